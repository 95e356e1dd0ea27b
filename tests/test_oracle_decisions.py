"""Pins for the adaptive decisions of Algorithm 5: s~ (eq. condy), the break
test (eq. newcondy), psi (eq. psiupd), c (eq. xiupd and the global-step gate)
and the kappa cut of reading C14.

Two kinds of pin:
- worked examples: hand-built kappa / phi / psi / c values chosen as powers of
  two, so every threshold is exact and the expected decision is worked out
  below from the paper's formula (boundary cases decide <= against <);
- solve records: a short solve is re-decided from its own recorded inputs, with
  the residual norms taken from a different computation than the one the
  oracle used (the previous block's coordinate estimate for ||r_m||, the per-step
  r'^T G r' values for phi), and psi is checked against the identity
  psi = ||r||^2 / ||p||^2 that eq. (psiupd) is derived from.
"""
import math

import numpy as np
import pytest

from oracle import cg
from oracle.operators import as_matrix
from sscg_inputs import generators as gen
from tests import pins

EPS = 2.0 ** -53


# ----------------------------------------------------------- worked examples
# tol = 2^-30, c = 2^3, eps = 2^-53, ||r_m|| = 2^-7, ||b|| = 2^3:
# relative residual 2^-10, so eq. (condy)'s bound is
# eps*/(c eps ||r||/||b||) = 2^-30 / (2^3 2^-53 2^-10) = 2^30.
TOL, C, NORMR, NORMB = 2.0 ** -30, 2.0 ** 3, 2.0 ** -7, 2.0 ** 3


def choose(kap, sbar, choose_stilde=cg.choose_stilde):
    return choose_stilde([math.nan] + list(kap), sbar, TOL, C, EPS, NORMR, NORMB)


def test_condy_largest_admissible_l_with_equality(choose_stilde=cg.choose_stilde):
    # kappa_3 = 2^30 equals the bound: admissible (kappa <= bound); kappa_4 above
    assert choose([1.0, 2.0 ** 10, 2.0 ** 30, 2.0 ** 31, math.inf], 5, choose_stilde) == 3
    # just above the bound at l = 3: s~ = 2
    assert choose([1.0, 2.0 ** 10, 2.0 ** 30 * (1 + 2.0 ** -52), 2.0 ** 31], 4, choose_stilde) == 2
    # the largest admissible l, not the last one before the first failure
    assert choose([1.0, 2.0 ** 31, 2.0 ** 29, math.inf], 4, choose_stilde) == 3
    # s~ never exceeds s-bar even when longer blocks would qualify
    assert choose([1.0, 2.0, 4.0, 8.0], 2, choose_stilde) == 2


def test_condy_uses_the_relative_residual(choose_stilde=cg.choose_stilde):
    # with ||r|| = 2^-7 alone (no division by ||b|| = 2^3) the bound would be
    # 2^27 and s~ = 1 here; with the relative residual (reading C10) it is 2^30
    assert choose([2.0 ** 27, 2.0 ** 28, 2.0 ** 30], 3, choose_stilde) == 3


def test_condy_no_admissible_l_gives_one(choose_stilde=cg.choose_stilde):
    # reading C12
    assert choose([2.0 ** 31, 2.0 ** 32, math.inf], 3, choose_stilde) == 1
    assert choose([math.inf, math.inf], 2, choose_stilde) == 1


def test_newcondy_break_at_equality(break_test=cg.break_test):
    # phi = 2^-7, ||b|| = 2^3: bound eps*/(c eps phi/||b||) = 2^30 as above
    assert break_test(2.0 ** 30, TOL, C, EPS, NORMR, NORMB) is True          # gamma >= bound
    assert break_test(2.0 ** 30 * (1 - 2.0 ** -53), TOL, C, EPS, NORMR, NORMB) is False
    assert break_test(math.inf, TOL, C, EPS, NORMR, NORMB) is True
    # relative form (C10): without /||b|| the bound would be 2^27
    assert break_test(2.0 ** 29, TOL, C, EPS, NORMR, NORMB) is False
    # a larger phi lowers the bound: phi = 2^-5 gives 2^28
    assert break_test(2.0 ** 29, TOL, C, EPS, 2.0 ** -5, NORMB) is True


def test_psi_recurrence_worked_values(psi_update=cg.psi_update):
    # eq. (psiupd), psi_0 = 1: with beta = 1 throughout, psi_n = 1/(n+1)
    psi = 1.0
    for n, want in enumerate([1 / 2, 1 / 3, 1 / 4, 1 / 5], start=1):
        psi = psi_update(psi, 1.0)
        assert abs(psi - want) <= 2e-16 * want, n
    # beta_0 = 3: 1/(1+3) = 1/4; then beta_1 = 1/3: (1/4)/(1/4 + 1/3) = 3/7
    psi = psi_update(psi_update(1.0, 3.0), 1.0 / 3.0)
    assert abs(psi - 3.0 / 7.0) <= 2e-16


def test_ritz_c_gate(uses_ritz_c=cg.uses_ritz_c):
    # global iteration m + j + 1: the first iteration (one alpha) keeps c;
    # from the second one on c comes from the Ritz estimates
    assert uses_ritz_c(0, 0) is False
    assert uses_ritz_c(0, 1) is True
    assert uses_ritz_c(1, 0) is True
    assert uses_ritz_c(7, 3) is True


def test_c_value_worked_values():
    # eq. (xiupd): c = max{1, lmax sqrt(psi/lmin)}; lmax = 4, lmin = 1/4, psi = 1/64:
    # 4 sqrt(4/64) = 1
    assert cg.c_value("xi", 0.25, 4.0, 1.0 / 64.0) == 1.0
    # psi = 1/4: 4 sqrt(1) = 4
    assert cg.c_value("xi", 0.25, 4.0, 0.25) == 4.0
    # below 1 it is clamped to 1: lmax = 1/2, lmin = 1, psi = 1/16 -> 1/8
    assert cg.c_value("xi", 1.0, 0.5, 1.0 / 16.0) == 1.0


def test_kappa_cut_boundary(kappa_estimates=cg.kappa_estimates):
    # reading C14: kappa = inf when lambda_min(G_l) <= 2^-44 lambda_max(G_l).
    # A diagonal G has its entries as eigenvalues.
    G = np.diag([1.0, 2.0 ** -44, 1.0])
    kap, _, _ = kappa_estimates(G, 1)
    assert math.isinf(kap[1])                       # at the cut: infinite
    G = np.diag([1.0, 2.0 ** -43, 1.0])
    kap, _, _ = kappa_estimates(G, 1)
    assert kap[1] == math.sqrt(2.0 ** 43)           # above it: sqrt(lmax/lmin)
    G = np.diag([4.0, 1.0, 2.0, 9.0, 1.0])
    kap, _, _ = kappa_estimates(G, 2)
    assert kap[1] == 2.0 and kap[2] == 3.0          # leading blocks (reading C9)


# -------------------------------------------------------------- solve records
def _short_solve(cgmod, n=24, seed=31, tol=1e-9, smax=8, basis="newton", bscale=100.0):
    st = gen.varcoef_stencil((n, n), seed=seed)
    A = as_matrix(st)
    b = bscale * gen.random_rhs(st.n, seed + 1)
    x, info = cgmod.sstep_cg(A, b, np.zeros(st.n), tol, cgmod.Options(smax=smax, basis=basis))
    return A, b, x, info


def check_condy_records(cgmod, tol=1e-9, **kw) -> int:
    """Number of outer loops whose s~ differs from eq. (condy) re-evaluated
    from the record (||r_m|| from the previous block's coordinate estimate)."""
    A, b, _, info = _short_solve(cgmod, tol=tol, **kw)
    normb = float(np.linalg.norm(b))
    bad = 0
    for k in range(1, len(info["hist"])):
        prev, h = info["hist"][k - 1], info["hist"][k]
        if prev.get("replaced"):
            continue
        assert h["c_start"] == prev["c"]            # c carried over from the last step (C11)
        rel = prev["relres_est"]                     # ||r_m||/||b|| of the recovered residual
        bound = tol / (h["c_start"] * EPS * rel)
        kap = h["kappa"]
        if any(math.isfinite(kap[l]) and abs(math.log(kap[l] / bound)) < 1e-6
               for l in range(1, h["sbar"] + 1)):
            continue                                 # too close to call in floating point
        want = max([l for l in range(1, h["sbar"] + 1) if kap[l] <= bound], default=1)
        bad += want != h["stilde"]
    return bad


def check_break_records(cgmod, tol=1e-9, **kw) -> int:
    """Number of outer loops whose block length differs from eqs. (newcondy)
    and C15 re-evaluated from the per-step records (phi rebuilt from r'^T G r')."""
    A, b, _, info = _short_solve(cgmod, tol=tol, **kw)
    normb = float(np.linalg.norm(b))
    bad = 0
    for h in info["hist"]:
        st, rr = h["stilde"], h["rr_steps"]
        kap = h["kappa"]
        phi = math.sqrt(h["rr0"])
        want, close = None, False
        for j, rj in enumerate(rr):
            phi = max(phi, math.sqrt(rj))
            if math.sqrt(rj) / normb <= tol:
                want = j + 1
                break
            if j < st - 1:
                bound = tol / (h["c_steps"][j] * EPS * phi / normb)
                g = kap[j + 2]                       # gamma_{j+1} = kappa(Y_{j+2}), reading C23
                if math.isfinite(g) and abs(math.log(g / bound)) < 1e-6:
                    close = True
                if g >= bound:
                    want = j + 1
                    break
        if want is None:
            want = st
        if not close:
            bad += want != h["sk"]
    return bad


def check_psi_records(cgmod, **kw) -> float:
    """Largest relative gap between psi and ||r||^2/||p||^2 = (r'^T G r')/(p'^T G p')
    at the end of the blocks that ended without a replacement.  The default
    problem keeps kappa(Y) small (Chebyshev, sigma = 6), so the identity holds
    to ~1e-9 over the whole solve in binary64."""
    kw = {**dict(n=20, smax=6, basis="chebyshev"), **kw}
    _, _, _, info = _short_solve(cgmod, **kw)
    worst = 0.0
    for h in info["hist"]:
        if h.get("replaced") or not h["rr_steps"]:
            continue
        ratio = h["rr_steps"][-1] / h["pGp_end"]
        worst = max(worst, abs(h["psi_end"] - ratio) / ratio)
    return worst


def check_first_ritz_c(cgmod) -> float:
    """Relative error of c after global iteration 2 against eq. (xiupd) from
    the closed-form eigenvalues of T_2 (eq. T) and psi_2 = ||r_2||^2/||p_2||^2
    of plain CG; also requires c = eps^-1/2 through iteration 1."""
    st = gen.varcoef_stencil((12, 12), seed=5)
    A = as_matrix(st)
    b = gen.random_rhs(st.n, 6)
    _, info = cgmod.sstep_cg(A, b, np.zeros(st.n), 1e-8, cgmod.Options(smax=4, basis="newton"))
    h0, h1 = info["hist"][0], info["hist"][1]
    assert h0["sk"] == 1                                   # p_0 = r_0: one step (C12)
    c1 = math.ldexp(math.sqrt(2.0), 26)                   # eps^-1/2 = 2^26.5 (Alg. 5 initialisation)
    if abs(h0["c"] - c1) > 4e-16 * c1 or h1["c_start"] != h0["c"]:
        return math.inf
    al, be, rs, ps = pins.cg_coefficients(A.toarray(), b, 2)
    t11 = 1.0 / al[0]
    t22 = 1.0 / al[1] + be[0] / al[0]
    t12 = math.sqrt(be[0]) / al[0]
    tr, det = t11 + t22, t11 * t22 - t12 * t12
    disc = math.sqrt(tr * tr / 4 - det)
    lmax, lmin = tr / 2 + disc, tr / 2 - disc
    psi2 = (rs[2] @ rs[2]) / (ps[2] @ ps[2])
    want = max(1.0, lmax * math.sqrt(psi2 / lmin))
    return abs(h1["c_steps"][0] - want) / want


def test_condy_matches_the_records():
    assert check_condy_records(cg) == 0


def test_break_step_matches_the_records():
    assert check_break_records(cg) == 0


def test_psi_identity_at_block_ends():
    assert check_psi_records(cg) <= 1e-8


def test_c_at_the_first_and_second_global_iteration():
    assert check_first_ritz_c(cg) <= 1e-10


@pytest.mark.parametrize("bscale", [2.0 ** -20, 2.0 ** 20])
def test_decisions_invariant_under_scaling_of_b(bscale):
    # Every quantity of eqs. (condy), (newcondy), (psiupd), (xiupd) is invariant
    # when b is scaled by a power of two (Y by the same factor, G by its square,
    # relative residuals, kappa, alpha, beta unchanged): same decisions, x scaled.
    A, b, x1, i1 = _short_solve(cg, bscale=1.0)
    _, _, x2, i2 = _short_solve(cg, bscale=bscale)
    assert [(h["stilde"], h["sk"]) for h in i1["hist"]] == [(h["stilde"], h["sk"]) for h in i2["hist"]]
    assert np.array_equal(x2, bscale * x1)
