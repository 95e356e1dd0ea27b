"""Pins for Algorithm 1 (HSCG) and Algorithm 5 (improved adaptive s-step CG)."""
import math

import numpy as np
import pytest

from oracle import cg
from oracle.operators import as_matrix
from sscg_inputs import generators as gen


def test_hscg_solves_tiny_dense_systems():
    for seed in range(4):
        rng = np.random.default_rng(seed)
        n = 24
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        A = Q @ np.diag(rng.uniform(0.5, 5.0, n)) @ Q.T
        b = rng.standard_normal(n)
        x, info = cg.hscg(A, b, np.zeros(n), 1e-12)
        assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-10 * np.linalg.norm(x)
        assert info["iters"] <= 2 * n


def test_hscg_finite_termination_few_eigenvalues():
    # A with 3 distinct eigenvalues: CG terminates in 3 steps (exact arithmetic)
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    A = Q @ np.diag(np.repeat([1.0, 2.0, 5.0], 10)) @ Q.T
    x, info = cg.hscg(A, rng.standard_normal(30), np.zeros(30), 1e-12)
    assert info["iters"] <= 4


def test_hscg_orthogonality_and_psi_identity():
    A = as_matrix(gen.varcoef_stencil((8, 8), seed=2)).toarray()
    b = np.random.default_rng(0).standard_normal(64)
    x = np.zeros(64)
    r = b.copy(); p = r.copy(); psi = 1.0
    rs = [r.copy()]
    _, info = cg.hscg(A, b, x, 1e-30, max_iters=10)
    for a, be in zip(info["alphas"], info["betas"]):
        q = A @ p
        r = r - a * q
        p = r + be * p
        psi = psi / (psi + be)                      # eq. (psiupd)
        assert abs(psi - (r @ r) / (p @ p)) < 1e-12 * psi
        rs.append(r.copy())
    R = np.array([v / np.linalg.norm(v) for v in rs])
    assert np.abs(R @ R.T - np.eye(len(rs))).max() < 1e-10   # residuals orthogonal


def test_sigma_one_reproduces_hscg():
    # With sigma = 1 every block is one step and the coordinate recurrences are
    # HSCG written in the 3-column basis [p, r, rho_1(A) p]: identical in exact
    # arithmetic.  On the 2D Poisson problem CG's coefficients are insensitive
    # to rounding, so the two sequences agree to ~1e-14 over the whole solve.
    A, b, x0, _ = gen.config_problem("poisson2d_64")
    M = as_matrix(A)
    xh, h = cg.hscg(M, b, x0, 1e-10)
    for basis in ("monomial", "newton", "chebyshev"):
        x, s = cg.sstep_cg(M, b, x0, 1e-10, cg.Options(smax=1, basis=basis))
        assert len(s["alphas"]) == len(h["alphas"])
        assert np.allclose(s["alphas"], h["alphas"], rtol=1e-12, atol=0)
        assert np.allclose(s["betas"], h["betas"], rtol=1e-12, atol=0)
        assert np.linalg.norm(x - xh) <= 1e-12 * np.linalg.norm(xh)
        assert all(hh["sk"] == 1 for hh in s["hist"])


@pytest.mark.parametrize("basis", ["newton", "chebyshev"])
def test_fixed_s_block_equals_hscg_in_exact_arithmetic(basis):
    # with a well-conditioned basis and small s, s-step coefficients track HSCG's
    A = as_matrix(gen.poisson2d_csr(24))
    b = A @ gen.uniform_vector(576, 6)
    _, h = cg.hscg(A, b, np.zeros(576), 1e-10)
    _, s = cg.sstep_cg(A, b, np.zeros(576), 1e-10,
                       cg.Options(smax=3, basis=basis, variant="fixed"))
    assert abs(len(s["alphas"]) - len(h["alphas"])) <= 1
    # agreement to rounding while the residual is large; near the attainable
    # accuracy the coefficients of both lose digits, as expected
    assert np.allclose(s["alphas"][:60], h["alphas"][:60], rtol=1e-11, atol=0)


def test_first_block_is_one_step_because_p_equals_r():
    # p_0 = r_0 makes P_l = R_l, so G is singular for every l >= 1 and kappa = inf:
    # no l satisfies (condy) and s~ = 1 (reading C12)
    A = as_matrix(gen.poisson2d_csr(16))
    b = A @ gen.uniform_vector(256, 1)
    _, info = cg.sstep_cg(A, b, np.zeros(256), 1e-10, cg.Options(smax=6, basis="chebyshev"))
    h0 = info["hist"][0]
    assert h0["stilde"] == 1 and h0["sk"] == 1
    assert all(math.isinf(k) for k in h0["kappa"][1:])


@pytest.mark.parametrize("basis", ["monomial", "newton", "chebyshev"])
def test_poisson64_converges_and_matches_xstar(basis):
    A, b, x0, extra = gen.config_problem("poisson2d_64")
    M = as_matrix(A)
    x, info = cg.sstep_cg(M, b, x0, 1e-10, cg.Options(smax=8, basis=basis))
    assert info["status"] == cg.OK
    assert info["relres_true"] <= 1e-10
    kappa = 7.995328907329306 / 4.671092670693646e-3
    err = np.linalg.norm(x - extra["xstar"]) / np.linalg.norm(extra["xstar"])
    assert err <= kappa * 1e-10
    # decision log invariants of Alg. 5
    prev = None
    for h in info["hist"]:
        assert 1 <= h["sk"] <= h["stilde"] <= h["sbar"] <= 8
        if prev is not None:
            assert h["sbar"] == min(prev + 8, 8)
        prev = h["sk"]
    # total inner iterations stay close to HSCG's (Section 5: independent of sigma)
    _, hh = cg.hscg(M, b, x0, 1e-10)
    assert abs(info["inner"] - hh["iters"]) <= 0.1 * hh["iters"]
    assert info["outer"] < hh["iters"] / 4


def test_kappa_estimates_monotone_and_break_rule():
    st = gen.varcoef_stencil((20, 20, 20), seed=9)
    A = as_matrix(st)
    b = gen.random_rhs(st.n, 3)
    _, info = cg.sstep_cg(A, b, np.zeros(st.n), 1e-10, cg.Options(smax=10, basis="newton"))
    assert info["status"] == cg.OK and info["relres_true"] <= 1e-10
    for h in info["hist"]:
        kap = np.array(h["kappa"][1:])
        fin = kap[np.isfinite(kap)]
        # interlacing: kappa(G_l) is non-decreasing in l
        assert np.all(np.diff(fin) >= -1e-8 * fin[1:])
        # once infinite, stays infinite
        if np.any(~np.isfinite(kap)):
            first = np.argmax(~np.isfinite(kap))
            assert np.all(~np.isfinite(kap[first:]))
        assert h["c"] >= 1.0


def test_c_modes():
    assert cg.c_value("xi", 0.1, 4.0, 0.01) == max(1.0, 4.0 * math.sqrt(0.01 / 0.1))
    assert cg.c_value("kappa_ratio", 0.1, 4.0, 0.5) == 40.0
    assert cg.c_value("one", 0.1, 4.0, 0.5) == 1.0
    assert cg.c_value("xi_scaled", 0.1, 4.0, 0.01) == max(1.0, 4.0 * 0.1 / 0.1)


def test_replay_of_own_log_is_identity():
    st = gen.varcoef_stencil((12, 10, 9), seed=11)
    b = gen.random_rhs(st.n, 12)
    A = as_matrix(st)
    x1, i1 = cg.sstep_cg(A, b, np.zeros(st.n), 1e-10, cg.Options(smax=8, basis="newton"))
    log = [dict(stilde=h["stilde"], sk=h["sk"], replaced=h.get("replaced", False)) for h in i1["hist"]]
    x2, i2 = cg.sstep_cg(A, b, np.zeros(st.n), 1e-10, cg.Options(smax=8, basis="newton", replay=log))
    assert np.array_equal(x1, x2) and i1["outer"] == i2["outer"]
    assert all(not h["margins"] for h in i2["hist"])


def test_replay_records_margin_of_a_forced_decision():
    st = gen.varcoef_stencil((12, 10, 9), seed=11)
    b = gen.random_rhs(st.n, 12)
    A = as_matrix(st)
    _, i1 = cg.sstep_cg(A, b, np.zeros(st.n), 1e-10, cg.Options(smax=8, basis="newton"))
    log = [dict(stilde=h["stilde"], sk=h["sk"]) for h in i1["hist"]]
    k = next(i for i, h in enumerate(log) if h["stilde"] >= 3 and h["sk"] >= 2)
    log[k] = dict(stilde=log[k]["stilde"] - 1, sk=min(log[k]["sk"], log[k]["stilde"] - 1))
    _, i2 = cg.sstep_cg(A, b, np.zeros(st.n), 1e-10, cg.Options(smax=8, basis="newton", replay=log[:k + 1]))
    assert "stilde" in i2["hist"][k]["margins"]


def test_old_adaptive_alg2_reduces_to_hscg_with_huge_c():
    # with c so large that condy admits no l, every block is one step: HSCG again
    A, b, x0, _ = gen.config_problem("poisson2d_64", scale=24)
    M = as_matrix(A)
    _, h = cg.hscg(M, b, x0, 1e-10)
    _, s = cg.sstep_cg(M, b, x0, 1e-10, cg.Options(smax=8, basis="monomial", variant="old", c_const=1e30))
    assert all(hh["sk"] == 1 for hh in s["hist"])
    assert np.allclose(s["alphas"], h["alphas"][: len(s["alphas"])], rtol=1e-10)


def test_old_adaptive_alg2_converges_with_c_one():
    A, b, x0, _ = gen.config_problem("poisson2d_64")
    x, s = cg.sstep_cg(as_matrix(A), b, x0, 1e-10, cg.Options(smax=8, basis="monomial", variant="old", c_const=1.0))
    assert s["status"] == cg.OK and s["relres_true"] <= 1e-10
    assert all(h["c"] == 1.0 for h in s["hist"])
    # the basis is never retuned: a Chebyshev request stays monomial
    _, s2 = cg.sstep_cg(as_matrix(A), b, x0, 1e-10, cg.Options(smax=8, basis="chebyshev", variant="old", c_const=1.0))
    assert [h["sk"] for h in s2["hist"]] == [h["sk"] for h in s["hist"]]


def test_failure_detection_on_the_host():
    # injected on the host: NaN in b, a non-SPD operator, an iteration cap
    A, b, x0, _ = gen.config_problem("poisson2d_64", scale=12)
    M = as_matrix(A)
    bn = b.copy()
    bn[5] = np.nan
    _, i1 = cg.sstep_cg(M, bn, x0, 1e-10, cg.Options(smax=4))
    assert i1["status"] == cg.NONFINITE
    _, i2 = cg.sstep_cg(-M, b, x0, 1e-10, cg.Options(smax=4))
    assert i2["status"] == cg.BREAKDOWN
    _, i3 = cg.sstep_cg(M, b, x0, 1e-14, cg.Options(smax=4, max_outer=3))
    assert i3["status"] == cg.NOT_CONVERGED and i3["outer"] == 3


@pytest.mark.parametrize("basis", ["newton", "chebyshev"])
def test_exact_ritz_mode_converges_and_tracks_t(basis):
    # f3: Options(ritz="exact") feeds the extremal eigenvalues of T_m itself
    # (eq. T) to the basis parameters and to c; the solve converges, and the
    # final values are the extreme eigenvalues of T built from all of the
    # solve's CG coefficients
    from oracle import ritz as oritz
    st = gen.varcoef_stencil((20, 18), seed=21)
    A = as_matrix(st)
    b = gen.random_rhs(st.n, 22)
    x, info = cg.sstep_cg(A, b, np.zeros(st.n), 1e-10, cg.Options(smax=8, basis=basis, ritz="exact"))
    assert info["status"] == cg.OK
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)
    al, be = info["alphas"], info["betas"]
    w = np.linalg.eigvalsh(oritz.lanczos_t(al, be[:len(al) - 1]))
    assert abs(info["lmax"] - w[-1]) <= 1e-12 * w[-1] and abs(info["lmin"] - w[0]) <= 1e-12 * w[-1]
    _, mt = cg.sstep_cg(A, b, np.zeros(st.n), 1e-10, cg.Options(smax=8, basis=basis))
    assert abs(info["inner"] - mt["inner"]) <= 0.3 * mt["inner"]
    with pytest.raises(ValueError):
        cg.sstep_cg(A, b, np.zeros(st.n), 1e-10, cg.Options(smax=8, basis=basis, ritz="lanczos"))
