"""Conjugate gradient solvers for the oracle (TEST INFRASTRUCTURE ONLY).

  hscg      Algorithm 1 (Hestenes-Stiefel CG, Section 1)
  sstep_cg  Algorithm 5 (improved adaptive s-step CG, Section 4), with the
            comparators of Section 5 as options: fixed s-step CG
            (variant="fixed": s_k = sigma, no break test) and the previous
            adaptive s-step CG, Algorithm 2 (variant="old": monomial basis never
            retuned, the user constant c = c_const, and the pessimistic break
            test gamma >= eps*/(c eps ||r_{m+j+1}||) with gamma = kappa(Y_{k,s~}),
            relative residual reading C10)

Readings of the paper used here (the CUDA path takes the same ones):
  C9   Y is stored interleaved, so Y_l is the leading 2l+1 columns.
  C10  conditions (condy) and (newcondy) use relative residuals ||r||/||b||, phi/||b||.
  C11  c starts at eps^{-1/2} and is the latest value thereafter.
  C12  if no l satisfies (condy), s~ = 1.
  C14  kappa_l = +inf when lambda_min(G_l) <= 2^-44 lambda_max(G_l): below that
       level the smallest eigenvalue is rounding noise of the N-term inner
       products in G (this also covers lambda_min <= 0).
  C15  besides the outer test, sqrt(r'^T G r')/||b|| <= tol is tested after
       every inner step (``inner_conv_check``), ending the block.
  C16  convergence is declared on the updated residual, then confirmed with the
       true residual b - A x; if that is above tol, r := b - A x, p := r,
       psi := 1 and the iteration continues (a "replacement").  A failed check
       whose true residual has not halved since the previous failed check
       means the attainable accuracy is above tol: the solve stops with
       NOT_CONVERGED.
  C17  alpha invalid (p'^T G B p' <= 0 or not finite) at inner step j > 0 ends
       the block with s_k = j; at j = 0 the solve stops with BREAKDOWN.
       r'^T G r' <= 0 after a step reads as "residual estimate zero": the step is
       kept and the convergence test fires.
  C21  the order inside the inner step is as printed in Alg. 5.
  C22  the Meurant-Tichy state is fed every alpha; the estimates are used from
       global iteration 2 on (m + j + 1 > 1).
  C23  gamma_l := kappa(Y_{l+1}) for l = 1..s~-1; the break test at step j uses gamma_{j+1}.
  C27  a Gram block G_l with a non-finite entry (a basis column that
       overflowed, possible with a binary32-stored basis) has kappa_l = +inf,
       so s~ stays below the first such column and the solve goes on; only a
       non-finite leading block makes the first coordinate step fail
       (BREAKDOWN, C17).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import basis as bs
from .ritz import ExactRitz, RitzTracker

EPS64 = 2.0 ** -53
KAPPA_CUT = 2.0 ** -44

OK, NOT_CONVERGED, BREAKDOWN, NONFINITE = 0, 3, 2, 4


def _norm(v) -> float:
    return float(np.sqrt(v @ v))


def hscg(A, b, x0, tol: float, max_iters: int = 100000):
    """Algorithm 1 (HSCG).  Stops when ||r_i||/||b|| <= tol on the updated
    residual, then confirms with the true residual (readings C16, C20).

    Returns (x, info) with info = {iters, alphas, betas, replacements, status,
    relres_true}.
    """
    normb = _norm(b)
    if normb == 0.0:  # b = 0: the solution is x = 0
        return np.zeros_like(np.asarray(x0, dtype=np.float64)), dict(
            iters=0, alphas=[], betas=[], replacements=0, status=OK, relres_true=0.0)
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - A @ x
    p = r.copy()
    rr = float(r @ r)
    alphas, betas = [], []
    it = 0
    replacements = 0
    status = NOT_CONVERGED
    prev_fail = 0.0
    while it < max_iters:
        if math.sqrt(rr) / normb <= tol:
            rt = b - A @ x
            rel = _norm(rt) / normb
            if rel <= tol:
                status = OK
                break
            if prev_fail > 0.0 and rel >= 0.5 * prev_fail:
                break                       # stagnation above tol (reading C16)
            prev_fail = rel
            r, p = rt, rt.copy()
            rr = float(r @ r)
            replacements += 1
        q = A @ p
        alpha = rr / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        rr_new = float(r @ r)
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        alphas.append(alpha)
        betas.append(beta)
        it += 1
    relres = _norm(b - A @ x) / normb
    return x, dict(iters=it, alphas=alphas, betas=betas, replacements=replacements,
                   status=status, relres_true=relres)


@dataclasses.dataclass
class Options:
    """Parameters of Algorithm 5 (sigma = smax, s̄_0 = s0, f) and the readings' switches."""
    smax: int = 8
    basis: str = "chebyshev"          # monomial | newton | chebyshev
    s0: int | None = None              # reading C13: s̄_0 = sigma
    f: int | None = None               # reading C13: f = sigma
    max_outer: int = 100000
    c_mode: str = "xi"                 # xi | xi_scaled | one | kappa_ratio | const
    c_const: float = 1.0
    newton_scale: str = "capacity"     # capacity | paper_unit   (reading C6)
    cheb_params: str = "standard"      # standard | paper_printed (reading C5)
    inner_conv_check: bool = True      # reading C15
    eps: float = EPS64
    kappa_cut: float = KAPPA_CUT       # reading C14
    y_fp32: bool = False               # store the basis rounded to FP32 (x, r, p stay FP64)
    # FP32-stored basis: replace r by b - A x at the end of a block once the
    # residual estimate has fallen by this factor since the last replacement
    fp32_replace_drop: float = 2.0 ** -4
    variant: str = "improved"          # improved (Alg. 5) | fixed (s_k = sigma) | old (Alg. 2)
    # ritz: "mt" = the Meurant-Tichy estimates of Algs. 3-4 (Section 4); "exact"
    # = the extremal eigenvalues of T_m itself (eq. T) after every iteration
    ritz: str = "mt"
    # replay: a decision log [{"stilde", "sk", "replaced"}, ...] from another
    # implementation.  The oracle then takes those decisions instead of its own,
    # evaluates its own ones beside them and records, for each decision, the
    # log-distance of the deciding quantity to its threshold ("margins"); the
    # solve ends after the last record.
    replay: list | None = None
    # gram: a callable Y -> G used instead of Y^T Y (G = Y^T Y of Section 2
    # computed another way, for studies of that arithmetic); None: Y.T @ Y
    gram: object = None
    # recover: a callable (Y, x', r', p', x) -> (x, r, p) used instead of
    # eq. (coords) as written (for studies of the recovery's rounding); None:
    # x + Y x', Y r', Y p'
    recover: object = None


def kappa_estimates(G: np.ndarray, sbar: int, kappa_cut: float = KAPPA_CUT):
    """kappa_l ~ kappa(Y_l) = sqrt(kappa(G_l)), l = 1..sbar (Section 3).

    G_l is the leading (2l+1) x (2l+1) block of G; its extreme eigenvalues come
    from a dense symmetric eigensolve.  Entry 0 is unused.  A block with a
    non-finite entry (a basis column that overflowed) has no eigenvalues:
    kappa_l = inf (reading C27).
    """
    kap = np.full(sbar + 1, np.nan)
    lmins = np.full(sbar + 1, np.nan)
    lmaxs = np.full(sbar + 1, np.nan)
    for l in range(1, sbar + 1):
        n = 2 * l + 1
        if not np.all(np.isfinite(G[:n, :n])):
            kap[l] = math.inf
            continue
        w = np.linalg.eigvalsh(G[:n, :n])
        lmins[l], lmaxs[l] = w[0], w[-1]
        if not (w[-1] > 0.0) or w[0] <= kappa_cut * w[-1]:
            kap[l] = math.inf
        else:
            kap[l] = math.sqrt(w[-1] / w[0])
    return kap, lmins, lmaxs


def choose_stilde(kap, sbar: int, tol: float, c: float, eps: float, normr: float, normb: float) -> int:
    """s~_k of eq. (condy): the largest l <= s-bar with kappa(Y_l) <= eps*/(c eps ||r_m||/||b||)
    (eq. (cond) with the relative residual, reading C10); 1 when no l qualifies (C12).

    ``kap[l]`` is the estimate kappa_l of kappa(Y_{k,l}), l = 1..sbar (entry 0 unused).
    """
    thr = tol / (c * eps * normr / normb)
    cands = [l for l in range(1, sbar + 1) if kap[l] <= thr]
    return max(cands) if cands else 1


def break_test(gam_next: float, tol: float, c: float, eps: float, phi: float, normb: float) -> bool:
    """The improved break test of eq. (newcondy): stop the block when
    gamma_{j+1} >= eps*/(c eps phi/||b||), phi the running maximum of the
    residual estimates of the block (reading C10 for the relative form)."""
    return gam_next >= tol / (c * eps * phi / normb)


def psi_update(psi: float, beta: float) -> float:
    """eq. (psiupd): psi_{n+1} = psi_n / (psi_n + beta_n), the ratio ||r_{n+1}||^2/||p_{n+1}||^2."""
    return psi / (psi + beta)


def uses_ritz_c(m: int, j: int) -> bool:
    """Alg. 5 updates c from the Ritz estimates once the global iteration count
    m + j + 1 exceeds 1 (two alphas known, reading C22)."""
    return m + j + 1 > 1


def c_value(mode: str, lmin: float, lmax: float, psi: float, c_const: float = 1.0) -> float:
    """c_{m+j+1} of Alg. 5 (eq. xiupd) and the alternatives of Section 5.1."""
    if mode == "xi":
        return max(1.0, lmax * math.sqrt(psi / lmin))
    if mode == "xi_scaled":
        return max(1.0, lmax * math.sqrt(psi) / lmin)
    if mode == "one":
        return 1.0
    if mode == "kappa_ratio":
        return lmax / lmin
    if mode == "const":
        return c_const
    raise ValueError(mode)


def sstep_cg(A, b, x0, tol: float, opts: Options | None = None, record_vectors: bool = False):
    """Algorithm 5 (improved adaptive s-step CG), step by step.

    A is anything with ``A @ v`` (a scipy sparse matrix).  Returns (x, info);
    info holds the status, counts, the alpha/beta sequence, the final Ritz
    estimates and a per-outer-loop decision log ``hist`` (list of dicts).
    """
    o = opts or Options()
    kind = bs.BASIS_NAMES[o.basis]
    sigma = o.smax
    s0 = o.s0 if o.s0 is not None else sigma
    f = o.f if o.f is not None else sigma
    eps = o.eps

    normb = _norm(b)
    if normb == 0.0:  # b = 0: the solution is x = 0
        return np.zeros_like(np.asarray(x0, dtype=np.float64)), dict(
            status=OK, outer=0, inner=0, alphas=[], betas=[], hist=[], replacements=0,
            relres_true=0.0, lmin=None, lmax=None, c=None, psi=1.0)
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - A @ x
    if not math.isfinite(normb) or not math.isfinite(_norm(r)):   # NaN/Inf in b, x0 or A
        return x, dict(status=NONFINITE, outer=0, inner=0, alphas=[], betas=[], hist=[], replacements=0,
                       relres_true=math.nan, lmin=None, lmax=None, c=None, psi=1.0)
    p = r.copy()
    psi = 1.0
    c = 1.0 / math.sqrt(eps)  # c_1 = eps^{-1/2}
    m = 0
    theta, gamma, mu = bs.basis_params(bs.MONOMIAL, sigma, None, None)
    if o.ritz not in ("mt", "exact"):
        raise ValueError(f"unknown ritz mode {o.ritz!r}")
    ritz = RitzTracker() if o.ritz == "mt" else ExactRitz()
    alphas, betas = [], []
    hist = []
    replacements = 0
    status = NOT_CONVERGED
    s_prev = None
    done = False
    rho_last = 1.0          # FP32 basis: relative residual at the last replacement
    fp32_replacements = 0
    prev_fail = 0.0         # relative true residual at the last failed convergence check
    for k in range(o.max_outer):
        sbar = s0 if k == 0 else min(s_prev + f, sigma)
        Y = bs.krylov_basis(A, p, r, sbar, theta, gamma, mu, store32=o.y_fp32)
        G = Y.T @ Y if o.gram is None else o.gram(Y)
        kap, _, _ = kappa_estimates(G, sbar, o.kappa_cut)
        normr = math.sqrt(G[1, 1])
        margins = {}
        if o.variant == "old":
            c = o.c_const            # Alg. 2: c_k is supplied by the user
        if o.variant == "fixed":
            stilde = sbar
        else:
            stilde = choose_stilde(kap, sbar, tol, c, eps, normr, normb)
            thr = tol / (c * eps * normr / normb)
            if o.replay is not None:
                own = stilde
                stilde = o.replay[k]["stilde"]
                if own != stilde:
                    lo, hi = min(own, stilde), max(own, stilde)
                    margins["stilde"] = min(abs(math.log(kap[l] / thr)) for l in range(lo, hi + 1)
                                            if 1 <= l <= sbar and math.isfinite(kap[l]) and kap[l] > 0) \
                        if any(math.isfinite(kap[l]) for l in range(lo, hi + 1) if 1 <= l <= sbar) else math.inf
        forced_sk = o.replay[k]["sk"] if o.replay is not None else None
        n = 2 * stilde + 1
        Gs = G[:n, :n]
        Bs = bs.b_matrix(stilde, theta, gamma, mu)
        gam = {l: kap[l + 1] for l in range(1, stilde)}
        pc = np.zeros(n); pc[bs.p_index(0)] = 1.0
        rc = np.zeros(n); rc[bs.r_index(0)] = 1.0
        xc = np.zeros(n)
        rr = float(rc @ Gs @ rc)
        phi = math.sqrt(max(rr, 0.0))
        c_start = c
        rr0 = rr
        rr_steps, c_steps = [], []     # per inner step: r'^T G r' and c after the step
        sk = 0
        converged_est = False
        breakdown = False
        for j in range(stilde):
            Bp = Bs @ pc
            den = float(pc @ (Gs @ Bp))
            alpha = rr / den if den > 0.0 else math.nan
            if not math.isfinite(alpha) or alpha <= 0.0:
                if j == 0:
                    breakdown = True
                break
            sk = j + 1
            xc = xc + alpha * pc
            rc = rc - alpha * Bp
            rr_new = float(rc @ Gs @ rc)
            if not (rr_new > 0.0) or not math.isfinite(rr_new):
                converged_est = True
                break
            alphas.append(alpha)
            beta = rr_new / rr
            pc = rc + beta * pc
            phi = max(phi, math.sqrt(rr_new))
            psi = psi_update(psi, beta)
            ritz.push(alpha, betas[-1] if betas else None)
            betas.append(beta)
            if uses_ritz_c(m, j) and o.variant != "old":
                c = c_value(o.c_mode, ritz.lmin, ritz.lmax, psi, o.c_const)
            rr = rr_new
            rr_steps.append(rr_new)
            c_steps.append(c)
            own_conv = o.inner_conv_check and math.sqrt(rr_new) / normb <= tol
            if o.variant == "old":   # Alg. 2: kappa of the whole block, current residual
                own_brk = (not own_conv) and kap[stilde] >= tol / (c * eps * math.sqrt(rr_new) / normb)
            else:
                own_brk = (not own_conv) and o.variant != "fixed" and j < stilde - 1 and \
                    break_test(gam[j + 1], tol, c, eps, phi, normb)
            if forced_sk is None:
                if own_conv:
                    converged_est = True
                    break
                if own_brk:
                    break
            else:
                stop = j + 1 >= forced_sk
                if stop != (own_conv or own_brk or j == stilde - 1):
                    qc = abs(math.log(math.sqrt(rr_new) / (normb * tol))) if o.inner_conv_check else math.inf
                    qb = abs(math.log(gam[j + 1] * c * eps * phi / (normb * tol))) \
                        if (j < stilde - 1 and math.isfinite(gam[j + 1])) else math.inf
                    margins[f"stop_j{j}"] = min(qc, qb)
                if stop:
                    converged_est = own_conv
                    break
        if breakdown:
            status = BREAKDOWN
            hist.append(dict(sbar=sbar, stilde=stilde, sk=0, kappa=kap.tolist(), c=c_start))
            break
        Yn = Y[:, :n]
        if o.recover is None:
            x = x + Yn @ xc
            r = Yn @ rc
            p = Yn @ pc
        else:
            x, r, p = o.recover(Yn, xc, rc, pc, x)
        m += sk
        s_prev = sk
        hist.append(dict(sbar=sbar, stilde=stilde, sk=sk, kappa=kap.tolist(), c_start=c_start,
                         c=c, phi=phi, lmin=ritz.lmin, lmax=ritz.lmax,
                         relres_est=math.sqrt(max(rr, 0.0)) / normb, m=m, margins=margins,
                         normr_start=normr, rr0=rr0, rr_steps=rr_steps, c_steps=c_steps,
                         psi_end=psi, pGp_end=float(pc @ Gs @ pc)))
        if m > 1 and kind != bs.MONOMIAL and o.variant != "old":
            theta, gamma, mu = bs.basis_params(kind, sigma, ritz.lmin, ritz.lmax,
                                               o.newton_scale, o.cheb_params)
        if not converged_est and not o.inner_conv_check:
            # outer-level test only (reading C15 off): the coordinate estimate
            # of the updated residual at the end of the block
            converged_est = math.sqrt(max(rr, 0.0)) / normb <= tol
        if o.y_fp32 and not converged_est:
            # FP32 basis: each block perturbs the updated residual at the 2^-24
            # level of the largest residual since the last replacement; put the
            # true residual back once the estimate has fallen far enough (p kept)
            est = math.sqrt(max(rr, 0.0)) / normb
            if est <= o.fp32_replace_drop * rho_last:
                r = b - A @ x
                rho_last = _norm(r) / normb
                fp32_replacements += 1
                hist[-1]["fp32_replaced"] = True
        if o.replay is not None:
            if k + 1 >= len(o.replay):
                status = OK if _norm(b - A @ x) / normb <= tol else NOT_CONVERGED
                break
            if o.replay[k].get("replaced"):
                rt = b - A @ x
                r, p = rt, rt.copy()
                psi = 1.0
                replacements += 1
                hist[-1]["replaced"] = True
            continue
        if converged_est:
            rt = b - A @ x
            rel = _norm(rt) / normb
            if not math.isfinite(rel):
                status = NONFINITE
                break
            if rel <= tol:
                status = OK
                done = True
            elif prev_fail > 0.0 and rel >= 0.5 * prev_fail:
                break                       # stagnation above tol (reading C16)
            else:
                prev_fail = rel
                r, p = rt, rt.copy()
                psi = 1.0
                replacements += 1
                hist[-1]["replaced"] = True
        if done:
            break
    relres = _norm(b - A @ x) / normb
    info = dict(status=status, outer=len(hist), inner=m, alphas=alphas, betas=betas,
                hist=hist, replacements=replacements, relres_true=relres,
                lmin=ritz.lmin, lmax=ritz.lmax, c=c, psi=psi, fp32_replacements=fp32_replacements)
    return x, info
