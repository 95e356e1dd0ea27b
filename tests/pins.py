"""Independent checks that pin the oracle to the mathematics (not to itself).

Each check takes the implementation under test as an argument so that the
mutation tests can hand it a deliberately broken copy and see it fail.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def poisson2d_eigs(n: int) -> np.ndarray:
    """Closed-form spectrum of the unit 5-point Dirichlet Laplacian on n x n."""
    j = np.arange(1, n + 1)
    s = 4.0 * np.sin(j * np.pi / (2 * (n + 1))) ** 2
    return np.sort((s[:, None] + s[None, :]).ravel())


def poisson3d_eigs(n: int) -> np.ndarray:
    j = np.arange(1, n + 1)
    s = 4.0 * np.sin(j * np.pi / (2 * (n + 1))) ** 2
    return np.sort((s[:, None, None] + s[None, :, None] + s[None, None, :]).ravel())


def check_chebyshev_closed_form(krylov_basis, basis_params, s=9, seed=3) -> float:
    """max |rho_l(z) - cos(l arccos y)| for the standard Chebyshev parameters.

    A = diag(z) with z in [lmin, lmax]: column l of P is rho_l(z_i) p_i, so with
    p = 1 it equals T_l((z - c)/h) exactly in exact arithmetic.
    """
    lmin, lmax = 0.3, 7.7
    z = np.random.default_rng(seed).uniform(lmin, lmax, 50)
    A = sp.diags(z)
    th, ga, mu = basis_params(2, s, lmin, lmax, "capacity", "standard")
    Y = krylov_basis(A, np.ones(50), np.ones(50), s, th, ga, mu)
    y = (z - 0.5 * (lmin + lmax)) / (0.5 * (lmax - lmin))
    err = 0.0
    for l in range(s + 1):
        err = max(err, np.max(np.abs(Y[:, 2 * l] - np.cos(l * np.arccos(y)))))
    for l in range(s):
        err = max(err, np.max(np.abs(Y[:, 2 * l + 1] - np.cos(l * np.arccos(y)))))
    return err


def check_newton_closed_form(krylov_basis, basis_params, s=7, seed=4) -> float:
    """max relative |rho_l(z) - prod_{m<l} (z - theta_m)/gamma_m| on A = diag(z)."""
    lmin, lmax = 0.2, 3.1
    z = np.random.default_rng(seed).uniform(lmin, lmax, 40)
    th, ga, mu = basis_params(1, s, lmin, lmax, "capacity", "standard")
    Y = krylov_basis(sp.diags(z), np.ones(40), np.ones(40), s, th, ga, mu)
    err = 0.0
    for l in range(s + 1):
        ref = np.ones(40)
        for mm in range(l):
            ref = ref * (z - th[mm]) / ga[mm]
        err = max(err, np.max(np.abs(Y[:, 2 * l] - ref)) / max(1.0, np.max(np.abs(ref))))
    return err


def check_avvb(krylov_basis, b_matrix, basis_params, A, kind, s, seed=5) -> float:
    """||A Ybar - Y B|| / (||A|| ||Y||) (eq. AVVB) for random p, r."""
    N = A.shape[0]
    rng = np.random.default_rng(seed)
    p, r = rng.standard_normal(N), rng.standard_normal(N)
    lmax = float(sp.linalg.norm(A, 1))
    th, ga, mu = basis_params(kind, s, 0.05 * lmax, lmax, "capacity", "standard")
    Y = krylov_basis(A, p, r, s, th, ga, mu)
    B = b_matrix(s, th, ga, mu)
    Yb = Y.copy()
    Yb[:, 2 * s] = 0.0
    Yb[:, 2 * (s - 1) + 1] = 0.0
    return np.linalg.norm(A @ Yb - Y @ B) / (lmax * np.linalg.norm(Y))


def check_mt_exact_at_two(tracker_cls, alpha0, alpha1, beta0) -> float:
    """|estimates - closed-form eigenvalues of the 2x2 T_2| / lambda_max."""
    t11 = 1.0 / alpha0
    t22 = 1.0 / alpha1 + beta0 / alpha0
    t12 = math.sqrt(beta0) / alpha0
    tr, det = t11 + t22, t11 * t22 - t12 * t12
    disc = math.sqrt(max(tr * tr / 4 - det, 0.0))
    lmax, lmin = tr / 2 + disc, tr / 2 - disc
    tr_ = tracker_cls()
    tr_.push(alpha0, None)
    est_min, est_max = tr_.push(alpha1, beta0)
    return max(abs(est_max - lmax), abs(est_min - lmin)) / lmax


def cg_coefficients(A, b, iters):
    """Plain Hestenes-Stiefel coefficients written out for the pins (dense numpy)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    al, be, rs, ps = [], [], [r.copy()], [p.copy()]
    for _ in range(iters):
        q = A @ p
        a = (r @ r) / (p @ q)
        x = x + a * p
        rn = r - a * q
        bb = (rn @ rn) / (r @ r)
        p = rn + bb * p
        r = rn
        al.append(a)
        be.append(bb)
        rs.append(r.copy())
        ps.append(p.copy())
    return al, be, rs, ps


def check_exact_ritz(tracker_cls, iters=16, seed=8) -> float:
    """Largest |extremal value - extremal eigenvalue of V_i^T A V_i| / lambda_max
    over i = 1..iters for a tracker fed CG's (alpha_i, beta_{i-1}): the Ritz
    values of A on the Krylov space, with V_i the normalised residuals of plain
    CG (a dense matrix product, independent of the tracker's T; 16 iterations
    on a 72-unknown system, before the residuals lose orthogonality).  Returns inf if
    the values violate interlacing (lmax rising, lmin falling with i)."""
    A = np.asarray(__import__("oracle.operators", fromlist=["as_matrix"]).as_matrix(
        __import__("sscg_inputs.generators", fromlist=["varcoef_stencil"]).varcoef_stencil((9, 8), seed=seed)).todense())
    b = np.random.default_rng(seed).standard_normal(A.shape[0])
    al, be, rs, _ = cg_coefficients(A, b, iters)
    tr = tracker_cls()
    worst, prev = 0.0, None
    for i in range(iters):
        lmin, lmax = tr.push(al[i], be[i - 1] if i else None)
        V = np.column_stack([rs[j] / np.linalg.norm(rs[j]) for j in range(i + 1)])
        w = np.linalg.eigvalsh(V.T @ A @ V)
        worst = max(worst, abs(lmin - w[0]) / w[-1], abs(lmax - w[-1]) / w[-1])
        if prev is not None and (lmax < prev[1] * (1 - 1e-13) or lmin > prev[0] * (1 + 1e-13)):
            return math.inf
        prev = (lmin, lmax)
    return worst
