"""Pins for eq. (T), eq. (lit), eq. (lest) and Algorithms 3-4 (Meurant-Tichy)."""
import math

import numpy as np
import pytest

from oracle import ritz
from oracle.operators import as_matrix
from sscg_inputs import generators as gen
from tests import pins


@pytest.fixture(scope="module")
def poisson64_cg():
    A = as_matrix(gen.poisson2d_csr(64))
    b = A @ gen.uniform_vector(A.shape[0], 1000)
    al, be, rs, ps = pins.cg_coefficients(A, b, 201)
    return A, al, be, rs, ps


def test_t_equals_lanczos_projection():
    # T_i = V^T A V with v_j = (-1)^j r_j / ||r_j|| (eq. T and the CG-Lanczos relation)
    A = as_matrix(gen.varcoef_stencil((6, 6), seed=4)).toarray()
    b = np.random.default_rng(1).standard_normal(36)
    al, be, rs, _ = pins.cg_coefficients(A, b, 8)
    V = np.column_stack([(-1) ** j * rs[j] / np.linalg.norm(rs[j]) for j in range(8)])
    T = ritz.lanczos_t(al, be[:7])
    assert np.allclose(V.T @ A @ V, T, rtol=0, atol=1e-12 * np.abs(T).max())


def test_ritz_values_converge_to_poisson_closed_form(poisson64_cg):
    _, al, be, _, _ = poisson64_cg
    w = np.linalg.eigvalsh(ritz.lanczos_t(al, be[:-1]))
    ex = pins.poisson2d_eigs(64)
    assert abs(w[0] - ex[0]) / ex[0] < 1e-9
    assert abs(w[-1] - ex[-1]) / ex[-1] < 1e-12


def test_cholesky_factor_of_t(poisson64_cg):
    _, al, be, _, _ = poisson64_cg
    zeta, eta = ritz.cholesky_lt(al[:30], be[:29])
    Lt = np.diag(zeta) + np.diag(eta, 1)
    T = ritz.lanczos_t(al[:30], be[:29])
    assert np.allclose(Lt.T @ Lt, T, rtol=1e-13, atol=0)


def test_mt_exact_at_i_two(poisson64_cg):
    _, al, be, _, _ = poisson64_cg
    assert pins.check_mt_exact_at_two(ritz.RitzTracker, al[0], al[1], be[0]) < 1e-14
    assert pins.check_mt_exact_at_two(ritz.RitzTracker, 0.3, 0.9, 0.6) < 1e-14


def test_mt_bounds_and_monotone(poisson64_cg):
    _, al, be, _, _ = poisson64_cg
    tr = ritz.RitzTracker()
    prev_min, prev_max = math.inf, -math.inf
    for i in range(len(al)):
        lmin, lmax = tr.push(al[i], be[i - 1] if i else None)
        if i >= 2 and i % 10 == 0:
            w = np.linalg.eigvalsh(ritz.lanczos_t(al[: i + 1], be[:i]))
            assert lmax <= w[-1] * (1 + 1e-14)       # Rayleigh quotient of T
            assert lmin >= w[0] * (1 - 1e-14)        # Rayleigh quotient of T^{-1}
        assert lmax >= prev_max * (1 - 1e-15) and lmin <= prev_min * (1 + 1e-15)
        prev_min, prev_max = lmin, lmax


def test_mt_incremental_equals_from_scratch(poisson64_cg):
    _, al, be, _, _ = poisson64_cg
    tr = ritz.RitzTracker()
    for i in range(60):
        inc = tr.push(al[i], be[i - 1] if i else None)
    scratch = ritz.mt_estimates(al[:60], be[:59])
    assert inc == scratch


def test_alg4_vector_is_a_unit_rayleigh_vector():
    # Alg. 4 keeps omega = ||y^T L^{-1}||^2 for a unit y built from the (g, h)
    # rotations: rebuild y densely and compare (pins d, a, g, h and the signs).
    rng = np.random.default_rng(3)
    alpha = rng.uniform(0.2, 2.0, 12)
    beta = rng.uniform(0.1, 0.9, 11)
    zeta, eta = ritz.cholesky_lt(alpha, beta)
    est = ritz.NormLinv(zeta[0])
    y = np.array([1.0])
    for l in range(11):
        est.step(zeta[l], eta[l], zeta[l + 1])
        y = np.concatenate([est.g * y, [est.h]])
        L = (np.diag(zeta[: l + 2]) + np.diag(eta[: l + 1], 1)).T
        w = y @ np.linalg.inv(L)
        assert abs(np.linalg.norm(y) - 1.0) < 1e-13
        assert abs(w @ w - est.omega) / est.omega < 1e-12


def test_alg3_vector_is_a_unit_rayleigh_vector():
    rng = np.random.default_rng(4)
    alpha = rng.uniform(0.2, 2.0, 12)
    beta = rng.uniform(0.1, 0.9, 11)
    zeta, eta = ritz.cholesky_lt(alpha, beta)
    est = ritz.NormL(zeta[0])
    T = ritz.lanczos_t(alpha, beta)
    v = np.array([1.0])
    for l in range(11):
        om_prev = est.omega
        est.step(zeta[l], eta[l], zeta[l + 1])
        # the 2x2 Rayleigh-Ritz step: the new unit vector is (c v, s) with s^2 = h
        Tl = T[: l + 2, : l + 2]
        s = math.sqrt(est.h)
        cands = []
        for sg in (1.0, -1.0):
            u = np.concatenate([math.sqrt(1 - est.h) * v, [sg * s]])
            cands.append((u @ Tl @ u, u))
        q, v = max(cands, key=lambda t: t[0])
        assert abs(q - est.omega) / est.omega < 1e-12
        assert est.omega >= om_prev


def test_exact_ritz_values_are_the_ritz_values():
    # f3: the exact tracker's values are the extreme eigenvalues of V^T A V
    assert pins.check_exact_ritz(ritz.ExactRitz) < 1e-13


def test_mt_estimates_lie_inside_the_exact_ritz_interval(poisson64_cg):
    # Algs. 3-4 give Rayleigh quotients of T_i (unit vectors), so they lie in
    # [lambda_min(T_i), lambda_max(T_i)]
    _, al, be, _, _ = poisson64_cg
    mt, ex = ritz.RitzTracker(), ritz.ExactRitz()
    for i in range(60):
        a, b_ = al[i], be[i - 1] if i else None
        mn, mx = mt.push(a, b_)
        en, exx = ex.push(a, b_)
        assert en * (1 - 1e-12) <= mn and mx <= exx * (1 + 1e-12), (i, en, mn, mx, exx)
