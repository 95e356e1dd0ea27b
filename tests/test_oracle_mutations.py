"""Plant plausible mistakes in a copy of the oracle and check that a pin catches each.

Each case rewrites one line of an oracle module's source (on the CPU, in a
fresh module object) and runs the pin that should fail.  The real oracle is
never modified.
"""
import importlib
import importlib.util
import math
import sys
import types

import numpy as np
import pytest

from oracle.operators import as_matrix
from sscg_inputs import generators as gen
from tests import pins


def mutated(modname: str, old: str, new: str, extra: dict | None = None) -> types.ModuleType:
    """A fresh copy of oracle.<modname> with one source substring replaced."""
    spec = importlib.util.find_spec(f"oracle.{modname}")
    src = open(spec.origin).read()
    assert src.count(old) == 1, f"mutation anchor not unique in {modname}: {old!r}"
    src = src.replace(old, new)
    mod = types.ModuleType(f"oracle._mut_{modname}")
    mod.__package__ = "oracle"
    mod.__file__ = spec.origin
    sys.modules[mod.__name__] = mod
    exec(compile(src, spec.origin, "exec"), mod.__dict__)
    for k, v in (extra or {}).items():
        setattr(mod, k, v)
    return mod


def test_dropped_mu_term_fails_chebyshev_pin():
    m = mutated("basis", "w = w - mu[l - 1] * Y[:, index(l - 1)]", "w = w")
    assert pins.check_chebyshev_closed_form(m.krylov_basis, m.basis_params) > 1e-3


def test_wrong_mu_sign_fails_chebyshev_pin():
    m = mutated("basis", "w = w - mu[l - 1] * Y[:, index(l - 1)]",
                "w = w + mu[l - 1] * Y[:, index(l - 1)]")
    assert pins.check_chebyshev_closed_form(m.krylov_basis, m.basis_params) > 1e-3


def test_transposed_b_fails_avvb_pin():
    m = mutated("basis", "B[index(l + 1), index(l)] = gamma[l]", "B[index(l), index(l + 1)] = gamma[l]")
    A = as_matrix(gen.varcoef_stencil((6, 6), seed=1))
    assert pins.check_avvb(m.krylov_basis, m.b_matrix, m.basis_params, A, 2, 4) > 1e-3


def test_shifted_theta_index_fails_newton_pin():
    m = mutated("basis", "w = A @ v - theta[l] * v", "w = A @ v - theta[max(l - 1, 0)] * v")
    assert pins.check_newton_closed_form(m.krylov_basis, m.basis_params) > 1e-6


def test_leja_tie_to_larger_fails_closed_form():
    m = mutated("basis", "elif abs(v - best_v) <= 1e-13 and t < best_t:",
                "elif abs(v - best_v) <= 1e-13 and t > best_t:")
    t = m.leja_points(4)
    assert abs(t[3] + 1.0 / math.sqrt(3.0)) > 1e-3


def test_alg3_wrong_index_fails_exactness():
    m = mutated("ritz", "a = eta_l * eta_l + zeta_l1 * zeta_l1", "a = eta_l * eta_l + zeta_l * zeta_l")
    assert pins.check_mt_exact_at_two(m.RitzTracker, 0.3, 0.9, 0.6) > 1e-6


def test_alg4_unsigned_h_fails_rayleigh_pin():
    m = mutated("ritz", "self.h = abs(h) * _sign(d1)", "self.h = abs(h)")
    rng = np.random.default_rng(3)
    alpha = rng.uniform(0.2, 2.0, 12)
    beta = rng.uniform(0.1, 0.9, 11)
    zeta, eta = m.cholesky_lt(alpha, beta)
    est = m.NormLinv(zeta[0])
    y = np.array([1.0])
    worst = 0.0
    for l in range(11):
        est.step(zeta[l], eta[l], zeta[l + 1])
        y = np.concatenate([est.g * y, [est.h]])
        L = (np.diag(zeta[: l + 2]) + np.diag(eta[: l + 1], 1)).T
        w = y @ np.linalg.inv(L)
        worst = max(worst, abs(w @ w - est.omega) / est.omega)
    assert worst > 1e-6


def test_alg4_bad_recurrence_fails_bounds():
    m = mutated("ritz", "a1 = (eta_l * eta_l * self.a + 1.0) / (zeta_l1 * zeta_l1)",
                "a1 = (eta_l * eta_l * self.a + 1.0) * (zeta_l1 * zeta_l1)")
    assert pins.check_mt_exact_at_two(m.RitzTracker, 0.3, 0.9, 0.6) > 1e-6


def _sigma_one_vs_hscg(cgmod):
    A, b, x0, _ = gen.config_problem("poisson2d_64", scale=24)
    M = as_matrix(A)
    _, h = cgmod.hscg(M, b, x0, 1e-10)
    _, s = cgmod.sstep_cg(M, b, x0, 1e-10, cgmod.Options(smax=1, basis="chebyshev",
                                                          max_outer=400))
    k = min(len(s["alphas"]), len(h["alphas"]), 30)
    return np.max(np.abs(np.array(s["alphas"][:k]) - np.array(h["alphas"][:k]))
                  / np.array(h["alphas"][:k]))


def test_inverted_beta_fails_sigma_one_pin():
    m = mutated("cg", "beta = rr_new / rr\n            pc = rc + beta * pc",
                "beta = rr / rr_new\n            pc = rc + beta * pc")
    assert _sigma_one_vs_hscg(m) > 1e-3


def test_wrong_alpha_denominator_fails_sigma_one_pin():
    m = mutated("cg", "den = float(pc @ (Gs @ Bp))", "den = float(pc @ (Gs @ pc))")
    assert _sigma_one_vs_hscg(m) > 1e-3


def test_forgotten_x_accumulation_fails_convergence():
    m = mutated("cg", "x = x + Yn @ xc", "x = Yn @ xc")
    A, b, x0, _ = gen.config_problem("poisson2d_64", scale=24)
    x, info = m.sstep_cg(as_matrix(A), b, x0, 1e-10, m.Options(smax=4, basis="chebyshev",
                                                                 max_outer=60))
    assert info["relres_true"] > 1e-6


def test_swapped_newton_endpoints_fail_explicit_pin():
    m = mutated("basis", "theta = c + h * leja_points(s)", "theta = c - h * leja_points(s)")
    th, _, _ = m.basis_params(1, 4, 0.5, 3.5)
    # eq. (newtbasis): theta_0 = lmax, theta_1 = lmin
    assert not (th[0] == 3.5 and th[1] == 0.5)
