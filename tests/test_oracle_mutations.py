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


# ------------------------------------------------- Alg. 5's adaptive decisions
from tests import test_oracle_decisions as dec  # noqa: E402


def _fails(pin, *args) -> bool:
    try:
        pin(*args)
    except AssertionError:
        return True
    return False


def test_condy_strict_inequality_fails_boundary_pin():
    m = mutated("cg", "if kap[l] <= thr]", "if kap[l] < thr]")
    assert _fails(dec.test_condy_largest_admissible_l_with_equality, m.choose_stilde)


def test_condy_without_relative_residual_fails_pin():
    m = mutated("cg", "thr = tol / (c * eps * normr / normb)\n    cands",
                "thr = tol / (c * eps * normr)\n    cands")
    assert _fails(dec.test_condy_uses_the_relative_residual, m.choose_stilde)


def test_condy_first_failure_instead_of_largest_fails_pin():
    m = mutated("cg", "return max(cands) if cands else 1",
                "return next((l - 1 for l in range(1, sbar + 1) if l not in cands), sbar) or 1")
    assert _fails(dec.test_condy_largest_admissible_l_with_equality, m.choose_stilde)


def test_condy_empty_set_not_one_fails_pin():
    m = mutated("cg", "return max(cands) if cands else 1", "return max(cands) if cands else sbar")
    assert _fails(dec.test_condy_no_admissible_l_gives_one, m.choose_stilde)


def test_condy_with_p_norm_fails_records_pin():
    m = mutated("cg", "normr = math.sqrt(G[1, 1])", "normr = math.sqrt(G[0, 0])")
    assert dec.check_condy_records(m) > 0


def test_newcondy_strict_inequality_fails_boundary_pin():
    m = mutated("cg", "return gam_next >= tol", "return gam_next > tol")
    assert _fails(dec.test_newcondy_break_at_equality, m.break_test)


def test_newcondy_without_relative_residual_fails_pin():
    m = mutated("cg", "(c * eps * phi / normb)", "(c * eps * phi)")
    assert _fails(dec.test_newcondy_break_at_equality, m.break_test)


def test_newcondy_with_current_residual_fails_records_pin():
    m = mutated("cg", "break_test(gam[j + 1], tol, c, eps, phi, normb)",
                "break_test(gam[j + 1], tol, c, eps, math.sqrt(rr_new), normb)")
    assert dec.check_break_records(m) > 0


def test_newcondy_gamma_index_fails_records_pin():
    m = mutated("cg", "gam = {l: kap[l + 1] for l in range(1, stilde)}",
                "gam = {l: kap[l] for l in range(1, stilde)}")
    assert dec.check_break_records(m) > 0


def test_psi_wrong_recurrence_fails_worked_values():
    m = mutated("cg", "return psi / (psi + beta)", "return psi / (1.0 + beta)")
    assert _fails(dec.test_psi_recurrence_worked_values, m.psi_update)


def test_psi_updated_with_previous_beta_fails_identity():
    m = mutated("cg", "psi = psi_update(psi, beta)",
                "psi = psi_update(psi, betas[-1] if betas else 0.0)")
    assert dec.check_psi_records(m) > 1e-6


def test_c_gate_from_first_iteration_fails_pins():
    m = mutated("cg", "return m + j + 1 > 1", "return m + j + 1 > 0")
    assert _fails(dec.test_ritz_c_gate, m.uses_ritz_c)
    assert dec.check_first_ritz_c(m) > 1e-6


def test_c_from_stale_psi_fails_first_ritz_pin():
    m = mutated("cg", "c = c_value(o.c_mode, ritz.lmin, ritz.lmax, psi, o.c_const)",
                "c = c_value(o.c_mode, ritz.lmin, ritz.lmax, 1.0, o.c_const)")
    assert dec.check_first_ritz_c(m) > 1e-6


def test_kappa_cut_strict_fails_boundary_pin():
    m = mutated("cg", "w[0] <= kappa_cut * w[-1]", "w[0] < kappa_cut * w[-1]")
    assert _fails(dec.test_kappa_cut_boundary, m.kappa_estimates)


def test_exact_ritz_offdiagonal_index_fails_pin():
    # f3: the coupling sqrt(beta_{i-1}) / alpha_{i-1} taken with alpha_i
    m = mutated("ritz", "self.e.append(math.sqrt(beta_prev) / self._alpha_prev)",
                "self.e.append(math.sqrt(beta_prev) / alpha)")
    assert pins.check_exact_ritz(m.ExactRitz) > 1e-6


def test_exact_ritz_diagonal_term_fails_pin():
    # f3: the diagonal 1/alpha_i + beta_{i-1}/alpha_{i-1} taken with alpha_i twice
    m = mutated("ritz", "self.d.append(1.0 / alpha + beta_prev / self._alpha_prev)",
                "self.d.append(1.0 / alpha + beta_prev / alpha)")
    assert pins.check_exact_ritz(m.ExactRitz) > 1e-6
