"""Pins for eq. (rho), eq. (B)/(AVVB), Leja points (eq. newtbasis) and the Chebyshev basis."""
import math

import numpy as np
import pytest

from oracle import basis as bs
from oracle.operators import stencil_matrix
from sscg_inputs import generators as gen
from tests import pins


def test_leja_closed_form_first_points():
    t = bs.leja_points(4)
    assert t[0] == 1.0 and t[1] == -1.0
    assert t[2] == 0.0                                   # maximiser of |1 - t^2|
    assert abs(t[3] + 1.0 / math.sqrt(3.0)) < 1e-15     # maximiser of |t^3 - t|, tie -> smaller t


def test_leja_points_brute_force_grid():
    t = bs.leja_points(12)
    grid = np.linspace(-1.0, 1.0, 400001)
    for l in range(2, 12):
        logp = np.sum(np.log(np.abs(grid[:, None] - t[None, :l]) + 1e-300), axis=1)
        g = grid[np.argmax(logp)]
        # the grid optimum is within one grid step of the computed point
        assert abs(g - t[l]) <= 1e-5, (l, g, t[l])
        # and nothing on the grid beats the computed product
        val = np.sum(np.log(np.abs(t[l] - t[:l])))
        assert val >= logp.max() - 1e-9


def test_chebyshev_standard_is_cos_l_arccos():
    assert pins.check_chebyshev_closed_form(bs.krylov_basis, bs.basis_params) < 1e-12


def test_newton_basis_is_product_form():
    assert pins.check_newton_closed_form(bs.krylov_basis, bs.basis_params) < 1e-13


def test_monomial_basis_powers():
    z = np.linspace(0.5, 1.5, 20)
    import scipy.sparse as sp
    th, ga, mu = bs.basis_params(bs.MONOMIAL, 5, None, None)
    Y = bs.krylov_basis(sp.diags(z), np.ones(20), 2 * np.ones(20), 5, th, ga, mu)
    for l in range(6):
        assert np.allclose(Y[:, 2 * l], z ** l, rtol=1e-15)
    for l in range(5):
        assert np.allclose(Y[:, 2 * l + 1], 2 * z ** l, rtol=1e-15)


def test_paper_printed_chebyshev_values():
    th, ga, mu = bs.basis_params(bs.CHEBYSHEV, 4, 1.0, 5.0, cheb_params="paper_printed")
    assert np.all(th == 3.0) and ga[0] == 4.0 and np.all(ga[1:] == 2.0) and np.all(mu == 8.0)


@pytest.mark.parametrize("kind", [bs.MONOMIAL, bs.NEWTON, bs.CHEBYSHEV])
@pytest.mark.parametrize("s", [1, 2, 5, 8])
def test_avvb_identity(kind, s):
    A = stencil_matrix(gen.varcoef_stencil((6, 7), seed=9))
    assert pins.check_avvb(bs.krylov_basis, bs.b_matrix, bs.basis_params, A, kind, s) < 1e-13


def test_b_matrix_s1_structure():
    B = bs.b_matrix(1, [0.7], [1.3], [0.0])
    expect = np.zeros((3, 3))
    expect[0, 0] = 0.7   # A P_0 = theta_0 P_0 + gamma_0 P_1
    expect[2, 0] = 1.3
    assert np.array_equal(B, expect)


def test_leading_block_is_smaller_basis():
    # Y_l of a larger basis equals the basis built with s = l (nesting, reading C9)
    A = stencil_matrix(gen.varcoef_stencil((5, 5), seed=1))
    rng = np.random.default_rng(0)
    p, r = rng.standard_normal(25), rng.standard_normal(25)
    th, ga, mu = bs.basis_params(bs.NEWTON, 6, 0.1, 6.0)
    Y6 = bs.krylov_basis(A, p, r, 6, th, ga, mu)
    Y3 = bs.krylov_basis(A, p, r, 3, th, ga, mu)
    assert np.array_equal(Y6[:, :7], Y3)


def test_newton_shifts_start_with_lmax_then_lmin():
    th, ga, mu = bs.basis_params(bs.NEWTON, 5, 0.5, 3.5)
    assert th[0] == 3.5 and th[1] == 0.5              # eq. (newtbasis)
    assert th[2] == 2.0                                # midpoint: t_2 = 0
    assert np.all(mu == 0) and np.all(ga == 0.75)     # capacity (lmax - lmin)/4 (reading C6)
    _, ga1, _ = bs.basis_params(bs.NEWTON, 5, 0.5, 3.5, newton_scale="paper_unit")
    assert np.all(ga1 == 1.0)
