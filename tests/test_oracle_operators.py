"""Pins for the stencil operator definition and the input generators."""
import numpy as np
import scipy.sparse as sp

from oracle.operators import as_matrix, stencil_matrix
from sscg_inputs import generators as gen
from tests.pins import poisson2d_eigs, poisson3d_eigs


def test_unit_stencil_2d_equals_poisson_csr():
    # two independent constructions of the same matrix
    A1 = stencil_matrix(gen.unit_stencil((7, 7)))
    A2 = gen.poisson2d_csr(7).scipy()
    assert abs(A1 - A2).max() == 0.0


def test_unit_stencil_spectra_closed_form():
    w2 = np.linalg.eigvalsh(stencil_matrix(gen.unit_stencil((6, 6))).toarray())
    assert np.allclose(w2, poisson2d_eigs(6), rtol=0, atol=1e-12)
    w3 = np.linalg.eigvalsh(stencil_matrix(gen.unit_stencil((4, 4, 4))).toarray())
    assert np.allclose(w3, poisson3d_eigs(4), rtol=0, atol=1e-12)


def test_varcoef_stencil_is_spd_and_flux_form():
    st = gen.varcoef_stencil((3, 4, 5), seed=11)
    A = stencil_matrix(st).toarray()
    assert np.allclose(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0
    # u = 1 gives the flux through the boundary faces only (flux form)
    nz, ny, nx = st.shape
    bnd = np.zeros(st.shape)
    bnd[:, :, 0] += st.kx[:, :, 0]
    bnd[:, :, -1] += st.kx[:, :, nx]
    bnd[:, 0, :] += st.ky[:, 0, :]
    bnd[:, -1, :] += st.ky[:, ny, :]
    bnd[0, :, :] += st.kz[0, :, :]
    bnd[-1, :, :] += st.kz[nz, :, :]
    assert np.allclose(A @ np.ones(A.shape[0]), bnd.ravel())
    # one interior coupling, checked by hand: cells (1,2,3) and (1,2,4) share kx[1,2,4]
    i = (1 * ny + 2) * nx + 3
    assert A[i, i + 1] == -st.kx[1, 2, 4]
    assert A[i, i + nx] == -st.ky[1, 3, 3]
    assert A[i, i + nx * ny] == -st.kz[2, 2, 3]


def test_varcoef_2d_quadratic_form():
    st = gen.varcoef_stencil((5, 6), seed=2)
    A = stencil_matrix(st)
    u = np.random.default_rng(0).standard_normal(30).reshape(5, 6)
    # u^T A u = sum over faces k_f (jump of u across f)^2 with u = 0 outside
    up = np.pad(u, 1)
    q = (st.kx * (up[1:-1, 1:] - up[1:-1, :-1]) ** 2).sum() + \
        (st.ky * (up[1:, 1:-1] - up[:-1, 1:-1]) ** 2).sum()
    assert np.isclose(u.ravel() @ (A @ u.ravel()), q, rtol=1e-13)


def test_generators_are_seeded():
    a = gen.varcoef_stencil((4, 4, 4), seed=5)
    b = gen.varcoef_stencil((4, 4, 4), seed=5)
    assert np.array_equal(a.kx, b.kx) and np.array_equal(a.kz, b.kz)
    assert np.array_equal(gen.random_rhs(10, 3), gen.random_rhs(10, 3))


def test_rgg_laplacian_small():
    P = gen.rgg_laplacian_csr(3000, seed=7)
    A = P.scipy()
    assert (A - A.T).count_nonzero() == 0 or abs(A - A.T).max() < 1e-12
    nnz_row = np.diff(P.rowptr).mean()
    assert 15 < nnz_row < 40
    w = sp.linalg.eigsh(A, k=1, which="SA", return_eigenvectors=False)
    assert w[0] > 0


def test_batched_generator_shapes():
    systems = gen.batched_stencils(6, seed=1, n_lo=100, n_hi=2000)
    for st, B in systems:
        assert B.shape[1] == st.n and 1 <= B.shape[0] <= 8
        assert 40 <= st.n <= 4000
    assert as_matrix(systems[0][0]).shape[0] == systems[0][0].n
