"""Pins for the dense adjoint: central finite differences of the dense solve."""
import copy

import numpy as np
import pytest

from oracle import adjoint
from sscg_inputs import generators as gen


@pytest.mark.parametrize("shape", [(6, 7), (4, 3, 5)])
def test_face_gradients_match_central_differences(shape):
    st = gen.varcoef_stencil(shape, seed=3)
    n = st.n
    b = gen.random_rhs(n, 1)
    xt = gen.random_rhs(n, 2)
    L, x, lam, gkx, gky, gkz = adjoint.face_gradients(st, b, xt)
    rng = np.random.default_rng(0)
    arrays = [("kx", gkx), ("ky", gky)] + ([("kz", gkz)] if gkz is not None else [])
    for name, g in arrays:
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in g.shape)
            h = 1e-4 * getattr(st, name)[idx]
            sp, sm = copy.deepcopy(st), copy.deepcopy(st)
            getattr(sp, name)[idx] += h
            getattr(sm, name)[idx] -= h
            fd = (adjoint.loss(sp, b, xt) - adjoint.loss(sm, b, xt)) / (2 * h)
            assert abs(fd - g[idx]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (name, idx, fd, g[idx])


def test_b_gradient_is_adjoint_state():
    st = gen.varcoef_stencil((5, 5), seed=1)
    b = gen.random_rhs(25, 1)
    xt = gen.random_rhs(25, 2)
    L, x, lam, *_ = adjoint.face_gradients(st, b, xt)
    for i in (0, 7, 24):
        h = 1e-4
        bp, bm = b.copy(), b.copy()
        bp[i] += h
        bm[i] -= h
        fd = (adjoint.loss(st, bp, xt) - adjoint.loss(st, bm, xt)) / (2 * h)
        assert abs(fd - lam[i]) <= 1e-7 * max(1.0, abs(fd))


def test_csr_value_gradients_match_central_differences():
    # each stored entry of a small RGG Laplacian (diagonally scaled, SPD) is a
    # free parameter; perturbing one entry alone gives a non-symmetric matrix,
    # solved densely in both the finite difference and the adjoint
    prob = gen.rgg_laplacian_csr(300, 7)
    A = prob.scipy()
    b = gen.random_rhs(A.shape[0], 1)
    xt = gen.random_rhs(A.shape[0], 2)
    L, x, lam, gval = adjoint.csr_value_gradients(A, b, xt)
    M = A.toarray()
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    rng = np.random.default_rng(4)

    def loss_of(Mp):
        xp = np.linalg.solve(Mp, b)
        return float((xp - xt) @ (xp - xt))

    for k in rng.choice(A.nnz, 12, replace=False):
        i, j = rows[k], A.indices[k]
        h = 1e-5 * abs(M[i, j])
        Mp, Mm = M.copy(), M.copy()
        Mp[i, j] += h
        Mm[i, j] -= h
        fd = (loss_of(Mp) - loss_of(Mm)) / (2 * h)
        assert abs(fd - gval[k]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(gval).max()), (i, j, fd, gval[k])
