"""Dense adjoint of the differentiable solve (TEST INFRASTRUCTURE ONLY).

For x(k) = A(k)^{-1} b with A(k) = sum over interior faces f = (i, j) of
k_f (e_i - e_j)(e_i - e_j)^T plus k_f e_i e_i^T for each boundary face of
cell i, and a loss L(x), the adjoint state lam = A^{-1} dL/dx gives
  dL/db   = lam
  dL/dk_f = -(lam_i - lam_j)(x_i - x_j)   (interior face)
  dL/dk_f = -lam_i x_i                   (boundary face)
  dL/dA_ij = -lam_i x_j                  (a free CSR entry)
This module evaluates them with dense solves for tiny grids; it is pinned by
central finite differences of the same dense solve.
"""
from __future__ import annotations

import numpy as np

from .operators import stencil_matrix


def face_gradients(st, b, x_target):
    """(L, x, lam, gkx, gky, gkz) for L = ||x - x_target||^2, dense solves."""
    A = stencil_matrix(st).toarray()
    x = np.linalg.solve(A, b)
    g = 2.0 * (x - x_target)
    lam = np.linalg.solve(A, g)
    L = float((x - x_target) @ (x - x_target))
    shape = st.shape
    X = x.reshape(shape)
    Lm = lam.reshape(shape)
    pad = [(1, 1)] * st.dim
    Xp = np.pad(X, pad)
    Lp = np.pad(Lm, pad)

    def grad_axis(axis):
        # face m along `axis` lies between padded cells m and m+1 (one of them may be padding = 0)
        sl_lo = [slice(1, -1)] * st.dim
        sl_hi = [slice(1, -1)] * st.dim
        n_ax = shape[axis]
        sl_lo[axis] = slice(0, n_ax + 1)
        sl_hi[axis] = slice(1, n_ax + 2)
        dx = Xp[tuple(sl_hi)] - Xp[tuple(sl_lo)]
        dl = Lp[tuple(sl_hi)] - Lp[tuple(sl_lo)]
        return -(dl * dx)

    gkx = grad_axis(st.dim - 1)
    gky = grad_axis(st.dim - 2)
    gkz = grad_axis(0) if st.dim == 3 else None
    return L, x, lam, gkx, gky, gkz


def loss(st, b, x_target):
    A = stencil_matrix(st).toarray()
    x = np.linalg.solve(A, b)
    return float((x - x_target) @ (x - x_target))


def csr_value_gradients(A, b, x_target):
    """(L, x, lam, gval) for L = ||x - x_target||^2 and a CSR matrix A (scipy),
    dense solves: gval[k] = dL/dA_ij = -lam_i x_j for the k-th stored entry
    (i, j) (row i of the CSR order), each entry a free parameter."""
    M = A.toarray()
    x = np.linalg.solve(M, b)
    lam = np.linalg.solve(M.T, 2.0 * (x - x_target))
    L = float((x - x_target) @ (x - x_target))
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    gval = -lam[rows] * x[A.indices]
    return L, x, lam, gval
