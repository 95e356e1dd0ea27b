"""Operator assembly for the oracle (TEST INFRASTRUCTURE ONLY).

A stencil problem is given by per-face conductivities k_f.  Its operator is
``(A u)_i = sum_{faces f of i} k_f (u_i - u_nb(f))`` with ``u_nb = 0``
outside the grid (homogeneous Dirichlet), i.e. A is the sum over interior
faces of k_f (e_i - e_j)(e_i - e_j)^T plus k_f e_i e_i^T for each boundary
face.  A is symmetric positive definite when every k_f > 0.  This is the
model problem class standing in for the paper's SuiteSparse matrices
(Section 5, Table 1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def stencil_matrix(st) -> sp.csr_matrix:
    """Assemble the sparse SPD matrix of a 2D 5-point or 3D 7-point stencil."""
    shape = st.shape
    N = int(np.prod(shape))
    idx = np.arange(N).reshape(shape)
    diag = np.zeros(shape)
    rows, cols, vals = [], [], []
    faces = [(st.kx, -1)]  # (array, axis) with axis counted from the end
    faces.append((st.ky, -2))
    if st.dim == 3:
        faces.append((st.kz, -3))
    for k, axis in faces:
        ax = st.dim + axis
        n_ax = shape[ax]
        # face m along this axis lies between cells m-1 and m (m = 0..n_ax)
        lo = [slice(None)] * st.dim
        hi = [slice(None)] * st.dim
        # cell c receives its low face k[c] and high face k[c+1]
        lo[ax] = slice(0, n_ax)
        hi[ax] = slice(1, n_ax + 1)
        diag += k[tuple(lo)] + k[tuple(hi)]
        # interior faces m = 1..n_ax-1 couple cells m-1 and m
        inner = [slice(None)] * st.dim
        inner[ax] = slice(1, n_ax)
        a = [slice(None)] * st.dim
        b = [slice(None)] * st.dim
        a[ax] = slice(0, n_ax - 1)
        b[ax] = slice(1, n_ax)
        kin = k[tuple(inner)].ravel()
        ia = idx[tuple(a)].ravel()
        ib = idx[tuple(b)].ravel()
        rows += [ia, ib]
        cols += [ib, ia]
        vals += [-kin, -kin]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N))
    A.sum_duplicates()
    A.sort_indices()
    return A


def as_matrix(op) -> sp.csr_matrix:
    """scipy CSR matrix of a Stencil or CsrProblem (or a scipy matrix)."""
    if sp.issparse(op):
        return op.tocsr()
    if hasattr(op, "kx"):
        return stencil_matrix(op)
    return sp.csr_matrix((op.val, op.col, op.rowptr), shape=(op.n, op.n))
