"""Seeded synthetic problem generators (numpy PCG64).

Every generator is deterministic in its ``seed``.  The workloads stand in for
the SuiteSparse matrices of the paper's Section 5 (Table 1), which are not
available here: SPD, sparse, at most 27 nonzeros per row, condition numbers
from about 1e3 to 1e8.

Stencil convention (both 2D and 3D): cells are indexed with x fastest, then y,
then z.  A stencil operator is given by per-face conductivities; the operator
is ``(A u)_i = sum over the faces f of cell i of k_f (u_i - u_nb(f))`` with
``u_nb = 0`` outside the grid (homogeneous Dirichlet), so boundary faces add
``k_f`` to the diagonal only.

Face arrays (C order):
  2D (ny, nx):  kx (ny, nx+1)  west face of (y,x) is kx[y,x], east is kx[y,x+1]
                ky (ny+1, nx)  south face is ky[y,x], north is ky[y+1,x]
  3D (nz, ny, nx): kx (nz, ny, nx+1), ky (nz, ny+1, nx), kz (nz+1, ny, nx)
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import reverse_cuthill_mckee

# seed = 1000 + index of the workload in the list of configurations
CONFIG_SEEDS = {"poisson2d_64": 1000, "varcoef3d_160": 1001, "rgg_2m": 1002,
                "batched_256": 1003, "adjoint2d_512": 1004}


@dataclasses.dataclass
class Stencil:
    """Per-face conductivities of a 2D 5-point or 3D 7-point stencil."""
    shape: tuple          # (ny, nx) or (nz, ny, nx)
    kx: np.ndarray
    ky: np.ndarray
    kz: np.ndarray | None = None

    @property
    def dim(self) -> int:
        return len(self.shape)

    @property
    def n(self) -> int:
        return int(np.prod(self.shape))


@dataclasses.dataclass
class CsrProblem:
    """A sparse symmetric matrix in CSR form (int64 row pointers, int32 columns)."""
    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    def scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))


def poisson2d_csr(n: int) -> CsrProblem:
    """Unit-coefficient 5-point Dirichlet Laplacian on an n x n grid, as CSR.

    Diagonal 4, off-diagonals -1 for the (up to four) grid neighbours.
    """
    N = n * n
    rows, cols, vals = [], [], []
    idx = np.arange(N).reshape(n, n)
    for dy, dx in ((0, 0), (0, -1), (0, 1), (-1, 0), (1, 0)):
        ys, xs = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        yn, xn = ys + dy, xs + dx
        ok = (yn >= 0) & (yn < n) & (xn >= 0) & (xn < n)
        rows.append(idx[ys[ok], xs[ok]])
        cols.append(idx[yn[ok], xn[ok]])
        vals.append(np.full(ok.sum(), 4.0 if (dy, dx) == (0, 0) else -1.0))
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N))
    A.sort_indices()
    return CsrProblem(N, A.indptr.astype(np.int64), A.indices.astype(np.int32),
                      A.data.astype(np.float64))


def varcoef_stencil(shape, seed: int, sigma: float = 1.0) -> Stencil:
    """Per-face conductivities k = exp(g), g i.i.d. N(0, sigma^2) per face."""
    rng = np.random.default_rng(seed)
    if len(shape) == 2:
        ny, nx = shape
        kx = np.exp(sigma * rng.standard_normal((ny, nx + 1)))
        ky = np.exp(sigma * rng.standard_normal((ny + 1, nx)))
        return Stencil(tuple(shape), kx, ky, None)
    nz, ny, nx = shape
    kx = np.exp(sigma * rng.standard_normal((nz, ny, nx + 1)))
    ky = np.exp(sigma * rng.standard_normal((nz, ny + 1, nx)))
    kz = np.exp(sigma * rng.standard_normal((nz + 1, ny, nx)))
    return Stencil(tuple(shape), kx, ky, kz)


def unit_stencil(shape) -> Stencil:
    """All face conductivities 1 (the constant-coefficient Dirichlet Laplacian)."""
    if len(shape) == 2:
        ny, nx = shape
        return Stencil(tuple(shape), np.ones((ny, nx + 1)), np.ones((ny + 1, nx)), None)
    nz, ny, nx = shape
    return Stencil(tuple(shape), np.ones((nz, ny, nx + 1)), np.ones((nz, ny + 1, nx)),
                   np.ones((nz + 1, ny, nx)))


def random_rhs(n: int, seed: int, nrhs: int | None = None) -> np.ndarray:
    """b ~ N(0, 1), seeded."""
    rng = np.random.default_rng(seed)
    if nrhs is None:
        return rng.standard_normal(n)
    return rng.standard_normal((nrhs, n))


def uniform_vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """x ~ U(lo, hi), seeded."""
    return np.random.default_rng(seed).uniform(lo, hi, n)


def rgg_laplacian_csr(N: int, seed: int, avg_nnz: float = 27.0, shift_frac: float = 1e-4,
                      scale_decades: float = 3.0) -> CsrProblem:
    """Graph Laplacian of a 3D random geometric graph, RCM-ordered, shifted and scaled.

    N points uniform in the unit cube; edges between points closer than
    r = ((avg_nnz - 1) / (N * 4 pi / 3))^(1/3) (found with cell lists), unit
    weights.  A = L + shift_frac * mean_degree * I, symmetrically permuted by
    reverse Cuthill-McKee, then S A S with S = diag(10^{U(0, scale_decades)/2})
    so that the diagonal scaling d_i = S_i^2 = 10^{U(0, scale_decades)}.
    """
    rng = np.random.default_rng(seed)
    pts = rng.random((N, 3))
    r = ((avg_nnz - 1.0) / (N * 4.0 * math.pi / 3.0)) ** (1.0 / 3.0)
    ncell = max(1, int(1.0 / r))
    cell = np.minimum((pts * ncell).astype(np.int64), ncell - 1)
    key = (cell[:, 2] * ncell + cell[:, 1]) * ncell + cell[:, 0]
    order = np.argsort(key, kind="stable")
    key_s = key[order]
    starts = np.searchsorted(key_s, np.arange(ncell ** 3), side="left")
    ends = np.searchsorted(key_s, np.arange(ncell ** 3), side="right")
    src_all, dst_all = [], []
    r2 = r * r
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                cz, cy, cx = cell[:, 2] + dz, cell[:, 1] + dy, cell[:, 0] + dx
                ok = (cz >= 0) & (cz < ncell) & (cy >= 0) & (cy < ncell) & (cx >= 0) & (cx < ncell)
                ii = np.nonzero(ok)[0]
                nk = (cz[ii] * ncell + cy[ii]) * ncell + cx[ii]
                s0, s1 = starts[nk], ends[nk]
                cnt = s1 - s0
                tot = int(cnt.sum())
                if tot == 0:
                    continue
                src = np.repeat(ii, cnt)
                offs = np.arange(tot) - np.repeat(np.cumsum(cnt) - cnt, cnt)
                dst = order[np.repeat(s0, cnt) + offs]
                d = pts[src] - pts[dst]
                keep = (np.einsum("ij,ij->i", d, d) < r2) & (src != dst)
                src_all.append(src[keep])
                dst_all.append(dst[keep])
    src = np.concatenate(src_all)
    dst = np.concatenate(dst_all)
    W = sp.csr_matrix((np.ones(src.size), (src, dst)), shape=(N, N))
    deg = np.asarray(W.sum(axis=1)).ravel()
    L = sp.diags(deg) - W
    A = (L + shift_frac * deg.mean() * sp.identity(N)).tocsr()
    perm = reverse_cuthill_mckee(A, symmetric_mode=True)
    A = A[perm][:, perm].tocsr()
    s = 10.0 ** (0.5 * rng.uniform(0.0, scale_decades, N))
    A = sp.diags(s) @ A @ sp.diags(s)
    A = A.tocsr()
    A.sort_indices()
    return CsrProblem(N, A.indptr.astype(np.int64), A.indices.astype(np.int32),
                      A.data.astype(np.float64))


def batched_stencils(count: int, seed: int, n_lo: float = 1e3, n_hi: float = 2.6e5,
                     max_rhs: int = 8):
    """Independent variable-coefficient Poisson systems of uneven sizes.

    Each system is 2D or 3D by a seeded coin; N is drawn log-uniform in
    [n_lo, n_hi] and rounded to n^2 or n^3; conductivities are log-normal;
    each system has 1..max_rhs right-hand sides b ~ N(0, 1).
    Returns a list of (Stencil, B) with B of shape (nrhs, N).
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        dim = 2 if rng.random() < 0.5 else 3
        N = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        n = max(4, int(round(N ** (1.0 / dim))))
        shape = (n,) * dim
        st = varcoef_stencil(shape, int(rng.integers(1 << 31)))
        nrhs = int(rng.integers(1, max_rhs + 1))
        B = random_rhs(st.n, int(rng.integers(1 << 31)), nrhs)
        out.append((st, B))
    return out


def config_problem(name: str, scale: int | None = None):
    """The synthetic problem of a named workload (optionally at a smaller grid size).

    Returns (operator, b, x0, extra) where operator is a Stencil or CsrProblem.
    """
    seed = CONFIG_SEEDS[name]
    if name == "poisson2d_64":
        n = scale or 64
        A = poisson2d_csr(n)
        xstar = uniform_vector(A.n, seed)
        b = A.scipy() @ xstar
        return A, b, np.zeros(A.n), {"xstar": xstar}
    if name == "varcoef3d_160":
        n = scale or 160
        st = varcoef_stencil((n, n, n), seed)
        b = random_rhs(st.n, seed + 7919)
        return st, b, np.zeros(st.n), {}
    if name == "rgg_2m":
        N = scale or 2_000_000
        A = rgg_laplacian_csr(N, seed)
        b = random_rhs(N, seed + 7919)
        return A, b, np.zeros(N), {}
    if name == "adjoint2d_512":
        n = scale or 512
        st = varcoef_stencil((n, n), seed)
        b = random_rhs(st.n, seed + 7919)
        xt = random_rhs(st.n, seed + 104729)
        return st, b, np.zeros(st.n), {"x_target": xt}
    raise KeyError(name)
