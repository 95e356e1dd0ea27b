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


def _exp_portable(y: np.ndarray) -> np.ndarray:
    """exp(y) from IEEE-rounded multiplies and adds only (no libm), so that the
    same inputs give the same bits on every platform: y = k ln2 + f with
    0 <= f < ln2, exp(f) by its Taylor series to degree 24 (Horner), times 2^k."""
    ln2 = 0.6931471805599453
    k = np.floor(y / ln2)
    f = y - k * ln2
    p = np.ones_like(f)
    for d in range(24, 0, -1):
        p = p * f
        p = p / float(d)
        p = p + 1.0
    return np.ldexp(p, k.astype(np.int64))


def _icbrt(v: int) -> int:
    """floor(v^(1/3)) for an integer v >= 0, by integer Newton steps."""
    if v < 2:
        return v
    x = 1 << ((v.bit_length() + 2) // 3)
    while True:
        y = (2 * x + v // (x * x)) // 3
        if y >= x:
            break
        x = y
    while x * x * x > v:
        x -= 1
    while (x + 1) ** 3 <= v:
        x += 1
    return x


def _rcm(A: sp.csr_matrix) -> np.ndarray:
    """Reverse Cuthill-McKee order of a structurally symmetric matrix with every
    tie broken by node index (a library's own ordering may break ties by its
    sort's order, which differs between platforms).  Level by level from the
    unvisited node of least degree: each level's new nodes are the frontier's
    unvisited neighbours, taken in frontier order, each parent's sorted by
    (degree, index), a node reached twice kept at its first parent."""
    N = A.shape[0]
    indptr, indices = A.indptr, A.indices
    deg = np.diff(indptr)
    visited = np.zeros(N, dtype=bool)
    order = []
    by_degree = np.lexsort((np.arange(N), deg))     # nodes by (degree, index)
    start_at = 0
    while True:
        while start_at < N and visited[by_degree[start_at]]:
            start_at += 1
        if start_at >= N:
            break
        frontier = np.array([by_degree[start_at]], dtype=np.int64)
        visited[frontier] = True
        order.append(frontier)
        while frontier.size:
            counts = deg[frontier]
            tot = int(counts.sum())
            if tot == 0:
                break
            starts = indptr[frontier]
            offs = np.arange(tot) - np.repeat(np.cumsum(counts) - counts, counts)
            nb = indices[np.repeat(starts, counts) + offs].astype(np.int64)
            parent = np.repeat(np.arange(frontier.size), counts)
            m = ~visited[nb]
            nb, parent = nb[m], parent[m]
            o = np.lexsort((nb, deg[nb], parent))
            nb = nb[o]
            _, first = np.unique(nb, return_index=True)
            nb = nb[np.sort(first)]
            visited[nb] = True
            order.append(nb)
            frontier = nb
    return np.concatenate(order)[::-1].astype(np.int64)


def rgg_laplacian_csr(N: int, seed: int, avg_nnz: float = 27.0, shift_frac: float = 1e-4,
                      scale_decades: float = 3.0) -> CsrProblem:
    """Graph Laplacian of a 3D random geometric graph, RCM-ordered, shifted and scaled.

    N points uniform in the unit cube; edges between points closer than
    r = ((avg_nnz - 1) / (N * 4 pi / 3))^(1/3) (found with cell lists), unit
    weights.  A = L + shift_frac * mean_degree * I, symmetrically permuted by
    reverse Cuthill-McKee, then S A S with S = diag(10^{U(0, scale_decades)/2})
    so that the diagonal scaling d_i = S_i^2 = 10^{U(0, scale_decades)}.

    Every step is exact or IEEE-rounded arithmetic with a fixed tie order, so
    the matrix is the same bit for bit on every platform: points on a 2^20
    integer grid with integer squared distances, the radius as an integer cube
    root, the ordering by _rcm, and 10^u from _exp_portable (a platform's libm
    or sort could round or order differently, which would move edges at the
    radius and with them the whole ordering).
    """
    rng = np.random.default_rng(seed)
    pts = rng.random((N, 3))
    Q = 1 << 20
    qp = np.floor(pts * Q).astype(np.int64)                   # exact: pts * 2^20 is exact
    c = (avg_nnz - 1.0) / (N * 4.0 * math.pi / 3.0)           # r^3
    R = _icbrt(int(c * float(Q) ** 3))                          # radius in grid units
    R2 = R * R
    ncell = max(1, Q // max(R, 1))                             # cells at least R wide
    cell = (qp * ncell) >> 20
    key = (cell[:, 2] * ncell + cell[:, 1]) * ncell + cell[:, 0]
    order = np.argsort(key, kind="stable")
    key_s = key[order]
    starts = np.searchsorted(key_s, np.arange(ncell ** 3), side="left")
    ends = np.searchsorted(key_s, np.arange(ncell ** 3), side="right")
    src_all, dst_all = [], []
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
                d = qp[src] - qp[dst]
                keep = (np.einsum("ij,ij->i", d, d) < R2) & (src != dst)
                src_all.append(src[keep])
                dst_all.append(dst[keep])
    src = np.concatenate(src_all)
    dst = np.concatenate(dst_all)
    W = sp.csr_matrix((np.ones(src.size), (src, dst)), shape=(N, N))
    deg = np.asarray(W.sum(axis=1)).ravel()
    L = sp.diags(deg) - W
    A = (L + shift_frac * deg.mean() * sp.identity(N)).tocsr()
    perm = _rcm(A)
    A = A[perm][:, perm].tocsr()
    A.sort_indices()
    s = _exp_portable(rng.uniform(0.0, scale_decades, N) * (0.5 * math.log(10.0)))
    rows = np.repeat(np.arange(N), np.diff(A.indptr))
    val = A.data * s[rows]
    val = val * s[A.indices]
    return CsrProblem(N, A.indptr.astype(np.int64), A.indices.astype(np.int32), val.astype(np.float64))


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
