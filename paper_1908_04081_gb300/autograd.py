"""Differentiable solves: x = A^{-1} b for a face-conductivity stencil or a CSR matrix.

``stencil_solve(kx, ky, kz, b)`` and ``csr_solve(rowptr, col, val, b)`` are
``torch.autograd.Function``s.  The forward pass is the adaptive s-step solve
(Algorithm 5); the backward pass is the adjoint s-step solve A lam = dL/dx
(A is symmetric) followed by the library's gradient-gather kernel:
dL/dk_f = -(lam_i - lam_j)(x_i - x_j) for a stencil's face conductivities,
dL/dA_ij = -lam_i x_j for each stored CSR entry (every stored value a free
parameter), and dL/db = lam.  Both solves and the gathers run in libsscg.
"""
from __future__ import annotations

import torch

from . import sscg

# statistics of the most recent forward and adjoint solves (for reporting)
last_stats: dict = {}


class StencilSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kx, ky, kz, b, tol=1e-10, s_max=16, basis="newton", gram_mode=0):
        solver = sscg.Solver.stencil(kx.detach().contiguous(), ky.detach().contiguous(),
                                     kz.detach().contiguous() if kz is not None else None)
        x = torch.zeros_like(b)
        st = solver.solve(b.detach().contiguous(), x, tol=tol, s_max=s_max, basis=basis, gram_mode=gram_mode)
        if st.status != sscg.OK:
            raise sscg.SscgError(f"forward solve status {st.status}")
        last_stats["forward"] = st
        ctx.solver = solver
        ctx.cfg = (tol, s_max, basis, gram_mode)
        ctx.has_kz = kz is not None
        ctx.save_for_backward(x)
        ctx.shapes = (kx.shape, ky.shape, kz.shape if kz is not None else None)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        tol, s_max, basis, gram_mode = ctx.cfg
        solver = ctx.solver
        lam = torch.zeros_like(x)
        st = solver.solve(gx.contiguous(), lam, tol=tol, s_max=s_max, basis=basis, gram_mode=gram_mode)
        if st.status != sscg.OK:
            raise sscg.SscgError(f"adjoint solve status {st.status}")
        last_stats["adjoint"] = st
        sx, sy, sz = ctx.shapes
        gkx = torch.empty(sx, dtype=x.dtype, device=x.device)
        gky = torch.empty(sy, dtype=x.dtype, device=x.device)
        gkz = torch.empty(sz, dtype=x.dtype, device=x.device) if ctx.has_kz else None
        sscg.sscg_stencil_face_grad(solver.h, lam, x, gkx, gky, gkz)
        solver.close()
        return gkx, gky, gkz, lam, None, None, None, None


def stencil_solve(kx, ky, kz, b, tol=1e-10, s_max=16, basis="newton", gram_mode=0):
    """x = A(k)^{-1} b, differentiable in kx, ky, kz and b.  gram_mode selects
    the Gram arithmetic of both solves (0: binary64 FMAs; 2: exact digit
    products on the tensor cores; see sscg_opts)."""
    return StencilSolve.apply(kx, ky, kz, b, tol, s_max, basis, gram_mode)


class CsrSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, val, b, rowptr, col, tol=1e-10, s_max=16, basis="newton", gram_mode=0):
        solver = sscg.Solver.csr(rowptr.contiguous(), col.contiguous(), val.detach().contiguous())
        x = torch.zeros_like(b)
        st = solver.solve(b.detach().contiguous(), x, tol=tol, s_max=s_max, basis=basis, gram_mode=gram_mode)
        if st.status != sscg.OK:
            raise sscg.SscgError(f"forward solve status {st.status}")
        last_stats["forward"] = st
        ctx.solver = solver
        ctx.cfg = (tol, s_max, basis, gram_mode)
        ctx.save_for_backward(x)
        ctx.nnz = val.numel()
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        tol, s_max, basis, gram_mode = ctx.cfg
        solver = ctx.solver
        lam = torch.zeros_like(x)
        st = solver.solve(gx.contiguous(), lam, tol=tol, s_max=s_max, basis=basis, gram_mode=gram_mode)
        if st.status != sscg.OK:
            raise sscg.SscgError(f"adjoint solve status {st.status}")
        last_stats["adjoint"] = st
        gval = torch.empty(ctx.nnz, dtype=x.dtype, device=x.device)
        sscg.sscg_csr_value_grad(solver.h, lam, x, gval)
        solver.close()
        return gval, lam, None, None, None, None, None, None


def csr_solve(rowptr, col, val, b, tol=1e-10, s_max=16, basis="newton", gram_mode=0):
    """x = A^{-1} b for the CSR matrix (rowptr int64, col int32, val float64;
    CUDA tensors), differentiable in val (each stored entry a free parameter,
    dL/dA_ij = -lam_i x_j) and b."""
    return CsrSolve.apply(val, b, rowptr, col, tol, s_max, basis, gram_mode)
