"""Thin ctypes binding of libsscg (include/sscg.h).

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels.  Functions keep the C names; ``Solver`` is a small convenience
wrapper that owns one handle.  Tensors must be contiguous float64 (int64/int32
for CSR indices) on the current CUDA device; numpy arrays are accepted where
the C function takes host pointers.  If the library or a CUDA device is
missing, the calls raise: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsscg.so")

SSCG_MAX_S = 16
MONOMIAL, NEWTON, CHEBYSHEV = 0, 1, 2
BASES = {"monomial": MONOMIAL, "newton": NEWTON, "chebyshev": CHEBYSHEV}
C_MODES = {"xi": 0, "xi_scaled": 1, "one": 2, "kappa_ratio": 3, "const": 4}
OK, BREAKDOWN, NOT_CONVERGED, NONFINITE = 0, 2, 3, 4


class SscgError(RuntimeError):
    pass


class Opts(C.Structure):
    _fields_ = [("s0", C.c_int), ("f", C.c_int), ("max_outer", C.c_int), ("c_mode", C.c_int),
                ("newton_scale", C.c_int), ("cheb_params", C.c_int), ("inner_conv_check", C.c_int),
                ("y_fp32", C.c_int), ("variant", C.c_int), ("check_every", C.c_int),
                ("use_graph", C.c_int), ("profile", C.c_int), ("c_const", C.c_double),
                ("eps", C.c_double), ("kappa_cut", C.c_double), ("gram_mode", C.c_int),
                ("batch_chunk_rows", C.c_int), ("batch_gram_rows", C.c_int), ("mpk_fp64_per16", C.c_int),
                ("rec_fp64_per16", C.c_int), ("ritz_exact", C.c_int),
                ("recompute_y", C.c_int)]


class OuterRecord(C.Structure):
    _fields_ = [("sbar", C.c_int), ("stilde", C.c_int), ("sk", C.c_int), ("replaced", C.c_int),
                ("c_start", C.c_double), ("c_end", C.c_double), ("phi", C.c_double),
                ("lmin", C.c_double), ("lmax", C.c_double), ("relres_est", C.c_double),
                ("kappa", C.c_double * (SSCG_MAX_S + 1))]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int), ("outer_iters", C.c_int), ("inner_iters", C.c_int),
                ("host_syncs", C.c_int), ("replacements", C.c_int), ("fp32_replacements", C.c_int),
                ("kernel_launches", C.c_int),
                ("lambda_min", C.c_double), ("lambda_max", C.c_double), ("c_last", C.c_double),
                ("true_relres", C.c_double), ("upd_relres", C.c_double),
                ("t_mpk_ms", C.c_double), ("t_gram_ms", C.c_double), ("t_kappa_ms", C.c_double),
                ("t_control_ms", C.c_double), ("t_recombine_ms", C.c_double), ("t_other_ms", C.c_double),
                ("n_gram_launches", C.c_int), ("gram_flops", C.c_double), ("mpk_spmvs", C.c_double),
                ("hist", C.POINTER(OuterRecord)), ("hist_cap", C.c_int), ("hist_len", C.c_int)]


class BatchStats(C.Structure):
    _fields_ = [("npairs", C.c_int), ("converged", C.c_int), ("outer_loops", C.c_int), ("host_syncs", C.c_int),
                ("kernel_launches", C.c_int), ("graph_launches", C.c_int), ("inner_iters", C.c_int64),
                ("max_true_relres", C.c_double), ("device_ms", C.c_double), ("pair_status", C.POINTER(C.c_int)),
                ("pair_outer", C.POINTER(C.c_int)), ("pair_inner", C.POINTER(C.c_int))]


_lib = None
_P = C.c_void_p
_I64 = C.c_int64


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load libsscg.so (built by ``paper_1908_04081_gb300.build``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise SscgError(f"{path} is missing: build it with __graft_entry__.build() "
                        "(there is no CPU fallback)")
    lib = C.CDLL(path)
    sig = {
        "sscg_version": (C.c_char_p, []),
        "sscg_strerror": (C.c_char_p, [C.c_int]),
        "sscg_last_cuda_error": (C.c_char_p, []),
        "sscg_opts_default": (None, [C.POINTER(Opts)]),
        "sscg_create_csr": (C.c_int, [C.POINTER(_P), _I64, _I64, _P, _P, _P, C.c_int, _P]),
        "sscg_create_stencil": (C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(_I64), _P, _P, _P, C.c_int, _P]),
        "sscg_destroy": (None, [_P]),
        "sscg_size": (_I64, [_P]),
        "sscg_solve": (C.c_int, [_P, _P, _P, C.c_double, C.c_int, C.c_int, C.POINTER(Opts), C.POINTER(Stats)]),
        "sscg_solve_host": (C.c_int, [_P, _P, _P, C.c_double, C.c_int, C.c_int, C.POINTER(Opts),
                                      C.POINTER(Stats)]),
        "sscg_solve_hscg": (C.c_int, [_P, _P, _P, C.c_double, C.c_int, C.POINTER(Stats)]),
        "sscg_ritz": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "sscg_spmv": (C.c_int, [_P, _P, _P]),
        "sscg_spmv_ex": (C.c_int, [_P, _P, _P, C.c_int]),
        "sscg_solve_hscg_ex": (C.c_int, [_P, _P, _P, C.c_double, C.c_int, C.c_int, C.POINTER(Stats)]),
        "sscg_build_basis": (C.c_int, [_P, _P, _P, C.c_int, _P, _P, _P, _P, _I64]),
        "sscg_wait_failures": (C.c_int, [_P, C.c_int]),
        "sscg_build_basis_ex": (C.c_int, [_P, _P, _P, C.c_int, _P, _P, _P, _P, _I64, C.c_int]),
        "sscg_gram": (C.c_int, [_P, _I64, _I64, C.c_int, _P, _P]),
        "sscg_gram_noalloc": (C.c_int, [_P, _I64, _I64, C.c_int, _P, _P]),
        "sscg_gram_ex": (C.c_int, [_P, _I64, _I64, C.c_int, _P, C.c_int, _P]),
        "sscg_kappa": (C.c_int, [_P, C.c_int, C.c_int, C.c_double, _P, _P, _P, _P]),
        "sscg_recombine": (C.c_int, [_P, C.c_int64, C.c_int64, C.c_int, _P, _P, C.c_int, _P]),
        "sscg_leja": (C.c_int, [C.c_int, _P]),
        "sscg_stencil_face_grad": (C.c_int, [_P, _P, _P, _P, _P, _P]),
        "sscg_csr_value_grad": (C.c_int, [_P, _P, _P, _P]),
        "sscg_solve_batch": (C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(C.c_int), _P, _P, C.c_double,
                                       C.POINTER(C.c_int), C.c_int, C.POINTER(Opts), C.POINTER(BatchStats), _P]),
        "sscg_autotune": (C.c_int, [_P, _P, C.c_double, C.POINTER(C.c_int), C.c_int, C.c_int, C.c_int,
                                    C.POINTER(C.c_int), C.POINTER(C.c_double)]),
        "sscg_solve_batch_hscg": (C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(C.c_int), _P, _P, C.c_double,
                                            C.c_int, C.c_int, C.POINTER(BatchStats), _P]),
        "sscg_autotune_batch": (C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(C.c_int), _P, C.c_double,
                                          C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                          C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double), _P]),
        "sscg_autotune_batch_ex": (C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(C.c_int), _P, C.c_double,
                                             C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                             C.POINTER(C.c_int), C.c_int, C.c_int, C.POINTER(C.c_int),
                                             C.POINTER(C.c_double), _P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, what: str, allow_status: bool = False) -> int:
    if rc == OK or (allow_status and rc > 0):
        return rc
    lib = load_library()
    msg = lib.sscg_strerror(rc).decode()
    if rc == -2:
        msg += ": " + lib.sscg_last_cuda_error().decode()
    raise SscgError(f"{what} failed ({rc}): {msg}")


def _dptr(t, dtype) -> int:
    """Device pointer of a contiguous CUDA tensor of the given torch dtype."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise SscgError("expected a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise SscgError(f"expected a contiguous {dtype} tensor, got {t.dtype}")
    return t.data_ptr()


def _f64(t) -> int:
    import torch
    return _dptr(t, torch.float64)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    return int(stream)


def _hptr(a: np.ndarray, dtype) -> int:
    if a.dtype != dtype or not a.flags.c_contiguous:
        raise SscgError(f"expected a C-contiguous {dtype} array")
    return a.ctypes.data


def sscg_opts_default(**kw) -> Opts:
    """Default options (sscg_opts_default), with fields overridden by keyword."""
    o = Opts()
    load_library().sscg_opts_default(C.byref(o))
    names = {name for name, _ in Opts._fields_}
    for k, v in kw.items():
        if k not in names:   # a ctypes Structure would take an unknown name as a plain attribute
            raise SscgError(f"unknown sscg_opts field {k!r}")
        if k == "c_mode" and isinstance(v, str):
            v = C_MODES[v]
        if k == "newton_scale" and isinstance(v, str):
            v = {"capacity": 0, "paper_unit": 1}[v]
        if k == "cheb_params" and isinstance(v, str):
            v = {"standard": 0, "paper_printed": 1}[v]
        if k == "variant" and isinstance(v, str):
            v = {"improved": 0, "fixed": 1, "old": 2}[v]
        if k == "gram_mode" and isinstance(v, str):
            v = {"binary64": 0, "binary32_pair": 1, "digits": 2, "digits_tcgen05": 3}[v]
        setattr(o, k, v)
    return o


def sscg_create_stencil(kx, ky, kz=None, stream=None) -> int:
    """Handle for a 2D (kz None) or 3D face-coefficient stencil; arrays are CUDA
    tensors or numpy arrays with the C-order shapes of include/sscg.h."""
    lib = load_library()
    dim = 2 if kz is None else 3
    if dim == 2:
        ny, nx1 = kx.shape
        shape = (_I64 * 3)(nx1 - 1, ny, 1)
    else:
        nz, ny, nx1 = kx.shape
        shape = (_I64 * 3)(nx1 - 1, ny, nz)
    h = _P()
    if isinstance(kx, np.ndarray):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) if a is not None else None for a in (kx, ky, kz)]
        ptrs = [a.ctypes.data if a is not None else None for a in arrs]
        on_dev = 0
    else:
        ptrs = [_f64(kx), _f64(ky), _f64(kz) if kz is not None else None]
        on_dev = 1
    _check(lib.sscg_create_stencil(C.byref(h), dim, shape, ptrs[0], ptrs[1], ptrs[2], on_dev,
                                   _stream_ptr(stream)), "sscg_create_stencil")
    return h.value


def sscg_create_csr(rowptr, col, val, stream=None) -> int:
    """Handle for a CSR matrix (int64 rowptr, int32 col, float64 val)."""
    lib = load_library()
    h = _P()
    if isinstance(rowptr, np.ndarray):
        rp = np.ascontiguousarray(rowptr, dtype=np.int64)
        cl = np.ascontiguousarray(col, dtype=np.int32)
        vl = np.ascontiguousarray(val, dtype=np.float64)
        n, nnz = rp.size - 1, cl.size
        rc = lib.sscg_create_csr(C.byref(h), n, nnz, rp.ctypes.data, cl.ctypes.data, vl.ctypes.data, 0,
                                 _stream_ptr(stream))
    else:
        import torch
        n, nnz = rowptr.numel() - 1, col.numel()
        rc = lib.sscg_create_csr(C.byref(h), n, nnz, _dptr(rowptr, torch.int64), _dptr(col, torch.int32),
                                 _f64(val), 1, _stream_ptr(stream))
    _check(rc, "sscg_create_csr")
    return h.value


def sscg_destroy(h: int) -> None:
    load_library().sscg_destroy(h)


def _stats(hist_cap: int) -> tuple[Stats, object]:
    st = Stats()
    buf = None
    if hist_cap > 0:
        buf = (OuterRecord * hist_cap)()
        st.hist = C.cast(buf, C.POINTER(OuterRecord))
        st.hist_cap = hist_cap
    return st, buf


def sscg_solve(h: int, b, x, tol: float, s_max: int, basis="chebyshev", opts: Opts | None = None,
               hist_cap: int = 0) -> Stats:
    """Algorithm 5 on device tensors b, x (x: x0 in, solution out)."""
    st, buf = _stats(hist_cap)
    rc = load_library().sscg_solve(h, _f64(b), _f64(x), tol, s_max, BASES.get(basis, basis),
                                   C.byref(opts) if opts is not None else None, C.byref(st))
    _check(rc, "sscg_solve", allow_status=True)
    st._hist_buf = buf
    return st


def sscg_solve_host(h: int, b: np.ndarray, x: np.ndarray, tol: float, s_max: int, basis="chebyshev",
                    opts: Opts | None = None, hist_cap: int = 0) -> Stats:
    """Algorithm 5 on host numpy arrays (copies inside the call)."""
    st, buf = _stats(hist_cap)
    rc = load_library().sscg_solve_host(h, _hptr(b, np.float64), _hptr(x, np.float64), tol, s_max,
                                        BASES.get(basis, basis),
                                        C.byref(opts) if opts is not None else None, C.byref(st))
    _check(rc, "sscg_solve_host", allow_status=True)
    st._hist_buf = buf
    return st


def sscg_solve_hscg(h: int, b, x, tol: float, max_iters: int = 0) -> Stats:
    """Algorithm 1 (HSCG) on device tensors."""
    st = Stats()
    rc = load_library().sscg_solve_hscg(h, _f64(b), _f64(x), tol, max_iters, C.byref(st))
    _check(rc, "sscg_solve_hscg", allow_status=True)
    return st


def sscg_solve_hscg_ex(h: int, b, x, tol: float, max_iters: int = 0, spmv_fp64_per16: int = -1) -> Stats:
    """Algorithm 1 (HSCG) with its SpMV split between FMA chains and exact integer products."""
    st = Stats()
    rc = load_library().sscg_solve_hscg_ex(h, _f64(b), _f64(x), tol, max_iters, spmv_fp64_per16, C.byref(st))
    _check(rc, "sscg_solve_hscg_ex", allow_status=True)
    return st


def sscg_ritz(h: int) -> tuple[float, float]:
    a, b = C.c_double(), C.c_double()
    _check(load_library().sscg_ritz(h, C.byref(a), C.byref(b)), "sscg_ritz")
    return a.value, b.value


def sscg_spmv(h: int, v, y) -> None:
    _check(load_library().sscg_spmv(h, _f64(v), _f64(y)), "sscg_spmv")


def sscg_spmv_ex(h: int, v, y, fp64_per16: int) -> None:
    _check(load_library().sscg_spmv_ex(h, _f64(v), _f64(y), fp64_per16), "sscg_spmv_ex")


def sscg_build_basis(h: int, p, r, s: int, theta, gamma, mu, Y, ldy: int, mpk_fp64_per16: int | None = None) -> None:
    th = np.ascontiguousarray(theta, dtype=np.float64)
    ga = np.ascontiguousarray(gamma, dtype=np.float64)
    mu_ = np.ascontiguousarray(mu, dtype=np.float64)
    if mpk_fp64_per16 is None:
        _check(load_library().sscg_build_basis(h, _f64(p), _f64(r), s, th.ctypes.data, ga.ctypes.data,
                                               mu_.ctypes.data, _f64(Y), ldy), "sscg_build_basis")
    else:
        _check(load_library().sscg_build_basis_ex(h, _f64(p), _f64(r), s, th.ctypes.data, ga.ctypes.data,
                                                  mu_.ctypes.data, _f64(Y), ldy, mpk_fp64_per16),
               "sscg_build_basis_ex")


def sscg_gram(Y, n: int, ldy: int, ncols: int, G, stream=None) -> None:
    _check(load_library().sscg_gram(_f64(Y), n, ldy, ncols, _f64(G), _stream_ptr(stream)), "sscg_gram")


def sscg_gram_ex(Y, n: int, ldy: int, ncols: int, G, mode: int, stream=None) -> None:
    """G = Y^T Y: binary64 products (mode 0), binary32-pair products (mode 1), exact
    digit products on the tensor cores by mma.sync (mode 2) or tcgen05.mma (mode 3)."""
    _check(load_library().sscg_gram_ex(_f64(Y), n, ldy, ncols, _f64(G), mode, _stream_ptr(stream)), "sscg_gram_ex")


def sscg_gram_noalloc(Y, n: int, ldy: int, ncols: int, G, stream=None) -> None:
    """G = Y^T Y with the library's fixed scratch (no device allocation)."""
    _check(load_library().sscg_gram_noalloc(_f64(Y), n, ldy, ncols, _f64(G), _stream_ptr(stream)),
           "sscg_gram_noalloc")


def sscg_wait_failures(clear: bool = True) -> int:
    """1 if a bounded in-kernel wait gave up since the last clear (see include/sscg.h)."""
    f = C.c_int(0)
    _check(load_library().sscg_wait_failures(C.byref(f), int(clear)), "sscg_wait_failures")
    return f.value


def sscg_kappa(G, ldg: int, sbar: int, kappa_cut: float, kappa, lmin, lmax, stream=None) -> None:
    _check(load_library().sscg_kappa(_f64(G), ldg, sbar, kappa_cut, _f64(kappa), _f64(lmin), _f64(lmax),
                                     _stream_ptr(stream)), "sscg_kappa")


def sscg_recombine(Y, n: int, ldy: int, ncols: int, coef, x, rec_fp64_per16: int = -1, stream=None) -> None:
    """x += Y x', Y[:, 0] = Y p', Y[:, 1] = Y r' on device buffers; coef (host) = x', r', p'."""
    c = np.ascontiguousarray(coef, dtype=np.float64).ravel()
    if c.size != 3 * ncols:
        raise ValueError("coef must hold x', r', p' (3 * ncols values)")
    _check(load_library().sscg_recombine(_f64(Y), n, ldy, ncols, c.ctypes.data, _f64(x), rec_fp64_per16,
                                         _stream_ptr(stream)), "sscg_recombine")


def sscg_leja(s: int) -> np.ndarray:
    t = np.zeros(s)
    _check(load_library().sscg_leja(s, t.ctypes.data), "sscg_leja")
    return t


def sscg_stencil_face_grad(h: int, lam, x, gkx, gky, gkz=None) -> None:
    _check(load_library().sscg_stencil_face_grad(h, _f64(lam), _f64(x), _f64(gkx), _f64(gky),
                                                 _f64(gkz) if gkz is not None else None),
           "sscg_stencil_face_grad")


def sscg_csr_value_grad(h: int, lam, x, gval) -> None:
    _check(load_library().sscg_csr_value_grad(h, _f64(lam), _f64(x), _f64(gval)), "sscg_csr_value_grad")


def sscg_solve_batch(handles, nrhs, b, x, tol: float, s_max, basis="newton", opts: Opts | None = None,
                     stream=None):
    """Batched Algorithm 5 over (system, right-hand side) pairs; b, x are the
    concatenated device vectors (system-major, right-hand-side-major).
    Returns (status, stats dict with per-pair arrays)."""
    nsys = len(handles)
    hs = (_P * nsys)(*handles)
    nr = (C.c_int * nsys)(*[int(k) for k in nrhs])
    sm = (C.c_int * nsys)(*[int(k) for k in s_max])
    npairs = int(sum(int(k) for k in nrhs))
    st = BatchStats()
    ps, po, pi = (C.c_int * max(npairs, 1))(), (C.c_int * max(npairs, 1))(), (C.c_int * max(npairs, 1))()
    st.pair_status = C.cast(ps, C.POINTER(C.c_int))
    st.pair_outer = C.cast(po, C.POINTER(C.c_int))
    st.pair_inner = C.cast(pi, C.POINTER(C.c_int))
    rc = load_library().sscg_solve_batch(hs, nsys, nr, _f64(b), _f64(x), tol, sm, BASES.get(basis, basis),
                                         C.byref(opts) if opts is not None else None, C.byref(st),
                                         _stream_ptr(stream))
    _check(rc, "sscg_solve_batch", allow_status=True)
    return rc, dict(npairs=st.npairs, converged=st.converged, outer_loops=st.outer_loops, host_syncs=st.host_syncs,
                    kernel_launches=st.kernel_launches, graph_launches=st.graph_launches,
                    inner_iters=st.inner_iters, max_true_relres=st.max_true_relres, device_ms=st.device_ms,
                    pair_status=list(ps)[:npairs], pair_outer=list(po)[:npairs], pair_inner=list(pi)[:npairs])


def sscg_solve_batch_hscg(handles, nrhs, b, x, tol: float, max_iters: int = 0, chunk_rows: int = 0, stream=None):
    """Batched plain CG (Algorithm 1) over the same pairs as sscg_solve_batch,
    in one graph launch.  Returns (status, stats dict with per-pair arrays)."""
    nsys = len(handles)
    hs = (_P * nsys)(*handles)
    nr = (C.c_int * nsys)(*[int(k) for k in nrhs])
    npairs = int(sum(int(k) for k in nrhs))
    st = BatchStats()
    ps, po, pi = (C.c_int * max(npairs, 1))(), (C.c_int * max(npairs, 1))(), (C.c_int * max(npairs, 1))()
    st.pair_status = C.cast(ps, C.POINTER(C.c_int))
    st.pair_outer = C.cast(po, C.POINTER(C.c_int))
    st.pair_inner = C.cast(pi, C.POINTER(C.c_int))
    rc = load_library().sscg_solve_batch_hscg(hs, nsys, nr, _f64(b), _f64(x), tol, int(max_iters), int(chunk_rows),
                                              C.byref(st), _stream_ptr(stream))
    _check(rc, "sscg_solve_batch_hscg", allow_status=True)
    return rc, dict(npairs=st.npairs, converged=st.converged, max_iters=st.outer_loops,
                    kernel_launches=st.kernel_launches, graph_launches=st.graph_launches,
                    inner_iters=st.inner_iters, max_true_relres=st.max_true_relres, device_ms=st.device_ms,
                    pair_status=list(ps)[:npairs], pair_iters=list(pi)[:npairs])


def sscg_autotune_batch(handles, nrhs, b, tol: float, s_max, shapes, trial_outer: int = 20, basis="newton",
                        stream=None):
    """Pick the batched solve's tile shapes among candidate (chunk_rows,
    gram_rows) pairs, or (chunk_rows, gram_rows, gram_mode) triples, by timed
    trial batches (the library's autotuner).  Returns (index of the best
    candidate, microseconds per inner iteration for each candidate)."""
    nsys = len(handles)
    hs = (_P * nsys)(*handles)
    nr = (C.c_int * nsys)(*[int(k) for k in nrhs])
    sm = (C.c_int * nsys)(*[int(k) for k in s_max])
    cr = (C.c_int * len(shapes))(*[int(c[0]) for c in shapes])
    gr = (C.c_int * len(shapes))(*[int(c[1]) for c in shapes])
    best = C.c_int()
    times = (C.c_double * len(shapes))()
    if all(len(c) == 2 for c in shapes):
        rc = load_library().sscg_autotune_batch(hs, nsys, nr, _f64(b), tol, sm, BASES.get(basis, basis), cr, gr,
                                                len(shapes), trial_outer, C.byref(best), times, _stream_ptr(stream))
    else:
        gm = (C.c_int * len(shapes))(*[int(c[2]) if len(c) > 2 else 0 for c in shapes])
        rc = load_library().sscg_autotune_batch_ex(hs, nsys, nr, _f64(b), tol, sm, BASES.get(basis, basis), cr, gr,
                                                   gm, len(shapes), trial_outer, C.byref(best), times,
                                                   _stream_ptr(stream))
    _check(rc, "sscg_autotune_batch")
    return best.value, list(times)


def sscg_autotune(h: int, b, tol: float, candidates, trial_outer: int = 12, basis="newton"):
    """Pick sigma among candidates by timed trial outer loops (the library's autotuner)."""
    cand = (C.c_int * len(candidates))(*candidates)
    best = C.c_int()
    times = (C.c_double * len(candidates))()
    _check(load_library().sscg_autotune(h, _f64(b), tol, cand, len(candidates), trial_outer,
                                        BASES.get(basis, basis), C.byref(best), times), "sscg_autotune")
    return best.value, list(times)


def history(st: Stats) -> list[dict]:
    """Per-outer-loop decision records of a solve as dicts."""
    out = []
    for k in range(st.hist_len):
        r = st.hist[k]
        out.append(dict(sbar=r.sbar, stilde=r.stilde, sk=r.sk, replaced=bool(r.replaced & 1),
                        fp32_replaced=bool(r.replaced & 2), c_start=r.c_start,
                        c=r.c_end, phi=r.phi, lmin=r.lmin, lmax=r.lmax, relres_est=r.relres_est,
                        kappa=[r.kappa[i] for i in range(r.sbar + 1)]))
    return out


class Solver:
    """One libsscg handle (a stencil or CSR operator) with Python conveniences."""

    def __init__(self, handle: int, n: int):
        self.h = handle
        self.n = n

    @classmethod
    def stencil(cls, kx, ky, kz=None, stream=None) -> "Solver":
        h = sscg_create_stencil(kx, ky, kz, stream)
        return cls(h, int(load_library().sscg_size(h)))

    @classmethod
    def csr(cls, rowptr, col, val, stream=None) -> "Solver":
        h = sscg_create_csr(rowptr, col, val, stream)
        return cls(h, int(load_library().sscg_size(h)))

    def solve(self, b, x, tol=1e-10, s_max=8, basis="chebyshev", hist_cap=0, **opts) -> Stats:
        o = sscg_opts_default(**opts) if opts else None
        return sscg_solve(self.h, b, x, tol, s_max, basis, o, hist_cap)

    def solve_host(self, b, x, tol=1e-10, s_max=8, basis="chebyshev", hist_cap=0, **opts) -> Stats:
        o = sscg_opts_default(**opts) if opts else None
        return sscg_solve_host(self.h, b, x, tol, s_max, basis, o, hist_cap)

    def hscg(self, b, x, tol=1e-10, max_iters=0, spmv_fp64_per16=None) -> Stats:
        if spmv_fp64_per16 is None:
            return sscg_solve_hscg(self.h, b, x, tol, max_iters)
        return sscg_solve_hscg_ex(self.h, b, x, tol, max_iters, spmv_fp64_per16)

    def spmv(self, v, y, fp64_per16=None) -> None:
        if fp64_per16 is None:
            sscg_spmv(self.h, v, y)
        else:
            sscg_spmv_ex(self.h, v, y, fp64_per16)

    def ritz(self) -> tuple[float, float]:
        return sscg_ritz(self.h)

    def close(self) -> None:
        if self.h:
            sscg_destroy(self.h)
            self.h = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
