// Vector kernels of the solvers: recovery of x, r, p from the basis
// coordinates (Carson 2019, eq. (coords), Algorithm 5), the initial and true
// residuals with their norms, residual replacement, and the Hestenes-Stiefel
// CG comparator (Algorithm 1).
//
// Reductions are deterministic: every block writes one partial, and the last
// block to arrive (atomic ticket) adds the partials in a fixed order.  Each
// thread first accumulates many rows so the FP64 adds of the reduction tree
// stay a small fraction of the FP64 work.
#include <math.h>

#include "exact_sum.cuh"
#include "sscg_internal.cuh"

namespace sscg {

namespace {

constexpr int kVecThreads = 256;

int vec_grid(int64_t n) {
  int64_t g = (n + (int64_t)kVecThreads * 8 - 1) / ((int64_t)kVecThreads * 8);
  if (g < 1) g = 1;
  if (g > 152 * 4) g = 152 * 4;
  return (int)g;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum to thread 0 (fixed order).
__device__ double block_sum(double v) {
  __shared__ double ws[kVecThreads / 32];
  v = warp_sum(v);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) ws[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kVecThreads / 32; ++i) s += ws[i];
  __syncthreads();
  return s;
}

// Write the block's partial; returns true (in every thread of the block) if
// this block is the last one and `*total` holds the fixed-order sum of all
// partials (valid in thread 0 only).
__device__ bool last_block_sum(double partial, double* partials, unsigned int* counter, double* total) {
  __shared__ bool is_last;
  const double bs = block_sum(partial);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = bs;
    __threadfence();
    const unsigned int ticket = atomicAdd(counter, 1u);
    is_last = ticket == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double s = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kVecThreads) s += __ldcg(partials + b);
  s = block_sum(s);
  if (threadIdx.x == 0) {
    *total = s;
    *counter = 0u;
  }
  return true;
}

// ------------------------------------------------------------- recovery
// x += Y x', r = Y r', p = Y p' over the first nc = 2 s_k + 1 columns.  With a
// binary64 basis the new p and r overwrite columns 0 and 1 of Y (each row
// reads its own row first); with a binary32 basis they go to the binary64
// vectors p64, r64 and their roundings to columns 0 and 1.
template <typename T>
__global__ void __launch_bounds__(kVecThreads) recombine_kernel(const SolveState* __restrict__ st,
                                                                T* __restrict__ Y, int64_t ld,
                                                                double* __restrict__ x, double* __restrict__ r64,
                                                                double* __restrict__ p64, int64_t n) {
  if (st->done) return;
  const int nc = st->nc;
  __shared__ double cx[kMaxCols], cr[kMaxCols], cp[kMaxCols];
  if (threadIdx.x < kMaxCols) {
    cx[threadIdx.x] = st->xc[threadIdx.x];
    cr[threadIdx.x] = st->rc[threadIdx.x];
    cp[threadIdx.x] = st->pc[threadIdx.x];
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double sx = 0.0, sr = 0.0, sp = 0.0;
    for (int c = 0; c < nc; ++c) {
      const double y = widen(Y[(int64_t)c * ld + i]);
      sx = fma(y, cx[c], sx);
      sr = fma(y, cr[c], sr);
      sp = fma(y, cp[c], sp);
    }
    x[i] += sx;
    if (r64 != nullptr) {
      r64[i] = sr;
      p64[i] = sp;
    }
    Y[i] = (T)sp;
    Y[ld + i] = (T)sr;
  }
}

// One row of the recovery as binary64 FMA chains (the order of
// recombine_kernel).  Out of line: the integer path calls it only for rows
// with Inf/NaN operands or a sum outside the normal range.
__device__ __noinline__ void recombine_row_fma(const double* __restrict__ Y, int64_t ld, int nc,
                                               const double* cx, const double* cr, const double* cp,
                                               int64_t i, double& sx, double& sr, double& sp) {
  sx = 0.0;
  sr = 0.0;
  sp = 0.0;
  for (int c = 0; c < nc; ++c) {
    const double y = Y[(int64_t)c * ld + i];
    sx = fma(y, cx[c], sx);
    sr = fma(y, cr[c], sr);
    sp = fma(y, cp[c], sp);
  }
}

// The recovery with a binary64 basis, its binary64 work split between two
// units (as the stencil matrix-powers level): rows go in groups of 32 (one
// warp), and of every 16 groups `fp64_per16` are summed as the binary64 FMA
// chains of recombine_kernel, the others as exact integer dot products
// (exact_sum.cuh): each of x + Y x', Y r', Y p' is a streamed sum of at most
// 34 products (x itself enters as x * 1), aligned online, rounded once.  The
// coefficients are the same for every row, so their limbs are formed once
// per block; each y is split once and feeds three sums.  A row's form
// depends only on its position, so results are reproducible.
constexpr int kRecHead = 6;   // headroom bits: up to 64 terms
static_assert(kMaxCols + 1 <= (1 << kRecHead), "recovery terms within the integer sum's headroom");

// Coefficients x', r', p' of a state into shared memory (values and limbs),
// by threads 0..kMaxCols-1; returns nonzero in every thread of the block when
// a coefficient is Inf/NaN (the block then takes the FMA chains).  Ends with
// a block barrier.
__device__ __forceinline__ int rec_load_coef(const SolveState* __restrict__ st, int nc, double* cx, double* cr,
                                             double* cp, int4 (*cl)[3]) {
  unsigned bad = 0;
  if (threadIdx.x < kMaxCols) {
    const int c = threadIdx.x;
    cx[c] = st->xc[c];
    cr[c] = st->rc[c];
    cp[c] = st->pc[c];
    if (c < nc) {
      const Limbs lx = to_limbs(cx[c], bad), lr = to_limbs(cr[c], bad), lp = to_limbs(cp[c], bad);
      cl[c][0] = make_int4(lx.a, lx.b, lx.e, 0);
      cl[c][1] = make_int4(lr.a, lr.b, lr.e, 0);
      cl[c][2] = make_int4(lp.a, lp.b, lp.e, 0);
    }
  }
  return __syncthreads_or((int)bad);
}

// Row i of the recovery: on the FMA chains when `fma_row`, else as exact
// integer dot products (falling back to the chains for non-finite operands or
// sums outside the normal range).  sx includes x_i.
__device__ __forceinline__ void rec_row(const double* __restrict__ Y, int64_t ld, int nc, const double* cx,
                                        const double* cr, const double* cp, const int4 (*cl)[3], int64_t i,
                                        double xi, bool fma_row, double& sx, double& sr, double& sp) {
  if (fma_row) {
    sx = 0.0;
    sr = 0.0;
    sp = 0.0;
    for (int c = 0; c < nc; ++c) {
      const double y = Y[(int64_t)c * ld + i];
      sx = fma(y, cx[c], sx);
      sr = fma(y, cr[c], sr);
      sp = fma(y, cp[c], sp);
    }
    sx += xi;
    return;
  }
  unsigned ybad = 0;
  OnlineSum<kRecHead> ax, ar, ap;
  ax.add(Limbs{1 << 30, 0, 1023}, to_limbs(xi, ybad));   // x * 1.0
#pragma unroll 2
  for (int c = 0; c < nc; ++c) {
    const Limbs ly = to_limbs(Y[(int64_t)c * ld + i], ybad);
    const int4 lx = cl[c][0], lr = cl[c][1], lp = cl[c][2];
    ax.add(Limbs{lx.x, lx.y, lx.z}, ly);
    ar.add(Limbs{lr.x, lr.y, lr.z}, ly);
    ap.add(Limbs{lp.x, lp.y, lp.z}, ly);
  }
  bool ok = true;
  sx = ax.result(ok);
  sr = ar.result(ok);
  sp = ap.result(ok);
  if (!ok || ybad) {
    recombine_row_fma(Y, ld, nc, cx, cr, cp, i, sx, sr, sp);
    sx += xi;
  }
}

__global__ void __launch_bounds__(kVecThreads, 4) recombine_hybrid_kernel(const SolveState* __restrict__ st,
                                                                          double* __restrict__ Y, int64_t ld,
                                                                          double* __restrict__ x, int64_t n,
                                                                          int fp64_per16) {
  if (st->done) return;
  const int nc = st->nc;
  __shared__ double cx[kMaxCols], cr[kMaxCols], cp[kMaxCols];
  __shared__ int4 cl[kMaxCols][3];   // limbs (a, b, e) of the x', r', p' coefficients
  const int coef_bad = rec_load_coef(st, nc, cx, cr, cp, cl);
  const unsigned f16 = (unsigned)fp64_per16;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned g = (unsigned)(i >> 5);   // the row group: the same for the 32 lanes of a warp
    double sx, sr, sp;
    rec_row(Y, ld, nc, cx, cr, cp, cl, i, x[i], coef_bad || ((g * f16) & 15u) < f16, sx, sr, sp);
    x[i] = sx;
    Y[i] = sp;
    Y[ld + i] = sr;
  }
}

// After r0 = b - A x0 has been formed: p0 = r0 into the basis columns (and
// the binary64 vectors of a binary32 basis), and ||b||.
template <typename T>
__global__ void __launch_bounds__(kVecThreads) init_norms_kernel(SolveState* __restrict__ st,
                                                                 const double* __restrict__ b,
                                                                 const double* __restrict__ r0,
                                                                 T* __restrict__ Y, int64_t ld,
                                                                 double* __restrict__ p64, int64_t n,
                                                                 double* __restrict__ partials) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i];
    s = fma(bi, bi, s);
    const double ri = r0[i];
    if (p64 != nullptr) p64[i] = ri;
    Y[i] = (T)ri;
    Y[ld + i] = (T)ri;
  }
  double tot;
  if (last_block_sum(s, partials, &st->red_counter, &tot) && threadIdx.x == 0) {
    st->normb = sqrt(tot);
    if (tot == 0.0) {  // b = 0: the solution is x = 0
      st->zero_rhs = 1;
      st->done = 1;
      st->status = SSCG_OK;
    } else if (!isfinite(tot)) {
      st->done = 1;
      st->status = SSCG_NONFINITE;
    }
  }
}

__global__ void __launch_bounds__(kVecThreads) zero_x_kernel(const SolveState* __restrict__ st, double* __restrict__ x,
                                                             int64_t n) {
  if (!st->zero_rhs) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = 0.0;
}

// True residual check after a converged coordinate estimate (reading C16).
__global__ void __launch_bounds__(kVecThreads) true_norm_kernel(SolveState* __restrict__ st,
                                                                const double* __restrict__ rt, int64_t n,
                                                                double* __restrict__ partials, int force) {
  if (!force && (st->done || !st->converged_est)) return;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = rt[i];
    s = fma(v, v, s);
  }
  double tot;
  if (last_block_sum(s, partials, &st->red_counter, &tot) && threadIdx.x == 0) {
    st->rt2 = tot;
    if (!force) {
      const double rel = sqrt(tot) / st->normb;
      if (!isfinite(rel)) {
        st->done = 1;
        st->status = SSCG_NONFINITE;
      } else if (rel <= st->tol) {
        st->done = 1;
        st->status = SSCG_OK;
      } else if (st->prev_fail > 0.0 && rel >= 0.5 * st->prev_fail) {
        st->done = 1;  // stagnation above tol: the attainable accuracy is reached
        st->status = SSCG_NOT_CONVERGED;
      } else {
        st->prev_fail = rel;
        st->replace_pending = 1;
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kVecThreads) replacement_kernel(const SolveState* __restrict__ st,
                                                                  const double* __restrict__ rt,
                                                                  T* __restrict__ Y, int64_t ld,
                                                                  double* __restrict__ r64, double* __restrict__ p64,
                                                                  int64_t n) {
  if (st->done || !st->replace_pending) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = rt[i];
    if (r64 != nullptr) {
      r64[i] = v;
      p64[i] = v;
    }
    Y[i] = (T)v;
    Y[ld + i] = (T)v;
  }
}

// FP32-stored basis: r := b - A x (already in r64) rounded into column 1, and
// the relative residual at this replacement; p is kept.
__global__ void __launch_bounds__(kVecThreads) fp32_replace_kernel(SolveState* __restrict__ st,
                                                                   const double* __restrict__ r64,
                                                                   float* __restrict__ Y, int64_t ld, int64_t n,
                                                                   double* __restrict__ partials,
                                                                   sscg_outer_record* __restrict__ hist) {
  if (st->done || !st->fp32_replace_pending) return;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = r64[i];
    Y[ld + i] = (float)v;
    s = fma(v, v, s);
  }
  double tot;
  if (last_block_sum(s, partials, &st->red_counter, &tot) && threadIdx.x == 0) {
    st->rho_last = sqrt(tot) / st->normb;
    st->fp32_replace_pending = 0;
    st->fp32_replacements += 1;
    const int k = st->k - 1;
    if (hist != nullptr && k >= 0 && k < st->hist_cap) hist[k].replaced |= 2;
  }
}

// Bookkeeping at the end of one outer loop: finish a replacement, enforce the
// outer-loop cap.
__global__ void end_of_loop_kernel(SolveState* st, sscg_outer_record* hist) {
  if (threadIdx.x != 0 || st->done) return;
  if (st->replace_pending) {
    st->replace_pending = 0;
    st->converged_est = 0;
    st->psi = 1.0;
    st->replacements += 1;
    const int k = st->k - 1;
    if (hist != nullptr && k >= 0 && k < st->hist_cap) hist[k].replaced |= 1;
  }
  if (st->k >= st->max_outer) {
    st->status = SSCG_NOT_CONVERGED;
    st->done = 1;
  }
}

// ------------------------------------------------------------------ HSCG
// Algorithm 1 with the updated-residual test ||r||/||b|| <= tol, confirmed by
// the true residual (readings C16, C20).  One iteration:
//   K1: q = A p, alpha = (r, r) / (p, q)          (reduction)
//   K2: x += alpha p, r -= alpha q, beta = (r+, r+)/(r, r)   (reduction)
//   K3: p = r + beta p
__global__ void __launch_bounds__(kVecThreads) hscg_pq_kernel(SolveState* __restrict__ st, const double* __restrict__ p,
                                                              const double* __restrict__ q, int64_t n,
                                                              double* __restrict__ partials) {
  if (st->done || st->converged_est) return;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(p[i], q[i], s);
  double tot;
  if (last_block_sum(s, partials, &st->red_counter, &tot) && threadIdx.x == 0) {
    st->h_pq = tot;
    st->h_alpha = st->h_rr / tot;
  }
}

__global__ void __launch_bounds__(kVecThreads) hscg_update_kernel(SolveState* __restrict__ st, double* __restrict__ x,
                                                                  double* __restrict__ r, const double* __restrict__ p,
                                                                  const double* __restrict__ q, int64_t n,
                                                                  double* __restrict__ partials) {
  if (st->done || st->converged_est) return;
  const double alpha = st->h_alpha;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    s = fma(ri, ri, s);
  }
  double tot;
  if (last_block_sum(s, partials, &st->red_counter, &tot) && threadIdx.x == 0) {
    st->h_beta = tot / st->h_rr;
    st->h_rr = tot;
    st->h_iters += 1;
    st->m = st->h_iters;
    if (sqrt(tot) / st->normb <= st->tol) st->converged_est = 1;
    if (st->h_iters >= st->h_max_iters && !st->converged_est) {
      st->status = SSCG_NOT_CONVERGED;
      st->done = 1;
    }
  }
}

__global__ void __launch_bounds__(kVecThreads) hscg_pupdate_kernel(const SolveState* __restrict__ st,
                                                                   const double* __restrict__ r, double* __restrict__ p,
                                                                   int64_t n) {
  if (st->done || st->converged_est) return;
  const double beta = st->h_beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], r[i]);
}

__global__ void __launch_bounds__(kVecThreads) hscg_init_kernel(SolveState* __restrict__ st,
                                                                const double* __restrict__ b,
                                                                const double* __restrict__ r, double* __restrict__ p,
                                                                int64_t n, double* __restrict__ partials,
                                                                double* __restrict__ partials2) {
  double sb = 0.0, sr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = r[i];
    p[i] = ri;
    sr = fma(ri, ri, sr);
    sb = fma(b[i], b[i], sb);
  }
  // two fixed-order sums: ||b||^2 into partials, ||r||^2 into partials2
  const double bsb = block_sum(sb);
  const double bsr = block_sum(sr);
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = bsb;
    partials2[blockIdx.x] = bsr;
    __threadfence();
    is_last = atomicAdd(&st->red_counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double a = 0.0, c = 0.0;
  for (int bi = threadIdx.x; bi < (int)gridDim.x; bi += kVecThreads) {
    a += __ldcg(partials + bi);
    c += __ldcg(partials2 + bi);
  }
  a = block_sum(a);
  c = block_sum(c);
  if (threadIdx.x == 0) {
    st->normb = sqrt(a);
    st->h_rr = c;
    st->red_counter = 0u;
    if (a == 0.0) {
      st->zero_rhs = 1;
      st->done = 1;
      st->status = SSCG_OK;
    } else if (!isfinite(a) || !isfinite(c)) {
      st->done = 1;
      st->status = SSCG_NONFINITE;
    } else if (sqrt(c) / st->normb <= st->tol) {
      st->converged_est = 1;
    }
  }
}

// HSCG true-residual confirmation: if converged_est, rt = b - A x was formed
// by the caller's residual launch; decide done or replace (r = p = rt).
__global__ void __launch_bounds__(kVecThreads) hscg_confirm_kernel(SolveState* __restrict__ st,
                                                                   const double* __restrict__ rt,
                                                                   double* __restrict__ r, double* __restrict__ p,
                                                                   int64_t n, double* __restrict__ partials) {
  if (st->done || !st->converged_est) return;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = rt[i];
    s = fma(v, v, s);
  }
  double tot;
  if (last_block_sum(s, partials, &st->red_counter, &tot) && threadIdx.x == 0) {
    st->rt2 = tot;
    const double rel = sqrt(tot) / st->normb;
    if (!isfinite(rel)) {
      st->done = 1;
      st->status = SSCG_NONFINITE;
    } else if (rel <= st->tol) {
      st->done = 1;
      st->status = SSCG_OK;
    } else if (st->prev_fail > 0.0 && rel >= 0.5 * st->prev_fail) {
      st->done = 1;  // stagnation above tol
      st->status = SSCG_NOT_CONVERGED;
    } else {
      st->prev_fail = rel;
      st->replace_pending = 1;
    }
  }
}

__global__ void __launch_bounds__(kVecThreads) hscg_replace_kernel(SolveState* __restrict__ st,
                                                                   const double* __restrict__ rt,
                                                                   double* __restrict__ r, double* __restrict__ p,
                                                                   int64_t n) {
  if (st->done || !st->replace_pending) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    r[i] = rt[i];
    p[i] = rt[i];
  }
}

__global__ void hscg_replace_finish_kernel(SolveState* st) {
  if (st->done || !st->replace_pending) return;
  st->replace_pending = 0;
  st->converged_est = 0;
  st->h_rr = st->rt2;
  st->replacements += 1;
}


// ------------------------------------------------------------------ batches
// (A v)_i for row i of a pair's operator (stencil or CSR); v is pair-local.
__device__ __forceinline__ double batch_apply(const Operator& A, const double* __restrict__ v, int64_t i) {
  if (A.kind == 1) {
    const int nx = A.nx, ny = A.ny, nz = A.nz;
    const int x = (int)(i % nx);
    const int64_t t = i / nx;
    const int y = (int)(t % ny);
    const int z = (int)(t / ny);
    const int64_t plane = (int64_t)nx * ny;
    const int64_t fx = ((int64_t)z * ny + y) * (nx + 1) + x;
    const int64_t fy = ((int64_t)z * (ny + 1) + y) * nx + x;
    double acc = A.diag[i] * v[i];
    acc = fma(-A.kx[fx], x > 0 ? v[i - 1] : 0.0, acc);
    acc = fma(-A.kx[fx + 1], x < nx - 1 ? v[i + 1] : 0.0, acc);
    acc = fma(-A.ky[fy], y > 0 ? v[i - nx] : 0.0, acc);
    acc = fma(-A.ky[fy + nx], y < ny - 1 ? v[i + nx] : 0.0, acc);
    if (A.dim == 3) {
      acc = fma(-A.kz[i], z > 0 ? v[i - plane] : 0.0, acc);
      acc = fma(-A.kz[i + plane], z < nz - 1 ? v[i + plane] : 0.0, acc);
    }
    return acc;
  }
  double acc = 0.0;
  for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) acc = fma(A.val[k], v[A.col[k]], acc);
  return acc;
}

// Per-pair fixed-order sum of chunk partials: the last chunk of pair j to
// arrive (ticket on the pair's counter) adds them; returns true there.
__device__ bool pair_last_sum(double partial, const BatchPair& bp, SolveState* st, double* partials, int c,
                              double* total) {
  __shared__ bool is_last;
  const double bs = block_sum(partial);
  if (threadIdx.x == 0) {
    partials[c] = bs;
    __threadfence();
    is_last = atomicAdd(&st->red_counter, 1u) == (unsigned)bp.nchunk - 1;
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double s = 0.0;
  for (int b = threadIdx.x; b < bp.nchunk; b += kVecThreads) s += __ldcg(partials + bp.chunk0 + b);
  s = block_sum(s);
  if (threadIdx.x == 0) {
    *total = s;
    st->red_counter = 0u;
  }
  return true;
}

// r0 = b - A x0 into basis columns 0 and 1 of every pair, and ||b|| per pair.
__global__ void __launch_bounds__(kVecThreads) batch_init_kernel(BatchView v, const double* __restrict__ b,
                                                                 const double* __restrict__ x, double* __restrict__ Y,
                                                                 int64_t LD, double* __restrict__ partials) {
  for (int c = blockIdx.x; c < v.nchunks; c += gridDim.x) {
    const int j = v.chunk_pair[c];
    const BatchPair& bp = v.pairs[j];
    SolveState* st = v.states + j;
    const int64_t r0 = (int64_t)(c - bp.chunk0) * v.chunk_rows;
    int64_t r1 = r0 + v.chunk_rows;
    if (r1 > bp.n) r1 = bp.n;
    const double* xb = x + bp.off;
    double s = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const double bi = b[bp.off + i];
      const double r = bi - batch_apply(bp.op, xb, i);
      Y[bp.off + i] = r;
      Y[LD + bp.off + i] = r;
      s = fma(bi, bi, s);
    }
    double tot;
    if (pair_last_sum(s, bp, st, partials, c, &tot) && threadIdx.x == 0) {
      st->normb = sqrt(tot);
      if (tot == 0.0) {
        st->zero_rhs = 1;
        st->done = 1;
        st->status = SSCG_OK;
      } else if (!isfinite(tot)) {
        st->done = 1;
        st->status = SSCG_NONFINITE;
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kVecThreads) batch_zero_x_kernel(BatchView v, double* __restrict__ x) {
  for (int c = blockIdx.x; c < v.nchunks; c += gridDim.x) {
    const int j = v.chunk_pair[c];
    const BatchPair& bp = v.pairs[j];
    if (!v.states[j].zero_rhs) continue;
    const int64_t r0 = (int64_t)(c - bp.chunk0) * v.chunk_rows;
    int64_t r1 = r0 + v.chunk_rows;
    if (r1 > bp.n) r1 = bp.n;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) x[bp.off + i] = 0.0;
  }
}

// The batched recovery: each chunk's rows with the coefficients of its pair,
// split between the FMA chains and exact integer dot products as
// recombine_hybrid_kernel (row groups of 32 rows counted from the pair's
// first row; fp64_per16 = 16: FMA chains only).
__global__ void __launch_bounds__(kVecThreads) batch_recombine_kernel(BatchView v, double* __restrict__ Y, int64_t LD,
                                                                      double* __restrict__ x, int fp64_per16) {
  __shared__ double cx[kMaxCols], cr[kMaxCols], cp[kMaxCols];
  __shared__ int4 cl[kMaxCols][3];
  const unsigned f16 = (unsigned)fp64_per16;
  for (int c = blockIdx.x; c < v.nchunks; c += gridDim.x) {
    const int j = v.chunk_pair[c];
    const BatchPair& bp = v.pairs[j];
    const SolveState* st = v.states + j;
    if (st->done) continue;
    const int nc = st->nc;
    __syncthreads();
    const int coef_bad = rec_load_coef(st, nc, cx, cr, cp, cl);
    const int64_t r0 = (int64_t)(c - bp.chunk0) * v.chunk_rows;
    int64_t r1 = r0 + v.chunk_rows;
    if (r1 > bp.n) r1 = bp.n;
    double* Yp = Y + bp.off;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const unsigned g = (unsigned)(i >> 5);
      double sx, sr, sp;
      rec_row(Yp, LD, nc, cx, cr, cp, cl, i, x[bp.off + i], f16 >= 16u || coef_bad || ((g * f16) & 15u) < f16, sx,
              sr, sp);
      x[bp.off + i] = sx;
      Yp[i] = sp;
      Yp[LD + i] = sr;
    }
  }
}

// True-residual confirmation of the pairs whose estimate reached tol (C16).
__global__ void __launch_bounds__(kVecThreads) batch_true_residual_kernel(BatchView v, const double* __restrict__ b,
                                                                          const double* __restrict__ x,
                                                                          double* __restrict__ rt,
                                                                          double* __restrict__ partials) {
  for (int c = blockIdx.x; c < v.nchunks; c += gridDim.x) {
    const int j = v.chunk_pair[c];
    const BatchPair& bp = v.pairs[j];
    SolveState* st = v.states + j;
    if (st->done || !st->converged_est) continue;
    const int64_t r0 = (int64_t)(c - bp.chunk0) * v.chunk_rows;
    int64_t r1 = r0 + v.chunk_rows;
    if (r1 > bp.n) r1 = bp.n;
    const double* xb = x + bp.off;
    double s = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const double r = b[bp.off + i] - batch_apply(bp.op, xb, i);
      rt[bp.off + i] = r;
      s = fma(r, r, s);
    }
    double tot;
    if (pair_last_sum(s, bp, st, partials, c, &tot) && threadIdx.x == 0) {
      st->rt2 = tot;
      const double rel = sqrt(tot) / st->normb;
      if (!isfinite(rel)) {
        st->done = 1;
        st->status = SSCG_NONFINITE;
      } else if (rel <= st->tol) {
        st->done = 1;
        st->status = SSCG_OK;
      } else if (st->prev_fail > 0.0 && rel >= 0.5 * st->prev_fail) {
        st->done = 1;
        st->status = SSCG_NOT_CONVERGED;
      } else {
        st->prev_fail = rel;
        st->replace_pending = 1;
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kVecThreads) batch_replacement_kernel(BatchView v, const double* __restrict__ rt,
                                                                        double* __restrict__ Y, int64_t LD) {
  for (int c = blockIdx.x; c < v.nchunks; c += gridDim.x) {
    const int j = v.chunk_pair[c];
    const BatchPair& bp = v.pairs[j];
    const SolveState* st = v.states + j;
    if (st->done || !st->replace_pending) continue;
    const int64_t r0 = (int64_t)(c - bp.chunk0) * v.chunk_rows;
    int64_t r1 = r0 + v.chunk_rows;
    if (r1 > bp.n) r1 = bp.n;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const double r = rt[bp.off + i];
      Y[bp.off + i] = r;
      Y[LD + bp.off + i] = r;
    }
  }
}

// End of one outer loop for every pair; counts the pairs still running.
__global__ void batch_end_kernel(BatchView v) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < v.npairs; j += gridDim.x * blockDim.x) {
    SolveState* st = v.states + j;
    if (st->done) continue;
    if (st->replace_pending) {
      st->replace_pending = 0;
      st->converged_est = 0;
      st->psi = 1.0;
      st->replacements += 1;
      const int k = st->k - 1;
      if (v.hist != nullptr && k >= 0 && k < v.hist_cap) v.hist[(int64_t)j * v.hist_cap + k].replaced |= 1;
    }
    if (st->k >= st->max_outer) {
      st->status = SSCG_NOT_CONVERGED;
      st->done = 1;
      continue;
    }
    atomicAdd(v.active, 1u);
  }
}

__global__ void batch_begin_kernel(BatchView v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *v.active = 0u;
    *v.bodies += 1u;
  }
}

// Loop condition of the batched graph: continue while a pair is running and
// the outer-loop budget is not spent.
__global__ void batch_cond_kernel(BatchView v, cudaGraphConditionalHandle cond) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    cudaGraphSetConditional(cond, (*v.active > 0u && *v.bodies < (unsigned)v.max_bodies) ? 1u : 0u);
}

// Loop condition of a single solve's graph: repeat the outer loop until the
// device has set done (convergence, breakdown, stagnation or the outer-loop cap).
// The configuration of a solve, passed by value: the host writes no device
// memory it would have to wait for before the solve's first kernel.
__global__ void set_state_kernel(SolveState* __restrict__ dst, const SolveState src) {
  const int nw = (int)(sizeof(SolveState) / sizeof(unsigned int));
  const unsigned int* s = reinterpret_cast<const unsigned int*>(&src);
  unsigned int* d = reinterpret_cast<unsigned int*>(dst);
  for (int i = threadIdx.x; i < nw; i += blockDim.x) d[i] = s[i];
}

__global__ void solve_cond_kernel(const SolveState* st, cudaGraphConditionalHandle cond) {
  if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(cond, st->done ? 0u : 1u);
}

__global__ void batch_arm_kernel(cudaGraphConditionalHandle cond) {
  if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(cond, 1u);
}

// ------------------------------------------------------------ batched HSCG
// Algorithm 1 for every pair in lock-step, the comparator of the batched
// s-step solve: per iteration q = A p with (p, q), then x, r and (r, r), then
// p; every pair keeps its own alpha, beta and test (reading C16 confirmation
// with the true residual at the end of each graph body).
__global__ void __launch_bounds__(kVecThreads) batch_hscg_init_kernel(BatchView v, const double* __restrict__ b,
                                                                      const double* __restrict__ x,
                                                                      double* __restrict__ r, double* __restrict__ p,
                                                                      double* __restrict__ partials) {
  // pass 1 of 2: r = p = b - A x and ||b||^2
  for (int c = blockIdx.x; c < v.nchunks; c += gridDim.x) {
    const int j = v.chunk_pair[c];
    const BatchPair& bp = v.pairs[j];
    SolveState* st = v.states + j;
    const int64_t r0 = (int64_t)(c - bp.chunk0) * v.chunk_rows;
    int64_t r1 = r0 + v.chunk_rows;
    if (r1 > bp.n) r1 = bp.n;
    const double* xb = x + bp.off;
    double s = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const double bi = b[bp.off + i];
      const double ri = bi - batch_apply(bp.op, xb, i);
      r[bp.off + i] = ri;
      p[bp.off + i] = ri;
      s = fma(bi, bi, s);
    }
    double tot;
    if (pair_last_sum(s, bp, st, partials, c, &tot) && threadIdx.x == 0) {
      st->normb = sqrt(tot);
      if (tot == 0.0) {
        st->zero_rhs = 1;
        st->done = 1;
        st->status = SSCG_OK;
      } else if (!isfinite(tot)) {
        st->done = 1;
        st->status = SSCG_NONFINITE;
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kVecThreads) batch_hscg_rr_kernel(BatchView v, const double* __restrict__ r,
                                                                    double* __restrict__ partials) {
  // pass 2 of 2: ||r0||^2 and the initial test
  for (int c = blockIdx.x; c < v.nchunks; c += gridDim.x) {
    const int j = v.chunk_pair[c];
    const BatchPair& bp = v.pairs[j];
    SolveState* st = v.states + j;
    if (st->done) continue;
    const int64_t r0 = (int64_t)(c - bp.chunk0) * v.chunk_rows;
    int64_t r1 = r0 + v.chunk_rows;
    if (r1 > bp.n) r1 = bp.n;
    double s = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) s = fma(r[bp.off + i], r[bp.off + i], s);
    double tot;
    if (pair_last_sum(s, bp, st, partials, c, &tot) && threadIdx.x == 0) {
      st->h_rr = tot;
      if (!isfinite(tot)) {
        st->done = 1;
        st->status = SSCG_NONFINITE;
      } else if (sqrt(tot) / st->normb <= st->tol) {
        st->converged_est = 1;
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ bool hscg_running(const SolveState* st) { return !st->done && !st->converged_est; }

__global__ void __launch_bounds__(kVecThreads) batch_hscg_q_kernel(BatchView v, const double* __restrict__ p,
                                                                   double* __restrict__ q,
                                                                   double* __restrict__ partials) {
  for (int c = blockIdx.x; c < v.nchunks; c += gridDim.x) {
    const int j = v.chunk_pair[c];
    const BatchPair& bp = v.pairs[j];
    SolveState* st = v.states + j;
    if (!hscg_running(st)) continue;
    const int64_t r0 = (int64_t)(c - bp.chunk0) * v.chunk_rows;
    int64_t r1 = r0 + v.chunk_rows;
    if (r1 > bp.n) r1 = bp.n;
    const double* pb = p + bp.off;
    double s = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const double qi = batch_apply(bp.op, pb, i);
      q[bp.off + i] = qi;
      s = fma(pb[i], qi, s);
    }
    double tot;
    if (pair_last_sum(s, bp, st, partials, c, &tot) && threadIdx.x == 0) {
      st->h_pq = tot;
      st->h_alpha = st->h_rr / tot;
      if (!(tot > 0.0) || !isfinite(st->h_alpha)) {
        st->done = 1;
        st->status = SSCG_BREAKDOWN;
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kVecThreads) batch_hscg_update_kernel(BatchView v, double* __restrict__ x,
                                                                        double* __restrict__ r,
                                                                        const double* __restrict__ p,
                                                                        const double* __restrict__ q,
                                                                        double* __restrict__ partials) {
  for (int c = blockIdx.x; c < v.nchunks; c += gridDim.x) {
    const int j = v.chunk_pair[c];
    const BatchPair& bp = v.pairs[j];
    SolveState* st = v.states + j;
    if (!hscg_running(st)) continue;
    const double alpha = st->h_alpha;
    const int64_t r0 = (int64_t)(c - bp.chunk0) * v.chunk_rows;
    int64_t r1 = r0 + v.chunk_rows;
    if (r1 > bp.n) r1 = bp.n;
    double s = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const int64_t k = bp.off + i;
      x[k] = fma(alpha, p[k], x[k]);
      const double ri = fma(-alpha, q[k], r[k]);
      r[k] = ri;
      s = fma(ri, ri, s);
    }
    double tot;
    if (pair_last_sum(s, bp, st, partials, c, &tot) && threadIdx.x == 0) {
      st->h_beta = tot / st->h_rr;
      st->h_rr = tot;
      st->h_iters += 1;
      st->m = st->h_iters;
      if (sqrt(tot) / st->normb <= st->tol) st->converged_est = 1;
      if (st->h_iters >= st->h_max_iters && !st->converged_est) {
        st->status = SSCG_NOT_CONVERGED;
        st->done = 1;
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kVecThreads) batch_hscg_p_kernel(BatchView v, const double* __restrict__ r,
                                                                   double* __restrict__ p) {
  for (int c = blockIdx.x; c < v.nchunks; c += gridDim.x) {
    const int j = v.chunk_pair[c];
    const BatchPair& bp = v.pairs[j];
    const SolveState* st = v.states + j;
    if (!hscg_running(st)) continue;
    const double beta = st->h_beta;
    const int64_t r0 = (int64_t)(c - bp.chunk0) * v.chunk_rows;
    int64_t r1 = r0 + v.chunk_rows;
    if (r1 > bp.n) r1 = bp.n;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const int64_t k = bp.off + i;
      p[k] = fma(beta, p[k], r[k]);
    }
  }
}

// r := p := b - A x for the pairs whose confirmation failed (C16)
__global__ void __launch_bounds__(kVecThreads) batch_hscg_replace_kernel(BatchView v, const double* __restrict__ rt,
                                                                         double* __restrict__ r,
                                                                         double* __restrict__ p) {
  for (int c = blockIdx.x; c < v.nchunks; c += gridDim.x) {
    const int j = v.chunk_pair[c];
    const BatchPair& bp = v.pairs[j];
    const SolveState* st = v.states + j;
    if (st->done || !st->replace_pending) continue;
    const int64_t r0 = (int64_t)(c - bp.chunk0) * v.chunk_rows;
    int64_t r1 = r0 + v.chunk_rows;
    if (r1 > bp.n) r1 = bp.n;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const int64_t k = bp.off + i;
      r[k] = rt[k];
      p[k] = rt[k];
    }
  }
}

__global__ void batch_hscg_end_kernel(BatchView v) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < v.npairs; j += gridDim.x * blockDim.x) {
    SolveState* st = v.states + j;
    if (st->done) continue;
    if (st->replace_pending) {
      st->replace_pending = 0;
      st->converged_est = 0;
      st->h_rr = st->rt2;
      st->replacements += 1;
    }
    atomicAdd(v.active, 1u);
  }
}

int chunk_grid(const BatchView& v) {
  int g = v.nchunks < 152 * 8 ? v.nchunks : 152 * 8;
  return g < 1 ? 1 : g;
}

}  // namespace

int reduce_blocks(int64_t n) { return vec_grid(n); }

cudaError_t launch_batch_init(const BatchView& v, const double* b, double* x, double* Y, int64_t LD,
                              double* partials, cudaStream_t st) {
  batch_init_kernel<<<chunk_grid(v), kVecThreads, 0, st>>>(v, b, x, Y, LD, partials);
  batch_zero_x_kernel<<<chunk_grid(v), kVecThreads, 0, st>>>(v, x);
  return cudaGetLastError();
}

cudaError_t launch_batch_recombine(const BatchView& v, double* Y, int64_t LD, double* x, cudaStream_t st,
                                   int fp64_per16) {
  batch_recombine_kernel<<<chunk_grid(v), kVecThreads, 0, st>>>(v, Y, LD, x,
                                                                fp64_per16 < 0 ? kRecFp64Per16 : fp64_per16);
  return cudaGetLastError();
}

cudaError_t launch_batch_check(const BatchView& v, const double* b, const double* x, double* rt, double* Y,
                               int64_t LD, double* partials, cudaStream_t st) {
  batch_true_residual_kernel<<<chunk_grid(v), kVecThreads, 0, st>>>(v, b, x, rt, partials);
  batch_replacement_kernel<<<chunk_grid(v), kVecThreads, 0, st>>>(v, rt, Y, LD);
  return cudaGetLastError();
}

cudaError_t launch_batch_hscg_init(const BatchView& v, const double* b, double* x, double* r, double* p,
                                   double* partials, cudaStream_t st) {
  batch_hscg_init_kernel<<<chunk_grid(v), kVecThreads, 0, st>>>(v, b, x, r, p, partials);
  batch_hscg_rr_kernel<<<chunk_grid(v), kVecThreads, 0, st>>>(v, r, partials);
  batch_zero_x_kernel<<<chunk_grid(v), kVecThreads, 0, st>>>(v, x);
  return cudaGetLastError();
}

cudaError_t launch_batch_hscg_iteration(const BatchView& v, double* x, double* r, double* p, double* q,
                                        double* partials, cudaStream_t st) {
  batch_hscg_q_kernel<<<chunk_grid(v), kVecThreads, 0, st>>>(v, p, q, partials);
  batch_hscg_update_kernel<<<chunk_grid(v), kVecThreads, 0, st>>>(v, x, r, p, q, partials);
  batch_hscg_p_kernel<<<chunk_grid(v), kVecThreads, 0, st>>>(v, r, p);
  return cudaGetLastError();
}

cudaError_t launch_batch_hscg_check(const BatchView& v, const double* b, const double* x, double* rt, double* r,
                                    double* p, double* partials, cudaGraphConditionalHandle cond, int use_cond,
                                    cudaStream_t st) {
  batch_true_residual_kernel<<<chunk_grid(v), kVecThreads, 0, st>>>(v, b, x, rt, partials);
  batch_hscg_replace_kernel<<<chunk_grid(v), kVecThreads, 0, st>>>(v, rt, r, p);
  const int g = (v.npairs + 255) / 256;
  batch_hscg_end_kernel<<<g < 1 ? 1 : g, 256, 0, st>>>(v);
  if (use_cond) batch_cond_kernel<<<1, 32, 0, st>>>(v, cond);
  return cudaGetLastError();
}

cudaError_t launch_batch_begin(const BatchView& v, cudaStream_t st) {
  batch_begin_kernel<<<1, 32, 0, st>>>(v);
  return cudaGetLastError();
}

cudaError_t launch_batch_end(const BatchView& v, cudaGraphConditionalHandle cond, int use_cond, cudaStream_t st) {
  const int g = (v.npairs + 255) / 256;
  batch_end_kernel<<<g < 1 ? 1 : g, 256, 0, st>>>(v);
  if (use_cond) batch_cond_kernel<<<1, 32, 0, st>>>(v, cond);
  return cudaGetLastError();
}

cudaError_t launch_set_state(SolveState* state, const SolveState& config, cudaStream_t st) {
  set_state_kernel<<<1, 128, 0, st>>>(state, config);
  return cudaGetLastError();
}

cudaError_t launch_solve_cond(const SolveState* state, cudaGraphConditionalHandle cond, cudaStream_t st) {
  solve_cond_kernel<<<1, 32, 0, st>>>(state, cond);
  return cudaGetLastError();
}

cudaError_t launch_batch_arm(cudaGraphConditionalHandle cond, cudaStream_t st) {
  batch_arm_kernel<<<1, 32, 0, st>>>(cond);
  return cudaGetLastError();
}

cudaError_t launch_recombine(const SolveState* state, void* Y, int64_t ld, double* x, double* r64, double* p64,
                             int64_t n, bool y32, cudaStream_t st, int fp64_per16) {
  const int f16 = fp64_per16 < 0 ? kRecFp64Per16 : fp64_per16;
  if (!y32 && f16 < 16)
    recombine_hybrid_kernel<<<vec_grid(n), kVecThreads, 0, st>>>(state, static_cast<double*>(Y), ld, x, n, f16);
  else if (y32)
    recombine_kernel<float><<<vec_grid(n), kVecThreads, 0, st>>>(state, static_cast<float*>(Y), ld, x, r64, p64, n);
  else
    recombine_kernel<double><<<vec_grid(n), kVecThreads, 0, st>>>(state, static_cast<double*>(Y), ld, x, nullptr,
                                                                  nullptr, n);
  return cudaGetLastError();
}

cudaError_t launch_init_state(SolveState* state, const Operator& A, const double* b, const double* x, void* Y,
                              int64_t ld, double* r64, double* p64, double* partials, int nblocks, bool y32,
                              cudaStream_t st) {
  if (y32) {
    cudaError_t e = launch_residual(A, b, x, r64, st);  // r0 in binary64
    if (e != cudaSuccess) return e;
    init_norms_kernel<float><<<nblocks, kVecThreads, 0, st>>>(state, b, r64, static_cast<float*>(Y), ld, p64, A.n,
                                                              partials);
  } else {
    double* Yd = static_cast<double*>(Y);
    cudaError_t e = launch_residual(A, b, x, Yd + ld, st);  // r0 into column 1
    if (e != cudaSuccess) return e;
    init_norms_kernel<double><<<nblocks, kVecThreads, 0, st>>>(state, b, Yd + ld, Yd, ld, nullptr, A.n, partials);
  }
  zero_x_kernel<<<vec_grid(A.n), kVecThreads, 0, st>>>(state, const_cast<double*>(x), A.n);
  return cudaGetLastError();
}

}  // namespace sscg

namespace sscg {

cudaError_t launch_true_residual(SolveState* state, const Operator& A, const double* b, const double* x, double* rt,
                                 double* partials, int nblocks, cudaStream_t st) {
  cudaError_t e = launch_residual(A, b, x, rt, st, state, 1);
  if (e != cudaSuccess) return e;
  true_norm_kernel<<<nblocks, kVecThreads, 0, st>>>(state, rt, A.n, partials, 0);
  return cudaGetLastError();
}

cudaError_t launch_final_norm(SolveState* state, const Operator& A, const double* b, const double* x, double* rt,
                              double* partials, int nblocks, cudaStream_t st) {
  cudaError_t e = launch_residual(A, b, x, rt, st);
  if (e != cudaSuccess) return e;
  true_norm_kernel<<<nblocks, kVecThreads, 0, st>>>(state, rt, A.n, partials, 1);
  return cudaGetLastError();
}

cudaError_t launch_apply_replacement(SolveState* state, const double* rt, void* Y, int64_t ld, double* r64,
                                     double* p64, int64_t n, bool y32, sscg_outer_record* hist, cudaStream_t st) {
  if (y32)
    replacement_kernel<float><<<vec_grid(n), kVecThreads, 0, st>>>(state, rt, static_cast<float*>(Y), ld, r64, p64,
                                                                   n);
  else
    replacement_kernel<double><<<vec_grid(n), kVecThreads, 0, st>>>(state, rt, static_cast<double*>(Y), ld, nullptr,
                                                                    nullptr, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  end_of_loop_kernel<<<1, 32, 0, st>>>(state, hist);
  return cudaGetLastError();
}

cudaError_t launch_fp32_replacement(SolveState* state, const Operator& A, const double* b, const double* x, void* Y,
                                    int64_t ld, double* r64, double* partials, int nblocks, sscg_outer_record* hist,
                                    cudaStream_t st) {
  cudaError_t e = launch_residual(A, b, x, r64, st, state, 3);
  if (e != cudaSuccess) return e;
  fp32_replace_kernel<<<nblocks, kVecThreads, 0, st>>>(state, r64, static_cast<float*>(Y), ld, A.n, partials, hist);
  return cudaGetLastError();
}

cudaError_t launch_hscg_init(SolveState* state, const Operator& A, const double* b, const double* x, double* r,
                             double* p, double* partials, int nblocks, cudaStream_t st) {
  cudaError_t e = launch_residual(A, b, x, r, st);
  if (e != cudaSuccess) return e;
  hscg_init_kernel<<<nblocks, kVecThreads, 0, st>>>(state, b, r, p, A.n, partials, partials + nblocks);
  zero_x_kernel<<<vec_grid(A.n), kVecThreads, 0, st>>>(state, const_cast<double*>(x), A.n);
  return cudaGetLastError();
}

cudaError_t launch_hscg_iteration(SolveState* state, const Operator& A, double* x, double* r, double* p, double* q,
                                  double* partials, int nblocks, cudaStream_t st, int spmv_fp64_per16) {
  cudaError_t e = launch_spmv_split(A, p, q, st, state, 2, spmv_fp64_per16);
  if (e != cudaSuccess) return e;
  hscg_pq_kernel<<<nblocks, kVecThreads, 0, st>>>(state, p, q, A.n, partials);
  hscg_update_kernel<<<nblocks, kVecThreads, 0, st>>>(state, x, r, p, q, A.n, partials);
  hscg_pupdate_kernel<<<nblocks, kVecThreads, 0, st>>>(state, r, p, A.n);
  return cudaGetLastError();
}

cudaError_t launch_hscg_check(SolveState* state, const Operator& A, const double* b, const double* x, double* r,
                              double* p, double* rt, double* partials, int nblocks, cudaStream_t st) {
  cudaError_t e = launch_residual(A, b, x, rt, st, state, 1);
  if (e != cudaSuccess) return e;
  hscg_confirm_kernel<<<nblocks, kVecThreads, 0, st>>>(state, rt, r, p, A.n, partials);
  hscg_replace_kernel<<<vec_grid(A.n), kVecThreads, 0, st>>>(state, rt, r, p, A.n);
  hscg_replace_finish_kernel<<<1, 1, 0, st>>>(state);
  return cudaGetLastError();
}

}  // namespace sscg
