// The outer loop of Algorithm 5 without a stored basis (recompute-Y), for
// 2D face-coefficient stencils.
//
// The s-step method needs the basis Y = [rho_0(A) p, rho_0(A) r, ..., rho_s(A) p]
// twice per outer loop: for its Gram matrix G = Y^T Y (Section 2) and for the
// recovery x += Y x', r = Y r', p = Y p' (eq. coords).  Here Y never reaches
// global memory.  Each 16 x 16 tile of the grid recomputes its part of the
// basis from p and r over the tile and a halo of s-bar cells (the matrix
// powers of eq. (rho) widen the dependence by one cell per level), first to
// sum its share of G, then, after the control step, again to form its rows of
// x, r and p.  Memory falls from (2 s-bar + 1) N to 4 N binary64 values; the
// stencil work grows by the halo (((16 + 2 s-bar) / 16)^2 at s-bar levels),
// so on GB300, whose binary64 rate binds the matrix powers, it is a memory
// saving, not a speed-up.
//
// Every basis value is formed with the arithmetic of stencil_mpk_grid_kernel
// (the same binary64 FMA order) and every recovery sum in the column order of
// recombine_kernel, so the columns are the stored path's (FMA form) bit for
// bit; only the Gram's summation order differs (per tile, then over tiles).
#include "sscg_internal.cuh"

namespace sscg {

namespace {

constexpr int kRT = 16;                          // tile edge
constexpr int kRThreads = kRT * kRT;             // one tile cell per thread
constexpr int kRMaxEdge = kRT + 2 * kMaxS;       // tile and halo of s-bar <= 16
constexpr int kRMaxCells = kRMaxEdge * kRMaxEdge;
constexpr int kRColStride = kRThreads + 1;       // padded: the pair sums read rows i and j at one cell

size_t rc_smem_bytes(bool gram) {
  return 4 * (size_t)kRMaxCells * sizeof(double) + (gram ? (size_t)kMaxCols * kRColStride * sizeof(double) : 0);
}

// GRAM = true: the tile's share of G (pairs i <= j of the 2 s-bar + 1
// columns) into partials[tile * kMaxPairs + pair], and the loop's recurrence
// coefficients (theta, 1/gamma, mu of eq. rho) into coef[0 .. 3 kMaxS): the
// control step replaces the state's with the next loop's before the recovery
// needs them again.  GRAM = false: the recovery over the nc = 2 s_k + 1
// columns with the saved coefficients: x += Y x', and the new p and r into
// PRnew (columns 0 and 1, leading dimension n).  PR holds the current p
// (column 0) and r (column 1), leading dimension n.
template <bool GRAM>
__global__ void __launch_bounds__(kRThreads) recompute_kernel(Operator A, const double* __restrict__ PR,
                                                              double* __restrict__ PRnew, double* __restrict__ x,
                                                              const SolveState* __restrict__ st,
                                                              double* __restrict__ partials,
                                                              double* __restrict__ coef) {
  if (st->done) return;
  const double* th = GRAM ? st->theta : coef;
  const double* ig_ = GRAM ? st->inv_gamma : coef + kMaxS;
  const double* mu_ = GRAM ? st->mu : coef + 2 * kMaxS;
  if (GRAM && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x < kMaxS) {
    coef[threadIdx.x] = st->theta[threadIdx.x];
    coef[kMaxS + threadIdx.x] = st->inv_gamma[threadIdx.x];
    coef[2 * kMaxS + threadIdx.x] = st->mu[threadIdx.x];
  }
  const int nx = A.nx, ny = A.ny;
  const int64_t n = (int64_t)nx * ny;
  const int sbar = st->sbar;
  const int nlev = GRAM ? sbar : st->sk;   // P_0..P_nlev and R_0..R_{nlev-1} (GRAM: as the stored levels)
  const int ncols = GRAM ? 2 * sbar + 1 : st->nc;
  const int h = nlev;
  const int E = kRT + 2 * h;
  const int t = threadIdx.x;
  const int tix = t % kRT, tiy = t / kRT;
  const int x0 = blockIdx.x * kRT - h, y0 = blockIdx.y * kRT - h;   // region origin

  extern __shared__ double rc_smem[];
  double* pm = rc_smem;                    // P_{l-1}, then P_{l+1}
  double* p0 = pm + kRMaxCells;            // P_l
  double* rm = p0 + kRMaxCells;
  double* r0 = rm + kRMaxCells;
  double* ycol = r0 + kRMaxCells;          // GRAM: column c of the tile at ycol[c * kRColStride + cell]
  __shared__ double cx[kMaxCols], cr[kMaxCols], cp[kMaxCols];
  if (!GRAM && t < kMaxCols) {
    cx[t] = st->xc[t];
    cr[t] = st->rc[t];
    cp[t] = st->pc[t];
  }
  for (int q = t; q < E * E; q += kRThreads) {
    const int gx = x0 + q % E, gy = y0 + q / E;
    const bool in = gx >= 0 && gx < nx && gy >= 0 && gy < ny;
    const int64_t gi = (int64_t)gy * nx + gx;
    pm[q] = 0.0;
    rm[q] = 0.0;
    p0[q] = in ? PR[gi] : 0.0;
    r0[q] = in ? PR[n + gi] : 0.0;
  }
  __syncthreads();

  // this thread's tile cell
  const int qc = (h + tiy) * E + (h + tix);
  const int cgx = blockIdx.x * kRT + tix, cgy = blockIdx.y * kRT + tiy;
  const bool cin = cgx < nx && cgy < ny;
  double sx = 0.0, sr = 0.0, sp = 0.0;
  auto take = [&](int c, double y) {   // column c at the tile cell, in column order
    if (GRAM) {
      ycol[c * kRColStride + t] = y;
    } else {
      sx = fma(y, cx[c], sx);
      sr = fma(y, cr[c], sr);
      sp = fma(y, cp[c], sp);
    }
  };
  take(0, p0[qc]);
  if (ncols > 1) take(1, r0[qc]);

  for (int l = 0; l < nlev; ++l) {
    const bool doR = l + 1 < nlev;   // R_{l+1} is a column only below the last level
    const double theta = th[l];
    const double ig = ig_[l];
    const double mu = l >= 1 ? mu_[l - 1] : 0.0;
    const int lo = l + 1, hi = E - l - 2;   // cells whose neighbours hold level l
    const int w = hi - lo + 1;
    for (int k = t; k < w * w; k += kRThreads) {
      const int rx = lo + k % w, ry = lo + k / w;
      const int gx = x0 + rx, gy = y0 + ry;
      if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) continue;   // outside the domain: zero at every level
      const int q = ry * E + rx;
      const int64_t i = (int64_t)gy * nx + gx;
      const int64_t fx = (int64_t)gy * (nx + 1) + gx;
      const int64_t fy = (int64_t)gy * nx + gx;
      const double kw = -__ldg(A.kx + fx), ke = -__ldg(A.kx + fx + 1);
      const double ks = -__ldg(A.ky + fy), kn = -__ldg(A.ky + fy + nx);
      const double ds = __ldg(A.diag + i) - theta;
      // the order of stencil_mpk_grid_kernel (2D)
      double acc = ds * p0[q];
      acc = fma(kw, p0[q - 1], acc);
      acc = fma(ke, p0[q + 1], acc);
      acc = fma(ks, p0[q - E], acc);
      acc = fma(kn, p0[q + E], acc);
      if (mu != 0.0) acc = fma(-mu, pm[q], acc);
      const double pn = acc * ig;
      double rn = 0.0;
      if (doR) {
        acc = ds * r0[q];
        acc = fma(kw, r0[q - 1], acc);
        acc = fma(ke, r0[q + 1], acc);
        acc = fma(ks, r0[q - E], acc);
        acc = fma(kn, r0[q + E], acc);
        if (mu != 0.0) acc = fma(-mu, rm[q], acc);
        rn = acc * ig;
      }
      pm[q] = pn;   // P_{l-1} at this cell is no longer needed
      if (doR) rm[q] = rn;
    }
    __syncthreads();
    double* tp = pm;
    pm = p0;
    p0 = tp;
    double* tr = rm;
    rm = r0;
    r0 = tr;
    take(2 * l + 2, cin ? p0[qc] : 0.0);
    if (doR) take(2 * l + 3, cin ? r0[qc] : 0.0);
    __syncthreads();
  }

  const int64_t tile = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
  if (GRAM) {
    // this tile's share of every pair (i <= j), cells in order
    const int np = ncols * (ncols + 1) / 2;
    for (int p = t; p < np; p += kRThreads) {
      int i = 0, rest = p;
      while (rest >= ncols - i) {
        rest -= ncols - i;
        ++i;
      }
      const int j = i + rest;
      const double* a = ycol + i * kRColStride;
      const double* b = ycol + j * kRColStride;
      double s = 0.0;
      for (int c = 0; c < kRThreads; ++c) s = fma(a[c], b[c], s);
      partials[tile * kMaxPairs + p] = s;
    }
  } else if (cin) {
    const int64_t i = (int64_t)cgy * nx + cgx;
    x[i] += sx;
    PRnew[i] = sp;
    PRnew[n + i] = sr;
  }
}

dim3 tile_grid(const Operator& A) { return dim3((A.nx + kRT - 1) / kRT, (A.ny + kRT - 1) / kRT); }

}  // namespace

bool recompute_supported(const Operator& A) {
  return A.kind == 1 && A.dim == 2 && (A.nx + kRT - 1) / kRT < 65536 && (A.ny + kRT - 1) / kRT < 65536;
}

int64_t recompute_partials(const Operator& A) {
  const dim3 g = tile_grid(A);
  return (int64_t)g.x * g.y * kMaxPairs;
}

cudaError_t recompute_prepare() {
  cudaError_t e = cudaFuncSetAttribute(recompute_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)rc_smem_bytes(true));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(recompute_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)rc_smem_bytes(false));
}

cudaError_t launch_recompute_gram(const Operator& A, const double* PR, const SolveState* state, double* partials,
                                  double* coef, double* G, int ldg, cudaStream_t st) {
  const dim3 g = tile_grid(A);
  recompute_kernel<true><<<g, kRThreads, rc_smem_bytes(true), st>>>(A, PR, nullptr, nullptr, state, partials, coef);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_gram_reduce(partials, (int)(g.x * g.y), state, 0, G, ldg, st);
}

cudaError_t launch_recompute_recover(const Operator& A, double* PR, double* PRnew, double* x,
                                     const SolveState* state, double* coef, cudaStream_t st) {
  recompute_kernel<false><<<tile_grid(A), kRThreads, rc_smem_bytes(false), st>>>(A, PR, PRnew, x, state, nullptr,
                                                                                 coef);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(PR, PRnew, 2 * (size_t)A.n * sizeof(double), cudaMemcpyDeviceToDevice, st);
}

}  // namespace sscg
