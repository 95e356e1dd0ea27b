// Sparse operator kernels: SpMV, residual and one matrix-powers level, for the
// face-coefficient stencil and for CSR.
//
// The matrix-powers level implements the three-term recurrence of Carson 2019,
// eq. (rho), for both chains of eq. (cg-krylovbasis) in one pass over A:
//   P_{l+1} = ((A - theta_l I) P_l - mu_{l-1} P_{l-1}) / gamma_l   (l < s-bar)
//   R_{l+1} = ((A - theta_l I) R_l - mu_{l-1} R_{l-1}) / gamma_l   (l + 1 < s-bar)
// so the coefficients of A are read once per level for both chains.  On GB300
// these kernels are bound by FP64 issue rate (2 DFMA/clk/SM), not by HBM, so
// they minimise FP64 instructions: theta is folded into the diagonal once per
// cell and shared by both chains, 1/gamma is a precomputed multiplier, and the
// mu term is skipped (uniform branch) when mu = 0.  Every lane of a warp does
// the same FP64 work (boundary neighbours read as 0 by predication), because
// masked lanes do not free FP64 issue slots.
#include "exact_sum.cuh"
#include "sscg_internal.cuh"

namespace sscg {

namespace {

constexpr int kOpThreads = 256;

__host__ __device__ inline int grid_for(int64_t n, int per_thread) {
  int64_t g = (n + (int64_t)kOpThreads * per_thread - 1) / ((int64_t)kOpThreads * per_thread);
  if (g < 1) g = 1;
  if (g > 152 * 16) g = 152 * 16;
  return (int)g;
}

template <typename T>
__device__ __forceinline__ double ld_val(const T* p) { return widen(__ldg(p)); }

// (A - shift I) v at cell i of a stencil, v read through `vp` (stride-1 vector).
// Coordinates (x, y, z) of cell i; boundary neighbours contribute 0.
template <bool DIM3, typename T>
__device__ __forceinline__ double stencil_apply(const Operator& A, const T* __restrict__ v, int64_t i,
                                                int x, int y, int z, double dshift) {
  const int nx = A.nx, ny = A.ny, nz = A.nz;
  const int64_t plane = (int64_t)nx * ny;
  const int64_t fx = ((int64_t)z * ny + y) * (nx + 1) + x;
  const int64_t fy = ((int64_t)z * (ny + 1) + y) * nx + x;
  double vi = ld_val(v + i);
  double vw = x > 0 ? ld_val(v + i - 1) : 0.0;
  double ve = x < nx - 1 ? ld_val(v + i + 1) : 0.0;
  double vs = y > 0 ? ld_val(v + i - nx) : 0.0;
  double vn = y < ny - 1 ? ld_val(v + i + nx) : 0.0;
  double acc = dshift * vi;
  acc = fma(-__ldg(A.kx + fx), vw, acc);
  acc = fma(-__ldg(A.kx + fx + 1), ve, acc);
  acc = fma(-__ldg(A.ky + fy), vs, acc);
  acc = fma(-__ldg(A.ky + fy + nx), vn, acc);
  if (DIM3) {
    double vd = z > 0 ? ld_val(v + i - plane) : 0.0;
    double vu = z < nz - 1 ? ld_val(v + i + plane) : 0.0;
    acc = fma(-__ldg(A.kz + i), vd, acc);
    acc = fma(-__ldg(A.kz + i + plane), vu, acc);
  }
  return acc;
}

// Launch gates read from the solve state: 0 = always run, 1 = only when a
// true-residual check is pending, 2 = only while the iteration is running,
// 3 = only when an FP32-basis residual replacement is pending.
__device__ __forceinline__ bool gate_closed(const SolveState* g, int mode) {
  if (mode == 0 || g == nullptr) return false;
  if (g->done) return true;
  if (mode == 3) return !g->fp32_replace_pending;
  return mode == 1 ? !g->converged_est : g->converged_est != 0;
}

template <bool DIM3>
__global__ void __launch_bounds__(kOpThreads) stencil_spmv_kernel(Operator A, const double* __restrict__ v,
                                                                  double* __restrict__ y, const SolveState* gate,
                                                                  int gmode) {
  if (gate_closed(gate, gmode)) return;
  const int64_t n = A.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int x = (int)(i % A.nx);
    int64_t t = i / A.nx;
    int yy = (int)(t % A.ny);
    int z = (int)(t / A.ny);
    y[i] = stencil_apply<DIM3>(A, v, i, x, yy, z, __ldg(A.diag + i));
  }
}

template <bool DIM3>
__global__ void __launch_bounds__(kOpThreads) stencil_residual_kernel(Operator A, const double* __restrict__ b,
                                                                      const double* __restrict__ xv,
                                                                      double* __restrict__ r, const SolveState* gate,
                                                                      int gmode) {
  if (gate_closed(gate, gmode)) return;
  const int64_t n = A.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int x = (int)(i % A.nx);
    int64_t t = i / A.nx;
    int yy = (int)(t % A.ny);
    int z = (int)(t / A.ny);
    r[i] = b[i] - stencil_apply<DIM3>(A, xv, i, x, yy, z, __ldg(A.diag + i));
  }
}

// One matrix-powers level for a stencil.  `sbar` is read from the solve state
// (device) unless sbar_fixed > 0.  T is the storage type of the basis
// (double, or float for the FP32-stored variant: loads widen to binary64,
// the recurrence runs in binary64, stores round to binary32).
template <bool DIM3, typename T>
__global__ void __launch_bounds__(kOpThreads) stencil_mpk_kernel(Operator A, T* __restrict__ Y, int64_t ld,
                                                                 int level, const SolveState* __restrict__ st,
                                                                 int sbar_fixed, LevelCoef coef) {
  int sbar = sbar_fixed;
  if (sbar <= 0) {
    if (st->done) return;
    sbar = st->sbar;
  }
  const bool doP = level < sbar;
  const bool doR = level + 1 < sbar;
  if (!doP) return;
  const double theta = coef.theta[level];
  const double ig = coef.inv_gamma[level];
  const double mu = level >= 1 ? coef.mu[level - 1] : 0.0;
  const T* Pl = Y + (int64_t)(2 * level) * ld;
  const T* Rl = Y + (int64_t)(2 * level + 1) * ld;
  const T* Pm = level >= 1 ? Y + (int64_t)(2 * level - 2) * ld : nullptr;
  const T* Rm = level >= 1 ? Y + (int64_t)(2 * level - 1) * ld : nullptr;
  T* Pn = Y + (int64_t)(2 * level + 2) * ld;
  T* Rn = Y + (int64_t)(2 * level + 3) * ld;
  const int64_t n = A.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int x = (int)(i % A.nx);
    int64_t t = i / A.nx;
    int yy = (int)(t % A.ny);
    int z = (int)(t / A.ny);
    const double ds = __ldg(A.diag + i) - theta;
    double wp = stencil_apply<DIM3>(A, Pl, i, x, yy, z, ds);
    if (mu != 0.0) wp = fma(-mu, ld_val(Pm + i), wp);
    Pn[i] = (T)(wp * ig);
    if (doR) {
      double wr = stencil_apply<DIM3>(A, Rl, i, x, yy, z, ds);
      if (mu != 0.0) wr = fma(-mu, ld_val(Rm + i), wr);
      Rn[i] = (T)(wr * ig);
    }
  }
}

// One matrix-powers level for a stencil, one cell per thread on a 3D grid
// (x in 32-lane rows, y in 8-row tiles, z per grid plane): the coordinates
// come from the launch indices, with no division.  The block first stages
// its 34 x 10 in-plane tile of P_l and R_l (halo included, zero outside the
// domain) in shared memory, so the four in-plane neighbours come from shared
// memory and only the centre tile and the two z neighbours from L1/L2; the
// sum is formed in stencil_apply's order (same bits as the grid-stride
// kernel).
template <bool DIM3, typename T>
__global__ void __launch_bounds__(256) stencil_mpk_grid_kernel(Operator A, T* __restrict__ Y, int64_t ld,
                                                                 int level, const SolveState* __restrict__ st,
                                                                 int sbar_fixed, LevelCoef coef) {
  int sbar = sbar_fixed;
  if (sbar <= 0) {
    if (st->done) return;
    sbar = st->sbar;
  }
  const bool doP = level < sbar;
  const bool doR = level + 1 < sbar;
  if (!doP) return;
  const int nx = A.nx, ny = A.ny, nz = A.nz;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 8;
  const int x = x0 + tx, yy = y0 + ty, z = blockIdx.z;
  const T* Pl = Y + (int64_t)(2 * level) * ld;
  const T* Rl = Y + (int64_t)(2 * level + 1) * ld;
  T* Pn = Y + (int64_t)(2 * level + 2) * ld;
  T* Rn = Y + (int64_t)(2 * level + 3) * ld;
  __shared__ double sP[10][34], sR[10][34];
  const int64_t zoff = (int64_t)z * ny * nx;
  for (int e = ty * 32 + tx; e < 340; e += 256) {
    const int ly = e / 34, lx = e - ly * 34;
    const int gx = x0 + lx - 1, gy = y0 + ly - 1;
    const bool in = gx >= 0 && gx < nx && gy >= 0 && gy < ny;
    const int64_t gi = zoff + (int64_t)gy * nx + gx;
    sP[ly][lx] = in ? ld_val(Pl + gi) : 0.0;
    sR[ly][lx] = (in && doR) ? ld_val(Rl + gi) : 0.0;
  }
  __syncthreads();
  if (x >= nx || yy >= ny) return;
  const int64_t plane = (int64_t)nx * ny;
  const int64_t i = zoff + (int64_t)yy * nx + x;
  const int64_t fx = ((int64_t)z * ny + yy) * (nx + 1) + x;
  const int64_t fy = ((int64_t)z * (ny + 1) + yy) * nx + x;
  const double kw = -__ldg(A.kx + fx), ke = -__ldg(A.kx + fx + 1);
  const double ks = -__ldg(A.ky + fy), kn = -__ldg(A.ky + fy + nx);
  double kd = 0.0, ku = 0.0;
  if (DIM3) {
    kd = -__ldg(A.kz + i);
    ku = -__ldg(A.kz + i + plane);
  }
  const double theta = coef.theta[level];
  const double ig = coef.inv_gamma[level];
  const double mu = level >= 1 ? coef.mu[level - 1] : 0.0;
  const double ds = __ldg(A.diag + i) - theta;
  const int ly = ty + 1, lx = tx + 1;
  {
    double acc = ds * sP[ly][lx];
    acc = fma(kw, sP[ly][lx - 1], acc);
    acc = fma(ke, sP[ly][lx + 1], acc);
    acc = fma(ks, sP[ly - 1][lx], acc);
    acc = fma(kn, sP[ly + 1][lx], acc);
    if (DIM3) {
      acc = fma(kd, z > 0 ? ld_val(Pl + i - plane) : 0.0, acc);
      acc = fma(ku, z < nz - 1 ? ld_val(Pl + i + plane) : 0.0, acc);
    }
    if (mu != 0.0) acc = fma(-mu, ld_val(Y + (int64_t)(2 * level - 2) * ld + i), acc);
    Pn[i] = (T)(acc * ig);
  }
  if (doR) {
    double acc = ds * sR[ly][lx];
    acc = fma(kw, sR[ly][lx - 1], acc);
    acc = fma(ke, sR[ly][lx + 1], acc);
    acc = fma(ks, sR[ly - 1][lx], acc);
    acc = fma(kn, sR[ly + 1][lx], acc);
    if (DIM3) {
      acc = fma(kd, z > 0 ? ld_val(Rl + i - plane) : 0.0, acc);
      acc = fma(ku, z < nz - 1 ? ld_val(Rl + i + plane) : 0.0, acc);
    }
    if (mu != 0.0) acc = fma(-mu, ld_val(Y + (int64_t)(2 * level - 1) * ld + i), acc);
    Rn[i] = (T)(acc * ig);
  }
}

// The binary64 FMA chain of one cell and chain of a matrix-powers level, from
// global memory (the rare cells whose integer form does not apply: Inf/NaN
// inputs, or a sum outside the normal binary64 range).  Kept out of line so
// that the integer path does not hold its operands in registers.
template <bool DIM3>
__device__ __noinline__ double mpk_cell_fma(const Operator& A, const double* __restrict__ Vl,
                                            const double* __restrict__ Vm, int64_t i, int x, int yy, int z,
                                            double ds, double mu) {
  double w = stencil_apply<DIM3>(A, Vl, i, x, yy, z, ds);
  if (mu != 0.0) w = fma(-mu, __ldg(Vm + i), w);
  return w;
}

// One matrix-powers level for a stencil with a binary64 basis, its binary64
// work split between two units: of every 16 warps, `fp64_per16` form their
// cells' sums as the binary64 FMA chain of stencil_mpk_grid_kernel, the others
// with exact integer products (exact_sum.cuh: the 5 or 7 stencil products and
// the mu term of each chain, in two passes: the largest exponent sum first,
// from the high words of the operands alone, then every product aligned to
// it, summed and rounded once, then times 1/gamma in binary64; the products
// of a chain are independent, and few values stay live, so five blocks fit
// on an SM).  GB300's FP64 unit and its integer pipes run concurrently, so
// the level's time falls towards that of the slower share.  Both forms are
// binary64-accurate (the integer one more so); a cell's result depends only
// on which form its warp takes, which depends only on the warp's position, so
// results are reproducible.  Inf or NaN among a cell's inputs, or a sum
// outside the normal binary64 range, sends that cell to the FMA chain.
template <bool DIM3>
__global__ void __launch_bounds__(256, 5) stencil_mpk_hybrid_kernel(Operator A, double* __restrict__ Y, int64_t ld,
                                                                      int level, const SolveState* __restrict__ st,
                                                                      int sbar_fixed, LevelCoef coef, int fp64_per16) {
  int sbar = sbar_fixed;
  if (sbar <= 0) {
    if (st->done) return;
    sbar = st->sbar;
  }
  const bool doP = level < sbar;
  const bool doR = level + 1 < sbar;
  if (!doP) return;
  const int nx = A.nx, ny = A.ny, nz = A.nz;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 8;
  const int x = x0 + tx, yy = y0 + ty, z = blockIdx.z;
  __shared__ double sv[2][10][34];   // P_l, R_l tiles (halo included, zero outside the domain)
  __shared__ int2 lv[2][10][34];     // their limbs a, b
  __shared__ int ev[2][10][34];      // and exponents
  const int64_t zoff = (int64_t)z * ny * nx;
  unsigned bad = 0;
  for (int e = ty * 32 + tx; e < 340; e += 256) {
    const int ly = e / 34, lx = e - ly * 34;
    const int gx = x0 + lx - 1, gy = y0 + ly - 1;
    const bool in = gx >= 0 && gx < nx && gy >= 0 && gy < ny;
    const int64_t gi = (int64_t)(2 * level) * ld + zoff + (int64_t)gy * nx + gx;
    const double vp = in ? __ldg(Y + gi) : 0.0;
    const double vr = in && doR ? __ldg(Y + gi + ld) : 0.0;
    sv[0][ly][lx] = vp;
    sv[1][ly][lx] = vr;
    const Limbs lp = to_limbs(vp, bad), lr = to_limbs(vr, bad);
    lv[0][ly][lx] = make_int2(lp.a, lp.b);
    ev[0][ly][lx] = lp.e;
    lv[1][ly][lx] = make_int2(lr.a, lr.b);
    ev[1][ly][lx] = lr.e;
  }
  const int tile_bad = __syncthreads_or((int)bad);
  if (x >= nx || yy >= ny) return;
  const int64_t plane = (int64_t)nx * ny;
  const int64_t i = zoff + (int64_t)yy * nx + x;
  const int64_t fx = ((int64_t)z * ny + yy) * (nx + 1) + x;
  const int64_t fy = ((int64_t)z * (ny + 1) + yy) * nx + x;
  const double theta = coef.theta[level];
  const double ig = coef.inv_gamma[level];
  const double mu = level >= 1 ? coef.mu[level - 1] : 0.0;
  const double ds = __ldg(A.diag + i) - theta;
  const int ly = ty + 1, lx = tx + 1;
  const unsigned warp = ((blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * 8u + (unsigned)ty;
  const bool fma_warp = ((warp * (unsigned)fp64_per16) & 15u) < (unsigned)fp64_per16;
  if (fma_warp || tile_bad) {
    // the binary64 FMA chain (the form and order of stencil_mpk_grid_kernel)
    const double kw = -__ldg(A.kx + fx), ke = -__ldg(A.kx + fx + 1);
    const double ks = -__ldg(A.ky + fy), kn = -__ldg(A.ky + fy + nx);
    const double kd = DIM3 ? -__ldg(A.kz + i) : 0.0, ku = DIM3 ? -__ldg(A.kz + i + plane) : 0.0;
#pragma unroll 1
    for (int ch = 0; ch < (doR ? 2 : 1); ++ch) {
      const double* Vl = Y + (int64_t)(2 * level + ch) * ld;
      double acc = ds * sv[ch][ly][lx];
      acc = fma(kw, sv[ch][ly][lx - 1], acc);
      acc = fma(ke, sv[ch][ly][lx + 1], acc);
      acc = fma(ks, sv[ch][ly - 1][lx], acc);
      acc = fma(kn, sv[ch][ly + 1][lx], acc);
      if (DIM3) {
        acc = fma(kd, z > 0 ? __ldg(Vl + i - plane) : 0.0, acc);
        acc = fma(ku, z < nz - 1 ? __ldg(Vl + i + plane) : 0.0, acc);
      }
      if (mu != 0.0) acc = fma(-mu, __ldg(Y + (int64_t)(2 * level - 2 + ch) * ld + i), acc);
      Y[(int64_t)(2 * level + 2 + ch) * ld + i] = acc * ig;
    }
    return;
  }
  // exact integer products in two passes: the largest exponent sum of each
  // chain, then every product aligned to it (3 guard bits) and summed
  const double* P = Y + (int64_t)(2 * level) * ld;
  const double* R = P + ld;
  const double* Pm = Y + (int64_t)(2 * level - 2) * ld;
  const int nch = doR ? 2 : 1;
  auto xe = [](double v) {
    const int e = (int)(((unsigned)__double2hiint(v) >> 20) & 0x7ffu);
    return e ? e : 1;
  };
  // pass-one loads of the high words only, opaque to the compiler so that
  // pass two loads again instead of holding the values
  auto ldhi = [](const double* p) {
    int h;
    asm volatile("ld.global.nc.b32 %0, [%1];" : "=r"(h) : "l"(reinterpret_cast<const char*>(p) + 4));
    return __hiloint2double(h, 0);
  };
  int Em0 = 0, Em1 = 0;
  auto e1 = [&](int ec, int e0, int e1v) {
    Em0 = max(Em0, ec + e0);
    Em1 = max(Em1, ec + e1v);
  };
  auto tev = [&](int ch, int oy, int ox) { return ev[ch][ly + oy][lx + ox]; };
  e1(xe(ds), tev(0, 0, 0), tev(1, 0, 0));
  e1(xe(ldhi(A.kx + fx)), tev(0, 0, -1), tev(1, 0, -1));
  e1(xe(ldhi(A.kx + fx + 1)), tev(0, 0, 1), tev(1, 0, 1));
  e1(xe(ldhi(A.ky + fy)), tev(0, -1, 0), tev(1, -1, 0));
  e1(xe(ldhi(A.ky + fy + nx)), tev(0, 1, 0), tev(1, 1, 0));
  if (DIM3) {
    e1(xe(ldhi(A.kz + i)), z > 0 ? xe(ldhi(P + i - plane)) : 1, z > 0 && nch > 1 ? xe(ldhi(R + i - plane)) : 1);
    e1(xe(ldhi(A.kz + i + plane)), z < nz - 1 ? xe(ldhi(P + i + plane)) : 1,
       z < nz - 1 && nch > 1 ? xe(ldhi(R + i + plane)) : 1);
  }
  if (mu != 0.0) e1(xe(mu), xe(ldhi(Pm + i)), nch > 1 ? xe(ldhi(Pm + ld + i)) : 1);
  unsigned bad2 = 0;
  long long S0 = 0, S1 = 0;
  auto term = [&](const Limbs& c, const Limbs& y0, const Limbs& y1) {
    S0 += aligned_product(c, y0, Em0);
    if (nch > 1) S1 += aligned_product(c, y1, Em1);
  };
  auto tile = [&](int ch, int oy, int ox) {
    const int2 t = lv[ch][ly + oy][lx + ox];
    return Limbs{t.x, t.y, ev[ch][ly + oy][lx + ox]};
  };
  term(to_limbs(ds, bad2), tile(0, 0, 0), tile(1, 0, 0));
  term(to_limbs<true>(__ldg(A.kx + fx), bad2), tile(0, 0, -1), tile(1, 0, -1));
  term(to_limbs<true>(__ldg(A.kx + fx + 1), bad2), tile(0, 0, 1), tile(1, 0, 1));
  term(to_limbs<true>(__ldg(A.ky + fy), bad2), tile(0, -1, 0), tile(1, -1, 0));
  term(to_limbs<true>(__ldg(A.ky + fy + nx), bad2), tile(0, 1, 0), tile(1, 1, 0));
  if (DIM3) {
    const Limbs zero{0, 0, 1};
    const Limbs cd = to_limbs<true>(__ldg(A.kz + i), bad2);
    term(cd, z > 0 ? to_limbs(__ldg(P + i - plane), bad2) : zero,
         z > 0 && nch > 1 ? to_limbs(__ldg(R + i - plane), bad2) : zero);
    const Limbs cu = to_limbs<true>(__ldg(A.kz + i + plane), bad2);
    term(cu, z < nz - 1 ? to_limbs(__ldg(P + i + plane), bad2) : zero,
         z < nz - 1 && nch > 1 ? to_limbs(__ldg(R + i + plane), bad2) : zero);
  }
  if (mu != 0.0)
    term(to_limbs<true>(mu, bad2), to_limbs(__ldg(Pm + i), bad2),
         nch > 1 ? to_limbs(__ldg(Pm + ld + i), bad2) : Limbs{0, 0, 1});
#pragma unroll 1
  for (int ch = 0; ch < nch; ++ch) {
    bool ok = true;
    double w = to_binary64(ch == 0 ? S0 : S1, ch == 0 ? Em0 : Em1, ok);
    if (!ok || bad2)
      w = mpk_cell_fma<DIM3>(A, Y + (int64_t)(2 * level + ch) * ld, Y + (int64_t)(2 * level - 2 + ch) * ld, i, x,
                             yy, z, ds, mu);
    Y[(int64_t)(2 * level + 2 + ch) * ld + i] = w * ig;
  }
}

// y = A v for a stencil, split between the two units like
// stencil_mpk_hybrid_kernel: of every 16 warps, `fp64_per16` sum their cells
// as the binary64 FMA chain of stencil_apply (the order of the other stencil
// apply kernels, so those cells are their bits), the others as exact integer
// products (exact_sum.cuh) rounded once.  Inf or NaN among a cell's inputs,
// or a sum outside the normal binary64 range, sends the cell to the FMA
// chain.  The SpMV of Algorithm 1 (HSCG) when the comparator is run with the
// same split as the s-step matrix powers.
template <bool DIM3>
__global__ void __launch_bounds__(256, 5) stencil_apply_hybrid_kernel(Operator A, const double* __restrict__ v,
                                                                        double* __restrict__ y,
                                                                        const SolveState* gate, int gmode,
                                                                        int fp64_per16) {
  if (gate_closed(gate, gmode)) return;
  const int nx = A.nx, ny = A.ny, nz = A.nz;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 8;
  const int x = x0 + tx, yy = y0 + ty, z = blockIdx.z;
  __shared__ double sv[10][34];   // v over the tile and its halo (zero outside the domain)
  __shared__ int2 lv[10][34];     // its limbs a, b
  __shared__ int ev[10][34];      // and exponents
  const int64_t zoff = (int64_t)z * ny * nx;
  unsigned bad = 0;
  for (int e = ty * 32 + tx; e < 340; e += 256) {
    const int ly = e / 34, lx = e - ly * 34;
    const int gx = x0 + lx - 1, gy = y0 + ly - 1;
    const bool in = gx >= 0 && gx < nx && gy >= 0 && gy < ny;
    const double val = in ? __ldg(v + zoff + (int64_t)gy * nx + gx) : 0.0;
    sv[ly][lx] = val;
    const Limbs l = to_limbs(val, bad);
    lv[ly][lx] = make_int2(l.a, l.b);
    ev[ly][lx] = l.e;
  }
  const int tile_bad = __syncthreads_or((int)bad);
  if (x >= nx || yy >= ny) return;
  const int64_t plane = (int64_t)nx * ny;
  const int64_t i = zoff + (int64_t)yy * nx + x;
  const int64_t fx = ((int64_t)z * ny + yy) * (nx + 1) + x;
  const int64_t fy = ((int64_t)z * (ny + 1) + yy) * nx + x;
  const double d = __ldg(A.diag + i);
  const int ly = ty + 1, lx = tx + 1;
  const unsigned warp = ((blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * 8u + (unsigned)ty;
  const bool fma_warp = ((warp * (unsigned)fp64_per16) & 15u) < (unsigned)fp64_per16;
  if (fma_warp || tile_bad) {
    double acc = d * sv[ly][lx];
    acc = fma(-__ldg(A.kx + fx), sv[ly][lx - 1], acc);
    acc = fma(-__ldg(A.kx + fx + 1), sv[ly][lx + 1], acc);
    acc = fma(-__ldg(A.ky + fy), sv[ly - 1][lx], acc);
    acc = fma(-__ldg(A.ky + fy + nx), sv[ly + 1][lx], acc);
    if (DIM3) {
      acc = fma(-__ldg(A.kz + i), z > 0 ? __ldg(v + i - plane) : 0.0, acc);
      acc = fma(-__ldg(A.kz + i + plane), z < nz - 1 ? __ldg(v + i + plane) : 0.0, acc);
    }
    y[i] = acc;
    return;
  }
  unsigned bad2 = 0;
  OnlineSum<3> acc;   // at most 7 terms
  auto tile = [&](int oy, int ox) {
    const int2 t = lv[ly + oy][lx + ox];
    return Limbs{t.x, t.y, ev[ly + oy][lx + ox]};
  };
  acc.add(to_limbs(d, bad2), tile(0, 0));
  acc.add(to_limbs<true>(__ldg(A.kx + fx), bad2), tile(0, -1));
  acc.add(to_limbs<true>(__ldg(A.kx + fx + 1), bad2), tile(0, 1));
  acc.add(to_limbs<true>(__ldg(A.ky + fy), bad2), tile(-1, 0));
  acc.add(to_limbs<true>(__ldg(A.ky + fy + nx), bad2), tile(1, 0));
  if (DIM3) {
    const Limbs zero{0, 0, 1};
    acc.add(to_limbs<true>(__ldg(A.kz + i), bad2), z > 0 ? to_limbs(__ldg(v + i - plane), bad2) : zero);
    acc.add(to_limbs<true>(__ldg(A.kz + i + plane), bad2), z < nz - 1 ? to_limbs(__ldg(v + i + plane), bad2) : zero);
  }
  bool ok = true;
  double w = acc.result(ok);
  if (!ok || bad2) w = mpk_cell_fma<DIM3>(A, v, v, i, x, yy, z, d, 0.0);
  y[i] = w;
}

// ---------------------------------------------------- CSR as sliced ELL
// One warp per slice of 32 rows whose lengths differ little (sorted within
// windows of 256 rows): on GB300 a binary64 instruction costs its warp the
// same 64 cycles whether 1 or 32 lanes are active, so thread-per-row CSR pays
// every warp's longest row on all lanes; here each lane loops to its own row
// length (lanes of shorter rows idle for the few steps up to the slice's
// longest row) and the loads of column indices and values are coalesced.
// Each row is summed in its CSR order, so results are the bits of the
// thread-per-row kernels.
template <int MODE>  // 0: y = A v; 1: y = b - A v
__global__ void __launch_bounds__(kOpThreads) sell_apply_kernel(Operator A, const double* __restrict__ v,
                                                                const double* __restrict__ b,
                                                                double* __restrict__ y, const SolveState* gate,
                                                                int gmode) {
  if (gate_closed(gate, gmode)) return;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t s = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); s < A.nslices; s += warps) {
    const int r = __ldg(A.s_row + s * kSliceRows + lane);
    if (r < 0) continue;
    const int len = (int)(__ldg(A.rowptr + r + 1) - __ldg(A.rowptr + r));
    const int64_t base = __ldg(A.s_off + s) + lane;
    double acc = 0.0;
    for (int j = 0; j < len; ++j) {
      const int64_t k = base + (int64_t)j * kSliceRows;
      acc = fma(__ldg(A.s_val + k), __ldg(v + __ldg(A.s_col + k)), acc);
    }
    y[r] = MODE == 0 ? acc : b[r] - acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(kOpThreads) sell_mpk_kernel(Operator A, T* __restrict__ Y, int64_t ld, int level,
                                                              const SolveState* __restrict__ st, int sbar_fixed,
                                                              LevelCoef coef) {
  int sbar = sbar_fixed;
  if (sbar <= 0) {
    if (st->done) return;
    sbar = st->sbar;
  }
  const bool doP = level < sbar;
  const bool doR = level + 1 < sbar;
  if (!doP) return;
  const double theta = coef.theta[level];
  const double ig = coef.inv_gamma[level];
  const double mu = level >= 1 ? coef.mu[level - 1] : 0.0;
  const T* Pl = Y + (int64_t)(2 * level) * ld;
  const T* Rl = Y + (int64_t)(2 * level + 1) * ld;
  const T* Pm = level >= 1 ? Y + (int64_t)(2 * level - 2) * ld : nullptr;
  const T* Rm = level >= 1 ? Y + (int64_t)(2 * level - 1) * ld : nullptr;
  T* Pn = Y + (int64_t)(2 * level + 2) * ld;
  T* Rn = Y + (int64_t)(2 * level + 3) * ld;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t s = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); s < A.nslices; s += warps) {
    const int r = __ldg(A.s_row + s * kSliceRows + lane);
    if (r < 0) continue;
    const int len = (int)(__ldg(A.rowptr + r + 1) - __ldg(A.rowptr + r));
    const int64_t base = __ldg(A.s_off + s) + lane;
    double ap = 0.0, ar = 0.0;
    if (doR) {
      for (int j = 0; j < len; ++j) {
        const int64_t k = base + (int64_t)j * kSliceRows;
        const double a = __ldg(A.s_val + k);
        const int c = __ldg(A.s_col + k);
        ap = fma(a, ld_val(Pl + c), ap);
        ar = fma(a, ld_val(Rl + c), ar);
      }
    } else {
      for (int j = 0; j < len; ++j) {
        const int64_t k = base + (int64_t)j * kSliceRows;
        ap = fma(__ldg(A.s_val + k), ld_val(Pl + __ldg(A.s_col + k)), ap);
      }
    }
    double wp = fma(-theta, ld_val(Pl + r), ap);
    if (mu != 0.0) wp = fma(-mu, ld_val(Pm + r), wp);
    Pn[r] = (T)(wp * ig);
    if (doR) {
      double wr = fma(-theta, ld_val(Rl + r), ar);
      if (mu != 0.0) wr = fma(-mu, ld_val(Rm + r), wr);
      Rn[r] = (T)(wr * ig);
    }
  }
}

// ------------------------------------------------- 3D stencil, z-marching
// The 3D SpMV and residual (the HSCG comparator's operator and the true
// residual) march along z: a block covers a 32 x 8 tile of (x, y) columns and
// a chunk of kZChunk planes; each thread keeps its column's values at z-1, z,
// z+1 (and the face coefficient below z) in registers, so per cell it loads
// the value above and the four lateral neighbours (L1 hits), and all indices
// advance by a constant per plane (no division).  The sum is formed in the
// same order as stencil_apply, so results are the same bits as the
// cell-parallel kernel.  (For the two-chain matrix-powers level the same
// scheme needs ~60 registers per thread and measured slower than the
// cell-parallel kernel, which it therefore keeps.)
constexpr int kZTx = 32, kZTy = 8, kZChunk = 4;

__host__ inline dim3 cell_grid3(const Operator& A) {
  return dim3((unsigned)((A.nx + 31) / 32), (unsigned)((A.ny + 7) / 8), (unsigned)A.nz);
}

__host__ inline int sell_grid(const Operator& A) {
  const int64_t warps_per_block = kOpThreads / 32;
  int64_t g = (A.nslices + warps_per_block - 1) / warps_per_block;
  if (g > 152 * 16) g = 152 * 16;
  return g < 1 ? 1 : (int)g;
}

__host__ inline dim3 zmarch_grid(const Operator& A) {
  return dim3((unsigned)((A.nx + kZTx - 1) / kZTx), (unsigned)((A.ny + kZTy - 1) / kZTy),
              (unsigned)((A.nz + kZChunk - 1) / kZChunk));
}

struct ZCol {  // per-thread column walk
  int x, y, z0, z1;
  int64_t i, fx, fy;
};

__device__ __forceinline__ bool zcol_begin(const Operator& A, ZCol& c) {
  c.x = blockIdx.x * kZTx + threadIdx.x;
  c.y = blockIdx.y * kZTy + threadIdx.y;
  c.z0 = blockIdx.z * kZChunk;
  if (c.x >= A.nx || c.y >= A.ny || c.z0 >= A.nz) return false;
  c.z1 = c.z0 + kZChunk < A.nz ? c.z0 + kZChunk : A.nz;
  c.i = ((int64_t)c.z0 * A.ny + c.y) * A.nx + c.x;
  c.fx = ((int64_t)c.z0 * A.ny + c.y) * (A.nx + 1) + c.x;
  c.fy = ((int64_t)c.z0 * (A.ny + 1) + c.y) * A.nx + c.x;
  return true;
}

// (A - shift I) v at the current cell from its column registers vd, vc, vu.
template <typename T>
__device__ __forceinline__ double zapply(const Operator& A, const T* __restrict__ v, const ZCol& c, double dshift,
                                         double kw, double ke, double ks, double kn, double kd, double ku,
                                         double vd, double vc, double vu) {
  const double vw = c.x > 0 ? ld_val(v + c.i - 1) : 0.0;
  const double ve = c.x < A.nx - 1 ? ld_val(v + c.i + 1) : 0.0;
  const double vs = c.y > 0 ? ld_val(v + c.i - A.nx) : 0.0;
  const double vn = c.y < A.ny - 1 ? ld_val(v + c.i + A.nx) : 0.0;
  double acc = dshift * vc;
  acc = fma(-kw, vw, acc);
  acc = fma(-ke, ve, acc);
  acc = fma(-ks, vs, acc);
  acc = fma(-kn, vn, acc);
  acc = fma(-kd, vd, acc);
  acc = fma(-ku, vu, acc);
  return acc;
}

// y = A v (mode 0) or r = b - A v (mode 1) for a 3D stencil, z-marching.
template <int MODE>
__global__ void __launch_bounds__(kZTx * kZTy, 6) stencil3d_apply_kernel(Operator A, const double* __restrict__ v,
                                                                      const double* __restrict__ b,
                                                                      double* __restrict__ y,
                                                                      const SolveState* gate, int gmode) {
  if (gate_closed(gate, gmode)) return;
  ZCol c;
  if (!zcol_begin(A, c)) return;
  const int64_t plane = (int64_t)A.nx * A.ny;
  const int64_t dfx = (int64_t)A.ny * (A.nx + 1), dfy = (int64_t)(A.ny + 1) * A.nx;
  double vd = c.z0 > 0 ? __ldg(v + c.i - plane) : 0.0, vc = __ldg(v + c.i);
  double kd = __ldg(A.kz + c.i);
#pragma unroll 2
  for (int z = c.z0; z < c.z1; ++z) {
    const double vu = z < A.nz - 1 ? __ldg(v + c.i + plane) : 0.0;
    const double ku = __ldg(A.kz + c.i + plane);
    const double av = zapply(A, v, c, __ldg(A.diag + c.i), __ldg(A.kx + c.fx), __ldg(A.kx + c.fx + 1),
                             __ldg(A.ky + c.fy), __ldg(A.ky + c.fy + A.nx), kd, ku, vd, vc, vu);
    y[c.i] = MODE == 0 ? av : b[c.i] - av;
    vd = vc;
    vc = vu;
    kd = ku;
    c.i += plane;
    c.fx += dfx;
    c.fy += dfy;
  }
}



__global__ void __launch_bounds__(kOpThreads) stencil_diag_kernel(Operator A, double* __restrict__ diag) {
  const int64_t n = A.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % A.nx);
    const int64_t t = i / A.nx;
    const int y = (int)(t % A.ny);
    const int z = (int)(t / A.ny);
    const int64_t fx = ((int64_t)z * A.ny + y) * (A.nx + 1) + x;
    const int64_t fy = ((int64_t)z * (A.ny + 1) + y) * A.nx + x;
    double d = A.kx[fx] + A.kx[fx + 1] + A.ky[fy] + A.ky[fy + A.nx];
    if (A.dim == 3) d += A.kz[i] + A.kz[i + (int64_t)A.nx * A.ny];
    diag[i] = d;
  }
}


// Both chains of one stencil cell of a matrix-powers level as exact integer
// products (exact_sum.cuh), every operand split from global memory (the
// batched level has no tiles): (A - theta I) v - mu v' for v = P_l and R_l
// (R only with doR), each sum rounded once.  Returns false when an input is
// Inf or NaN or a sum leaves the normal binary64 range; the caller then takes
// the FMA chain.
template <bool DIM3>
__device__ __forceinline__ bool mpk_cell_int(const Operator& A, const double* __restrict__ Pl,
                                             const double* __restrict__ Rl, const double* __restrict__ Pm,
                                             const double* __restrict__ Rm, int64_t i, int x, int yy, int z,
                                             double ds, double mu, bool doR, double& wp, double& wr) {
  const int nx = A.nx, ny = A.ny, nz = A.nz;
  const int64_t plane = (int64_t)nx * ny;
  const int64_t fx = ((int64_t)z * ny + yy) * (nx + 1) + x;
  const int64_t fy = ((int64_t)z * (ny + 1) + yy) * nx + x;
  unsigned bad = 0;
  OnlineSum<3> a0, a1;
  const Limbs zero{0, 0, 1};
  auto term = [&](const Limbs& c, int64_t j, bool in) {
    a0.add(c, in ? to_limbs(__ldg(Pl + j), bad) : zero);
    if (doR) a1.add(c, in ? to_limbs(__ldg(Rl + j), bad) : zero);
  };
  term(to_limbs(ds, bad), i, true);
  term(to_limbs<true>(__ldg(A.kx + fx), bad), i - 1, x > 0);
  term(to_limbs<true>(__ldg(A.kx + fx + 1), bad), i + 1, x < nx - 1);
  term(to_limbs<true>(__ldg(A.ky + fy), bad), i - nx, yy > 0);
  term(to_limbs<true>(__ldg(A.ky + fy + nx), bad), i + nx, yy < ny - 1);
  if (DIM3) {
    term(to_limbs<true>(__ldg(A.kz + i), bad), i - plane, z > 0);
    term(to_limbs<true>(__ldg(A.kz + i + plane), bad), i + plane, z < nz - 1);
  }
  if (mu != 0.0) {
    const Limbs cm = to_limbs<true>(mu, bad);
    a0.add(cm, to_limbs(__ldg(Pm + i), bad));
    if (doR) a1.add(cm, to_limbs(__ldg(Rm + i), bad));
  }
  bool ok = true;
  wp = a0.result(ok);
  wr = doR ? a1.result(ok) : 0.0;
  return ok && !bad;
}

// Batched matrix-powers level: every chunk belongs to one pair, whose state
// gives its own s-bar and recurrence coefficients (eq. rho); pairs that are
// done or whose block is shorter than this level skip their chunks.  Stencil
// pairs split their warps like stencil_mpk_hybrid_kernel: of every 16 groups
// of 32 rows, fp64_per16 take the binary64 FMA chain and the others exact
// integer products (mpk_cell_int), by the group's position alone.
__global__ void __launch_bounds__(kOpThreads, 4) batch_mpk_kernel(BatchView v, double* __restrict__ Y, int64_t LD,
                                                               int level, int fp64_per16) {
  for (int c = blockIdx.x; c < v.nchunks; c += gridDim.x) {
    const int j = v.chunk_pair[c];
    const BatchPair& bp = v.pairs[j];
    const SolveState* st = v.states + j;
    if (st->done) continue;
    const int sbar = st->sbar;
    if (level >= sbar) continue;
    const bool doR = level + 1 < sbar;
    const double theta = st->theta[level];
    const double ig = st->inv_gamma[level];
    const double mu = level >= 1 ? st->mu[level - 1] : 0.0;
    const Operator& A = bp.op;
    double* base = Y + bp.off;
    const double* Pl = base + (int64_t)(2 * level) * LD;
    const double* Rl = base + (int64_t)(2 * level + 1) * LD;
    const double* Pm = level >= 1 ? base + (int64_t)(2 * level - 2) * LD : nullptr;
    const double* Rm = level >= 1 ? base + (int64_t)(2 * level - 1) * LD : nullptr;
    double* Pn = base + (int64_t)(2 * level + 2) * LD;
    double* Rn = base + (int64_t)(2 * level + 3) * LD;
    const int64_t r0 = (int64_t)(c - bp.chunk0) * v.chunk_rows;
    int64_t r1 = r0 + v.chunk_rows;
    if (r1 > bp.n) r1 = bp.n;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      double wp, wr = 0.0;
      // the row group of this warp (i - r0 is a multiple of 32 on lane 0)
      const unsigned grp = (unsigned)c * 64u + (unsigned)((i - r0) >> 5);
      if (A.kind == 1 && ((grp * (unsigned)fp64_per16) & 15u) >= (unsigned)fp64_per16) {
        const int x = (int)(i % A.nx);
        const int64_t t = i / A.nx;
        const int yy = (int)(t % A.ny);
        const int z = (int)(t / A.ny);
        const double ds = __ldg(A.diag + i) - theta;
        const bool ok = A.dim == 3 ? mpk_cell_int<true>(A, Pl, Rl, Pm, Rm, i, x, yy, z, ds, mu, doR, wp, wr)
                                   : mpk_cell_int<false>(A, Pl, Rl, Pm, Rm, i, x, yy, z, ds, mu, doR, wp, wr);
        if (ok) {
          Pn[i] = wp * ig;
          if (doR) Rn[i] = wr * ig;
          continue;
        }
      }
      if (A.kind == 1) {
        const int x = (int)(i % A.nx);
        const int64_t t = i / A.nx;
        const int yy = (int)(t % A.ny);
        const int z = (int)(t / A.ny);
        const double ds = __ldg(A.diag + i) - theta;
        if (A.dim == 3) {
          wp = stencil_apply<true>(A, Pl, i, x, yy, z, ds);
          if (doR) wr = stencil_apply<true>(A, Rl, i, x, yy, z, ds);
        } else {
          wp = stencil_apply<false>(A, Pl, i, x, yy, z, ds);
          if (doR) wr = stencil_apply<false>(A, Rl, i, x, yy, z, ds);
        }
      } else {
        const int64_t kb = __ldg(A.rowptr + i), ke = __ldg(A.rowptr + i + 1);
        double ap = 0.0, ar = 0.0;
        for (int64_t k = kb; k < ke; ++k) {
          const double a = __ldg(A.val + k);
          const int cc = __ldg(A.col + k);
          ap = fma(a, __ldg(Pl + cc), ap);
          if (doR) ar = fma(a, __ldg(Rl + cc), ar);
        }
        wp = fma(-theta, __ldg(Pl + i), ap);
        wr = fma(-theta, __ldg(Rl + i), ar);
      }
      if (mu != 0.0) wp = fma(-mu, __ldg(Pm + i), wp);
      Pn[i] = wp * ig;
      if (doR) {
        if (mu != 0.0) wr = fma(-mu, __ldg(Rm + i), wr);
        Rn[i] = wr * ig;
      }
    }
  }
}

}  // namespace

cudaError_t launch_batch_mpk(const BatchView& v, double* Y, int64_t LD, int level, cudaStream_t st,
                             int fp64_per16) {
  int g = v.nchunks < 152 * 8 ? v.nchunks : 152 * 8;
  const int f16 = fp64_per16 < 0 ? kBatchMpkFp64Per16 : fp64_per16;
  batch_mpk_kernel<<<g < 1 ? 1 : g, kOpThreads, 0, st>>>(v, Y, LD, level, f16);
  return cudaGetLastError();
}

cudaError_t launch_stencil_diag(const Operator& A, double* diag, cudaStream_t st) {
  stencil_diag_kernel<<<grid_for(A.n, 4), kOpThreads, 0, st>>>(A, diag);
  return cudaGetLastError();
}

cudaError_t launch_spmv(const Operator& A, const double* v, double* y, cudaStream_t st, const SolveState* gate,
                        int gmode) {
  int g = grid_for(A.n, 4);
  if (A.kind == 0) sell_apply_kernel<0><<<sell_grid(A), kOpThreads, 0, st>>>(A, v, nullptr, y, gate, gmode);
  else if (A.dim == 3)
    stencil3d_apply_kernel<0><<<zmarch_grid(A), dim3(kZTx, kZTy), 0, st>>>(A, v, nullptr, y, gate, gmode);
  else stencil_spmv_kernel<false><<<g, kOpThreads, 0, st>>>(A, v, y, gate, gmode);
  return cudaGetLastError();
}

bool spmv_split_supported(const Operator& A) {
  return A.kind == 1 && A.nz <= 65535 && (A.ny + 7) / 8 <= 65535;
}

cudaError_t launch_spmv_split(const Operator& A, const double* v, double* y, cudaStream_t st, const SolveState* gate,
                              int gmode, int fp64_per16) {
  const int f16 = fp64_per16 < 0 ? kMpkFp64Per16 : fp64_per16;
  if (f16 >= 16 || !spmv_split_supported(A)) return launch_spmv(A, v, y, st, gate, gmode);
  if (A.dim == 3)
    stencil_apply_hybrid_kernel<true><<<cell_grid3(A), dim3(32, 8), 0, st>>>(A, v, y, gate, gmode, f16);
  else
    stencil_apply_hybrid_kernel<false><<<cell_grid3(A), dim3(32, 8), 0, st>>>(A, v, y, gate, gmode, f16);
  return cudaGetLastError();
}

cudaError_t launch_residual(const Operator& A, const double* b, const double* x, double* r, cudaStream_t st,
                            const SolveState* gate, int gmode) {
  int g = grid_for(A.n, 4);
  if (A.kind == 0) sell_apply_kernel<1><<<sell_grid(A), kOpThreads, 0, st>>>(A, x, b, r, gate, gmode);
  else if (A.dim == 3)
    stencil3d_apply_kernel<1><<<zmarch_grid(A), dim3(kZTx, kZTy), 0, st>>>(A, x, b, r, gate, gmode);
  else stencil_residual_kernel<false><<<g, kOpThreads, 0, st>>>(A, b, x, r, gate, gmode);
  return cudaGetLastError();
}

cudaError_t launch_mpk_level(const Operator& A, void* Y, int64_t ld, int level, const SolveState* state,
                             int sbar_fixed, LevelCoef coef, bool y32, cudaStream_t st, int fp64_per16) {
  int g = grid_for(A.n, 4);
  if (y32) {
    float* Yf = static_cast<float*>(Y);
    if (A.kind == 0)
      sell_mpk_kernel<float><<<sell_grid(A), kOpThreads, 0, st>>>(A, Yf, ld, level, state, sbar_fixed, coef);
    else if (A.nz > 65535)  // beyond the grid's z extent: grid-stride kernel
      stencil_mpk_kernel<true, float><<<g, kOpThreads, 0, st>>>(A, Yf, ld, level, state, sbar_fixed, coef);
    else if (A.dim == 3)
      stencil_mpk_grid_kernel<true, float><<<cell_grid3(A), dim3(32, 8), 0, st>>>(A, Yf, ld, level, state,
                                                                                 sbar_fixed, coef);
    else
      stencil_mpk_grid_kernel<false, float><<<cell_grid3(A), dim3(32, 8), 0, st>>>(A, Yf, ld, level, state,
                                                                                  sbar_fixed, coef);
  } else {
    double* Yd = static_cast<double*>(Y);
    const int f16 = fp64_per16 < 0 ? kMpkFp64Per16 : fp64_per16;
    if (A.kind == 0)
      sell_mpk_kernel<double><<<sell_grid(A), kOpThreads, 0, st>>>(A, Yd, ld, level, state, sbar_fixed, coef);
    else if (A.nz > 65535)  // beyond the grid's z extent: grid-stride kernel
      stencil_mpk_kernel<true, double><<<g, kOpThreads, 0, st>>>(A, Yd, ld, level, state, sbar_fixed, coef);
    else if (f16 >= 16 && A.dim == 3)
      stencil_mpk_grid_kernel<true, double><<<cell_grid3(A), dim3(32, 8), 0, st>>>(A, Yd, ld, level, state,
                                                                                  sbar_fixed, coef);
    else if (f16 >= 16)
      stencil_mpk_grid_kernel<false, double><<<cell_grid3(A), dim3(32, 8), 0, st>>>(A, Yd, ld, level, state,
                                                                                   sbar_fixed, coef);
    else if (A.dim == 3)
      stencil_mpk_hybrid_kernel<true><<<cell_grid3(A), dim3(32, 8), 0, st>>>(A, Yd, ld, level, state, sbar_fixed,
                                                                            coef, f16);
    else
      stencil_mpk_hybrid_kernel<false><<<cell_grid3(A), dim3(32, 8), 0, st>>>(A, Yd, ld, level, state, sbar_fixed,
                                                                             coef, f16);
  }
  return cudaGetLastError();
}

}  // namespace sscg
