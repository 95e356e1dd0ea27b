// Device-side control of Algorithm 5 (Carson 2019, Sections 3-4): the basis
// condition estimates, the choice of s-tilde, the coordinate-space CG steps,
// the Meurant-Tichy Ritz estimates (Algorithms 3-4), the error/residual ratio
// c (eq. xiupd), the break test (eq. newcondy) and the next basis parameters
// (eqs. newtbasis, chebbasis).  Everything is O(s^3) scalar work on tiny
// matrices, done by single blocks so the host never waits inside a solve.
//
// This file is compiled with FMA contraction disabled: its scalar formulas are
// evaluated operation by operation in the order they are written, so equal
// inputs give equal decisions on any IEEE binary64 implementation.  Fused
// multiply-adds appear only where written out (fma()): in the small matrix
// kernels (Householder, Sturm sequences, G times a vector), whose summation
// order differs from any reference anyway.
#include <math.h>

#include "sscg_internal.cuh"

namespace sscg {

namespace {

constexpr int kKappaThreads = 128;
constexpr int kControlThreads = 128;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ kappa
// On GB300 every binary64 instruction occupies its SM sub-partition's FP64
// unit for about 64 cycles per warp, whether 1 or 32 lanes are active, so the
// latency of these one-block kernels is the count of binary64 instructions on
// each warp's path.  The kappa step therefore keeps sign and zero tests in
// integer arithmetic, brackets each extreme eigenvalue with a cheap binary32
// Sturm multisection first, and spends binary64 Sturm sequences only on the
// last ~35 bits.

// Number of eigenvalues of the symmetric tridiagonal (d, e2 = squared
// off-diagonals) that are smaller than x: sign changes of the Sturm sequence
// p_0 = 1, p_i = (d_{i-1} - x) p_{i-1} - e2_{i-2} p_{i-2}.  Division free, three
// binary64 operations per step.  The guards stay off the binary64 unit: one
// integer test of q's exponent (outside [2^-600, 2^600], or zero) leads to a
// warp-uniform rare branch that replaces an exact zero by a tiny value of the
// opposite sign of p_{i-1} and rescales the sequence by a power of two; sign
// changes are counted on the sign bits.  Called by whole warps.
__device__ __forceinline__ int sturm_count(const double* d, const double* e2, int n, double x) {
  double pm = 1.0;
  double p = d[0] - x;
  long long pb = __double_as_longlong(p);
  if ((pb << 1) == 0) {
    p = -1e-300;
    pb = __double_as_longlong(p);
  }
  int cnt = (int)((unsigned long long)pb >> 63);
  for (int i = 1; i < n; ++i) {
    double q = fma(d[i] - x, p, -(e2[i - 1] * pm));
    long long qb = __double_as_longlong(q);
    const unsigned ex = (unsigned)(qb >> 52) & 0x7ffu;
    const bool odd = ex - 423u > 1200u;  // biased exponent outside [423, 1623]
    if (__any_sync(0xffffffffu, odd)) {
      if (odd) {
        if ((qb << 1) == 0) q = pb < 0 ? 1e-300 : -1e-300;
        const unsigned eq = (unsigned)(__double_as_longlong(q) >> 52) & 0x7ffu;
        const double sc = eq > 1023u ? 0x1p-600 : 0x1p600;
        q *= sc;
        p *= sc;
        qb = __double_as_longlong(q);
      }
    }
    cnt += (int)((unsigned long long)(qb ^ pb) >> 63);
    pm = p;
    p = q;
    pb = qb;
  }
  return cnt;
}

// The same count in binary32 with the ratio form q_i = (d_i - x) - e2_{i-1} / q_{i-1}
// (negative q_i counted; |q_i| below pivmin replaced by -pivmin).  Used only to
// bracket an eigenvalue; the bracket is checked in binary64 before use.
__device__ __forceinline__ int sturm_count32(const float* d, const float* e2, int n, float x) {
  const float pivmin = 1e-30f;
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int cnt = q < 0.f ? 1 : 0;
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += q < 0.f ? 1 : 0;
  }
  return cnt;
}

// binary32 multisection by one warp: 32 points per round in (lo, hi); the
// result brackets the point where count first reaches `target`.
__device__ void warp_bracket32(const float* d, const float* e2, int n, float lo, float hi, int target, int rounds,
                               float* out_lo, float* out_hi) {
  const int lane = threadIdx.x & 31;
  for (int round = 0; round < rounds; ++round) {
    const float step = (hi - lo) * (1.0f / 33.0f);
    const float x = lo + step * (float)(lane + 1);
    const unsigned ball = __ballot_sync(0xffffffffu, sturm_count32(d, e2, n, x) >= target);
    const int f = ball ? __ffs(ball) - 1 : 32;
    const float xf = __shfl_sync(0xffffffffu, x, f & 31);
    const float xfm = __shfl_sync(0xffffffffu, x, (f - 1) & 31);
    const float nlo = f == 0 ? lo : xfm;
    const float nhi = f == 32 ? hi : xf;
    lo = nlo;
    hi = nhi;
  }
  *out_lo = lo;
  *out_hi = hi;
}

// One block per l = 1..sbar: Householder tridiagonalisation of the leading
// (2l+1) block of G, then its extreme eigenvalues by multisection;
// kappa_l = sqrt(lmax/lmin) (Section 3: kappa(Y_l) ~ sqrt(kappa(G_l))).
// Four warps: the Householder steps use all of them; in the multisection warps
// 0-1 find lambda_min and warps 2-3 lambda_max (64 binary64 points per round).
__device__ void kappa_body(const double* __restrict__ G, int ldg, int l, double kappa_cut,
                           double* __restrict__ kap, double* __restrict__ lmin_out, double* __restrict__ lmax_out) {
  static_assert(kKappaThreads == 128, "four warps");
  const int n = 2 * l + 1;
  const int t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5;

  __shared__ double A[kMaxCols][kMaxCols + 1];
  __shared__ double v[kMaxCols], w[kMaxCols], spart[3][32];
  __shared__ double dd[kMaxCols], ee[kMaxCols], e2[kMaxCols];
  __shared__ float df[kMaxCols], ef2[kMaxCols];
  __shared__ double sh[2];
  __shared__ int sh_skip;
  __shared__ unsigned masks[2][4];
  constexpr int kTri = 32 * 33 / 2;  // lower triangle of the largest trailing block
  __shared__ unsigned char tri_i[kTri], tri_j[kTri];

  int nonfinite = 0;
  for (int e = t; e < n * n; e += kKappaThreads) {
    const int i = e / n, j = e - (e / n) * n;
    const double g = G[i * ldg + j];
    nonfinite |= ((__double_as_longlong(g) >> 52) & 0x7ff) == 0x7ff;
    A[i][j] = g;
  }
  // a block with a non-finite entry (a basis column that overflowed) has no
  // eigenvalues: kappa_l = inf, so s-tilde stays below that column
  if (__syncthreads_or(nonfinite)) {
    if (t == 0) {
      lmin_out[l] = NAN;
      lmax_out[l] = NAN;
      kap[l] = INFINITY;
    }
    return;
  }
  if (t < 32) {  // entry e = i (i + 1) / 2 + j of the lower triangle, j <= i; thread t fills row t
    const int base = t * (t + 1) / 2;
    for (int j = 0; j <= t; ++j) {
      tri_i[base + j] = (unsigned char)t;
      tri_j[base + j] = (unsigned char)j;
    }
  }
  __syncthreads();

  // Householder step k with x = A(k+1:n-1, k), v = x - alpha e_0:
  //   warp 0:    rest = |x(1:)|^2, alpha = -sign(x_0) |x|, tau = 2 / (v^T v)
  //   warps 1-3: s = A_sub x, concurrently (3 threads per row)
  //   warp 0:    p = tau (s - alpha A_sub e_0) = tau A_sub v, K = tau p^T v / 2, w = p - K v
  //   all:       A_sub -= v w^T + w v^T on the lower triangle (balanced), mirrored
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;  // trailing block rows k+1..n-1, m <= 32
    if (warp == 0) {
      const double xi = lane < m ? A[k + 1 + lane][k] : 0.0;
      const double rest = warp_sum(lane >= 1 ? xi * xi : 0.0);
      if (lane == 0) {
        if (__double_as_longlong(rest) == 0) {  // already tridiagonal in this column
          sh_skip = 1;
          dd[k] = A[k][k];
          ee[k] = xi;
        } else {
          const long long xb = __double_as_longlong(xi);
          const double sig2 = fma(xi, xi, rest);
          const double r = sqrt(sig2);
          const double alpha = (xb >= 0 || (xb << 1) == 0) ? -r : r;
          const double v0 = xi - alpha;
          sh_skip = 0;
          sh[0] = 2.0 / (rest + v0 * v0);  // tau
          sh[1] = alpha;
          v[0] = v0;
        }
      } else if (lane < m) {
        v[lane] = xi;
      }
    } else {
      const int u = t - 32, i = u / 3, slot = u - 3 * i;
      if (i < m) {
        double sacc = 0.0;
        for (int j = slot; j < m; j += 3) sacc = fma(A[k + 1 + i][k + 1 + j], A[k + 1 + j][k], sacc);
        spart[slot][i] = sacc;
      }
    }
    __syncthreads();
    if (sh_skip) {
      __syncthreads();  // the next step's warp 0 rewrites what every thread just read
      continue;
    }
    if (warp == 0) {
      const double tau = sh[0], alpha = sh[1];
      double pl = 0.0, vl = 0.0;
      if (lane < m) {
        const double sl = (spart[0][lane] + spart[1][lane]) + spart[2][lane];
        pl = tau * fma(-alpha, A[k + 1 + lane][k + 1], sl);
        vl = v[lane];
      }
      const double pv = warp_sum(pl * vl);
      const double K = 0.5 * tau * pv;
      if (lane < m) w[lane] = fma(-K, vl, pl);
    }
    __syncthreads();
    for (int e = t; e < m * (m + 1) / 2; e += kKappaThreads) {
      const int i = tri_i[e], j = tri_j[e];
      const double val = fma(-v[i], w[j], fma(-w[i], v[j], A[k + 1 + i][k + 1 + j]));
      A[k + 1 + i][k + 1 + j] = val;
      A[k + 1 + j][k + 1 + i] = val;
    }
    if (t == 0) {
      dd[k] = A[k][k];
      ee[k] = sh[1];
    }
    __syncthreads();
  }
  if (t == 0) {
    dd[n - 2] = A[n - 2][n - 2];
    dd[n - 1] = A[n - 1][n - 1];
    ee[n - 2] = A[n - 1][n - 2];
  }
  __syncthreads();

  // Gershgorin interval (warp 0, lanes over rows), then normalisation by a
  // power of two near its largest magnitude (exact scaling)
  __shared__ double glo, ghi;
  __shared__ int sc_exp;
  if (warp == 0) {
    double lo = 1e308, hi = -1e308;
    for (int i = lane; i < n; i += 32) {
      const double r = (i > 0 ? fabs(ee[i - 1]) : 0.0) + (i < n - 1 ? fabs(ee[i]) : 0.0);
      lo = fmin(lo, dd[i] - r);
      hi = fmax(hi, dd[i] + r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      const double mag = fmax(fabs(lo), fabs(hi));
      const int ex = mag > 0.0 ? (int)((__double_as_longlong(mag) >> 52) & 0x7ff) - 1023 : 0;
      sc_exp = ex;
      const double sc = ldexp(1.0, -ex);
      glo = lo * sc - 0x1p-50;
      ghi = hi * sc + 0x1p-50;
    }
  }
  __syncthreads();
  {
    const double sc = ldexp(1.0, -sc_exp);
    if (t < n) {
      dd[t] = dd[t] * sc;
      df[t] = (float)dd[t];
      if (t < n - 1) {
        const double es = ee[t] * sc;
        e2[t] = es * es;
        ef2[t] = (float)e2[t];
      }
    }
  }
  __syncthreads();

  // warps 0-1: lambda_min (count reaches 1); warps 2-3: lambda_max (count reaches n)
  const int pair = warp >> 1;
  const int target = pair == 0 ? 1 : n;
  const double g_lo = glo, g_hi = ghi;
  __shared__ double br[2][2];
  if ((warp & 1) == 0) {  // binary32 bracket by the pair's first warp
    float blo, bhi;
    warp_bracket32(df, ef2, n, (float)g_lo, (float)g_hi, target, 4, &blo, &bhi);
    if (lane == 0) {
      br[pair][0] = fmax(g_lo, (double)blo - 0x1p-16);
      br[pair][1] = fmin(g_hi, (double)bhi + 0x1p-16);
    }
  }
  __syncthreads();
  double lo = br[pair][0], hi = br[pair][1];
  const int k64 = lane + 32 * (warp & 1);  // this thread's point, 0..63
  bool done = false;
  constexpr int kRounds = 10;
  for (int round = 0; round < kRounds; ++round) {
    // round 0: points lo + (hi - lo) k / 63 including both ends (checks the
    // binary32 bracket); later rounds: interior points lo + (hi - lo)(k + 1) / 65
    const double step = round == 0 ? (hi - lo) * (1.0 / 63.0) : (hi - lo) * (1.0 / 65.0);
    const double x = lo + step * (double)(round == 0 ? k64 : k64 + 1);
    if (!done) {
      const unsigned ball = __ballot_sync(0xffffffffu, sturm_count(dd, e2, n, x) >= target);
      if (lane == 0) masks[round & 1][warp] = ball;
    }
    __syncthreads();
    if (!done) {
      const unsigned long long M = (unsigned long long)masks[round & 1][2 * pair] |
                                   ((unsigned long long)masks[round & 1][2 * pair + 1] << 32);
      if (round == 0) {
        if ((M & 1ull) || !(M >> 63)) {  // the bracket does not hold: start from Gershgorin
          lo = g_lo;
          hi = g_hi;
        } else {
          const int f = __ffsll((long long)M) - 1;  // >= 1
          const double nlo = lo + step * (double)(f - 1);
          const double nhi = lo + step * (double)f;
          lo = nlo;
          hi = nhi;
        }
      } else {
        const int f = M ? __ffsll((long long)M) - 1 : 64;
        const double nlo = f == 0 ? lo : lo + step * (double)f;
        const double nhi = f == 64 ? hi : lo + step * (double)(f + 1);
        lo = nlo;
        hi = nhi;
      }
      // 2^-56 absolute on the normalised matrix (small lambda_min keeps its
      // relative accuracy), or 4 ulps of the larger endpoint
      done = hi - lo <= fmax(0x1p-56, 0x1p-50 * fmax(fabs(lo), fabs(hi)));
    }
  }
  __shared__ double ev[2];
  if ((warp & 1) == 0 && lane == 0) ev[pair] = 0.5 * (lo + hi);
  __syncthreads();
  if (t == 0) {
    const double lmn = ldexp(ev[0], sc_exp), lmx = ldexp(ev[1], sc_exp);
    lmin_out[l] = lmn;
    lmax_out[l] = lmx;
    kap[l] = (!(lmx > 0.0) || lmn <= kappa_cut * lmx) ? INFINITY : sqrt(lmx / lmn);
  }
}

__global__ void __launch_bounds__(kKappaThreads) kappa_kernel(const double* __restrict__ G, int ldg,
                                                              const SolveState* __restrict__ st, int sbar_fixed,
                                                              double kappa_cut, double* __restrict__ kap,
                                                              double* __restrict__ lmin_out,
                                                              double* __restrict__ lmax_out) {
  int sbar = sbar_fixed;
  if (sbar <= 0) {
    if (st->done) return;
    sbar = st->sbar;
    kappa_cut = st->kappa_cut;
  }
  const int l = blockIdx.x + 1;
  if (l > sbar) return;
  kappa_body(G, ldg, l, kappa_cut, kap, lmin_out, lmax_out);
}

// --------------------------------------------------------------- control
// (B p)_i for the interleaved B of eq. (B): A P_l = gamma_l P_{l+1} + theta_l P_l
// + mu_{l-1} P_{l-1} for l < s (P chain) and l < s-1 (R chain); the last P and
// the last R column of B are zero.
__device__ __forceinline__ double b_times(const double* pc, int i, int s, const double* th, const double* ga,
                                          const double* mu) {
  const int chain = i & 1;           // 0: P, 1: R
  const int l = i >> 1;              // index within the chain
  const int len = chain ? s : s + 1; // number of columns of the chain
  double acc = 0.0;
  if (l >= 1) acc += ga[l - 1] * pc[i - 2];                       // gamma_{l-1} from column l-1
  if (l < len - 1) acc += th[l] * pc[i];                          // diagonal theta_l
  if (l + 1 < len - 1) acc += mu[l] * pc[i + 2];                  // mu_l from column l+1
  return acc;
}

__device__ __forceinline__ void group_sync(int bar, int nthr) {
  if (bar == 0) __syncthreads();
  else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthr) : "memory");
}

// w^T G x over the leading n x n block of Gs (shared memory) by threads
// 0..nthr-1 (whole warps; `bar` = 0: all threads of the block, else a named
// barrier over those nthr threads).  Every product G_ij x_j is issued once and
// the binary64 work is spread evenly: rows 0..31 by nthr/32 threads each
// (columns slot, slot + nthr/32, ...), row 32 (n = 33) one column per thread.
// The fixed-order reduction returns the sum to thread 0 (others get 0).
__device__ double gdot(const double (*Gs)[kMaxCols + 1], const double* x, const double* w, int n, int nthr, int bar,
                       double* red) {
  const int t = threadIdx.x;
  const int S = nthr >> 5;  // threads per row
  const int i = t / S, slot = t - i * S;
  double part = 0.0;
  if (i < n) {
    double s = 0.0;
    for (int j = slot; j < n; j += S) s = fma(Gs[i][j], x[j], s);
    part = w[i] * s;
  }
  if (n > 32 && t < n) part = fma(w[32] * Gs[32][t], x[t], part);
  part = warp_sum(part);
  if ((t & 31) == 0) red[t >> 5] = part;
  group_sync(bar, nthr);
  double q = 0.0;
  if (t == 0) {
    q = red[0];
    for (int k = 1; k < S; ++k) q = q + red[k];
  }
  group_sync(bar, nthr);
  return q;
}

__device__ __forceinline__ double clamp01(double v) { return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v); }

// One loop step of Algorithm 3 (upper estimate, xi read as zeta) for alpha_i and
// beta_{i-1}, with zeta_i = alpha_i^{-1/2} and eta_{i-1} = sqrt(beta_{i-1} /
// alpha_{i-1}) (eq. lit); the first push initialises.  Reads the state, writes
// out[0..2] = (omega, h, zeta).
__device__ void mt_upper(const SolveState* st, double alpha, double beta_prev, double* out) {
  const double zeta = 1.0 / sqrt(alpha);
  out[2] = zeta;
  if (st->mt_n == 0) {
    out[0] = zeta * zeta;
    out[1] = 1.0;
    return;
  }
  const double zl = st->zeta_prev, zl1 = zeta;
  const double eta = sqrt(beta_prev / st->alpha_prev);
  const double d = zl * zl * eta * eta * st->up_h;
  const double a = eta * eta + zl1 * zl1;
  const double dm = st->up_omega - a;
  const double chi = sqrt(dm * dm + 4.0 * d);
  if (chi == 0.0) {
    out[0] = st->up_omega;
    out[1] = 1.0;
  } else {
    const double h = clamp01(0.5 * (1.0 - (st->up_omega - a) / chi));
    out[1] = h;
    out[0] = st->up_omega + chi * h;
  }
}

// One loop step of Algorithm 4 (lower estimate); out[0..5] = (omega, a, d, g,
// h, lambda_min = 1/omega).
__device__ void mt_lower(const SolveState* st, double alpha, double beta_prev, double* out) {
  const double zeta = 1.0 / sqrt(alpha);
  if (st->mt_n == 0) {
    const double om = 1.0 / (zeta * zeta);
    out[0] = om;
    out[1] = om;
    out[2] = 0.0;
    out[3] = 0.0;
    out[4] = 1.0;
    out[5] = 1.0 / om;
    return;
  }
  const double zl1 = zeta;
  const double eta = sqrt(beta_prev / st->alpha_prev);
  const double d1 = -(eta / zl1) * (st->lo_g * st->lo_d + st->lo_h * st->lo_a);
  const double a1 = (eta * eta * st->lo_a + 1.0) / (zl1 * zl1);
  const double dm = st->lo_omega - a1;
  const double chi = sqrt(dm * dm + 4.0 * d1 * d1);
  double om = st->lo_omega, h, g;
  if (chi == 0.0) {
    h = 1.0;
    g = 0.0;
  } else {
    const double h2 = clamp01(0.5 * (1.0 - (st->lo_omega - a1) / chi));
    om = st->lo_omega + chi * h2;
    h = sqrt(h2);
    g = sqrt(clamp01(1.0 - h2));
  }
  out[0] = om;
  out[1] = a1;
  out[2] = d1;
  out[3] = g;
  out[4] = fabs(h) * (d1 < 0.0 ? -1.0 : 1.0);
  out[5] = 1.0 / om;
}

__device__ double c_value(int mode, double lmin, double lmax, double psi, double c_const) {
  switch (mode) {
    case SSCG_C_XI: return fmax(1.0, lmax * sqrt(psi / lmin));
    case SSCG_C_XI_SCALED: return fmax(1.0, lmax * sqrt(psi) / lmin);
    case SSCG_C_ONE: return 1.0;
    case SSCG_C_KAPPA_RATIO: return lmax / lmin;
    default: return c_const;
  }
}

// Recurrence coefficients of level l for the next outer loops from the Ritz
// estimates (one thread per level).
__device__ void basis_update_level(SolveState* st, const double* leja, int l) {
  const double lmin = st->lmin, lmax = st->lmax;
  const double c = 0.5 * (lmax + lmin);
  const double h = 0.5 * (lmax - lmin);
  double th = 0.0, ga = 1.0, mu = 0.0;
  if (st->basis == SSCG_NEWTON) {
    th = c + h * leja[l];
    ga = st->newton_scale == 0 ? (lmax - lmin) / 4.0 : 1.0;
  } else if (st->basis == SSCG_CHEBYSHEV) {
    th = c;
    if (st->cheb_params == 0) {
      ga = l == 0 ? h : 0.5 * h;
      mu = 0.5 * h;
    } else {
      ga = l == 0 ? lmax - lmin : 0.5 * (lmax - lmin);
      mu = 2.0 * (lmax - lmin);
    }
  }
  st->theta[l] = th;
  st->gamma[l] = ga;
  st->inv_gamma[l] = 1.0 / ga;
  st->mu[l] = mu;
}

// Thread roles (128 threads).  Each inner step: all threads form p'^T G (B p');
// then warps 2 and 3 run the two Meurant-Tichy recurrences (they need only
// alpha_j and beta_{j-1}) while warps 0-1 update x', r' and form r'^T G r' and
// thread 0 the scalars that do not depend on the Ritz values; thread 0 then
// commits the Ritz state and takes the c update and the break test.
// ------------------------------------------------------- exact Ritz values
// ritz_exact = 1: the extremal eigenvalues of T_m (eq. T) after every inner
// iteration, in place of the Meurant-Tichy estimates of Algs. 3-4.  T grows by
// one row per CG step (diagonal 1/alpha_m + beta_{m-1}/alpha_{m-1}, squared
// coupling beta_{m-1}/alpha_{m-1}^2, kept in global memory); each extremal
// eigenvalue is bracketed from its previous value (interlacing: lambda_max
// never falls and lambda_min never rises as T grows; Weyl: bordering T by the
// new row moves them by at most the coupling) and narrowed by multisection,
// 64 Sturm counts per round on one half of the block.

// Eigenvalues of the m x m tridiagonal (d, e2) below x: the sign changes of
// p_0 = 1, p_k = det(T_k - x I) = (d_k - x) p_{k-1} - e2_{k-1} p_{k-2} (a zero
// takes the sign opposite to its predecessor), p_k and p_{k-1} rescaled
// together by a power of two whenever the larger leaves [2^-400, 2^400].
__device__ int sturm_below(const double* d, const double* e2, int m, double x) {
  double p2 = 1.0, p1 = d[0] - x;
  int s1 = p1 > 0.0 ? 1 : -1;
  int cnt = s1 < 0 ? 1 : 0;
  for (int k = 1; k < m; ++k) {
    const double p = fma(d[k] - x, p1, -e2[k - 1] * p2);
    const int s = p > 0.0 ? 1 : (p < 0.0 ? -1 : -s1);
    cnt += s != s1;
    p2 = p1;
    p1 = p;
    s1 = s;
    const int E1 = (int)(((unsigned long long)__double_as_longlong(p1) >> 52) & 0x7ff);
    const int E2 = (int)(((unsigned long long)__double_as_longlong(p2) >> 52) & 0x7ff);
    const int Em = E1 > E2 ? E1 : E2;
    if ((Em > 1423 && Em < 2047) || Em < 623) {
      const double sc = __longlong_as_double((long long)(2046 - Em) << 52);   // 2^(1023 - Em), exact
      p1 *= sc;
      p2 *= sc;
    }
  }
  return cnt;
}

// Narrow [lo, hi] around the largest (largest = true) or the smallest
// eigenvalue by the 64 threads of one half of the block (ht = 0..63, named
// barrier BAR): each round counts at 64 interior points and keeps the gap
// between the last point below the eigenvalue and the first above it; every
// thread computes the same brackets.
template <int BAR>
__device__ double multisect(const double* d, const double* e2, int m, double lo, double hi, bool largest, int ht,
                            unsigned* ball) {
  for (int round = 0; round < 16; ++round) {
    if (!(hi - lo > 0x1p-51 * fmax(fabs(lo), fabs(hi)))) break;
    const double w = hi - lo;
    const double x = lo + w * ((double)(ht + 1) * (1.0 / 65.0));
    const int c = sturm_below(d, e2, m, x);
    const bool above = largest ? c >= m : c >= 1;
    const unsigned b = __ballot_sync(0xffffffffu, above);
    if ((ht & 31) == 0) ball[ht >> 5] = b;
    group_sync(BAR, 64);
    const unsigned long long all = (unsigned long long)ball[0] | ((unsigned long long)ball[1] << 32);
    const int first = all ? __ffsll((long long)all) - 1 : 64;
    const double nlo = first == 0 ? lo : lo + w * ((double)first * (1.0 / 65.0));
    const double nhi = first == 64 ? hi : lo + w * ((double)(first + 1) * (1.0 / 65.0));
    group_sync(BAR, 64);
    lo = nlo;
    hi = nhi;
  }
  return 0.5 * (lo + hi);
}

// One push of (alpha, beta_prev) into T (row n = st->mt_n) and its extremal
// eigenvalues into out[0] (lambda_min), out[1] (lambda_max); *full = 1 when T
// has no room for the row (out keeps the previous values).  All threads.
__device__ __forceinline__ void exact_ritz_step(SolveState* __restrict__ st, double alpha, double* out, int* full) {
  static_assert(kControlThreads == 128, "two halves of 64 threads");
  __shared__ unsigned ball[2][2];
  const int t = threadIdx.x;
  const int n = st->mt_n;
  if (n >= st->ritz_cap) {
    if (t == 0) {
      *full = 1;
      out[0] = st->lmin;
      out[1] = st->lmax;
    }
    __syncthreads();
    return;
  }
  if (t == 0) {
    const double bp = st->beta_prev, ap = st->alpha_prev;
    st->ritz_d[n] = 1.0 / alpha + (n >= 1 ? bp / ap : 0.0);
    if (n >= 1) st->ritz_e2[n - 1] = bp / (ap * ap);
  }
  __syncthreads();
  const double* d = st->ritz_d;
  const double* e2 = st->ritz_e2;
  const int m = n + 1;
  if (m == 1) {
    if (t == 0) out[0] = out[1] = d[0];
    __syncthreads();
    return;
  }
  const double dn = d[n], e = sqrt(e2[n - 1]);
  const double pmin = st->lmin, pmax = st->lmax;
  const int half = t >> 6, ht = t & 63;
  double lo, hi;
  if (half == 0) {
    lo = pmax - 0x1p-50 * fabs(pmax);
    hi = fmax(pmax, dn) + e;
    hi += 0x1p-50 * fabs(hi);
  } else {
    lo = fmin(pmin, dn) - e;
    lo -= 0x1p-50 * fabs(lo);
    hi = pmin + 0x1p-50 * fabs(pmin);
  }
  const double v = half == 0 ? multisect<2>(d, e2, m, lo, hi, true, ht, ball[0])
                             : multisect<3>(d, e2, m, lo, hi, false, ht, ball[1]);
  if (ht == 0) out[half == 0 ? 1 : 0] = v;
  __syncthreads();
}

// EXACT: the control step of ritz_exact = 1 (its own kernel, so that the
// default step keeps its registers)
template <bool EXACT>
__device__ void control_body(SolveState* __restrict__ st, const double* __restrict__ G, int ldg,
                             const double* __restrict__ leja, sscg_outer_record* __restrict__ hist) {
  static_assert(kControlThreads == 128, "four warps");
  const int t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  __shared__ double Gs[kMaxCols][kMaxCols + 1];
  __shared__ double xc[kMaxCols], rc[kMaxCols], pc[kMaxCols], bp[kMaxCols];
  __shared__ double th[kMaxS], ga[kMaxS], mu[kMaxS];
  __shared__ double red[4], red2[2];
  __shared__ double mt_up[3], mt_lo[6];
  __shared__ int s_stilde, s_flag, s_valid, s_basis, s_rfull;
  __shared__ double s_alpha, s_beta;
  __shared__ double ex_ritz[2];   // ritz_exact: lambda_min, lambda_max of T after this step

  const int sbar = st->sbar;
  if (warp == 0) {
    // s-tilde (eq. condy): the largest l <= s-bar with kappa_l below the threshold
    const double c0 = st->variant == 2 ? st->c_const : st->c;  // Alg. 2: c_k supplied by the user
    int stl = 1;
    if (st->variant == 1) {
      stl = sbar;
    } else {
      const double normr = sqrt(G[1 * ldg + 1]);
      const double thr = st->tol / (c0 * st->eps * normr / st->normb);
      const unsigned ball = __ballot_sync(0xffffffffu, lane >= 1 && lane <= sbar && st->kappa[lane] <= thr);
      if (ball) stl = 31 - __clz(ball);
    }
    if (lane == 0) {
      if (st->variant == 2) st->c = st->c_const;
      s_stilde = stl;
      s_rfull = 0;
    }
  }
  if (t < kMaxS) {
    th[t] = st->theta[t];
    ga[t] = st->gamma[t];
    mu[t] = st->mu[t];
  }
  __syncthreads();
  const int stl = s_stilde;
  const int n = 2 * stl + 1;
  for (int e = t; e < n * n; e += kControlThreads) {
    const int i = e / n, j = e - (e / n) * n;
    Gs[i][j] = G[i * ldg + j];
  }
  if (t < kMaxCols) {
    xc[t] = 0.0;
    rc[t] = t == 1 ? 1.0 : 0.0;
    pc[t] = t == 0 ? 1.0 : 0.0;
  }
  __syncthreads();

  // thread-0 scalars of the inner loop
  double rr = Gs[1][1];
  double phi = sqrt(rr > 0.0 ? rr : 0.0);
  const double c_start = st->c;
  int sk = 0;
  int conv = 0, breakdown = 0;
  const int m0 = st->m;

  for (int j = 0; j < stl; ++j) {
    if (t < n) bp[t] = b_times(pc, t, stl, th, ga, mu);
    __syncthreads();
    const double pGBp = gdot(Gs, bp, pc, n, kControlThreads, 0, red);  // p'^T G (B p')
    if (t == 0) {
      const double alpha = pGBp > 0.0 ? rr / pGBp : NAN;
      s_flag = 0;
      if (!(alpha > 0.0) || !isfinite(alpha)) {
        s_flag = 1;
        if (j == 0) breakdown = 1;
      }
      s_alpha = alpha;
    }
    __syncthreads();
    if (s_flag) break;
    const double alpha = s_alpha;
    if constexpr (EXACT) exact_ritz_step(st, alpha, ex_ritz, &s_rfull);
    double beta = 0.0;
    if (warp >= 2) {
      if (lane == 0) {
        if (warp == 2) mt_upper(st, alpha, st->beta_prev, mt_up);
        else mt_lower(st, alpha, st->beta_prev, mt_lo);
      }
    } else {
      if (t < n) {
        xc[t] = xc[t] + alpha * pc[t];
        rc[t] = rc[t] - alpha * bp[t];
      }
      group_sync(1, 64);
      const double rr_new = gdot(Gs, rc, rc, n, 64, 1, red2);
      if (t == 0) {
        sk = j + 1;
        s_flag = 0;
        s_valid = 0;
        if (!(rr_new > 0.0) || !isfinite(rr_new)) {
          conv = 1;
          s_flag = 1;
        } else {
          s_valid = 1;
          beta = rr_new / rr;
          s_beta = beta;
          phi = fmax(phi, sqrt(rr_new));
          st->psi = st->psi / (st->psi + beta);
          rr = rr_new;
          if (st->inner_conv_check && sqrt(rr_new) / st->normb <= st->tol) {
            conv = 1;
            s_flag = 2;
          }
        }
      }
    }
    __syncthreads();
    if (t == 0 && s_valid) {
      // commit Algorithms 3-4 for (alpha_j, beta_{j-1})
      st->up_omega = mt_up[0];
      st->up_h = mt_up[1];
      st->lo_omega = mt_lo[0];
      st->lo_a = mt_lo[1];
      st->lo_d = mt_lo[2];
      st->lo_g = mt_lo[3];
      st->lo_h = mt_lo[4];
      if constexpr (EXACT) {
        st->lmax = ex_ritz[1];
        st->lmin = ex_ritz[0];
        if (s_rfull) {   // no room left for T: stop
          st->status = SSCG_NOT_CONVERGED;
          st->done = 1;
          s_flag = 1;
        }
      } else {
        st->lmax = mt_up[0];
        st->lmin = mt_lo[5];
      }
      st->zeta_prev = mt_up[2];
      st->alpha_prev = alpha;
      st->mt_n += 1;
      st->beta_prev = beta;
      if (m0 + j + 1 > 1 && st->variant != 2)
        st->c = c_value(st->c_mode, st->lmin, st->lmax, st->psi, st->c_const);
      if (s_flag != 2) {
        if (st->variant == 2) {
          // Alg. 2's break test: kappa of the whole block against the current residual
          if (st->kappa[stl] >= st->tol / (st->c * st->eps * sqrt(rr) / st->normb)) s_flag = 2;
        } else if (st->variant != 1 && j < stl - 1 &&
                   st->kappa[j + 2] >= st->tol / (st->c * st->eps * phi / st->normb)) {
          s_flag = 2;
        }
      }
    }
    __syncthreads();
    if (s_flag == 1) break;
    const double b_ = s_beta;
    if (t < n) pc[t] = rc[t] + b_ * pc[t];
    __syncthreads();
    if (s_flag == 2) break;
  }
  __syncthreads();

  if (t == 0) {
    const int k = st->k;
    s_basis = 0;
    if (breakdown) {
      st->status = SSCG_BREAKDOWN;
      st->done = 1;
      st->nc = 0;
    } else {
      // outer-level convergence test when the per-step test is off (reading C15)
      if (!conv && !st->inner_conv_check && sqrt(rr > 0.0 ? rr : 0.0) / st->normb <= st->tol) conv = 1;
      st->stilde = stl;
      st->sk = sk;
      st->nc = 2 * sk + 1;
      st->m = m0 + sk;
      st->converged_est = conv;
      st->upd_relres = sqrt(rr > 0.0 ? rr : 0.0) / st->normb;
      if (st->m > 1 && st->basis != SSCG_MONOMIAL && st->variant != 2) {
        s_basis = 1;
        st->have_ritz = 1;
      }
      int nsb = sk + st->f;
      st->sbar = nsb < st->sigma ? nsb : st->sigma;
      // FP32-stored basis: put the true residual back once the estimate has
      // fallen by fp32_drop since the last replacement (p is kept)
      if (st->y_fp32 && !conv && st->upd_relres <= st->fp32_drop * st->rho_last) st->fp32_replace_pending = 1;
    }
    if (hist != nullptr && k < st->hist_cap) {
      sscg_outer_record& h = hist[k];
      h.sbar = sbar;
      h.stilde = stl;
      h.sk = breakdown ? 0 : sk;
      h.replaced = 0;
      h.c_start = c_start;
      h.c_end = st->c;
      h.phi = phi;
      h.lmin = st->lmin;
      h.lmax = st->lmax;
      h.relres_est = st->upd_relres;
      for (int l = 0; l <= kMaxS; ++l) h.kappa[l] = (l >= 1 && l <= sbar) ? st->kappa[l] : 0.0;
    }
    st->k = k + 1;
  }
  if (t < kMaxCols) {
    st->xc[t] = t < n ? xc[t] : 0.0;
    st->rc[t] = t < n ? rc[t] : 0.0;
    st->pc[t] = t < n ? pc[t] : 0.0;
  }
  __syncthreads();
  if (s_basis && t < st->sigma) basis_update_level(st, leja, t);
}

template <bool EXACT>
__global__ void __launch_bounds__(kControlThreads) control_kernel(SolveState* __restrict__ st,
                                                                  const double* __restrict__ G, int ldg,
                                                                  const double* __restrict__ leja,
                                                                  sscg_outer_record* __restrict__ hist) {
  if (st->done) return;
  control_body<EXACT>(st, G, ldg, leja, hist);
}


// Batched kappa: block (j, l) computes kappa_l of pair j.
__global__ void __launch_bounds__(kKappaThreads) batch_kappa_kernel(BatchView v, int sigma_max) {
  const int j = blockIdx.x / sigma_max;
  const int l = blockIdx.x % sigma_max + 1;
  SolveState* st = v.states + j;
  if (st->done || l > st->sbar) return;
  const double* G = v.G + (int64_t)j * kMaxCols * kMaxCols;
  kappa_body(G, kMaxCols, l, st->kappa_cut, st->kappa, st->glmin, st->glmax);
}

// Batched control: one block per pair.
__global__ void __launch_bounds__(kControlThreads) batch_control_kernel(BatchView v, const double* __restrict__ leja) {
  const int j = blockIdx.x;
  SolveState* st = v.states + j;
  if (st->done) return;
  const double* G = v.G + (int64_t)j * kMaxCols * kMaxCols;
  sscg_outer_record* h = v.hist != nullptr ? v.hist + (int64_t)j * v.hist_cap : nullptr;
  control_body<false>(st, G, kMaxCols, leja, h);
}

// ------------------------------------------------------------------ Leja
// Leja points of [-1, 1] (eq. newtbasis on the reference interval): t_0 = 1,
// t_1 = -1, then the maximiser of prod |t - t_m|.  In each gap between sorted
// points the log-product is concave, so its maximiser is the zero of the
// derivative sum 1/(t - t_m), found by bisection to the last bit; the gap with
// the largest product wins, ties (within 1e-13 in log) go to the smaller t.
__device__ void leja_points(double* out, int s) {
  double pts[kMaxS];
  double srt[kMaxS];
  int np = 0;
  if (s >= 1) pts[np++] = 1.0;
  if (s >= 2) pts[np++] = -1.0;
  while (np < s) {
    for (int i = 0; i < np; ++i) srt[i] = pts[i];
    for (int i = 1; i < np; ++i) {  // insertion sort, ascending
      double key = srt[i];
      int j = i - 1;
      while (j >= 0 && srt[j] > key) {
        srt[j + 1] = srt[j];
        --j;
      }
      srt[j + 1] = key;
    }
    double best_t = 0.0, best_v = -INFINITY;
    bool have = false;
    for (int g = 0; g + 1 < np; ++g) {
      double lo = srt[g], hi = srt[g + 1];
      while (true) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double dv = 0.0;
        for (int i = 0; i < np; ++i) dv = dv + 1.0 / (mid - pts[i]);
        if (dv == 0.0) {
          lo = hi = mid;
          break;
        }
        if (dv > 0.0) lo = mid;
        else hi = mid;
      }
      const double tt = 0.5 * (lo + hi);
      double v = 0.0;
      for (int i = 0; i < np; ++i) v = v + log(fabs(tt - pts[i]));
      if (!have || v > best_v + 1e-13) {
        best_t = tt;
        best_v = v;
        have = true;
      } else if (fabs(v - best_v) <= 1e-13 && tt < best_t) {
        best_t = tt;
        best_v = fmax(v, best_v);
      }
    }
    pts[np++] = best_t;
  }
  for (int i = 0; i < s; ++i) out[i] = pts[i];
}

__global__ void leja_kernel(double* out, int s) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  leja_points(out, s);
}

// The process-wide table of the first kMaxS Leja points (every s-bar uses a
// prefix of it): it lives in this module's device memory, so each device
// holds its own copy, and a device reset reloads the module with the flag
// cleared.  The kernel computes the table only while the flag is clear; the
// flag is set after the points are written, so a later reader on any stream
// either sees it set with the points in place, or computes them itself.
__device__ double g_leja[kMaxS];
__device__ int g_leja_ready;

__global__ void leja_table_kernel() {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (*(volatile int*)&g_leja_ready) return;
  leja_points(g_leja, kMaxS);
  __threadfence();
  *(volatile int*)&g_leja_ready = 1;
}

}  // namespace

cudaError_t leja_table(const double** table, cudaStream_t st) {
  leja_table_kernel<<<1, 32, 0, st>>>();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaGetSymbolAddress((void**)table, g_leja);
}

cudaError_t launch_kappa(const double* G, int ldg, const SolveState* state, int sbar_fixed, double kappa_cut,
                         double* kappa, double* lmin, double* lmax, int grid, cudaStream_t st) {
  kappa_kernel<<<grid, kKappaThreads, 0, st>>>(G, ldg, state, sbar_fixed, kappa_cut, kappa, lmin, lmax);
  return cudaGetLastError();
}

cudaError_t launch_control(SolveState* state, const double* G, int ldg, const double* leja,
                           sscg_outer_record* hist, cudaStream_t st, bool ritz_exact) {
  if (ritz_exact)
    control_kernel<true><<<1, kControlThreads, 0, st>>>(state, G, ldg, leja, hist);
  else
    control_kernel<false><<<1, kControlThreads, 0, st>>>(state, G, ldg, leja, hist);
  return cudaGetLastError();
}

cudaError_t launch_batch_kappa(const BatchView& v, int sigma_max, cudaStream_t st) {
  batch_kappa_kernel<<<v.npairs * sigma_max, kKappaThreads, 0, st>>>(v, sigma_max);
  return cudaGetLastError();
}

cudaError_t launch_batch_control(const BatchView& v, const double* leja, cudaStream_t st) {
  batch_control_kernel<<<v.npairs, kControlThreads, 0, st>>>(v, leja);
  return cudaGetLastError();
}

cudaError_t launch_leja(double* t, int s, cudaStream_t st) {
  leja_kernel<<<1, 32, 0, st>>>(t, s);
  return cudaGetLastError();
}

}  // namespace sscg
