// Gram matrix G = Y^T Y of the s-step basis (Carson 2019, Section 2: the one
// block inner product per outer loop of Algorithm 5, computed once and kept on
// the device).
//
// Design for GB300: a tall-skinny contraction (n rows, at most 33 columns)
// that is bound by FP64 issue rate (561 DFMA per row at s = 16 against 264
// bytes per row), so the kernel gives every lane one unique (i <= j) entry of
// G and streams row tiles of Y through shared memory: each DFMA needs two
// shared loads and nothing else.  When fewer pairs than threads exist, the
// spare threads take interleaved rows of the same tile (row lanes) so that all
// lanes issue DFMAs.  Rows are split into contiguous chunks per block; each
// block writes one partial sum per pair, and a second kernel adds the partials
// of every pair in a fixed order, so G is bitwise reproducible run to run.
#include <mutex>

#include "sscg_internal.cuh"

namespace sscg {

namespace {

__device__ __forceinline__ void pair_of(int q, int ncols, int* pi, int* pj) {
  int i = 0, rem = q;
  while (rem >= ncols - i) {
    rem -= ncols - i;
    ++i;
  }
  *pi = i;
  *pj = i + rem;
}

template <typename T>
__global__ void __launch_bounds__(kGramThreads, 2)
gram_partial_kernel(const T* __restrict__ Y, int64_t n, int64_t ld, const SolveState* __restrict__ st,
                    int ncols_fixed, double* __restrict__ partials) {
  int ncols = ncols_fixed;
  if (ncols <= 0) {
    if (st->done) return;
    ncols = 2 * st->sbar + 1;
  }
  const int np = ncols * (ncols + 1) / 2;
  const int R = kGramThreads / np;  // row lanes, >= 1
  const int t = threadIdx.x;
  const bool active = t < R * np;
  const int q = t % np;
  const int rl = t / np;
  int pi = 0, pj = 0;
  pair_of(q, ncols, &pi, &pj);

  __shared__ double tile[kGramTileRows][kMaxCols + 1];
  __shared__ double red[kGramThreads];

  // contiguous row chunk of this block, a multiple of the tile height
  const int64_t tiles = (n + kGramTileRows - 1) / kGramTileRows;
  const int64_t tpb = (tiles + gridDim.x - 1) / gridDim.x;
  const int64_t r_begin = (int64_t)blockIdx.x * tpb * kGramTileRows;
  int64_t r_end = r_begin + tpb * kGramTileRows;
  if (r_end > n) r_end = n;

  double acc = 0.0;
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kGramTileRows) {
    for (int e = t; e < kGramTileRows * ncols; e += kGramThreads) {
      const int c = e / kGramTileRows;
      const int r = e - c * kGramTileRows;
      const int64_t row = r0 + r;
      tile[r][c] = row < r_end ? widen(__ldg(Y + (int64_t)c * ld + row)) : 0.0;
    }
    __syncthreads();
    if (active) {
#pragma unroll 8
      for (int r = rl; r < kGramTileRows; r += R) acc = fma(tile[r][pi], tile[r][pj], acc);
    }
    __syncthreads();
  }
  red[t] = acc;
  __syncthreads();
  if (t < np) {
    double s = 0.0;
    for (int l = 0; l < R; ++l) s += red[l * np + t];
    partials[(int64_t)blockIdx.x * kMaxPairs + t] = s;
  }
}


// ------------------------------------------------------------------------
// Gram with binary32-pair products (gram_mode = 1).
//
// GB300 issues binary32 FMAs 62 times faster than binary64 ones, so this
// variant forms each product y_i y_j on the FP32 pipes and keeps binary64 only
// for the accumulation across tiles.  Per 256-row tile every column c gets a
// power-of-two scale 2^-e_c (e_c = its largest exponent in the tile); each
// scaled value is split exactly by integer operations into hi (its leading 24
// bits) + lo (the next 24 bits, truncated; |y - hi - lo| < 2^-46 |y|).  Then
//   y_i y_j ~ hi_i hi_j + (hi_i lo_j + lo_i hi_j + lo_i lo_j),
// with hi_i hi_j exact as the pair (p, fma(hi_i, hi_j, -p)); the tile sum is a
// compensated (TwoSum) binary32 pair, added into the binary64 accumulator times
// 2^(e_i + e_j) once per tile.  Values more than 2^125 below their column's
// largest in the tile are dropped (they are below binary64's resolution of
// the sum).
//
// Work layout: columns are taken in groups of two (the last group padded with
// a zero column), each thread owns one 2 x 2 block (I <= J) of G, so one pair
// of 16-byte shared loads feeds 4 products (13 binary32 operations each); the
// spare threads take interleaved rows of the tile.  One block per SM; the next
// tile's global loads are issued into registers before the current tile is
// reduced, and the split tiles are double-buffered in shared memory.
__device__ __forceinline__ void split_scaled(double y, int cexp, float* hi, float* lo) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(y);
  const unsigned int sign = (unsigned int)(bits >> 32) & 0x80000000u;
  const int E = (int)((bits >> 52) & 0x7ff);
  if (E == 0) {  // zero (and subnormals, far below any column's largest value)
    *hi = 0.f;
    *lo = 0.f;
    return;
  }
  if (E == 0x7ff) {  // Inf/NaN propagate
    *hi = (float)y;
    *lo = 0.f;
    return;
  }
  const int e = E - 1023 - cexp;  // <= 0
  if (e < -125) {
    *hi = 0.f;
    *lo = 0.f;
    return;
  }
  const unsigned long long m = bits & ((1ull << 52) - 1);
  *hi = __uint_as_float(sign | ((unsigned int)(e + 127) << 23) | (unsigned int)(m >> 29));
  const unsigned int rem = (unsigned int)(m & ((1u << 29) - 1));
  if (rem == 0u) {
    *lo = 0.f;
    return;
  }
  const int lz = __clz(rem) - 3;       // leading zeros inside the 29-bit remainder
  const int el = e - 24 - lz;          // exponent of the remainder's leading bit
  if (el < -126) {
    *lo = 0.f;
    return;
  }
  const unsigned int ml = (rem << (lz + 4)) >> 9;  // bits after the leading one, 23 kept
  *lo = __uint_as_float(sign | ((unsigned int)(el + 127) << 23) | ml);
}

// unbiased exponent of a finite nonzero y; -1100 for zero and subnormals,
// 1024 for Inf and NaN (so that they reach the sum)
__device__ __forceinline__ int exp_key(double y) {
  const int E = (int)(((unsigned long long)__double_as_longlong(y) >> 52) & 0x7ff);
  return E == 0 ? -1100 : E - 1023;
}

// 2^k as a binary64 built from its bits (k in the normal range), else ldexp
__device__ __forceinline__ double pow2(int k) {
  return (k >= -1022 && k <= 1023) ? __longlong_as_double((long long)(k + 1023) << 52) : ldexp(1.0, k);
}

constexpr int kFFThreads = 640;
constexpr int kFFRows = 256;
constexpr int kFFCols = kMaxCols + 1;                           // 34: padded to whole groups
constexpr int kFFGroups = kFFCols / 2;                          // 17
constexpr int kFFLoads = (kFFRows * kMaxCols + kFFThreads - 1) / kFFThreads;  // 14 per thread
constexpr size_t kFFSmem = 2 * (size_t)kFFRows * kFFCols * sizeof(float2);  // 139,264 B

// one binary32-pair product hi_a*hi_b + (hi_a*lo_b + lo_a*hi_b + lo_a*lo_b)
// added into the compensated sum (shi, slo)
__device__ __forceinline__ void ff_madd(float ah, float al, float bh, float bl, float& shi, float& slo) {
  const float p = ah * bh;
  const float pe = fmaf(ah, bh, -p);
  const float cr = fmaf(ah, bl, fmaf(al, bh, al * bl));
  const float s = shi + p;  // TwoSum(shi, p)
  const float bb = s - shi;
  const float err = (shi - (s - bb)) + (p - bb);
  shi = s;
  slo = slo + (err + (pe + cr));
}

template <typename T>
__global__ void __launch_bounds__(kFFThreads, 1)
gram_partial_ff_kernel(const T* __restrict__ Y, int64_t n, int64_t ld, const SolveState* __restrict__ st,
                       int ncols_fixed, double* __restrict__ partials) {
  int ncols = ncols_fixed;
  if (ncols <= 0) {
    if (st->done) return;
    ncols = 2 * st->sbar + 1;
  }
  const int ng = (ncols + 1) / 2;             // column groups
  const int nbp = ng * (ng + 1) / 2;          // 2 x 2 blocks with I <= J
  const int R = kFFThreads / nbp;             // row lanes, >= 4
  const int t = threadIdx.x;
  const bool active = t < R * nbp;
  const int q = t % nbp;
  const int rl = t / nbp;
  int I = 0, J = 0;
  pair_of(q, ng, &I, &J);
  const int i0 = 2 * I, j0 = 2 * J;

  extern __shared__ __align__(16) unsigned char ff_smem[];
  float2* tiles = reinterpret_cast<float2*>(ff_smem);  // [2][kFFRows][kFFCols]
  __shared__ int cexp[2][kFFCols];

  const int64_t ntiles = (n + kFFRows - 1) / kFFRows;
  const int64_t tpb = (ntiles + gridDim.x - 1) / gridDim.x;
  const int64_t r_begin = (int64_t)blockIdx.x * tpb * kFFRows;
  int64_t r_end = r_begin + tpb * kFFRows;
  if (r_end > n) r_end = n;

  // padding columns (index >= ncols) of both buffers stay zero
  for (int e = t; e < 2 * kFFRows; e += kFFThreads)
    for (int c = ncols; c < kFFCols; ++c) tiles[(size_t)e * kFFCols + c] = make_float2(0.f, 0.f);
  if (t < 2 * kFFCols) cexp[t / kFFCols][t % kFFCols] = -1100;

  // element k of this thread in a tile: e = t + k * kFFThreads -> (column e / kFFRows,
  // row e % kFFRows); a warp's 32 elements share one column
  double pre[kFFLoads];
  auto prefetch = [&](int64_t r0) {
#pragma unroll
    for (int k = 0; k < kFFLoads; ++k) {
      const int e = t + k * kFFThreads;
      const int c = e / kFFRows;
      const int64_t row = r0 + (e - c * kFFRows);
      pre[k] = (c < ncols && row < r_end) ? widen(__ldg(Y + (int64_t)c * ld + row)) : 0.0;
    }
  };
  if (r_begin < r_end) prefetch(r_begin);
  __syncthreads();

  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  int buf = 0;
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kFFRows, buf ^= 1) {
    // column exponents of this tile: warp maximum, then one shared atomic per warp
#pragma unroll
    for (int k = 0; k < kFFLoads; ++k) {
      const int e = t + k * kFFThreads;
      const int c = e / kFFRows;
      if (c < ncols) {  // warp-uniform
        const int m = __reduce_max_sync(0xffffffffu, exp_key(pre[k]));
        if ((t & 31) == 0) atomicMax(&cexp[buf][c], m);
      }
    }
    __syncthreads();
    float2* tile = tiles + (size_t)buf * kFFRows * kFFCols;
#pragma unroll
    for (int k = 0; k < kFFLoads; ++k) {
      const int e = t + k * kFFThreads;
      const int c = e / kFFRows;
      if (c < ncols) {
        float h, l;
        split_scaled(pre[k], cexp[buf][c], &h, &l);
        tile[(e - c * kFFRows) * kFFCols + c] = make_float2(h, l);
      }
    }
    // the other buffer's exponents were last read before the barrier above
    if (t < kFFCols) cexp[buf ^ 1][t] = -1100;
    if (r0 + kFFRows < r_end) prefetch(r0 + kFFRows);
    __syncthreads();
    if (active) {
      float shi[4] = {0.f, 0.f, 0.f, 0.f}, slo[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
      for (int r = rl; r < kFFRows; r += R) {
        const float4 a = *reinterpret_cast<const float4*>(&tile[r * kFFCols + i0]);
        const float4 b = *reinterpret_cast<const float4*>(&tile[r * kFFCols + j0]);
        ff_madd(a.x, a.y, b.x, b.y, shi[0], slo[0]);
        ff_madd(a.x, a.y, b.z, b.w, shi[1], slo[1]);
        ff_madd(a.z, a.w, b.x, b.y, shi[2], slo[2]);
        ff_madd(a.z, a.w, b.z, b.w, shi[3], slo[3]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int ci = i0 + (u >> 1), cj = j0 + (u & 1);
        if (ci < ncols && cj < ncols) {
          const int sc = cexp[buf][ci] + cexp[buf][cj];
          if (sc > -2100) acc[u] = fma(pow2(sc), (double)shi[u] + (double)slo[u], acc[u]);
        }
      }
    }
  }
  __syncthreads();
  // row-lane reduction through shared memory (reusing the tiles): red[rl][q][u]
  double* red = reinterpret_cast<double*>(ff_smem);
  if (active) {
#pragma unroll
    for (int u = 0; u < 4; ++u) red[((size_t)rl * nbp + q) * 4 + u] = acc[u];
  }
  __syncthreads();
  const int np = ncols * (ncols + 1) / 2;
  for (int pq = t; pq < np; pq += kFFThreads) {
    int pi = 0, pj = 0;
    pair_of(pq, ncols, &pi, &pj);
    const int bI = pi >> 1, bJ = pj >> 1;
    const int bq = bI * ng - bI * (bI - 1) / 2 + (bJ - bI);
    const int u = ((pi & 1) << 1) | (pj & 1);
    double s = 0.0;
    for (int l = 0; l < R; ++l) s += red[((size_t)l * nbp + bq) * 4 + u];
    partials[(int64_t)blockIdx.x * kMaxPairs + pq] = s;
  }
}

// One warp per pair: fixed-order sum of the per-block partials.
__global__ void __launch_bounds__(256) gram_reduce_kernel(const double* __restrict__ partials, int nblocks,
                                                          const SolveState* __restrict__ st, int ncols_fixed,
                                                          double* __restrict__ G, int ldg) {
  int ncols = ncols_fixed;
  if (ncols <= 0) {
    if (st->done) return;
    ncols = 2 * st->sbar + 1;
  }
  const int np = ncols * (ncols + 1) / 2;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= np) return;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += partials[(int64_t)b * kMaxPairs + warp];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    int i, j;
    pair_of(warp, ncols, &i, &j);
    G[i * ldg + j] = s;
    G[j * ldg + i] = s;
  }
}


// Batched Gram: each block owns gram_rows rows of one pair and writes the
// pair's (2s-bar+1)(2s-bar+2)/2 partial sums; the reduction adds each pair's
// block partials in a fixed order (one block per pair).
__global__ void __launch_bounds__(kGramThreads, 2)
batch_gram_partial_kernel(BatchView v, const double* __restrict__ Y, int64_t LD, double* __restrict__ partials) {
  const int g = blockIdx.x;
  const int j = v.gblk_pair[g];
  const BatchPair& bp = v.pairs[j];
  const SolveState* st = v.states + j;
  if (st->done) return;
  const int ncols = 2 * st->sbar + 1;
  const int np = ncols * (ncols + 1) / 2;
  const int R = kGramThreads / np;
  const int t = threadIdx.x;
  const bool active = t < R * np;
  const int q = t % np;
  const int rl = t / np;
  int pi = 0, pj = 0;
  pair_of(q, ncols, &pi, &pj);
  __shared__ double tile[kGramTileRows][kMaxCols + 1];
  __shared__ double red[kGramThreads];
  const double* Yp = Y + bp.off;
  const int64_t r_begin = (int64_t)(g - bp.gblk0) * v.gram_rows;
  int64_t r_end = r_begin + v.gram_rows;
  if (r_end > bp.n) r_end = bp.n;
  double acc = 0.0;
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kGramTileRows) {
    for (int e = t; e < kGramTileRows * ncols; e += kGramThreads) {
      const int c = e / kGramTileRows;
      const int r = e - c * kGramTileRows;
      const int64_t row = r0 + r;
      tile[r][c] = row < r_end ? __ldg(Yp + (int64_t)c * LD + row) : 0.0;
    }
    __syncthreads();
    if (active) {
#pragma unroll 8
      for (int r = rl; r < kGramTileRows; r += R) acc = fma(tile[r][pi], tile[r][pj], acc);
    }
    __syncthreads();
  }
  red[t] = acc;
  __syncthreads();
  if (t < np) {
    double s = 0.0;
    for (int l = 0; l < R; ++l) s += red[l * np + t];
    partials[(int64_t)g * kMaxPairs + t] = s;
  }
}

__global__ void __launch_bounds__(256) batch_gram_reduce_kernel(BatchView v, const double* __restrict__ partials) {
  const int j = blockIdx.x;
  const BatchPair& bp = v.pairs[j];
  const SolveState* st = v.states + j;
  if (st->done) return;
  const int ncols = 2 * st->sbar + 1;
  const int np = ncols * (ncols + 1) / 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* G = v.G + (int64_t)j * kMaxCols * kMaxCols;
  for (int q = warp; q < np; q += blockDim.x / 32) {
    double s = 0.0;
    for (int b = lane; b < bp.ngblk; b += 32) s += partials[(int64_t)(bp.gblk0 + b) * kMaxPairs + q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      int i, jj;
      pair_of(q, ncols, &i, &jj);
      G[i * kMaxCols + jj] = s;
      G[jj * kMaxCols + i] = s;
    }
  }
}

}  // namespace

cudaError_t launch_batch_gram(const BatchView& v, const double* Y, int64_t LD, double* partials, cudaStream_t st) {
  batch_gram_partial_kernel<<<v.ngblk, kGramThreads, 0, st>>>(v, Y, LD, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_gram_reduce_kernel<<<v.npairs, 256, 0, st>>>(v, partials);
  return cudaGetLastError();
}

int gram_blocks(int64_t n) {
  int64_t tiles = (n + kGramTileRows - 1) / kGramTileRows;
  int64_t b = 152 * 2;
  if (tiles < b) b = tiles;
  return b < 1 ? 1 : (int)b;
}

cudaError_t gram_prepare() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(gram_partial_ff_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFFSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(gram_partial_ff_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFFSmem);
  if (e != cudaSuccess) return e;
  done[dev] = true;
  return cudaSuccess;
}

cudaError_t launch_gram(const void* Y, int64_t n, int64_t ld, const int* /*ncols_dev*/, int ncols_fixed,
                        const SolveState* state, double* partials, int nblocks, double* G, int ldg, bool y32,
                        cudaStream_t st, int gram_mode) {
  if (gram_mode == 1) {
    // one block per SM, at most one block per 256-row tile
    const int64_t ntiles = (n + kFFRows - 1) / kFFRows;
    int nb = nblocks < 152 ? nblocks : 152;
    if (ntiles < nb) nb = (int)ntiles;
    if (nb < 1) nb = 1;
    nblocks = nb;
    if (y32)
      gram_partial_ff_kernel<float><<<nblocks, kFFThreads, kFFSmem, st>>>(static_cast<const float*>(Y), n, ld,
                                                                         state, ncols_fixed, partials);
    else
      gram_partial_ff_kernel<double><<<nblocks, kFFThreads, kFFSmem, st>>>(static_cast<const double*>(Y), n, ld,
                                                                          state, ncols_fixed, partials);
  } else if (y32) {
    gram_partial_kernel<float><<<nblocks, kGramThreads, 0, st>>>(static_cast<const float*>(Y), n, ld, state,
                                                                 ncols_fixed, partials);
  } else {
    gram_partial_kernel<double><<<nblocks, kGramThreads, 0, st>>>(static_cast<const double*>(Y), n, ld, state,
                                                                  ncols_fixed, partials);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int warps_per_block = 256 / 32;
  gram_reduce_kernel<<<(kMaxPairs + warps_per_block - 1) / warps_per_block, 256, 0, st>>>(
      partials, nblocks, state, ncols_fixed, G, ldg);
  return cudaGetLastError();
}

}  // namespace sscg
