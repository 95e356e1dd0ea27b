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

// ------------------------------------------------------------------------
// Gram on the tensor cores by exact digit products (gram_mode = 2).
//
// GB300 runs `mma.sync` f16 with binary32 accumulation at about 600 TFLOP/s
// against 1.2 TFLOP/s of binary64 FMA, so this variant writes every value of
// Y as 12 signed 5-bit digits and lets the tensor cores form all digit
// products, exactly.  Rows are grouped in scale chunks of kDgChunkRows;
// within a chunk column c has the power-of-two scale of its largest value
// (biased exponent ce_c, from a pre-pass over Y), and each value becomes the
// 60-bit integer
//   F = round(|y| 2^(1082 - ce_c)),  |y| ~ F 2^(ce_c - 1082)
// (exact when y is within 2^7 of the column's largest value, else rounded at
// bit 60), F = sum_t d_t 32^(11 - t), d_t in [0, 31], each digit carrying
// y's sign.  The f16 bit pattern k (0 <= k <= 1023) is the subnormal k 2^-24,
// so a digit is its own encoding.  For u = s + t <= 11 the tensor cores
// accumulate H_u = 2^-48 sum_rows sum_{s+t=u} d_s(y_i) d_t(y_j) in binary32;
// every partial sum is an integer times 2^-48 below 2^24 2^-48 (at most
// 1024 rows x 12 products x 961), so it is exact.  Every 1024 rows the
// block adds
//   G_ij += 2^(ce_i + ce_j - 2006) sum_{u <= 11} H_u 2^(-5u)
// (the sum formed exactly in two 64-bit integers, then two binary64 adds).
// Per row, the rounding of F (2^-60 of the column's largest value) and the
// terms dropped (s + t > 11: about 2^-56.5 of the product of the two columns'
// largest values) bound the error, so normwise the result is at least as
// accurate as binary64 FMAs (below 2^-53 ||y_i|| ||y_j|| in the tests, where
// binary64 FMAs are only bounded by n 2^-53 ||y_i|| ||y_j||); componentwise it
// is not: an entry whose products all lie far below the two columns' largest
// values keeps only that absolute accuracy.  A column with an Inf or NaN in a
// chunk makes its entries NaN.
//
// Work layout (warp specialised): eight MMA warps own one 16 x 8 tile
// (m16n8k16) of the upper triangle of G each, with all 12 accumulators
// H_0..H_11 of the tile (48 registers).  Per 16-row k-step a warp loads the
// B fragments of all 12 digit planes once, then for each plane s one A
// fragment feeding 12 - s MMAs (78 per k-step).  Eight conversion warps fetch
// the raw values of the stages ahead by cp.async (each thread the rows it
// converts) and write their digits; the digits of a 64-row stage sit in
// shared memory as [plane][8-row block][column][16 bytes] (one 16-byte
// ldmatrix row per column and block), double buffered, handed over with
// named barriers (full: conversion warps arrive, MMA warps wait; empty: the
// reverse), so conversion overlaps the MMAs.  When ncols = 16 m + 1
// (ncols = 17, 33) the last tile row holds only the diagonal entry of the
// last column; it is summed with binary64 FMAs by the threads that convert
// that column instead, which leaves 2 MMA warps per sub-partition at
// ncols = 33.
constexpr int kDgPlanes = 12;
constexpr int kDgStageRows = 64;
constexpr int kDgKBlocks = kDgStageRows / 8;    // 8-row blocks per stage
constexpr int kDgChunkRows = 4096;              // scale granularity
constexpr int kDgChunkShift = 12;
constexpr int kDgFlushShift = 10;               // exact binary32 sums over 1024 rows
constexpr int kDgColPad = 48;                   // 3 m-tiles of 16 columns
constexpr int kDgTileWarps = 8;                 // MMA warps: one per tile (8 tiles at ncols = 33)
constexpr int kDgConvWarps = 8;                 // conversion warps
constexpr int kDgWarps = kDgTileWarps + kDgConvWarps;
constexpr int kDgThreads = kDgWarps * 32;
constexpr int kDgConvThreads = kDgConvWarps * 32;
// named barriers (0 is __syncthreads): stage buffer b full (1 + b) and
// empty (3 + b)
constexpr int kBarFull = 1, kBarEmpty = 3;
constexpr int kDgPlaneBytes = kDgKBlocks * kDgColPad * 16;             // 6,144
constexpr size_t kDgStageBytes = (size_t)kDgPlanes * kDgPlaneBytes;    // 73,728
// raw stage row stride (elements): 16-byte rows (for 16-byte copies and
// reads) whose 16-byte reads by 8 consecutive columns fall in distinct bank
// groups (528 or 272 bytes per column: 16 mod 128)
template <typename T>
constexpr int dg_raw_ld() { return sizeof(T) == 8 ? kDgStageRows + 2 : kDgStageRows + 4; }
template <typename T>
constexpr size_t dg_raw_bytes() { return (size_t)kMaxCols * dg_raw_ld<T>() * sizeof(T); }
template <typename T>
constexpr size_t dg_smem_bytes() { return 2 * kDgStageBytes + 2 * dg_raw_bytes<T>(); }  // 182,304 for binary64
static_assert(kDgChunkRows == (1 << kDgChunkShift) && kDgChunkShift >= kDgFlushShift &&
              (1 << kDgFlushShift) % kDgStageRows == 0, "chunk");
static_assert(kDgConvThreads == 32 * kDgKBlocks && kDgConvWarps == kDgKBlocks && kMaxCols <= 33,
              "conversion: one thread per (column < 32, 8-row block), column 32 split over the warps");
static_assert(kMaxCols <= 33, "tile layout assumes at most kDgTileWarps tiles");

// biased binary64 exponent of the value, at least 1 (zero and subnormals
// count as exponent 1: |y| = M 2^(max(E,1) - 1075)); 2047 for Inf/NaN
__device__ __forceinline__ int dg_exp(double y) {
  const int E = (int)(((unsigned long long)__double_as_longlong(y) >> 52) & 0x7ff);
  return E > 1 ? E : 1;
}

// 60-bit digit integer F of |y| at column exponent ce (see above)
__device__ __forceinline__ unsigned long long dg_fixed(double y, int ce) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(y);
  const int E = (int)((bits >> 52) & 0x7ff);
  if (E == 0x7ff) return 0ull;
  const unsigned long long M = (bits & ((1ull << 52) - 1)) | (E ? (1ull << 52) : 0ull);
  const int sh = (E > 1 ? E : 1) - ce + 7;  // <= 7
  if (sh >= 0) return M << sh;
  const int r = -sh;
  if (r > 54) return 0ull;
  return (M + (1ull << (r - 1))) >> r;
}

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], unsigned addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(unsigned (&r)[2], unsigned addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(addr));
}
__device__ __forceinline__ void mma_f16(float (&c)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
               : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// largest biased exponent (dg_exp) of every column within every chunk of
// kDgChunkRows rows: cexp[chunk * kMaxCols + column]
template <typename T>
__global__ void __launch_bounds__(256)
gram_chunk_exp_kernel(const T* __restrict__ Y, int64_t n, int64_t ld, const SolveState* __restrict__ st,
                      int ncols_fixed, int* __restrict__ cexp, int c0 = 0) {
  int ncols = ncols_fixed;
  if (ncols <= 0) {
    if (st->done) return;
    ncols = 2 * st->sbar + 1;
  }
  const int c = c0 + (int)blockIdx.y;   // columns c0 .. c0 + gridDim.y - 1
  if (c >= ncols) return;
  const int64_t r0 = (int64_t)blockIdx.x * kDgChunkRows;
  const T* col = Y + (int64_t)c * ld;
  int m = 1;
#pragma unroll 4
  for (int k = threadIdx.x; k < kDgChunkRows; k += 256) {
    const int64_t r = r0 + k;
    if (r < n) m = max(m, dg_exp(widen(__ldg(col + r))));
  }
  m = __reduce_max_sync(0xffffffffu, m);
  __shared__ int wm[8];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    int v = wm[0];
    for (int w = 1; w < 8; ++w) v = max(v, wm[w]);
    cexp[(int64_t)blockIdx.x * kMaxCols + c] = v;
  }
}

// Raw stage: every conversion thread copies, by cp.async, the rows it will
// convert (8 rows of column 8 (cw % 4) + lane % 8 from row 8 (4 (cw / 4) +
// lane / 8), and for ncols = 33 lanes 0..3 two rows of column 32) into
// [column][dg_raw_ld] of the stage buffer, zero filled past the thread
// block's last row; it later waits for its own copies only, so the conversion
// warps need no barrier among themselves.  vec16: Y 16-byte aligned and ld a
// multiple of 16 bytes / sizeof(T), so 16-byte copies (else one element per
// copy).
template <typename T>
__device__ __forceinline__ void cp_async_elems(unsigned dst, const T* src, int nvalid, int nelems, bool vec16) {
  constexpr int E = 16 / sizeof(T);  // elements per 16-byte copy
  if (vec16) {
    for (int q = 0; q < nelems; q += E) {
      int v = nvalid - q;
      v = v < 0 ? 0 : (v > E ? E : v);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst + (unsigned)(q * sizeof(T))),
                   "l"(v > 0 ? src + q : src), "r"(v * (int)sizeof(T))
                   : "memory");
    }
  } else {
    for (int q = 0; q < nelems; ++q) {
      const int v = q < nvalid ? (int)sizeof(T) : 0;
      if (sizeof(T) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst + (unsigned)(q * 8)),
                     "l"(v ? src + q : src), "r"(v)
                     : "memory");
      else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst + (unsigned)(q * 4)),
                     "l"(v ? src + q : src), "r"(v)
                     : "memory");
    }
  }
}

template <typename T>
__device__ __forceinline__ void dg_issue_raw(T* raw, const T* __restrict__ Y, int64_t ld, int64_t r0, int64_t r_end,
                                             int ncols, int cw, bool vec16) {
  constexpr int LD = dg_raw_ld<T>();
  const int lane = threadIdx.x & 31;
  const unsigned rbase = (unsigned)__cvta_generic_to_shared(raw);
  const int c = 8 * (cw & 3) + (lane & 7), kb = 4 * (cw >> 2) + (lane >> 3);
  if (c < ncols) {
    const int64_t row = r0 + 8 * kb;
    const int64_t nv = r_end - row;
    // rows past the end are zero filled; their source address is never read
    // but stays inside Y (row 0 of the column)
    cp_async_elems<T>(rbase + (unsigned)((c * LD + 8 * kb) * sizeof(T)), Y + (int64_t)c * ld + (nv > 0 ? row : 0),
                      nv < 0 ? 0 : (nv > 8 ? 8 : (int)nv), 8, vec16);
  }
  if (ncols > 32 && lane < 4) {
    const int64_t row = r0 + 8 * cw + 2 * lane;
    const int64_t nv = r_end - row;
    const int nvalid = nv < 0 ? 0 : (nv > 2 ? 2 : (int)nv);
    const unsigned dst = rbase + (unsigned)((32 * LD + 8 * cw + 2 * lane) * sizeof(T));
    // two elements: one 16-byte copy for binary64, element copies otherwise
    cp_async_elems<T>(dst, Y + 32 * ld + (nvalid > 0 ? row : 0), nvalid, 2, vec16 && sizeof(T) == 8);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// digit t (0 = most significant) of the 60-bit F = (h << 32) | l: bits
// 55 - 5t .. 59 - 5t
template <int t>
__device__ __forceinline__ unsigned dg_digit(unsigned h, unsigned l) {
  if constexpr (t < 5)
    return (h >> (23 - 5 * t)) & 31u;
  else if constexpr (t == 5)
    return __funnelshift_r(l, h, 30) & 31u;
  else
    return (l >> (55 - 5 * t)) & 31u;
}

// digits of 8 consecutive rows of one column (one 8-row block kb): plane t
// gets the 16-byte ldmatrix row (two f16 bit patterns per word, row 2w in
// the low half of word w)
__device__ __forceinline__ void dg_store8(const double (&v)[8], int ce, unsigned char* stage, int kb, int c) {
  unsigned h[8], l[8], sg[4];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const unsigned long long F = dg_fixed(v[k], ce);
    h[k] = (unsigned)(F >> 32);
    l[k] = (unsigned)F;
  }
#pragma unroll
  for (int w = 0; w < 4; ++w)
    sg[w] = (((unsigned)((unsigned long long)__double_as_longlong(v[2 * w]) >> 63)) << 15) |
            (((unsigned)((unsigned long long)__double_as_longlong(v[2 * w + 1]) >> 63)) << 31);
  unsigned char* row = stage + (kb * kDgColPad + c) * 16;
#define DG_PLANE(t)                                                                                      \
  *reinterpret_cast<uint4*>(row + (t) * kDgPlaneBytes) =                                                 \
      make_uint4(dg_digit<t>(h[0], l[0]) | (dg_digit<t>(h[1], l[1]) << 16) | sg[0],                      \
                 dg_digit<t>(h[2], l[2]) | (dg_digit<t>(h[3], l[3]) << 16) | sg[1],                      \
                 dg_digit<t>(h[4], l[4]) | (dg_digit<t>(h[5], l[5]) << 16) | sg[2],                      \
                 dg_digit<t>(h[6], l[6]) | (dg_digit<t>(h[7], l[7]) << 16) | sg[3]);
  DG_PLANE(0) DG_PLANE(1) DG_PLANE(2) DG_PLANE(3) DG_PLANE(4) DG_PLANE(5)
  DG_PLANE(6) DG_PLANE(7) DG_PLANE(8) DG_PLANE(9) DG_PLANE(10) DG_PLANE(11)
#undef DG_PLANE
}

// digits of 2 consecutive rows (2 w4, 2 w4 + 1 of block kb) of one column:
// word w4 of every plane's ldmatrix row
__device__ __forceinline__ void dg_store2(double v0, double v1, int ce, unsigned char* stage, int kb, int c, int w4) {
  const unsigned long long F0 = dg_fixed(v0, ce), F1 = dg_fixed(v1, ce);
  const unsigned h0 = (unsigned)(F0 >> 32), l0 = (unsigned)F0;
  const unsigned h1 = (unsigned)(F1 >> 32), l1 = (unsigned)F1;
  const unsigned sgn = (((unsigned)((unsigned long long)__double_as_longlong(v0) >> 63)) << 15) |
                       (((unsigned)((unsigned long long)__double_as_longlong(v1) >> 63)) << 31);
  unsigned* wb = reinterpret_cast<unsigned*>(stage + (kb * kDgColPad + c) * 16) + w4;
  constexpr int kPW = kDgPlaneBytes / 4;
#define DG_WORD(t) wb[(t) * kPW] = dg_digit<t>(h0, l0) | (dg_digit<t>(h1, l1) << 16) | sgn;
  DG_WORD(0) DG_WORD(1) DG_WORD(2) DG_WORD(3) DG_WORD(4) DG_WORD(5)
  DG_WORD(6) DG_WORD(7) DG_WORD(8) DG_WORD(9) DG_WORD(10) DG_WORD(11)
#undef DG_WORD
}

// Conversion of one stage by the conversion threads ct = 0..255: thread
// (warp cw, lane) takes column 8 (cw % 4) + lane % 8 and 8-row block
// 4 (cw / 4) + lane / 8 (8 consecutive columns per 8-lane phase: the 16-byte
// shared stores do not conflict); column 32 (ncols = 33) is split over the
// warps, warp cw taking its block cw with lanes 0..3 (two rows each).
template <typename T>
__device__ __forceinline__ void dg_convert(const T* raw, unsigned char* stage, const int* __restrict__ ce_g,
                                           int ncols, int cw, bool diag_fp64, double& dg) {
  constexpr int LD = dg_raw_ld<T>();
  const int lane = threadIdx.x & 31;
  const int c = 8 * (cw & 3) + (lane & 7), kb = 4 * (cw >> 2) + (lane >> 3);
  if (c < ncols) {
    const T* src = raw + c * LD + 8 * kb;  // 16-byte aligned
    double v[8];
    if (sizeof(T) == 8) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double2 p = reinterpret_cast<const double2*>(src)[k];
        v[2 * k] = p.x;
        v[2 * k + 1] = p.y;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const float4 p = reinterpret_cast<const float4*>(src)[k];
        v[4 * k] = widen(p.x);
        v[4 * k + 1] = widen(p.y);
        v[4 * k + 2] = widen(p.z);
        v[4 * k + 3] = widen(p.w);
      }
    }
    if (diag_fp64 && c == ncols - 1) {
#pragma unroll
      for (int k = 0; k < 8; ++k) dg = fma(v[k], v[k], dg);
    }
    dg_store8(v, __ldg(ce_g + c), stage, kb, c);
  }
  if (ncols > 32 && lane < 4) {
    const T* src = raw + 32 * LD + 8 * cw + 2 * lane;
    const double v0 = widen(src[0]), v1 = widen(src[1]);
    if (diag_fp64) dg = fma(v1, v1, fma(v0, v0, dg));
    dg_store2(v0, v1, __ldg(ce_g + 32), stage, cw, 32, lane);
  }
}

// v 2^k for any k a sum of two exponents can give (two factors when 2^k
// itself is out of the normal range)
__device__ __forceinline__ double dg_scale(double v, int k) {
  return (k >= -1022 && k <= 1023) ? v * pow2(k) : (v * pow2(k / 2)) * pow2(k - k / 2);
}

// add the digit sums of this lane's four tile entries into gacc (binary64)
// and clear them.  Each H_u is an integer times 2^-48 below 2^24 2^-48, so
// 2^48 H_u converts to int32 exactly; Horner in base 32 over u = 0..5 and
// u = 6..11 gives two integers below 2^49 (exact in int64 and in binary64),
// and G_ij += 2^(ce_i + ce_j - 2006) (S_hi 2^-73 + S_lo 2^-103).
__device__ __forceinline__ void dg_flush(float (&acc)[kDgPlanes][4], double (&gacc)[4], const int* ce_s, int ncols,
                                         int m0, int n0, int g, int tig) {
  constexpr int kHalf = kDgPlanes / 2;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int i = m0 + g + (e >> 1) * 8, j = n0 + 2 * tig + (e & 1);
    if (i < ncols && j < ncols && i <= j) {
      const int ci = ce_s[i], cj = ce_s[j];
      long long shi = 0, slo = 0;
#pragma unroll
      for (int u = 0; u < kHalf; ++u) {
        shi = shi * 32 + __float2int_rz(acc[u][e] * 0x1p48f);
        slo = slo * 32 + __float2int_rz(acc[u + kHalf][e] * 0x1p48f);
      }
      const int k = ci + cj - 2006;
      double& ge = gacc[e];
      if (ci == 2047 || cj == 2047) {
        ge = __longlong_as_double(0x7ff8000000000000ll);
      } else {
        if (shi != 0) ge += dg_scale((double)shi, k - 5 * (kHalf - 1) - 48);
        if (slo != 0) ge += dg_scale((double)slo, k - 5 * (kDgPlanes - 1) - 48);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kDgPlanes; ++u) acc[u][0] = acc[u][1] = acc[u][2] = acc[u][3] = 0.f;
}

// all digit products of one 64-row stage for this warp's tile
__device__ __forceinline__ void dg_mma_stage(float (&acc)[kDgPlanes][4], unsigned sbase, unsigned a_off,
                                             unsigned b_off) {
#pragma unroll 1
  for (int ks = 0; ks < kDgKBlocks / 2; ++ks) {
    const unsigned kofs = (unsigned)(ks * 2 * kDgColPad * 16);
    unsigned bf[kDgPlanes][2];
#pragma unroll
    for (int s = 0; s < kDgPlanes; ++s) ldsm_x2(bf[s], sbase + s * kDgPlaneBytes + kofs + b_off);
#pragma unroll
    for (int s = 0; s < kDgPlanes; ++s) {
      unsigned af[4];
      ldsm_x4(af, sbase + s * kDgPlaneBytes + kofs + a_off);
#pragma unroll
      for (int q = 0; q < kDgPlanes - s; ++q) mma_f16(acc[s + q], af, bf[q]);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kDgThreads, 1)
gram_partial_dg_kernel(const T* __restrict__ Y, int64_t n, int64_t ld, const SolveState* __restrict__ st,
                       int ncols_fixed, const int* __restrict__ cexp, double* __restrict__ partials, bool vec16) {
  int ncols = ncols_fixed;
  if (ncols <= 0) {
    if (st->done) return;
    ncols = 2 * st->sbar + 1;
  }
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int g = lane >> 2, tig = lane & 3;
  const bool conv = warp >= kDgTileWarps;

  // tiles (mt, nt) with nt >= 2 mt, in order; the diagonal-only last tile row
  // (ncols = 16 m + 1) is left to binary64
  const int MT = (ncols + 15) >> 4, NT = (ncols + 7) >> 3;
  const bool diag_fp64 = (ncols & 15) == 1;
  int ntiles = 0, mt = 0, nt = 0;
  for (int a = 0; a < MT; ++a) {
    if (diag_fp64 && a == MT - 1) break;
    for (int b = 2 * a; b < NT; ++b) {
      if (ntiles == warp) {
        mt = a;
        nt = b;
      }
      ++ntiles;
    }
  }
  const bool mma_warp = !conv && warp < ntiles;
  const int m0 = 16 * mt, n0 = 8 * nt;

  extern __shared__ __align__(16) unsigned char dg_smem[];
  T* raw[2] = {reinterpret_cast<T*>(dg_smem + 2 * kDgStageBytes),
               reinterpret_cast<T*>(dg_smem + 2 * kDgStageBytes + dg_raw_bytes<T>())};
  __shared__ int ce_buf[2][kMaxCols];  // exponents of the stage in digit buffer b
  __shared__ double dred[kDgThreads];

  const int64_t nst_all = (n + kDgStageRows - 1) / kDgStageRows;
  const int64_t spb = (nst_all + gridDim.x - 1) / gridDim.x;
  const int64_t r_begin = (int64_t)blockIdx.x * spb * kDgStageRows;
  int64_t r_end = r_begin + spb * kDgStageRows;
  if (r_end > n) r_end = n;
  const int64_t nst = r_begin < r_end ? (r_end - r_begin + kDgStageRows - 1) / kDgStageRows : 0;

  // both digit buffers zero: columns >= ncols are never written again
  for (int e = t; e < (int)(2 * kDgStageBytes / 16); e += kDgThreads)
    reinterpret_cast<uint4*>(dg_smem)[e] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();

  double dg = 0.0;  // binary64 diagonal entry of the last column (diag_fp64)
  double gacc[4] = {0.0, 0.0, 0.0, 0.0};
  if (conv) {
    // ---- conversion warps: stage k into digit buffer k & 1.  Every stage
    // commits one cp.async group (possibly empty), so "wait_group 1" means
    // that raw stage k has landed.
    const int ct = t - kDgTileWarps * 32, cw = warp - kDgTileWarps;
    dg_issue_raw(raw[0], Y, ld, r_begin, r_end, ncols, cw, vec16);
    dg_issue_raw(raw[1], Y, ld, r_begin + kDgStageRows, r_end, ncols, cw, vec16);
    for (int64_t k = 0; k < nst; ++k) {
      const int b = (int)(k & 1);
      const int64_t r0 = r_begin + k * kDgStageRows;
      const int* ce_g = cexp + (r0 >> kDgChunkShift) * kMaxCols;
      asm volatile("cp.async.wait_group 1;" ::: "memory");  // this thread's rows of stage k have landed
      if (k >= 2) bar_sync(kBarEmpty + b, kDgThreads);      // the MMA warps are done with stage k - 2
      if (ct < ncols) ce_buf[b][ct] = __ldg(ce_g + ct);
      dg_convert(raw[b], dg_smem + (size_t)b * kDgStageBytes, ce_g, ncols, cw, diag_fp64, dg);
      dg_issue_raw(raw[b], Y, ld, r0 + 2 * kDgStageRows, r_end, ncols, cw, vec16);  // own rows, read above
      bar_arrive(kBarFull + b, kDgThreads);                 // digit buffer b holds stage k
    }
    // the empty signals of the last two stages
    for (int64_t k = nst > 2 ? nst - 2 : 0; k < nst; ++k) bar_sync(kBarEmpty + (int)(k & 1), kDgThreads);
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else {
    // ---- MMA warps
    const unsigned smem0 = (unsigned)__cvta_generic_to_shared(dg_smem);
    // per-lane ldmatrix row offsets within a plane (k-step 0): x4 matrices
    // (m0..+7, kb0), (m0+8..+15, kb0), (m0..+7, kb0+1), (m0+8..+15, kb0+1);
    // x2 matrices (n0..+7, kb0), (n0..+7, kb0+1)
    const unsigned a_off = (unsigned)(((lane >> 4) * kDgColPad + m0 + ((lane >> 3) & 1) * 8 + (lane & 7)) * 16);
    const unsigned b_off = (unsigned)((((lane >> 3) & 1) * kDgColPad + n0 + (lane & 7)) * 16);
    float acc[kDgPlanes][4];
#pragma unroll
    for (int u = 0; u < kDgPlanes; ++u) acc[u][0] = acc[u][1] = acc[u][2] = acc[u][3] = 0.f;
    for (int64_t k = 0; k < nst; ++k) {
      const int b = (int)(k & 1);
      const int64_t r0 = r_begin + k * kDgStageRows, r1 = r0 + kDgStageRows;
      bar_sync(kBarFull + b, kDgThreads);
      if (mma_warp) {
        dg_mma_stage(acc, smem0 + (unsigned)(b * kDgStageBytes), a_off, b_off);
        // exact binary32 sums end at every 1024-row boundary and at the end
        if (k + 1 == nst || (r1 >> kDgFlushShift) != (r0 >> kDgFlushShift))
          dg_flush(acc, gacc, ce_buf[b], ncols, m0, n0, g, tig);
      }
      bar_arrive(kBarEmpty + b, kDgThreads);
    }
  }
  __syncthreads();

  // binary64 diagonal entry of the last column: fixed-order sum over threads
  if (diag_fp64) {
    dred[t] = dg;
    __syncthreads();
    if (t == 0) {
      double s = 0.0;
      for (int k = 0; k < kDgThreads; ++k) s += dred[k];
      const int i = ncols - 1;
      partials[(int64_t)blockIdx.x * kMaxPairs + i * ncols - i * (i - 1) / 2] = s;
    }
  }
  if (mma_warp) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int i = m0 + g + (e >> 1) * 8, j = n0 + 2 * tig + (e & 1);
      if (i < ncols && j < ncols && i <= j)
        partials[(int64_t)blockIdx.x * kMaxPairs + i * ncols - i * (i - 1) / 2 + (j - i)] = gacc[e];
    }
  }
}

// ------------------------------------------------------------------------
// The digit Gram on the 5th-generation tensor cores (gram_mode = 3).
//
// Columns 0..31: the 60-bit integers F of gram_mode 2 (the same per-value,
// per-chunk scales), here written as ten signed 6-bit digits (|d| <= 63) as
// f16 subnormals, with exact binary32 sums of digit products combined in two
// 64-bit integers per entry and added in binary64 once per 4096-row scale
// chunk (each accumulator sums a single plane pair: below 4096 * 63^2 < 2^24,
// exact), run as tcgen05.mma (kind::f16, M = 128, N = 128 or 64, K = 16, f32
// accumulators in tensor memory) issued by one thread.  Since
// H_u = sum_{s+t=u} D_s^T D_t (D_s the digit plane s of the columns) is
// symmetric, it is formed from the pairs s <= t only:
//   H_u = sum_{s<t, s+t=u} (X_st + X_st^T) + [u even] X_{u/2,u/2},
//   X_st = D_s^T D_t,
// 30 plane pairs (s + t <= 9; the pairs beyond weigh at most about 2^-57 of
// the product of the two columns' largest values per row).  Each MMA takes
// four consecutive planes on the A side (planes a..a+3 x 32 columns = 128
// rows) and four or two on the B side, so block (k, l) of its accumulator is
// X_{a+k, b+l}; the four accumulators (a, b) = (0, 0), (0, 4) (N = 128) and
// (0, 8), (4, 4) (N = 64, planes b, b+1) hold every pair with s <= t and
// s + t <= 9 in 384 tensor-memory columns.  Four MMAs per 16 rows; 30 of the
// 48 plane-pair blocks computed are used.  (Six-bit digits need ten planes
// where five-bit ones need twelve: a sixth less conversion work, a quarter
// less MMA work.)
// Column 32 (ncols = 33): its 33 entries are binary64 FMA sums (the FP64
// unit is otherwise idle here), formed by three warps from Y in global memory.
//
// Shared memory holds each 64-row stage in the no-swizzle canonical K-major
// layout: the 16-byte unit of 8 rows of (plane, column) at
// [8-row block][plane][column] (LBO = one 8-row block, 5,120 bytes; SBO = 128
// bytes between groups of 8 operand rows).
//
// Warp roles (768 threads): warp 0 allocates tensor memory and one of its
// threads issues the MMAs; warps 1..3 the column-32 dot products; warps 4..7
// the epilogue of each scale chunk (tcgen05.ld reaches lane quadrant w % 4
// from warp w); warps 8..23 stage and convert the rows (four rows per
// thread).  Hand-offs are mbarriers: full[b] (conversion -> MMA, per
// stage buffer), empty[b] (tcgen05.commit -> conversion), tfull
// (tcgen05.commit -> epilogue), tempty (epilogue -> MMA, before a block's
// first MMA overwrites the accumulators).  Every wait gives up after about a
// second of clock cycles, records the failure in g_gram_tc_error and lets the
// block finish (G is then not to be trusted; the flag is the error report).
constexpr int kTcStageRows = 64;
constexpr int kTcKB = kTcStageRows / 8;
constexpr int kTcCols = 32;
constexpr uint32_t kTcCore = 128;                                      // 8 rows x 16 bytes
constexpr uint32_t kTcPlaneBytes = (kTcCols / 8) * kTcCore;            // 512: one plane of 32 columns
constexpr int kTcPlanes = 10;                                          // six-bit digit planes
constexpr uint32_t kTcKBBytes = kTcPlanes * kTcPlaneBytes;             // 5,120: LBO
constexpr uint32_t kTcStage = kTcKB * kTcKBBytes;                      // 40,960
constexpr int kTcConvWarps = 16;                                       // conversion warps (4 rows per thread)
constexpr int kTcThreads = 32 * (8 + kTcConvWarps);                    // 768
constexpr int kTcC32W0 = 1, kTcEpi0 = 4, kTcConv0 = 8;                 // first column-32 / epilogue / conversion warp
constexpr uint32_t kTcTmemCols = 512;
constexpr int kTcAcc = 4;                                              // accumulators (a, b)
__device__ __constant__ int kTcAccA[kTcAcc] = {0, 0, 0, 4};
__device__ __constant__ int kTcAccB[kTcAcc] = {0, 4, 8, 4};
__device__ __constant__ int kTcAccL[kTcAcc] = {4, 4, 2, 2};            // B planes (N / 32)
__device__ __constant__ int kTcAccCol[kTcAcc] = {0, 128, 256, 320};    // tensor-memory column of each
static_assert(kTcStageRows == kDgStageRows, "the raw stages of gram_mode 2 are reused");
template <typename T>
constexpr size_t tc_smem_bytes() { return 2 * (size_t)kTcStage + 2 * dg_raw_bytes<T>(); }   // 116,768 for binary64

__device__ int g_gram_tc_error;   // set when a wait of gram_partial_tc_kernel gave up

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major; start, LBO and SBO in
// 16-byte units, descriptor version 1 (bits 46-47) for tcgen05
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: f32 accumulator (bits 4-5 = 1), A and
// B f16 (0), both K-major, N / 8 at bits 17-22, M / 16 at bits 24-28
constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
               "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
// wait for the phase of the given parity to complete, for about a second at
// most; a give-up is recorded (block-wide, so later waits return at once)
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, volatile int* abort) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile("{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
    if (ok) return true;
    if (*abort) return false;
    if (clock64() - t0 > 2000000000ll) {
      *abort = 1;
      atomicOr(&g_gram_tc_error, 1);
      return false;
    }
  }
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 8 consecutive accumulator columns of this warp's lane quadrant (raw bits)
__device__ __forceinline__ void tc_ld8(uint32_t (&r)[8], uint32_t taddr) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// six-bit digit t (0 = most significant) of the 60-bit F = (h << 32) | l:
// bits 54 - 6t .. 59 - 6t
template <int t>
__device__ __forceinline__ unsigned tc_digit(unsigned h, unsigned l) {
  constexpr int lo = 54 - 6 * t;
  if constexpr (lo >= 32)
    return (h >> (lo - 32)) & 63u;
  else if constexpr (lo + 6 <= 32)
    return (l >> lo) & 63u;
  else
    return __funnelshift_r(l, h, lo) & 63u;
}

// the 10 digit planes of 4 consecutive rows of one column: words 2h, 2h + 1
// of the 16-byte units unit + t * plane_stride
__device__ __forceinline__ void tc_store4(const double (&v)[4], int ce, unsigned char* unit, uint32_t plane_stride,
                                          int h2) {
  unsigned h[4], l[4], sg[2];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const unsigned long long F = dg_fixed(v[k], ce);
    h[k] = (unsigned)(F >> 32);
    l[k] = (unsigned)F;
  }
#pragma unroll
  for (int w = 0; w < 2; ++w)
    sg[w] = (((unsigned)((unsigned long long)__double_as_longlong(v[2 * w]) >> 63)) << 15) |
            (((unsigned)((unsigned long long)__double_as_longlong(v[2 * w + 1]) >> 63)) << 31);
  unsigned char* u = unit + 8 * h2;
#define TC_PLANE4(t)                                                                                      \
  *reinterpret_cast<uint2*>(u + (t) * plane_stride) =                                                     \
      make_uint2(tc_digit<t>(h[0], l[0]) | (tc_digit<t>(h[1], l[1]) << 16) | sg[0],                       \
                 tc_digit<t>(h[2], l[2]) | (tc_digit<t>(h[3], l[3]) << 16) | sg[1]);
  TC_PLANE4(0) TC_PLANE4(1) TC_PLANE4(2) TC_PLANE4(3) TC_PLANE4(4) TC_PLANE4(5)
  TC_PLANE4(6) TC_PLANE4(7) TC_PLANE4(8) TC_PLANE4(9)
#undef TC_PLANE4
}

// Conversion threads: warp cw (0..15), lane: column 8 (cw % 4) + lane % 8,
// 4-row group q = 4 (cw / 4) + lane / 8 (8-row block q / 2, half q % 2), so 8
// consecutive columns per 8-lane phase (the 8-byte shared stores do not
// conflict).  Each thread stages its own rows by cp.async into
// [column][dg_raw_ld] and waits for its own copies only.
__device__ __forceinline__ void tc_conv_slot(int cw, int lane, int& c, int& kb, int& h2) {
  c = 8 * (cw & 3) + (lane & 7);
  const int q = 4 * (cw >> 2) + (lane >> 3);
  kb = q >> 1;
  h2 = q & 1;
}

template <typename T>
__device__ __forceinline__ void tc_issue_raw(T* raw, const T* __restrict__ Y, int64_t ld, int64_t r0, int64_t r_end,
                                             int ncols, int cw, bool vec16) {
  constexpr int LD = dg_raw_ld<T>();
  int c, kb, h2;
  tc_conv_slot(cw, threadIdx.x & 31, c, kb, h2);
  if (c < ncols) {
    const int off = 8 * kb + 4 * h2;
    const int64_t row = r0 + off;
    const int64_t nv = r_end - row;
    // rows past the end are zero filled; their source address is never read
    // but stays inside Y (row 0 of the column)
    cp_async_elems<T>((unsigned)__cvta_generic_to_shared(raw) + (unsigned)((c * LD + off) * sizeof(T)),
                      Y + (int64_t)c * ld + (nv > 0 ? row : 0), nv < 0 ? 0 : (nv > 4 ? 4 : (int)nv), 4, vec16);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <typename T>
__device__ __forceinline__ void tc_convert(const T* raw, unsigned char* stage, const int* __restrict__ ce_g,
                                           int ncols, int cw) {
  constexpr int LD = dg_raw_ld<T>();
  int c, kb, h2;
  tc_conv_slot(cw, threadIdx.x & 31, c, kb, h2);
  if (c < ncols) {
    const T* src = raw + c * LD + 8 * kb + 4 * h2;
    double v[4];
    if (sizeof(T) == 8) {
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const double2 p = reinterpret_cast<const double2*>(src)[k];
        v[2 * k] = p.x;
        v[2 * k + 1] = p.y;
      }
    } else {
      const float4 p = *reinterpret_cast<const float4*>(src);
      v[0] = widen(p.x);
      v[1] = widen(p.y);
      v[2] = widen(p.z);
      v[3] = widen(p.w);
    }
    tc_store4(v, ce_g[c], stage + kb * kTcKBBytes + c * 16, kTcPlaneBytes, h2);
  }
}

// Each accumulator sums one plane pair: below 3969 R for R rows, exact in
// binary32 up to R = 4227, so the block sums are read out once per scale
// chunk (4096 rows), where the scales change.
constexpr int kTcFlushShift = kDgChunkShift;
static_assert((1 << kTcFlushShift) * 63 * 63 < (1 << 24), "exact binary32 sums of one plane pair");

// whether stage rows r0..r0+63 end a flush block within [.., r_end)
__device__ __forceinline__ bool tc_block_end(int64_t r0, int64_t r_end) {
  const int64_t r1 = r0 + kTcStageRows;
  return r1 >= r_end || (r1 >> kTcFlushShift) != (r0 >> kTcFlushShift);
}

// BATCH = false: one basis Y (n rows), thread blocks over contiguous ranges of
// 64-row stages, scales from the pre-pass (cexp, per 4096-row chunk).
// BATCH = true: thread block g is Gram block g of a batch (one pair's
// v.gram_rows rows, at most 16,384), its column scales computed here over its
// own rows, its partials in row g of `partials`.
template <typename T, bool BATCH>
__global__ void __launch_bounds__(kTcThreads, 1)
gram_partial_tc_kernel(const T* __restrict__ Y, int64_t n, int64_t ld, const SolveState* __restrict__ st,
                       int ncols_fixed, const int* __restrict__ cexp, double* __restrict__ partials, bool vec16,
                       BatchView v) {
  int ncols = ncols_fixed;
  int64_t r_begin, r_end;
  __shared__ int ce_blk[kMaxCols];   // BATCH: the block's column scales
  if (BATCH) {
    const int j = v.gblk_pair[blockIdx.x];
    const BatchPair& bp = v.pairs[j];
    const SolveState* sj = v.states + j;
    if (sj->done) return;
    ncols = 2 * sj->sbar + 1;
    Y += bp.off;
    n = bp.n;
    // 16-byte copies need every column of this pair 16-byte aligned
    vec16 = vec16 && ((uintptr_t)Y % 16 == 0);
    r_begin = (int64_t)(blockIdx.x - bp.gblk0) * v.gram_rows;
    r_end = r_begin + v.gram_rows < n ? r_begin + v.gram_rows : n;
  } else {
    if (ncols <= 0) {
      if (st->done) return;
      ncols = 2 * st->sbar + 1;
    }
    const int64_t nst_all = (n + kTcStageRows - 1) / kTcStageRows;
    const int64_t spb = (nst_all + gridDim.x - 1) / gridDim.x;
    r_begin = (int64_t)blockIdx.x * spb * kTcStageRows;
    r_end = r_begin + spb * kTcStageRows;
    if (r_end > n) r_end = n;
  }
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const bool c32 = ncols > kTcCols;
  const int np = ncols * (ncols + 1) / 2;
  const int nct = ncols < kTcCols ? ncols : kTcCols;   // columns on the tensor cores

  extern __shared__ __align__(1024) unsigned char tc_smem[];
  T* raw[2] = {reinterpret_cast<T*>(tc_smem + 2 * kTcStage),
               reinterpret_cast<T*>(tc_smem + 2 * kTcStage + dg_raw_bytes<T>())};
  __shared__ __align__(8) uint64_t bars[7];          // full[2], empty[2], tfull, tempty, drain
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ unsigned long long s_hi[kMaxPairs], s_lo[kMaxPairs];
  __shared__ double gacc[kMaxPairs];
  __shared__ double c32sum[1][kMaxCols];
  const uint32_t b_full = smem_addr(&bars[0]), b_empty = smem_addr(&bars[2]);
  const uint32_t b_tfull = smem_addr(&bars[4]), b_tempty = smem_addr(&bars[5]), b_drain = smem_addr(&bars[6]);

  const int64_t nst = r_begin < r_end ? (r_end - r_begin + kTcStageRows - 1) / kTcStageRows : 0;
  if (BATCH) {
    // the largest biased exponent (dg_exp) of every column over this block's rows
    for (int c = warp; c < ncols; c += kTcThreads / 32) {
      int m = 1;
      for (int64_t r = r_begin + lane; r < r_end; r += 32) m = max(m, dg_exp(widen(__ldg(Y + (int64_t)c * ld + r))));
      m = (int)__reduce_max_sync(0xffffffffu, (unsigned)m);
      if (lane == 0) ce_blk[c] = m;
    }
  }
  // scale exponents of the columns for the stage starting at row r0
  auto ce_for = [&](int64_t r0) -> const int* {
    return BATCH ? ce_blk : cexp + (r0 >> kDgChunkShift) * kMaxCols;
  };

  // both stage buffers zero (columns >= ncols are never written)
  for (int e = t; e < (int)(2 * kTcStage / 16); e += kTcThreads)
    reinterpret_cast<uint4*>(tc_smem)[e] = make_uint4(0u, 0u, 0u, 0u);
  for (int e = t; e < kMaxPairs; e += kTcThreads) {
    s_hi[e] = 0ull;
    s_lo[e] = 0ull;
    gacc[e] = 0.0;
  }
  if (t == 0) {
    abort_flag = 0;
    mbar_init(b_full, kTcConvWarps);   // one arrival per conversion warp
    mbar_init(b_full + 8, kTcConvWarps);
    mbar_init(b_empty, 1);
    mbar_init(b_empty + 8, 1);
    mbar_init(b_tfull, 1);
    mbar_init(b_tempty, 4);   // one arrival per epilogue warp
    mbar_init(b_drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"(kTcTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  volatile int* abort = &abort_flag;

  if (warp >= kTcConv0) {
    // ---- conversion warps (as in gram_partial_dg_kernel; buffer b = k & 1)
    const int cw = warp - kTcConv0;
    tc_issue_raw(raw[0], Y, ld, r_begin, r_end, nct, cw, vec16);
    tc_issue_raw(raw[1], Y, ld, r_begin + kTcStageRows, r_end, nct, cw, vec16);
    for (int64_t k = 0; k < nst; ++k) {
      const int b = (int)(k & 1);
      const int64_t r0 = r_begin + k * kTcStageRows;
      const int* ce_g = ce_for(r0);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
      if (k >= 2) mbar_wait(b_empty + 8 * b, (uint32_t)(((k - 2) >> 1) & 1), abort);   // MMAs of stage k - 2 done
      tc_convert(raw[b], tc_smem + (size_t)b * kTcStage, ce_g, nct, cw);
      tc_issue_raw(raw[b], Y, ld, r0 + 2 * kTcStageRows, r_end, nct, cw, vec16);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // digits visible to the tensor cores
      __syncwarp();
      if (lane == 0) mbar_arrive(b_full + 8 * b);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp == 0) {
    // ---- MMA issue (one thread)
    if (lane == 0) {
      const uint32_t sbase = smem_addr(tc_smem);
      constexpr uint32_t idesc128 = tc_idesc(128, 128), idesc64 = tc_idesc(128, 64);
      int64_t blk = -1;
      bool new_block = true;
      for (int64_t k = 0; k < nst; ++k) {
        const int b = (int)(k & 1);
        const int64_t r0 = r_begin + k * kTcStageRows;
        if (new_block) {
          ++blk;
          if (blk >= 1) mbar_wait(b_tempty, (uint32_t)((blk - 1) & 1), abort);   // previous block read out
        }
        mbar_wait(b_full + 8 * b, (uint32_t)((k >> 1) & 1), abort);
        tc_fence_after();
        const uint32_t stb = sbase + (uint32_t)b * kTcStage;
#pragma unroll
        for (int ks = 0; ks < kTcKB / 2; ++ks) {
          const uint32_t km = stb + (uint32_t)(2 * ks) * kTcKBBytes;
          const uint32_t acc = (new_block && ks == 0) ? 0u : 1u;
#pragma unroll
          for (int q = 0; q < kTcAcc; ++q) {
            const uint64_t da = tc_desc(km + (uint32_t)kTcAccA[q] * kTcPlaneBytes, kTcKBBytes, kTcCore);
            const uint64_t db = tc_desc(km + (uint32_t)kTcAccB[q] * kTcPlaneBytes, kTcKBBytes, kTcCore);
            tc_mma(tmem + (uint32_t)kTcAccCol[q], da, db, kTcAccL[q] == 4 ? idesc128 : idesc64, acc);
          }
        }
        tc_commit(b_empty + 8 * b);                     // stage buffer b may be refilled
        new_block = tc_block_end(r0, r_end);
        if (new_block) tc_commit(b_tfull);              // the block's sums are complete
      }
      // every MMA of this thread complete before tensor memory is freed
      tc_commit(b_drain);
      mbar_wait(b_drain, 0u, abort);
    }
    __syncwarp();
  } else if (warp < kTcEpi0) {
    // ---- column 32: binary64 FMA sums of y_i y_32, warp w taking i = 11 w .. 11 w + 10
    if (c32) {
      const int w = warp - kTcC32W0;
      double acc[11];
#pragma unroll
      for (int k = 0; k < 11; ++k) acc[k] = 0.0;
      for (int64_t r = r_begin + lane; r < r_end; r += 32) {
        const double y32 = widen(__ldg(Y + 32 * ld + r));
#pragma unroll
        for (int k = 0; k < 11; ++k) acc[k] = fma(widen(__ldg(Y + (int64_t)(11 * w + k) * ld + r)), y32, acc[k]);
      }
#pragma unroll
      for (int k = 0; k < 11; ++k) {
        double v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) c32sum[0][11 * w + k] = v;
      }
    }
  } else {
    // ---- epilogue: warp q = warp - 4 reads lane quadrant q: rows s = a + q
    // of accumulator (a, b), i = lane, column 32 l + j = (t = b + l, column j)
    const int q = warp - kTcEpi0, i = lane;
    int64_t blk = -1;
    for (int64_t k = 0; k < nst; ++k) {
      const int64_t r0 = r_begin + k * kTcStageRows;
      if (!tc_block_end(r0, r_end)) continue;
      ++blk;
      const int* ce_g = ce_for(r0);
      mbar_wait(b_tfull, (uint32_t)(blk & 1), abort);
      tc_fence_after();
      const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16);
      // Half a row of columns j at a time, summed over every plane-pair block
      // of this quadrant: 2^48 X is an integer below 2^24; u = s + t < 6 goes
      // to the high Horner sum (weight 64^(4 - u)), u >= 5 to the low one
      // (64^(9 - u)).  X_st (s < t) enters entry (min(i,j), max(i,j)) from
      // both (i, j) and (j, i) (twice on the diagonal); X_ss only once, from
      // i <= j.
#pragma unroll 1
      for (int half = 0; half < 4; ++half) {
        long long hi[8], lo[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) hi[jj] = lo[jj] = 0;
#pragma unroll 1
        for (int acc = 0; acc < kTcAcc; ++acc) {
          const int s = kTcAccA[acc] + q;
#pragma unroll 1
          for (int l = 0; l < kTcAccL[acc]; ++l) {
            const int tt = kTcAccB[acc] + l;
            if (s > tt || s + tt > 9) continue;        // uniform: pairs s <= t, s + t <= 9
            uint32_t x[8];
            tc_ld8(x, tq + (uint32_t)(kTcAccCol[acc] + 32 * l + 8 * half));
            tc_wait_ld();
            const int u = s + tt;
            const long long w = u < 5 ? (1ll << (6 * (4 - u))) : (1ll << (6 * (9 - u)));
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
              const int j = 8 * half + jj;
              if (s < tt || i <= j) {
                const long long v =
                    (long long)__float2int_rz(__uint_as_float(x[jj]) * 0x1p48f) * (s < tt && i == j ? 2 * w : w);
                if (u < 5) hi[jj] += v;
                else lo[jj] += v;
              }
            }
          }
        }
        if (i < nct) {
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int j = 8 * half + jj;
            if (j < nct) {
              const int a = i < j ? i : j, bb = i < j ? j : i;
              const int p = a * ncols - a * (a - 1) / 2 + (bb - a);
              if (hi[jj] != 0) atomicAdd(&s_hi[p], (unsigned long long)hi[jj]);
              if (lo[jj] != 0) atomicAdd(&s_lo[p], (unsigned long long)lo[jj]);
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(b_tempty);              // the accumulators may be overwritten
      bar_sync(1, 128);                                 // all four quadrants added
      for (int p = t - 32 * kTcEpi0; p < np; p += 128) {
        int pi, pj;
        pair_of(p, ncols, &pi, &pj);
        if (pj >= kTcCols) continue;                    // column 32: binary64 sums
        const long long shi = (long long)s_hi[p], slo = (long long)s_lo[p];
        s_hi[p] = 0ull;
        s_lo[p] = 0ull;
        const int ci_ = ce_g[pi], cj_ = ce_g[pj];
        if (ci_ == 2047 || cj_ == 2047) {
          gacc[p] = __longlong_as_double(0x7ff8000000000000ll);
        } else {
          // y_i y_j = F_i F_j 2^(ce_i + ce_j - 2164), F_i F_j = sum_u H_u 2^(108 - 6u):
          // the high sum at 2^84, the low one at 2^54
          const int kk = ci_ + cj_ - 2164;
          if (shi != 0) gacc[p] += dg_scale((double)shi, kk + 84);
          if (slo != 0) gacc[p] += dg_scale((double)slo, kk + 54);
        }
      }
      bar_sync(1, 128);                                 // sums cleared before the next block
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols));
  for (int p = t; p < np; p += kTcThreads) {
    int pi, pj;
    pair_of(p, ncols, &pi, &pj);
    const double v = pj >= kTcCols ? c32sum[0][pi] : gacc[p];
    partials[(int64_t)blockIdx.x * kMaxPairs + p] = v;
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

cudaError_t launch_batch_gram(const BatchView& v, const double* Y, int64_t LD, double* partials, cudaStream_t st,
                              int gram_mode) {
  if (gram_mode == 3) {
    if (v.gram_rows > (1 << 14)) return cudaErrorInvalidValue;   // exact binary32 sums of one plane pair
    const bool vec16 = ((uintptr_t)Y % 16 == 0) && ((size_t)LD * 8) % 16 == 0;
    gram_partial_tc_kernel<double, true><<<v.ngblk, kTcThreads, tc_smem_bytes<double>(), st>>>(
        Y, 0, LD, nullptr, 0, nullptr, partials, vec16, v);
  } else {
    batch_gram_partial_kernel<<<v.ngblk, kGramThreads, 0, st>>>(v, Y, LD, partials);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_gram_reduce_kernel<<<v.npairs, 256, 0, st>>>(v, partials);
  return cudaGetLastError();
}

cudaError_t launch_chunk_exp(const void* Y, int64_t n, int64_t ld, const SolveState* state, int c0, int count,
                             bool y32, int* chunk_exp, cudaStream_t st) {
  const int64_t nchunks = (n + kDgChunkRows - 1) / kDgChunkRows;
  if (c0 + count > kMaxCols) count = kMaxCols - c0;   // columns past the basis: nothing to do
  if (count < 1) return cudaSuccess;
  if (nchunks > 0x7fffffff || c0 < 0) return cudaErrorInvalidValue;
  const dim3 egrid((unsigned)nchunks, (unsigned)count);
  if (y32)
    gram_chunk_exp_kernel<float><<<egrid, 256, 0, st>>>(static_cast<const float*>(Y), n, ld, state, 0, chunk_exp,
                                                        c0);
  else
    gram_chunk_exp_kernel<double><<<egrid, 256, 0, st>>>(static_cast<const double*>(Y), n, ld, state, 0, chunk_exp,
                                                         c0);
  return cudaGetLastError();
}

cudaError_t launch_gram_reduce(const double* partials, int nblocks, const SolveState* state, int ncols_fixed,
                               double* G, int ldg, cudaStream_t st) {
  const int warps_per_block = 256 / 32;
  gram_reduce_kernel<<<(kMaxPairs + warps_per_block - 1) / warps_per_block, 256, 0, st>>>(partials, nblocks, state,
                                                                                          ncols_fixed, G, ldg);
  return cudaGetLastError();
}

int gram_blocks(int64_t n) {
  int64_t tiles = (n + kGramTileRows - 1) / kGramTileRows;
  int64_t b = kGramMaxBlocks;
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
  e = cudaFuncSetAttribute(gram_partial_dg_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)dg_smem_bytes<double>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(gram_partial_dg_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)dg_smem_bytes<float>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(gram_partial_tc_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tc_smem_bytes<double>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(gram_partial_tc_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tc_smem_bytes<float>());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(gram_partial_tc_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)tc_smem_bytes<double>());
  if (e != cudaSuccess) return e;
  done[dev] = true;
  return cudaSuccess;
}

cudaError_t gram_tc_error(int* flag, bool clear) {
  cudaError_t e = cudaMemcpyFromSymbol(flag, g_gram_tc_error, sizeof(int));
  if (e != cudaSuccess || !clear) return e;
  const int zero = 0;
  return cudaMemcpyToSymbol(g_gram_tc_error, &zero, sizeof(int));
}

int64_t gram_exp_ints(int64_t n) { return ((n + kDgChunkRows - 1) / kDgChunkRows) * kMaxCols; }

cudaError_t launch_gram(const void* Y, int64_t n, int64_t ld, const int* /*ncols_dev*/, int ncols_fixed,
                        const SolveState* state, double* partials, int nblocks, double* G, int ldg, bool y32,
                        cudaStream_t st, int gram_mode, int* chunk_exp, bool exp_ready) {
  if (gram_mode == 2 || gram_mode == 3) {
    if (!chunk_exp) return cudaErrorInvalidValue;
    const int64_t nchunks = (n + kDgChunkRows - 1) / kDgChunkRows;
    if (nchunks > 0x7fffffff) return cudaErrorInvalidValue;
    const dim3 egrid((unsigned)nchunks, ncols_fixed > 0 ? ncols_fixed : kMaxCols);
    // one block per SM, at most one block per 64-row stage
    const int64_t nstages = (n + kDgStageRows - 1) / kDgStageRows;
    int nb = nblocks < 152 ? nblocks : 152;
    if (nstages < nb) nb = (int)nstages;
    if (nb < 1) nb = 1;
    nblocks = nb;
    const size_t esz = y32 ? 4 : 8;
    const bool vec16 = ((uintptr_t)Y % 16 == 0) && ((size_t)ld * esz) % 16 == 0;
    if (y32) {
      if (!exp_ready)
        gram_chunk_exp_kernel<float><<<egrid, 256, 0, st>>>(static_cast<const float*>(Y), n, ld, state,
                                                            ncols_fixed, chunk_exp);
      if (gram_mode == 3)
        gram_partial_tc_kernel<float, false><<<nblocks, kTcThreads, tc_smem_bytes<float>(), st>>>(
            static_cast<const float*>(Y), n, ld, state, ncols_fixed, chunk_exp, partials, vec16, BatchView{});
      else
        gram_partial_dg_kernel<float><<<nblocks, kDgThreads, dg_smem_bytes<float>(), st>>>(
            static_cast<const float*>(Y), n, ld, state, ncols_fixed, chunk_exp, partials, vec16);
    } else {
      if (!exp_ready)
        gram_chunk_exp_kernel<double><<<egrid, 256, 0, st>>>(static_cast<const double*>(Y), n, ld, state,
                                                             ncols_fixed, chunk_exp);
      if (gram_mode == 3)
        gram_partial_tc_kernel<double, false><<<nblocks, kTcThreads, tc_smem_bytes<double>(), st>>>(
            static_cast<const double*>(Y), n, ld, state, ncols_fixed, chunk_exp, partials, vec16, BatchView{});
      else
        gram_partial_dg_kernel<double><<<nblocks, kDgThreads, dg_smem_bytes<double>(), st>>>(
            static_cast<const double*>(Y), n, ld, state, ncols_fixed, chunk_exp, partials, vec16);
    }
  } else if (gram_mode == 1) {
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
