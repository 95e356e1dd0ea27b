// Internal declarations shared by the libsscg translation units.
//
// Layout of the s-step basis in device memory: Y is column major with leading
// dimension ld (n rounded up to a multiple of 32), 2*sigma+1 columns, stored in
// the interleaved order [P_0, R_0, P_1, R_1, ..., P_{s-1}, R_{s-1}, P_s]; column
// 2l is P_l and column 2l+1 is R_l, so the basis of the first l inner steps is
// the leading 2l+1 columns (Carson 2019, eq. (reqsub)).  Columns 0 and 1 hold
// the current p and r between outer loops.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sscg.h"

namespace sscg {

constexpr int kMaxS = SSCG_MAX_S;
constexpr int kMaxCols = 2 * kMaxS + 1;                    // 33
constexpr int kMaxPairs = kMaxCols * (kMaxCols + 1) / 2;   // 561
constexpr int kGramThreads = 576;                          // >= kMaxPairs, multiple of 32
constexpr int kGramTileRows = 128;
constexpr int kGramMaxBlocks = 152 * 2;   // most thread blocks (and partial sums per pair) of one Gram

// ---------------------------------------------------------------- operator
// A sparse SPD operator: a CSR matrix or a 2D/3D face-coefficient stencil.
struct Operator {
  int kind;            // 0 = CSR, 1 = stencil
  int64_t n;
  // CSR
  const int64_t* rowptr;
  const int32_t* col;
  const double* val;
  // the same CSR matrix in sliced ELL (slices of kSliceRows rows, rows sorted
  // by length within windows of kSliceWindow rows): lane t of slice s owns
  // row s_row[32 s + t] (-1: padding), whose j-th entry sits at
  // s_off[s] + 32 j + t of s_col / s_val; s_len[s] = the slice's longest row
  int64_t nslices;
  const int32_t* s_row;
  const int64_t* s_off;
  const int32_t* s_len;
  const int32_t* s_col;
  const double* s_val;
  // stencil: cells x fastest; kx [nz][ny][nx+1], ky [nz][ny+1][nx], kz [nz+1][ny][nx]
  int dim, nx, ny, nz;
  const double* kx;
  const double* ky;
  const double* kz;
  const double* diag;  // sum of the faces of each cell (the diagonal of A)
};

constexpr int kSliceRows = 32;     // one warp per slice
constexpr int kSliceWindow = 256;  // rows sorted by length within each window

// binary32 -> binary64, exact, by integer operations on the bits only (the
// FP64 unit's own conversion costs a 64-cycle binary64 slot per warp on
// GB300): normal numbers rebias the exponent; a subnormal m 2^-149 is
// renormalised at its leading bit p (value 2^(p-149) (1 + ...)); zero, Inf and
// NaN keep their class (NaN payloads are kept as they are)
__device__ __forceinline__ double widen(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xffu;
  const unsigned int m = u & 0x7fffffu;
  const int p = 31 - __clz(m | 1u);  // leading bit of a subnormal's mantissa
  const unsigned long long m_norm = (unsigned long long)m << 29;
  const unsigned long long m_sub = (unsigned long long)(m ^ (1u << p)) << (52 - p);
  const unsigned long long e_norm = e == 255u ? 2047ull : (unsigned long long)(e + 896u);
  const unsigned long long e_sub = m == 0u ? 0ull : (unsigned long long)(p + 874);
  const unsigned long long bits = ((unsigned long long)(u >> 31) << 63) |
                                  ((e == 0u ? e_sub : e_norm) << 52) | (e == 0u ? (m == 0u ? 0ull : m_sub) : m_norm);
  return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double widen(double d) { return d; }

// ------------------------------------------------------------ solver state
// Device-resident state of one s-step solve (Algorithm 5).  Only kernels read
// and write it during a solve; the host reads `done`/`status` to stop.
struct SolveState {
  // configuration
  int sigma, s0, f, basis, c_mode, newton_scale, cheb_params, inner_conv_check, variant;
  int max_outer, y_fp32, hist_cap;
  double tol, eps, kappa_cut, c_const;
  // running scalars
  int k;              // outer loop index (0-based) of the loop in progress
  int m;              // inner iterations done (global index of the next alpha)
  int sbar;           // s-bar_k of the loop in progress
  int stilde, sk;     // s-tilde_k, s_k of the last finished control step
  int done, status;
  int converged_est;  // coordinate estimate <= tol: a true-residual check is pending
  int replace_pending;
  int replacements;
  int have_ritz;      // basis parameters come from Ritz values (m > 1)
  int zero_rhs;       // b = 0: x = 0 is returned without iterating
  // FP32-stored basis: periodic residual replacement (r := b - A x, p kept)
  double fp32_drop, rho_last;
  double prev_fail;   // relative true residual at the last failed convergence check
  int gram_mode;      // 0: binary64 Gram; 1: binary32-pair products; 2, 3: f16 digit products (mma.sync, tcgen05)
  int mpk_fp64_per16; // warps (of 16) on the binary64 FMA chain in stencil levels; -1: library default
  int rec_fp64_per16; // row groups (of 16) on the binary64 FMA chains in the recovery; -1: library default
  int recompute_y;    // 1: no stored basis (recompute.cu)
  int fp32_replace_pending, fp32_replacements;
  double c, psi, normb, upd_relres;
  // Meurant-Tichy state (Algs. 3-4)
  int mt_n;
  double up_omega, up_h;
  double lo_omega, lo_a, lo_d, lo_g, lo_h;
  double alpha_prev, zeta_prev, beta_prev;
  double lmin, lmax;
  // exact Ritz values (ritz_exact = 1): T_m of eq. (T) kept as its diagonal
  // ritz_d[0..m) and squared off-diagonal ritz_e2[0..m-1), room for ritz_cap rows
  int ritz_exact, ritz_cap;
  double* ritz_d;
  double* ritz_e2;
  // recurrence coefficients of the loop in progress (eq. rho)
  double theta[kMaxS], gamma[kMaxS], inv_gamma[kMaxS], mu[kMaxS];
  // control output: coordinates of x - x_m, r, p in the basis (eq. coords)
  int nc;             // 2 s_k + 1 columns used by the recombination
  double xc[kMaxCols], rc[kMaxCols], pc[kMaxCols];
  // kappa step output (entry l = 1..sbar)
  double kappa[kMaxS + 1], glmin[kMaxS + 1], glmax[kMaxS + 1];
  // true residual check
  double rt2;
  unsigned int red_counter;   // arrival counter of the last-block reductions
  // HSCG comparator scalars
  double h_rr, h_pq, h_alpha, h_beta;
  int h_iters, h_max_iters;
};
static_assert(sizeof(SolveState) % sizeof(unsigned int) == 0, "SolveState is copied as 32-bit words");
static_assert(sizeof(SolveState) <= 4000, "SolveState travels as a kernel argument");

// ----------------------------------------------------------------- launchers
// operator kernels (ops_stencil.cu / ops_csr.cu)
// gmode: 0 = always run; 1 = only when a true-residual check is pending
// (state->converged_est and not done); 2 = only while iterating (not done and
// no check pending); 3 = only when an FP32-basis replacement is pending.
cudaError_t launch_spmv(const Operator& A, const double* v, double* y, cudaStream_t st,
                        const SolveState* gate = nullptr, int gmode = 0);
// diag_i = sum of the faces of cell i (the diagonal of a stencil operator)
cudaError_t launch_stencil_diag(const Operator& A, double* diag, cudaStream_t st);
// residual r = b - A x, written to r
cudaError_t launch_residual(const Operator& A, const double* b, const double* x, double* r,
                            cudaStream_t st, const SolveState* gate = nullptr, int gmode = 0);
// one matrix-powers level l (computes P_{l+1} and R_{l+1} when within the block size
// read from st->sbar, or from `sbar_fixed` when > 0, with coefficients from `coef`).
// Stencil levels with a binary64 basis: fp64_per16 of every 16 warps form the
// binary64 FMA chain, the others exact integer products (16: FMA chain only;
// negative: kMpkFp64Per16).
struct LevelCoef { const double* theta; const double* inv_gamma; const double* mu; };
constexpr int kMpkFp64Per16 = 8;
cudaError_t launch_mpk_level(const Operator& A, void* Y, int64_t ld, int level,
                             const SolveState* state, int sbar_fixed, LevelCoef coef, bool y32,
                             cudaStream_t st, int fp64_per16 = -1);
// y = A v with a stencil's cells split the same way (fp64_per16 as above; CSR
// operators, 16, and grids beyond the launch's extents take launch_spmv)
bool spmv_split_supported(const Operator& A);
cudaError_t launch_spmv_split(const Operator& A, const double* v, double* y, cudaStream_t st,
                              const SolveState* gate, int gmode, int fp64_per16);

// gram.cu
int gram_blocks(int64_t n);
// G from per-block partial sums (nblocks x kMaxPairs, fixed order)
cudaError_t launch_gram_reduce(const double* partials, int nblocks, const SolveState* state, int ncols_fixed,
                               double* G, int ldg, cudaStream_t st);

// recompute.cu: the outer loop without a stored basis (2D stencils).  PR
// holds p (column 0) and r (column 1) with leading dimension n.
bool recompute_supported(const Operator& A);
int64_t recompute_partials(const Operator& A);     // doubles of partial sums
cudaError_t recompute_prepare();                   // shared-memory limits (once per device)
// coef (3 kMaxS doubles): the loop's recurrence coefficients, saved by the
// Gram pass for the recovery pass
cudaError_t launch_recompute_gram(const Operator& A, const double* PR, const SolveState* state, double* partials,
                                  double* coef, double* G, int ldg, cudaStream_t st);   // G (2 kernels)
cudaError_t launch_recompute_recover(const Operator& A, double* PR, double* PRnew, double* x,
                                     const SolveState* state, double* coef, cudaStream_t st);   // 1 kernel + copy
// per-device one-time setup of the gram_mode 1 and 2 kernels (shared memory
// above the 48 KB default); call outside stream capture, before launch_gram
cudaError_t gram_prepare();
// gram_mode 0: binary64 products and sums; 1: binary32-pair products on the
// FP32 pipes, compensated binary32 sums per tile, binary64 across tiles;
// 2: exact products of 5-bit digits on the f16 tensor cores (mma.sync), exact
// binary32 sums over 1024 rows, binary64 across them; 3: the same digit
// arithmetic as tcgen05.mma with tensor-memory accumulators (modes 2 and 3
// need `chunk_exp`, an int scratch of gram_exp_ints(n) entries).
int64_t gram_exp_ints(int64_t n);
// the give-up flag of the gram_mode 3 kernel's bounded waits (read, optionally cleared)
cudaError_t gram_tc_error(int* flag, bool clear);
cudaError_t launch_gram(const void* Y, int64_t n, int64_t ld, const int* ncols_dev, int ncols_fixed,
                        const SolveState* state, double* partials, int nblocks, double* G, int ldg,
                        bool y32, cudaStream_t st, int gram_mode = 0, int* chunk_exp = nullptr,
                        bool exp_ready = false);
// gram_mode 2, 3: the column scales of columns c0 .. c0 + count - 1 (those
// below the state's 2 s-bar + 1) into chunk_exp; launch_gram with exp_ready
// then skips its own pass over Y
cudaError_t launch_chunk_exp(const void* Y, int64_t n, int64_t ld, const SolveState* state, int c0, int count,
                             bool y32, int* chunk_exp, cudaStream_t st);

// control.cu
cudaError_t launch_kappa(const double* G, int ldg, const SolveState* state, int sbar_fixed,
                         double kappa_cut, double* kappa, double* lmin, double* lmax, int grid,
                         cudaStream_t st);
// ritz_exact: the step with exact Ritz values (state->ritz_exact = 1)
cudaError_t launch_control(SolveState* state, const double* G, int ldg, const double* leja,
                           sscg_outer_record* hist, cudaStream_t st, bool ritz_exact = false);
cudaError_t launch_leja(double* t, int s, cudaStream_t st);
// the device's table of the first kMaxS Leja points (computed on `st` by the
// first call on a device, a no-op kernel afterwards) and its device address
cudaError_t leja_table(const double** table, cudaStream_t st);

// vec.cu
// Basis storage: y32 = false: Y is double and columns 0/1 are p and r
// themselves; y32 = true: Y is float and p, r live in the binary64 vectors
// p64, r64 (columns 0/1 of Y hold their binary32 roundings).
// With a binary64 basis, fp64_per16 of every 16 groups of 32 rows are summed
// by binary64 FMAs and the others by exact integer dot products (16: FMA only;
// negative: kRecFp64Per16); a binary32 basis always takes the FMA chains.
constexpr int kRecFp64Per16 = 9;
cudaError_t launch_recombine(const SolveState* state, void* Y, int64_t ld, double* x, double* r64, double* p64,
                             int64_t n, bool y32, cudaStream_t st, int fp64_per16 = 16);
cudaError_t launch_init_state(SolveState* state, const Operator& A, const double* b, const double* x,
                              void* Y, int64_t ld, double* r64, double* p64, double* partials, int nblocks,
                              bool y32, cudaStream_t st);
cudaError_t launch_fp32_replacement(SolveState* state, const Operator& A, const double* b, const double* x,
                                    void* Y, int64_t ld, double* r64, double* partials, int nblocks,
                                    sscg_outer_record* hist, cudaStream_t st);
cudaError_t launch_true_residual(SolveState* state, const Operator& A, const double* b, const double* x,
                                 double* rt, double* partials, int nblocks, cudaStream_t st);
cudaError_t launch_apply_replacement(SolveState* state, const double* rt, void* Y, int64_t ld, double* r64,
                                     double* p64, int64_t n, bool y32, sscg_outer_record* hist, cudaStream_t st);
cudaError_t launch_final_norm(SolveState* state, const Operator& A, const double* b, const double* x,
                              double* rt, double* partials, int nblocks, cudaStream_t st);
// HSCG
cudaError_t launch_hscg_init(SolveState* state, const Operator& A, const double* b, const double* x,
                             double* r, double* p, double* partials, int nblocks, cudaStream_t st);
cudaError_t launch_hscg_iteration(SolveState* state, const Operator& A, double* x, double* r,
                                  double* p, double* q, double* partials, int nblocks,
                                  cudaStream_t st, int spmv_fp64_per16 = 16);
cudaError_t launch_hscg_check(SolveState* state, const Operator& A, const double* b, const double* x,
                              double* r, double* p, double* rt, double* partials, int nblocks,
                              cudaStream_t st);
int reduce_blocks(int64_t n);

// adjoint.cu
cudaError_t launch_face_grad(const Operator& A, const double* lam, const double* x, double* gkx, double* gky,
                             double* gkz, cudaStream_t st);
cudaError_t launch_csr_grad(const Operator& A, const double* lam, const double* x, double* gval, cudaStream_t st);


// ------------------------------------------------------------------ batches
// A batched solve runs many independent (system, right-hand side) pairs in
// lock-step outer loops.  Every vector of pair j lives at rows
// [off, off + n) of the concatenated arrays; basis column c of pair j starts
// at Y + c * LD + off.  Row work is cut into chunks of chunk_rows rows, each
// owned by one pair; the Gram uses its own blocks of gram_rows rows (both
// chosen per call, default kBatchChunk / kBatchGramRows).
constexpr int kBatchChunk = 2048;
constexpr int kBatchGramRows = 2048;

struct BatchPair {
  Operator op;      // the pair's system (operator storage owned by its handle)
  int64_t off, n;
  int chunk0, nchunk;
  int gblk0, ngblk;
};

struct BatchView {
  const BatchPair* pairs;
  int npairs;
  const int* chunk_pair;  // chunk -> pair
  int nchunks;
  const int* gblk_pair;   // Gram block -> pair
  int ngblk;
  SolveState* states;     // one per pair
  double* G;              // kMaxCols x kMaxCols per pair
  sscg_outer_record* hist;  // hist_cap records per pair, or null
  int hist_cap;
  unsigned int* active;   // pairs still iterating after the last outer loop
  unsigned int* bodies;   // outer loops run so far (all pairs)
  int max_bodies;
  int chunk_rows;         // rows per work chunk
  int gram_rows;          // rows per Gram block
};

// batch.cu / per-file batched kernels
// stencil pairs: fp64_per16 of every 16 groups of 32 rows on binary64 FMA
// chains, the others exact integer products (negative: kBatchMpkFp64Per16,
// all on FMA chains: without the single-system kernel's shared-memory tiles
// the integer form costs more than it saves here)
constexpr int kBatchMpkFp64Per16 = 16;
cudaError_t launch_batch_mpk(const BatchView& v, double* Y, int64_t LD, int level, cudaStream_t st,
                             int fp64_per16 = -1);
// gram_mode 0: binary64 FMAs; 3: the tcgen05 digit Gram (v.gram_rows <= 16384)
cudaError_t launch_batch_gram(const BatchView& v, const double* Y, int64_t LD, double* partials, cudaStream_t st,
                              int gram_mode = 0);
cudaError_t launch_batch_kappa(const BatchView& v, int sigma_max, cudaStream_t st);
cudaError_t launch_batch_control(const BatchView& v, const double* leja, cudaStream_t st);
cudaError_t launch_batch_recombine(const BatchView& v, double* Y, int64_t LD, double* x, cudaStream_t st,
                                   int fp64_per16 = -1);
cudaError_t launch_batch_check(const BatchView& v, const double* b, const double* x, double* rt, double* Y,
                               int64_t LD, double* partials, cudaStream_t st);
cudaError_t launch_batch_init(const BatchView& v, const double* b, double* x, double* Y, int64_t LD,
                              double* partials, cudaStream_t st);
cudaError_t launch_batch_begin(const BatchView& v, cudaStream_t st);
// batched HSCG (the comparator of the batched s-step solve)
cudaError_t launch_batch_hscg_init(const BatchView& v, const double* b, double* x, double* r, double* p,
                                   double* partials, cudaStream_t st);
cudaError_t launch_batch_hscg_iteration(const BatchView& v, double* x, double* r, double* p, double* q,
                                        double* partials, cudaStream_t st);
cudaError_t launch_batch_hscg_check(const BatchView& v, const double* b, const double* x, double* rt, double* r,
                                    double* p, double* partials, cudaGraphConditionalHandle cond, int use_cond,
                                    cudaStream_t st);
cudaError_t launch_batch_end(const BatchView& v, cudaGraphConditionalHandle cond, int use_cond, cudaStream_t st);
cudaError_t launch_batch_arm(cudaGraphConditionalHandle cond, cudaStream_t st);
cudaError_t launch_solve_cond(const SolveState* state, cudaGraphConditionalHandle cond, cudaStream_t st);
// *state = config, by a kernel on `st` (the configuration travels as a kernel argument)
cudaError_t launch_set_state(SolveState* state, const SolveState& config, cudaStream_t st);

}  // namespace sscg
