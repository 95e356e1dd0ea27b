/*
 * sscg.h - C ABI of libsscg: adaptive s-step conjugate gradient on one GB300.
 *
 * The method is the improved adaptive s-step CG of E. C. Carson, "An Adaptive
 * s-step Conjugate Gradient Algorithm with Dynamic Basis Updating" (2019),
 * Algorithm 5, for sparse symmetric positive definite A.  Every step of a solve
 * runs in this library's CUDA kernels; the host only enqueues work and polls a
 * device-side "done" flag.
 *
 * Conventions for every entry point
 *  - Return value: 0 (SSCG_OK) or a negative SSCG_ERR_* code; solver outcomes
 *    (SSCG_NOT_CONVERGED, SSCG_BREAKDOWN) are positive.  No C++ exception
 *    crosses this boundary.  sscg_strerror() names every code.
 *  - Floating point is IEEE binary64 throughout unless stated.
 *  - "device pointer" means memory of the current CUDA device (cudaMalloc or a
 *    torch CUDA tensor's data_ptr()); "host pointer" means ordinary host memory.
 *  - A handle owns a CUDA stream given at creation (NULL = the legacy default
 *    stream); all of its work is ordered on that stream.  Calls on one handle
 *    must not overlap from several host threads.
 *  - Vectors are dense, contiguous, length n, with the row numbering of A.
 */
#ifndef SSCG_H
#define SSCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SSCG_MAX_S 16 /* largest sigma (maximum s_k) the kernels support */

typedef struct sscg_ctx* sscg_t;

/* Polynomial basis of the s-step Krylov basis, Section 2 eqs. (rho),
 * (newtbasis), (chebbasis).  Until two iterations have run, Algorithm 5 uses
 * the monomial basis whatever is chosen here. */
typedef enum { SSCG_MONOMIAL = 0, SSCG_NEWTON = 1, SSCG_CHEBYSHEV = 2 } sscg_basis;

/* c in conditions (condy)/(newcondy): Alg. 5 sets c = max{1, lmax sqrt(psi/lmin)}
 * (eq. xiupd, SSCG_C_XI).  The other modes are the alternatives of Section 5.1:
 * the scale-consistent form max{1, lmax sqrt(psi)/lmin}, c = 1, c = lmax/lmin,
 * and a user constant. */
typedef enum { SSCG_C_XI = 0, SSCG_C_XI_SCALED = 1, SSCG_C_ONE = 2, SSCG_C_KAPPA_RATIO = 3,
               SSCG_C_CONST = 4 } sscg_c_mode;

/* Status codes. */
enum {
  SSCG_OK = 0,
  SSCG_BREAKDOWN = 2,        /* p'^T G B p' <= 0 at the first step of a block: A not SPD (numerically) */
  SSCG_NOT_CONVERGED = 3,    /* max_outer (or max_iters) reached, or stagnation above tol */
  SSCG_NONFINITE = 4,        /* a NaN or Inf in b, x0, A or the iteration */
  SSCG_ERR_INVALID_ARG = -1,
  SSCG_ERR_CUDA = -2,        /* a CUDA runtime call failed; sscg_last_cuda_error() has the text */
  SSCG_ERR_NO_MEMORY = -3,
  SSCG_ERR_UNSUPPORTED = -4
};

/* Options of Algorithm 5 and of the readings the library takes where the paper
 * leaves a choice.  sscg_opts_default() fills the defaults given per field. */
typedef struct {
  int s0;                /* initial s (s-bar_0, Alg. 5 input); default 0 = sigma */
  int f;                 /* maximum basis growth per outer loop (Alg. 5 input); default 0 = sigma */
  int max_outer;         /* outer-loop cap; default 100000 */
  int c_mode;            /* sscg_c_mode; default SSCG_C_XI */
  int newton_scale;      /* 0: gamma_l = (lmax - lmin)/4 (interval capacity); 1: gamma_l = 1 as printed; default 0 */
  int cheb_params;       /* 0: rho_l(z) = T_l((z-c)/h); 1: eq. (chebbasis) as printed; default 0 */
  int inner_conv_check;  /* 1: test sqrt(r'^T G r')/||b|| <= tol after every inner step; default 1 */
  int y_fp32;            /* 1: store the basis Y in binary32 (recurrence, Gram, x, r, p stay binary64;
                            r := b - A x whenever the residual estimate has fallen by 2^-4 since the
                            last such replacement); default 0 */
  int variant;           /* 0: Algorithm 5; 1: fixed s-step CG (s_k = sigma, no break test); 2: the previous
                            adaptive s-step CG, Algorithm 2 (basis never retuned from Ritz values, c = c_const,
                            break when kappa(Y_{k,s~}) >= tol/(c eps ||r||/||b||)); default 0 */
  int check_every;       /* outer loops enqueued between two polls of the done flag; default 4 */
  int use_graph;         /* 1: replay one outer loop as a CUDA graph; default 1 */
  int profile;           /* 1: time each kernel phase with CUDA events (direct launches); default 0 */
  double c_const;        /* c for SSCG_C_CONST; default 1 */
  double eps;            /* unit roundoff in (condy)/(newcondy); default 2^-53 */
  double kappa_cut;      /* kappa_l = inf when lambda_min(G_l) <= kappa_cut * lambda_max(G_l); default 2^-44 */
  int gram_mode;         /* 0: G by binary64 FMAs (the method as written); 1: binary32-pair products on the
                            FP32 pipes (each within ~2^-46 of Y_i Y_j), compensated binary32 sums over
                            256-row tiles, binary64 across tiles; 2: every value written as 12 signed
                            5-bit digits after a per-4096-row-chunk power-of-two column scale, all digit
                            products on the f16 tensor cores with exact binary32 sums over 1024 rows,
                            binary64 across them (normwise error below binary64 FMAs'); 3: the arithmetic of
                            mode 2 run as tcgen05.mma with the sums in tensor memory (the same G up to the
                            order of the final binary64 additions); default 0 */
  int batch_chunk_rows;  /* sscg_solve_batch only: rows per work chunk of the row kernels (matrix powers,
                            recombination, residual checks); 0 = 2048, else 128..1048576 */
  int batch_gram_rows;   /* sscg_solve_batch only: rows per Gram block; 0 = 2048, else 128..1048576 */
  int mpk_fp64_per16;    /* stencil matrix-powers levels with a binary64 basis (also the stencil pairs of
                            sscg_solve_batch, by groups of 32 rows): of every 16 warps, this many
                            form each cell's (A - theta I) v - mu v' as the binary64 FMA chain and the others
                            as exact integer products summed exactly and rounded once (both binary64-accurate;
                            the two share the level between GB300's FP64 unit and its integer pipes);
                            16 = FMA chain only, 0 = integer products only; default -1 = the library's
                            tuned share (8 for a single system; 16 in sscg_solve_batch, whose untiled
                            level gains nothing from the integer form) */
  int rec_fp64_per16;    /* the recovery x += Y x', r = Y r', p = Y p' (eq. coords) with a binary64 basis:
                            of every 16 groups of 32 rows, this many are summed by binary64 FMA chains and
                            the others as exact integer dot products rounded once per output (within
                            m (1 + 2^-5) 2^-54 of the largest term before that rounding, m <= 34 terms;
                            an FMA chain is bounded by m 2^-53 sum|terms|); 16 = FMA only, 0 = integer
                            only; default -1 = the library's tuned share */
  int ritz_exact;        /* 0: the extremal Ritz value estimates of Algorithms 3-4 (Section 4, the method as
                            written); 1: the extremal eigenvalues of T_m (eq. T) themselves after every inner
                            iteration, by multisection with Sturm counts on one thread block (O(m) binary64
                            operations per count, so the control step grows with the iteration count m; for
                            studies, not speed).  The solve stops SSCG_NOT_CONVERGED if m reaches
                            min(max_outer * s_max, 2^20).  Not supported by sscg_solve_batch.  Default 0 */
  int recompute_y;       /* 1: no stored basis (2D stencils, gram_mode 0, binary64 basis): each outer loop forms
                            the basis of eq. (rho) tile by tile from p and r with a halo of s-bar cells, once
                            to sum G = Y^T Y and once more, after the control step, to form x += Y x',
                            r = Y r', p = Y p' (eq. coords).  The (2 s + 1) N basis values are never stored
                            (4 N instead); the stencil work grows with the halo.  Other operators or options:
                            SSCG_ERR_UNSUPPORTED.  Not supported by sscg_solve_batch.  Default 0 */
} sscg_opts;

/* Per-outer-loop decision record (Alg. 5): s-bar_k, s-tilde_k, s_k, c at the
 * start and end of the block, phi, the Ritz estimates after the block, the
 * coordinate residual estimate, and kappa_l ~ kappa(Y_l) for l = 1..s-bar_k
 * (kappa[0] unused; +inf when numerically singular). */
typedef struct {
  int sbar, stilde, sk;
  int replaced;          /* bit 0: true-residual replacement (convergence check failed); bit 1: FP32-basis replacement */
  double c_start, c_end, phi, lmin, lmax, relres_est;
  double kappa[SSCG_MAX_S + 1];
} sscg_outer_record;

/* Statistics of the last solve.  `hist` is caller-owned and optional: when
 * non-NULL, up to hist_cap records are written, one per outer loop. */
typedef struct {
  int status;            /* SSCG_OK / SSCG_NOT_CONVERGED / SSCG_BREAKDOWN */
  int outer_iters;       /* outer loops = global synchronisations of the method */
  int inner_iters;       /* total CG iterations m */
  int host_syncs;        /* times the host waited on the device during the solve */
  int replacements;      /* residual replacements after a failed true-residual check */
  int fp32_replacements; /* y_fp32 only: r := b - A x after the residual fell by 2^-4 since the last one */
  int kernel_launches;   /* kernels of this library launched by the solve (graph nodes counted) */
  double lambda_min, lambda_max; /* final Ritz estimates (Algs. 3-4) */
  double c_last;         /* final c */
  double true_relres;    /* ||b - A x|| / ||b|| at exit, computed on the device */
  double upd_relres;     /* coordinate estimate of the updated residual at exit */
  /* profile == 1 only: summed kernel time per phase (ms) and launch counts */
  double t_mpk_ms, t_gram_ms, t_kappa_ms, t_control_ms, t_recombine_ms, t_other_ms;
  int n_gram_launches;
  double gram_flops;     /* algorithmic flops of all Gram launches: sum of 2 * n * (2s+1)(2s+2)/2 */
  double mpk_spmvs;      /* shifted SpMVs of all matrix-powers levels: sum over loops of 2 s-bar_k - 1 */
  sscg_outer_record* hist;
  int hist_cap;
  int hist_len;
} sscg_stats;

/* ---------------------------------------------------------------- handles */

/* Create a handle for a CSR matrix (Section 1: sparse SPD A).
 * rowptr: n+1 int64 offsets; col: nnz int32 column indices (sorted or not);
 * val: nnz binary64 values.  A must be symmetric positive definite; this is not
 * checked (a non-SPD A ends a solve with SSCG_BREAKDOWN or no convergence).
 * on_device: 1 if the three arrays are device pointers, 0 if host pointers.
 * The handle copies A into its own device memory (CSR, plus a sliced-ELL copy
 * in 32-row slices for the row kernels, about 1.1x the CSR arrays); the caller
 * keeps ownership of its arrays.  cuda_stream: a cudaStream_t or NULL.
 * Errors: INVALID_ARG (n <= 0, nnz < 0, NULL pointers, rowptr[0] != 0,
 * rowptr[n] != nnz, a decreasing rowptr, a column index outside [0, n)),
 * NO_MEMORY, CUDA. */
int sscg_create_csr(sscg_t* out, int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                    const double* val, int on_device, void* cuda_stream);

/* Create a handle for a 2D 5-point or 3D 7-point variable-coefficient stencil
 * with homogeneous Dirichlet boundary: (A u)_i = sum over the faces f of cell i
 * of k_f (u_i - u_nb(f)), u_nb = 0 outside the grid.  Cells are numbered x
 * fastest, then y, then z.  shape = {nx, ny, nz} (nz = 1 for dim = 2).
 * Face arrays, C order (slowest first):
 *   kx: [nz][ny][nx+1]  (west face of cell x is kx[..][..][x], east is x+1)
 *   ky: [nz][ny+1][nx]
 *   kz: [nz+1][ny][nx]  (dim = 3 only; NULL for dim = 2)
 * All k_f must be > 0.  on_device/cuda_stream as for sscg_create_csr; the
 * handle copies the coefficients.  Errors: INVALID_ARG, NO_MEMORY, CUDA. */
int sscg_create_stencil(sscg_t* out, int dim, const int64_t shape[3], const double* kx,
                        const double* ky, const double* kz, int on_device, void* cuda_stream);

/* Release the handle and all device memory it owns (safe on NULL). */
void sscg_destroy(sscg_t h);

/* Problem size n of the handle, or a negative error code. */
int64_t sscg_size(sscg_t h);

/* ---------------------------------------------------------------- solves */

/* Fill opts with the defaults documented in sscg_opts. */
void sscg_opts_default(sscg_opts* opts);

/* Solve A x = b by Algorithm 5 (improved adaptive s-step CG, Section 4).
 * b: device pointer, length n (read only).  x: device pointer, length n; on
 * entry the initial guess x0, on exit the solution.  tol = eps* (relative
 * residual ||b - A x||/||b||), s_max = sigma in [1, SSCG_MAX_S].
 * opts may be NULL (defaults); stats may be NULL.
 * Convergence is declared on the coordinate residual estimate and confirmed by
 * a true residual computed on the device; if that check fails, r := b - A x,
 * p := r and the iteration continues (counted in stats->replacements).  A
 * failed check whose true residual has not halved since the previous failed
 * check ends the solve with SSCG_NOT_CONVERGED (tol below the attainable
 * accuracy).
 * Returns SSCG_OK, SSCG_NOT_CONVERGED, SSCG_BREAKDOWN or a negative error.
 * The call returns after the solve has finished on the device. */
int sscg_solve(sscg_t h, const double* b, double* x, double tol, int s_max, sscg_basis basis,
               const sscg_opts* opts, sscg_stats* stats);

/* As sscg_solve with b and x in HOST memory: copies b and x0 to the device,
 * solves, copies x back (all on the handle's stream). */
int sscg_solve_host(sscg_t h, const double* b_host, double* x_host, double tol, int s_max,
                    sscg_basis basis, const sscg_opts* opts, sscg_stats* stats);

/* Hestenes-Stiefel CG (Algorithm 1, Section 1), the comparator.  Same b, x,
 * tol conventions and true-residual confirmation as sscg_solve.  max_iters
 * caps the iterations (<= 0: 100000).  stats->inner_iters is the iteration
 * count; outer_iters = inner_iters. */
int sscg_solve_hscg(sscg_t h, const double* b, double* x, double tol, int max_iters,
                    sscg_stats* stats);

/* sscg_solve_hscg with its SpMV q = A p split like the s-step matrix powers
 * (sscg_opts.mpk_fp64_per16): for a stencil operator, of every 16 warps
 * spmv_fp64_per16 sum their rows as the binary64 FMA chain and the others as
 * exact integer products rounded once (binary64-accurate, the integer form
 * more so), so that the comparator can use GB300's integer pipes the way the
 * s-step path does.  16 = FMA chain only (sscg_solve_hscg), 0 = integer
 * products only, -1 = the library's tuned share; CSR operators always take
 * the FMA chain.  Other arguments, results and errors as sscg_solve_hscg;
 * spmv_fp64_per16 outside -1..16 returns SSCG_ERR_INVALID_ARG. */
int sscg_solve_hscg_ex(sscg_t h, const double* b, double* x, double tol, int max_iters,
                       int spmv_fp64_per16, sscg_stats* stats);

/* Statistics of a batched solve.  The per-pair arrays are caller-owned and
 * optional (length = total number of right-hand sides when non-NULL). */
typedef struct {
  int npairs;            /* (system, right-hand side) pairs solved */
  int converged;         /* pairs that reached tol (true residual) */
  int outer_loops;       /* outer loops run by the batch (the slowest pair's count) */
  int host_syncs;        /* host waits inside the call */
  int kernel_launches;   /* kernels launched (graph nodes counted once per replay) */
  int graph_launches;    /* CUDA graph launches */
  int64_t inner_iters;   /* sum over pairs */
  double max_true_relres;/* largest ||b - A x||/||b|| over the pairs */
  double device_ms;      /* device time of the outer loops (CUDA events around the graph launch or the
                            polled loop; set-up and copies excluded) */
  int* pair_status;      /* optional, per pair */
  int* pair_outer;       /* optional, per pair */
  int* pair_inner;       /* optional, per pair */
} sscg_batch_stats;

/* Solve many independent systems, each with several right-hand sides, by
 * Algorithm 5 in one batched launch sequence: every (system, right-hand side)
 * pair keeps its own s-step state (its own s-bar_k, s-tilde_k, basis
 * parameters, Ritz estimates and c) while all pairs advance through the same
 * kernels, one outer loop at a time; the loop runs inside one CUDA graph
 * launch (a device-side WHILE node repeats the outer loop until every pair
 * has finished), so the host does not take part.
 * systems: nsys handles (their operators are used, not modified).
 * nrhs: right-hand sides per system (>= 0).  b, x: device arrays holding the
 * pairs back to back, system-major then right-hand-side-major: pair (s, k) at
 * offset sum_{s' < s} nrhs[s'] n_{s'} + k n_s; x holds the initial guesses on
 * entry and the solutions on exit.  s_max: per-system sigma in
 * [1, SSCG_MAX_S] (e.g. from sscg_autotune).  opts: as for sscg_solve
 * (y_fp32 and gram_mode 1 and 2 are unsupported here: SSCG_ERR_UNSUPPORTED;
 * gram_mode 3, the tcgen05 digit Gram, runs one thread block per Gram block
 * and needs batch_gram_rows <= 16384, else SSCG_ERR_INVALID_ARG;
 * batch_chunk_rows / batch_gram_rows set the tile shapes; use_graph = 0
 * replaces the WHILE node by host polling every check_every outer loops).
 * Returns SSCG_OK if every pair
 * converged, SSCG_NOT_CONVERGED / SSCG_BREAKDOWN if some did not, or a
 * negative error.  Device memory for the batch is allocated for the call. */
int sscg_solve_batch(const sscg_t* systems, int nsys, const int* nrhs, const double* b, double* x,
                     double tol, const int* s_max, sscg_basis basis, const sscg_opts* opts,
                     sscg_batch_stats* stats, void* cuda_stream);

/* Autotuner for sigma (the paper leaves sigma to "offline auto-tuning",
 * Section 3): for each candidate sigma (ncand values in [1, SSCG_MAX_S]) run
 * at most trial_outer outer loops of Algorithm 5 with tolerance tol on the
 * handle's operator and right-hand side b (device, length n) from x0 = 0,
 * time them with CUDA events on the handle's stream, and return in *best the
 * candidate with the least device time per inner iteration.  times
 * (optional, host, length ncand) receives milliseconds per inner iteration. */
int sscg_autotune(sscg_t h, const double* b, double tol, const int* candidates, int ncand, int trial_outer,
                  sscg_basis basis, int* best, double* times);

/* Plain CG (Algorithm 1, as sscg_solve_hscg) for the same batch layout as
 * sscg_solve_batch, every pair in lock-step inside one CUDA graph launch
 * (WHILE over bodies of 8 iterations and a true-residual confirmation per
 * pair): the comparator of the batched s-step solve.  systems, nsys, nrhs, b,
 * x, tol, stats: as for sscg_solve_batch (stats->outer_loops = the largest
 * iteration count; pair_outer = pair_inner = each pair's iterations).
 * max_iters caps each pair's iterations (<= 0: 100000); chunk_rows: rows per
 * work chunk (0 = 2048, else 128..1048576).  Returns SSCG_OK if every pair
 * converged, else the first non-OK pair status, or a negative error. */
int sscg_solve_batch_hscg(const sscg_t* systems, int nsys, const int* nrhs, const double* b, double* x, double tol,
                          int max_iters, int chunk_rows, sscg_batch_stats* stats, void* cuda_stream);

/* Autotuner for the batched solve's tile shapes (rows per work chunk and per
 * Gram block, sscg_opts.batch_chunk_rows / batch_gram_rows): for each of the
 * ncand candidates (chunk_rows[i], gram_rows[i]) run sscg_solve_batch on the
 * given batch (same arguments as there; x0 = 0 in a scratch array, b
 * unchanged) for at most trial_outer outer loops, and return in *best the
 * index of the candidate with the least device time per inner iteration
 * (summed over pairs).  times (optional, host, length ncand) receives
 * microseconds per inner iteration.  Device memory is allocated per trial. */
int sscg_autotune_batch(const sscg_t* systems, int nsys, const int* nrhs, const double* b, double tol,
                        const int* s_max, sscg_basis basis, const int* chunk_rows, const int* gram_rows, int ncand,
                        int trial_outer, int* best, double* times, void* cuda_stream);

/* sscg_autotune_batch with the Gram of each candidate as a third dimension:
 * gram_modes[i] (0: binary64 FMAs, 3: the tcgen05 digit Gram; other values
 * return SSCG_ERR_INVALID_ARG) is the sscg_opts.gram_mode of trial i; NULL
 * means 0 for every candidate (sscg_autotune_batch).  Which Gram is faster
 * depends on the batch's block sizes: the digit Gram's cost does not shrink
 * with the number of columns below 32, the binary64 Gram's does. */
int sscg_autotune_batch_ex(const sscg_t* systems, int nsys, const int* nrhs, const double* b, double tol,
                           const int* s_max, sscg_basis basis, const int* chunk_rows, const int* gram_rows,
                           const int* gram_modes, int ncand, int trial_outer, int* best, double* times,
                           void* cuda_stream);

/* Ritz estimates (Algs. 3-4, eq. lest) of the handle's last s-step solve. */
int sscg_ritz(sscg_t h, double* lmin, double* lmax);

/* ----------------------------------------------------- single steps (tests) */

/* y = A v (device pointers, length n). */
int sscg_spmv(sscg_t h, const double* v, double* y);

/* y = A v with a stencil's rows split between binary64 FMA chains and exact
 * integer products as in sscg_solve_hscg_ex (fp64_per16: -1..16; 16 is
 * sscg_spmv; CSR operators take the FMA chain).  Waits for the result. */
int sscg_spmv_ex(sscg_t h, const double* v, double* y, int fp64_per16);

/* The s-step basis of eq. (cg-krylovbasis) by the recurrence eq. (rho):
 * Y = [P_0, R_0, P_1, R_1, ..., P_{s-1}, R_{s-1}, P_s] (interleaved column
 * order: the basis Y_l of the first l inner steps is the leading 2l+1 columns),
 * P_0 = p, R_0 = r, P_{l+1} = ((A - theta_l) P_l - mu_{l-1} P_{l-1}) / gamma_l.
 * p, r: device, length n.  theta, gamma, mu: HOST arrays of length s (mu[l]
 * multiplies rho_l in the recurrence for rho_{l+2}).  Y: device, column major,
 * leading dimension ldy >= n, 2s+1 columns, written.  1 <= s <= SSCG_MAX_S. */
int sscg_build_basis(sscg_t h, const double* p, const double* r, int s, const double* theta,
               const double* gamma, const double* mu, double* Y, int64_t ldy);

/* sscg_build_basis with the split of sscg_opts.mpk_fp64_per16 for stencil
 * operators (0..16 warps of every 16 on the binary64 FMA chain, the others on
 * exact integer products; -1: the library's default).  Outside -1..16:
 * SSCG_ERR_INVALID_ARG. */
int sscg_build_basis_ex(sscg_t h, const double* p, const double* r, int s, const double* theta,
                        const double* gamma, const double* mu, double* Y, int64_t ldy, int mpk_fp64_per16);

/* G = Y^T Y (Section 2, the block inner product of Alg. 5), Y device column
 * major n x ncols with leading dimension ldy, G device ncols x ncols row major
 * (symmetric, both triangles written).  1 <= ncols <= 2*SSCG_MAX_S+1.
 * Deterministic: a fixed blocking and reduction order independent of timing.
 * cuda_stream: cudaStream_t or NULL.  Scratch for the block partial sums is
 * allocated and freed inside the call. */
int sscg_gram(const double* Y, int64_t n, int64_t ldy, int ncols, double* G, void* cuda_stream);

/* sscg_gram with a choice of product arithmetic: mode 0 as sscg_gram; mode 1
 * forms every product from binary32 pairs on the FP32 pipes (each value split
 * exactly into two 24-bit parts after a per-tile power-of-two column scale,
 * compensated binary32 sums over 256-row tiles, binary64 across tiles), which
 * GB300 executes far faster than binary64 FMAs; mode 2 writes every value as
 * the integer F = round(|y| 2^(1082 - e_c)) (e_c the biased exponent of
 * column c's largest value in its 4096-row chunk) split into 12 signed 5-bit
 * digits, forms all digit products (pairs s + t <= 11) on the f16 tensor
 * cores with exact binary32 sums over 1024 rows, and adds those in binary64
 * (normwise error below binary64 FMAs'; componentwise, an entry made only of
 * products far below the two columns' largest values keeps just that
 * absolute accuracy); a column with an Inf or NaN in a chunk gives NaN
 * entries.  Mode 3 is mode 2's arithmetic on the 5th-generation tensor
 * cores (tcgen05.mma, accumulators in tensor memory).  Modes 2 and 3 also
 * allocate an integer scratch of 33 entries per 4096 rows.  Same arguments
 * and allocation behaviour as sscg_gram otherwise; mode outside 0..3:
 * SSCG_ERR_INVALID_ARG. */
int sscg_gram_ex(const double* Y, int64_t n, int64_t ldy, int ncols, double* G, int mode, void* cuda_stream);

/* Same result as sscg_gram, for callers that cannot allocate device memory
 * during a call: programs whose device-memory budget is fixed at start-up,
 * and hosts whose own memory manager owns the device memory (a cudaMalloc or
 * cudaFree inside a library call bypasses it, and cudaFree waits for the whole
 * device).  The paper has no counterpart: this is an interface variant.
 * The block partial sums live in a fixed device array inside the library
 * (304 x 561 doubles, 1.36 MB, held by every device that loads the library
 * until exit); the call allocates nothing.  n is unlimited; ncols must be in
 * [1, 33], else SSCG_ERR_INVALID_ARG.  The first call on a device looks up the
 * array's device address (with that device current), so make that first call
 * before any stream capture.  That address is kept for the process: do not
 * call this entry point on a device after a cudaDeviceReset of it (the reset
 * moves the array).  All calls on a device share the array: calls
 * that overlap on the GPU (other streams, other host threads) race and must
 * be serialised by the caller.  Enqueued on cuda_stream (NULL: legacy
 * default stream); the call does not wait for the result. */
int sscg_gram_noalloc(const double* Y, int64_t n, int64_t ldy, int ncols, double* G, void* cuda_stream);

/* Whether a bounded wait inside a kernel of this library gave up since the
 * flag was last cleared (the gram_mode 3 kernel's hand-offs between its
 * warps: each wait ends after about a second, records the failure and lets
 * the kernel finish, so a result computed after it is not to be trusted).
 * Synchronises the current device, writes 0 or 1 to *flag (host) and
 * clears the flag when `clear` is nonzero. */
int sscg_wait_failures(int* flag, int clear);

/* kappa_l ~ sqrt(kappa(G_l)) for the leading (2l+1) blocks of G, l = 1..sbar
 * (Section 3), from the extreme eigenvalues of each block.  G: device,
 * ldg x ldg row major, ldg >= 2*sbar+1.  kappa, lmin, lmax: device arrays of
 * length sbar+1 (entry 0 unused).  kappa_l = +inf when lmin <= kappa_cut * lmax. */
int sscg_kappa(const double* G, int ldg, int sbar, double kappa_cut, double* kappa, double* lmin,
               double* lmax, void* cuda_stream);

/* The recovery of eq. (coords), Algorithm 5: x += Y x', then Y[:,0] = Y p'
 * and Y[:,1] = Y r' (p and r overwrite columns 0 and 1, as in a solve), over
 * the first ncols columns of Y (1 <= ncols <= 33).  Y: device, column major,
 * leading dimension ldy >= n, at least max(ncols, 2) columns, read and written.  coef: HOST array of 3*ncols
 * doubles, x' then r' then p'.  x: device, length n, read and written.
 * rec_fp64_per16: the split of sscg_opts.rec_fp64_per16 (-1..16).  Waits for
 * the stream; SSCG_ERR_INVALID_ARG on bad sizes or split. */
int sscg_recombine(double* Y, int64_t n, int64_t ldy, int ncols, const double* coef, double* x, int rec_fp64_per16,
                   void* cuda_stream);

/* The first s Leja points of [-1, 1] starting 1, -1 (eq. newtbasis on the
 * reference interval), computed on the device.  t: HOST array of length s. */
int sscg_leja(int s, double* t);

/* --------------------------------------------------- differentiable solve */

/* Gradient of a loss L(x) with respect to the face conductivities of a stencil
 * handle, for x = A^{-1} b: with the adjoint state lam = A^{-1} dL/dx (A is
 * symmetric, so the adjoint solve is another sscg_solve), dA/dk_f is
 * (e_i - e_j)(e_i - e_j)^T for the interior face between cells i and j and
 * e_i e_i^T for a boundary face of cell i, so
 *   dL/dk_f = -(lam_i - lam_j)(x_i - x_j)   (lam = x = 0 outside the grid).
 * dL/db = lam needs no call.  lam, x: device, length n.  gkx, gky, gkz:
 * device arrays with the shapes of kx, ky, kz (gkz NULL for dim = 2),
 * overwritten.  Errors: INVALID_ARG (NULL pointers, not a stencil handle). */
int sscg_stencil_face_grad(sscg_t h, const double* lam, const double* x, double* gkx, double* gky,
                           double* gkz);

/* dL/dA_ij = -lam_i x_j for every stored entry of a CSR handle (each stored
 * value treated as an independent parameter).  gval: device, length nnz,
 * overwritten.  Errors: INVALID_ARG (NULL pointers, not a CSR handle). */
int sscg_csr_value_grad(sscg_t h, const double* lam, const double* x, double* gval);

/* ------------------------------------------------------------------ misc */

const char* sscg_strerror(int code);
const char* sscg_last_cuda_error(void);
/* Library version string. */
const char* sscg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SSCG_H */
