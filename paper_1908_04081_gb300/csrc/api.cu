// Host side of libsscg: handles, the outer-loop driver of Algorithm 5 (Carson
// 2019, Section 4), the HSCG comparator (Algorithm 1) and the step-level entry
// points.  The host only enqueues kernels: every decision of a solve is taken
// by device code, and the host polls a device "done" flag once every
// `check_every` outer loops (bodies after convergence exit immediately).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sscg_internal.cuh"

using namespace sscg;

namespace {

thread_local std::string g_last_cuda_error;

int cuda_fail(cudaError_t e, const char* what) {
  g_last_cuda_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? SSCG_ERR_NO_MEMORY : SSCG_ERR_CUDA;
}

#define CK(call)                                        \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return cuda_fail(_e, #call); \
  } while (0)

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }  // frees on every return path of the entry points
  cudaError_t ensure(size_t count) {
    if (count <= n) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e == cudaSuccess) n = count;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

}  // namespace

struct sscg_ctx {
  Operator op{};
  int64_t n = 0;
  cudaStream_t user_stream = nullptr;
  cudaStream_t stream = nullptr;  // private stream (stream capture needs a non-legacy stream)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // digit Grams: the column scales of each level's new columns are found on
  // a side stream while the next level runs (ev_lvl[l]: level l - 1 done,
  // ev_lvl[kMaxS + 1]: the side stream's last pass done)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_lvl[kMaxS + 2] = {};
  // operator storage
  DevBuf<int64_t> rowptr, s_off;
  DevBuf<int32_t> col, s_row, s_len, s_col;
  DevBuf<double> val, s_val, kx, ky, kz, diag;
  // solve storage
  int64_t ld = 0;
  DevBuf<double> Y, G, partials, rt, b, x, r, p, q;
  DevBuf<double> ritz_t;   // T_m of eq. (T) for ritz_exact: diagonal, then squared off-diagonal
  DevBuf<double> pr;       // recompute_y: p, r (columns 0, 1, leading dimension n), the new p, r, the
                           // loop's recurrence coefficients (3 kMaxS)
  const double* leja = nullptr;  // the device's Leja table (not owned)
  DevBuf<int> chunk_exp;  // gram_mode 2 scratch
  DevBuf<SolveState> state;
  DevBuf<sscg_outer_record> hist;
  SolveState* host_state = nullptr;  // pinned mirror
  // cached graph of one outer loop
  cudaGraphExec_t graph = nullptr;
  int graph_sigma = -1;
  bool graph_y32 = false;
  int graph_gram_mode = 0;
  int graph_mpk_split = -1;
  int graph_rec_split = -1;
  int graph_ritz_exact = -1;
  int graph_recompute = -1;
  int graph_launches = 0;
  double last_lmin = 0.0, last_lmax = 0.0;
};

namespace {

int init_common(sscg_ctx* h, void* cuda_stream) {
  h->user_stream = (cudaStream_t)cuda_stream;
  CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
  CK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
  for (auto& e : h->ev_lvl) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  CK(cudaMallocHost(&h->host_state, sizeof(SolveState)));
  CK(leja_table(&h->leja, h->stream));
  CK(h->state.ensure(1));
  CK(h->G.ensure(kMaxCols * kMaxCols));
  return SSCG_OK;
}

// order the private stream after the caller's stream (start) and the caller's
// stream after the private one (end)
int join_in(sscg_ctx* h) {
  CK(cudaEventRecord(h->ev_in, h->user_stream));
  CK(cudaStreamWaitEvent(h->stream, h->ev_in, 0));
  return SSCG_OK;
}
int join_out(sscg_ctx* h) {
  CK(cudaEventRecord(h->ev_out, h->stream));
  CK(cudaStreamWaitEvent(h->user_stream, h->ev_out, 0));
  return SSCG_OK;
}

template <typename T>
cudaMemcpyKind kind_of(int on_device) {
  return on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}

int ensure_solve_buffers(sscg_ctx* h, int sigma, int hist_cap, bool y32 = false, bool recompute = false) {
  const int64_t n = h->n;
  h->ld = round_up(n, 32);
  auto drop_graph = [&]() {
    if (h->graph) {
      cudaGraphExecDestroy(h->graph);
      h->graph = nullptr;
      h->graph_sigma = -1;
    }
  };
  const int gb = gram_blocks(n);
  const int rb = reduce_blocks(n);
  size_t npart = std::max((size_t)gb * kMaxPairs, (size_t)4 * rb);
  if (recompute) {
    // no basis: p and r twice, and one partial Gram per tile
    if (h->pr.n < 4 * (size_t)n + 3 * kMaxS) drop_graph();
    CK(h->pr.ensure(4 * (size_t)n + 3 * kMaxS));
    CK(recompute_prepare());
    npart = std::max(npart, (size_t)recompute_partials(h->op));
  } else {
    const size_t ycount = (size_t)h->ld * (2 * sigma + 1);
    if (ycount > h->Y.n) drop_graph();
    CK(h->Y.ensure(ycount));
  }
  CK(gram_prepare());
  if (npart > h->partials.n) drop_graph();
  CK(h->partials.ensure(npart));
  CK(h->chunk_exp.ensure((size_t)gram_exp_ints(n)));
  CK(h->rt.ensure(n));
  CK(h->b.ensure(n));
  CK(h->x.ensure(n));
  if (y32) {
    if (h->r.n < (size_t)n || h->p.n < (size_t)n) {
      if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
        h->graph_sigma = -1;
      }
    }
    CK(h->r.ensure(n));
    CK(h->p.ensure(n));
  }
  if (hist_cap > 0 && (size_t)hist_cap > h->hist.n) {
    if (h->graph) {
      cudaGraphExecDestroy(h->graph);
      h->graph = nullptr;
      h->graph_sigma = -1;
    }
    CK(h->hist.ensure(hist_cap));
  }
  return SSCG_OK;
}

// Enqueue one outer loop of Algorithm 5.  Returns the number of kernels.
// One outer loop without a stored basis (recompute_y, 2D stencils): the
// basis is formed tile by tile twice, for G and for the recovery.
int enqueue_body_recompute(sscg_ctx* h, cudaStream_t st, std::vector<cudaEvent_t>* evs, int* nlaunch) {
  SolveState* ds = h->state.p;
  double* PR = h->pr.p;
  int count = 0;
  auto mark = [&](int i) -> int {
    if (evs) CK(cudaEventRecord((*evs)[i], st));
    return SSCG_OK;
  };
  int rc;
  if ((rc = mark(0))) return rc;
  if ((rc = mark(1))) return rc;
  CK(launch_recompute_gram(h->op, PR, ds, h->partials.p, PR + 4 * h->n, h->G.p, kMaxCols, st));
  count += 2;
  if ((rc = mark(2))) return rc;
  CK(launch_kappa(h->G.p, kMaxCols, ds, 0, 0.0 /* taken from the state */, ds->kappa, ds->glmin,
                  ds->glmax, h->host_state->sigma, st));
  ++count;
  if ((rc = mark(3))) return rc;
  CK(launch_control(ds, h->G.p, kMaxCols, h->leja, h->hist.n ? h->hist.p : nullptr, st,
                    h->host_state->ritz_exact != 0));
  ++count;
  if ((rc = mark(4))) return rc;
  CK(launch_recompute_recover(h->op, PR, PR + 2 * h->n, h->x.p, ds, PR + 4 * h->n, st));
  ++count;
  if ((rc = mark(5))) return rc;
  CK(launch_true_residual(ds, h->op, h->b.p, h->x.p, h->rt.p, h->partials.p, reduce_blocks(h->n), st));
  CK(launch_apply_replacement(ds, h->rt.p, PR, h->n, nullptr, nullptr, h->n, false,
                              h->hist.n ? h->hist.p : nullptr, st));
  count += 4;
  if ((rc = mark(6))) return rc;
  *nlaunch = count;
  return SSCG_OK;
}

int enqueue_body(sscg_ctx* h, int sigma, bool y32, cudaStream_t st, std::vector<cudaEvent_t>* evs, int* nlaunch) {
  if (h->host_state->recompute_y) return enqueue_body_recompute(h, st, evs, nlaunch);
  SolveState* ds = h->state.p;
  LevelCoef coef{ds->theta, ds->inv_gamma, ds->mu};
  int count = 0;
  auto mark = [&](int i) -> int {
    if (evs) CK(cudaEventRecord((*evs)[i], st));
    return SSCG_OK;
  };
  int rc;
  if ((rc = mark(0))) return rc;
  // digit Grams: each pair of new columns gets its scales on the side stream
  // while the next level runs on st (the levels are bound by the FP64 unit
  // and the integer pipes, the scale pass by memory); only the last pair's
  // pass is on the path to the Gram
  const bool digit = h->host_state->gram_mode >= 2;
  bool forked = false;
  auto join = [&]() -> cudaError_t {   // the side stream back into st (also before an error return)
    if (!forked) return cudaSuccess;
    forked = false;
    cudaError_t e = cudaEventRecord(h->ev_lvl[kMaxS + 1], h->side);
    cudaError_t e2 = cudaStreamWaitEvent(st, h->ev_lvl[kMaxS + 1], 0);
    return e != cudaSuccess ? e : e2;
  };
  auto scales = [&](int l) -> cudaError_t {   // after level l - 1 (l = 0: columns 0, 1 from the last loop)
    cudaError_t e = cudaEventRecord(h->ev_lvl[l], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->ev_lvl[l], 0);
    if (e == cudaSuccess) {
      forked = true;
      e = launch_chunk_exp(h->Y.p, h->n, h->ld, ds, 2 * l, 2, y32, h->chunk_exp.p, h->side);
    }
    if (e == cudaSuccess) ++count;
    return e;
  };
  cudaError_t ef = digit ? scales(0) : cudaSuccess;
  for (int l = 0; l < sigma && ef == cudaSuccess; ++l) {
    ef = launch_mpk_level(h->op, h->Y.p, h->ld, l, ds, 0, coef, y32, st, h->host_state->mpk_fp64_per16);
    if (ef == cudaSuccess) ++count;
    if (ef == cudaSuccess && digit) ef = scales(l + 1);
  }
  const cudaError_t ej = join();
  CK(ef);
  CK(ej);
  if ((rc = mark(1))) return rc;
  CK(launch_gram(h->Y.p, h->n, h->ld, nullptr, 0, ds, h->partials.p, gram_blocks(h->n), h->G.p, kMaxCols, y32,
                 st, h->host_state->gram_mode, h->chunk_exp.p, digit));
  count += 2;
  if ((rc = mark(2))) return rc;
  CK(launch_kappa(h->G.p, kMaxCols, ds, 0, 0.0 /* taken from the state */, ds->kappa, ds->glmin,
                  ds->glmax, sigma, st));
  ++count;
  if ((rc = mark(3))) return rc;
  CK(launch_control(ds, h->G.p, kMaxCols, h->leja, h->hist.n ? h->hist.p : nullptr, st,
                    h->host_state->ritz_exact != 0));
  ++count;
  if ((rc = mark(4))) return rc;
  CK(launch_recombine(ds, h->Y.p, h->ld, h->x.p, y32 ? h->r.p : nullptr, y32 ? h->p.p : nullptr, h->n, y32, st,
                      h->host_state->rec_fp64_per16));
  ++count;
  if ((rc = mark(5))) return rc;
  if (y32) {
    CK(launch_fp32_replacement(ds, h->op, h->b.p, h->x.p, h->Y.p, h->ld, h->r.p, h->partials.p, reduce_blocks(h->n),
                               h->hist.n ? h->hist.p : nullptr, st));
    count += 2;
  }
  CK(launch_true_residual(ds, h->op, h->b.p, h->x.p, h->rt.p, h->partials.p, reduce_blocks(h->n), st));
  CK(launch_apply_replacement(ds, h->rt.p, h->Y.p, h->ld, y32 ? h->r.p : nullptr, y32 ? h->p.p : nullptr, h->n, y32,
                              h->hist.n ? h->hist.p : nullptr, st));
  count += 4;
  if ((rc = mark(6))) return rc;
  *nlaunch = count;
  return SSCG_OK;
}

// The whole solve loop as one graph: a kernel arms the loop condition, then a
// WHILE node repeats one outer loop until the device sets done.
int build_graph(sscg_ctx* h, int sigma, bool y32) {
  if (h->graph && h->graph_sigma == sigma && h->graph_y32 == y32 && h->graph_gram_mode == h->host_state->gram_mode &&
      h->graph_mpk_split == h->host_state->mpk_fp64_per16 && h->graph_rec_split == h->host_state->rec_fp64_per16 &&
      h->graph_ritz_exact == h->host_state->ritz_exact && h->graph_recompute == h->host_state->recompute_y)
    return SSCG_OK;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  cudaGraph_t g;
  CK(cudaGraphCreate(&g, 0));
  auto fail = [&](cudaError_t e, const char* w) {
    cudaGraphDestroy(g);
    return cuda_fail(e, w);
  };
  cudaGraphConditionalHandle cond;
  cudaError_t e = cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return fail(e, "cudaGraphConditionalHandleCreate");
  if ((e = cudaStreamBeginCaptureToGraph(h->stream, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess)
    return fail(e, "capture arm");
  cudaError_t ea = launch_batch_arm(cond, h->stream);
  cudaGraph_t tmp;
  e = cudaStreamEndCapture(h->stream, &tmp);
  if (ea != cudaSuccess) return fail(ea, "arm kernel");
  if (e != cudaSuccess) return fail(e, "end capture arm");
  size_t nn = 1;
  cudaGraphNode_t arm_node;
  if ((e = cudaGraphGetNodes(g, &arm_node, &nn)) != cudaSuccess) return fail(e, "cudaGraphGetNodes");
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wnode;
  if ((e = cudaGraphAddNode(&wnode, g, &arm_node, nullptr, 1, &cp)) != cudaSuccess) return fail(e, "while node");
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if ((e = cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
      cudaSuccess)
    return fail(e, "capture body");
  int nl = 0;
  int rc = enqueue_body(h, sigma, y32, h->stream, nullptr, &nl);
  cudaError_t ec = rc ? cudaSuccess : launch_solve_cond(h->state.p, cond, h->stream);
  e = cudaStreamEndCapture(h->stream, &tmp);
  if (rc) {
    cudaGraphDestroy(g);
    return rc;
  }
  if (ec != cudaSuccess) return fail(ec, "cond kernel");
  if (e != cudaSuccess) return fail(e, "end capture body");
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  h->graph_sigma = sigma;
  h->graph_y32 = y32;
  h->graph_gram_mode = h->host_state->gram_mode;
  h->graph_mpk_split = h->host_state->mpk_fp64_per16;
  h->graph_rec_split = h->host_state->rec_fp64_per16;
  h->graph_ritz_exact = h->host_state->ritz_exact;
  h->graph_recompute = h->host_state->recompute_y;
  h->graph_launches = nl + 1;
  return SSCG_OK;
}

void fill_state_config(SolveState& s, int sigma, double tol, int basis, const sscg_opts& o, int hist_cap) {
  std::memset(&s, 0, sizeof(s));
  s.sigma = sigma;
  s.s0 = o.s0 > 0 ? std::min(o.s0, sigma) : sigma;
  s.f = o.f > 0 ? o.f : sigma;
  s.basis = basis;
  s.c_mode = o.c_mode;
  s.newton_scale = o.newton_scale;
  s.cheb_params = o.cheb_params;
  s.inner_conv_check = o.inner_conv_check;
  s.variant = o.variant;
  s.max_outer = o.max_outer > 0 ? o.max_outer : 100000;
  s.y_fp32 = o.y_fp32;
  s.hist_cap = hist_cap;
  s.tol = tol;
  s.eps = o.eps;
  s.kappa_cut = o.kappa_cut;
  s.c_const = o.c_const;
  s.sbar = s.s0;
  s.status = SSCG_NOT_CONVERGED;
  s.c = 1.0 / std::sqrt(o.eps);  // c_1 = eps^{-1/2} (Alg. 5)
  s.psi = 1.0;
  s.fp32_drop = std::ldexp(1.0, -4);  // FP32 basis: replace r after a 2^-4 drop
  s.gram_mode = o.gram_mode;
  s.mpk_fp64_per16 = o.mpk_fp64_per16;
  s.rec_fp64_per16 = o.rec_fp64_per16;
  s.ritz_exact = o.ritz_exact;
  s.recompute_y = o.recompute_y;
  s.rho_last = 1.0;
  for (int l = 0; l < kMaxS; ++l) {
    s.theta[l] = 0.0;  // monomial basis until Ritz values exist
    s.gamma[l] = 1.0;
    s.inv_gamma[l] = 1.0;
    s.mu[l] = 0.0;
  }
}

int validate_opts(const sscg_opts& o) {
  if (o.c_mode < 0 || o.c_mode > SSCG_C_CONST) return SSCG_ERR_INVALID_ARG;
  if (o.gram_mode < 0 || o.gram_mode > 3) return SSCG_ERR_INVALID_ARG;
  if (o.batch_chunk_rows != 0 && (o.batch_chunk_rows < 128 || o.batch_chunk_rows > (1 << 20)))
    return SSCG_ERR_INVALID_ARG;
  if (o.batch_gram_rows != 0 && (o.batch_gram_rows < 128 || o.batch_gram_rows > (1 << 20)))
    return SSCG_ERR_INVALID_ARG;
  if (!(o.eps > 0.0) || !(o.kappa_cut >= 0.0)) return SSCG_ERR_INVALID_ARG;
  if (o.mpk_fp64_per16 < -1 || o.mpk_fp64_per16 > 16) return SSCG_ERR_INVALID_ARG;
  if (o.rec_fp64_per16 < -1 || o.rec_fp64_per16 > 16) return SSCG_ERR_INVALID_ARG;
  if (o.ritz_exact != 0 && o.ritz_exact != 1) return SSCG_ERR_INVALID_ARG;
  if (o.recompute_y != 0 && o.recompute_y != 1) return SSCG_ERR_INVALID_ARG;
  return SSCG_OK;
}

}  // namespace

// ===================================================================== API
extern "C" {

const char* sscg_version(void) { return "sscg 0.1 (sm_103a)"; }

const char* sscg_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

const char* sscg_strerror(int code) {
  switch (code) {
    case SSCG_OK: return "ok";
    case SSCG_BREAKDOWN: return "breakdown: p'^T G B p' <= 0 at the first step of a block (A not SPD?)";
    case SSCG_NOT_CONVERGED: return "not converged (iteration cap, or stagnation above tol)";
    case SSCG_NONFINITE: return "non-finite value (NaN or Inf) in b, x0, A or the iteration";
    case SSCG_ERR_INVALID_ARG: return "invalid argument";
    case SSCG_ERR_CUDA: return "CUDA runtime error (see sscg_last_cuda_error)";
    case SSCG_ERR_NO_MEMORY: return "out of device memory";
    case SSCG_ERR_UNSUPPORTED: return "unsupported option";
    default: return "unknown status";
  }
}

void sscg_opts_default(sscg_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->s0 = 0;
  o->f = 0;
  o->max_outer = 100000;
  o->c_mode = SSCG_C_XI;
  o->newton_scale = 0;
  o->cheb_params = 0;
  o->inner_conv_check = 1;
  o->y_fp32 = 0;
  o->variant = 0;
  o->check_every = 4;
  o->use_graph = 1;
  o->profile = 0;
  o->c_const = 1.0;
  o->eps = std::ldexp(1.0, -53);
  o->kappa_cut = std::ldexp(1.0, -44);
  o->gram_mode = 0;
  o->batch_chunk_rows = 0;
  o->batch_gram_rows = 0;
  o->mpk_fp64_per16 = -1;
  o->rec_fp64_per16 = -1;
  o->ritz_exact = 0;
  o->recompute_y = 0;
}

int sscg_create_csr(sscg_t* out, int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                    const double* val, int on_device, void* cuda_stream) {
  if (!out || n <= 0 || nnz < 0 || !rowptr || (nnz > 0 && (!col || !val))) return SSCG_ERR_INVALID_ARG;
  if (n > (int64_t)INT32_MAX) return SSCG_ERR_INVALID_ARG;  // int32 column indices
  *out = nullptr;
  sscg_ctx* h = new (std::nothrow) sscg_ctx();
  if (!h) return SSCG_ERR_NO_MEMORY;
  int rc = init_common(h, cuda_stream);
  if (rc) {
    sscg_destroy(h);
    return rc;
  }
  h->n = n;
  auto fail = [&](cudaError_t e, const char* w) {
    int r = cuda_fail(e, w);
    sscg_destroy(h);
    return r;
  };
  cudaError_t e;
  if ((e = h->rowptr.ensure(n + 1)) != cudaSuccess) return fail(e, "alloc rowptr");
  if ((e = h->col.ensure(std::max<int64_t>(nnz, 1))) != cudaSuccess) return fail(e, "alloc col");
  if ((e = h->val.ensure(std::max<int64_t>(nnz, 1))) != cudaSuccess) return fail(e, "alloc val");
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if ((e = cudaMemcpyAsync(h->rowptr.p, rowptr, (n + 1) * sizeof(int64_t), k, h->stream)) != cudaSuccess)
    return fail(e, "copy rowptr");
  if (nnz > 0) {
    if ((e = cudaMemcpyAsync(h->col.p, col, nnz * sizeof(int32_t), k, h->stream)) != cudaSuccess)
      return fail(e, "copy col");
    if ((e = cudaMemcpyAsync(h->val.p, val, nnz * sizeof(double), k, h->stream)) != cudaSuccess)
      return fail(e, "copy val");
  }
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return fail(e, "create_csr sync");
  // sliced ELL copy for the row kernels: every lane of a warp walks a row of
  // nearly the same length, and the loads of a slice are coalesced
  std::vector<int64_t> hrp(n + 1);
  std::vector<int32_t> hcol(std::max<int64_t>(nnz, 1));
  std::vector<double> hval(std::max<int64_t>(nnz, 1));
  if ((e = cudaMemcpy(hrp.data(), h->rowptr.p, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return fail(e, "read rowptr");
  if (nnz > 0) {
    if ((e = cudaMemcpy(hcol.data(), h->col.p, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return fail(e, "read col");
    if ((e = cudaMemcpy(hval.data(), h->val.p, nnz * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return fail(e, "read val");
  }
  // the kernels index with these: reject a malformed matrix here
  auto bad = [&](const char* what) {
    g_last_cuda_error = std::string("create_csr: ") + what;
    sscg_destroy(h);
    return SSCG_ERR_INVALID_ARG;
  };
  if (hrp[0] != 0 || hrp[n] != nnz) return bad("rowptr[0] must be 0 and rowptr[n] = nnz");
  for (int64_t i = 0; i < n; ++i)
    if (hrp[i + 1] < hrp[i]) return bad("rowptr must not decrease");
  for (int64_t k = 0; k < nnz; ++k)
    if (hcol[k] < 0 || hcol[k] >= n) return bad("column index out of range");
  const int64_t nslices = (n + kSliceRows - 1) / kSliceRows;
  std::vector<int32_t> srow(nslices * kSliceRows, -1), slen(nslices);
  std::vector<int64_t> soff(nslices + 1, 0);
  for (int64_t w = 0; w < n; w += kSliceWindow) {
    const int64_t cnt = std::min<int64_t>(kSliceWindow, n - w);
    for (int64_t i = 0; i < cnt; ++i) srow[w + i] = (int32_t)(w + i);
    std::stable_sort(srow.begin() + w, srow.begin() + w + cnt, [&](int32_t a, int32_t b) {
      return hrp[a + 1] - hrp[a] > hrp[b + 1] - hrp[b];
    });
  }
  for (int64_t sl = 0; sl < nslices; ++sl) {
    int64_t mx = 0;
    for (int t = 0; t < kSliceRows; ++t) {
      const int32_t r = srow[sl * kSliceRows + t];
      if (r >= 0) mx = std::max<int64_t>(mx, hrp[r + 1] - hrp[r]);
    }
    if (mx > INT32_MAX) return fail(cudaErrorInvalidValue, "row length");
    slen[sl] = (int32_t)mx;
    soff[sl + 1] = soff[sl] + mx * kSliceRows;
  }
  const int64_t scount = std::max<int64_t>(soff[nslices], 1);
  std::vector<int32_t> scol(scount, 0);
  std::vector<double> sval(scount, 0.0);
  for (int64_t sl = 0; sl < nslices; ++sl)
    for (int t = 0; t < kSliceRows; ++t) {
      const int32_t r = srow[sl * kSliceRows + t];
      if (r < 0) continue;
      for (int64_t k = hrp[r], j = 0; k < hrp[r + 1]; ++k, ++j) {
        scol[soff[sl] + j * kSliceRows + t] = hcol[k];
        sval[soff[sl] + j * kSliceRows + t] = hval[k];
      }
    }
  if ((e = h->s_row.ensure(srow.size())) != cudaSuccess) return fail(e, "alloc s_row");
  if ((e = h->s_len.ensure(std::max<int64_t>(nslices, 1))) != cudaSuccess) return fail(e, "alloc s_len");
  if ((e = h->s_off.ensure(nslices + 1)) != cudaSuccess) return fail(e, "alloc s_off");
  if ((e = h->s_col.ensure(scount)) != cudaSuccess) return fail(e, "alloc s_col");
  if ((e = h->s_val.ensure(scount)) != cudaSuccess) return fail(e, "alloc s_val");
  if ((e = cudaMemcpy(h->s_row.p, srow.data(), srow.size() * sizeof(int32_t), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->s_len.p, slen.data(), nslices * sizeof(int32_t), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->s_off.p, soff.data(), (nslices + 1) * sizeof(int64_t), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->s_col.p, scol.data(), scount * sizeof(int32_t), cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(h->s_val.p, sval.data(), scount * sizeof(double), cudaMemcpyHostToDevice)))
    return fail(e, "copy sliced ELL");
  h->op.kind = 0;
  h->op.n = n;
  h->op.rowptr = h->rowptr.p;
  h->op.col = h->col.p;
  h->op.val = h->val.p;
  h->op.nslices = nslices;
  h->op.s_row = h->s_row.p;
  h->op.s_off = h->s_off.p;
  h->op.s_len = h->s_len.p;
  h->op.s_col = h->s_col.p;
  h->op.s_val = h->s_val.p;
  *out = h;
  return SSCG_OK;
}

int sscg_create_stencil(sscg_t* out, int dim, const int64_t shape[3], const double* kx, const double* ky,
                        const double* kz, int on_device, void* cuda_stream) {
  if (!out || !shape || (dim != 2 && dim != 3) || !kx || !ky || (dim == 3 && !kz)) return SSCG_ERR_INVALID_ARG;
  const int64_t nx = shape[0], ny = shape[1], nz = dim == 3 ? shape[2] : 1;
  if (nx <= 0 || ny <= 0 || nz <= 0 || nx > (1 << 30) || ny > (1 << 30) || nz > (1 << 30))
    return SSCG_ERR_INVALID_ARG;
  *out = nullptr;
  sscg_ctx* h = new (std::nothrow) sscg_ctx();
  if (!h) return SSCG_ERR_NO_MEMORY;
  int rc = init_common(h, cuda_stream);
  if (rc) {
    sscg_destroy(h);
    return rc;
  }
  const int64_t n = nx * ny * nz;
  h->n = n;
  auto fail = [&](cudaError_t e, const char* w) {
    int r = cuda_fail(e, w);
    sscg_destroy(h);
    return r;
  };
  const size_t cx = (size_t)nz * ny * (nx + 1), cy = (size_t)nz * (ny + 1) * nx, cz = (size_t)(nz + 1) * ny * nx;
  cudaError_t e;
  if ((e = h->kx.ensure(cx)) != cudaSuccess) return fail(e, "alloc kx");
  if ((e = h->ky.ensure(cy)) != cudaSuccess) return fail(e, "alloc ky");
  if (dim == 3 && (e = h->kz.ensure(cz)) != cudaSuccess) return fail(e, "alloc kz");
  if ((e = h->diag.ensure(n)) != cudaSuccess) return fail(e, "alloc diag");
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if ((e = cudaMemcpyAsync(h->kx.p, kx, cx * sizeof(double), k, h->stream)) != cudaSuccess) return fail(e, "copy kx");
  if ((e = cudaMemcpyAsync(h->ky.p, ky, cy * sizeof(double), k, h->stream)) != cudaSuccess) return fail(e, "copy ky");
  if (dim == 3 && (e = cudaMemcpyAsync(h->kz.p, kz, cz * sizeof(double), k, h->stream)) != cudaSuccess)
    return fail(e, "copy kz");
  h->op.kind = 1;
  h->op.n = n;
  h->op.dim = dim;
  h->op.nx = (int)nx;
  h->op.ny = (int)ny;
  h->op.nz = (int)nz;
  h->op.kx = h->kx.p;
  h->op.ky = h->ky.p;
  h->op.kz = dim == 3 ? h->kz.p : nullptr;
  h->op.diag = h->diag.p;
  if ((e = launch_stencil_diag(h->op, h->diag.p, h->stream)) != cudaSuccess) return fail(e, "stencil diag");
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return fail(e, "create_stencil sync");
  *out = h;
  return SSCG_OK;
}

void sscg_destroy(sscg_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->rowptr.release();
  h->col.release();
  h->val.release();
  h->s_off.release();
  h->s_row.release();
  h->s_len.release();
  h->s_col.release();
  h->s_val.release();
  h->kx.release();
  h->ky.release();
  h->kz.release();
  h->diag.release();
  h->Y.release();
  h->G.release();
  h->partials.release();
  h->chunk_exp.release();
  h->rt.release();
  h->b.release();
  h->x.release();
  h->r.release();
  h->p.release();
  h->q.release();
  h->state.release();
  h->ritz_t.release();
  h->pr.release();
  h->hist.release();
  if (h->host_state) cudaFreeHost(h->host_state);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  for (auto& e : h->ev_lvl)
    if (e) cudaEventDestroy(e);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

int64_t sscg_size(sscg_t h) { return h ? h->n : SSCG_ERR_INVALID_ARG; }

int sscg_solve(sscg_t h, const double* b, double* x, double tol, int s_max, sscg_basis basis, const sscg_opts* opts,
               sscg_stats* stats) {
  if (!h || !b || !x || !(tol > 0.0) || s_max < 1 || s_max > kMaxS) return SSCG_ERR_INVALID_ARG;
  if (basis < SSCG_MONOMIAL || basis > SSCG_CHEBYSHEV) return SSCG_ERR_INVALID_ARG;
  sscg_opts o;
  sscg_opts_default(&o);
  if (opts) o = *opts;
  int rc = validate_opts(o);
  if (rc) return rc;
  const int sigma = s_max;
  int hist_cap = 0;
  if (stats && stats->hist && stats->hist_cap > 0) hist_cap = stats->hist_cap;
  if (o.profile && hist_cap == 0) hist_cap = std::min(o.max_outer > 0 ? o.max_outer : 100000, 100000);
  hist_cap = std::min(hist_cap, o.max_outer > 0 ? o.max_outer : 100000);
  const bool y32 = o.y_fp32 != 0;
  const bool recompute = o.recompute_y != 0;
  if (recompute && (!recompute_supported(h->op) || y32 || o.gram_mode != 0)) return SSCG_ERR_UNSUPPORTED;
  if ((rc = ensure_solve_buffers(h, sigma, hist_cap, y32, recompute))) return rc;
  if ((rc = join_in(h))) return rc;
  cudaStream_t st = h->stream;
  const int64_t n = h->n;
  CK(cudaMemcpyAsync(h->b.p, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(h->x.p, x, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  // configuration -> device state, as a kernel argument (no host wait); the
  // pinned mirror keeps a copy for the host-side choices below
  fill_state_config(*h->host_state, sigma, tol, (int)basis, o, hist_cap);
  if (o.ritz_exact) {
    const int64_t mo = o.max_outer > 0 ? o.max_outer : 100000;
    const int cap = (int)std::min<int64_t>(mo * sigma, (int64_t)1 << 20);
    CK(h->ritz_t.ensure(2 * (size_t)cap));
    h->host_state->ritz_cap = cap;
    h->host_state->ritz_d = h->ritz_t.p;
    h->host_state->ritz_e2 = h->ritz_t.p + cap;
  }
  CK(launch_set_state(h->state.p, *h->host_state, st));
  CK(launch_init_state(h->state.p, h->op, h->b.p, h->x.p, recompute ? h->pr.p : h->Y.p, recompute ? h->n : h->ld,
                       y32 ? h->r.p : nullptr,
                       y32 ? h->p.p : nullptr, h->partials.p, reduce_blocks(n), y32, st));
  int launches = 3;
  int host_syncs = 0;

  const bool prof = o.profile != 0;
  const bool graph = o.use_graph && !prof;
  if (graph && (rc = build_graph(h, sigma, y32))) return rc;
  const int every = std::max(1, o.check_every);
  double tph[6] = {0, 0, 0, 0, 0, 0};
  std::vector<cudaEvent_t> evs;
  if (prof) {
    evs.resize(7 * every);
    for (auto& e : evs) CK(cudaEventCreate(&e));
  }
  int bodies = 0;
  if (graph) {
    // one launch runs the whole solve; the host waits once, at the end
    CK(cudaGraphLaunch(h->graph, st));
  }
  while (!graph) {
    for (int b2 = 0; b2 < every; ++b2) {
      {
        std::vector<cudaEvent_t> sub;
        if (prof) sub.assign(evs.begin() + 7 * b2, evs.begin() + 7 * b2 + 7);
        int nl = 0;
        if ((rc = enqueue_body(h, sigma, y32, st, prof ? &sub : nullptr, &nl))) return rc;
        launches += nl;
      }
      ++bodies;
    }
    CK(cudaMemcpyAsync(h->host_state, h->state.p, sizeof(SolveState), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    ++host_syncs;
    if (prof) {
      for (int b2 = 0; b2 < every; ++b2)
        for (int ph = 0; ph < 6; ++ph) {
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, evs[7 * b2 + ph], evs[7 * b2 + ph + 1]));
          tph[ph] += ms;
        }
    }
    if (h->host_state->done) break;
  }
  for (auto& e : evs) cudaEventDestroy(e);
  if (graph) launches += 1;  // the arm kernel; bodies are counted from the outer-loop count below
  // final true residual for the statistics
  CK(launch_final_norm(h->state.p, h->op, h->b.p, h->x.p, h->rt.p, h->partials.p, reduce_blocks(n), st));
  launches += 2;
  CK(cudaMemcpyAsync(x, h->x.p, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(h->host_state, h->state.p, sizeof(SolveState), cudaMemcpyDeviceToHost, st));
  std::vector<sscg_outer_record> hh;
  const SolveState& s0 = *h->host_state;
  CK(cudaStreamSynchronize(st));
  ++host_syncs;
  const SolveState s = s0;
  const int outer = s.k;
  if (graph) launches += std::max(outer, 1) * h->graph_launches;  // one body per outer loop
  const int nh = std::min(outer, hist_cap);
  if (nh > 0) {
    hh.resize(nh);
    CK(cudaMemcpy(hh.data(), h->hist.p, nh * sizeof(sscg_outer_record), cudaMemcpyDeviceToHost));
  }
  h->last_lmin = s.lmin;
  h->last_lmax = s.lmax;
  if ((rc = join_out(h))) return rc;
  if (stats) {
    stats->status = s.status;
    stats->outer_iters = outer;
    stats->inner_iters = s.m;
    stats->host_syncs = host_syncs;
    stats->replacements = s.replacements;
    stats->fp32_replacements = s.fp32_replacements;
    stats->kernel_launches = launches;
    stats->lambda_min = s.lmin;
    stats->lambda_max = s.lmax;
    stats->c_last = s.c;
    stats->true_relres = s.normb > 0.0 ? std::sqrt(s.rt2) / s.normb : 0.0;
    stats->upd_relres = s.upd_relres;
    stats->t_mpk_ms = tph[0];
    stats->t_gram_ms = tph[1];
    stats->t_kappa_ms = tph[2];
    stats->t_control_ms = tph[3];
    stats->t_recombine_ms = tph[4];
    stats->t_other_ms = tph[5];
    stats->n_gram_launches = prof ? outer : 0;
    double gf = 0.0, mf = 0.0;
    for (int k = 0; k < nh; ++k) {
      const int nc = 2 * hh[k].sbar + 1;
      gf += 2.0 * (double)n * (nc * (nc + 1) / 2);
      mf += (double)(2 * hh[k].sbar - 1);
    }
    stats->gram_flops = gf;
    stats->mpk_spmvs = mf;
    if (stats->hist && stats->hist_cap > 0) {
      const int cp = std::min(nh, stats->hist_cap);
      std::memcpy(stats->hist, hh.data(), cp * sizeof(sscg_outer_record));
      stats->hist_len = cp;
    } else {
      stats->hist_len = 0;
    }
  }
  (void)bodies;
  return s.status;
}

int sscg_solve_host(sscg_t h, const double* b_host, double* x_host, double tol, int s_max, sscg_basis basis,
                    const sscg_opts* opts, sscg_stats* stats) {
  if (!h || !b_host || !x_host) return SSCG_ERR_INVALID_ARG;
  const int64_t n = h->n;
  DevBuf<double> db, dx;
  CK(db.ensure(n));
  CK(dx.ensure(n));
  CK(cudaMemcpyAsync(db.p, b_host, n * sizeof(double), cudaMemcpyHostToDevice, h->user_stream));
  CK(cudaMemcpyAsync(dx.p, x_host, n * sizeof(double), cudaMemcpyHostToDevice, h->user_stream));
  int rc = sscg_solve(h, db.p, dx.p, tol, s_max, basis, opts, stats);
  if (rc < 0) {
    db.release();
    dx.release();
    return rc;
  }
  cudaError_t e = cudaMemcpyAsync(x_host, dx.p, n * sizeof(double), cudaMemcpyDeviceToHost, h->user_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->user_stream);
  db.release();
  dx.release();
  if (e != cudaSuccess) return cuda_fail(e, "solve_host copy back");
  return rc;
}

int sscg_solve_hscg(sscg_t h, const double* b, double* x, double tol, int max_iters, sscg_stats* stats) {
  return sscg_solve_hscg_ex(h, b, x, tol, max_iters, 16, stats);
}

int sscg_solve_hscg_ex(sscg_t h, const double* b, double* x, double tol, int max_iters, int spmv_fp64_per16,
                       sscg_stats* stats) {
  if (!h || !b || !x || !(tol > 0.0)) return SSCG_ERR_INVALID_ARG;
  if (spmv_fp64_per16 < -1 || spmv_fp64_per16 > 16) return SSCG_ERR_INVALID_ARG;
  const int64_t n = h->n;
  cudaStream_t st = h->stream;
  int rc;
  if ((rc = ensure_solve_buffers(h, 1, 0))) return rc;
  CK(h->r.ensure(n));
  CK(h->p.ensure(n));
  CK(h->q.ensure(n));
  if ((rc = join_in(h))) return rc;
  CK(cudaMemcpyAsync(h->b.p, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(h->x.p, x, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  SolveState& hs = *h->host_state;
  std::memset(&hs, 0, sizeof(hs));
  hs.tol = tol;
  hs.status = SSCG_NOT_CONVERGED;
  hs.h_max_iters = max_iters > 0 ? max_iters : 100000;
  hs.max_outer = hs.h_max_iters;
  CK(launch_set_state(h->state.p, hs, st));
  const int nb = reduce_blocks(n);
  CK(launch_hscg_init(h->state.p, h->op, h->b.p, h->x.p, h->r.p, h->p.p, h->partials.p, nb, st));
  int launches = 3, host_syncs = 0;
  // Iterations run inside one graph: WHILE (not done) { 8 iterations, then the
  // true-residual confirmation }.  Kernels of iterations past convergence exit
  // at once.
  const int per_check = 8;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  int body_kernels = 0;
  {
    cudaError_t e;
    auto fail = [&](cudaError_t er, const char* w) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(er, w);
    };
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return fail(e, "cudaGraphCreate");
    cudaGraphConditionalHandle cond;
    if ((e = cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
      return fail(e, "cond handle");
    if ((e = cudaStreamBeginCaptureToGraph(st, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
      return fail(e, "capture arm");
    cudaError_t ea = launch_batch_arm(cond, st);
    cudaGraph_t tmp;
    e = cudaStreamEndCapture(st, &tmp);
    if (ea != cudaSuccess) return fail(ea, "arm");
    if (e != cudaSuccess) return fail(e, "end capture arm");
    size_t nn = 1;
    cudaGraphNode_t arm_node;
    if ((e = cudaGraphGetNodes(g, &arm_node, &nn)) != cudaSuccess) return fail(e, "nodes");
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    if ((e = cudaGraphAddNode(&wnode, g, &arm_node, nullptr, 1, &cp)) != cudaSuccess) return fail(e, "while node");
    if ((e = cudaStreamBeginCaptureToGraph(st, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return fail(e, "capture body");
    cudaError_t eb = cudaSuccess;
    for (int it = 0; it < per_check && eb == cudaSuccess; ++it)
      eb = launch_hscg_iteration(h->state.p, h->op, h->x.p, h->r.p, h->p.p, h->q.p, h->partials.p, nb, st,
                                 spmv_fp64_per16);
    if (eb == cudaSuccess)
      eb = launch_hscg_check(h->state.p, h->op, h->b.p, h->x.p, h->r.p, h->p.p, h->rt.p, h->partials.p, nb, st);
    if (eb == cudaSuccess) eb = launch_solve_cond(h->state.p, cond, st);
    e = cudaStreamEndCapture(st, &tmp);
    if (eb != cudaSuccess) return fail(eb, "hscg body");
    if (e != cudaSuccess) return fail(e, "end capture body");
    body_kernels = 4 * per_check + 4 + 1;
    if ((e = cudaGraphInstantiate(&ge, g, 0)) != cudaSuccess) return fail(e, "instantiate");
    cudaGraphDestroy(g);
    g = nullptr;
  }
  cudaError_t el = cudaGraphLaunch(ge, st);
  if (el != cudaSuccess) {
    cudaGraphExecDestroy(ge);
    return cuda_fail(el, "hscg graph launch");
  }
  CK(launch_final_norm(h->state.p, h->op, h->b.p, h->x.p, h->rt.p, h->partials.p, nb, st));
  CK(cudaMemcpyAsync(x, h->x.p, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(h->host_state, h->state.p, sizeof(SolveState), cudaMemcpyDeviceToHost, st));
  const cudaError_t es = cudaStreamSynchronize(st);
  cudaGraphExecDestroy(ge);
  CK(es);
  ++host_syncs;
  const SolveState s = *h->host_state;
  launches += 1 + ((s.h_iters + per_check - 1) / per_check + 1) * body_kernels;
  if ((rc = join_out(h))) return rc;
  if (stats) {
    stats->status = s.status;
    stats->outer_iters = s.h_iters;
    stats->inner_iters = s.h_iters;
    stats->host_syncs = host_syncs;
    stats->replacements = s.replacements;
    stats->kernel_launches = launches + 2;
    stats->true_relres = s.normb > 0.0 ? std::sqrt(s.rt2) / s.normb : 0.0;
    stats->upd_relres = s.normb > 0.0 ? std::sqrt(s.h_rr) / s.normb : 0.0;
    stats->hist_len = 0;
  }
  return s.status;
}


int sscg_solve_batch(const sscg_t* systems, int nsys, const int* nrhs, const double* b, double* x, double tol,
                     const int* s_max, sscg_basis basis, const sscg_opts* opts, sscg_batch_stats* stats,
                     void* cuda_stream) {
  if (!systems || nsys <= 0 || !nrhs || !b || !x || !s_max || !(tol > 0.0)) return SSCG_ERR_INVALID_ARG;
  if (basis < SSCG_MONOMIAL || basis > SSCG_CHEBYSHEV) return SSCG_ERR_INVALID_ARG;
  sscg_opts o;
  sscg_opts_default(&o);
  if (opts) o = *opts;
  int rc = validate_opts(o);
  if (rc) return rc;
  if (o.y_fp32 || (o.gram_mode != 0 && o.gram_mode != 3) || o.ritz_exact || o.recompute_y)
    return SSCG_ERR_UNSUPPORTED;
  // ---- pairs, chunks and Gram blocks (host)
  const int chunk_rows = o.batch_chunk_rows > 0 ? o.batch_chunk_rows : kBatchChunk;
  const int gram_rows = o.batch_gram_rows > 0 ? o.batch_gram_rows : kBatchGramRows;
  if (o.gram_mode == 3) {
    if (gram_rows > (1 << 14)) return SSCG_ERR_INVALID_ARG;   // one tcgen05 Gram block sums at most 16384 rows
    CK(gram_prepare());
  }
  std::vector<BatchPair> pairs;
  std::vector<int> chunk_pair, gblk_pair, pair_sigma;
  int64_t off = 0;
  int sigma_max = 1;
  for (int s = 0; s < nsys; ++s) {
    if (!systems[s] || nrhs[s] < 0 || s_max[s] < 1 || s_max[s] > kMaxS) return SSCG_ERR_INVALID_ARG;
    const int64_t n = systems[s]->n;
    for (int k = 0; k < nrhs[s]; ++k) {
      BatchPair bp;
      bp.op = systems[s]->op;
      bp.off = off;
      bp.n = n;
      bp.chunk0 = (int)chunk_pair.size();
      bp.nchunk = (int)((n + chunk_rows - 1) / chunk_rows);
      bp.gblk0 = (int)gblk_pair.size();
      bp.ngblk = (int)((n + gram_rows - 1) / gram_rows);
      const int j = (int)pairs.size();
      for (int c = 0; c < bp.nchunk; ++c) chunk_pair.push_back(j);
      for (int g = 0; g < bp.ngblk; ++g) gblk_pair.push_back(j);
      pairs.push_back(bp);
      pair_sigma.push_back(s_max[s]);
      sigma_max = std::max(sigma_max, s_max[s]);
      off += n;
    }
  }
  const int P = (int)pairs.size();
  if (P == 0) return SSCG_OK;
  const int64_t total = off;
  const int64_t LD = round_up(total, 32);
  const int hist_cap = 0;
  // ---- device buffers for the call
  DevBuf<BatchPair> d_pairs;
  DevBuf<int> d_cp, d_gp;
  DevBuf<SolveState> d_st;
  DevBuf<double> d_G, d_Y, d_part, d_rt;
  const double* d_leja = nullptr;
  DevBuf<unsigned int> d_cnt;
  auto release = [&]() {
    d_pairs.release(); d_cp.release(); d_gp.release(); d_st.release(); d_G.release(); d_Y.release();
    d_part.release(); d_rt.release(); d_cnt.release();
  };
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr, t0 = nullptr, t1 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int result = SSCG_OK;
  float device_ms = 0.f;
  std::vector<SolveState> hs(P);
  int launches = 0, host_syncs = 0, graph_launches = 0;
  unsigned int bodies_run = 0;
  do {
    cudaError_t e;
#define BK(call)                                  \
  if ((e = (call)) != cudaSuccess) {              \
    result = cuda_fail(e, #call);                 \
    break;                                        \
  }
    BK(d_pairs.ensure(P));
    BK(d_cp.ensure(chunk_pair.size()));
    BK(d_gp.ensure(gblk_pair.size()));
    BK(d_st.ensure(P));
    BK(d_G.ensure((size_t)P * kMaxCols * kMaxCols));
    BK(d_Y.ensure((size_t)LD * (2 * sigma_max + 1)));
    BK(d_part.ensure(std::max(gblk_pair.size() * (size_t)kMaxPairs, chunk_pair.size())));
    BK(d_rt.ensure(total));
    BK(d_cnt.ensure(2));
    BK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    BK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    BK(cudaEventCreate(&t0));
    BK(cudaEventCreate(&t1));
    BK(cudaEventRecord(ev, (cudaStream_t)cuda_stream));
    BK(cudaStreamWaitEvent(st, ev, 0));
    for (int j = 0; j < P; ++j) fill_state_config(hs[j], pair_sigma[j], tol, (int)basis, o, hist_cap);
    BK(cudaMemcpyAsync(d_pairs.p, pairs.data(), P * sizeof(BatchPair), cudaMemcpyHostToDevice, st));
    BK(cudaMemcpyAsync(d_cp.p, chunk_pair.data(), chunk_pair.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    BK(cudaMemcpyAsync(d_gp.p, gblk_pair.data(), gblk_pair.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    BK(cudaMemcpyAsync(d_st.p, hs.data(), P * sizeof(SolveState), cudaMemcpyHostToDevice, st));
    BK(cudaMemsetAsync(d_cnt.p, 0, 2 * sizeof(unsigned int), st));
    BK(leja_table(&d_leja, st));
    BatchView v;
    v.pairs = d_pairs.p;
    v.npairs = P;
    v.chunk_pair = d_cp.p;
    v.nchunks = (int)chunk_pair.size();
    v.gblk_pair = d_gp.p;
    v.ngblk = (int)gblk_pair.size();
    v.states = d_st.p;
    v.G = d_G.p;
    v.hist = nullptr;
    v.hist_cap = 0;
    v.active = d_cnt.p;
    v.bodies = d_cnt.p + 1;
    v.max_bodies = (o.max_outer > 0 ? o.max_outer : 100000) + 2;
    v.chunk_rows = chunk_rows;
    v.gram_rows = gram_rows;
    BK(launch_batch_init(v, b, x, d_Y.p, LD, d_part.p, st));
    launches += 3;
    auto body = [&](cudaGraphConditionalHandle cond, int use_cond) -> cudaError_t {
      cudaError_t e2;
      if ((e2 = launch_batch_begin(v, st)) != cudaSuccess) return e2;
      for (int l = 0; l < sigma_max; ++l)
        if ((e2 = launch_batch_mpk(v, d_Y.p, LD, l, st, o.mpk_fp64_per16)) != cudaSuccess) return e2;
      if ((e2 = launch_batch_gram(v, d_Y.p, LD, d_part.p, st, o.gram_mode)) != cudaSuccess) return e2;
      if ((e2 = launch_batch_kappa(v, sigma_max, st)) != cudaSuccess) return e2;
      if ((e2 = launch_batch_control(v, d_leja, st)) != cudaSuccess) return e2;
      if ((e2 = launch_batch_recombine(v, d_Y.p, LD, x, st, o.rec_fp64_per16)) != cudaSuccess) return e2;
      if ((e2 = launch_batch_check(v, b, x, d_rt.p, d_Y.p, LD, d_part.p, st)) != cudaSuccess) return e2;
      return launch_batch_end(v, cond, use_cond, st);
    };
    const int body_kernels = sigma_max + 9;
    if (o.use_graph) {
      // one graph: arm the condition, then WHILE (condition) { one outer loop }
      BK(cudaGraphCreate(&graph, 0));
      cudaGraphConditionalHandle cond;
      BK(cudaGraphConditionalHandleCreate(&cond, graph, 0, cudaGraphCondAssignDefault));
      BK(cudaStreamBeginCaptureToGraph(st, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      cudaError_t ea = launch_batch_arm(cond, st);
      cudaGraph_t tmp;
      cudaError_t ee = cudaStreamEndCapture(st, &tmp);
      BK(ea);
      BK(ee);
      size_t nn = 1;
      cudaGraphNode_t arm_node;
      BK(cudaGraphGetNodes(graph, &arm_node, &nn));
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = cond;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t wnode;
      BK(cudaGraphAddNode(&wnode, graph, &arm_node, nullptr, 1, &cp));
      cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
      BK(cudaStreamBeginCaptureToGraph(st, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      cudaError_t eb = body(cond, 1);
      ee = cudaStreamEndCapture(st, &tmp);
      BK(eb);
      BK(ee);
      BK(cudaGraphInstantiate(&gexec, graph, 0));
      BK(cudaEventRecord(t0, st));
      BK(cudaGraphLaunch(gexec, st));
      BK(cudaEventRecord(t1, st));
      ++graph_launches;
    } else {
      BK(cudaEventRecord(t0, st));
      const int every = std::max(1, o.check_every);
      unsigned int cnt[2] = {1u, 0u};
      while (true) {
        for (int i = 0; i < every; ++i) {
          cudaError_t eb = body(cudaGraphConditionalHandle(), 0);
          BK(eb);
        }
        if (result) break;
        BK(cudaMemcpyAsync(cnt, d_cnt.p, sizeof(cnt), cudaMemcpyDeviceToHost, st));
        BK(cudaStreamSynchronize(st));
        ++host_syncs;
        if (cnt[0] == 0u || cnt[1] >= (unsigned)v.max_bodies) break;
      }
      if (result) break;
      BK(cudaEventRecord(t1, st));
    }
    BK(cudaMemcpyAsync(hs.data(), d_st.p, P * sizeof(SolveState), cudaMemcpyDeviceToHost, st));
    BK(cudaMemcpyAsync(&bodies_run, d_cnt.p + 1, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    BK(cudaStreamSynchronize(st));
    ++host_syncs;
    launches += (int)bodies_run * body_kernels;
    BK(cudaEventElapsedTime(&device_ms, t0, t1));
    BK(cudaEventRecord(ev, st));
    BK(cudaStreamWaitEvent((cudaStream_t)cuda_stream, ev, 0));
#undef BK
  } while (0);
  if (gexec) cudaGraphExecDestroy(gexec);
  if (graph) cudaGraphDestroy(graph);
  if (st) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  if (ev) cudaEventDestroy(ev);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  release();
  if (result) return result;
  int conv = 0, worst = SSCG_OK, max_outer = 0;
  int64_t inner = 0;
  double max_rel = 0.0;
  for (int j = 0; j < P; ++j) {
    const SolveState& q = hs[j];
    const int status = q.done ? q.status : SSCG_NOT_CONVERGED;
    if (status == SSCG_OK) ++conv;
    else if (worst == SSCG_OK) worst = status;
    max_outer = std::max(max_outer, q.k);
    inner += q.m;
    const double rel = q.normb > 0.0 ? std::sqrt(q.rt2) / q.normb : 0.0;
    max_rel = std::max(max_rel, rel);
    if (stats) {
      if (stats->pair_status) stats->pair_status[j] = status;
      if (stats->pair_outer) stats->pair_outer[j] = q.k;
      if (stats->pair_inner) stats->pair_inner[j] = q.m;
    }
  }
  if (stats) {
    stats->npairs = P;
    stats->converged = conv;
    stats->outer_loops = max_outer;
    stats->host_syncs = host_syncs;
    stats->kernel_launches = launches;
    stats->graph_launches = graph_launches;
    stats->inner_iters = inner;
    stats->max_true_relres = max_rel;
    stats->device_ms = device_ms;
  }
  return worst;
}

int sscg_solve_batch_hscg(const sscg_t* systems, int nsys, const int* nrhs, const double* b, double* x, double tol,
                          int max_iters, int chunk_rows_opt, sscg_batch_stats* stats, void* cuda_stream) {
  if (!systems || nsys <= 0 || !nrhs || !b || !x || !(tol > 0.0)) return SSCG_ERR_INVALID_ARG;
  if (chunk_rows_opt != 0 && (chunk_rows_opt < 128 || chunk_rows_opt > (1 << 20))) return SSCG_ERR_INVALID_ARG;
  const int chunk_rows = chunk_rows_opt > 0 ? chunk_rows_opt : kBatchChunk;
  const int iters_cap = max_iters > 0 ? max_iters : 100000;
  constexpr int kItersPerBody = 8;
  std::vector<BatchPair> pairs;
  std::vector<int> chunk_pair;
  int64_t off = 0;
  for (int s = 0; s < nsys; ++s) {
    if (!systems[s] || nrhs[s] < 0) return SSCG_ERR_INVALID_ARG;
    const int64_t n = systems[s]->n;
    for (int k = 0; k < nrhs[s]; ++k) {
      BatchPair bp;
      bp.op = systems[s]->op;
      bp.off = off;
      bp.n = n;
      bp.chunk0 = (int)chunk_pair.size();
      bp.nchunk = (int)((n + chunk_rows - 1) / chunk_rows);
      bp.gblk0 = 0;
      bp.ngblk = 0;
      const int j = (int)pairs.size();
      for (int c = 0; c < bp.nchunk; ++c) chunk_pair.push_back(j);
      pairs.push_back(bp);
      off += n;
    }
  }
  const int P = (int)pairs.size();
  if (P == 0) return SSCG_OK;
  const int64_t total = off;
  DevBuf<BatchPair> d_pairs;
  DevBuf<int> d_cp;
  DevBuf<SolveState> d_st;
  DevBuf<double> d_r, d_p, d_q, d_rt, d_part;
  DevBuf<unsigned int> d_cnt;
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr, t0 = nullptr, t1 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int result = SSCG_OK;
  float device_ms = 0.f;
  std::vector<SolveState> hs(P);
  int launches = 0;
  unsigned int bodies_run = 0;
  do {
    cudaError_t e;
#define BK(call)                                  \
  if ((e = (call)) != cudaSuccess) {              \
    result = cuda_fail(e, #call);                 \
    break;                                        \
  }
    BK(d_pairs.ensure(P));
    BK(d_cp.ensure(chunk_pair.size()));
    BK(d_st.ensure(P));
    BK(d_r.ensure(total));
    BK(d_p.ensure(total));
    BK(d_q.ensure(total));
    BK(d_rt.ensure(total));
    BK(d_part.ensure(chunk_pair.size()));
    BK(d_cnt.ensure(2));
    BK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    BK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    BK(cudaEventCreate(&t0));
    BK(cudaEventCreate(&t1));
    BK(cudaEventRecord(ev, (cudaStream_t)cuda_stream));
    BK(cudaStreamWaitEvent(st, ev, 0));
    for (int j = 0; j < P; ++j) {
      std::memset(&hs[j], 0, sizeof(SolveState));
      hs[j].tol = tol;
      hs[j].status = SSCG_NOT_CONVERGED;
      hs[j].h_max_iters = iters_cap;
    }
    BK(cudaMemcpyAsync(d_pairs.p, pairs.data(), P * sizeof(BatchPair), cudaMemcpyHostToDevice, st));
    BK(cudaMemcpyAsync(d_cp.p, chunk_pair.data(), chunk_pair.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    BK(cudaMemcpyAsync(d_st.p, hs.data(), P * sizeof(SolveState), cudaMemcpyHostToDevice, st));
    BK(cudaMemsetAsync(d_cnt.p, 0, 2 * sizeof(unsigned int), st));
    BatchView v;
    std::memset(&v, 0, sizeof(v));
    v.pairs = d_pairs.p;
    v.npairs = P;
    v.chunk_pair = d_cp.p;
    v.nchunks = (int)chunk_pair.size();
    v.states = d_st.p;
    v.active = d_cnt.p;
    v.bodies = d_cnt.p + 1;
    v.max_bodies = (iters_cap + kItersPerBody - 1) / kItersPerBody + 2;
    v.chunk_rows = chunk_rows;
    v.gram_rows = kBatchGramRows;
    BK(launch_batch_hscg_init(v, b, x, d_r.p, d_p.p, d_part.p, st));
    launches += 3;
    // one graph: arm the condition, then WHILE (a pair is running) { 8 iterations, confirmation }
    BK(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle cond;
    BK(cudaGraphConditionalHandleCreate(&cond, graph, 0, cudaGraphCondAssignDefault));
    BK(cudaStreamBeginCaptureToGraph(st, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    cudaError_t ea = launch_batch_arm(cond, st);
    cudaGraph_t tmp;
    cudaError_t ee = cudaStreamEndCapture(st, &tmp);
    BK(ea);
    BK(ee);
    size_t nn = 1;
    cudaGraphNode_t arm_node;
    BK(cudaGraphGetNodes(graph, &arm_node, &nn));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    BK(cudaGraphAddNode(&wnode, graph, &arm_node, nullptr, 1, &cp));
    cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
    BK(cudaStreamBeginCaptureToGraph(st, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    cudaError_t eb = launch_batch_begin(v, st);
    for (int i = 0; i < kItersPerBody && eb == cudaSuccess; ++i)
      eb = launch_batch_hscg_iteration(v, x, d_r.p, d_p.p, d_q.p, d_part.p, st);
    if (eb == cudaSuccess) eb = launch_batch_hscg_check(v, b, x, d_rt.p, d_r.p, d_p.p, d_part.p, cond, 1, st);
    ee = cudaStreamEndCapture(st, &tmp);
    BK(eb);
    BK(ee);
    BK(cudaGraphInstantiate(&gexec, graph, 0));
    BK(cudaEventRecord(t0, st));
    BK(cudaGraphLaunch(gexec, st));
    BK(cudaEventRecord(t1, st));
    BK(cudaMemcpyAsync(hs.data(), d_st.p, P * sizeof(SolveState), cudaMemcpyDeviceToHost, st));
    BK(cudaMemcpyAsync(&bodies_run, d_cnt.p + 1, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    BK(cudaStreamSynchronize(st));
    BK(cudaEventElapsedTime(&device_ms, t0, t1));
    launches += 1 + (int)bodies_run * (1 + 3 * kItersPerBody + 4);
    BK(cudaEventRecord(ev, st));
    BK(cudaStreamWaitEvent((cudaStream_t)cuda_stream, ev, 0));
#undef BK
  } while (0);
  if (gexec) cudaGraphExecDestroy(gexec);
  if (graph) cudaGraphDestroy(graph);
  if (st) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  if (ev) cudaEventDestroy(ev);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (result) return result;
  int conv = 0, worst = SSCG_OK, max_it = 0;
  int64_t inner = 0;
  double max_rel = 0.0;
  for (int j = 0; j < P; ++j) {
    const SolveState& q = hs[j];
    const int status = q.done ? q.status : SSCG_NOT_CONVERGED;
    if (status == SSCG_OK) ++conv;
    else if (worst == SSCG_OK) worst = status;
    max_it = std::max(max_it, q.h_iters);
    inner += q.h_iters;
    const double rel = q.normb > 0.0 ? std::sqrt(q.rt2) / q.normb : 0.0;
    max_rel = std::max(max_rel, rel);
    if (stats) {
      if (stats->pair_status) stats->pair_status[j] = status;
      if (stats->pair_outer) stats->pair_outer[j] = q.h_iters;
      if (stats->pair_inner) stats->pair_inner[j] = q.h_iters;
    }
  }
  if (stats) {
    stats->npairs = P;
    stats->converged = conv;
    stats->outer_loops = max_it;
    stats->host_syncs = 1;
    stats->kernel_launches = launches;
    stats->graph_launches = 1;
    stats->inner_iters = inner;
    stats->max_true_relres = max_rel;
    stats->device_ms = device_ms;
  }
  return worst;
}

int sscg_autotune_batch(const sscg_t* systems, int nsys, const int* nrhs, const double* b, double tol,
                        const int* s_max, sscg_basis basis, const int* chunk_rows, const int* gram_rows, int ncand,
                        int trial_outer, int* best, double* times, void* cuda_stream) {
  return sscg_autotune_batch_ex(systems, nsys, nrhs, b, tol, s_max, basis, chunk_rows, gram_rows, nullptr, ncand,
                                trial_outer, best, times, cuda_stream);
}

int sscg_autotune_batch_ex(const sscg_t* systems, int nsys, const int* nrhs, const double* b, double tol,
                           const int* s_max, sscg_basis basis, const int* chunk_rows, const int* gram_rows,
                           const int* gram_modes, int ncand, int trial_outer, int* best, double* times,
                           void* cuda_stream) {
  if (!systems || nsys <= 0 || !nrhs || !b || !s_max || !chunk_rows || !gram_rows || ncand <= 0 ||
      trial_outer <= 0 || !best || !(tol > 0.0))
    return SSCG_ERR_INVALID_ARG;
  int64_t total = 0;
  for (int s = 0; s < nsys; ++s) {
    if (!systems[s] || nrhs[s] < 0) return SSCG_ERR_INVALID_ARG;
    total += (int64_t)nrhs[s] * systems[s]->n;
  }
  if (total == 0) {
    *best = 0;
    return SSCG_OK;
  }
  DevBuf<double> dx;
  int rc = SSCG_OK;
  cudaError_t e = dx.ensure(total);
  if (e != cudaSuccess) rc = cuda_fail(e, "autotune_batch scratch");
  double best_t = 0.0;
  *best = -1;
  for (int i = 0; i < ncand && rc == SSCG_OK; ++i) {
    sscg_opts o;
    sscg_opts_default(&o);
    o.max_outer = trial_outer;
    o.batch_chunk_rows = chunk_rows[i];
    o.batch_gram_rows = gram_rows[i];
    o.gram_mode = gram_modes ? gram_modes[i] : 0;
    if (validate_opts(o) || (o.gram_mode != 0 && o.gram_mode != 3)) {
      rc = SSCG_ERR_INVALID_ARG;
      break;
    }
    e = cudaMemsetAsync(dx.p, 0, total * sizeof(double), (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "autotune_batch memset");
      break;
    }
    sscg_batch_stats bs;
    std::memset(&bs, 0, sizeof(bs));
    const int r = sscg_solve_batch(systems, nsys, nrhs, b, dx.p, tol, s_max, basis, &o, &bs, cuda_stream);
    if (r < 0) {
      rc = r;
      break;
    }
    const double t = bs.inner_iters > 0 ? 1e3 * bs.device_ms / (double)bs.inner_iters : 0.0;
    if (times) times[i] = t;
    if (*best < 0 || t < best_t) {
      *best = i;
      best_t = t;
    }
  }
  if (rc == SSCG_OK) {
    e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "autotune_batch sync");
  }
  dx.release();
  return rc;
}

int sscg_autotune(sscg_t h, const double* b, double tol, const int* candidates, int ncand, int trial_outer,
                  sscg_basis basis, int* best, double* times) {
  if (!h || !b || !(tol > 0.0) || !candidates || ncand <= 0 || trial_outer <= 0 || !best) return SSCG_ERR_INVALID_ARG;
  for (int i = 0; i < ncand; ++i)
    if (candidates[i] < 1 || candidates[i] > kMaxS) return SSCG_ERR_INVALID_ARG;
  DevBuf<double> dx;
  CK(dx.ensure(h->n));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best_t = 0.0;
  int rc = SSCG_OK;
  for (int i = 0; i < ncand && rc >= 0; ++i) {
    sscg_opts o;
    sscg_opts_default(&o);
    o.max_outer = trial_outer;
    sscg_stats stt;
    std::memset(&stt, 0, sizeof(stt));
    cudaError_t e = cudaMemsetAsync(dx.p, 0, h->n * sizeof(double), h->user_stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, h->user_stream);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "autotune");
      break;
    }
    int r = sscg_solve(h, b, dx.p, tol, candidates[i], basis, &o, &stt);
    if (r < 0) {
      rc = r;
      break;
    }
    if ((e = cudaEventRecord(e1, h->user_stream)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) {
      rc = cuda_fail(e, "autotune");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double per = stt.inner_iters > 0 ? ms / stt.inner_iters : 1e30;
    if (times) times[i] = per;
    if (i == 0 || per < best_t) {
      best_t = per;
      *best = candidates[i];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dx.release();
  return rc < 0 ? rc : SSCG_OK;
}

int sscg_ritz(sscg_t h, double* lmin, double* lmax) {
  if (!h || !lmin || !lmax) return SSCG_ERR_INVALID_ARG;
  *lmin = h->last_lmin;
  *lmax = h->last_lmax;
  return SSCG_OK;
}

int sscg_spmv(sscg_t h, const double* v, double* y) { return sscg_spmv_ex(h, v, y, 16); }

int sscg_spmv_ex(sscg_t h, const double* v, double* y, int fp64_per16) {
  if (!h || !v || !y || fp64_per16 < -1 || fp64_per16 > 16) return SSCG_ERR_INVALID_ARG;
  int rc;
  if ((rc = join_in(h))) return rc;
  CK(launch_spmv_split(h->op, v, y, h->stream, nullptr, 0, fp64_per16));
  if ((rc = join_out(h))) return rc;
  CK(cudaStreamSynchronize(h->stream));
  return SSCG_OK;
}

int sscg_build_basis(sscg_t h, const double* p, const double* r, int s, const double* theta, const double* gamma,
               const double* mu, double* Y, int64_t ldy) {
  return sscg_build_basis_ex(h, p, r, s, theta, gamma, mu, Y, ldy, -1);
}

int sscg_build_basis_ex(sscg_t h, const double* p, const double* r, int s, const double* theta,
                        const double* gamma, const double* mu, double* Y, int64_t ldy, int mpk_fp64_per16) {
  if (!h || !p || !r || !theta || !gamma || !mu || !Y || s < 1 || s > kMaxS || ldy < h->n)
    return SSCG_ERR_INVALID_ARG;
  if (mpk_fp64_per16 < -1 || mpk_fp64_per16 > 16) return SSCG_ERR_INVALID_ARG;
  double coef[3 * kMaxS];
  for (int l = 0; l < s; ++l) {
    if (!(gamma[l] != 0.0)) return SSCG_ERR_INVALID_ARG;
    coef[l] = theta[l];
    coef[kMaxS + l] = 1.0 / gamma[l];
    coef[2 * kMaxS + l] = mu[l];
  }
  DevBuf<double> dc;
  CK(dc.ensure(3 * kMaxS));
  int rc;
  if ((rc = join_in(h))) return rc;
  cudaStream_t st = h->stream;
  CK(cudaMemcpyAsync(dc.p, coef, sizeof(coef), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(Y, p, h->n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(Y + ldy, r, h->n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  LevelCoef lc{dc.p, dc.p + kMaxS, dc.p + 2 * kMaxS};
  for (int l = 0; l < s; ++l) CK(launch_mpk_level(h->op, Y, ldy, l, nullptr, s, lc, false, st, mpk_fp64_per16));
  CK(cudaStreamSynchronize(st));
  if ((rc = join_out(h))) return rc;
  dc.release();
  return SSCG_OK;
}

int sscg_gram(const double* Y, int64_t n, int64_t ldy, int ncols, double* G, void* cuda_stream) {
  if (!Y || !G || n <= 0 || ldy < n || ncols < 1 || ncols > kMaxCols) return SSCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int nb = gram_blocks(n);
  DevBuf<double> part;
  CK(part.ensure((size_t)nb * kMaxPairs));
  CK(launch_gram(Y, n, ldy, nullptr, ncols, nullptr, part.p, nb, G, ncols, false, st));
  CK(cudaStreamSynchronize(st));
  part.release();
  return SSCG_OK;
}

int sscg_gram_ex(const double* Y, int64_t n, int64_t ldy, int ncols, double* G, int mode, void* cuda_stream) {
  if (!Y || !G || n <= 0 || ldy < n || ncols < 1 || ncols > kMaxCols || mode < 0 || mode > 3)
    return SSCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int nb = gram_blocks(n);
  CK(gram_prepare());
  DevBuf<double> part;
  DevBuf<int> cexp;
  CK(part.ensure((size_t)nb * kMaxPairs));
  if (mode >= 2) CK(cexp.ensure((size_t)gram_exp_ints(n)));
  CK(launch_gram(Y, n, ldy, nullptr, ncols, nullptr, part.p, nb, G, ncols, false, st, mode, cexp.p));
  CK(cudaStreamSynchronize(st));
  part.release();
  return SSCG_OK;
}

int sscg_wait_failures(int* flag, int clear) {
  if (!flag) return SSCG_ERR_INVALID_ARG;
  CK(cudaDeviceSynchronize());
  CK(gram_tc_error(flag, clear != 0));
  return SSCG_OK;
}

int sscg_kappa(const double* G, int ldg, int sbar, double kappa_cut, double* kappa, double* lmin, double* lmax,
               void* cuda_stream) {
  if (!G || !kappa || !lmin || !lmax || sbar < 1 || sbar > kMaxS || ldg < 2 * sbar + 1) return SSCG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  CK(launch_kappa(G, ldg, nullptr, sbar, kappa_cut, kappa, lmin, lmax, sbar, st));
  CK(cudaStreamSynchronize(st));
  return SSCG_OK;
}

int sscg_recombine(double* Y, int64_t n, int64_t ldy, int ncols, const double* coef, double* x, int rec_fp64_per16,
                   void* cuda_stream) {
  if (!Y || !coef || !x || n <= 0 || ldy < n || ncols < 1 || ncols > kMaxCols) return SSCG_ERR_INVALID_ARG;
  if (rec_fp64_per16 < -1 || rec_fp64_per16 > 16) return SSCG_ERR_INVALID_ARG;
  SolveState hs;
  std::memset(&hs, 0, sizeof(hs));
  hs.nc = ncols;
  for (int c = 0; c < ncols; ++c) {
    hs.xc[c] = coef[c];
    hs.rc[c] = coef[ncols + c];
    hs.pc[c] = coef[2 * ncols + c];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  DevBuf<SolveState> ds;
  CK(ds.ensure(1));
  CK(cudaMemcpyAsync(ds.p, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
  CK(launch_recombine(ds.p, Y, ldy, x, nullptr, nullptr, n, false, st, rec_fp64_per16));
  CK(cudaStreamSynchronize(st));
  ds.release();
  return SSCG_OK;
}

int sscg_stencil_face_grad(sscg_t h, const double* lam, const double* x, double* gkx, double* gky, double* gkz) {
  if (!h || !lam || !x || !gkx || !gky || h->op.kind != 1 || (h->op.dim == 3 && !gkz)) return SSCG_ERR_INVALID_ARG;
  int rc;
  if ((rc = join_in(h))) return rc;
  CK(launch_face_grad(h->op, lam, x, gkx, gky, gkz, h->stream));
  if ((rc = join_out(h))) return rc;
  return SSCG_OK;
}

int sscg_csr_value_grad(sscg_t h, const double* lam, const double* x, double* gval) {
  if (!h || !lam || !x || !gval || h->op.kind != 0) return SSCG_ERR_INVALID_ARG;
  int rc;
  if ((rc = join_in(h))) return rc;
  CK(launch_csr_grad(h->op, lam, x, gval, h->stream));
  if ((rc = join_out(h))) return rc;
  return SSCG_OK;
}

int sscg_leja(int s, double* t) {
  if (!t || s < 1 || s > kMaxS) return SSCG_ERR_INVALID_ARG;
  DevBuf<double> d;
  CK(d.ensure(kMaxS));
  CK(launch_leja(d.p, s, nullptr));
  CK(cudaMemcpy(t, d.p, s * sizeof(double), cudaMemcpyDeviceToHost));
  d.release();
  return SSCG_OK;
}

}  // extern "C"
