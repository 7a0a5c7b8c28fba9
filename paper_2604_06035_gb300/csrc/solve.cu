// solve.cu -- the level solve: V-cycles (App. G Alg. (vcycle), one GPU, no
// halo exchanges) iterated to a relative residual, in FP64 or as FP32
// V-cycles inside FP64 iterative refinement.
//
// The whole solve is one CUDA graph: set-up kernels, then a conditional
// WHILE node whose body is one V-cycle plus the residual norm and a check
// kernel that decides on the device whether to run another cycle, then the
// periodic mean removal and a copy of the statistics to pinned host memory.
// The host waits once per solve.  With profiling on, the same kernels are
// launched one by one from a host loop instead (conditional bodies cannot
// hold event nodes), so that every launch can be bracketed by CUDA events.
#include <cmath>

#include "cmg_internal.cuh"

namespace cmg {

struct SolveCtrl {
  double n0sq, rel_initial, rel_final, blowup;
  int cycles, status, zero, go;
  int err;           // sticky device error of this solve (a grid-barrier timeout)
  unsigned bar[2];   // grid barrier word of the tail kernel (bar[0]), spare
  double hist[256];
};

struct CachedGraph {
  cmg_solve_params p;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches_pre = 0, launches_body = 0, launches_post = 0;
  int64_t updates_per_cycle = 0;
};

namespace {

// The scale of a mixed-precision solve's FP32 correction problem: the power
// of two of the residual norm's binade (a positive finite norm), else the
// norm itself.  A power of two makes the scalings exact.
__global__ void k_pow2_scale(double *dst, const double *src) {
  const double v = *src;
  if (v > 0.0 && v < INFINITY) {
    int e;
    (void)frexp(v, &e);
    *dst = ldexp(1.0, e - 1);
  } else {
    *dst = v;
  }
}

__device__ void decide(SolveCtrl *c, double tol, int fixed, int maxc, cudaGraphConditionalHandle h,
                       int use_handle) {
  int go;
  const double rel = c->rel_final;
  if (c->err != 0) {
    c->status = c->err;
    go = 0;
  } else if (!(rel == rel) || rel > c->blowup || isinf(rel)) {
    c->status = CMG_ERR_DIVERGED;
    go = 0;
  } else if (fixed > 0) {
    c->status = CMG_OK;
    go = c->cycles < fixed;
  } else if (rel <= tol) {
    c->status = CMG_OK;
    go = 0;
  } else {
    c->status = CMG_ERR_NOT_CONVERGED;
    go = c->cycles < maxc;
  }
  c->go = go;
  if (use_handle) cudaGraphSetConditional(h, go ? 1u : 0u);
}

// scal: [0] ||f - L0||^2, [2] ||r||^2 of the initial guess
__global__ void k_ctrl_init(SolveCtrl *c, const double *scal, double tol, int fixed, int maxc,
                            cudaGraphConditionalHandle h, int use_handle) {
  const double n0sq = scal[0];
  c->n0sq = n0sq;
  c->cycles = 0;
  c->err = 0;
  c->bar[0] = c->bar[1] = 0u;
  if (n0sq == 0.0) {
    c->zero = 1;
    c->status = CMG_OK;
    c->rel_initial = c->rel_final = 0.0;
    c->blowup = 0.0;
    c->go = 0;
    if (use_handle) cudaGraphSetConditional(h, 0u);
    return;
  }
  c->zero = 0;
  const double rel = sqrt(scal[2] / n0sq);
  c->rel_initial = rel;
  c->rel_final = rel;
  c->blowup = 1e3 * (rel > 1.0 ? rel : 1.0);
  if (fixed > 0) {
    c->status = CMG_OK;
    c->go = 1;
    if (use_handle) cudaGraphSetConditional(h, 1u);
    return;
  }
  decide(c, tol, 0, maxc, h, use_handle);
}

// The check after a cycle: record rel = sqrt(||r||^2 / ||f - L0||^2), decide.
__device__ void record_and_decide(SolveCtrl *c, double n2, double tol, int fixed, int maxc,
                                  cudaGraphConditionalHandle h, int use_handle) {
  const double rel = sqrt(n2 / c->n0sq);
  const int k = c->cycles;
  if (k < 256) c->hist[k] = rel;
  c->cycles = k + 1;
  c->rel_final = rel;
  decide(c, tol, fixed, maxc, h, use_handle);
}

__global__ void k_ctrl_check(SolveCtrl *c, const double *scal, double tol, int fixed, int maxc,
                             cudaGraphConditionalHandle h, int use_handle) {
  record_and_decide(c, scal[2], tol, fixed, maxc, h, use_handle);
}

// The last step of the residual norm fused with the check (one launch per
// cycle fewer): the block reduction of the residual kernel's per-block
// partial sums in k_finalize's order (the norm is bit-identical), written to
// scal[2] (||r||^2) and scal[3] (||r||), then the check.  One block of 1024
// threads.
__global__ void __launch_bounds__(1024) k_norm_check(const double *__restrict__ partials, int np, double scale,
                                                     double *scal, SolveCtrl *c, double tol, int fixed, int maxc,
                                                     cudaGraphConditionalHandle h, int use_handle) {
  pdl_enter();
  __shared__ double ws[32];
  double v = 0.0;
  for (int t = threadIdx.x; t < np; t += blockDim.x) v += partials[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) {
      const double n2 = scale * w;
      scal[2] = n2;
      scal[3] = sqrt(n2);
      record_and_decide(c, n2, tol, fixed, maxc, h, use_handle);
    }
  }
}

__global__ void k_zero_if(const SolveCtrl *c, double *phi, int64_t n, int64_t n_alloc) {
  if (!c->zero) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 8 * n) return;
  const int p = (int)((t >> 2) & 1);
  phi[(p * n_alloc + (t >> 3)) * 4 + (t & 3)] = 0.0;
}

// Coarse phi must start at zero unless the next operation on it overwrites
// it without reading it (first sweep in zero-init mode, or the exact solve).
bool coarse_needs_zero(const cmg_level *L, int m, const cmg_solve_params *p) {
  const int last = (int)L->mg.size() - 1;
  if (m + 1 < last) return p->n_pre == 0;
  return !L->exact_coarse && p->coarse_sweeps == 0;
}

// First MG level (>= 1) from which every level down to the coarsest has at
// most the schedule's tail size: those levels run in one tail launch.
template <typename T>
int tail_start(const cmg_level *L) {
  const int64_t lim = sizeof(T) == 8 ? L->tail_octs_fp64 : L->tail_octs_fp32;
  if (lim <= 0) return -1;
  int m0 = -1;
  for (int m = (int)L->mg.size() - 1; m >= 1; --m) {
    if (L->mg[m].n > lim) break;
    m0 = m;
  }
  return m0;
}

template <typename T>
void vcycle(cmg_level *L, int m, const cmg_solve_params *p, bool zero_top, int64_t *updates) {
  const int last = (int)L->mg.size() - 1;
  const int prec = sizeof(T) == 8 ? CMG_PREC_FP64 : CMG_PREC_MIXED;
  if (m > 0 && m == tail_start<T>(L)) {
    bool zc[64] = {};
    for (int j = m; j < last && j < 64; ++j) zc[j] = coarse_needs_zero(L, j, p);
    tail_vcycle<T>(L, m, p, zc);
    for (int j = m; j < last; ++j) *updates += (int64_t)(p->n_pre + p->n_post) * 8 * L->mg[j].n;
    if (!L->exact_coarse) *updates += (int64_t)p->coarse_sweeps * 8 * L->mg[last].n;
    return;
  }
  if (m == last) {
    coarse_solve(L, prec, p->coarse_sweeps);
    if (!L->exact_coarse) *updates += (int64_t)p->coarse_sweeps * 8 * L->mg[m].n;
    return;
  }
  for (int k = 0; k < p->n_pre; ++k) sweep<T>(L, m, k == 0 && (m > 0 || zero_top));
  resid_restrict<T>(L, m, true, false, coarse_needs_zero(L, m, p), nullptr, nullptr, p->n_pre >= 1);
  vcycle<T>(L, m + 1, p, false, updates);
  prolong<T>(L, m, p->n_post >= 1);
  for (int k = 0; k < p->n_post; ++k) sweep<T>(L, m, false);
  *updates += (int64_t)(p->n_pre + p->n_post) * 8 * L->mg[m].n;
}

SolveCtrl *ctrl_dev(cmg_level *L) { return reinterpret_cast<SolveCtrl *>(L->ctrl); }

// Whether a V-cycle's last operation on MG level 0 is a colour-1 pass over
// all of it: post-smoothing, or the sweeps of a one-level hierarchy.
bool vcycle_ends_with_colour1(const cmg_level *L, const cmg_solve_params *p) {
  if (L->mg.size() > 1) return p->n_post >= 1;
  return !L->exact_coarse && p->coarse_sweeps >= 1;
}

// Set-up: ghosts, ||f - L0||, initial residual (and, in mixed mode, the
// first FP32 right-hand side), control block.
void segment_pre(cmg_level *L, const cmg_solve_params *p, cudaGraphConditionalHandle h, int use_handle) {
  cudaStream_t s = L->ctx->stream;
  double *scal = L->scal;
  if (p->krylov == 1) {
    pcg_pre(L);
    LaunchScope ls(L->ctx, K_REDUCE, 64.0, 0.0);
    k_ctrl_init<<<1, 1, 0, s>>>(ctrl_dev(L), scal, p->tol, p->fixed_cycles, p->max_cycles, h, use_handle);
    CMG_CUDA(cudaGetLastError());
    return;
  }
  fill_ghosts(L);
  zero_phi_norm(L, scal + 0);
  if (p->precision != CMG_PREC_FP64) {
    LaunchScope ls(L->ctx, K_REDUCE, 16.0, 0.0);
    k_pow2_scale<<<1, 1, 0, s>>>(scal + 4, scal + 1);
    CMG_CUDA(cudaGetLastError());
    resid_restrict<double>(L, 0, false, true, false, scal + 2, scal + 4);
  } else {
    resid_restrict<double>(L, 0, false, true, false, scal + 2);
  }
  LaunchScope ls(L->ctx, K_REDUCE, 64.0, 0.0);
  k_ctrl_init<<<1, 1, 0, s>>>(ctrl_dev(L), scal, p->tol, p->fixed_cycles, p->max_cycles, h, use_handle);
  CMG_CUDA(cudaGetLastError());
}

// The residual norm's reduction (its partial sums written by a residual
// launch with finalize = false) and the check, in one launch.
void norm_check(cmg_level *L, const cmg_solve_params *p, cudaGraphConditionalHandle h, int use_handle) {
  const MgLev &g = L->mg[0];
  const unsigned nb = blocks_for(g.n);
  LaunchScope ls(L->ctx, K_REDUCE, nb * 8.0 + 64.0, nb);
  launch_k(k_norm_check, 1, 1024, L->ctx->stream, L->partials, (int)nb, 36.0 / (g.h * g.h * g.h * g.h), L->scal,
           ctrl_dev(L), p->tol, p->fixed_cycles, p->max_cycles, h, use_handle);
  CMG_CUDA(cudaGetLastError());
}

// One iteration: a V-cycle (FP64), or an FP32 V-cycle (mixed) or FP32 FFT
// solve (fft) of the scaled correction equation + FP64 accumulation, then
// the FP64 residual norm and the check.
void segment_body(cmg_level *L, const cmg_solve_params *p, cudaGraphConditionalHandle h, int use_handle,
                  int64_t *updates) {
  cudaStream_t s = L->ctx->stream;
  double *scal = L->scal;
  if (p->krylov == 1) {
    pcg_body(L, p, updates);
  } else if (p->precision == CMG_PREC_FP64) {
    vcycle<double>(L, 0, p, false, updates);
    resid_restrict<double>(L, 0, false, true, false, scal + 2, nullptr, vcycle_ends_with_colour1(L, p), false);
    norm_check(L, p, h, use_handle);
    return;
  } else {
    MgLev &g = L->mg[0];
    if (p->precision == CMG_PREC_FFT) {
      fft_solve32(L);
    } else {
      if (p->n_pre == 0) {
        CMG_CUDA(cudaMemsetAsync(g.phi32, 0, sizeof(float) * 4 * g.n, s));
        CMG_CUDA(cudaMemsetAsync(g.phi32 + 4 * g.n_alloc, 0, sizeof(float) * 4 * g.n, s));
      }
      for (int k = 0; k < p->inner_cycles; ++k) vcycle<float>(L, 0, p, k == 0, updates);
    }
    accumulate(L, scal + 4);
    {
      LaunchScope ls(L->ctx, K_REDUCE, 16.0, 0.0);
      k_pow2_scale<<<1, 1, 0, s>>>(scal + 4, scal + 3);
    }
    resid_restrict<double>(L, 0, false, true, false, scal + 2, scal + 4, false, false);
    norm_check(L, p, h, use_handle);
    return;
  }
  LaunchScope ls(L->ctx, K_REDUCE, 64.0, 0.0);
  k_ctrl_check<<<1, 1, 0, s>>>(ctrl_dev(L), scal, p->tol, p->fixed_cycles, p->max_cycles, h, use_handle);
  CMG_CUDA(cudaGetLastError());
}

void segment_post(cmg_level *L, const cmg_solve_params *p) {
  MgLev &g = L->mg[0];
  if (p->krylov == 1) pcg_post(L);
  {
    LaunchScope ls(L->ctx, K_CONVERT, 0.0, 0.0);
    k_zero_if<<<blocks_for(8 * g.n), kThreads, 0, L->ctx->stream>>>(ctrl_dev(L), g.phi, g.n, g.n_alloc);
    CMG_CUDA(cudaGetLastError());
  }
  if (L->periodic_full) subtract_mean(L);
}

void copy_ctrl_to_host(cmg_level *L) {
  CMG_CUDA(cudaMemcpyAsync(L->h_ctrl, L->ctrl, sizeof(SolveCtrl), cudaMemcpyDeviceToHost, L->ctx->stream));
}

void fill_stats(cmg_level *L, cmg_solve_stats &S, int64_t updates_per_cycle) {
  const SolveCtrl &c = *reinterpret_cast<const SolveCtrl *>(L->h_ctrl);
  S.cycles = c.cycles;
  S.status = c.status;
  S.rel_initial = c.rel_initial;
  S.rel_final = c.rel_final;
  S.norm0 = std::sqrt(c.n0sq);
  for (int k = 0; k < c.cycles && k < 256; ++k) S.rel_history[k] = c.hist[k];
  S.cell_updates = updates_per_cycle * c.cycles;
}

bool same_params(const cmg_solve_params &a, const cmg_solve_params &b) {
  return a.tol == b.tol && a.max_cycles == b.max_cycles && a.n_pre == b.n_pre && a.n_post == b.n_post &&
         a.coarse_sweeps == b.coarse_sweeps && a.fixed_cycles == b.fixed_cycles && a.precision == b.precision &&
         a.krylov == b.krylov &&
         a.inner_cycles == b.inner_cycles;
}

// Records the solve into a graph on a private stream (capture on the
// caller's stream is impossible when it is the legacy default stream).
CachedGraph *build_graph(cmg_level *L, const cmg_solve_params *p) {
  cmg_ctx *ctx = L->ctx;
  if (!ctx->cap_stream) {
    CMG_CUDA(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    CMG_CUDA(cudaStreamCreateWithFlags(&ctx->cap_stream2, cudaStreamNonBlocking));
  }
  auto *cg = new CachedGraph();
  cg->p = *p;
  cudaStream_t user = ctx->stream;
  CMG_CUDA(cudaGraphCreate(&cg->graph, 0));
  cudaGraphConditionalHandle h;
  CMG_CUDA(cudaGraphConditionalHandleCreate(&h, cg->graph, 0, cudaGraphCondAssignDefault));
  ctx->capturing = true;
  try {
    ctx->stream = ctx->cap_stream;
    CMG_CUDA(cudaStreamBeginCaptureToGraph(ctx->stream, cg->graph, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeRelaxed));
    ctx->captured = 0;
    segment_pre(L, p, h, 1);
    cg->launches_pre = ctx->captured;
    // conditional WHILE node after everything captured so far
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaGraph_t capg = nullptr;
    CMG_CUDA(cudaStreamGetCaptureInfo(ctx->stream, &st, nullptr, &capg, &deps, nullptr, &ndeps));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t cond;
    CMG_CUDA(cudaGraphAddNode(&cond, capg, deps, nullptr, ndeps, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    CMG_CUDA(cudaStreamUpdateCaptureDependencies(ctx->stream, &cond, nullptr, 1, cudaStreamSetCaptureDependencies));
    // body, captured on the second private stream
    cudaStream_t main_cap = ctx->stream;
    ctx->stream = ctx->cap_stream2;
    CMG_CUDA(cudaStreamBeginCaptureToGraph(ctx->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    ctx->captured = 0;
    segment_body(L, p, h, 1, &cg->updates_per_cycle);
    cg->launches_body = ctx->captured;
    cudaGraph_t body_out = nullptr;
    CMG_CUDA(cudaStreamEndCapture(ctx->stream, &body_out));
    ctx->stream = main_cap;
    ctx->captured = 0;
    segment_post(L, p);
    copy_ctrl_to_host(L);
    cg->launches_post = ctx->captured;
    cudaGraph_t out = nullptr;
    CMG_CUDA(cudaStreamEndCapture(ctx->stream, &out));
    CMG_CUDA(cudaGraphInstantiate(&cg->exec, cg->graph, 0));
  } catch (...) {
    cudaStreamCaptureStatus st;
    if (cudaStreamIsCapturing(ctx->cap_stream2, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
      cudaGraph_t g;
      cudaStreamEndCapture(ctx->cap_stream2, &g);
    }
    if (cudaStreamIsCapturing(ctx->cap_stream, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
      cudaGraph_t g;
      cudaStreamEndCapture(ctx->cap_stream, &g);
    }
    cudaGetLastError();
    ctx->stream = user;
    ctx->capturing = false;
    if (cg->graph) cudaGraphDestroy(cg->graph);
    delete cg;
    throw;
  }
  ctx->stream = user;
  ctx->capturing = false;
  return cg;
}

}  // namespace

// One FP64 V-cycle from zero on the level's right-hand side (the CG
// preconditioner, pcg.cu).
int *solve_err_word(cmg_level *L) { return &reinterpret_cast<SolveCtrl *>(L->ctrl)->err; }
unsigned *solve_bar_words(cmg_level *L) { return reinterpret_cast<SolveCtrl *>(L->ctrl)->bar; }

void vcycle64_from_zero(cmg_level *L, const cmg_solve_params *p, int64_t *updates) {
  vcycle<double>(L, 0, p, true, updates);
}

// inner_cycles FP32 V-cycles on MG level 0's FP32 right-hand side, from zero
void vcycle32_from_zero(cmg_level *L, const cmg_solve_params *p, int64_t *updates) {
  MgLev &g = L->mg[0];
  if (p->n_pre == 0) {
    CMG_CUDA(cudaMemsetAsync(g.phi32, 0, sizeof(float) * 4 * g.n, L->ctx->stream));
    CMG_CUDA(cudaMemsetAsync(g.phi32 + 4 * g.n_alloc, 0, sizeof(float) * 4 * g.n, L->ctx->stream));
  }
  for (int k = 0; k < p->inner_cycles; ++k) vcycle<float>(L, 0, p, k == 0, updates);
}

void destroy_graphs(cmg_level *L) {
  for (void *v : L->graphs) {
    auto *cg = static_cast<CachedGraph *>(v);
    if (cg->exec) cudaGraphExecDestroy(cg->exec);
    if (cg->graph) cudaGraphDestroy(cg->graph);
    delete cg;
  }
  L->graphs.clear();
}

// Queue a solve of the level on the context's stream: the cached graph (built
// on first use) and a copy of the control block to pinned host memory, with
// the level's own timing events around them; with profiling on, the
// host-driven loop (which waits every cycle).  solve_wait() completes it.
void solve_launch(cmg_level *L, const cmg_solve_params *p) {
  if (!p || p->n_pre < 0 || p->n_post < 0 || p->coarse_sweeps < 0 || p->max_cycles < 0 || p->max_cycles > 256 ||
      p->fixed_cycles < 0 || p->fixed_cycles > 256 || !(p->tol >= 0.0) ||
      (p->precision != CMG_PREC_FP64 && p->precision != CMG_PREC_MIXED && p->precision != CMG_PREC_FFT) ||
      (p->precision == CMG_PREC_MIXED && p->inner_cycles < 1) || (p->krylov != 0 && p->krylov != 1))
    throw Error(CMG_ERR_INVALID_ARG, "invalid solve parameters");
  if (p->krylov == 1 && p->precision == CMG_PREC_FFT)
    throw Error(CMG_ERR_INVALID_ARG, "the CG outer iteration takes a V-cycle preconditioner (FP64 or MIXED)");
  if (L->periodic_full && L->nx != 1)
    throw Error(CMG_ERR_INVALID_ARG, "periodic base levels need n_x = 1 (exact 2^3 coarsest solve)");
  if (p->precision == CMG_PREC_MIXED && L->mg.size() < 2)
    throw Error(CMG_ERR_INVALID_ARG, "mixed precision needs at least two multigrid levels");
  if (p->precision == CMG_PREC_FFT && !fft_supported(L))
    throw Error(CMG_ERR_INVALID_ARG, "the FFT solve needs a full periodic level of 4^3 .. 512^3 cells");
  if (L->solve_pending) throw Error(CMG_ERR_INVALID_ARG, "a solve of this level is still pending");
  cmg_ctx *ctx = L->ctx;
  if (p->precision != CMG_PREC_FP64) ensure_fp32(L);
  if (p->precision == CMG_PREC_FFT) fft_prepare(L);
  if (p->krylov == 1) pcg_prepare(L);
  if (!L->h_ctrl) CMG_CUDA(cudaMallocHost(&L->h_ctrl, sizeof(SolveCtrl)));
  if (!L->ctrl) L->ctrl = L->mem.alloc<uint8_t>(sizeof(SolveCtrl), true, ctx->stream);
  if (!L->ev_start) CMG_CUDA(cudaEventCreate(&L->ev_start));
  if (!L->ev_end) CMG_CUDA(cudaEventCreate(&L->ev_end));
  L->pend = cmg_level::Pending{};
  if (L->n == 0) {
    L->pend.empty = true;
    L->solve_pending = true;
    return;
  }
  CMG_CUDA(cudaEventRecord(L->ev_start, ctx->stream));
  if (!ctx->profiling) {
    CachedGraph *cg = nullptr;
    for (void *v : L->graphs)
      if (same_params(static_cast<CachedGraph *>(v)->p, *p)) cg = static_cast<CachedGraph *>(v);
    if (!cg) {
      if (L->graphs.size() >= 4) destroy_graphs(L);
      cg = build_graph(L, p);
      L->graphs.push_back(cg);
    }
    CMG_CUDA(cudaGraphLaunch(cg->exec, ctx->stream));
    CMG_CUDA(cudaEventRecord(L->ev_end, ctx->stream));
    L->pend.launches_fixed = cg->launches_pre + cg->launches_post;
    L->pend.launches_body = cg->launches_body;
    L->pend.updates_per_cycle = cg->updates_per_cycle;
  } else {
    // host-driven loop, every launch visible to the profiler
    cudaGraphConditionalHandle none{};
    segment_pre(L, p, none, 0);
    copy_ctrl_to_host(L);
    CMG_CUDA(cudaStreamSynchronize(ctx->stream));
    const SolveCtrl &c = *reinterpret_cast<const SolveCtrl *>(L->h_ctrl);
    int64_t updates_per_cycle = 0;
    while (c.go) {
      int64_t u = 0;
      segment_body(L, p, none, 0, &u);
      updates_per_cycle = u;
      copy_ctrl_to_host(L);
      CMG_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    segment_post(L, p);
    copy_ctrl_to_host(L);
    CMG_CUDA(cudaEventRecord(L->ev_end, ctx->stream));
    L->pend.updates_per_cycle = updates_per_cycle;
  }
  L->solve_pending = true;
}

// Wait for the level's queued solve and report it.
int solve_wait(cmg_level *L, cmg_solve_stats *st) {
  if (!L->solve_pending) throw Error(CMG_ERR_INVALID_ARG, "no solve of this level is pending");
  L->solve_pending = false;
  cmg_solve_stats local;
  cmg_solve_stats &S = st ? *st : local;
  S = cmg_solve_stats{};
  if (L->pend.empty) {
    S.status = CMG_OK;
    return CMG_OK;
  }
  CMG_CUDA(cudaEventSynchronize(L->ev_end));
  const SolveCtrl &c = *reinterpret_cast<const SolveCtrl *>(L->h_ctrl);
  L->ctx->launches += L->pend.launches_fixed + (int64_t)c.cycles * L->pend.launches_body;
  fill_stats(L, S, L->pend.updates_per_cycle);
  float ms = 0.f;
  CMG_CUDA(cudaEventElapsedTime(&ms, L->ev_start, L->ev_end));
  S.ms = ms;
  return S.status;
}

int solve(cmg_level *L, const cmg_solve_params *p, cmg_solve_stats *st) {
  solve_launch(L, p);
  return solve_wait(L, st);
}

}  // namespace cmg
