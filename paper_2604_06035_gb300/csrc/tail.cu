// tail.cu -- the small multigrid levels of a V-cycle in one launch.
//
// Below a few thousand octs a level's work no longer fills the GPU and each
// operation would cost a full kernel launch.  The tail kernel runs, in one
// thread-block cluster (16 CTAs on GB300 when the non-portable size is
// available, else 8), every operation of the V-cycle from MG level m0 down to
// the coarsest and back up: pre-smoothing, residual + restriction, the
// coarsest solve (exact 2^3 transform or red-black sweeps), prolongation and
// post-smoothing.  Operations are separated by hardware cluster barriers
// (barrier.cluster arrive.release / wait.acquire); data written by one CTA is
// read by the others through L2 (ld.global.cg).  The arithmetic is the same
// per-oct code as the one-launch-per-operation path (oct_ops.cuh), so the two
// paths give the same results.
#include <cooperative_groups.h>

#include "cmg_internal.cuh"
#include "oct_ops.cuh"

namespace cg = cooperative_groups;

namespace cmg {

namespace {

constexpr int kTailThreads = 512;
constexpr int kMaxTail = 24;

struct TailLevel {
  int64_t n, n_alloc;
  const int32_t *nbr;
  const uint8_t *active;
  const int32_t *father;
  const int32_t *blk;
  const uint64_t *keys;
  void *phi, *g;           // T planes
  double *phi64, *g64;     // FP64 planes (coarsest level of a mixed solve)
  int all_active;
  int zero_coarse;         // restriction from this level zeroes the coarse phi
};

struct TailPlan {
  int m0, last, n_pre, n_post, coarse_sweeps, exact, mixed;
  double h_last;
  TailLevel lv[kMaxTail];
};

// CG: loads through L2 only (another CTA of the cluster may have written the
// data); a single-CTA tail reads through L1.
template <typename T, bool MASK, bool CG>
__device__ void pass(const TailLevel &L, int P, bool zero, int64_t tid, int64_t nthr) {
  T *phi = static_cast<T *>(L.phi);
  const T *g = static_cast<const T *>(L.g);
  const int64_t st = L.n_alloc * 4;
  for (int64_t i = tid; i < L.n; i += nthr) {
    if (P == 0) {
      if (zero)
        dev::sweep_oct<T, 0, true, MASK, CG>(i, L.nbr, phi + st, phi, g, L.active, L.n);
      else
        dev::sweep_oct<T, 0, false, MASK, CG>(i, L.nbr, phi + st, phi, g, L.active, L.n);
    } else {
      dev::sweep_oct<T, 1, false, MASK, CG>(i, L.nbr, phi, phi + st, g + L.n * 4, L.active, L.n);
    }
  }
}

template <typename T, bool CG>
__device__ void colour_pass(const TailLevel &L, int P, bool zero, int64_t tid, int64_t nthr) {
  if (L.all_active)
    pass<T, false, CG>(L, P, zero, tid, nthr);
  else
    pass<T, true, CG>(L, P, zero, tid, nthr);
}

template <typename T, bool CG, class Sync>
__device__ void sweeps(const TailLevel &L, int n_sweeps, bool zero_first, int64_t tid, int64_t nthr, Sync &sync) {
  for (int k = 0; k < n_sweeps; ++k) {
    colour_pass<T, CG>(L, 0, zero_first && k == 0, tid, nthr);
    sync();
    colour_pass<T, CG>(L, 1, false, tid, nthr);
    sync();
  }
}

// The V-cycle from MG level plan.m0 down to the coarsest and back up, by
// nthr threads (thread tid), operations separated by sync().
template <typename T, bool CG, class Sync>
__device__ void tail_body(const TailPlan &plan, int64_t tid, int64_t nthr, Sync &sync) {
  // descend: pre-smoothing, residual + restriction
  for (int m = plan.m0; m < plan.last; ++m) {
    const TailLevel &L = plan.lv[m];
    const TailLevel &C = plan.lv[m + 1];
    sweeps<T, CG>(L, plan.n_pre, true, tid, nthr, sync);
    const T *phi = static_cast<const T *>(L.phi);
    const T *g = static_cast<const T *>(L.g);
    for (int64_t i = tid; i < L.n; i += nthr)
      dev::resid_oct<T, false, true, false, false, false, CG>(
          i, L.nbr, phi, g, L.all_active ? nullptr : L.active, L.n, L.n_alloc, L.father, static_cast<T *>(C.g),
          static_cast<T *>(C.phi), C.n, C.n_alloc, L.zero_coarse, nullptr, 0.0, nullptr, 0.0);
    sync();
  }
  // coarsest level
  {
    const TailLevel &L = plan.lv[plan.last];
    if (plan.exact) {
      if (tid == 0) dev::wht_solve<T, T, CG>(static_cast<const T *>(L.g), static_cast<T *>(L.phi), L.n_alloc,
                                             plan.h_last);
      sync();
    } else if (!plan.mixed) {
      sweeps<T, CG>(L, plan.coarse_sweeps, plan.last > 0, tid, nthr, sync);
    } else {
      // mixed precision: the coarsest level is solved in FP64
      TailLevel L64 = L;
      L64.phi = L.phi64;
      L64.g = L.g64;
      const float *g32 = static_cast<const float *>(L.g);
      for (int64_t t = tid; t < 8 * L.n; t += nthr) L.g64[t] = (double)(CG ? __ldcg(g32 + t) : g32[t]);
      sync();
      sweeps<double, CG>(L64, plan.coarse_sweeps, true, tid, nthr, sync);
      float *p32 = static_cast<float *>(L.phi);
      for (int64_t t = tid; t < 8 * L.n_alloc; t += nthr) p32[t] = (float)(CG ? __ldcg(L.phi64 + t) : L.phi64[t]);
      sync();
    }
  }
  // ascend: prolongation + correction, post-smoothing
  for (int m = plan.last - 1; m >= plan.m0; --m) {
    const TailLevel &L = plan.lv[m];
    const TailLevel &C = plan.lv[m + 1];
    T *phi = static_cast<T *>(L.phi);
    const T *cphi = static_cast<const T *>(C.phi);
    for (int64_t i = tid; i < L.n; i += nthr) {
      if (L.all_active)
        dev::prolong_oct<T, false, CG>(i, L.keys, L.blk, L.n, L.n_alloc, phi, L.active, cphi, C.n_alloc);
      else
        dev::prolong_oct<T, true, CG>(i, L.keys, L.blk, L.n, L.n_alloc, phi, L.active, cphi, C.n_alloc);
    }
    sync();
    sweeps<T, CG>(L, plan.n_post, false, tid, nthr, sync);
  }
}

struct ClusterSync {
  cg::cluster_group cl;
  __device__ void operator()() { cl.sync(); }
};
struct BlockSync {
  __device__ void operator()() { __syncthreads(); }
};

template <typename T>
__global__ void __launch_bounds__(kTailThreads) k_tail(const __grid_constant__ TailPlan plan) {
  ClusterSync sync{cg::this_cluster()};
  const int64_t nthr = (int64_t)sync.cl.num_threads();
  const int64_t tid = (int64_t)sync.cl.block_rank() * blockDim.x + threadIdx.x;
  tail_body<T, true>(plan, tid, nthr, sync);
}

// The same V-cycle tail in one CTA: block barriers, loads through L1.  For
// levels so small that a launch costs more than their arithmetic on one SM.
constexpr int kTail1Threads = 1024;
template <typename T>
__global__ void __launch_bounds__(kTail1Threads) k_tail1(const __grid_constant__ TailPlan plan) {
  BlockSync sync;
  tail_body<T, false>(plan, threadIdx.x, blockDim.x, sync);
}

template <typename T>
int tail_cluster_size() {
  static int size = 0;
  if (size) return size;
  int s = 8;
  if (cudaFuncSetAttribute(k_tail<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(kTailThreads);
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 16;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k_tail<T>, &cfg) == cudaSuccess && clusters > 0) s = 16;
  }
  cudaGetLastError();
  size = s;
  return size;
}

}  // namespace

// Largest first tail level run by one CTA: one SM does ~2 FP64 FMAs per
// clock but ~64 FP32 ones, so the single-CTA tail pays for far larger FP32
// levels than FP64 ones.
template <typename T>
int64_t tail1_max_octs() {
  return sizeof(T) == 8 ? 64 : 4096;
}

template <typename T>
void tail_vcycle(cmg_level *L, int m0, const cmg_solve_params *p, const bool *zero_coarse) {
  const int last = (int)L->mg.size() - 1;
  if (last >= kMaxTail) throw Error(CMG_ERR_INVALID_ARG, "too many multigrid levels for the tail kernel");
  TailPlan plan = {};
  plan.m0 = m0;
  plan.last = last;
  plan.n_pre = p->n_pre;
  plan.n_post = p->n_post;
  plan.coarse_sweeps = p->coarse_sweeps;
  plan.exact = L->exact_coarse ? 1 : 0;
  plan.mixed = sizeof(T) == 4 ? 1 : 0;
  plan.h_last = L->mg[last].h;
  for (int m = m0; m <= last; ++m) {
    MgLev &g = L->mg[m];
    TailLevel &t = plan.lv[m];
    t.n = g.n;
    t.n_alloc = g.n_alloc;
    t.nbr = g.nbr;
    t.active = g.active;
    t.father = g.father;
    t.blk = g.blk;
    t.keys = g.keys;
    t.phi = sizeof(T) == 8 ? (void *)g.phi : (void *)g.phi32;
    t.g = sizeof(T) == 8 ? (void *)g.g : (void *)g.g32;
    t.phi64 = g.phi;
    t.g64 = g.g;
    t.all_active = g.all_active ? 1 : 0;
    t.zero_coarse = (m < last && zero_coarse[m]) ? 1 : 0;
  }
  double cells = 0.0;
  for (int m = m0; m <= last; ++m) cells += 8.0 * L->mg[m].n;
  LaunchScope ls(L->ctx, K_COARSE, cells * (p->n_pre + p->n_post + 2) * 3.0 * sizeof(T),
                 cells * (p->n_pre + p->n_post) * 7.0);
  if (L->mg[m0].n <= tail1_max_octs<T>()) {
    k_tail1<T><<<1, kTail1Threads, 0, L->ctx->stream>>>(plan);
    CMG_CUDA(cudaGetLastError());
    return;
  }
  const int cs = tail_cluster_size<T>();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(kTailThreads);
  cfg.stream = L->ctx->stream;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = cs;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  CMG_CUDA(cudaLaunchKernelEx(&cfg, k_tail<T>, plan));
}

template void tail_vcycle<double>(cmg_level *, int, const cmg_solve_params *, const bool *);
template void tail_vcycle<float>(cmg_level *, int, const cmg_solve_params *, const bool *);

}  // namespace cmg
