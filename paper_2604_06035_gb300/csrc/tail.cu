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

template <typename T, bool MASK>
__device__ void pass(const TailLevel &L, int P, bool zero, int64_t tid, int64_t nthr) {
  T *phi = static_cast<T *>(L.phi);
  const T *g = static_cast<const T *>(L.g);
  const int64_t st = L.n_alloc * 4;
  for (int64_t i = tid; i < L.n; i += nthr) {
    if (P == 0) {
      if (zero)
        dev::sweep_oct<T, 0, true, MASK, true>(i, L.nbr, phi + st, phi, g, L.active, L.n);
      else
        dev::sweep_oct<T, 0, false, MASK, true>(i, L.nbr, phi + st, phi, g, L.active, L.n);
    } else {
      dev::sweep_oct<T, 1, false, MASK, true>(i, L.nbr, phi, phi + st, g + L.n * 4, L.active, L.n);
    }
  }
}

template <typename T>
__device__ void colour_pass(const TailLevel &L, int P, bool zero, int64_t tid, int64_t nthr) {
  if (L.all_active)
    pass<T, false>(L, P, zero, tid, nthr);
  else
    pass<T, true>(L, P, zero, tid, nthr);
}

template <typename T>
__device__ void sweeps(const TailLevel &L, int n_sweeps, bool zero_first, int64_t tid, int64_t nthr,
                       cg::cluster_group &cl) {
  for (int k = 0; k < n_sweeps; ++k) {
    colour_pass<T>(L, 0, zero_first && k == 0, tid, nthr);
    cl.sync();
    colour_pass<T>(L, 1, false, tid, nthr);
    cl.sync();
  }
}

template <typename T>
__global__ void __launch_bounds__(kTailThreads) k_tail(const __grid_constant__ TailPlan plan) {
  cg::cluster_group cl = cg::this_cluster();
  const int64_t nthr = (int64_t)cl.num_threads();
  const int64_t tid = (int64_t)cl.block_rank() * blockDim.x + threadIdx.x;
  // descend: pre-smoothing, residual + restriction
  for (int m = plan.m0; m < plan.last; ++m) {
    const TailLevel &L = plan.lv[m];
    const TailLevel &C = plan.lv[m + 1];
    sweeps<T>(L, plan.n_pre, true, tid, nthr, cl);
    const T *phi = static_cast<const T *>(L.phi);
    const T *g = static_cast<const T *>(L.g);
    for (int64_t i = tid; i < L.n; i += nthr)
      dev::resid_oct<T, false, true, false, false, false, true>(
          i, L.nbr, phi, g, L.all_active ? nullptr : L.active, L.n, L.n_alloc, L.father, static_cast<T *>(C.g),
          static_cast<T *>(C.phi), C.n, C.n_alloc, L.zero_coarse, nullptr, 0.0, nullptr, 0.0);
    cl.sync();
  }
  // coarsest level
  {
    const TailLevel &L = plan.lv[plan.last];
    if (plan.exact) {
      if (tid == 0) dev::wht_solve<T, T, true>(static_cast<const T *>(L.g), static_cast<T *>(L.phi), L.n_alloc,
                                               plan.h_last);
      cl.sync();
    } else if (!plan.mixed) {
      sweeps<T>(L, plan.coarse_sweeps, plan.last > 0, tid, nthr, cl);
    } else {
      // mixed precision: the coarsest level is solved in FP64
      TailLevel L64 = L;
      L64.phi = L.phi64;
      L64.g = L.g64;
      const float *g32 = static_cast<const float *>(L.g);
      for (int64_t t = tid; t < 8 * L.n; t += nthr) L.g64[t] = (double)__ldcg(g32 + t);
      cl.sync();
      sweeps<double>(L64, plan.coarse_sweeps, true, tid, nthr, cl);
      float *p32 = static_cast<float *>(L.phi);
      for (int64_t t = tid; t < 8 * L.n_alloc; t += nthr) p32[t] = (float)__ldcg(L.phi64 + t);
      cl.sync();
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
        dev::prolong_oct<T, false, true>(i, L.keys, L.blk, L.n, L.n_alloc, phi, L.active, cphi, C.n_alloc);
      else
        dev::prolong_oct<T, true, true>(i, L.keys, L.blk, L.n, L.n_alloc, phi, L.active, cphi, C.n_alloc);
    }
    cl.sync();
    sweeps<T>(L, plan.n_post, false, tid, nthr, cl);
  }
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
  double cells = 0.0;
  for (int m = m0; m <= last; ++m) cells += 8.0 * L->mg[m].n;
  LaunchScope ls(L->ctx, K_COARSE, cells * (p->n_pre + p->n_post + 2) * 3.0 * sizeof(T),
                 cells * (p->n_pre + p->n_post) * 7.0);
  CMG_CUDA(cudaLaunchKernelEx(&cfg, k_tail<T>, plan));
}

template void tail_vcycle<double>(cmg_level *, int, const cmg_solve_params *, const bool *);
template void tail_vcycle<float>(cmg_level *, int, const cmg_solve_params *, const bool *);

}  // namespace cmg
