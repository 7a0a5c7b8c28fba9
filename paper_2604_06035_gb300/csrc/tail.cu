// tail.cu -- the small multigrid levels of a V-cycle in one launch.
//
// Below a few ten thousand octs a level's work no longer fills the GPU and
// each operation would cost a full kernel launch.  The tail kernel runs every
// operation of the V-cycle from MG level m0 down to the coarsest and back up:
// pre-smoothing, residual + restriction, the coarsest solve (exact 2^3
// transform or red-black sweeps), prolongation and post-smoothing.
//   * Grid tail: one cooperative launch of one CTA per SM.  A level's octs
//     are split into one contiguous chunk per CTA; operations are separated
//     by a grid barrier (a word in the solve's control block, bounded waits
//     that record CMG_ERR_TIMEOUT); loads go through L2
//     (ld.global.cg), since another CTA may have written the data.  Levels
//     small enough for one SM run inside the same launch on CTA 0 alone,
//     with block barriers, while the others wait at the next grid barrier.
//   * Single-CTA tail: when even the first tail level fits one SM, one CTA of
//     1024 threads with block barriers and L1 loads.
// The arithmetic is the same per-oct code as the one-launch-per-operation
// path (oct_ops.cuh), so every schedule gives the same results.
#include "cmg_internal.cuh"
#include "gridsync.cuh"
#include "oct_ops.cuh"

namespace cmg {

namespace {

constexpr int kTailThreads = 512;
constexpr int kMaxTail = 48;  // MG levels of a level at up to level 43 (128-bit keys)

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
  int split;  // grid tail: first level run by CTA 0 alone (last + 1: none)
  double h_last;
  int *err;       // sticky error word of the solve (grid-barrier timeout)
  unsigned *bar;  // grid barrier word
  long long spin_budget;
  TailLevel lv[kMaxTail];
};

// The items a thread handles: a, a + s, ... below e; a - base is the same
// offset for every stride (the thread's rank among the s threads).
struct Span {
  int64_t a, e, s, base;
};
// every thread of one CTA strides over the whole range
struct FlatMap {
  int64_t tid, nthr;
  // octs (or values) [0, n)
  __device__ Span span(int64_t n) const { return {tid, n, nthr, 0}; }
  // k work units per oct over octs [0, n): units [0, k n)
  __device__ Span units(int64_t n, int k) const { return {tid, k * n, nthr, 0}; }
  // whether a colour pass over n octs takes one round of threads per cell
  __device__ bool fits_per_cell(int64_t n) const { return 4 * n <= nthr; }
  __device__ bool first_warp() const { return tid < 32; }
};
// one contiguous chunk of octs per CTA, the CTA's threads striding over it
struct ChunkMap {
  int64_t b, nb, t, nt;
  __device__ Span span(int64_t n) const { return units(n, 1); }
  __device__ Span units(int64_t n, int k) const {
    const int64_t c = (n + nb - 1) / nb;
    const int64_t a = b * c;
    return {k * a + t, k * (a + c < n ? a + c : n), nt, k * a};
  }
  __device__ bool fits_per_cell(int64_t n) const { return 4 * ((n + nb - 1) / nb) <= nt; }
  __device__ bool first_warp() const { return b == 0 && t < 32; }
};

// Small FP64 levels run one thread per cell (4 per oct in a colour pass and
// in a prolongation that only corrects colour 1, 8 in the residual and in a
// full prolongation); FP32 levels and FP64 levels with
// more than a quarter as many octs per CTA as threads run one thread per
// oct.  A GB300 SM sub-partition issues one FP64 warp instruction about
// every 68 clocks however many of its lanes are active, so where a CTA
// holds a few octs, one thread per oct leaves each FP64 instruction mostly
// idle and serialises the oct's arithmetic in one lane, while one thread per
// cell fills the lanes and shortens each thread's FP64 chain 4 to 8 fold.
// Where the per-oct warps are already full, per-cell threads only add
// instructions (the residual's restriction sum runs in every lane of the
// 8-lane group).  The per-cell bodies are bit-identical to the per-oct ones.
template <typename T, class Map>
__device__ bool per_cell(const Map &map, int64_t n) {
  return sizeof(T) == 8 && map.fits_per_cell(n);
}

// CG: loads through L2 only; otherwise plain loads (see k_tailg).
template <typename T, bool MASK, bool CG, class Map>
__device__ void pass(const TailLevel &L, int P, bool zero, const Map &map) {
  T *phi = static_cast<T *>(L.phi);
  const T *g = static_cast<const T *>(L.g);
  const int64_t st = L.n_alloc * 4;
  if (per_cell<T>(map, L.n)) {
    const Span su = map.units(L.n, 4);
    for (int64_t u = su.a; u < su.e; u += su.s) {
      const int64_t i = u >> 2;
      const int q = (int)(u & 3);
      if (P == 0) {
        if (zero)
          dev::sweep_cell<T, 0, true, MASK, CG>(i, q, L.nbr, phi + st, phi, g, L.active, L.n);
        else
          dev::sweep_cell<T, 0, false, MASK, CG>(i, q, L.nbr, phi + st, phi, g, L.active, L.n);
      } else {
        dev::sweep_cell<T, 1, false, MASK, CG>(i, q, L.nbr, phi, phi + st, g + L.n * 4, L.active, L.n);
      }
    }
    return;
  }
  const Span sp = map.span(L.n);
  for (int64_t i = sp.a; i < sp.e; i += sp.s) {
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

template <typename T, bool CG, class Map>
__device__ void colour_pass(const TailLevel &L, int P, bool zero, const Map &map) {
  if (L.all_active)
    pass<T, false, CG>(L, P, zero, map);
  else
    pass<T, true, CG>(L, P, zero, map);
}

template <typename T, bool CG, class Map, class Sync>
__device__ void sweeps(const TailLevel &L, int n_sweeps, bool zero_first, const Map &map, Sync &sync) {
  for (int k = 0; k < n_sweeps; ++k) {
    colour_pass<T, CG>(L, 0, zero_first && k == 0, map);
    sync();
    colour_pass<T, CG>(L, 1, false, map);
    sync();
  }
}

// Down leg over levels [m_from, m_to): pre-smoothing of m, residual of m
// restricted to the right-hand side of m + 1.
template <typename T, bool CG, class Map, class Sync>
__device__ void descend(const TailPlan &plan, int m_from, int m_to, const Map &map, Sync &sync) {
  for (int m = m_from; m < m_to; ++m) {
    const TailLevel &L = plan.lv[m];
    const TailLevel &C = plan.lv[m + 1];
    sweeps<T, CG>(L, plan.n_pre, true, map, sync);
    const T *phi = static_cast<const T *>(L.phi);
    const T *g = static_cast<const T *>(L.g);
    if (per_cell<T>(map, L.n)) {
      // every thread of the CTA runs the same number of rounds: the 8 lanes
      // of an oct exchange values by shuffles
      const Span su = map.units(L.n, 8);
      for (int64_t u0 = su.base; u0 < su.e; u0 += su.s) {
        const int64_t u = u0 + (su.a - su.base);
        dev::resid_restrict_cell<T, CG>(u < su.e, u >> 3, L.nbr, phi, g, L.all_active ? nullptr : L.active, L.n,
                                        L.n_alloc, L.father, static_cast<T *>(C.g), static_cast<T *>(C.phi), C.n,
                                        C.n_alloc, L.zero_coarse);
      }
    } else {
      // after pre-smoothing (n_pre >= 1) the colour-1 residuals are exactly 0
      const Span sp = map.span(L.n);
      if (plan.n_pre >= 1) {
        for (int64_t i = sp.a; i < sp.e; i += sp.s)
          dev::resid_oct<T, false, true, false, false, false, CG, true>(
              i, L.nbr, phi, g, L.all_active ? nullptr : L.active, L.n, L.n_alloc, L.father, static_cast<T *>(C.g),
              static_cast<T *>(C.phi), C.n, C.n_alloc, L.zero_coarse, nullptr, 0.0, nullptr, 0.0);
      } else {
        for (int64_t i = sp.a; i < sp.e; i += sp.s)
          dev::resid_oct<T, false, true, false, false, false, CG>(
              i, L.nbr, phi, g, L.all_active ? nullptr : L.active, L.n, L.n_alloc, L.father, static_cast<T *>(C.g),
              static_cast<T *>(C.phi), C.n, C.n_alloc, L.zero_coarse, nullptr, 0.0, nullptr, 0.0);
      }
    }
    sync();
  }
}

// The coarsest level: exact 2^3 transform or red-black sweeps (in FP64 in a
// mixed-precision solve).
template <typename T, bool CG, class Map, class Sync>
__device__ void coarsest(const TailPlan &plan, const Map &map, Sync &sync) {
  const TailLevel &L = plan.lv[plan.last];
  if (plan.exact) {
    if (map.first_warp())
      dev::wht_solve_warp<T, T, CG>(static_cast<const T *>(L.g), static_cast<T *>(L.phi), L.n_alloc, plan.h_last);
    sync();
  } else if (!plan.mixed) {
    sweeps<T, CG>(L, plan.coarse_sweeps, plan.last > 0, map, sync);
  } else {
    TailLevel L64 = L;
    L64.phi = L.phi64;
    L64.g = L.g64;
    const float *g32 = static_cast<const float *>(L.g);
    const Span sg = map.span(8 * L.n);
    for (int64_t t = sg.a; t < sg.e; t += sg.s) L.g64[t] = (double)(CG ? __ldcg(g32 + t) : g32[t]);
    sync();
    sweeps<double, CG>(L64, plan.coarse_sweeps, true, map, sync);
    float *p32 = static_cast<float *>(L.phi);
    const Span sq = map.span(8 * L.n_alloc);
    for (int64_t t = sq.a; t < sq.e; t += sq.s) p32[t] = (float)(CG ? __ldcg(L.phi64 + t) : L.phi64[t]);
    sync();
  }
}

// Up leg from level m_from down to m_to: prolongation of m + 1 added to m,
// post-smoothing of m.
template <typename T, bool CG, class Map, class Sync>
__device__ void ascend(const TailPlan &plan, int m_from, int m_to, const Map &map, Sync &sync) {
  for (int m = m_from; m >= m_to; --m) {
    const TailLevel &L = plan.lv[m];
    const TailLevel &C = plan.lv[m + 1];
    T *phi = static_cast<T *>(L.phi);
    const T *cphi = static_cast<const T *>(C.phi);
    // with post-smoothing (n_post >= 1) the colour-0 corrections are
    // overwritten unread by the next pass: only colour-1 cells are corrected
    const bool c0d = plan.n_post >= 1;
    if (per_cell<T>(map, L.n)) {
      const int k = c0d ? 4 : 8;  // cells per oct: colour 1, or all
      const Span su = map.units(L.n, k);
      for (int64_t u = su.a; u < su.e; u += su.s) {
        const int64_t i = c0d ? u >> 2 : u >> 3;
        const int c = c0d ? plane_cell(1, (int)(u & 3)) : (int)(u & 7);
        if (L.all_active)
          dev::prolong_cell<T, false, CG>(i, c, L.keys, L.blk, L.n, L.n_alloc, phi, L.active, cphi, C.n_alloc);
        else
          dev::prolong_cell<T, true, CG>(i, c, L.keys, L.blk, L.n, L.n_alloc, phi, L.active, cphi, C.n_alloc);
      }
    } else {
      const Span sp = map.span(L.n);
      for (int64_t i = sp.a; i < sp.e; i += sp.s) {
        if (L.all_active && c0d)
          dev::prolong_oct<T, false, CG, true>(i, L.keys, L.blk, L.n, L.n_alloc, phi, L.active, cphi, C.n_alloc);
        else if (L.all_active)
          dev::prolong_oct<T, false, CG>(i, L.keys, L.blk, L.n, L.n_alloc, phi, L.active, cphi, C.n_alloc);
        else if (c0d)
          dev::prolong_oct<T, true, CG, true>(i, L.keys, L.blk, L.n, L.n_alloc, phi, L.active, cphi, C.n_alloc);
        else
          dev::prolong_oct<T, true, CG>(i, L.keys, L.blk, L.n, L.n_alloc, phi, L.active, cphi, C.n_alloc);
      }
    }
    sync();
    sweeps<T, CG>(L, plan.n_post, false, map, sync);
  }
}

// The V-cycle from MG level m0 down to the coarsest and back up.
template <typename T, bool CG, class Map, class Sync>
__device__ void tail_body(const TailPlan &plan, int m0, const Map &map, Sync &sync) {
  descend<T, CG>(plan, m0, plan.last, map, sync);
  coarsest<T, CG>(plan, map, sync);
  ascend<T, CG>(plan, plan.last - 1, m0, map, sync);
}

struct BlockSync {
  __device__ void operator()() { __syncthreads(); }
};

// Grid-wide barrier of a cooperative launch (gridsync.cuh); after a wait
// gives up (CMG_ERR_TIMEOUT in the solve's error word) no barrier waits any
// more, so the launch ends with its results void.
struct GridSync {
  unsigned *bar;
  int *err;
  long long budget;
  __device__ void operator()() { dev::grid_barrier(bar, err, budget); }
};

constexpr int kTailThreads1 = 1024;

// Grid tail: levels [m0, split) on all CTAs, [split, last] on CTA 0.
//
// The level fields are read with plain (L1-cacheable) loads (kTailCG =
// false): a CTA reads values another CTA wrote only after a grid barrier,
// whose release add and acquire load at GPU scope, with the block barriers
// around them, order those writes before the reads in the PTX memory model.
// CMG_TAIL_CG = 1 routes them through L2 only.
#ifndef CMG_TAIL_CG
#define CMG_TAIL_CG 0
#endif
constexpr bool kTailCG = CMG_TAIL_CG != 0;

template <typename T>
__global__ void __launch_bounds__(kTailThreads) k_tailg(const __grid_constant__ TailPlan plan) {
  GridSync gs{plan.bar, plan.err, plan.spin_budget};
  const ChunkMap map{(int64_t)blockIdx.x, (int64_t)gridDim.x, (int64_t)threadIdx.x, (int64_t)blockDim.x};
  const int split = plan.split;
  if (split <= plan.last) {
    descend<T, kTailCG>(plan, plan.m0, split, map, gs);
    if (blockIdx.x == 0) {
      // CTA 0 alone from split down: block barriers, loads through L1
      BlockSync bs;
      const FlatMap fm{(int64_t)threadIdx.x, (int64_t)blockDim.x};
      tail_body<T, false>(plan, split, fm, bs);
    }
    gs();
    ascend<T, kTailCG>(plan, split - 1, plan.m0, map, gs);
  } else {
    tail_body<T, kTailCG>(plan, plan.m0, map, gs);
  }
}

// The whole tail in one CTA: block barriers, loads through L1.  For levels
// so small that a launch costs more than their arithmetic on one SM.
template <typename T>
__global__ void __launch_bounds__(kTailThreads1) k_tail1(const __grid_constant__ TailPlan plan) {
  BlockSync sync;
  const FlatMap fm{(int64_t)threadIdx.x, (int64_t)blockDim.x};
  tail_body<T, false>(plan, plan.m0, fm, sync);
}

template <typename T>
int tailg_grid(const cmg_ctx *ctx) {
  static int per_sm = -1;
  if (per_sm < 0) {
    int b = 0;
    CMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_tailg<T>, kTailThreads, 0));
    per_sm = b;
  }
  if (per_sm < 1) throw Error(CMG_ERR_CUDA, "the grid tail kernel does not fit on an SM");
  return ctx->num_sms;  // one CTA per SM: co-resident, as the cooperative launch requires
}

}  // namespace

// Largest level one CTA runs: one SM does ~2 FP64 FMAs per clock but ~128
// FP32 ones, so a single SM pays for far larger FP32 levels than FP64 ones.
// The coarsest level of a mixed-precision solve is swept in FP64.
template <typename T>
int64_t one_cta_octs() {
  return sizeof(T) == 8 ? 64 : 512;
}

// Whether levels m .. last fit one CTA.
template <typename T>
bool one_cta(const cmg_level *L, int m) {
  const int last = (int)L->mg.size() - 1;
  if (L->mg[m].n > one_cta_octs<T>()) return false;
  if (sizeof(T) == 4 && !L->exact_coarse && L->mg[last].n > one_cta_octs<double>()) return false;
  return true;
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
  if (one_cta<T>(L, m0)) {
    k_tail1<T><<<1, kTailThreads1, 0, L->ctx->stream>>>(plan);
    CMG_CUDA(cudaGetLastError());
    return;
  }
  // grid tail; CTA 0 alone takes the levels from the first that fits it
  plan.split = last + 1;
  for (int m = m0 + 1; m <= last; ++m)
    if (one_cta<T>(L, m)) {
      plan.split = m;
      break;
    }
  plan.err = solve_err_word(L);
  plan.bar = solve_bar_words(L);
  plan.spin_budget = L->tail_spin_budget;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tailg_grid<T>(L->ctx));
  cfg.blockDim = dim3(kTailThreads);
  cfg.stream = L->ctx->stream;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeCooperative;
  attr.val.cooperative = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  CMG_CUDA(cudaLaunchKernelEx(&cfg, k_tailg<T>, plan));
}

template void tail_vcycle<double>(cmg_level *, int, const cmg_solve_params *, const bool *);
template void tail_vcycle<float>(cmg_level *, int, const cmg_solve_params *, const bool *);

}  // namespace cmg
