// batch.cu -- batched solve of many independent refined patches in one
// persistent cooperative kernel launch (recorded in a CUDA graph), with an
// autotuner for its block shape and sweep schedule.
//
// The patches are the octs of one level (patch k = a contiguous range of the
// level's keys), so the level's hash table, neighbour cache, ghost octs and
// multigrid hierarchy serve all of them; isolation between patches is
// checked at build time on every MG level.  The persistent kernel walks the
// whole V-cycle schedule with grid-stride loops over octs and a grid barrier
// between dependent operations; per-patch residual norms are accumulated
// with warp-aggregated atomics, and the stopping test runs on the device.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "cmg_internal.cuh"
#include "gridsync.cuh"
#include "oct_ops.cuh"

namespace cmg {

namespace {

constexpr int kBMaxLevels = 48;

struct BLevel {
  int64_t n, n_alloc;
  const int32_t *nbr;
  const uint8_t *active;
  const int32_t *father;
  const int32_t *blk;
  const uint64_t *keys;
  double *phi, *g;
  float *phi32, *g32;
  int all_active;
};

struct BatchPlan {
  int depth, n_pre, n_post, inner, max_cycles, fixed_cycles, n_patches;
  double tol;
  long long spin_budget;
  BLevel lv[kBMaxLevels];
  const int32_t *pid;  // patch of each top-level oct
  // Dirichlet ghosts of the top level
  int64_t n_ghost;
  const uint64_t *gkeys;
  const int32_t *gblk;
  const uint32_t *gmask;
  const double *pphi;
  int64_t pn_alloc;
  // per-patch state (d-units: d = fma(s, 1/6, g) - phi)
  double *n0, *norm, *s_emit, *s_acc, *rel;
  int32_t *conv_at;
  // control: [0] status, [1] cycles, [2..3] unconverged counters, [4] barriers, [5] n_converged
  int *ctrl;
  unsigned *bar;  // grid barrier word
  // conjugate gradients (krylov = 1): top-level vectors in the phi layout
  // ([2][n_alloc][4]; gsave in the g layout) and per-patch scalars
  double *cx, *cp0, *cp1, *cq, *gsave;
  double *zr, *zq, *zr_old, *beta, *pq, *alpha;
  int32_t *done;
};

// Grid-wide barrier (gridsync.cuh): waits give up after spin_budget SM clock
// cycles with CMG_ERR_TIMEOUT in the status word, and every block then leaves
// at its next barrier, so a failed launch always ends.  CTA 0 counts the
// barriers passed.
__device__ bool grid_sync(const BatchPlan &P) {
  if (!dev::grid_barrier(P.bar, P.ctrl, P.spin_budget)) return false;
  if (blockIdx.x == 0 && threadIdx.x == 0) P.ctrl[4] += 1;
  return true;
}

// Sum v over the lanes of the warp that share patch p (p < 0: no value).
__device__ __forceinline__ void patch_add(double *arr, int p, double v) {
  const int lane = threadIdx.x & 31;
  const int p0 = __shfl_sync(0xffffffffu, p, 0);
  if (__all_sync(0xffffffffu, p == p0 || p < 0)) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0 && p0 >= 0) atomicAdd(arr + p0, v);
  } else if (p >= 0) {
    atomicAdd(arr + p, v);
  }
}

template <typename T>
__device__ __forceinline__ T *phi_t(const BLevel &L) {
  if constexpr (sizeof(T) == 8) return L.phi; else return L.phi32;
}
template <typename T>
__device__ __forceinline__ T *g_t(const BLevel &L) {
  if constexpr (sizeof(T) == 8) return L.g; else return L.g32;
}

// The per-oct bodies read the level fields through L1 (kCG = false) or
// through L2 only (true).  Plain loads are enough: a block reads values
// another block wrote only after a grid barrier, whose release add and
// acquire load at GPU scope (with the block barriers around them) order those
// writes before the reads in the PTX memory model; per-patch scalars and the
// control words keep their L2 loads.  CMG_BATCH_CG = 1 restores L2-only
// loads for the fields.
#ifndef CMG_BATCH_CG
#define CMG_BATCH_CG 0
#endif
constexpr bool kCG = CMG_BATCH_CG != 0;

template <typename T>
__device__ void colour_pass(const BLevel &L, int P, bool zero, int64_t tid, int64_t nthr, T *phi, const T *g) {
  const int64_t st = L.n_alloc * 4;
  for (int64_t i = tid; i < L.n; i += nthr) {
    if (P == 0) {
      if (zero) {
        if (L.all_active) dev::sweep_oct<T, 0, true, false, kCG>(i, L.nbr, phi + st, phi, g, L.active, L.n);
        else dev::sweep_oct<T, 0, true, true, kCG>(i, L.nbr, phi + st, phi, g, L.active, L.n);
      } else {
        if (L.all_active) dev::sweep_oct<T, 0, false, false, kCG>(i, L.nbr, phi + st, phi, g, L.active, L.n);
        else dev::sweep_oct<T, 0, false, true, kCG>(i, L.nbr, phi + st, phi, g, L.active, L.n);
      }
    } else {
      if (L.all_active) dev::sweep_oct<T, 1, false, false, kCG>(i, L.nbr, phi, phi + st, g + L.n * 4, L.active, L.n);
      else dev::sweep_oct<T, 1, false, true, kCG>(i, L.nbr, phi, phi + st, g + L.n * 4, L.active, L.n);
    }
  }
}

template <typename T>
__device__ bool sweeps(const BatchPlan &Pl, const BLevel &L, int n_sweeps, bool zero_first, int64_t tid,
                       int64_t nthr, T *phi, const T *g) {
  for (int k = 0; k < n_sweeps; ++k) {
    colour_pass<T>(L, 0, zero_first && k == 0, tid, nthr, phi, g);
    if (!grid_sync(Pl)) return false;
    colour_pass<T>(L, 1, false, tid, nthr, phi, g);
    if (!grid_sync(Pl)) return false;
  }
  return true;
}

// One V-cycle over every MG level of the batch; T = double works on phi/g
// (solution at the top, with ghosts), T = float on the FP32 correction.
template <typename T>
__device__ bool vcycle(const BatchPlan &P, bool zero_top, int64_t tid, int64_t nthr) {
  const int last = P.depth - 1;
  const int nsw = P.n_pre + P.n_post;  // coarsest solve = n_pre + n_post sweeps
  for (int m = 0; m < last; ++m) {
    const BLevel &L = P.lv[m];
    const BLevel &C = P.lv[m + 1];
    if (!sweeps<T>(P, L, P.n_pre, m > 0 || zero_top, tid, nthr, phi_t<T>(L), g_t<T>(L))) return false;
    const int zc = (m + 1 < last) ? (P.n_pre == 0) : (nsw == 0);
    // after pre-smoothing (n_pre >= 1) the colour-1 residuals are exactly 0
    if (P.n_pre >= 1) {
      for (int64_t i = tid; i < L.n; i += nthr)
        dev::resid_oct<T, false, true, false, false, false, kCG, true>(
            i, L.nbr, phi_t<T>(L), g_t<T>(L), L.all_active ? nullptr : L.active, L.n, L.n_alloc, L.father,
            g_t<T>(C), phi_t<T>(C), C.n, C.n_alloc, zc, nullptr, 0.0, nullptr, 0.0);
    } else {
      for (int64_t i = tid; i < L.n; i += nthr)
        dev::resid_oct<T, false, true, false, false, false, kCG>(
            i, L.nbr, phi_t<T>(L), g_t<T>(L), L.all_active ? nullptr : L.active, L.n, L.n_alloc, L.father,
            g_t<T>(C), phi_t<T>(C), C.n, C.n_alloc, zc, nullptr, 0.0, nullptr, 0.0);
    }
    if (!grid_sync(P)) return false;
  }
  {
    const BLevel &L = P.lv[last];
    if (sizeof(T) == 4) {
      // the coarsest level is solved in FP64 on FP64 copies
      for (int64_t t = tid; t < 8 * L.n; t += nthr) L.g[t] = (double)__ldcg(L.g32 + t);
      if (!grid_sync(P)) return false;
      if (!sweeps<double>(P, L, nsw, last > 0, tid, nthr, L.phi, L.g)) return false;
      for (int64_t t = tid; t < 8 * L.n_alloc; t += nthr) L.phi32[t] = (float)__ldcg(L.phi + t);
      if (!grid_sync(P)) return false;
    } else {
      if (!sweeps<T>(P, L, nsw, last > 0, tid, nthr, phi_t<T>(L), g_t<T>(L))) return false;
    }
  }
  for (int m = last - 1; m >= 0; --m) {
    const BLevel &L = P.lv[m];
    const BLevel &C = P.lv[m + 1];
    // with post-smoothing, the colour-0 corrections are overwritten unread
    for (int64_t i = tid; i < L.n; i += nthr) {
      if (L.all_active && P.n_post >= 1)
        dev::prolong_oct<T, false, kCG, true>(i, L.keys, L.blk, L.n, L.n_alloc, phi_t<T>(L), L.active, phi_t<T>(C),
                                               C.n_alloc);
      else if (L.all_active)
        dev::prolong_oct<T, false, kCG>(i, L.keys, L.blk, L.n, L.n_alloc, phi_t<T>(L), L.active, phi_t<T>(C),
                                         C.n_alloc);
      else if (P.n_post >= 1)
        dev::prolong_oct<T, true, kCG, true>(i, L.keys, L.blk, L.n, L.n_alloc, phi_t<T>(L), L.active, phi_t<T>(C),
                                              C.n_alloc);
      else
        dev::prolong_oct<T, true, kCG>(i, L.keys, L.blk, L.n, L.n_alloc, phi_t<T>(L), L.active, phi_t<T>(C),
                                        C.n_alloc);
    }
    if (!grid_sync(P)) return false;
    if (!sweeps<T>(P, L, P.n_post, false, tid, nthr, phi_t<T>(L), g_t<T>(L))) return false;
  }
  return true;
}

// Top-level FP64 residual, per-patch norms into P.norm; MIXED also writes the
// FP32 right-hand side g32 = d / s_emit[patch].  C1Z: right after an FP64
// V-cycle whose last operation on the top level is a colour-1 pass (the
// colour-1 residuals are exactly zero and are not evaluated).
template <bool MIXED, bool ZPHI, bool C1Z = false>
__device__ void top_residual(const BatchPlan &P, double *acc_out, int64_t tid, int64_t nthr) {
  const BLevel &L = P.lv[0];
  const int64_t wbase = tid & ~(int64_t)31;
  for (int64_t base = wbase; base < L.n; base += nthr) {
    const int64_t i = base + (threadIdx.x & 31);
    double acc = 0.0;
    int p = -1;
    if (i < L.n) {
      p = __ldg(P.pid + i);
      const double inv_s = MIXED ? 1.0 / __ldcg(P.s_emit + p) : 0.0;
      acc = dev::resid_oct<double, true, false, MIXED, false, ZPHI, kCG, C1Z>(
          i, L.nbr, L.phi, L.g, nullptr, L.n, L.n_alloc, nullptr, nullptr, nullptr, 0, 0, 0, L.g32, inv_s, nullptr,
          0.0);
    }
    patch_add(acc_out, p, acc);
  }
}

// Dirichlet ghosts of the top level from the parent's phi.
__device__ void fill_top_ghosts(const BatchPlan &P, int64_t tid, int64_t nthr) {
  const BLevel &T0 = P.lv[0];
  for (int64_t t = tid; t < P.n_ghost; t += nthr) {
    const int cc = (int)(__ldg(P.gkeys + t) & 7);
    int32_t b[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) b[k] = __ldg(P.gblk + k * P.n_ghost + t);
    double val[8];
    dev::interp8<double, false>(P.pphi, P.pn_alloc, b, cc, val);
    const uint32_t m = __ldg(P.gmask + t);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      double v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = plane_cell(p, q);
        v[q] = ((m >> c) & 1) ? val[c] : 0.0;
      }
      dev::store4(T0.phi + (p * T0.n_alloc + T0.n + t) * 4, v);
    }
  }
}

// ---- flexible (Polak-Ribiere) conjugate gradients per patch (krylov = 1),
// the multigrid V-cycle from zero as the preconditioner (the paper names
// multigrid as a CG preconditioner, App. D.2): the level solve's PCG
// (pcg.cu) with a separate alpha and beta for every patch.  A patch that has
// reached tol keeps alpha = beta = 0 (frozen) while the others iterate.

__device__ __forceinline__ int64_t at_phi(int64_t o, int c, int64_t ps) {
  return (int64_t)cell_parity(c) * ps + o * 4 + (c >> 1);
}

// z at phi-layout index k of a cell of patch p: the FP64 V-cycle leaves z in
// phi; the FP32 one leaves e = z / s_acc in phi32
template <bool MIXED>
__device__ __forceinline__ double zval(const BatchPlan &P, int64_t k, double s) {
  if constexpr (MIXED) return s * (double)__ldcg(P.lv[0].phi32 + k);
  else return __ldcg(P.lv[0].phi + k);
}

template <bool MIXED>
__device__ bool krylov_solve(const BatchPlan &P, int64_t tid, int64_t nthr) {
  const BLevel &T = P.lv[0];
  const int64_t n = T.n, ps = T.n_alloc * 4, gs = n * 4;
  const int64_t wbase = tid & ~(int64_t)31;
  // r0 = f - L phi0 (Dirichlet ghosts) in place of g (saved), x = phi0, ||r0||^2
  for (int64_t base = wbase; base < n; base += nthr) {
    const int64_t i = base + (threadIdx.x & 31);
    double acc = 0.0;
    int pp = -1;
    if (i < n) {
      pp = __ldg(P.pid + i);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        double sum = 0.0;
#pragma unroll
        for (int d = 0; d < 6; ++d) {
          const int a = d >> 1, side = d & 1, c2 = c ^ (1 << a);
          const int64_t o = (((c >> a) & 1) != side) ? i : (int64_t)__ldg(T.nbr + d * n + i);
          sum += __ldcg(T.phi + at_phi(o, c2, ps));
        }
        const int64_t gi = at_phi(i, c, gs), k = at_phi(i, c, ps);
        const double gv = __ldcg(T.g + gi), ph = __ldcg(T.phi + k);
        const double v = fma(sum, 1.0 / 6.0, gv) - ph;
        P.gsave[gi] = gv;
        T.g[gi] = v;
        P.cx[k] = ph;
        acc += v * v;
      }
    }
    patch_add(P.norm, pp, acc);
  }
  for (int64_t p = tid; p < P.n_patches; p += nthr) {
    P.zr[p] = P.zq[p] = P.zr_old[p] = P.beta[p] = P.pq[p] = P.alpha[p] = 0.0;
    P.done[p] = 0;
  }
  if (!grid_sync(P)) return false;
  // corrections see zero coarse-fine values: clear phi's ghost octs
  for (int64_t t = tid; t < 8 * (T.n_alloc - n); t += nthr) {
    const int pl = (int)(t / (4 * (T.n_alloc - n)));
    const int64_t r = t - pl * 4 * (T.n_alloc - n);
    T.phi[pl * ps + 4 * n + r] = 0.0;
  }
  for (int64_t p = tid; p < P.n_patches; p += nthr) {
    const double nr = __ldcg(P.norm + p);
    P.s_emit[p] = nr > 0.0 ? sqrt(nr) : 1.0;
  }
  if (!grid_sync(P)) return false;
  if (MIXED) {  // the first FP32 right-hand side r0 / s
    for (int64_t t = tid; t < 8 * n; t += nthr) {
      const int64_t i = (t >> 2) % n;
      T.g32[t] = (float)(T.g[t] / __ldcg(P.s_emit + __ldg(P.pid + i)));
    }
    if (!grid_sync(P)) return false;
  }
  int cur = 0;  // direction buffer written this iteration
  for (int cycle = 0;; ++cycle) {
    // stop test on ||r||; alpha of the last step kept for the next beta
    for (int64_t p = tid; p < P.n_patches; p += nthr) {
      const double n0 = __ldcg(P.n0 + p), nr = __ldcg(P.norm + p);
      const double rel = n0 > 0.0 ? sqrt(nr / n0) : 0.0;
      P.rel[p] = rel;
      if (!(rel == rel) || isinf(rel)) atomicCAS(P.ctrl, 0, CMG_ERR_DIVERGED);
      const int was_done = __ldcg(P.done + p);
      if (cycle > 0) {
        const double pq = __ldcg(P.pq + p), zo = __ldcg(P.zr_old + p);
        P.alpha[p] = (was_done || pq == 0.0) ? 0.0 : zo / pq;
      }
      if (rel <= P.tol) {
        if (__ldcg(P.conv_at + p) < 0) P.conv_at[p] = cycle;
        P.done[p] = 1;
      } else {
        atomicAdd(P.ctrl + 2 + (cycle & 1), 1);
      }
      if (MIXED) {
        P.s_acc[p] = __ldcg(P.s_emit + p);
        P.s_emit[p] = nr > 0.0 ? sqrt(nr) : 1.0;
      }
      P.norm[p] = 0.0;
    }
    if (!grid_sync(P)) return false;
    const int unconverged = __ldcg(P.ctrl + 2 + (cycle & 1));
    const int status = __ldcg(P.ctrl);
    bool stop = status != 0;
    if (P.fixed_cycles > 0) stop = stop || cycle >= P.fixed_cycles;
    else stop = stop || unconverged == 0 || cycle >= P.max_cycles;
    if (stop) {
      if (tid == 0) {
        P.ctrl[1] = cycle;
        P.ctrl[5] = P.n_patches - unconverged;
        if (status == 0 && P.fixed_cycles == 0 && unconverged > 0) P.ctrl[0] = CMG_ERR_NOT_CONVERGED;
      }
      break;
    }
    if (tid == 0) P.ctrl[2 + ((cycle + 1) & 1)] = 0;
    // z = M r: one V-cycle from zero (FP64 on g = r, or FP32 on g32 = r / s)
    if (MIXED) {
      for (int k = 0; k < P.inner; ++k)
        if (!vcycle<float>(P, k == 0, tid, nthr)) return false;
    } else {
      if (!vcycle<double>(P, true, tid, nthr)) return false;
    }
    // (z, r) and (z, q) per patch; q is the last iteration's L0 p
    for (int64_t base = wbase; base < n; base += nthr) {
      const int64_t i = base + (threadIdx.x & 31);
      double a = 0.0, b = 0.0;
      int pp = -1;
      if (i < n) {
        pp = __ldg(P.pid + i);
        const double sz = MIXED ? __ldcg(P.s_acc + pp) : 1.0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int64_t k = at_phi(i, c, ps);
          const double z = zval<MIXED>(P, k, sz);
          a += z * __ldcg(T.g + at_phi(i, c, gs));
          b += z * __ldcg(P.cq + k);
        }
      }
      patch_add(P.zr, pp, a);
      patch_add(P.zq, pp, b);
    }
    if (!grid_sync(P)) return false;
    // beta = -alpha (z', q) / (z, r)_old (0 on the first iteration and once frozen)
    for (int64_t p = tid; p < P.n_patches; p += nthr) {
      const double zo = __ldcg(P.zr_old + p);
      const bool fresh = cycle == 0 || __ldcg(P.done + p) || zo == 0.0;
      P.beta[p] = fresh ? 0.0 : -__ldcg(P.alpha + p) * __ldcg(P.zq + p) / zo;
      P.zr_old[p] = __ldcg(P.zr + p);
      P.zr[p] = 0.0;
      P.zq[p] = 0.0;
      P.pq[p] = 0.0;
    }
    if (!grid_sync(P)) return false;
    // p = z + beta p_old into the other direction buffer (ghost and zero octs
    // stay zero), then q = L0 p and (p, q) per patch (neighbours share the
    // patch).  Two passes: forming the neighbours' p on the fly would cost six
    // more FP64 FMAs per cell than the extra pass costs bandwidth.
    double *pn = cur ? P.cp1 : P.cp0;
    const double *po = cur ? P.cp0 : P.cp1;
    for (int64_t i = tid; i < n; i += nthr) {
      const int pp = __ldg(P.pid + i);
      const double bt = __ldcg(P.beta + pp), sz = MIXED ? __ldcg(P.s_acc + pp) : 1.0;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int64_t k = at_phi(i, c, ps);
        pn[k] = fma(bt, __ldcg(po + k), zval<MIXED>(P, k, sz));
      }
    }
    if (!grid_sync(P)) return false;
    for (int64_t base = wbase; base < n; base += nthr) {
      const int64_t i = base + (threadIdx.x & 31);
      double acc = 0.0;
      int pp = -1;
      if (i < n) {
        pp = __ldg(P.pid + i);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int64_t k = at_phi(i, c, ps);
          const double pv = __ldcg(pn + k);
          double sum = 0.0;
#pragma unroll
          for (int d = 0; d < 6; ++d) {
            const int a = d >> 1, side = d & 1, c2 = c ^ (1 << a);
            const int64_t o = (((c >> a) & 1) != side) ? i : (int64_t)__ldg(T.nbr + d * n + i);
            sum += __ldcg(pn + at_phi(o, c2, ps));
          }
          const double qv = pv - sum * (1.0 / 6.0);
          P.cq[k] = qv;
          acc += pv * qv;
        }
      }
      patch_add(P.pq, pp, acc);
    }
    if (!grid_sync(P)) return false;
    // alpha = (z, r) / (p, q); x += alpha p; r -= alpha q; ||r||^2 per patch;
    // MIXED: the next FP32 right-hand side r / s
    for (int64_t base = wbase; base < n; base += nthr) {
      const int64_t i = base + (threadIdx.x & 31);
      double acc = 0.0;
      int pp = -1;
      if (i < n) {
        pp = __ldg(P.pid + i);
        const double pq = __ldcg(P.pq + pp);
        const double al = (__ldcg(P.done + pp) || pq == 0.0) ? 0.0 : __ldcg(P.zr_old + pp) / pq;
        const double inv_s = MIXED ? 1.0 / __ldcg(P.s_emit + pp) : 0.0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int64_t k = at_phi(i, c, ps), gi = at_phi(i, c, gs);
          P.cx[k] += al * __ldcg(pn + k);
          const double rv = __ldcg(T.g + gi) - al * __ldcg(P.cq + k);
          T.g[gi] = rv;
          if (MIXED) T.g32[gi] = (float)(rv * inv_s);
          acc += rv * rv;
        }
      }
      patch_add(P.norm, pp, acc);
    }
    if (!grid_sync(P)) return false;
    cur ^= 1;
  }
  // wrap-up: phi = x, the source restored, the coarse-fine ghosts refilled
  for (int64_t t = tid; t < 8 * n; t += nthr) {
    const int pl = (int)(t / (4 * n));
    const int64_t r = t - pl * 4 * n;
    T.phi[pl * ps + r] = __ldcg(P.cx + pl * ps + r);
    T.g[t] = __ldcg(P.gsave + t);
  }
  fill_top_ghosts(P, tid, nthr);
  return grid_sync(P);
}

// The stationary iteration: V-cycles (FP64, or FP32 inside FP64 refinement)
// until every patch reaches tol.
template <bool MIXED>
__device__ void stationary_solve(const BatchPlan &P, int64_t tid, int64_t nthr) {
  const BLevel &T0 = P.lv[0];
  for (int64_t p = tid; p < P.n_patches; p += nthr) {
    const double n0 = __ldcg(P.n0 + p);
    P.s_emit[p] = n0 > 0.0 ? sqrt(n0) : 1.0;
  }
  if (!grid_sync(P)) return;
  top_residual<MIXED, false>(P, P.norm, tid, nthr);
  if (!grid_sync(P)) return;
  for (int cycle = 0;; ++cycle) {
    // per-patch test; unconverged patches counted in ctrl[2 + parity]
    for (int64_t p = tid; p < P.n_patches; p += nthr) {
      const double n0 = __ldcg(P.n0 + p), nr = __ldcg(P.norm + p);
      const double rel = n0 > 0.0 ? sqrt(nr / n0) : 0.0;
      P.rel[p] = rel;
      if (!(rel == rel) || isinf(rel)) atomicCAS(P.ctrl, 0, CMG_ERR_DIVERGED);
      if (rel <= P.tol) {
        if (__ldcg(P.conv_at + p) < 0) P.conv_at[p] = cycle;
      } else {
        atomicAdd(P.ctrl + 2 + (cycle & 1), 1);
      }
      if (MIXED) {
        P.s_acc[p] = __ldcg(P.s_emit + p);
        P.s_emit[p] = nr > 0.0 ? sqrt(nr) : 1.0;
      }
      P.norm[p] = 0.0;
    }
    if (!grid_sync(P)) return;
    const int unconverged = __ldcg(P.ctrl + 2 + (cycle & 1));
    const int status = __ldcg(P.ctrl);
    bool stop = status != 0;
    if (P.fixed_cycles > 0) stop = stop || cycle >= P.fixed_cycles;
    else stop = stop || unconverged == 0 || cycle >= P.max_cycles;
    if (stop) {
      if (tid == 0) {
        P.ctrl[1] = cycle;
        P.ctrl[5] = P.n_patches - unconverged;
        if (status == 0 && P.fixed_cycles == 0 && unconverged > 0) P.ctrl[0] = CMG_ERR_NOT_CONVERGED;
      }
      return;
    }
    if (tid == 0) P.ctrl[2 + ((cycle + 1) & 1)] = 0;
    if (MIXED) {
      for (int k = 0; k < P.inner; ++k)
        if (!vcycle<float>(P, k == 0, tid, nthr)) return;
      for (int64_t t = tid; t < 2 * T0.n; t += nthr) {  // phi64 += s_acc * e
        const int pl = (int)(t / T0.n);
        const int64_t i = t - pl * T0.n;
        const double S = __ldcg(P.s_acc + __ldg(P.pid + i));
        double v[4];
        float w[4];
        dev::load4<true>(T0.phi + (pl * T0.n_alloc + i) * 4, v);
        dev::load4<true>(T0.phi32 + (pl * T0.n_alloc + i) * 4, w);
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = fma(S, (double)w[q], v[q]);
        dev::store4(T0.phi + (pl * T0.n_alloc + i) * 4, v);
      }
      if (!grid_sync(P)) return;
      top_residual<MIXED, false>(P, P.norm, tid, nthr);
    } else {
      if (!vcycle<double>(P, false, tid, nthr)) return;
      const bool c1 = P.depth > 1 ? P.n_post >= 1 : P.n_pre + P.n_post >= 1;
      if (c1)
        top_residual<false, false, true>(P, P.norm, tid, nthr);
      else
        top_residual<false, false>(P, P.norm, tid, nthr);
    }
    if (!grid_sync(P)) return;
  }
}

template <bool MIXED, bool KRYLOV>
__global__ void __launch_bounds__(512, 1) k_batch(const __grid_constant__ BatchPlan P) {
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // Dirichlet ghosts from the parent's phi; per-patch accumulators cleared
  fill_top_ghosts(P, tid, nthr);
  for (int64_t p = tid; p < P.n_patches; p += nthr) {
    P.n0[p] = 0.0;
    P.norm[p] = 0.0;
    P.conv_at[p] = -1;
  }
  if (!grid_sync(P)) return;
  top_residual<false, true>(P, P.n0, tid, nthr);  // ||f - L 0||^2 per patch
  if (!grid_sync(P)) return;
  if constexpr (KRYLOV)
    krylov_solve<MIXED>(P, tid, nthr);
  else
    stationary_solve<MIXED>(P, tid, nthr);
}

__global__ void k_patch_ids(const int64_t *__restrict__ offsets, int n_patches, int32_t *__restrict__ pid, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = n_patches - 1;  // patch k: offsets[k] <= i < offsets[k+1]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (offsets[mid] <= i) lo = mid; else hi = mid - 1;
  }
  pid[i] = lo;
}

// Coarse patch ids from the fully active children (pushed through father).
__global__ void k_patch_up(const int32_t *__restrict__ pid, const int32_t *__restrict__ father, int64_t n,
                           int32_t *__restrict__ cpid) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t f = father[i];
  if (f >= 0) cpid[f >> 3] = pid[i];
}

// Isolation check: every fully active child agrees with its coarse oct and
// every real same-level neighbour belongs to the same patch.
__global__ void k_patch_check(const int32_t *__restrict__ pid, const int32_t *__restrict__ nbr,
                              const int32_t *__restrict__ father, const int32_t *__restrict__ cpid, int64_t n,
                              int *err) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t p = pid[i];
  for (int d = 0; d < 6; ++d) {
    const int32_t o = nbr[d * n + i];
    if (o < n && pid[o] != p) set_error(err, CMG_ERR_INVALID_ARG);
  }
  if (father && cpid) {
    const int32_t f = father[i];
    if (f >= 0 && cpid[f >> 3] != p) set_error(err, CMG_ERR_INVALID_ARG);
  }
}

}  // namespace

}  // namespace cmg

namespace cmg {
namespace {

void drop_graph(cmg_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

bool same_sched(const cmg_batch_schedule &a, const cmg_batch_schedule &b) {
  return a.threads == b.threads && a.blocks_per_sm == b.blocks_per_sm && a.n_pre == b.n_pre &&
         a.n_post == b.n_post && a.inner_cycles == b.inner_cycles;
}

bool same_params(const cmg_solve_params &a, const cmg_solve_params &b) {
  return a.tol == b.tol && a.max_cycles == b.max_cycles && a.fixed_cycles == b.fixed_cycles &&
         a.precision == b.precision && a.krylov == b.krylov;
}

const void *batch_kernel(bool mixed, bool krylov) {
  if (mixed) return krylov ? (const void *)k_batch<true, true> : (const void *)k_batch<true, false>;
  return krylov ? (const void *)k_batch<false, true> : (const void *)k_batch<false, false>;
}

// Blocks of this many threads can launch the kernel (its launch bounds).
bool block_fits(const void *fn, int threads) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return threads <= fa.maxThreadsPerBlock;
}

int grid_size(cmg_batch *b, bool mixed, bool krylov) {
  const void *fn = batch_kernel(mixed, krylov);
  if (!block_fits(fn, b->sched.threads))
    throw Error(CMG_ERR_INVALID_ARG, "the batch kernel does not take blocks of this size");
  int per_sm = 0;
  CMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, b->sched.threads, 0));
  if (per_sm < 1) throw Error(CMG_ERR_INVALID_ARG, "the batch kernel does not fit this block size");
  return b->lvl->ctx->num_sms * std::min(per_sm, b->sched.blocks_per_sm);
}

BatchPlan make_plan(cmg_batch *b, const cmg_solve_params *p) {
  cmg_level *L = b->lvl;
  BatchPlan P = {};
  P.depth = (int)L->mg.size();
  P.n_pre = b->sched.n_pre;
  P.n_post = b->sched.n_post;
  P.inner = b->sched.inner_cycles;
  P.max_cycles = p->max_cycles;
  P.fixed_cycles = p->fixed_cycles;
  P.n_patches = b->n_patches;
  P.tol = p->tol;
  P.spin_budget = b->spin_budget;
  for (int m = 0; m < P.depth; ++m) {
    MgLev &g = L->mg[m];
    BLevel &t = P.lv[m];
    t.n = g.n;
    t.n_alloc = g.n_alloc;
    t.nbr = g.nbr;
    t.active = g.active;
    t.father = g.father;
    t.blk = g.blk;
    t.keys = g.keys;
    t.phi = g.phi;
    t.g = g.g;
    t.phi32 = g.phi32;
    t.g32 = g.g32;
    t.all_active = g.all_active ? 1 : 0;
  }
  P.pid = b->pid[0];
  P.n_ghost = L->mg[0].n_ghost;
  P.gkeys = L->ghost_keys;
  P.gblk = L->ghost_blk;
  P.gmask = L->ghost_mask;
  P.pphi = L->parent ? L->parent->mg[0].phi : nullptr;
  P.pn_alloc = L->parent ? L->parent->mg[0].n_alloc : 0;
  const int n = b->n_patches;
  P.n0 = b->pstate;
  P.norm = b->pstate + n;
  P.s_emit = b->pstate + 2 * n;
  P.s_acc = b->pstate + 3 * n;
  P.rel = b->pstate + 4 * n;
  P.conv_at = b->conv_at;
  P.ctrl = b->ctrl;
  P.bar = b->bar;
  if (b->cg) {
    const int64_t nv = 8 * L->mg[0].n_alloc;
    P.cx = b->cg;
    P.cp0 = P.cx + nv;
    P.cp1 = P.cp0 + nv;
    P.cq = P.cp1 + nv;
    P.gsave = P.cq + nv;
    P.zr = P.gsave + 8 * L->mg[0].n;
    P.zq = P.zr + n;
    P.zr_old = P.zq + n;
    P.beta = P.zr_old + n;
    P.pq = P.beta + n;
    P.alpha = P.pq + n;
    P.done = b->cg_done;
  }
  return P;
}

// CG vectors and per-patch scalars (krylov = 1), allocated on first use
void ensure_cg(cmg_batch *b) {
  if (b->cg) return;
  cmg_level *L = b->lvl;
  const int64_t nv = 8 * L->mg[0].n_alloc;
  // b->cg (the "allocated" mark) is set last
  double *cg = b->mem.alloc<double>(4 * nv + 8 * L->mg[0].n + 6 * (int64_t)b->n_patches, true, L->ctx->stream);
  b->cg_done = b->mem.alloc<int32_t>(b->n_patches, true, L->ctx->stream);
  CMG_CUDA(cudaStreamSynchronize(L->ctx->stream));
  b->cg = cg;
}

// Records: clear control words (and the CG direction buffers), the
// cooperative persistent kernel, copy of the control words to pinned host
// memory.
void record(cmg_batch *b, const cmg_solve_params *p) {
  cmg_level *L = b->lvl;
  cmg_ctx *ctx = L->ctx;
  const bool mixed = p->precision == CMG_PREC_MIXED, krylov = p->krylov == 1;
  BatchPlan P = make_plan(b, p);
  const int grid = grid_size(b, mixed, krylov);
  if (!ctx->cap_stream) {
    CMG_CUDA(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    CMG_CUDA(cudaStreamCreateWithFlags(&ctx->cap_stream2, cudaStreamNonBlocking));
  }
  drop_graph(b);
  cudaStream_t s = ctx->cap_stream;
  CMG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
  try {
    CMG_CUDA(cudaMemsetAsync(b->ctrl, 0, 8 * sizeof(int), s));
    CMG_CUDA(cudaMemsetAsync(b->bar, 0, 2 * sizeof(unsigned), s));
    if (krylov)  // both direction buffers and q start at zero (finite) every solve
      CMG_CUDA(cudaMemsetAsync(P.cp0, 0, sizeof(double) * 3 * 8 * L->mg[0].n_alloc, s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(b->sched.threads);
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeCooperative;
    attr.val.cooperative = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    if (mixed && krylov)
      CMG_CUDA(cudaLaunchKernelEx(&cfg, k_batch<true, true>, P));
    else if (mixed)
      CMG_CUDA(cudaLaunchKernelEx(&cfg, k_batch<true, false>, P));
    else if (krylov)
      CMG_CUDA(cudaLaunchKernelEx(&cfg, k_batch<false, true>, P));
    else
      CMG_CUDA(cudaLaunchKernelEx(&cfg, k_batch<false, false>, P));
    CMG_CUDA(cudaMemcpyAsync(b->h_ctrl, b->ctrl, 8 * sizeof(int), cudaMemcpyDeviceToHost, s));
  } catch (...) {
    cudaGraph_t g;
    cudaStreamEndCapture(s, &g);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    throw;
  }
  CMG_CUDA(cudaStreamEndCapture(s, &b->graph));
  CMG_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
  b->g_sched = b->sched;
  b->g_params = *p;
  b->g_grid = grid;
  b->g_budget = b->spin_budget;
}

int64_t updates_per_cycle(const cmg_batch *b, bool mixed) {
  const cmg_level *L = b->lvl;
  const int nsw = b->sched.n_pre + b->sched.n_post;
  int64_t u = 0;
  for (size_t m = 0; m < L->mg.size(); ++m) u += (int64_t)nsw * 8 * L->mg[m].n;
  return mixed ? u * b->sched.inner_cycles : u;
}


}  // namespace

int batch_solve(cmg_batch *b, const cmg_solve_params *p, cmg_batch_stats *st) {
  if (!p || !(p->tol >= 0.0) || p->max_cycles < 0 || p->fixed_cycles < 0 ||
      (p->precision != CMG_PREC_FP64 && p->precision != CMG_PREC_MIXED) || (p->krylov != 0 && p->krylov != 1))
    throw Error(CMG_ERR_INVALID_ARG, "invalid solve parameters");
  cmg_level *L = b->lvl;
  cmg_ctx *ctx = L->ctx;
  const bool mixed = p->precision == CMG_PREC_MIXED;
  if (p->krylov == 1 && mixed && L->mg.size() < 2)
    throw Error(CMG_ERR_INVALID_ARG, "mixed-precision CG needs at least two multigrid levels");
  if (mixed) ensure_fp32(L);
  if (p->krylov == 1) ensure_cg(b);
  if (!b->exec || !same_sched(b->sched, b->g_sched) || !same_params(*p, b->g_params) ||
      b->spin_budget != b->g_budget)
    record(b, p);
  CMG_CUDA(cudaEventRecord(ctx->ev0, ctx->stream));
  CMG_CUDA(cudaGraphLaunch(b->exec, ctx->stream));
  CMG_CUDA(cudaEventRecord(ctx->ev1, ctx->stream));
  CMG_CUDA(cudaEventSynchronize(ctx->ev1));
  float ms = 0.f;
  CMG_CUDA(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
  const int *c = b->h_ctrl;
  ctx->launches += 1;
  cmg_batch_stats S = {};
  S.status = c[0];
  S.cycles = c[1];
  S.n_patches = b->n_patches;
  S.n_converged = c[5];
  S.ms = ms;
  S.cell_updates = updates_per_cycle(b, mixed) * c[1];
  S.grid_barriers = c[4];
  std::vector<double> rel(b->n_patches);
  CMG_CUDA(cudaMemcpy(rel.data(), b->pstate + 4 * b->n_patches, sizeof(double) * b->n_patches,
                      cudaMemcpyDeviceToHost));
  for (double r : rel) S.rel_max = std::max(S.rel_max, r);
  if (st) *st = S;
  return S.status;
}

void batch_create(cmg_level *L, const int64_t *offsets, int n_patches, cmg_batch **out) {
  if (!L || !offsets || n_patches < 1) throw Error(CMG_ERR_INVALID_ARG, "bad batch arguments");
  if (offsets[0] != 0 || offsets[n_patches] != L->n) throw Error(CMG_ERR_INVALID_ARG, "offsets must span the level");
  for (int k = 0; k < n_patches; ++k)
    if (offsets[k + 1] <= offsets[k]) throw Error(CMG_ERR_INVALID_ARG, "empty or decreasing patch range");
  if (!L->parent) throw Error(CMG_ERR_INVALID_ARG, "a batch needs a refined level (Dirichlet patches)");
  if ((int)L->mg.size() > kBMaxLevels) throw Error(CMG_ERR_INVALID_ARG, "too many multigrid levels");
  cmg_ctx *ctx = L->ctx;
  cudaStream_t s = ctx->stream;
  auto *b = new cmg_batch();
  try {
    b->lvl = L;
    b->n_patches = n_patches;
    int64_t *d_off = b->mem.alloc<int64_t>(n_patches + 1);
    CMG_CUDA(cudaMemcpyAsync(d_off, offsets, sizeof(int64_t) * (n_patches + 1), cudaMemcpyHostToDevice, s));
    for (size_t m = 0; m < L->mg.size(); ++m) b->pid.push_back(b->mem.alloc<int32_t>(L->mg[m].n));
    k_patch_ids<<<blocks_for(L->n), kThreads, 0, s>>>(d_off, n_patches, b->pid[0], L->n);
    CMG_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s));
    for (size_t m = 0; m + 1 < L->mg.size(); ++m)
      k_patch_up<<<blocks_for(L->mg[m].n), kThreads, 0, s>>>(b->pid[m], L->mg[m].father, L->mg[m].n, b->pid[m + 1]);
    for (size_t m = 0; m < L->mg.size(); ++m) {
      const bool has_c = m + 1 < L->mg.size();
      k_patch_check<<<blocks_for(L->mg[m].n), kThreads, 0, s>>>(b->pid[m], L->mg[m].nbr,
                                                                  has_c ? L->mg[m].father : nullptr,
                                                                  has_c ? b->pid[m + 1] : nullptr, L->mg[m].n,
                                                                  ctx->d_err);
    }
    CMG_CUDA(cudaGetLastError());
    int err = 0;
    CMG_CUDA(cudaMemcpyAsync(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    if (err) {
      CMG_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s));
      throw Error(CMG_ERR_INVALID_ARG, "patches are not independent: a neighbour link joins two patches");
    }
    b->pstate = b->mem.alloc<double>(5 * (int64_t)n_patches, true, s);
    b->conv_at = b->mem.alloc<int32_t>(n_patches, true, s);
    b->ctrl = b->mem.alloc<int>(8, true, s);
    b->bar = b->mem.alloc<unsigned>(2, true, s);
    CMG_CUDA(cudaMallocHost(&b->h_ctrl, 8 * sizeof(int)));
    CMG_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    cudaStreamSynchronize(s);
    if (b->h_ctrl) cudaFreeHost(b->h_ctrl);
    b->mem.release();
    delete b;
    throw;
  }
  *out = b;
}

void batch_destroy(cmg_batch *b) {
  cudaStreamSynchronize(b->lvl->stream);
  drop_graph(b);
  if (b->h_ctrl) cudaFreeHost(b->h_ctrl);
  b->mem.release();
  delete b;
}

void batch_patch_stats(cmg_batch *b, double *rel, int32_t *conv, double *norm0) {
  const int n = b->n_patches;
  std::vector<double> st(5 * (size_t)n);
  CMG_CUDA(cudaMemcpy(st.data(), b->pstate, sizeof(double) * 5 * n, cudaMemcpyDeviceToHost));
  if (rel)
    for (int k = 0; k < n; ++k) rel[k] = st[4 * (size_t)n + k];
  if (norm0) {
    // d-units to r-units: r = -6 / h^2 d
    const double h = b->lvl->mg[0].h;
    for (int k = 0; k < n; ++k) norm0[k] = std::sqrt(st[k]) * 6.0 / (h * h);
  }
  if (conv) CMG_CUDA(cudaMemcpy(conv, b->conv_at, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
}

void batch_set_schedule(cmg_batch *b, const cmg_batch_schedule *s) {
  if (!s || s->threads < 32 || s->threads > 1024 || s->threads % 32 || s->blocks_per_sm < 1 || s->n_pre < 0 ||
      s->n_post < 0 || s->n_pre + s->n_post < 1 || s->inner_cycles < 1)
    throw Error(CMG_ERR_INVALID_ARG, "invalid batch schedule");
  b->sched = *s;
}

void batch_autotune(cmg_batch *b, const cmg_solve_params *p, cmg_batch_schedule *best, double *best_ms) {
  cmg_level *L = b->lvl;
  cudaStream_t s = L->ctx->stream;
  const bool mixed = p->precision == CMG_PREC_MIXED;
  MgLev &top = L->mg[0];
  const int64_t cnt = 8 * top.n_alloc;
  double *saved = nullptr;
  CMG_CUDA(cudaMalloc(&saved, sizeof(double) * cnt));
  CMG_CUDA(cudaMemcpyAsync(saved, top.phi, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, s));
  // two stages: the block shape (and inner cycles) with V(2,2), then the
  // sweep schedule with the best shape
  const cmg_batch_schedule keep = b->sched;
  double best_t = 1e300;
  cmg_batch_schedule best_s = keep;
  auto time_candidate = [&](const cmg_batch_schedule &c) {
    b->sched = c;
    int per_sm = 0;
    const void *fn = batch_kernel(mixed, p->krylov == 1);
    if (!block_fits(fn, c.threads)) return;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, c.threads, 0) != cudaSuccess || per_sm < 1) {
      cudaGetLastError();
      return;
    }
    if (c.blocks_per_sm > per_sm) return;
    double t = 0.0;
    for (int rep = 0; rep < 2; ++rep) {  // first run records the graph
      CMG_CUDA(cudaMemcpyAsync(top.phi, saved, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, s));
      cmg_batch_stats st;
      const int rc = batch_solve(b, p, &st);
      t = (rc == CMG_OK || rc == CMG_ERR_NOT_CONVERGED) && st.n_converged == b->n_patches ? st.ms : 1e300;
    }
    if (t < best_t) {
      best_t = t;
      best_s = c;
    }
  };
  try {
    for (int th : {256, 512})
      for (int bps : {1, 2, 4})
        for (int inner : {1, 2}) {
          if (!mixed && inner == 2) continue;
          time_candidate({th, bps, 2, 2, inner});
        }
    const cmg_batch_schedule shape = best_s;
    const int sweeps[][2] = {{1, 1}, {2, 3}, {3, 2}, {3, 3}};
    for (const auto &sw : sweeps) time_candidate({shape.threads, shape.blocks_per_sm, sw[0], sw[1], shape.inner_cycles});
  } catch (...) {
    b->sched = keep;
    cudaMemcpyAsync(top.phi, saved, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, s);
    cudaStreamSynchronize(s);
    cudaFree(saved);
    throw;
  }
  b->sched = best_s;
  CMG_CUDA(cudaMemcpyAsync(top.phi, saved, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, s));
  CMG_CUDA(cudaStreamSynchronize(s));
  cudaFree(saved);
  if (best) *best = best_s;
  if (best_ms) *best_ms = best_t;
}

}  // namespace cmg
