// kernels.cuh -- one-operation-per-launch kernels of the multigrid V-cycle
// (thread per oct), built on the per-oct bodies of oct_ops.cuh:
//   red-black Gauss-Seidel colour pass      App. D.2 Eq. (gs_update)
//   residual (+ squared norm, + restriction) Sec. 5.1.1 item (iii); restriction = mean of 8 children
//   prolongation + correction               Sec. 5.1.1 (trilinear interpolation)
//   coarse-fine Dirichlet ghost values      interpolation of the parent's phi (morton_nbor_cell, App. B)
//   coarsest periodic 2^3 solve             exact (Walsh-Hadamard diagonalisation)
// Included by launch.cu only.
#pragma once

#include "oct_ops.cuh"

namespace cmg {
namespace {

// Deterministic block sum of one double per thread -> partials[blockIdx.x].
__device__ void block_sum_to(double v, double *partials) {
  __shared__ double ws[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) partials[blockIdx.x] = w;
  }
}

// FP32 kernels read their oct's index data (written only by the level build)
// before the grid-dependency wait, overlapping the preceding kernel's tail:
// measured on the two-level 128^3 workload, the mixed-precision solves got
// 2-3 % faster.  FP64 kernels, bound by GB300's FP64 issue rate, keep every
// load after the wait: with the early reads the refined level's FP64 solve
// got ~1-3 % slower.  FP32 colour passes preload only on levels of at most
// kPreloadSweepOcts octs: the HBM-bound pass over a 512^3 level got 3 %
// slower with it (the residual there got faster).
template <typename T>
constexpr bool kPreloadIdx = sizeof(T) == 4;
constexpr int64_t kPreloadSweepOcts = int64_t(1) << 20;

template <typename T, int P, bool ZERO, bool MASK, bool PRE>
__global__ void __launch_bounds__(kThreads) k_sweep(const int32_t *__restrict__ nbr, const T *__restrict__ src,
                                                   T *__restrict__ dst, const T *__restrict__ g,
                                                   const uint8_t *__restrict__ active, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if constexpr (PRE) {
    dev::SweepIdx x;
    if (i < n) x = dev::sweep_idx<ZERO, MASK>(i, nbr, active, n);
    pdl_enter();
    if (i >= n) return;
    dev::sweep_oct_idx<T, P, ZERO, MASK, false>(i, x, src, dst, g);
  } else {
    pdl_enter();
    if (i >= n) return;
    dev::sweep_oct<T, P, ZERO, MASK, false>(i, nbr, src, dst, g, active, n);
  }
}

template <typename T, bool NORM, bool RESTRICT, bool EMIT, bool ROUT, bool ZPHI, bool C1Z = false>
__global__ void __launch_bounds__(kThreads) k_resid(const int32_t *__restrict__ nbr, const T *__restrict__ phi,
                                                   const T *__restrict__ g, const uint8_t *__restrict__ active,
                                                   int64_t n, int64_t n_alloc, const int32_t *__restrict__ father,
                                                   T *__restrict__ cg, T *__restrict__ cphi, int64_t cn,
                                                   int64_t cn_alloc, int zero_cphi, double *__restrict__ partials,
                                                   float *__restrict__ g32, const double *__restrict__ emit_scale,
                                                   double *__restrict__ rout, double rscale) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double acc = 0.0;
  if constexpr (kPreloadIdx<T>) {
    dev::ResidIdx x;
    if (i < n) x = dev::resid_idx<RESTRICT>(i, nbr, active, n, father);
    pdl_enter();
    if (i < n) {
      const double inv_s = EMIT ? 1.0 / *emit_scale : 0.0;
      acc = dev::resid_oct_idx<T, NORM, RESTRICT, EMIT, ROUT, ZPHI, false, C1Z>(i, x, phi, g, n, n_alloc, cg, cphi, cn,
                                                                           cn_alloc, zero_cphi, g32, inv_s, rout,
                                                                           rscale);
    }
  } else {
    pdl_enter();
    if (i < n) {
      const double inv_s = EMIT ? 1.0 / *emit_scale : 0.0;
      acc = dev::resid_oct<T, NORM, RESTRICT, EMIT, ROUT, ZPHI, false, C1Z>(i, nbr, phi, g, active, n, n_alloc, father,
                                                                       cg, cphi, cn, cn_alloc, zero_cphi, g32, inv_s,
                                                                       rout, rscale);
    }
  }
  if (NORM) block_sum_to(acc, partials);
}

template <typename T, bool MASK, bool C0D>
__global__ void __launch_bounds__(kThreads) k_prolong(const uint64_t *__restrict__ keys, const int32_t *__restrict__ blk,
                                                     int64_t n, int64_t n_alloc, T *__restrict__ phi,
                                                     const uint8_t *__restrict__ active,
                                                     const T *__restrict__ cphi, int64_t cn_alloc) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if constexpr (kPreloadIdx<T>) {
    dev::ProlongIdx x;
    if (i < n) x = dev::prolong_idx<MASK>(i, keys, blk, n, active);
    pdl_enter();
    if (i >= n) return;
    dev::prolong_oct_idx<T, MASK, false, C0D>(i, x, n_alloc, phi, cphi, cn_alloc);
  } else {
    pdl_enter();
    if (i >= n) return;
    dev::prolong_oct<T, MASK, false, C0D>(i, keys, blk, n, n_alloc, phi, active, cphi, cn_alloc);
  }
}

__global__ void __launch_bounds__(kThreads) k_ghost_fill(const uint64_t *__restrict__ gkeys,
                                                        const int32_t *__restrict__ gblk,
                                                        const uint32_t *__restrict__ gmask, int64_t n_ghost,
                                                        int64_t n, int64_t n_alloc, double *__restrict__ phi,
                                                        const double *__restrict__ pphi, int64_t pn_alloc) {
  pdl_enter();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n_ghost) return;
  const int cc = (int)(gkeys[t] & 7);
  int32_t b[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) b[k] = __ldg(gblk + k * n_ghost + t);
  double val[8];
  dev::interp8<double, false>(pphi, pn_alloc, b, cc, val);
  const uint32_t m = gmask[t];
  const int64_t oct = n + t;
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    double v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = plane_cell(p, q);
      v[q] = ((m >> c) & 1) ? val[c] : 0.0;
    }
    dev::store4(phi + (p * n_alloc + oct) * 4, v);
  }
}

// Ghost values in the [n][6][4] API layout (NaN where the neighbour exists).
__global__ void k_get_ghosts(const int32_t *__restrict__ nbr, int64_t n, int64_t n_ghost, int64_t n_alloc,
                             const double *__restrict__ phi, double *__restrict__ out) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int d = 0; d < 6; ++d) {
    const int64_t o = nbr[d * n + i];
    const bool ghost = o >= n && o < n + n_ghost;
    const int a = d >> 1, side = d & 1;
    int q = 0;
    for (int c = 0; c < 8; ++c) {
      if (((c >> a) & 1) != side) continue;
      const int c2 = c ^ (1 << a);
      out[(i * 6 + d) * 4 + q] = ghost ? phi[((int64_t)cell_parity(c2) * n_alloc + o) * 4 + (c2 >> 1)]
                                       : __longlong_as_double(0x7ff8000000000000ll);
      ++q;
    }
  }
}

template <typename T>
__global__ void k_wht(const T *__restrict__ g, T *__restrict__ phi, int64_t n_alloc, double h) {
  pdl_enter();
  if (threadIdx.x >= 32 || blockIdx.x != 0) return;
  dev::wht_solve_warp<T, T, false>(g, phi, n_alloc, h);
}

__global__ void k_set_density(const double *__restrict__ rho, int64_t n, double rho_bar, double scale,
                              double *__restrict__ g) {
  pdl_enter();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 8 * n) return;
  const int64_t i = t >> 3;
  const int c = (int)(t & 7);
  g[((int64_t)cell_parity(c) * n + i) * 4 + (c >> 1)] = scale * (rho[t] - rho_bar);
}

// oct-major [n][8] <-> planar [2][stride][4], with a scale factor
template <typename S, typename D>
__global__ void k_pack(const S *__restrict__ in, int64_t n, int64_t stride, double scale, D *__restrict__ out) {
  pdl_enter();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 8 * n) return;
  const int64_t i = t >> 3;
  const int c = (int)(t & 7);
  out[((int64_t)cell_parity(c) * stride + i) * 4 + (c >> 1)] = (D)(scale * (double)in[t]);
}

template <typename S, typename D>
__global__ void k_unpack(const S *__restrict__ in, int64_t n, int64_t stride, double scale, D *__restrict__ out) {
  pdl_enter();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 8 * n) return;
  const int64_t i = t >> 3;
  const int c = (int)(t & 7);
  out[t] = (D)(scale * (double)in[((int64_t)cell_parity(c) * stride + i) * 4 + (c >> 1)]);
}

__global__ void k_sum_phi(const double *__restrict__ phi, int64_t n, int64_t n_alloc, double *__restrict__ partials) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (i < n) {
    double a[4], b[4];
    dev::load4<false>(phi + i * 4, a);
    dev::load4<false>(phi + (n_alloc + i) * 4, b);
    acc = ((a[0] + a[1]) + (a[2] + a[3])) + ((b[0] + b[1]) + (b[2] + b[3]));
  }
  block_sum_to(acc, partials);
}

__global__ void k_sub_scalar(double *__restrict__ phi, int64_t n, int64_t n_alloc, const double *__restrict__ s) {
  pdl_enter();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 8 * n) return;
  const int64_t i = t >> 3;
  const int p = (int)((t >> 2) & 1);
  const int q = (int)(t & 3);
  phi[(p * n_alloc + i) * 4 + q] -= *s;
}

// phi64 += S * phi32 on the real octs (solution accumulation, FP64)
__global__ void k_accumulate(double *__restrict__ phi, const float *__restrict__ e, int64_t n, int64_t n_alloc,
                             const double *__restrict__ scale) {
  pdl_enter();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 2 * n) return;
  const int p = (int)(t / n);
  const int64_t i = t - p * n;
  const double S = *scale;
  double v[4];
  float w[4];
  dev::load4<false>(phi + (p * n_alloc + i) * 4, v);
  dev::load4<false>(e + (p * n_alloc + i) * 4, w);
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = fma(S, (double)w[q], v[q]);
  dev::store4(phi + (p * n_alloc + i) * 4, v);
}

// Sum partials in a fixed order; out[0] = scale * sum (and its sqrt to out[1]).
__global__ void k_finalize(const double *__restrict__ partials, int np, double scale, double *__restrict__ out,
                           int with_sqrt) {
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
      out[0] = scale * w;
      if (with_sqrt) out[1] = sqrt(scale * w);
    }
  }
}

__global__ void k_copy_convert_f2d(const float *__restrict__ a, double *__restrict__ b, int64_t m) {
  pdl_enter();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < m) b[t] = (double)a[t];
}
__global__ void k_copy_convert_d2f(const double *__restrict__ a, float *__restrict__ b, int64_t m) {
  pdl_enter();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < m) b[t] = (float)a[t];
}

template <typename T>
T *phi_of(MgLev &g);
template <>
double *phi_of<double>(MgLev &g) { return g.phi; }
template <>
float *phi_of<float>(MgLev &g) { return g.phi32; }
template <typename T>
T *g_of(MgLev &g);
template <>
double *g_of<double>(MgLev &g) { return g.g; }
template <>
float *g_of<float>(MgLev &g) { return g.g32; }

}  // namespace
}  // namespace cmg
