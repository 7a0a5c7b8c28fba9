// shard.cu -- operations of the V-cycle restricted to a range of octs, and
// cell-granular gather / scatter of level fields: the device side of the
// sharded level solve (App. G, GPU V-cycle algorithm: every rank smooths,
// evaluates the residual, restricts and prolongs on the octs it owns, and
// exchanges boundary values between the steps; Sec. 9.5 describes the
// halo exchange between GPUs).
//
// The range kernels run the same per-oct bodies as the whole-level kernels
// (oct_ops.cuh), so an oct's result does not depend on which launch computed
// it.  FP64 only.
#include "oct_ops.cuh"

namespace cmg {
namespace {

constexpr int kT = 256;

unsigned grid_of(int64_t n) { return (unsigned)((n + kT - 1) / kT); }

template <int P, bool ZERO, bool MASK>
__global__ void __launch_bounds__(kT) k_sweep_range(const int32_t *__restrict__ nbr, const double *__restrict__ src,
                                                    double *__restrict__ dst, const double *__restrict__ g,
                                                    const uint8_t *__restrict__ active, int64_t n, int64_t lo,
                                                    int64_t hi) {
  const int64_t i = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= hi) return;
  dev::sweep_oct<double, P, ZERO, MASK, false>(i, nbr, src, dst, g, active, n);
}

// Deterministic block sum of one double per thread -> partials[blockIdx.x].
__device__ void block_sum(double v, double *partials) {
  __shared__ double ws[kT / 32];
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

// Residual of the octs [lo, hi): NORM sums d^2 per block; RESTRICT writes the
// father cells' source and zeroes their phi (the children in the range only).
template <bool NORM, bool RESTRICT, bool C1Z>
__global__ void __launch_bounds__(kT)
    k_resid_range(const int32_t *__restrict__ nbr, const double *__restrict__ phi, const double *__restrict__ g,
                  const uint8_t *__restrict__ active, int64_t n, int64_t n_alloc, const int32_t *__restrict__ father,
                  double *__restrict__ cg, double *__restrict__ cphi, int64_t cn, int64_t cn_alloc, int64_t lo,
                  int64_t hi, double *__restrict__ partials) {
  const int64_t i = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (i < hi)
    acc = dev::resid_oct<double, NORM, RESTRICT, false, false, false, false, C1Z>(
        i, nbr, phi, g, active, n, n_alloc, father, cg, cphi, cn, cn_alloc, 1, nullptr, 0.0, nullptr, 0.0);
  if (NORM) block_sum(acc, partials);
}

template <bool MASK, bool C0D>
__global__ void __launch_bounds__(kT) k_prolong_range(const uint64_t *__restrict__ keys,
                                                      const int32_t *__restrict__ blk, int64_t n, int64_t n_alloc,
                                                      double *__restrict__ phi, const uint8_t *__restrict__ active,
                                                      const double *__restrict__ cphi, int64_t cn_alloc, int64_t lo,
                                                      int64_t hi) {
  const int64_t i = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= hi) return;
  dev::prolong_oct<double, MASK, false, C0D>(i, keys, blk, n, n_alloc, phi, active, cphi, cn_alloc);
}

__global__ void __launch_bounds__(kT) k_sum_phi_range(const double *__restrict__ phi, int64_t n_alloc, int64_t lo,
                                                      int64_t hi, double *__restrict__ partials) {
  const int64_t i = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (i < hi) {
    double a[4], b[4];
    dev::load4<false>(phi + i * 4, a);
    dev::load4<false>(phi + (n_alloc + i) * 4, b);
    acc = ((a[0] + a[1]) + (a[2] + a[3])) + ((b[0] + b[1]) + (b[2] + b[3]));
  }
  block_sum(acc, partials);
}

__global__ void __launch_bounds__(kT) k_shift_phi_range(double *__restrict__ phi, int64_t n_alloc, int64_t lo,
                                                        int64_t hi, double s) {
  const int64_t t = lo * 8 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= hi * 8) return;
  const int64_t i = t >> 3;
  const int p = (int)((t >> 2) & 1), q = (int)(t & 3);
  phi[(p * n_alloc + i) * 4 + q] -= s;
}

// Sum of partials in a fixed order, times scale -> *out.
__global__ void k_finish(const double *__restrict__ partials, int np, double scale, double *__restrict__ out) {
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
    if (threadIdx.x == 0) *out = scale * w;
  }
}

// Cell c of oct i in the planar layout [2][stride][4].
__device__ __forceinline__ int64_t cell_at(int64_t cell, int64_t stride) {
  const int64_t i = cell >> 3;
  const int c = (int)(cell & 7);
  return ((int64_t)cell_parity(c) * stride + i) * 4 + (c >> 1);
}

__global__ void k_gather_cells(const double *__restrict__ f, int64_t stride, int64_t n, const int32_t *__restrict__ idx,
                               int64_t cnt, double *__restrict__ out, int *__restrict__ bad) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int64_t c = idx[t];
  if (c < 0 || c >= 8 * n) {
    atomicCAS(bad, 0, (int)CMG_ERR_INVALID_ARG);
    return;
  }
  out[t] = f[cell_at(c, stride)];
}

__global__ void k_scatter_cells(double *__restrict__ f, int64_t stride, int64_t n, const int32_t *__restrict__ idx,
                                int64_t cnt, const double *__restrict__ in, int *__restrict__ bad) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int64_t c = idx[t];
  if (c < 0 || c >= 8 * n) {
    atomicCAS(bad, 0, (int)CMG_ERR_INVALID_ARG);
    return;
  }
  f[cell_at(c, stride)] = in[t];
}

}  // namespace

void range_sweep_pass(cmg_level *L, int m, int colour, bool zero_other, int64_t lo, int64_t hi) {
  MgLev &g = L->mg[m];
  if (hi <= lo) return;
  cudaStream_t s = L->ctx->stream;
  const int64_t st = g.n_alloc * 4;
  const bool mask = !g.all_active;
  const unsigned nb = grid_of(hi - lo);
  double *src = g.phi + (1 - colour) * st, *dst = g.phi + colour * st;
  const double *gg = g.g + colour * g.n * 4;
#define CMG_RSWEEP(P, Z, M) \
  k_sweep_range<P, Z, M><<<nb, kT, 0, s>>>(g.nbr, src, dst, gg, g.active, g.n, lo, hi)
  if (colour == 0) {
    if (zero_other) {
      if (mask) CMG_RSWEEP(0, true, true); else CMG_RSWEEP(0, true, false);
    } else {
      if (mask) CMG_RSWEEP(0, false, true); else CMG_RSWEEP(0, false, false);
    }
  } else {
    if (zero_other) {
      if (mask) CMG_RSWEEP(1, true, true); else CMG_RSWEEP(1, true, false);
    } else {
      if (mask) CMG_RSWEEP(1, false, true); else CMG_RSWEEP(1, false, false);
    }
  }
#undef CMG_RSWEEP
  CMG_CUDA(cudaGetLastError());
}

// norm_out (device): scale * sum d^2 = sum r^2 over the range (NORM);
// restriction of the range's fully active octs to the father cells.
void range_residual(cmg_level *L, int m, bool restrict_to_coarse, bool c1_swept, int64_t lo, int64_t hi,
                    double *norm_out) {
  MgLev &g = L->mg[m];
  cudaStream_t s = L->ctx->stream;
  const uint8_t *act = g.all_active ? nullptr : g.active;
  MgLev *c = restrict_to_coarse ? &L->mg[m + 1] : nullptr;
  const unsigned nb = grid_of(hi > lo ? hi - lo : 1);
  if (!restrict_to_coarse) {
    if (hi > lo) {
      if (c1_swept)
        k_resid_range<true, false, true><<<nb, kT, 0, s>>>(g.nbr, g.phi, g.g, act, g.n, g.n_alloc, nullptr, nullptr,
                                                          nullptr, 0, 0, lo, hi, L->partials);
      else
        k_resid_range<true, false, false><<<nb, kT, 0, s>>>(g.nbr, g.phi, g.g, act, g.n, g.n_alloc, nullptr,
                                                           nullptr, nullptr, 0, 0, lo, hi, L->partials);
      k_finish<<<1, 1024, 0, s>>>(L->partials, (int)nb, 36.0 / (g.h * g.h * g.h * g.h), norm_out);
    } else {
      CMG_CUDA(cudaMemsetAsync(norm_out, 0, sizeof(double), s));
    }
  } else if (hi > lo) {
    if (c1_swept)
      k_resid_range<false, true, true><<<nb, kT, 0, s>>>(g.nbr, g.phi, g.g, act, g.n, g.n_alloc, g.father, c->g,
                                                        c->phi, c->n, c->n_alloc, lo, hi, nullptr);
    else
      k_resid_range<false, true, false><<<nb, kT, 0, s>>>(g.nbr, g.phi, g.g, act, g.n, g.n_alloc, g.father, c->g,
                                                         c->phi, c->n, c->n_alloc, lo, hi, nullptr);
  }
  CMG_CUDA(cudaGetLastError());
}

void range_prolong(cmg_level *L, int m, bool c0_dead, int64_t lo, int64_t hi) {
  MgLev &g = L->mg[m];
  MgLev &c = L->mg[m + 1];
  if (hi <= lo) return;
  cudaStream_t s = L->ctx->stream;
  const unsigned nb = grid_of(hi - lo);
  if (g.all_active && c0_dead)
    k_prolong_range<false, true><<<nb, kT, 0, s>>>(g.keys, g.blk, g.n, g.n_alloc, g.phi, g.active, c.phi, c.n_alloc,
                                                   lo, hi);
  else if (g.all_active)
    k_prolong_range<false, false><<<nb, kT, 0, s>>>(g.keys, g.blk, g.n, g.n_alloc, g.phi, g.active, c.phi,
                                                    c.n_alloc, lo, hi);
  else if (c0_dead)
    k_prolong_range<true, true><<<nb, kT, 0, s>>>(g.keys, g.blk, g.n, g.n_alloc, g.phi, g.active, c.phi, c.n_alloc,
                                                  lo, hi);
  else
    k_prolong_range<true, false><<<nb, kT, 0, s>>>(g.keys, g.blk, g.n, g.n_alloc, g.phi, g.active, c.phi, c.n_alloc,
                                                   lo, hi);
  CMG_CUDA(cudaGetLastError());
}

void range_sum_phi(cmg_level *L, int m, int64_t lo, int64_t hi, double *out) {
  MgLev &g = L->mg[m];
  cudaStream_t s = L->ctx->stream;
  if (hi <= lo) {
    CMG_CUDA(cudaMemsetAsync(out, 0, sizeof(double), s));
    return;
  }
  const unsigned nb = grid_of(hi - lo);
  k_sum_phi_range<<<nb, kT, 0, s>>>(g.phi, g.n_alloc, lo, hi, L->partials);
  k_finish<<<1, 1024, 0, s>>>(L->partials, (int)nb, 1.0, out);
  CMG_CUDA(cudaGetLastError());
}

void range_shift_phi(cmg_level *L, int m, int64_t lo, int64_t hi, double v) {
  MgLev &g = L->mg[m];
  if (hi <= lo) return;
  k_shift_phi_range<<<grid_of(8 * (hi - lo)), kT, 0, L->ctx->stream>>>(g.phi, g.n_alloc, lo, hi, v);
  CMG_CUDA(cudaGetLastError());
}

// field 0 = phi ([2][n_alloc][4]), 1 = the stored source g ([2][n][4]).
void gather_cells(cmg_level *L, int m, int field, const int32_t *idx, int64_t cnt, double *out, int *bad) {
  MgLev &g = L->mg[m];
  if (cnt <= 0) return;
  const double *f = field == 0 ? g.phi : g.g;
  const int64_t stride = field == 0 ? g.n_alloc : g.n;
  k_gather_cells<<<grid_of(cnt), kT, 0, L->ctx->stream>>>(f, stride, g.n, idx, cnt, out, bad);
  CMG_CUDA(cudaGetLastError());
}

void scatter_cells(cmg_level *L, int m, int field, const int32_t *idx, int64_t cnt, const double *in, int *bad) {
  MgLev &g = L->mg[m];
  if (cnt <= 0) return;
  double *f = field == 0 ? g.phi : g.g;
  const int64_t stride = field == 0 ? g.n_alloc : g.n;
  k_scatter_cells<<<grid_of(cnt), kT, 0, L->ctx->stream>>>(f, stride, g.n, idx, cnt, in, bad);
  CMG_CUDA(cudaGetLastError());
}

}  // namespace cmg
