// ops.cu -- numerical kernels of the multigrid V-cycle on colour-planar oct
// fields (see cmg_internal.cuh for the layout):
//   red-black Gauss-Seidel colour pass      App. D.2 Eq. (gs_update)
//   residual (+ squared norm, + restriction) Sec. 5.1.1 item (iii), restriction = mean of 8 children
//   prolongation + correction               Sec. 5.1.1 (trilinear interpolation)
//   coarse-fine Dirichlet ghost values      interpolation of the parent's phi (morton_nbor_cell, App. B)
//   coarsest periodic 2^3 solve             exact (Walsh-Hadamard diagonalisation)
// All kernels run one thread per oct; FP64 and FP32 (mixed precision) share
// the same templates.
#include <cmath>

#include "cmg_internal.cuh"

namespace cmg {
namespace {

// ------------------------------------------------------------ vector I/O

__device__ __forceinline__ void load4(const double *p, double v[4]) {
  const double2 a = *reinterpret_cast<const double2 *>(p);
  const double2 b = *reinterpret_cast<const double2 *>(p + 2);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}
__device__ __forceinline__ void load4(const float *p, float v[4]) {
  const float4 a = *reinterpret_cast<const float4 *>(p);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = a.z;
  v[3] = a.w;
}
__device__ __forceinline__ void store4(double *p, const double v[4]) {
  *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
  *reinterpret_cast<double2 *>(p + 2) = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void store4(float *p, const float v[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

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

// ------------------------------------------------------------ colour pass

// One colour pass of red-black Gauss-Seidel: plane P of every oct from the
// other plane of the oct and of its six face neighbours.  ZERO: the other
// plane is known to be zero (first sweep after restriction), so phi = g.
template <typename T, int P, bool ZERO, bool MASK>
__global__ void __launch_bounds__(kThreads) k_sweep(const int32_t *__restrict__ nbr, const T *__restrict__ src,
                                                   T *__restrict__ dst, const T *__restrict__ g,
                                                   const uint8_t *__restrict__ active, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  T gv[4], out[4];
  load4(g + i * 4, gv);
  if (ZERO) {
#pragma unroll
    for (int q = 0; q < 4; ++q) out[q] = gv[q];
  } else {
    T own[4];
    load4(src + i * 4, own);
    int32_t nb[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) nb[d] = __ldg(nbr + d * n + i);
    const T inv6 = T(1) / T(6);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = plane_cell(P, q);
      T s = T(0);
#pragma unroll
      for (int d = 0; d < 6; ++d) {
        const int a = d >> 1, side = d & 1, c2 = c ^ (1 << a);
        const T v = (((c >> a) & 1) != side) ? own[c2 >> 1] : src[(int64_t)nb[d] * 4 + (c2 >> 1)];
        s = d == 0 ? v : s + v;
      }
      out[q] = fma_t(s, inv6, gv[q]);
    }
  }
  if (MASK) {
    const unsigned m = active[i];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (!((m >> plane_cell(P, q)) & 1)) out[q] = T(0);
  }
  store4(dst + i * 4, out);
}

// ------------------------------------------------------------ residual

// d = fma(s, 1/6, g) - phi per cell; r = (-6 / h^2) d.
//  NORM:     partials[block] = sum of d^2
//  RESTRICT: a fully active oct writes its father cell g_c = 0.5 * sum_8 d
//            (= -h_c^2/6 * mean_8 r), and optionally zeroes the coarse phi
//  EMIT:     g32 = (float)(d / S), S = *emit_scale (mixed precision)
//  ROUT:     r written oct-major (masked by the active cells)
//  ZPHI:     phi taken as zero on real octs (ghost octs keep their values)
template <typename T, bool NORM, bool RESTRICT, bool EMIT, bool ROUT, bool ZPHI>
__global__ void __launch_bounds__(kThreads) k_resid(const int32_t *__restrict__ nbr, const T *__restrict__ phi,
                                                   const T *__restrict__ g, const uint8_t *__restrict__ active,
                                                   int64_t n, int64_t n_alloc, const int32_t *__restrict__ father,
                                                   T *__restrict__ cg, T *__restrict__ cphi, int64_t cn,
                                                   int64_t cn_alloc, int zero_cphi, double *__restrict__ partials,
                                                   float *__restrict__ g32, const double *__restrict__ emit_scale,
                                                   double *__restrict__ rout, double rscale) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (i < n) {
    T pl[2][4], gv[2][4];
    if (ZPHI) {
#pragma unroll
      for (int q = 0; q < 4; ++q) pl[0][q] = pl[1][q] = T(0);
    } else {
      load4(phi + i * 4, pl[0]);
      load4(phi + (n_alloc + i) * 4, pl[1]);
    }
    load4(g + i * 4, gv[0]);
    load4(g + (n + i) * 4, gv[1]);
    int32_t nb[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) nb[d] = __ldg(nbr + d * n + i);
    const T inv6 = T(1) / T(6);
    const unsigned m = active ? active[i] : 0xFFu;
    T rsum = T(0);
    double inv_s = 0.0;
    if (EMIT) inv_s = 1.0 / *emit_scale;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = plane_cell(p, q);
        T s = T(0);
#pragma unroll
        for (int d = 0; d < 6; ++d) {
          const int a = d >> 1, side = d & 1, c2 = c ^ (1 << a);
          T v;
          if (((c >> a) & 1) != side) {
            v = pl[1 - p][c2 >> 1];
          } else {
            const int64_t o = nb[d];
            v = (ZPHI && o < n) ? T(0) : phi[((1 - p) * n_alloc + o) * 4 + (c2 >> 1)];
          }
          s = d == 0 ? v : s + v;
        }
        T dv = fma_t(s, inv6, gv[p][q]) - pl[p][q];
        if (!((m >> c) & 1)) dv = T(0);
        if (NORM) acc = fma((double)dv, (double)dv, acc);
        if (RESTRICT) rsum += dv;
        if (EMIT) g32[(p * n + i) * 4 + q] = (float)((double)dv * inv_s);
        if (ROUT) rout[i * 8 + c] = rscale * (double)dv;
      }
    }
    if (RESTRICT) {
      const int32_t fa = father[i];
      if (fa >= 0) {
        const int64_t pc = fa >> 3;
        const int cc = fa & 7;
        const int64_t o = ((int64_t)cell_parity(cc) * cn + pc) * 4 + (cc >> 1);
        cg[o] = T(0.5) * rsum;
        if (zero_cphi) cphi[((int64_t)cell_parity(cc) * cn_alloc + pc) * 4 + (cc >> 1)] = T(0);
      }
    }
  }
  if (NORM) block_sum_to(acc, partials);
}

// ----------------------------------------------------- interpolation

// Block index and child bit of the coarse cell at offset e - 1 (e = 0, 1, 2)
// along one axis from a father cell whose octant bit is cx; the block of 8
// coarse octs is displaced toward the father's octant.
__device__ __forceinline__ void axis_cell(int cx, int e, int &a, int &bit) {
  if (cx == 0) {
    a = (e == 0);
    bit = (e != 1);
  } else {
    a = (e == 2);
    bit = (e == 1);
  }
}

// Trilinear cell-centred interpolation of a coarse field onto the 8 children
// of the coarse cell (block octs b, octant cc): per axis weight 3/4 for the
// father, 1/4 for its neighbour toward the child.
template <typename T>
__device__ __forceinline__ void interp8(const T *__restrict__ cphi, int64_t cn_alloc, const int32_t b[8], int cc,
                                        T out[8]) {
  T v[27];
#pragma unroll
  for (int ez = 0; ez < 3; ++ez)
#pragma unroll
    for (int ey = 0; ey < 3; ++ey)
#pragma unroll
      for (int ex = 0; ex < 3; ++ex) {
        int ax, bx, ay, by, az, bz;
        axis_cell(cc & 1, ex, ax, bx);
        axis_cell((cc >> 1) & 1, ey, ay, by);
        axis_cell((cc >> 2) & 1, ez, az, bz);
        const int ch = bx | (by << 1) | (bz << 2);
        const int64_t oct = b[ax | (ay << 1) | (az << 2)];
        v[ex + 3 * ey + 9 * ez] = cphi[((int64_t)cell_parity(ch) * cn_alloc + oct) * 4 + (ch >> 1)];
      }
  const T w0 = T(0.75), w1 = T(0.25);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int fx = c & 1, fy = (c >> 1) & 1, fz = (c >> 2) & 1;
    const int ex1 = fx ? 2 : 0, ey1 = fy ? 2 : 0, ez1 = fz ? 2 : 0;
    T acc = w0 * w0 * w0 * v[1 + 3 * 1 + 9 * 1];
    acc = fma_t(w1 * w0 * w0, v[ex1 + 3 * 1 + 9 * 1], acc);
    acc = fma_t(w0 * w1 * w0, v[1 + 3 * ey1 + 9 * 1], acc);
    acc = fma_t(w1 * w1 * w0, v[ex1 + 3 * ey1 + 9 * 1], acc);
    acc = fma_t(w0 * w0 * w1, v[1 + 3 * 1 + 9 * ez1], acc);
    acc = fma_t(w1 * w0 * w1, v[ex1 + 3 * 1 + 9 * ez1], acc);
    acc = fma_t(w0 * w1 * w1, v[1 + 3 * ey1 + 9 * ez1], acc);
    acc = fma_t(w1 * w1 * w1, v[ex1 + 3 * ey1 + 9 * ez1], acc);
    out[c] = acc;
  }
}

template <typename T, bool MASK>
__global__ void __launch_bounds__(kThreads) k_prolong(const uint64_t *__restrict__ keys, const int32_t *__restrict__ blk,
                                                     int64_t n, int64_t n_alloc, T *__restrict__ phi,
                                                     const uint8_t *__restrict__ active,
                                                     const T *__restrict__ cphi, int64_t cn_alloc) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int cc = (int)(keys[i] & 7);
  int32_t b[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) b[t] = __ldg(blk + t * n + i);
  T corr[8];
  interp8(cphi, cn_alloc, b, cc, corr);
  const unsigned m = MASK ? active[i] : 0xFFu;
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    T v[4];
    load4(phi + (p * n_alloc + i) * 4, v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = plane_cell(p, q);
      if ((m >> c) & 1) v[q] += corr[c];
    }
    store4(phi + (p * n_alloc + i) * 4, v);
  }
}

__global__ void __launch_bounds__(kThreads) k_ghost_fill(const uint64_t *__restrict__ gkeys,
                                                        const int32_t *__restrict__ gblk,
                                                        const uint32_t *__restrict__ gmask, int64_t n_ghost,
                                                        int64_t n, int64_t n_alloc, double *__restrict__ phi,
                                                        const double *__restrict__ pphi, int64_t pn_alloc) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n_ghost) return;
  const int cc = (int)(gkeys[t] & 7);
  int32_t b[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) b[k] = __ldg(gblk + k * n_ghost + t);
  double val[8];
  interp8(pphi, pn_alloc, b, cc, val);
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
    store4(phi + (p * n_alloc + oct) * 4, v);
  }
}

// Ghost values in the [n][6][4] API layout (NaN where the neighbour exists).
__global__ void k_get_ghosts(const int32_t *__restrict__ nbr, int64_t n, int64_t n_ghost, int64_t n_alloc,
                             const double *__restrict__ phi, double *__restrict__ out) {
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
      out[(i * 6 + d) * 4 + q] =
          ghost ? phi[((int64_t)cell_parity(c2) * n_alloc + o) * 4 + (c2 >> 1)] : __longlong_as_double(0x7ff8000000000000ll);
      ++q;
    }
  }
}

// --------------------------------------------------------- coarsest solve

// Periodic 2^3 oct: eigenvectors (-1)^{k.b}, eigenvalues -4 |k|_1 / h^2;
// the mean (k = 0) is dropped.  Computed in FP64 whatever T is.
template <typename T>
__global__ void k_wht(const T *__restrict__ g, T *__restrict__ phi, int64_t n_alloc, double h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double f[8], fh[8];
  for (int c = 0; c < 8; ++c) f[c] = (double)g[cell_parity(c) * 4 + (c >> 1)] * (-6.0 / (h * h));
  for (int k = 0; k < 8; ++k) {
    double s = 0.0;
    for (int b = 0; b < 8; ++b) s += cell_parity(k & b) ? -f[b] : f[b];
    fh[k] = s * 0.125;
  }
  for (int b = 0; b < 8; ++b) {
    double s = 0.0;
    for (int k = 1; k < 8; ++k) {
      const int odd = (k & 1) + ((k >> 1) & 1) + ((k >> 2) & 1);
      const double x = fh[k] / (-4.0 * odd / (h * h));
      s += cell_parity(k & b) ? -x : x;
    }
    phi[(int64_t)cell_parity(b) * n_alloc * 4 + (b >> 1)] = (T)s;
  }
}

// ------------------------------------------------------------- misc

__global__ void k_set_density(const double *__restrict__ rho, int64_t n, double rho_bar, double scale,
                              double *__restrict__ g) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 8 * n) return;
  const int64_t i = t >> 3;
  const int c = (int)(t & 7);
  g[((int64_t)cell_parity(c) * n + i) * 4 + (c >> 1)] = scale * (rho[t] - rho_bar);
}

// oct-major [n][8] <-> planar [2][stride][4], with a scale factor
template <typename S, typename D>
__global__ void k_pack(const S *__restrict__ in, int64_t n, int64_t stride, double scale, D *__restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 8 * n) return;
  const int64_t i = t >> 3;
  const int c = (int)(t & 7);
  out[((int64_t)cell_parity(c) * stride + i) * 4 + (c >> 1)] = (D)(scale * (double)in[t]);
}

template <typename S, typename D>
__global__ void k_unpack(const S *__restrict__ in, int64_t n, int64_t stride, double scale, D *__restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 8 * n) return;
  const int64_t i = t >> 3;
  const int c = (int)(t & 7);
  out[t] = (D)(scale * (double)in[((int64_t)cell_parity(c) * stride + i) * 4 + (c >> 1)]);
}

__global__ void k_sum_phi(const double *__restrict__ phi, int64_t n, int64_t n_alloc, double *__restrict__ partials) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (i < n) {
    double a[4], b[4];
    load4(phi + i * 4, a);
    load4(phi + (n_alloc + i) * 4, b);
    acc = ((a[0] + a[1]) + (a[2] + a[3])) + ((b[0] + b[1]) + (b[2] + b[3]));
  }
  block_sum_to(acc, partials);
}

__global__ void k_sub_scalar(double *__restrict__ phi, int64_t n, int64_t n_alloc, const double *__restrict__ s) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 8 * n) return;
  const int64_t i = t >> 2 >> 1;
  const int p = (int)((t >> 2) & 1);
  const int q = (int)(t & 3);
  phi[(p * n_alloc + i) * 4 + q] -= *s;
}

// phi64 += S * phi32 on the real octs (solution accumulation, FP64)
__global__ void k_accumulate(double *__restrict__ phi, const float *__restrict__ e, int64_t n, int64_t n_alloc,
                             const double *__restrict__ scale) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 2 * n) return;
  const int p = (int)(t / n);
  const int64_t i = t - p * n;
  const double S = *scale;
  double v[4];
  float w[4];
  load4(phi + (p * n_alloc + i) * 4, v);
  load4(e + (p * n_alloc + i) * 4, w);
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = fma(S, (double)w[q], v[q]);
  store4(phi + (p * n_alloc + i) * 4, v);
}

// Sum partials in a fixed order; out = scale * sum (and, with root, its sqrt
// to out[1]).
__global__ void k_finalize(const double *__restrict__ partials, int np, double scale, double *__restrict__ out,
                           int with_sqrt) {
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
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < m) b[t] = (double)a[t];
}
__global__ void k_copy_convert_d2f(const double *__restrict__ a, float *__restrict__ b, int64_t m) {
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

// ------------------------------------------------------------ launchers
// Algorithmic work per launch (for the profile): bytes are the minimum
// traffic of the operation, flops its floating-point operations (FMA = 2).

template <typename T>
void sweep(cmg_level *L, int m, bool zero_init) {
  MgLev &g = L->mg[m];
  if (g.n == 0) return;
  cudaStream_t s = L->ctx->stream;
  T *phi = phi_of<T>(g);
  T *gg = g_of<T>(g);
  const int64_t st = g.n_alloc * 4;
  const unsigned nb = blocks_for(g.n);
  const bool mask = !g.all_active;
  const int cls = sizeof(T) == 8 ? K_SWEEP64 : K_SWEEP32;
  const double u = 4.0 * (double)g.n;  // cells updated per colour pass
  const double full_bytes = 3.0 * u * sizeof(T), full_flops = 7.0 * u;
#define CMG_SWEEP(P, Z, M)                                                                                  \
  do {                                                                                                      \
    LaunchScope ls(L->ctx, cls, (Z) ? 2.0 * u * sizeof(T) : full_bytes, (Z) ? 0.0 : full_flops);            \
    k_sweep<T, P, Z, M><<<nb, kThreads, 0, s>>>(g.nbr, phi + (1 - P) * st, phi + P * st, gg + P * g.n * 4, \
                                                g.active, g.n);                                             \
  } while (0)
  if (mask) {
    if (zero_init) CMG_SWEEP(0, true, true); else CMG_SWEEP(0, false, true);
    CMG_SWEEP(1, false, true);
  } else {
    if (zero_init) CMG_SWEEP(0, true, false); else CMG_SWEEP(0, false, false);
    CMG_SWEEP(1, false, false);
  }
#undef CMG_SWEEP
  CMG_CUDA(cudaGetLastError());
}
template void sweep<double>(cmg_level *, int, bool);
template void sweep<float>(cmg_level *, int, bool);

template <typename T>
void resid_restrict(cmg_level *L, int m, bool restrict_to_coarse, bool norm, bool zero_coarse_phi, double *norm_out,
                    const double *emit_scale) {
  MgLev &g = L->mg[m];
  cudaStream_t s = L->ctx->stream;
  const unsigned nb = blocks_for(g.n);
  MgLev *c = restrict_to_coarse ? &L->mg[m + 1] : nullptr;
  T *cg = c ? g_of<T>(*c) : nullptr;
  T *cphi = c ? phi_of<T>(*c) : nullptr;
  const int64_t cn = c ? c->n : 0, cna = c ? c->n_alloc : 0;
  const uint8_t *act = g.all_active ? nullptr : g.active;
  const double cells = 8.0 * (double)g.n;
  const double bytes = cells * 2.0 * sizeof(T) + (restrict_to_coarse ? g.n * sizeof(T) : 0.0) +
                       (emit_scale ? cells * 4.0 : 0.0);
  const double flops = cells * (8.0 + (norm ? 2.0 : 0.0) + (restrict_to_coarse ? 1.0 : 0.0));
  const int cls = sizeof(T) == 8 ? K_RESID64 : K_RESID32;
  if (g.n > 0) {
    LaunchScope ls(L->ctx, cls, bytes, flops);
    if (restrict_to_coarse && !norm && !emit_scale)
      k_resid<T, false, true, false, false, false><<<nb, kThreads, 0, s>>>(
          g.nbr, phi_of<T>(g), g_of<T>(g), act, g.n, g.n_alloc, g.father, cg, cphi, cn, cna, zero_coarse_phi,
          nullptr, nullptr, nullptr, nullptr, 0.0);
    else if (restrict_to_coarse && norm && !emit_scale)
      k_resid<T, true, true, false, false, false><<<nb, kThreads, 0, s>>>(
          g.nbr, phi_of<T>(g), g_of<T>(g), act, g.n, g.n_alloc, g.father, cg, cphi, cn, cna, zero_coarse_phi,
          L->partials, nullptr, nullptr, nullptr, 0.0);
    else if (!restrict_to_coarse && norm && !emit_scale)
      k_resid<T, true, false, false, false, false><<<nb, kThreads, 0, s>>>(
          g.nbr, phi_of<T>(g), g_of<T>(g), act, g.n, g.n_alloc, nullptr, nullptr, nullptr, 0, 0, 0, L->partials,
          nullptr, nullptr, nullptr, 0.0);
    else if (!restrict_to_coarse && norm && emit_scale)
      k_resid<T, true, false, true, false, false><<<nb, kThreads, 0, s>>>(
          g.nbr, phi_of<T>(g), g_of<T>(g), act, g.n, g.n_alloc, nullptr, nullptr, nullptr, 0, 0, 0, L->partials,
          g.g32, emit_scale, nullptr, 0.0);
    else
      throw Error(CMG_ERR_INVALID_ARG, "unsupported residual variant");
    CMG_CUDA(cudaGetLastError());
  }
  if (norm) {
    const double scale = 36.0 / (g.h * g.h * g.h * g.h);
    if (g.n == 0) {
      CMG_CUDA(cudaMemsetAsync(norm_out, 0, 2 * sizeof(double), s));
    } else {
      LaunchScope ls(L->ctx, K_REDUCE, nb * 8.0, nb);
      k_finalize<<<1, 1024, 0, s>>>(L->partials, (int)nb, scale, norm_out, 1);
      CMG_CUDA(cudaGetLastError());
    }
  }
}
template void resid_restrict<double>(cmg_level *, int, bool, bool, bool, double *, const double *);
template void resid_restrict<float>(cmg_level *, int, bool, bool, bool, double *, const double *);

void residual_out(cmg_level *L, int m, int prec, double *out) {
  MgLev &g = L->mg[m];
  if (g.n == 0) return;
  cudaStream_t s = L->ctx->stream;
  const uint8_t *act = g.all_active ? nullptr : g.active;
  const double rscale = -6.0 / (g.h * g.h);
  LaunchScope ls(L->ctx, prec == CMG_PREC_FP64 ? K_RESID64 : K_RESID32, 8.0 * g.n * 24.0, 8.0 * g.n * 9.0);
  if (prec == CMG_PREC_FP64)
    k_resid<double, false, false, false, true, false><<<blocks_for(g.n), kThreads, 0, s>>>(
        g.nbr, g.phi, g.g, act, g.n, g.n_alloc, nullptr, nullptr, nullptr, 0, 0, 0, nullptr, nullptr, nullptr, out,
        rscale);
  else
    k_resid<float, false, false, false, true, false><<<blocks_for(g.n), kThreads, 0, s>>>(
        g.nbr, g.phi32, g.g32, act, g.n, g.n_alloc, nullptr, nullptr, nullptr, 0, 0, 0, nullptr, nullptr, nullptr,
        out, rscale);
  CMG_CUDA(cudaGetLastError());
}

// ||f - L 0||^2 at level 0 (ghost forcing included) -> out[0], sqrt -> out[1]
void zero_phi_norm(cmg_level *L, double *out) {
  MgLev &g = L->mg[0];
  cudaStream_t s = L->ctx->stream;
  const unsigned nb = blocks_for(g.n);
  if (g.n == 0) {
    CMG_CUDA(cudaMemsetAsync(out, 0, 2 * sizeof(double), s));
    return;
  }
  {
    LaunchScope ls(L->ctx, K_RESID64, 8.0 * g.n * 8.0, 8.0 * g.n * 9.0);
    k_resid<double, true, false, false, false, true><<<nb, kThreads, 0, s>>>(
        g.nbr, g.phi, g.g, nullptr, g.n, g.n_alloc, nullptr, nullptr, nullptr, 0, 0, 0, L->partials, nullptr,
        nullptr, nullptr, 0.0);
  }
  {
    LaunchScope ls(L->ctx, K_REDUCE, nb * 8.0, nb);
    k_finalize<<<1, 1024, 0, s>>>(L->partials, (int)nb, 36.0 / (g.h * g.h * g.h * g.h), out, 1);
  }
  CMG_CUDA(cudaGetLastError());
}

template <typename T>
void prolong(cmg_level *L, int m) {
  MgLev &g = L->mg[m];
  MgLev &c = L->mg[m + 1];
  if (g.n == 0) return;
  cudaStream_t s = L->ctx->stream;
  LaunchScope ls(L->ctx, sizeof(T) == 8 ? K_PROLONG64 : K_PROLONG32,
                 g.n * 17.0 * sizeof(T), g.n * 128.0);
  if (g.all_active)
    k_prolong<T, false><<<blocks_for(g.n), kThreads, 0, s>>>(g.keys, g.blk, g.n, g.n_alloc, phi_of<T>(g), g.active,
                                                             phi_of<T>(c), c.n_alloc);
  else
    k_prolong<T, true><<<blocks_for(g.n), kThreads, 0, s>>>(g.keys, g.blk, g.n, g.n_alloc, phi_of<T>(g), g.active,
                                                            phi_of<T>(c), c.n_alloc);
  CMG_CUDA(cudaGetLastError());
}
template void prolong<double>(cmg_level *, int);
template void prolong<float>(cmg_level *, int);

void fill_ghosts(cmg_level *L) {
  MgLev &g = L->mg[0];
  if (!L->parent || g.n_ghost == 0) return;
  MgLev &pg = L->parent->mg[0];
  LaunchScope ls(L->ctx, K_GHOST, g.n_ghost * (64.0 + 8.0 + 32.0 + 4.0), g.n_ghost * 120.0);
  k_ghost_fill<<<blocks_for(g.n_ghost), kThreads, 0, L->ctx->stream>>>(
      L->ghost_keys, L->ghost_blk, L->ghost_mask, g.n_ghost, g.n, g.n_alloc, g.phi, pg.phi, pg.n_alloc);
  CMG_CUDA(cudaGetLastError());
}

void get_ghosts(cmg_level *L, double *out) {
  MgLev &g = L->mg[0];
  if (g.n == 0) return;
  LaunchScope ls(L->ctx, K_CONVERT, g.n * 24.0 * 8.0, 0.0);
  k_get_ghosts<<<blocks_for(g.n), kThreads, 0, L->ctx->stream>>>(g.nbr, g.n, g.n_ghost, g.n_alloc, g.phi, out);
  CMG_CUDA(cudaGetLastError());
}

void coarse_solve(cmg_level *L, int prec, int coarse_sweeps) {
  const int m = (int)L->mg.size() - 1;
  MgLev &g = L->mg[m];
  cudaStream_t s = L->ctx->stream;
  if (L->exact_coarse) {
    LaunchScope ls(L->ctx, K_COARSE, 128.0, 256.0);
    if (prec == CMG_PREC_FP64)
      k_wht<double><<<1, 32, 0, s>>>(g.g, g.phi, g.n_alloc, g.h);
    else
      k_wht<float><<<1, 32, 0, s>>>(g.g32, g.phi32, g.n_alloc, g.h);
    CMG_CUDA(cudaGetLastError());
    return;
  }
  if (prec == CMG_PREC_FP64) {
    for (int k = 0; k < coarse_sweeps; ++k) sweep<double>(L, m, k == 0 && m > 0);
    return;
  }
  // mixed: the coarsest level is solved in FP64 on FP64 copies
  const int64_t mg = 8 * g.n, ma = 8 * g.n_alloc;
  {
    LaunchScope ls(L->ctx, K_CONVERT, 12.0 * (mg + ma), 0.0);
    k_copy_convert_f2d<<<blocks_for(mg), kThreads, 0, s>>>(g.g32, g.g, mg);
  }
  {
    LaunchScope ls(L->ctx, K_CONVERT, 12.0 * ma, 0.0);
    k_copy_convert_f2d<<<blocks_for(ma), kThreads, 0, s>>>(g.phi32, g.phi, ma);
  }
  CMG_CUDA(cudaGetLastError());
  for (int k = 0; k < coarse_sweeps; ++k) sweep<double>(L, m, k == 0 && m > 0);
  {
    LaunchScope ls(L->ctx, K_CONVERT, 12.0 * ma, 0.0);
    k_copy_convert_d2f<<<blocks_for(ma), kThreads, 0, s>>>(g.phi, g.phi32, ma);
  }
  CMG_CUDA(cudaGetLastError());
}

void subtract_mean(cmg_level *L) {
  MgLev &g = L->mg[0];
  if (g.n == 0) return;
  cudaStream_t s = L->ctx->stream;
  const unsigned nb = blocks_for(g.n);
  {
    LaunchScope ls(L->ctx, K_REDUCE, 64.0 * g.n, 8.0 * g.n);
    k_sum_phi<<<nb, kThreads, 0, s>>>(g.phi, g.n, g.n_alloc, L->partials);
  }
  {
    LaunchScope ls(L->ctx, K_REDUCE, nb * 8.0, nb);
    k_finalize<<<1, 1024, 0, s>>>(L->partials, (int)nb, 1.0 / (8.0 * (double)g.n), L->scal + 6, 0);
  }
  {
    LaunchScope ls(L->ctx, K_CONVERT, 128.0 * g.n, 8.0 * g.n);
    k_sub_scalar<<<blocks_for(8 * g.n), kThreads, 0, s>>>(g.phi, g.n, g.n_alloc, L->scal + 6);
  }
  CMG_CUDA(cudaGetLastError());
}

void accumulate(cmg_level *L, const double *scale) {
  MgLev &g = L->mg[0];
  if (g.n == 0) return;
  LaunchScope ls(L->ctx, K_CONVERT, g.n * 8.0 * (16.0 + 4.0), g.n * 16.0);
  k_accumulate<<<blocks_for(2 * g.n), kThreads, 0, L->ctx->stream>>>(g.phi, g.phi32, g.n, g.n_alloc, scale);
  CMG_CUDA(cudaGetLastError());
}

void set_density(cmg_level *L, const double *rho, double rho_bar, double four_pi_g) {
  MgLev &g = L->mg[0];
  if (g.n == 0) return;
  const double scale = -g.h * g.h / 6.0 * four_pi_g;
  LaunchScope ls(L->ctx, K_CONVERT, g.n * 8.0 * 16.0, g.n * 16.0);
  k_set_density<<<blocks_for(8 * g.n), kThreads, 0, L->ctx->stream>>>(rho, g.n, rho_bar, scale, g.g);
  CMG_CUDA(cudaGetLastError());
}

void ensure_fp32(cmg_level *L) {
  if (L->has32) return;
  for (auto &g : L->mg) {
    g.phi32 = L->mem.alloc<float>(8 * g.n_alloc, true, L->ctx->stream);
    g.g32 = L->mem.alloc<float>(8 * g.n, true, L->ctx->stream);
  }
  L->has32 = true;
}

// field 0 = phi, 1 = f (stored as g = -h^2 f / 6)
void pack_field(cmg_level *L, int m, int field, int prec, const void *in) {
  MgLev &g = L->mg[m];
  if (g.n == 0) return;
  cudaStream_t s = L->ctx->stream;
  const double scale = field == 0 ? 1.0 : -g.h * g.h / 6.0;
  const int64_t stride = field == 0 ? g.n_alloc : g.n;
  const unsigned nb = blocks_for(8 * g.n);
  LaunchScope ls(L->ctx, K_CONVERT, g.n * 8.0 * 2.0 * (prec == CMG_PREC_FP64 ? 8.0 : 4.0), 0.0);
  if (prec == CMG_PREC_FP64)
    k_pack<double, double><<<nb, kThreads, 0, s>>>((const double *)in, g.n, stride, scale, field == 0 ? g.phi : g.g);
  else
    k_pack<float, float><<<nb, kThreads, 0, s>>>((const float *)in, g.n, stride, scale, field == 0 ? g.phi32 : g.g32);
  CMG_CUDA(cudaGetLastError());
}

void unpack_field(cmg_level *L, int m, int field, int prec, void *out) {
  MgLev &g = L->mg[m];
  if (g.n == 0) return;
  cudaStream_t s = L->ctx->stream;
  const double scale = field == 0 ? 1.0 : -6.0 / (g.h * g.h);
  const int64_t stride = field == 0 ? g.n_alloc : g.n;
  const unsigned nb = blocks_for(8 * g.n);
  LaunchScope ls(L->ctx, K_CONVERT, g.n * 8.0 * 2.0 * (prec == CMG_PREC_FP64 ? 8.0 : 4.0), 0.0);
  if (prec == CMG_PREC_FP64)
    k_unpack<double, double><<<nb, kThreads, 0, s>>>(field == 0 ? g.phi : g.g, g.n, stride, scale, (double *)out);
  else
    k_unpack<float, float><<<nb, kThreads, 0, s>>>(field == 0 ? g.phi32 : g.g32, g.n, stride, scale, (float *)out);
  CMG_CUDA(cudaGetLastError());
}

}  // namespace cmg
