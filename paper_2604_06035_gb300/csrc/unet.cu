// unet.cu -- the learned warm start: a 3-level 3-D U-Net (16/32/64 channels)
// mapping (rho, phi_prev) on a periodic D^3 block to the change of phi, with
// hand-written BF16 x BF16 -> FP32 tensor-core training and inference kernels.
// (No counterpart in the paper; the layer graph is listed in include/cmg.h.)
//
// Layout: activations are channels-last bf16 [B][D^3][C] (voxel v = (z D + y)
// D + x); conv weights are bf16 [Cout][27][Cin] for the forward pass and
// [Cin][27][Cout] for the input gradient, tap t = 9 (dz+1) + 3 (dy+1) + (dx+1);
// master parameters, gradients and Adam moments are FP32.
//
// Convolutions are implicit GEMMs on mma.sync m16n8k16 (bf16 in, fp32
// accumulate).  A block owns a 4x4x4 voxel brick: per 16-channel slice it
// stages the brick's 6x6x6 periodic halo (216 rows of 32 B) and the 27 taps of
// the weight slice in shared memory, and every tap's A fragment is an ldmatrix
// of halo rows shifted by the tap offset -- each input value is read from
// global memory once per slice instead of 27 times.  The weight gradient uses
// the same halo with ldmatrix.trans fragments and reduces over bricks.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

#include "cmg_internal.cuh"
#include "conv_tc.cuh"

namespace cmg {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kConvThreads = 128;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void mma16816(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ int wrap(int a, int D) { return a < 0 ? a + D : (a >= D ? a - D : a); }

// Global voxel row of halo cell (hz, hy, hx) (0..5) around brick (bz, by, bx).
__device__ __forceinline__ int64_t halo_row(int64_t sbase, int D, int bz, int by, int bx, int hz, int hy, int hx) {
  const int z = wrap(bz * 4 + hz - 1, D), y = wrap(by * 4 + hy - 1, D), x = wrap(bx * 4 + hx - 1, D);
  return sbase + ((int64_t)z * D + y) * D + x;
}

// out[v][n] = sum_t sum_k in[v + SIGN d_t][k] * W[n][t][k] (+ bias, ReLU).
// SIGN = +1: forward conv (W = [Cout][27][Cin]); SIGN = -1: input gradient
// (in = output gradient, W = [Cin][27][Cout]).  N = 8 NT output channels.
template <int NT, int SIGN, bool BIAS_RELU>
__global__ void __launch_bounds__(kConvThreads) k_conv(const bf16 *__restrict__ in, int K, const bf16 *__restrict__ W,
                                                      const float *__restrict__ bias, bf16 *__restrict__ out, int D) {
  extern __shared__ __align__(16) uint8_t smem[];
  constexpr int N = NT * 8;
  bf16 *halo = reinterpret_cast<bf16 *>(smem);  // [216][16]
  bf16 *wt = halo + 216 * 16;                   // [N][27][16]
  const int D4 = D >> 2;
  const int brick = blockIdx.x;
  const int bx = brick % D4, by = (brick / D4) % D4, bz = brick / (D4 * D4);
  const int64_t sbase = (int64_t)blockIdx.y * D * D * D;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  // A-fragment row of this lane: voxel m of the warp's 16 (z = warp)
  const int am = (lane & 7) + ((lane >> 3) & 1) * 8, akofs = (lane >> 4) * 8;
  const int ay = am >> 2, ax = am & 3;
  const int bn = (lane & 7) + ((lane >> 4) & 1) * 8, bkofs = ((lane >> 3) & 1) * 8;
  for (int kc = 0; kc < K / 16; ++kc) {
    for (int p = threadIdx.x; p < 432; p += kConvThreads) {
      const int row = p >> 1, half = p & 1;
      const int hz = row / 36, hy = (row / 6) % 6, hx = row % 6;
      const int64_t g = halo_row(sbase, D, bz, by, bx, hz, hy, hx);
      *reinterpret_cast<uint4 *>(halo + row * 16 + half * 8) =
          *reinterpret_cast<const uint4 *>(in + g * K + kc * 16 + half * 8);
    }
    for (int p = threadIdx.x; p < N * 27 * 2; p += kConvThreads) {
      const int r = p >> 1, half = p & 1;
      *reinterpret_cast<uint4 *>(wt + r * 16 + half * 8) =
          *reinterpret_cast<const uint4 *>(W + (int64_t)r * K + kc * 16 + half * 8);
    }
    __syncthreads();
#pragma unroll 1
    for (int t = 0; t < 27; ++t) {
      const int dz = SIGN * (t / 9 - 1), dy = SIGN * ((t / 3) % 3 - 1), dx = SIGN * (t % 3 - 1);
      const int hrow = ((warp + dz + 1) * 6 + (ay + dy + 1)) * 6 + (ax + dx + 1);
      uint32_t a0, a1, a2, a3;
      ldsm_x4(smem_u32(halo + hrow * 16 + akofs), a0, a1, a2, a3);
#pragma unroll
      for (int np = 0; np < NT / 2; ++np) {
        uint32_t b0, b1, b2, b3;
        ldsm_x4(smem_u32(wt + ((np * 16 + bn) * 27 + t) * 16 + bkofs), b0, b1, b2, b3);
        mma16816(acc[2 * np], a0, a1, a2, a3, b0, b1);
        mma16816(acc[2 * np + 1], a0, a1, a2, a3, b2, b3);
      }
    }
    __syncthreads();
  }
  const int g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int c0 = j * 8 + q * 2;
    float bv0 = 0.f, bv1 = 0.f;
    if (BIAS_RELU) {
      bv0 = bias[c0];
      bv1 = bias[c0 + 1];
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = g + h * 8;
      const int64_t v = sbase + ((int64_t)(bz * 4 + warp) * D + by * 4 + (m >> 2)) * D + bx * 4 + (m & 3);
      float x0 = acc[j][2 * h] + bv0, x1 = acc[j][2 * h + 1] + bv1;
      if (BIAS_RELU) {
        x0 = fmaxf(x0, 0.f);
        x1 = fmaxf(x1, 0.f);
      }
      *reinterpret_cast<__nv_bfloat162 *>(out + v * N + c0) = __floats2bfloat162_rn(x0, x1);
    }
  }
}

// dW[co][t][ci] += sum_v dout[v][co] * in[v + d_t][ci] over the bricks of
// this block, for the TG taps t0 = TG blockIdx.y ... t0 + TG - 1: each
// brick's 6x6x6 halo and output gradient are staged once and serve all TG
// taps.  A tile is (tap, 16 output channels, 16 input channels): two
// m16n8k16 accumulators; tiles go round-robin to the 8 warps.
constexpr int kWgThreads = 256;

template <int CIN, int COUT, int TG>
__global__ void __launch_bounds__(kWgThreads) k_conv_wgrad(const bf16 *__restrict__ dout, const bf16 *__restrict__ in,
                                                          float *__restrict__ dW, int D, int nbricks,
                                                          int bricks_per_block) {
  constexpr int NMB = COUT / 16, NJP = CIN / 16, TILES = TG * NMB * NJP, MAXT = (TILES + 7) / 8;
  extern __shared__ __align__(16) uint8_t smem[];
  bf16 *halo = reinterpret_cast<bf16 *>(smem);  // [216][CIN]
  bf16 *dt = halo + 216 * CIN;                  // [64][COUT]
  const int t0 = blockIdx.y * TG;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[MAXT][2][4];
#pragma unroll
  for (int i = 0; i < MAXT; ++i)
#pragma unroll
    for (int h = 0; h < 2; ++h) acc[i][h][0] = acc[i][h][1] = acc[i][h][2] = acc[i][h][3] = 0.f;
  const int D4 = D >> 2, per = D4 * D4 * D4;
  const int b_first = blockIdx.x * bricks_per_block;
  for (int bi = b_first; bi < b_first + bricks_per_block && bi < nbricks; ++bi) {
    const int s = bi / per, brick = bi % per;
    const int bx = brick % D4, by = (brick / D4) % D4, bz = brick / (D4 * D4);
    const int64_t sbase = (int64_t)s * D * D * D;
    for (int p = threadIdx.x; p < 216 * (CIN / 8); p += kWgThreads) {
      const int row = p / (CIN / 8), piece = p % (CIN / 8);
      const int hz = row / 36, hy = (row / 6) % 6, hx = row % 6;
      const int64_t g = halo_row(sbase, D, bz, by, bx, hz, hy, hx);
      *reinterpret_cast<uint4 *>(halo + row * CIN + piece * 8) =
          *reinterpret_cast<const uint4 *>(in + g * CIN + piece * 8);
    }
    for (int p = threadIdx.x; p < 64 * (COUT / 8); p += kWgThreads) {
      const int vi = p / (COUT / 8), piece = p % (COUT / 8);
      const int64_t v = sbase + ((int64_t)(bz * 4 + vi / 16) * D + by * 4 + (vi / 4) % 4) * D + bx * 4 + vi % 4;
      *reinterpret_cast<uint4 *>(dt + vi * COUT + piece * 8) =
          *reinterpret_cast<const uint4 *>(dout + v * COUT + piece * 8);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < MAXT; ++i) {
      const int tile = warp + 8 * i;
      if (tile < TILES) {
        const int tl = tile / (NMB * NJP), r = tile % (NMB * NJP), mb = r / NJP, jp = r % NJP;
        const int t = t0 + tl;
        const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
#pragma unroll
        for (int k16 = 0; k16 < 4; ++k16) {
          // A = dout^T (co x voxel) from dt [voxel][co] via ldmatrix.trans
          const int av = k16 * 16 + (lane & 7) + ((lane >> 4) & 1) * 8;
          const int aco = mb * 16 + ((lane >> 3) & 1) * 8;
          uint32_t a0, a1, a2, a3;
          ldsm_x4_t(smem_u32(dt + av * COUT + aco), a0, a1, a2, a3);
          // B = in shifted by the tap (voxel x ci) from halo rows via ldmatrix.trans
          const int bv = k16 * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
          const int hrow = ((bv / 16 + dz + 1) * 6 + ((bv / 4) % 4 + dy + 1)) * 6 + (bv % 4 + dx + 1);
          const int ci = jp * 16 + ((lane >> 4) & 1) * 8;
          uint32_t b0, b1, b2, b3;
          ldsm_x4_t(smem_u32(halo + hrow * CIN + ci), b0, b1, b2, b3);
          mma16816(acc[i][0], a0, a1, a2, a3, b0, b1);
          mma16816(acc[i][1], a0, a1, a2, a3, b2, b3);
        }
      }
    }
    __syncthreads();
  }
  const int g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int i = 0; i < MAXT; ++i) {
    const int tile = warp + 8 * i;
    if (tile >= TILES) continue;
    const int tl = tile / (NMB * NJP), r = tile % (NMB * NJP), mb = r / NJP, jp = r % NJP;
    const int t = t0 + tl;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int ci = (2 * jp + h) * 8 + q * 2;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int co = mb * 16 + g + hh * 8;
        float *dst = dW + ((int64_t)co * 27 + t) * CIN + ci;
        atomicAdd(dst, acc[i][h][2 * hh]);
        atomicAdd(dst + 1, acc[i][h][2 * hh + 1]);
      }
    }
  }
}

// ---- per-sample input statistics and the network input
// stats[b] = {sum rho, sum rho^2, sum phi^2}: per-thread FP32 partial sums,
// combined in FP64 (GB300's FP64 rate is a small fraction of FP32's)
__global__ void k_stats(const float *__restrict__ rho, const float *__restrict__ phi, int64_t V,
                        double *__restrict__ stats) {
  const int b = blockIdx.y;
  float f0 = 0.f, f1 = 0.f, f2 = 0.f;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    const float r = rho[b * V + v], p = phi[b * V + v];
    f0 += r;
    f1 = fmaf(r, r, f1);
    f2 = fmaf(p, p, f2);
  }
  double s0 = f0, s1 = f1, s2 = f2;
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(stats + 3 * b, s0);
    atomicAdd(stats + 3 * b + 1, s1);
    atomicAdd(stats + 3 * b + 2, s2);
  }
}

// norm[b] = {mean, 1/std, out_scale * rms}, plus 1/rms at norm_in[b] (one thread per sample)
__global__ void k_norm(const double *__restrict__ stats, int64_t V, int B, float out_scale, float *__restrict__ norm,
                       float *__restrict__ inv_rms) {
  const int b = threadIdx.x;
  if (b >= B) return;
  const double n = (double)V;
  const double mean = stats[3 * b] / n;
  const double var = fmax(stats[3 * b + 1] / n - mean * mean, 1e-300);
  const double rms = sqrt(stats[3 * b + 2] / n);
  norm[3 * b] = (float)mean;
  norm[3 * b + 1] = (float)(1.0 / sqrt(var));
  norm[3 * b + 2] = (float)(out_scale * rms);
  inv_rms[b] = (float)(1.0 / rms);
}

// x[b][v][0] = (rho - mean) / std, x[..][1] = phi / rms, channels 2..15 = 0
__global__ void k_input(const float *__restrict__ rho, const float *__restrict__ phi, int64_t V,
                        const float *__restrict__ norm, const float *__restrict__ inv_rms, bf16 *__restrict__ x) {
  const int b = blockIdx.y;
  const float mean = norm[3 * b], inv_std = norm[3 * b + 1], ir = inv_rms[b];
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    __align__(16) __nv_bfloat162 row[8];
    row[0] = __floats2bfloat162_rn((rho[b * V + v] - mean) * inv_std, phi[b * V + v] * ir);
#pragma unroll
    for (int c = 1; c < 8; ++c) row[c] = __floats2bfloat162_rn(0.f, 0.f);
    uint4 *dst = reinterpret_cast<uint4 *>(x + (b * V + v) * 16);
    dst[0] = reinterpret_cast<const uint4 *>(row)[0];
    dst[1] = reinterpret_cast<const uint4 *>(row)[1];
  }
}

// 2x2x2 mean pooling: in [B][D^3][C] -> out [B][(D/2)^3][C]
__global__ void k_pool(const bf16 *__restrict__ in, int D, int C, int B, bf16 *__restrict__ out) {
  const int Dh = D / 2;
  const int64_t total = (int64_t)B * Dh * Dh * Dh * C;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const int64_t u = e / C;
    const int64_t b = u / ((int64_t)Dh * Dh * Dh);
    const int64_t r = u % ((int64_t)Dh * Dh * Dh);
    const int z = (int)(r / (Dh * Dh)), y = (int)((r / Dh) % Dh), x = (int)(r % Dh);
    float s = 0.f;
    for (int k = 0; k < 8; ++k) {
      const int64_t v = b * D * D * D + ((int64_t)(2 * z + (k >> 2)) * D + 2 * y + ((k >> 1) & 1)) * D + 2 * x + (k & 1);
      s += __bfloat162float(in[v * C + c]);
    }
    out[e] = __float2bfloat16_rn(s * 0.125f);
  }
}

// out [B][D^3][Ca+Cb] = [nearest-upsampled a (D/2 grid, Ca), b (D grid, Cb)]
__global__ void k_up_concat(const bf16 *__restrict__ a, int Ca, const bf16 *__restrict__ b, int Cb, int D, int B,
                            bf16 *__restrict__ out) {
  const int C = Ca + Cb, Dh = D / 2;
  const int64_t total = (int64_t)B * D * D * D * C;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const int64_t v = e / C;
    const int64_t s = v / ((int64_t)D * D * D);
    const int64_t r = v % ((int64_t)D * D * D);
    if (c < Ca) {
      const int z = (int)(r / (D * D)), y = (int)((r / D) % D), x = (int)(r % D);
      const int64_t u = s * Dh * Dh * Dh + ((int64_t)(z >> 1) * Dh + (y >> 1)) * Dh + (x >> 1);
      out[e] = a[u * Ca + c];
    } else {
      out[e] = b[v * Cb + (c - Ca)];
    }
  }
}

// head: delta[v] = sum_c d0[v][c] w[c] + b; phi_pred = phi_prev + rms delta
__global__ void k_head(const bf16 *__restrict__ d0, const float *__restrict__ hw, const float *__restrict__ hb,
                       const float *__restrict__ phi_prev, const float *__restrict__ norm, int64_t V, int B,
                       float *__restrict__ delta, float *__restrict__ phi_pred) {
  const int64_t total = (int64_t)B * V;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    float s = hb[0];
#pragma unroll
    for (int c = 0; c < 16; ++c) s = fmaf(__bfloat162float(d0[e * 16 + c]), hw[c], s);
    if (delta) delta[e] = s;
    if (phi_pred) phi_pred[e] = phi_prev[e] + norm[3 * (e / V) + 2] * s;
  }
}

// loss = mean (delta - target)^2, target = (phi_next - phi_prev) / rms;
// ddelta = 2 (delta - target) / (B V); dact = bf16(ddelta w); head grads.
__global__ void k_head_grad(const bf16 *__restrict__ d0, const float *__restrict__ hw, const float *__restrict__ delta,
                            const float *__restrict__ phi_prev, const float *__restrict__ phi_next,
                            const float *__restrict__ norm, int64_t V, int B, bf16 *__restrict__ dact,
                            float *__restrict__ ghw, float *__restrict__ ghb, double *__restrict__ loss) {
  __shared__ float sh[17][32];
  const int64_t total = (int64_t)B * V;
  const float inv_n = 1.f / (float)total;
  float acc[17];
#pragma unroll
  for (int c = 0; c < 17; ++c) acc[c] = 0.f;
  double l = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const float target = (phi_next[e] - phi_prev[e]) / norm[3 * (e / V) + 2];
    const float diff = delta[e] - target;
    l += (double)diff * diff;
    const float dd = 2.f * diff * inv_n;
    acc[16] += dd;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      acc[c] = fmaf(__bfloat162float(d0[e * 16 + c]), dd, acc[c]);
      dact[e * 16 + c] = __float2bfloat16_rn(dd * hw[c]);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 17; ++c) {
    float v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[c][warp] = v;
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
  if (lane == 0) atomicAdd(loss, l);
  __syncthreads();
  if (threadIdx.x < 17) {
    float v = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[threadIdx.x][w];
    if (threadIdx.x < 16) atomicAdd(ghw + threadIdx.x, v); else atomicAdd(ghb, v);
  }
}

// g = bf16(g * (act > 0)) in place (ReLU derivative from the stored output)
__global__ void k_relu_mask(bf16 *__restrict__ g, const bf16 *__restrict__ act, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    if (!(__bfloat162float(act[e]) > 0.f)) g[e] = __float2bfloat16_rn(0.f);
}

// db[c] += sum_v g[v][c]
__global__ void k_bias_grad(const bf16 *__restrict__ g, int64_t rows, int C, float *__restrict__ db) {
  const int c = threadIdx.x % C;
  const int lanes = blockDim.x / C;
  const int r0 = threadIdx.x / C;
  float s = 0.f;
  for (int64_t r = blockIdx.x * (int64_t)lanes + r0; r < rows; r += (int64_t)gridDim.x * lanes)
    s += __bfloat162float(g[r * C + c]);
  if (r0 < lanes) atomicAdd(db + c, s);
}

// gradient split of a concat [up(a) (Ca), b (Cb)] on the D grid:
//   da[u][c] = bf16(sum over the 8 children of dcat[..][c]), c < Ca  (D/2 grid)
__global__ void k_up_grad(const bf16 *__restrict__ dcat, int Ca, int Cb, int D, int B, bf16 *__restrict__ da) {
  const int C = Ca + Cb, Dh = D / 2;
  const int64_t total = (int64_t)B * Dh * Dh * Dh * Ca;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % Ca);
    const int64_t u = e / Ca;
    const int64_t s = u / ((int64_t)Dh * Dh * Dh), r = u % ((int64_t)Dh * Dh * Dh);
    const int z = (int)(r / (Dh * Dh)), y = (int)((r / Dh) % Dh), x = (int)(r % Dh);
    float acc = 0.f;
    for (int k = 0; k < 8; ++k) {
      const int64_t v = s * D * D * D + ((int64_t)(2 * z + (k >> 2)) * D + 2 * y + ((k >> 1) & 1)) * D + 2 * x + (k & 1);
      acc += __bfloat162float(dcat[v * C + c]);
    }
    da[e] = __float2bfloat16_rn(acc);
  }
}

// skip gradient: ds[v][c] = bf16(dcat[v][Ca + c] + dpool[parent(v)][c] / 8)
__global__ void k_skip_grad(const bf16 *__restrict__ dcat, int Ca, int Cb, const bf16 *__restrict__ dpool, int D,
                            int B, bf16 *__restrict__ ds) {
  const int C = Ca + Cb, Dh = D / 2;
  const int64_t total = (int64_t)B * D * D * D * Cb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % Cb);
    const int64_t v = e / Cb;
    const int64_t s = v / ((int64_t)D * D * D), r = v % ((int64_t)D * D * D);
    const int z = (int)(r / (D * D)), y = (int)((r / D) % D), x = (int)(r % D);
    const int64_t u = s * Dh * Dh * Dh + ((int64_t)(z >> 1) * Dh + (y >> 1)) * Dh + (x >> 1);
    ds[e] = __float2bfloat16_rn(__bfloat162float(dcat[v * C + Ca + c]) + __bfloat162float(dpool[u * Cb + c]) * 0.125f);
  }
}

// Sum of squares of the gradient into clip[0] (block sums, one atomic each).
__global__ void k_grad_sq(const float *__restrict__ g, int64_t n, double *__restrict__ clip) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)g[i] * (double)g[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
  __shared__ double ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    atomicAdd(clip, t);
  }
}

// The clipping scale of this step: the gradient's 2-norm is capped at k times
// the running mean of the earlier steps' (capped) norms, once 20 steps have
// formed that mean; the mean then takes the capped norm.  Resets the sum.
__global__ void k_clip_scale(double *clip, float k) {
  const double norm = sqrt(clip[0]);
  const double mean = clip[1], seen = clip[2];
  double scale = 1.0, kept = norm;
  if (seen >= 20.0 && norm > k * mean && norm > 0.0) {
    scale = k * mean / norm;
    kept = k * mean;
    clip[4] += 1.0;
  }
  clip[1] = seen == 0.0 ? kept : 0.95 * mean + 0.05 * kept;
  clip[2] = seen + 1.0;
  clip[3] = scale;
  clip[5] = norm;
  clip[0] = 0.0;
}

// Adam on the FP32 master parameters; with clip, the gradient is scaled by
// clip[3] first.
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2,
                       const double *__restrict__ clip) {
  const float gs = clip ? (float)clip[3] : 1.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i] * gs;
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// bf16 weight copies: W [co][t][ci] and WT [ci][t][co] from the master slice
__global__ void k_cast_w(const float *__restrict__ w, int co_n, int ci_n, bf16 *__restrict__ W, bf16 *__restrict__ WT) {
  const int64_t n = (int64_t)co_n * 27 * ci_n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int ci = (int)(e % ci_n);
    const int t = (int)((e / ci_n) % 27);
    const int co = (int)(e / (27 * ci_n));
    const bf16 x = __float2bfloat16_rn(w[e]);
    W[e] = x;
    WT[((int64_t)ci * 27 + t) * co_n + co] = x;
  }
}

// dense [B][D^3] (z, y, x) <-> oct-major [n][8] of a full periodic level whose
// octs are listed x fastest (child c = bx + 2 by + 4 bz)
__global__ void k_dense_octs(const double *__restrict__ src, int D, int64_t n, double *__restrict__ dst, int to_octs) {
  const int Do = D / 2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 8 * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = e >> 3;
    const int c = (int)(e & 7);
    const int ox = (int)(o % Do), oy = (int)((o / Do) % Do), oz = (int)(o / ((int64_t)Do * Do));
    const int64_t v = ((int64_t)(2 * oz + ((c >> 2) & 1)) * D + 2 * oy + ((c >> 1) & 1)) * D + 2 * ox + (c & 1);
    if (to_octs) dst[e] = src[v]; else dst[v] = src[e];
  }
}

unsigned gsz(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 4096); }

}  // namespace
}  // namespace cmg

// ----------------------------------------------------------------- network

namespace {

struct LayerSpec {
  const char *name;
  int cin, cout, lvl;
};
constexpr LayerSpec kLayers[10] = {{"enc0a", 16, 16, 0}, {"enc0b", 16, 16, 0}, {"enc1a", 16, 32, 1},
                                   {"enc1b", 32, 32, 1}, {"bota", 32, 64, 2},  {"botb", 64, 64, 2},
                                   {"dec1a", 96, 32, 1}, {"dec1b", 32, 32, 1}, {"dec0a", 48, 16, 0},
                                   {"dec0b", 16, 16, 0}};

int64_t layer_offset(int l) {
  int64_t o = 0;
  for (int k = 0; k < l; ++k) o += (int64_t)kLayers[k].cout * 27 * kLayers[k].cin + kLayers[k].cout;
  return o;
}
int64_t total_params() { return layer_offset(10) + 17; }

}  // namespace

struct cmg_unet {
  cmg_ctx *ctx = nullptr;
  int D = 0, max_batch = 0;
  int64_t np = 0;
  float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *W[10] = {}, *WT[10] = {};
  // the same weights arranged for the tcgen05 kernels (conv_tc.cuh)
  __nv_bfloat16 *WI[10] = {}, *WTI[10] = {};
  int *d_err = nullptr;  // device status word of the bounded waits
  bool use_tc = true;    // tcgen05 convolutions where the grid allows
  // activations (bf16) and their gradients, per batch sample
  __nv_bfloat16 *x = nullptr, *a[10] = {}, *p0 = nullptr, *p1 = nullptr, *c1 = nullptr, *c0 = nullptr;
  __nv_bfloat16 *g0 = nullptr, *g1 = nullptr, *gc = nullptr, *gx = nullptr, *gs0 = nullptr, *gs1 = nullptr;
  __nv_bfloat16 *gp = nullptr, *gu = nullptr;
  float *delta = nullptr, *norm = nullptr;
  double *stats = nullptr, *loss = nullptr;
  // inputs: rho, field (its rms scales the output), base (the output is
  // base + rms(field) delta), target (training); out = the prediction
  float *in_rho = nullptr, *in_phi = nullptr, *in_base = nullptr, *in_next = nullptr, *out_phi = nullptr;
  // the prediction is base + out_scale * rms(field) * delta
  float out_scale = 1.f;
  int adam_t = 0;
  // gradient-norm clipping (cmg_unet_set_grad_clip): clip_k = 0 off; clip on
  // the device: [0] sum of squares of the step's gradient, [1] running mean
  // of the (clipped) norm, [2] steps seen, [3] scale applied, [4] steps
  // clipped, [5] last norm
  float clip_k = 0.f;
  double *clip = nullptr;
  bool weights_ready = false;
  cmg::DeviceBuffers mem;
};

namespace cmg {
namespace {

using bf16 = __nv_bfloat16;

template <int N, int ZB, bool FWD>
void conv_tc_launch(cmg_unet *U, const bf16 *in, int K, const bf16 *skip, int Cb, const bf16 *WI, const float *bias,
                    bf16 *out, int D, int B, const tc::ConvEpi &ep) {
  using G = tc::ConvGeom<N, ZB>;
  static int attr_dev = -1;
  if (attr_dev != U->ctx->device) {
    CMG_CUDA(cudaFuncSetAttribute(tc::k_conv_tc<N, ZB, FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  227 * 1024));
    attr_dev = U->ctx->device;
  }
  const int total = (D / 8) * (D / 16) * (D / ZB) * B;
  const int grid = std::min(total, U->ctx->num_sms);
  LaunchScope ls(U->ctx, FWD ? K_CONV_FWD : K_CONV_DGRAD, 0.0, 2.0 * 27 * K * N * (double)D * D * D * B);
  tc::k_conv_tc<N, ZB, FWD><<<grid, tc::kConvThreads, G::smem_bytes(K), U->ctx->stream>>>(in, K, skip, Cb, WI, bias, out,
                                                                                     D, total, U->d_err, ep);
  CMG_CUDA(cudaGetLastError());
}

template <int NT, int SIGN, bool BR>
void conv_launch(cmg_unet *U, const bf16 *in, int K, const bf16 *W, const float *bias, bf16 *out, int D, int B) {
  const size_t smem = (216 * 16 + (size_t)NT * 8 * 27 * 16) * sizeof(bf16);
  static bool attr = false;
  if (!attr) {
    CMG_CUDA(cudaFuncSetAttribute(k_conv<NT, SIGN, BR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
    attr = true;
  }
  const int nb = (D / 4) * (D / 4) * (D / 4);
  LaunchScope ls(U->ctx, SIGN > 0 ? K_CONV_FWD : K_CONV_DGRAD, 0.0, 2.0 * 27 * K * NT * 8 * (double)D * D * D * B);
  k_conv<NT, SIGN, BR><<<dim3(nb, B), kConvThreads, smem, U->ctx->stream>>>(in, K, W, bias, out, D);
  CMG_CUDA(cudaGetLastError());
}

// The tcgen05 path needs bricks of 8 x 16 x ZB voxels: D a multiple of 16.
bool tc_eligible(const cmg_unet *U, int N, int D) {
  return U->use_tc && D >= 16 && D % 16 == 0 && (N == 16 || N == 32 || N == 48 || N == 64 || N == 96);
}

// Deep bricks (ZB = 8 for N = 16, 4 for N = 32, 2 above) when they still
// give every SM a brick, else one-slice bricks.  The epilogue extras need
// N <= 32 (head: N = 16), and the pooling also needs the deep (even) ZB:
// returns whether ep.pool was done (else the caller pools separately).
bool conv_tc(cmg_unet *U, const bf16 *in, int K, const bf16 *skip, int Cb, const bf16 *WI, const float *bias,
             bf16 *out, int N, int D, int B, bool fwd, tc::ConvEpi ep = tc::ConvEpi()) {
  const int zb = N == 16 ? 8 : N == 32 ? 4 : 2;
  const bool deep = (D / 8) * (D / 16) * (D / zb) * B >= U->ctx->num_sms;
  const bool pooled = ep.pool != nullptr && deep && N <= 32;
  tc::ConvEpi e = ep;
  if (!pooled) e.pool = nullptr;
#define CMG_CONV_TC(NN, ZB)                                                                           \
  case NN:                                                                                            \
    if (deep) {                                                                                       \
      if (fwd) conv_tc_launch<NN, ZB, true>(U, in, K, skip, Cb, WI, bias, out, D, B, e);              \
      else conv_tc_launch<NN, ZB, false>(U, in, K, nullptr, 0, WI, nullptr, out, D, B, e);            \
    } else {                                                                                          \
      if (fwd) conv_tc_launch<NN, 1, true>(U, in, K, skip, Cb, WI, bias, out, D, B, e);               \
      else conv_tc_launch<NN, 1, false>(U, in, K, nullptr, 0, WI, nullptr, out, D, B, e);             \
    }                                                                                                 \
    break;
  switch (N) {
    CMG_CONV_TC(16, 8)
    CMG_CONV_TC(32, 4)
    CMG_CONV_TC(48, 2)
    CMG_CONV_TC(64, 2)
    CMG_CONV_TC(96, 2)
    default: throw Error(CMG_ERR_INVALID_ARG, "unsupported channel count");
  }
#undef CMG_CONV_TC
  return pooled;
}

// Convolution of layer l: forward (in = activations, N = cout) or input
// gradient (in = output gradient, N = cin).
void conv(cmg_unet *U, int l, const bf16 *in, int K, const float *bias, bf16 *out, int N, int D, int B, bool fwd) {
  if (tc_eligible(U, N, D)) {
    conv_tc(U, in, K, nullptr, 0, fwd ? U->WI[l] : U->WTI[l], bias, out, N, D, B, fwd);
    return;
  }
  const bf16 *W = fwd ? U->W[l] : U->WT[l];
#define CMG_CONV(NT)                                                             \
  case NT:                                                                       \
    if (fwd) conv_launch<NT, 1, true>(U, in, K, W, bias, out, D, B);             \
    else conv_launch<NT, -1, false>(U, in, K, W, nullptr, out, D, B);            \
    break;
  switch (N / 8) {
    CMG_CONV(2)
    CMG_CONV(4)
    CMG_CONV(6)
    CMG_CONV(8)
    CMG_CONV(12)
    default: throw Error(CMG_ERR_INVALID_ARG, "unsupported channel count");
  }
#undef CMG_CONV
}

template <int CIN, int COUT, int TG>
void wgrad_launch(cmg_unet *U, const bf16 *dout, const bf16 *in, float *dW, int D, int B) {
  const size_t smem = ((size_t)216 * CIN + 64 * (size_t)COUT) * sizeof(bf16);
  static int attr_dev = -1;
  if (attr_dev != U->ctx->device) {
    CMG_CUDA(cudaFuncSetAttribute(k_conv_wgrad<CIN, COUT, TG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    attr_dev = U->ctx->device;
  }
  const int nbricks = B * (D / 4) * (D / 4) * (D / 4);
  const int gy = 27 / TG;
  const int bx = std::max(1, std::min(nbricks, 4 * U->ctx->num_sms / gy));
  const int per_block = (nbricks + bx - 1) / bx;
  const int blocks = (nbricks + per_block - 1) / per_block;
  LaunchScope ls(U->ctx, K_CONV_WGRAD, 0.0, 2.0 * 27 * COUT * CIN * (double)D * D * D * B);
  k_conv_wgrad<CIN, COUT, TG><<<dim3(blocks, gy), kWgThreads, smem, U->ctx->stream>>>(dout, in, dW, D, nbricks,
                                                                                     per_block);
  CMG_CUDA(cudaGetLastError());
}

// Taps per block: as many (27, 9 or 3) as keep the accumulators of a warp
// within 12 tiles (96 registers).
void wgrad(cmg_unet *U, const bf16 *dout, int Cout, const bf16 *in, int Cin, float *dW, int D, int B) {
#define CMG_WG(CI, CO, TG)                                      \
  if (Cin == CI && Cout == CO) {                                \
    wgrad_launch<CI, CO, TG>(U, dout, in, dW, D, B);            \
    return;                                                     \
  }
  CMG_WG(16, 16, 27)
  CMG_WG(16, 32, 27)
  CMG_WG(32, 32, 9)
  CMG_WG(32, 64, 9)
  CMG_WG(64, 64, 3)
  CMG_WG(96, 32, 3)
  CMG_WG(48, 16, 27)
#undef CMG_WG
  throw Error(CMG_ERR_INVALID_ARG, "unsupported channel count");
}

// After a synchronisation: a bounded wait that expired in a tcgen05
// convolution is reported (and the status word cleared).
void check_status(cmg_unet *U) {
  int e = 0;
  CMG_CUDA(cudaMemcpy(&e, U->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e != 0) {
    CMG_CUDA(cudaMemset(U->d_err, 0, sizeof(int)));
    throw Error(e, "U-Net convolution: a bounded wait expired (tensor-core pipeline stalled)");
  }
}

int dim_of(const cmg_unet *U, int lvl) { return U->D >> lvl; }
int64_t vox(const cmg_unet *U, int lvl) {
  const int64_t d = dim_of(U, lvl);
  return d * d * d;
}

void prepare_weights(cmg_unet *U) {
  if (U->weights_ready) return;
  cudaStream_t s = U->ctx->stream;
  for (int l = 0; l < 10; ++l) {
    const LayerSpec &L = kLayers[l];
    const int64_t n = (int64_t)L.cout * 27 * L.cin;
    k_cast_w<<<gsz(n), 256, 0, s>>>(U->params + layer_offset(l), L.cout, L.cin, U->W[l], U->WT[l]);
    tc::k_weight_image<<<gsz(n), 256, 0, s>>>(U->W[l], L.cout, L.cin, 1, U->WI[l]);
    tc::k_weight_image<<<gsz(n), 256, 0, s>>>(U->WT[l], L.cin, L.cout, -1, U->WTI[l]);
  }
  CMG_CUDA(cudaGetLastError());
  U->weights_ready = true;
}

const float *bias_of(cmg_unet *U, int l) {
  return U->params + layer_offset(l) + (int64_t)kLayers[l].cout * 27 * kLayers[l].cin;
}

// Forward pass on U->in_rho / U->in_phi (B samples); leaves activations,
// delta and (if phi_pred) phi_prev + rms * delta.
void forward(cmg_unet *U, int B, float *phi_pred, bool training) {
  cudaStream_t s = U->ctx->stream;
  prepare_weights(U);
  const int64_t V0 = vox(U, 0);
  CMG_CUDA(cudaMemsetAsync(U->stats, 0, sizeof(double) * 3 * B, s));
  k_stats<<<dim3(64, B), 256, 0, s>>>(U->in_rho, U->in_phi, V0, U->stats);
  k_norm<<<1, (B + 31) / 32 * 32, 0, s>>>(U->stats, V0, B, U->out_scale, U->norm, U->norm + 3 * U->max_batch);
  k_input<<<dim3(gsz(V0), B), 256, 0, s>>>(U->in_rho, U->in_phi, V0, U->norm, U->norm + 3 * U->max_batch, U->x);
  CMG_CUDA(cudaGetLastError());
  const int D0 = dim_of(U, 0), D1 = dim_of(U, 1), D2 = dim_of(U, 2);
  auto layer = [&](int l, const bf16 *in, bf16 *out) {
    const LayerSpec &L = kLayers[l];
    conv(U, l, in, L.cin, bias_of(U, l), out, L.cout, dim_of(U, L.lvl), B, true);
  };
  // encoder convolution + 2x2x2 pooling (fused into the tcgen05 epilogue
  // where the bricks allow it)
  auto layer_pool = [&](int l, const bf16 *in, bf16 *out, bf16 *pooled) {
    const LayerSpec &L = kLayers[l];
    const int D = dim_of(U, L.lvl);
    bool done = false;
    if (tc_eligible(U, L.cout, D)) {
      tc::ConvEpi ep;
      ep.pool = pooled;
      done = conv_tc(U, in, L.cin, nullptr, 0, U->WI[l], bias_of(U, l), out, L.cout, D, B, true, ep);
    } else {
      layer(l, in, out);
    }
    if (!done) k_pool<<<gsz(B * (int64_t)(D / 2) * (D / 2) * (D / 2) * L.cout), 256, 0, s>>>(out, D, L.cout, B, pooled);
  };
  layer(0, U->x, U->a[0]);
  layer_pool(1, U->a[0], U->a[1], U->p0);  // s0
  layer(2, U->p0, U->a[2]);
  layer_pool(3, U->a[2], U->a[3], U->p1);  // s1
  layer(4, U->p1, U->a[4]);
  layer(5, U->a[4], U->a[5]);
  // decoder convolutions: in inference the tcgen05 kernels read the
  // upsampled coarse map and the skip map directly; training keeps the
  // concatenation (the backward pass needs it)
  auto up_layer = [&](int l, const bf16 *coarse, int Ca, const bf16 *skipm, int Cb, bf16 *cat, bf16 *out) {
    const LayerSpec &L = kLayers[l];
    const int D = dim_of(U, L.lvl);
    if (!training && tc_eligible(U, L.cout, D)) {
      conv_tc(U, coarse, Ca + Cb, skipm, Cb, U->WI[l], bias_of(U, l), out, L.cout, D, B, true);
      return;
    }
    k_up_concat<<<gsz(B * (int64_t)D * D * D * (Ca + Cb)), 256, 0, s>>>(coarse, Ca, skipm, Cb, D, B, cat);
    layer(l, cat, out);
  };
  up_layer(6, U->a[5], 64, U->a[3], 32, U->c1, U->a[6]);
  layer(7, U->a[6], U->a[7]);
  up_layer(8, U->a[7], 32, U->a[1], 16, U->c0, U->a[8]);
  const float *hw = U->params + layer_offset(10);
  if (!training && tc_eligible(U, 16, D0)) {
    // last convolution + head in one kernel; its activations are not kept
    tc::ConvEpi ep;
    ep.hw = hw;
    ep.base = U->in_base;
    ep.norm = U->norm;
    ep.delta = U->delta;
    ep.pred = phi_pred;
    ep.store_out = 0;
    conv_tc(U, U->a[8], 16, nullptr, 0, U->WI[9], bias_of(U, 9), U->a[9], 16, D0, B, true, ep);
  } else {
    layer(9, U->a[8], U->a[9]);
    k_head<<<gsz(B * V0), 256, 0, s>>>(U->a[9], hw, hw + 16, U->in_base, U->norm, V0, B, U->delta, phi_pred);
  }
  CMG_CUDA(cudaGetLastError());
  (void)D2;
}

// Backward pass after forward(): gradients (summed over the batch's voxels,
// loss = mean over all voxels) into U->grads; loss into U->loss.
void backward(cmg_unet *U, int B) {
  cudaStream_t s = U->ctx->stream;
  const int64_t V0 = vox(U, 0), V1 = vox(U, 1), V2 = vox(U, 2);
  const int D0 = dim_of(U, 0), D1 = dim_of(U, 1), D2 = dim_of(U, 2);
  CMG_CUDA(cudaMemsetAsync(U->grads, 0, sizeof(float) * U->np, s));
  CMG_CUDA(cudaMemsetAsync(U->loss, 0, sizeof(double), s));
  float *ghw = U->grads + layer_offset(10);
  k_head_grad<<<gsz(B * V0), 256, 0, s>>>(U->a[9], U->params + layer_offset(10), U->delta, U->in_base, U->in_next,
                                          U->norm, V0, B, U->g0, ghw, ghw + 16, U->loss);
  CMG_CUDA(cudaGetLastError());
  // back through layer l: g (grad of its output, bf16) -> grad of its input
  auto back = [&](int l, bf16 *g, const bf16 *in, bf16 *gin) {
    const LayerSpec &L = kLayers[l];
    const int D = dim_of(U, L.lvl);
    const int64_t rows = (int64_t)B * vox(U, L.lvl);
    k_relu_mask<<<gsz(rows * L.cout), 256, 0, s>>>(g, U->a[l], rows * L.cout);
    float *gw = U->grads + layer_offset(l);
    k_bias_grad<<<256, 256, 0, s>>>(g, rows, L.cout, gw + (int64_t)L.cout * 27 * L.cin);
    CMG_CUDA(cudaGetLastError());
    wgrad(U, g, L.cout, in, L.cin, gw, D, B);
    if (gin) conv(U, l, g, L.cout, nullptr, gin, L.cin, D, B, false);
  };
  // decoder level 0
  back(9, U->g0, U->a[8], U->g1);            // g1 = grad a8 (16 ch, V0)
  back(8, U->g1, U->c0, U->gc);              // gc = grad c0 (48 ch, V0)
  k_up_grad<<<gsz(B * V1 * 32), 256, 0, s>>>(U->gc, 32, 16, D0, B, U->gu);  // grad a7 (32 ch, V1)
  // decoder level 1
  back(7, U->gu, U->a[6], U->gx);            // gx = grad a6 (32 ch, V1)
  back(6, U->gx, U->c1, U->g0);              // g0 reused: grad c1 (96 ch, V1)
  k_up_grad<<<gsz(B * V2 * 64), 256, 0, s>>>(U->g0, 64, 32, D1, B, U->gu);  // grad a5 (64 ch, V2)
  // bottleneck
  back(5, U->gu, U->a[4], U->gx);            // grad a4 (64, V2)
  back(4, U->gx, U->p1, U->gp);              // grad p1 (32, V2)
  k_skip_grad<<<gsz(B * V1 * 32), 256, 0, s>>>(U->g0, 64, 32, U->gp, D1, B, U->gs1);  // grad s1 = a3
  // encoder level 1
  back(3, U->gs1, U->a[2], U->gx);           // grad a2 (32, V1)
  back(2, U->gx, U->p0, U->gp);              // grad p0 (16, V1)
  k_skip_grad<<<gsz(B * V0 * 16), 256, 0, s>>>(U->gc, 32, 16, U->gp, D0, B, U->gs0);  // grad s0 = a1
  // encoder level 0
  back(1, U->gs0, U->a[0], U->g1);           // grad a0 (16, V0)
  back(0, U->g1, U->x, nullptr);
  CMG_CUDA(cudaGetLastError());
  (void)D2;
}

void copy_in(cmg_unet *U, float *dst, const float *src, int64_t n, int mem) {
  CMG_CUDA(cudaMemcpyAsync(dst, src, sizeof(float) * n,
                           mem == CMG_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, U->ctx->stream));
}

}  // namespace
}  // namespace cmg

// ------------------------------------------------------------------ C ABI

namespace {
template <class F>
int unet_guard(F &&f) {
  try {
    cmg::record_error("");
    return f();
  } catch (const cmg::Error &e) {
    cmg::record_error(e.what());
    return e.code;
  } catch (const std::exception &e) {
    cmg::record_error(e.what());
    return CMG_ERR_CUDA;
  }
}
}  // namespace

extern "C" {

int cmg_unet_create(cmg_ctx *ctx, int grid_dim, int max_batch, cmg_unet **out) {
  return unet_guard([&] {
    if (!out || !ctx || grid_dim < 16 || grid_dim % 16 || max_batch < 1) return (int)CMG_ERR_INVALID_ARG;
    *out = nullptr;
    cudaSetDevice(ctx->device);
    auto *U = new cmg_unet();
    try {
      U->ctx = ctx;
      U->D = grid_dim;
      U->max_batch = max_batch;
      U->np = total_params();
      cudaStream_t s = ctx->stream;
      auto &M = U->mem;
      U->params = M.alloc<float>(U->np, true, s);
      U->grads = M.alloc<float>(U->np, true, s);
      U->m = M.alloc<float>(U->np, true, s);
      U->v = M.alloc<float>(U->np, true, s);
      U->clip = M.alloc<double>(8, true, s);
      for (int l = 0; l < 10; ++l) {
        const int64_t n = (int64_t)kLayers[l].cout * 27 * kLayers[l].cin;
        U->W[l] = reinterpret_cast<__nv_bfloat16 *>(M.alloc<uint16_t>(n));
        U->WT[l] = reinterpret_cast<__nv_bfloat16 *>(M.alloc<uint16_t>(n));
        U->WI[l] = reinterpret_cast<__nv_bfloat16 *>(M.alloc<uint16_t>(n));
        U->WTI[l] = reinterpret_cast<__nv_bfloat16 *>(M.alloc<uint16_t>(n));
      }
      const int64_t B = max_batch;
      const int64_t V0 = (int64_t)grid_dim * grid_dim * grid_dim, V1 = V0 / 8, V2 = V0 / 64;
      auto act = [&](int64_t n) { return reinterpret_cast<__nv_bfloat16 *>(M.alloc<uint16_t>(n)); };
      U->x = act(B * V0 * 16);
      const int64_t vox_of[3] = {V0, V1, V2};
      for (int l = 0; l < 10; ++l) U->a[l] = act(B * vox_of[kLayers[l].lvl] * kLayers[l].cout);
      U->p0 = act(B * V1 * 16);
      U->p1 = act(B * V2 * 32);
      U->c1 = act(B * V1 * 96);
      U->c0 = act(B * V0 * 48);
      const int64_t big = B * std::max(V0 * 48, V1 * 96);
      U->g0 = act(big);
      U->g1 = act(B * V0 * 16);
      U->gc = act(B * V0 * 48);
      U->gx = act(B * std::max(V1 * 32, V2 * 64));
      U->gs0 = act(B * V0 * 16);
      U->gs1 = act(B * V1 * 32);
      U->gp = act(B * std::max(V1 * 16, V2 * 32));
      U->gu = act(B * std::max(V1 * 32, V2 * 64));
      U->delta = M.alloc<float>(B * V0);
      U->norm = M.alloc<float>(4 * B);  // {mean, 1/std, c rms} per sample, then 1/rms per sample
      U->stats = M.alloc<double>(3 * B);
      U->loss = M.alloc<double>(1);
      U->d_err = M.alloc<int32_t>(1, true, s);
      U->in_rho = M.alloc<float>(B * V0);
      U->in_phi = M.alloc<float>(B * V0);
      U->in_base = M.alloc<float>(B * V0);
      U->in_next = M.alloc<float>(B * V0);
      U->out_phi = M.alloc<float>(B * V0);
      CMG_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
      U->mem.release();
      delete U;
      throw;
    }
    *out = U;
    return (int)CMG_OK;
  });
}

int cmg_unet_destroy(cmg_unet *U) {
  if (!U) return CMG_OK;
  cudaSetDevice(U->ctx->device);
  cudaStreamSynchronize(U->ctx->stream);
  U->mem.release();
  delete U;
  return CMG_OK;
}

int cmg_unet_n_params(const cmg_unet *U, int64_t *n) {
  if (!U || !n) return CMG_ERR_INVALID_ARG;
  *n = U->np;
  return CMG_OK;
}

int cmg_unet_set_params(cmg_unet *U, const float *params, cmg_mem mem) {
  return unet_guard([&] {
    if (!U || !params) return (int)CMG_ERR_INVALID_ARG;
    cudaSetDevice(U->ctx->device);
    cmg::copy_in(U, U->params, params, U->np, mem);
    cudaStream_t s = U->ctx->stream;
    CMG_CUDA(cudaMemsetAsync(U->m, 0, sizeof(float) * U->np, s));
    CMG_CUDA(cudaMemsetAsync(U->v, 0, sizeof(float) * U->np, s));
    CMG_CUDA(cudaMemsetAsync(U->clip, 0, sizeof(double) * 8, s));
    U->adam_t = 0;
    U->weights_ready = false;
    CMG_CUDA(cudaStreamSynchronize(s));
    return (int)CMG_OK;
  });
}

int cmg_unet_set_kernels(cmg_unet *U, int tensor_path) {
  if (!U || (tensor_path != 0 && tensor_path != 1)) return CMG_ERR_INVALID_ARG;
  U->use_tc = tensor_path == 1;
  return CMG_OK;
}

int cmg_unet_set_output_scale(cmg_unet *U, float scale) {
  if (!U || !(scale > 0.f) || !std::isfinite(scale)) return CMG_ERR_INVALID_ARG;
  U->out_scale = scale;
  return CMG_OK;
}

int cmg_unet_get_output_scale(const cmg_unet *U, float *scale) {
  if (!U || !scale) return CMG_ERR_INVALID_ARG;
  *scale = U->out_scale;
  return CMG_OK;
}

int cmg_unet_get_params(cmg_unet *U, float *out, cmg_mem mem) {
  return unet_guard([&] {
    if (!U || !out) return (int)CMG_ERR_INVALID_ARG;
    cudaSetDevice(U->ctx->device);
    CMG_CUDA(cudaMemcpyAsync(out, U->params, sizeof(float) * U->np,
                             mem == CMG_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                             U->ctx->stream));
    CMG_CUDA(cudaStreamSynchronize(U->ctx->stream));
    return (int)CMG_OK;
  });
}

int cmg_unet_forward(cmg_unet *U, const float *rho, const float *field, const float *base, int batch,
                     float *phi_pred, float *delta, cmg_mem mem) {
  return unet_guard([&] {
    if (!U || !rho || !field || batch < 1 || batch > U->max_batch) return (int)CMG_ERR_INVALID_ARG;
    cudaSetDevice(U->ctx->device);
    const int64_t n = (int64_t)batch * U->D * U->D * U->D;
    cudaStream_t s = U->ctx->stream;
    cmg::copy_in(U, U->in_rho, rho, n, mem);
    cmg::copy_in(U, U->in_phi, field, n, mem);
    cmg::copy_in(U, U->in_base, base ? base : field, n, mem);
    cmg::forward(U, batch, U->out_phi, false);
    const cudaMemcpyKind k = mem == CMG_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (phi_pred) CMG_CUDA(cudaMemcpyAsync(phi_pred, U->out_phi, sizeof(float) * n, k, s));
    if (delta) CMG_CUDA(cudaMemcpyAsync(delta, U->delta, sizeof(float) * n, k, s));
    if (mem == CMG_MEM_HOST) {
      CMG_CUDA(cudaStreamSynchronize(s));
      cmg::check_status(U);
    }
    return (int)CMG_OK;
  });
}

int cmg_unet_gradients(cmg_unet *U, const float *rho, const float *field, const float *base, const float *target,
                       int batch, float *grads, double *loss, cmg_mem mem) {
  return unet_guard([&] {
    if (!U || !rho || !field || !target || batch < 1 || batch > U->max_batch) return (int)CMG_ERR_INVALID_ARG;
    cudaSetDevice(U->ctx->device);
    const int64_t n = (int64_t)batch * U->D * U->D * U->D;
    cudaStream_t s = U->ctx->stream;
    cmg::copy_in(U, U->in_rho, rho, n, mem);
    cmg::copy_in(U, U->in_phi, field, n, mem);
    cmg::copy_in(U, U->in_base, base ? base : field, n, mem);
    cmg::copy_in(U, U->in_next, target, n, mem);
    cmg::forward(U, batch, nullptr, true);
    cmg::backward(U, batch);
    const cudaMemcpyKind k = mem == CMG_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (grads) CMG_CUDA(cudaMemcpyAsync(grads, U->grads, sizeof(float) * U->np, k, s));
    if (loss) {
      CMG_CUDA(cudaMemcpyAsync(loss, U->loss, sizeof(double), k, s));
    }
    if (mem == CMG_MEM_HOST || loss) {
      CMG_CUDA(cudaStreamSynchronize(s));
      cmg::check_status(U);
    }
    if (loss && mem == CMG_MEM_HOST) *loss /= (double)n;
    return (int)CMG_OK;
  });
}

int cmg_unet_adam_step(cmg_unet *U, float lr, float beta1, float beta2, float eps) {
  return unet_guard([&] {
    if (!U || !(lr >= 0.f)) return (int)CMG_ERR_INVALID_ARG;
    cudaSetDevice(U->ctx->device);
    U->adam_t += 1;
    const float c1 = 1.f - std::pow(beta1, (float)U->adam_t), c2 = 1.f - std::pow(beta2, (float)U->adam_t);
    const bool clip = U->clip_k > 0.f;
    if (clip) {
      cmg::k_grad_sq<<<cmg::gsz(U->np), 256, 0, U->ctx->stream>>>(U->grads, U->np, U->clip);
      cmg::k_clip_scale<<<1, 1, 0, U->ctx->stream>>>(U->clip, U->clip_k);
    }
    cmg::k_adam<<<cmg::gsz(U->np), 256, 0, U->ctx->stream>>>(U->params, U->grads, U->m, U->v, U->np, lr, beta1,
                                                              beta2, eps, c1, c2, clip ? U->clip : nullptr);
    CMG_CUDA(cudaGetLastError());
    U->weights_ready = false;
    return (int)CMG_OK;
  });
}

int cmg_unet_set_grad_clip(cmg_unet *U, float k) {
  return unet_guard([&] {
    if (!U || !(k == 0.f || k >= 1.f)) return (int)CMG_ERR_INVALID_ARG;
    U->clip_k = k;
    return (int)CMG_OK;
  });
}

int cmg_unet_grad_clip_stats(cmg_unet *U, double *last_norm, double *mean_norm, int64_t *steps, int64_t *clipped) {
  return unet_guard([&] {
    if (!U) return (int)CMG_ERR_INVALID_ARG;
    cudaSetDevice(U->ctx->device);
    double h[8];
    CMG_CUDA(cudaMemcpyAsync(h, U->clip, sizeof(h), cudaMemcpyDeviceToHost, U->ctx->stream));
    CMG_CUDA(cudaStreamSynchronize(U->ctx->stream));
    if (last_norm) *last_norm = h[5];
    if (mean_norm) *mean_norm = h[1];
    if (steps) *steps = (int64_t)h[2];
    if (clipped) *clipped = (int64_t)h[4];
    return (int)CMG_OK;
  });
}

int cmg_dense_octs(cmg_ctx *ctx, const double *src, int grid_dim, double *dst, int to_octs) {
  return unet_guard([&] {
    if (!ctx || !src || !dst || grid_dim < 2 || grid_dim % 2) return (int)CMG_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    const int64_t n = (int64_t)(grid_dim / 2) * (grid_dim / 2) * (grid_dim / 2);
    cmg::k_dense_octs<<<cmg::gsz(8 * n), 256, 0, ctx->stream>>>(src, grid_dim, n, dst, to_octs);
    CMG_CUDA(cudaGetLastError());
    return (int)CMG_OK;
  });
}

}  // extern "C"
