// conv_tc.cuh -- 3x3x3 periodic convolutions of the warm-start U-Net on the
// 5th-generation tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// Implicit GEMM: out[v][n] = sum_t sum_k in[v + SIGN d_t][k] W[n][t][k] with
// M = voxels, N = output channels, K = 27 taps x input channels.  A CTA owns
// a brick of 8 (x) x 16 (y) x ZB (z) voxels: ZB accumulators of 128 rows
// (row m = 8 y + x of one z slice) x N fp32 columns in TMEM.  Per 16-channel
// input slice the CTA stages
//   * the brick's periodic halo, 10 x 18 x (ZB + 2) rows of 16 channels, as
//     two K-halves ("planes") of 16-byte rows: plane p holds channels
//     8p..8p+7 of every halo row, rows x fastest;
//   * the slice's weights for all 27 taps in the same canonical form (one
//     bulk copy of a pre-arranged image, tap-major, then K-half, then n).
// In that form every tap's A operand is a plain shared-memory descriptor:
// eight consecutive x rows are one 128-byte core matrix, the 16 y rows of a
// z slice are core matrices 10 rows (160 B) apart (SBO), the second K-half is
// a plane further (LBO), and the tap offset only moves the start address --
// no im2col copy.  One thread issues the 27 x ZB MMAs of a slice and commits
// them to an mbarrier; the slices are double-buffered so the copies of slice
// k+1 overlap the MMAs of slice k.  The epilogue reads TMEM (each warp its 32
// lanes), adds the bias, applies the ReLU and stores bf16.
//
// Every wait is bounded (clock64 budget); on expiry the kernel records
// CMG_ERR_TIMEOUT in *err, stops issuing work, frees its TMEM and returns.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace cmg {
namespace tc {

constexpr int kThreads = 128;
constexpr long long kWaitBudget = 2000000000LL;  // clock cycles (~1 s)

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, SWIZZLE_NONE, K-major canonical layout:
// start address, LBO = byte distance between the two 8-element K halves,
// SBO = byte distance between consecutive 8-row core matrices along M (N);
// bits 46-47 = 1 (descriptor version of this architecture).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: D fp32, A and B bf16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t d;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(d)
      : "r"(mbar), "r"(parity)
      : "memory");
  return d != 0;
}

// Bounded wait for the completion of phase `parity`; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try(mbar, parity))
    if (clock64() - t0 > kWaitBudget) return false;
  return true;
}

// One-thread bulk copy global -> shared completing `bytes` on mbar.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__host__ __device__ constexpr int pow2_cols(int c) { return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : c <= 256 ? 256 : 512; }

// Geometry of one configuration (shared by host and device).
template <int N, int ZB>
struct ConvGeom {
  static constexpr int kHaloRows = (ZB + 2) * 18 * 10;
  static constexpr int kHaloBytes = kHaloRows * 32;     // two planes of 16-byte rows
  static constexpr int kWBytes = 27 * N * 32;           // one slice, all taps
  static constexpr int kBufBytes = kHaloBytes + kWBytes;
  static constexpr int kBarOffset = 2 * kBufBytes;      // 4 mbarriers + TMEM slot + abort flag
  static constexpr int kSmemBytes = kBarOffset + 64 + 1024;  // + alignment slack
  static constexpr int kCols = pow2_cols(ZB * N);
};

template <int N, int ZB, int SIGN, bool BIAS_RELU>
__global__ void __launch_bounds__(kThreads) k_conv_tc(const __nv_bfloat16 *__restrict__ in, int K,
                                                     const __nv_bfloat16 *__restrict__ wimg,
                                                     const float *__restrict__ bias, __nv_bfloat16 *__restrict__ out,
                                                     int D, int *__restrict__ err) {
  using G = ConvGeom<N, ZB>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + G::kBarOffset);  // [0,1] weights, [2,3] mma
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + G::kBarOffset + 32);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + G::kBarOffset + 40);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const int nbx = D >> 3, nby = D >> 4;
  const int brick = blockIdx.x;
  const int bx = brick % nbx, by = (brick / nbx) % nby, bz = brick / (nbx * nby);
  const int64_t sbase = (int64_t)blockIdx.y * D * D * D;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(G::kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(smem_addr(bars + i), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  constexpr uint32_t kIdesc = idesc_bf16(128, N);

  const int nk = K >> 4;
  for (int kc = 0; kc < nk; ++kc) {
    const int b = kc & 1;
    uint8_t *halo = smem + b * G::kBufBytes;
    uint8_t *wsm = halo + G::kHaloBytes;
    if (kc >= 2 && !mbar_wait(smem_addr(bars + 2 + b), ((kc - 2) >> 1) & 1)) *abort_flag = 1;
    __syncthreads();
    if (*abort_flag) break;
    if (tid == 0)
      bulk_load(smem_addr(wsm), wimg + (int64_t)kc * 27 * N * 16, G::kWBytes, smem_addr(bars + b));
    for (int p = tid; p < 2 * G::kHaloRows; p += kThreads) {
      const int row = p >> 1, half = p & 1;
      const int hz = row / 180, hy = (row / 10) % 18, hx = row % 10;
      int z = bz * ZB + hz - 1, y = by * 16 + hy - 1, x = bx * 8 + hx - 1;
      z += z < 0 ? D : (z >= D ? -D : 0);
      y += y < 0 ? D : (y >= D ? -D : 0);
      x += x < 0 ? D : (x >= D ? -D : 0);
      const int64_t v = sbase + ((int64_t)z * D + y) * D + x;
      cp_async16(smem_addr(halo + half * (G::kHaloRows * 16) + row * 16), in + v * K + kc * 16 + half * 8);
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    fence_async_shared();
    __syncthreads();
    if (tid == 0) {
      if (mbar_wait(smem_addr(bars + b), (kc >> 1) & 1)) {
        tc_fence_after();
        const uint32_t hbase = smem_addr(halo), wbase = smem_addr(wsm);
#pragma unroll 1
        for (int t = 0; t < 27; ++t) {
          const int dz = SIGN * (t / 9 - 1), dy = SIGN * ((t / 3) % 3 - 1), dx = SIGN * (t % 3 - 1);
          const uint64_t bdesc = sdesc(wbase + t * N * 32, N * 16, 128);
#pragma unroll
          for (int zz = 0; zz < ZB; ++zz) {
            const int row0 = ((zz + dz + 1) * 18 + (dy + 1)) * 10 + (dx + 1);
            const uint64_t adesc = sdesc(hbase + row0 * 16, G::kHaloRows * 16, 160);
            mma_bf16(tbase + zz * N, adesc, bdesc, kIdesc, (kc | t) != 0);
          }
        }
      } else {
        *abort_flag = 1;
      }
      mma_commit(smem_addr(bars + 2 + b));  // arrives even when nothing was issued
    }
  }
  // all MMAs of the last slice done (each commit covers every earlier MMA)
  if (!*abort_flag && !mbar_wait(smem_addr(bars + 2 + ((nk - 1) & 1)), ((nk - 1) >> 1) & 1)) *abort_flag = 1;
  __syncthreads();
  tc_fence_after();
  if (!*abort_flag) {
    const int m = warp * 32 + lane;  // TMEM lane = accumulator row
    const int y = by * 16 + (m >> 3), x = bx * 8 + (m & 7);
#pragma unroll 1
    for (int zz = 0; zz < ZB; ++zz) {
      const int z = bz * ZB + zz;
      __nv_bfloat16 *dst = out + (sbase + ((int64_t)z * D + y) * D + x) * N;
#pragma unroll 1
      for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16];
        tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + zz * N + c0, v);
        __align__(16) __nv_bfloat162 o[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float a = v[2 * j], c = v[2 * j + 1];
          if (BIAS_RELU) {
            a = fmaxf(a + bias[c0 + 2 * j], 0.f);
            c = fmaxf(c + bias[c0 + 2 * j + 1], 0.f);
          }
          o[j] = __floats2bfloat162_rn(a, c);
        }
        reinterpret_cast<uint4 *>(dst + c0)[0] = reinterpret_cast<const uint4 *>(o)[0];
        reinterpret_cast<uint4 *>(dst + c0)[1] = reinterpret_cast<const uint4 *>(o)[1];
      }
    }
  } else if (tid == 0) {
    atomicExch(err, (int)CMG_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(G::kCols));
}

// Weight image for k_conv_tc: src [N][27][K] (bf16) -> dst [K/16][27][2][N][8]
// (slice, tap, K-half, output channel, 8 channels).
__global__ void k_weight_image(const __nv_bfloat16 *__restrict__ src, int N, int K, __nv_bfloat16 *__restrict__ dst) {
  const int64_t total = (int64_t)N * 27 * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % K);
    const int t = (int)((e / K) % 27);
    const int n = (int)(e / (27 * K));
    const int kc = k >> 4, p = (k >> 3) & 1, j = k & 7;
    dst[((((int64_t)kc * 27 + t) * 2 + p) * N + n) * 8 + j] = src[e];
  }
}

}  // namespace tc
}  // namespace cmg
