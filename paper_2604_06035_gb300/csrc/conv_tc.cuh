// conv_tc.cuh -- 3x3x3 periodic convolutions of the warm-start U-Net on the
// 5th-generation tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// Implicit GEMM: out[v][n] = sum_t sum_k in[v + SIGN d_t][k] W[n][t][k] with
// M = voxels, N = output channels, K = 27 taps x input channels.  A CTA owns
// bricks of 8 (x) x 16 (y) x ZB (z) voxels: one accumulator of 128 rows
// (row m = 8 y + x of one z slice) per z slice, fp32 in TMEM.  Per 16-channel
// input slice the CTA stages
//   * the brick's periodic halo, 10 x 18 x (ZB + 2) rows of 16 channels, as
//     two K-halves ("planes") of 16-byte rows: plane p holds channels
//     8p..8p+7 of every halo row, rows x fastest;
//   * the slice's weights for all 27 taps in the canonical form (one bulk
//     copy of a pre-arranged image).
// In that form every A operand is a plain shared-memory descriptor: eight
// consecutive x rows are one 128-byte core matrix, the 16 y rows of a z slab
// are core matrices 10 rows (160 B) apart (SBO), the second K-half is a plane
// further (LBO), and a tap's (dy, dx) offset only moves the start address --
// no im2col copy.
//
// A z slab of the halo is the A operand of three taps (dz = -1, 0, +1 of
// three consecutive output slices).  For N <= 32 ("stacked" form) one MMA
// with N' = 3N covers all three: B stacks the three taps' weights, and D
// spans three consecutive accumulators (output slices s - 2, s - 1, s for
// halo slab s; the accumulator of slice zz sits at column (zz + 2) N, the
// slices -2, -1, ZB, ZB + 1 are scratch).  That is 9 (ZB + 2) MMAs per slice
// and brick instead of 27 ZB, each with three times the N -- the MMA cost
// at small N is set by the A operand, not by N.  The accumulators are then
// zeroed by the epilogue (tcgen05.st) instead of by the first MMA.  For
// N >= 48 every tap is its own MMA (27 ZB per slice and brick).
//
// The kernel is persistent and warp-specialised: one CTA per SM walks the
// work items (brick, slice) of bricks blockIdx.x, + gridDim.x, ...; warps
// 0-3 run the epilogues (TMEM -> bias, ReLU -> bf16; warp w owns TMEM lanes
// 32w..32w+31), warps 4-7 load the halo stages (cp.async), and one thread of
// warp 8 issues every MMA in work-item order (one issuer keeps each mbarrier
// waited in phase order and the summation order fixed).  The accumulators
// are double-buffered in TMEM so that a brick's epilogue overlaps the next
// brick's MMAs, and the producers never wait for an epilogue.
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

// 16 consecutive fp32 columns of this thread's TMEM lane, without the wait
// (several loads in flight, one tcgen05.wait::ld after them).
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__host__ __device__ constexpr int pow2_cols(int c) { return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : c <= 256 ? 256 : 512; }

__device__ __forceinline__ void tmem_st16_zero(uint32_t taddr) {
  const uint32_t z = 0;
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
      "r"(z)
      : "memory");
}

// Geometry of one configuration (shared by host and device).
template <int N, int ZB>
struct ConvGeom {
  static constexpr bool kStack = N <= 32;
  static constexpr int kHaloRows = (ZB + 2) * 18 * 10;
  static constexpr int kHaloBytes = kHaloRows * 32;  // two planes of 16-byte rows
  static constexpr int kWBytes = 27 * N * 32;        // one 16-channel slice, all taps
  static constexpr int kAccCols = kStack ? (ZB + 4) * N : ZB * N;  // one accumulator set
  static constexpr int kCols = pow2_cols(2 * kAccCols);            // two sets
  static constexpr int kBarBytes = 192;  // 14 mbarriers, TMEM slot, abort flag
  // Weights stay resident (one bulk copy per CTA) when they fit beside a
  // three-stage halo ring; otherwise every stage carries its slice's weights
  // and the ring has two stages.
  __host__ __device__ static constexpr bool resident(int K) {
    return 3 * kHaloBytes + (K / 16) * kWBytes + kBarBytes + 1024 <= 227 * 1024;
  }
  __host__ __device__ static constexpr int stages(int K) { return resident(K) ? 3 : 2; }
  __host__ __device__ static constexpr int stage_bytes(int K) { return kHaloBytes + (resident(K) ? 0 : kWBytes); }
  __host__ __device__ static constexpr int wres_offset(int K) { return stages(K) * stage_bytes(K); }
  __host__ __device__ static constexpr int bar_offset(int K) {
    return wres_offset(K) + (resident(K) ? (K / 16) * kWBytes : 0);
  }
  // at least 116 KB so that a single CTA fits per SM (the TMEM allocation
  // assumes it)
  __host__ __device__ static constexpr int smem_bytes(int K) {
    return bar_offset(K) + kBarBytes + 1024 > 116 * 1024 ? bar_offset(K) + kBarBytes + 1024 : 116 * 1024;
  }
};

// Optional work of a forward convolution's epilogue (nullptr = off):
//   pool  the 2x2x2 mean of the (bf16-rounded) outputs on the D/2 grid,
//         N <= 32 and ZB even (both z slices of a pair are in the thread,
//         the x / y partners are lanes ^1 / ^8 of the warp);
//   hw    the linear head (N = 16): delta = hb + sum_c out_c hw_c,
//         pred = base + norm[3 sample + 2] delta (float fields [B][D^3]);
//         with store_out = 0 the activations themselves are not written.
struct ConvEpi {
  __nv_bfloat16 *pool = nullptr;
  const float *hw = nullptr, *base = nullptr, *norm = nullptr;
  float *delta = nullptr, *pred = nullptr;
  int store_out = 1;
};

// Barriers:
//   full[s]     halo of stage s landed (128 producer arrivals)
//   empty[s]    MMAs that read stage s done (tcgen05.commit of its issuer)
//   wfull[s]    stage weights landed (bulk copy); wres: resident weights
//   accfull[b]  brick accumulators in TMEM set b complete (commit)
//   accempty[b] the epilogue has read (and, stacked, zeroed) set b (128 arrivals)
// FWD: out = ReLU(conv(in, W) + bias); else out = conv^T (SIGN = -1, no bias).
// With `skip` set (forward only) the input is the channel concatenation of
// the nearest-upsampled `in` (K - Cb channels on the D/2 grid) and `skip`
// (Cb channels on the D grid), read directly by the halo loader.
constexpr int kConvThreads = 288;
constexpr int kProducers = 128;

template <int N, int ZB, bool FWD>
__global__ void __launch_bounds__(kConvThreads, 1) k_conv_tc(const __nv_bfloat16 *__restrict__ in, int K,
                                                            const __nv_bfloat16 *__restrict__ skip, int Cb,
                                                            const __nv_bfloat16 *__restrict__ wimg,
                                                            const float *__restrict__ bias,
                                                            __nv_bfloat16 *__restrict__ out, int D, int total_bricks,
                                                            int *__restrict__ err, const ConvEpi ep) {
  using G = ConvGeom<N, ZB>;
  constexpr int SIGN = FWD ? 1 : -1;
  constexpr bool STACK = G::kStack;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const bool wres = G::resident(K);
  const int NS = G::stages(K), sbytes = G::stage_bytes(K);
  uint8_t *wres_sm = smem + G::wres_offset(K);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + G::bar_offset(K));
  uint64_t *full = bars, *empty = bars + 3, *wfull = bars + 6, *wresb = bars + 9, *accfull = bars + 10,
           *accempty = bars + 12;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 14);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 15);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nk = K >> 4, Ca = K - Cb, Dh = D >> 1;
  const int nbx = D >> 3, nby = D >> 4, nbps = nbx * nby * (D / ZB);
  const int my_bricks = blockIdx.x < total_bricks ? (total_bricks - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int n_items = my_bricks * nk;

  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(G::kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < 3; ++i) {
      mbar_init(smem_addr(full + i), kProducers);
      mbar_init(smem_addr(empty + i), 1);
      mbar_init(smem_addr(wfull + i), 1);
    }
    mbar_init(smem_addr(wresb), 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_addr(accfull + i), 1);
      mbar_init(smem_addr(accempty + i), kProducers);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  if (STACK && warp < 4) {
    // both accumulator sets start at zero (the MMAs always accumulate)
    const uint32_t lanes = (uint32_t)(warp * 32) << 16;
    for (int c0 = 0; c0 < 2 * G::kAccCols; c0 += 16) tmem_st16_zero(tbase + lanes + c0);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  // bounded wait that also gives up as soon as another thread has
  auto wait = [&](uint64_t *bar, int parity) -> bool {
    const uint32_t a = smem_addr(bar);
    const long long t0 = clock64();
    while (!mbar_try(a, (uint32_t)parity)) {
      if (*abort_flag) return false;
      if (clock64() - t0 > kWaitBudget) {
        *abort_flag = 1;
        return false;
      }
    }
    return true;
  };

  if (warp >= 4 && warp < 8) {
    // ---------------------------------------------------------- producers
    const int ptid = tid - 128;
    if (wres && ptid == 0 && n_items > 0)
      bulk_load(smem_addr(wres_sm), wimg, (uint32_t)(nk * G::kWBytes), smem_addr(wresb));
    // each thread copies halo columns (hy, hx, half): slots ptid, + 128, + 256 (< 360)
    auto produce = [&](int j) {
      const int bi = blockIdx.x + (j / nk) * gridDim.x, kc = j % nk;
      const int sample = bi / nbps, brick = bi % nbps;
      const int bx = brick % nbx, by = (brick / nbx) % nby, bz = brick / (nbx * nby);
      uint8_t *halo = smem + (j % NS) * sbytes;
      const bool up = skip != nullptr && kc * 16 < Ca;
      const int cbase = up ? kc * 16 : (skip != nullptr ? kc * 16 - Ca : kc * 16);
      const int cstride = up ? Ca : (skip != nullptr ? Cb : K);
      const __nv_bfloat16 *srcT = (skip != nullptr && !up) ? skip : in;
      const int Dg = up ? Dh : D;  // grid of the tensor read
      const int64_t s_off = (int64_t)sample * Dg * Dg * Dg;
      for (int slot = ptid; slot < 360; slot += kProducers) {
        const int col = slot >> 1, half = slot & 1;
        const int hy = col / 10, hx = col % 10;
        int y = by * 16 + hy - 1, x = bx * 8 + hx - 1;
        y += y < 0 ? D : (y >= D ? -D : 0);
        x += x < 0 ? D : (x >= D ? -D : 0);
        if (up) {
          y >>= 1;
          x >>= 1;
        }
        const __nv_bfloat16 *src = srcT + (s_off + (int64_t)y * Dg + x) * cstride + cbase + half * 8;
        const uint32_t dst = smem_addr(halo + half * (G::kHaloRows * 16) + col * 16);
#pragma unroll
        for (int hz = 0; hz < ZB + 2; ++hz) {
          int z = bz * ZB + hz - 1;
          z += z < 0 ? D : (z >= D ? -D : 0);
          if (up) z >>= 1;
          cp_async16(dst + hz * 180 * 16, src + (int64_t)z * Dg * Dg * cstride);
        }
      }
      if (!wres && ptid == 0)
        bulk_load(smem_addr(halo + G::kHaloBytes), wimg + (int64_t)kc * 27 * N * 16, G::kWBytes,
                  smem_addr(wfull + j % NS));
    };
    for (int s = 0; s < NS - 1; ++s) {
      if (s < n_items) produce(s);
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int j = 0; j < n_items; ++j) {
      // item j's copies landed (its group is NS - 2 groups older than the
      // newest): hand the stage to the MMA warp
      if (NS == 3) asm volatile("cp.async.wait_group 1;" ::: "memory");
      else asm volatile("cp.async.wait_group 0;" ::: "memory");
      fence_async_shared();
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(full + j % NS)) : "memory");
      // refill the stage of item j - 1 once its MMAs are done
      const int jn = j + NS - 1;
      if (jn < n_items) {
        if (jn >= NS && !wait(empty + jn % NS, ((jn - NS) / NS) & 1)) break;
        produce(jn);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  } else if (warp < 4) {
    // ----------------------------------------------------------- epilogue
    const int m = warp * 32 + lane;  // TMEM lane = accumulator row
    for (int c = 0; c < my_bricks; ++c) {
      if (!wait(accfull + (c & 1), (c >> 1) & 1)) break;
      tc_fence_after();
      const int bi = blockIdx.x + c * gridDim.x;
      const int sample = bi / nbps, brick = bi % nbps;
      const int bx = brick % nbx, by = (brick / nbx) % nby, bz = brick / (nbx * nby);
      const uint32_t set = tbase + (c & 1) * G::kAccCols + ((uint32_t)(warp * 32) << 16);
      const int y = by * 16 + (m >> 3), x = bx * 8 + (m & 7);
      // the ZB accumulators are ZB * N consecutive columns; 32 per wait
      const uint32_t acc0 = set + (STACK ? 2 * N : 0);
      const int64_t vbase = (int64_t)sample * D * D * D + (int64_t)y * D + x;
      if constexpr (FWD && N <= 32) {
        if (ep.pool != nullptr || ep.hw != nullptr) {
          // per z slice: all N columns, bias + ReLU + bf16 rounding, then
          // the optional pooling (pairs of slices) and head
          float keep[N];
          const int Dh = D >> 1;
#pragma unroll 1
          for (int zz = 0; zz < ZB; ++zz) {
            float v[N];
#pragma unroll
            for (int c0 = 0; c0 < N; c0 += 16) tmem_ld16_nowait(acc0 + zz * N + c0, v + c0);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int z = bz * ZB + zz;
            const int64_t vox = vbase + (int64_t)z * D * D;
#pragma unroll
            for (int c0 = 0; c0 < N; c0 += 16) {
              __align__(16) __nv_bfloat162 o[8];
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                o[q] = __floats2bfloat162_rn(fmaxf(v[c0 + 2 * q] + __ldg(bias + c0 + 2 * q), 0.f),
                                             fmaxf(v[c0 + 2 * q + 1] + __ldg(bias + c0 + 2 * q + 1), 0.f));
                v[c0 + 2 * q] = __low2float(o[q]);
                v[c0 + 2 * q + 1] = __high2float(o[q]);
              }
              if (ep.store_out) {
                __nv_bfloat16 *dst = out + vox * N + c0;
                reinterpret_cast<uint4 *>(dst)[0] = reinterpret_cast<const uint4 *>(o)[0];
                reinterpret_cast<uint4 *>(dst)[1] = reinterpret_cast<const uint4 *>(o)[1];
              }
            }
            if (N == 16 && ep.hw != nullptr) {
              float dlt = __ldg(ep.hw + 16);  // the head's bias
#pragma unroll
              for (int c = 0; c < 16; ++c) dlt = fmaf(v[c], __ldg(ep.hw + c), dlt);
              ep.delta[vox] = dlt;
              if (ep.pred) ep.pred[vox] = ep.base[vox] + ep.norm[3 * sample + 2] * dlt;
            }
            if (ep.pool != nullptr) {
              if ((zz & 1) == 0) {
#pragma unroll
                for (int c = 0; c < N; ++c) keep[c] = v[c];
              } else {
                const bool writer = (lane & 1) == 0 && (lane & 8) == 0;
                __nv_bfloat16 *pdst =
                    ep.pool + (((int64_t)sample * Dh + (z >> 1)) * Dh * Dh + (int64_t)(y >> 1) * Dh + (x >> 1)) * N;
#pragma unroll
                for (int c0 = 0; c0 < N; c0 += 16) {
                  __align__(16) __nv_bfloat162 o[8];
#pragma unroll
                  for (int q = 0; q < 8; ++q) {
                    float a = keep[c0 + 2 * q] + v[c0 + 2 * q], b2 = keep[c0 + 2 * q + 1] + v[c0 + 2 * q + 1];
                    a += __shfl_xor_sync(0xffffffffu, a, 1);
                    b2 += __shfl_xor_sync(0xffffffffu, b2, 1);
                    a += __shfl_xor_sync(0xffffffffu, a, 8);
                    b2 += __shfl_xor_sync(0xffffffffu, b2, 8);
                    o[q] = __floats2bfloat162_rn(a * 0.125f, b2 * 0.125f);
                  }
                  if (writer) {
                    reinterpret_cast<uint4 *>(pdst + c0)[0] = reinterpret_cast<const uint4 *>(o)[0];
                    reinterpret_cast<uint4 *>(pdst + c0)[1] = reinterpret_cast<const uint4 *>(o)[1];
                  }
                }
              }
            }
          }
          goto epilogue_done;
        }
      }
#pragma unroll 1
      for (int col0 = 0; col0 < ZB * N; col0 += 32) {
        const int ng = (ZB * N - col0) >= 32 ? 2 : 1;  // 16-column groups in this chunk
        float v[32];
        tmem_ld16_nowait(acc0 + col0, v);
        if (ng == 2) tmem_ld16_nowait(acc0 + col0 + 16, v + 16);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          if (g >= ng) break;
          const int col = col0 + 16 * g, zz = col / N, c0 = col % N;
          __nv_bfloat16 *dst = out + (vbase + (int64_t)(bz * ZB + zz) * D * D) * N + c0;
          __align__(16) __nv_bfloat162 o[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            float a = v[16 * g + 2 * q], b2 = v[16 * g + 2 * q + 1];
            if (FWD) {
              a = fmaxf(a + __ldg(bias + c0 + 2 * q), 0.f);
              b2 = fmaxf(b2 + __ldg(bias + c0 + 2 * q + 1), 0.f);
            }
            o[q] = __floats2bfloat162_rn(a, b2);
          }
          reinterpret_cast<uint4 *>(dst)[0] = reinterpret_cast<const uint4 *>(o)[0];
          reinterpret_cast<uint4 *>(dst)[1] = reinterpret_cast<const uint4 *>(o)[1];
        }
      }
    epilogue_done:
      if (STACK) {
        // zero the whole set (scratch slices included) for its next brick
        for (int c0 = 0; c0 < G::kAccCols; c0 += 16) tmem_st16_zero(set + c0);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      }
      tc_fence_before();
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(accempty + (c & 1))) : "memory");
    }
  } else if (warp == 8 && lane == 0) {
    // ------------------------------------------------------------ MMA issue
    constexpr uint32_t kIdesc = idesc_bf16(128, STACK ? 3 * N : N);
    for (int j = 0; j < n_items; ++j) {
      const int st = j % NS, kc = j % nk, c = j / nk, h = c & 1;
      if (kc == 0 && c >= 2 && !wait(accempty + h, ((c - 2) >> 1) & 1)) break;
      if (!wait(full + st, (j / NS) & 1)) break;
      if (!(wres ? wait(wresb, 0) : wait(wfull + st, (j / NS) & 1))) break;
      fence_async_shared();
      tc_fence_after();
      const uint32_t hbase = smem_addr(smem + st * sbytes);
      const uint32_t wbase = wres ? smem_addr(wres_sm) + kc * G::kWBytes : hbase + G::kHaloBytes;
      const uint64_t a0 = sdesc(hbase, G::kHaloRows * 16, 160);
      const uint32_t set = tbase + h * G::kAccCols;
      if (STACK) {
        // B for (dy, dx) = q: the taps dz = +1, 0, -1 (times SIGN) stacked
        const uint64_t b0 = sdesc(wbase, 3 * N * 16, 128);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          const int qoff = (q / 3) * 10 + (q % 3);  // (dy + 1) * 10 + (dx + 1) in halo rows
          const uint64_t bdesc = b0 + (uint64_t)(q * 6 * N);  // + q 3N 32 bytes (>> 4)
#pragma unroll
          for (int sl = 0; sl < ZB + 2; ++sl)
            mma_bf16(set + sl * N, a0 + (uint64_t)(sl * 180 + qoff), bdesc, kIdesc, 1u);
        }
      } else {
        const uint64_t b0 = sdesc(wbase, N * 16, 128);
#pragma unroll
        for (int t = 0; t < 27; ++t) {
          const int dz = SIGN * (t / 9 - 1), dy = SIGN * ((t / 3) % 3 - 1), dx = SIGN * (t % 3 - 1);
          const int toff = ((dz + 1) * 18 + (dy + 1)) * 10 + (dx + 1);  // halo row of (0, 0, 0) at this tap
          const uint64_t bdesc = b0 + (uint64_t)(t * N * 2);          // + t N 32 bytes (>> 4)
#pragma unroll
          for (int zz = 0; zz < ZB; ++zz)
            mma_bf16(set + zz * N, a0 + (uint64_t)(zz * 180 + toff), bdesc, kIdesc, (t > 0 || kc > 0) ? 1u : 0u);
        }
      }
      mma_commit(smem_addr(empty + st));
      if (kc == nk - 1) mma_commit(smem_addr(accfull + h));
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (*abort_flag && tid == 0) atomicExch(err, (int)CMG_ERR_TIMEOUT);
  if (warp == 8) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(G::kCols));
}

// Weight images for k_conv_tc from src [N][27][K] (bf16):
//   per tap (N >= 48):  [K/16][27 taps][2 K-halves][N][8]
//   stacked (N <= 32):  [K/16][9 (dy, dx)][2 K-halves][3 (dz = +1, 0, -1)][N][8]
// with the tap offsets of the stacked form scaled by `sign` (-1 for the
// input-gradient convolution, whose taps are mirrored).
__global__ void k_weight_image(const __nv_bfloat16 *__restrict__ src, int N, int K, int sign,
                               __nv_bfloat16 *__restrict__ dst) {
  const int64_t total = (int64_t)N * 27 * K;
  const bool stack = N <= 32;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % K);
    const int t = (int)((e / K) % 27);
    const int n = (int)(e / (27 * K));
    const int kc = k >> 4, p = (k >> 3) & 1, j = k & 7;
    int64_t o;
    if (!stack) {
      o = ((((int64_t)kc * 27 + t) * 2 + p) * N + n) * 8 + j;
    } else {
      // applied offsets (dzs, dys, dxs) = sign (dz, dy, dx) of tap t
      const int dzs = sign * (t / 9 - 1), dys = sign * ((t / 3) % 3 - 1), dxs = sign * (t % 3 - 1);
      const int q = (dys + 1) * 3 + (dxs + 1), st = 1 - dzs;  // dzs = +1 -> 0, 0 -> 1, -1 -> 2
      o = (((((int64_t)kc * 9 + q) * 2 + p) * 3 + st) * N + n) * 8 + j;
    }
    dst[o] = src[e];
  }
}

}  // namespace tc
}  // namespace cmg
