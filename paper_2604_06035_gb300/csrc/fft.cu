// fft.cu -- direct FP32 FFT solve of the correction equation on a full
// periodic level (the paper's FFT base-level solve, Sec. 5.2, here inside the
// FP64 iterative refinement of the mixed-precision path).
//
// On a full periodic level the 7-point operator is diagonalised by the 3-D
// DFT.  The FP32 inner problem of the refinement loop is the smoother's fixed
// point e = (sum of the 6 neighbours) / 6 + g, i.e.
//   sum_nb e - 6 e = -6 g,
// whose symbol is -4 (sin^2(pi kx/n) + sin^2(pi ky/n) + sin^2(pi kz/n)), so
//   e^(k) = 1.5 g^(k) / (sin^2 + sin^2 + sin^2),  e^(0) = 0 (zero mean).
// Five passes over a dense complex FP32 array [z][y][x]: x forward (gathering
// g from the colour-planar oct layout through an oct map), y forward, z
// forward + scaling + z inverse (one kernel, the line stays in shared
// memory), y inverse, x inverse (scattering e into the oct layout).  Each
// pass runs batched radix-2 FFTs of whole lines in shared memory: forward
// transforms decimate in time from a bit-reversed load, inverse ones
// decimate in frequency to a bit-reversed store, so no pass reorders
// separately.  Twiddles exp(-2 pi i k / n) come from an FP64 table rounded to
// FP32, laid out by stage; lines are padded by one element per 16 against
// shared-memory bank conflicts.  Each refinement step gains ~6 digits (FP32 transform error), so the
// FP64 loop reaches 1e-10 in two or three steps.
#include <algorithm>
#include <cmath>
#include <vector>

#include "cmg_internal.cuh"

namespace cmg {
namespace {

constexpr int kFftThreads = 256;
constexpr int kLoads = 8;  // global loads each thread keeps in flight per batch

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 conjf2(float2 w) { return make_float2(w.x, -w.y); }

__device__ __forceinline__ int brev(int i, int logn) { return (int)(__brev((unsigned)i) >> (32 - logn)); }

// Shared-memory position of element i of a line: one float2 of padding per 16
// elements, so that bit-reversed and power-of-two-strided accesses of a warp
// spread over the banks.
__host__ __device__ constexpr int pad(int i) { return i + (i >> 4); }

// Twiddles by stage: stage s (span 2^s) uses w_s(p) = exp(-2 pi i p / 2^s),
// p < 2^(s-1), stored at (2^(s-1) - 1) + p, so a stage's threads read
// consecutive entries.  The FP64-rounded values are those of exp(-2 pi i k / n)
// at k = p n / 2^s.
__device__ __forceinline__ float2 twid(const float2 *tws, int s, int p) { return tws[(1 << (s - 1)) - 1 + p]; }

// In-place radix-2 transforms of `lines` lines of length n = 2^logn in
// shared memory (line l at s + l ld, element i at pad(i)).  DIT (forward:
// input bit-reversed, output natural) with twiddles w^k; DIF (inverse: input
// natural, output bit-reversed) with conj(w)^k.  Three stages per pass where
// they fit (eight points per thread in registers), then two, then one: the
// same butterflies in the same order as stage by stage, with a third of the
// shared-memory round trips and barriers.
__device__ void fft_dit(float2 *s, int logn, int ld, int lines, const float2 *tws) {
  const int n = 1 << logn;
  int st = 1;
  for (; st + 2 <= logn; st += 3) {
    const int h = 1 << (st - 1), ng = lines << (logn - 3);
    for (int b = threadIdx.x; b < ng; b += blockDim.x) {
      const int line = b >> (logn - 3), g = b & ((n >> 3) - 1);
      const int pos = g & (h - 1), i = ((g >> (st - 1)) << (st + 2)) | pos;
      float2 *x = s + line * ld;
      float2 v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = x[pad(i + k * h)];
      const float2 w1 = twid(tws, st, pos);
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
        const float2 c = cmul(v[k + 1], w1);
        v[k + 1] = csub(v[k], c);
        v[k] = cadd(v[k], c);
      }
      const float2 w2a = twid(tws, st + 1, pos), w2b = twid(tws, st + 1, pos + h);
#pragma unroll
      for (int k0 = 0; k0 < 8; k0 += 4) {
        const float2 c0 = cmul(v[k0 + 2], w2a), c1 = cmul(v[k0 + 3], w2b);
        v[k0 + 2] = csub(v[k0], c0);
        v[k0] = cadd(v[k0], c0);
        v[k0 + 3] = csub(v[k0 + 1], c1);
        v[k0 + 1] = cadd(v[k0 + 1], c1);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 c = cmul(v[k + 4], twid(tws, st + 2, pos + k * h));
        v[k + 4] = csub(v[k], c);
        v[k] = cadd(v[k], c);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) x[pad(i + k * h)] = v[k];
    }
    __syncthreads();
  }
  for (; st + 1 <= logn; st += 2) {
    const int h = 1 << (st - 1), ng = lines << (logn - 2);
    for (int b = threadIdx.x; b < ng; b += blockDim.x) {
      const int line = b >> (logn - 2), g = b & ((n >> 2) - 1);
      const int pos = g & (h - 1), i = ((g >> (st - 1)) << (st + 1)) | pos;
      float2 *x = s + line * ld;
      const float2 w1 = twid(tws, st, pos), w2 = twid(tws, st + 1, pos), w3 = twid(tws, st + 1, pos + h);
      const float2 x0 = x[pad(i)], x1 = cmul(x[pad(i + h)], w1), x2 = x[pad(i + 2 * h)],
                   x3 = cmul(x[pad(i + 3 * h)], w1);
      const float2 y0 = cadd(x0, x1), y1 = csub(x0, x1), y2 = cadd(x2, x3), y3 = csub(x2, x3);
      const float2 u = cmul(y2, w2), v = cmul(y3, w3);
      x[pad(i)] = cadd(y0, u);
      x[pad(i + 2 * h)] = csub(y0, u);
      x[pad(i + h)] = cadd(y1, v);
      x[pad(i + 3 * h)] = csub(y1, v);
    }
    __syncthreads();
  }
  if (st == logn) {  // one stage left
    const int h = 1 << (st - 1), nb = lines << (logn - 1);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      const int line = b >> (logn - 1), bb = b & ((n >> 1) - 1);
      const int pos = bb & (h - 1), i = ((bb >> (st - 1)) << st) | pos;
      float2 *x = s + line * ld;
      const float2 a = x[pad(i)], c = cmul(x[pad(i + h)], twid(tws, st, pos));
      x[pad(i)] = cadd(a, c);
      x[pad(i + h)] = csub(a, c);
    }
    __syncthreads();
  }
}

__device__ void fft_dif_inv(float2 *s, int logn, int ld, int lines, const float2 *tws) {
  const int n = 1 << logn;
  int st = logn;
  for (; st - 2 >= 1; st -= 3) {
    const int q = 1 << (st - 3), ng = lines << (logn - 3);
    for (int b = threadIdx.x; b < ng; b += blockDim.x) {
      const int line = b >> (logn - 3), g = b & ((n >> 3) - 1);
      const int p = g & (q - 1), i = ((g >> (st - 3)) << st) | p;
      float2 *x = s + line * ld;
      float2 v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = x[pad(i + k * q)];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 d = csub(v[k], v[k + 4]);
        v[k] = cadd(v[k], v[k + 4]);
        v[k + 4] = cmul(d, conjf2(twid(tws, st, p + k * q)));
      }
      const float2 wa = conjf2(twid(tws, st - 1, p)), wb = conjf2(twid(tws, st - 1, p + q));
#pragma unroll
      for (int k0 = 0; k0 < 8; k0 += 4) {
        const float2 d0 = csub(v[k0], v[k0 + 2]), d1 = csub(v[k0 + 1], v[k0 + 3]);
        v[k0] = cadd(v[k0], v[k0 + 2]);
        v[k0 + 1] = cadd(v[k0 + 1], v[k0 + 3]);
        v[k0 + 2] = cmul(d0, wa);
        v[k0 + 3] = cmul(d1, wb);
      }
      const float2 wc = conjf2(twid(tws, st - 2, p));
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
        const float2 d = csub(v[k], v[k + 1]);
        v[k] = cadd(v[k], v[k + 1]);
        v[k + 1] = cmul(d, wc);
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) x[pad(i + k * q)] = v[k];
    }
    __syncthreads();
  }
  for (; st - 1 >= 1; st -= 2) {
    const int q = 1 << (st - 2), ng = lines << (logn - 2);
    for (int b = threadIdx.x; b < ng; b += blockDim.x) {
      const int line = b >> (logn - 2), g = b & ((n >> 2) - 1);
      const int p = g & (q - 1), i = ((g >> (st - 2)) << st) | p;
      float2 *x = s + line * ld;
      const float2 wa = conjf2(twid(tws, st, p)), wb = conjf2(twid(tws, st, p + q));
      const float2 wc = conjf2(twid(tws, st - 1, p));
      const float2 x0 = x[pad(i)], x1 = x[pad(i + q)], x2 = x[pad(i + 2 * q)], x3 = x[pad(i + 3 * q)];
      const float2 y0 = cadd(x0, x2), y2 = cmul(csub(x0, x2), wa);
      const float2 y1 = cadd(x1, x3), y3 = cmul(csub(x1, x3), wb);
      x[pad(i)] = cadd(y0, y1);
      x[pad(i + q)] = cmul(csub(y0, y1), wc);
      x[pad(i + 2 * q)] = cadd(y2, y3);
      x[pad(i + 3 * q)] = cmul(csub(y2, y3), wc);
    }
    __syncthreads();
  }
  if (st == 1) {  // one stage left (twiddle 1)
    const int nb = lines << (logn - 1);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      const int line = b >> (logn - 1), i = (b & ((n >> 1) - 1)) << 1;
      float2 *x = s + line * ld;
      const float2 a = x[pad(i)], c = x[pad(i + 1)];
      x[pad(i)] = cadd(a, c);
      x[pad(i + 1)] = csub(a, c);
    }
    __syncthreads();
  }
}

// the per-stage twiddle table (n - 1 entries) into shared memory
__device__ void load_tw(float2 *stw, const float2 *tw, int n) {
  for (int k = threadIdx.x; k < n - 1; k += blockDim.x) stw[k] = tw[k];
}

// line stride in shared memory: padded length plus one (odd in float2 units,
// so the y/z passes' column-wise loads spread over the banks)
__host__ __device__ constexpr int line_ld(int n) { return pad(n) + 1; }

// cell (x, y, z) of the level -> (oct, plane, slot) through the oct map
__device__ __forceinline__ int64_t cell_index(const int32_t *map, int no, int x, int y, int z, int64_t plane_stride) {
  const int o = map[((int64_t)(z >> 1) * no + (y >> 1)) * no + (x >> 1)];
  const int c = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
  return (int64_t)cell_parity(c) * plane_stride + (int64_t)o * 4 + (c >> 1);
}

// x forward: lines (y, z), `lines` per block; input g (plane stride ps)
__global__ void k_fft_x_fwd(const float *__restrict__ g, int64_t ps, const int32_t *__restrict__ map,
                            const float2 *__restrict__ tw, int n, int logn, int lines, float2 *__restrict__ buf) {
  extern __shared__ float2 sm[];
  float2 *stw = sm, *s = sm + n;
  load_tw(stw, tw, n);
  const int line0 = blockIdx.x * lines, no = n >> 1, ld = line_ld(n), total = lines * n;
  // batches of kLoads independent gathers per thread (oct map, then g)
  for (int e0 = threadIdx.x; e0 < total; e0 += kLoads * blockDim.x) {
    int64_t idx[kLoads];
    float v[kLoads];
#pragma unroll
    for (int u = 0; u < kLoads; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < total) {
        const int l = e >> logn, x = e & (n - 1), yz = line0 + l;
        idx[u] = cell_index(map, no, x, yz & (n - 1), yz >> logn, ps);
      }
    }
#pragma unroll
    for (int u = 0; u < kLoads; ++u)
      if (e0 + u * blockDim.x < total) v[u] = g[idx[u]];
#pragma unroll
    for (int u = 0; u < kLoads; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < total) s[(e >> logn) * ld + pad(brev(e & (n - 1), logn))] = make_float2(v[u], 0.f);
    }
  }
  __syncthreads();
  fft_dit(s, logn, ld, lines, stw);
  for (int e = threadIdx.x; e < lines * n; e += blockDim.x)
    buf[(int64_t)line0 * n + e] = s[(e >> logn) * ld + pad(e & (n - 1))];
}

// y or z pass on tiles of `tx` consecutive x columns: AXIS 1 = y (block =
// (z, x tile)), AXIS 2 = z (block = (y, x tile)).  MODE 0: forward;
// 1: inverse; 2 (z only): forward, scale by the inverse symbol, inverse.
// The tile's lines are n + 1 apart in shared memory (the load writes one
// element of each line per thread: no bank conflicts).
template <int AXIS, int MODE>
__global__ void k_fft_yz(float2 *__restrict__ buf, const float2 *__restrict__ tw, int n, int logn, int logtx) {
  extern __shared__ float2 sm[];
  float2 *stw = sm, *s = sm + n;
  load_tw(stw, tw, n);
  const int tx = 1 << logtx, logtile = logn - logtx;
  const int x0 = (blockIdx.x & ((1 << logtile) - 1)) << logtx, other = blockIdx.x >> logtile;  // z (AXIS 1) or y (AXIS 2)
  const int64_t nn = (int64_t)n * n;
  const int ld = line_ld(n);
  auto addr = [&](int a, int t) -> int64_t {  // element a along the axis, column x0 + t
    return AXIS == 1 ? ((int64_t)other * nn + (int64_t)a * n + x0 + t) : ((int64_t)a * nn + (int64_t)other * n + x0 + t);
  };
  // pairs of consecutive x columns as one 16-byte load (tx even: n >= 2)
  const int pairs = (tx * n) >> 1, logpx = logtx - 1;
  for (int e0 = threadIdx.x; e0 < pairs; e0 += kLoads * blockDim.x) {
    float4 v[kLoads];
#pragma unroll
    for (int u = 0; u < kLoads; ++u) {
      const int e = e0 + u * blockDim.x;  // consecutive threads read consecutive x pairs
      if (e < pairs) v[u] = *reinterpret_cast<const float4 *>(buf + addr(e >> logpx, (e & ((1 << logpx) - 1)) << 1));
    }
#pragma unroll
    for (int u = 0; u < kLoads; ++u) {
      const int e = e0 + u * blockDim.x, a = e >> logpx, t = (e & ((1 << logpx) - 1)) << 1;
      if (e < pairs) {
        const int j = pad(MODE == 1 ? a : brev(a, logn));
        s[t * ld + j] = make_float2(v[u].x, v[u].y);
        s[(t + 1) * ld + j] = make_float2(v[u].z, v[u].w);
      }
    }
  }
  __syncthreads();
  if (MODE == 1) {
    fft_dif_inv(s, logn, ld, tx, stw);
  } else {
    fft_dit(s, logn, ld, tx, stw);
    if (MODE == 2) {
      // natural-order spectrum along z; x and y are already frequencies
      const float sy = sinpif((float)other / (float)n);
      for (int e = threadIdx.x; e < tx * n; e += blockDim.x) {
        const int t = e >> logn, kz = e & (n - 1);
        const float sx = sinpif((float)(x0 + t) / (float)n), sz = sinpif((float)kz / (float)n);
        const float d = sx * sx + sy * sy + sz * sz;
        const float f = d > 0.f ? 1.5f / d : 0.f;
        float2 &v = s[t * ld + pad(kz)];
        v = make_float2(v.x * f, v.y * f);
      }
      __syncthreads();
      fft_dif_inv(s, logn, ld, tx, stw);
    }
  }
  for (int e = threadIdx.x; e < tx * n; e += blockDim.x) {
    const int a = e >> logtx, t = e & (tx - 1);
    buf[addr(a, t)] = s[t * ld + pad(MODE == 0 ? a : brev(a, logn))];
  }
}

// x inverse and scatter: e = Re / n^3 into the colour-planar FP32 field
__global__ void k_fft_x_inv(const float2 *__restrict__ buf, const int32_t *__restrict__ map,
                            const float2 *__restrict__ tw, int n, int logn, int lines, float inv_n3,
                            float *__restrict__ e_out, int64_t ps) {
  extern __shared__ float2 sm[];
  float2 *stw = sm, *s = sm + n;
  load_tw(stw, tw, n);
  const int line0 = blockIdx.x * lines, no = n >> 1, ld = line_ld(n);
  const int pairs = (lines * n) >> 1;  // two consecutive elements of a line per 16-byte load
  for (int e0 = threadIdx.x; e0 < pairs; e0 += kLoads * blockDim.x) {
    float4 v[kLoads];
#pragma unroll
    for (int u = 0; u < kLoads; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < pairs) v[u] = *reinterpret_cast<const float4 *>(buf + (int64_t)line0 * n + 2 * e);
    }
#pragma unroll
    for (int u = 0; u < kLoads; ++u) {
      const int e = 2 * (e0 + u * blockDim.x);
      if (e < 2 * pairs) {
        float2 *d = s + (e >> logn) * ld;
        d[pad(e & (n - 1))] = make_float2(v[u].x, v[u].y);
        d[pad((e & (n - 1)) + 1)] = make_float2(v[u].z, v[u].w);
      }
    }
  }
  __syncthreads();
  fft_dif_inv(s, logn, ld, lines, stw);
  for (int e = threadIdx.x; e < lines * n; e += blockDim.x) {
    const int l = e >> logn, x = e & (n - 1), yz = line0 + l;
    const int y = yz & (n - 1), z = yz >> logn;
    e_out[cell_index(map, no, x, y, z, ps)] = s[l * ld + pad(brev(x, logn))].x * inv_n3;
  }
}

__global__ void k_fft_map(const uint64_t *__restrict__ keys, int64_t n_octs, int no, int32_t *__restrict__ map) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_octs; o += (int64_t)gridDim.x * blockDim.x) {
    uint32_t i, j, k;
    morton_decode(keys[o], i, j, k);
    map[((int64_t)k * no + j) * no + i] = (int32_t)o;
  }
}

}  // namespace

bool fft_supported(const cmg_level *L) { return L->periodic_full && L->lev >= 2 && L->lev <= 9; }

void fft_prepare(cmg_level *L) {
  if (L->fft_buf) return;
  if (!fft_supported(L)) throw Error(CMG_ERR_INVALID_ARG, "the FFT solve needs a full periodic level of at most 512^3 cells");
  const int n = 1 << L->lev, no = n >> 1;
  cudaStream_t s = L->ctx->stream;
  // L->fft_buf (the "prepared" mark) is set last, after every allocation
  float2 *buf = reinterpret_cast<float2 *>(L->mem.alloc<float>((int64_t)2 * n * n * n));
  L->fft_map = L->mem.alloc<int32_t>((int64_t)no * no * no, true, s);  // zeroed: every entry a valid oct
  // per-stage twiddles: stage st (span 2^st) at (2^(st-1) - 1) + p, p < 2^(st-1),
  // the value of exp(-2 pi i k / n) at k = p n / 2^st
  L->fft_tw = reinterpret_cast<float2 *>(L->mem.alloc<float>(2 * n));
  std::vector<float> tw(2 * n, 0.f);
  for (int st = 1; st <= L->lev; ++st)
    for (int p = 0; p < (1 << (st - 1)); ++p) {
      const int k = p << (L->lev - st);
      const double a = -2.0 * M_PI * (double)k / (double)n;
      const int t = (1 << (st - 1)) - 1 + p;
      tw[2 * t] = (float)std::cos(a);
      tw[2 * t + 1] = (float)std::sin(a);
    }
  CMG_CUDA(cudaMemcpyAsync(L->fft_tw, tw.data(), sizeof(float) * 2 * n, cudaMemcpyHostToDevice, s));
  const MgLev &g = L->mg[0];
  k_fft_map<<<blocks_for(g.n), kThreads, 0, s>>>(g.keys, g.n, no, L->fft_map);
  CMG_CUDA(cudaGetLastError());
  CMG_CUDA(cudaStreamSynchronize(s));
  L->fft_buf = buf;
}

// e (phi32 of MG level 0) = the FFT solution of the FP32 correction equation
// whose right-hand side is g32 of MG level 0.
void fft_solve32(cmg_level *L) {
  const MgLev &g = L->mg[0];
  const int n = 1 << L->lev, logn = L->lev;
  cudaStream_t s = L->ctx->stream;
  const int lines = std::max(1, std::min(2048 / n, n * n));  // x passes: <= 16 KB of lines per block
  const int tx = std::min(16, n);                           // y / z passes: columns per block (128-byte rows)
  int logtx = 0;
  while ((1 << logtx) < tx) ++logtx;
  const size_t smx = sizeof(float2) * ((size_t)n + (size_t)lines * line_ld(n));
  const size_t smyz = sizeof(float2) * ((size_t)n + (size_t)tx * line_ld(n));
  const int64_t lines_total = (int64_t)n * n;
  const unsigned bx = (unsigned)(lines_total / lines), byz = (unsigned)((int64_t)n * (n / tx));
  // algorithmic work per pass: one read and one write of the dense complex
  // array (x passes: one FP32 field value per cell instead), 5 n log2 n flops
  // per line transform
  const double cells = (double)n * n * n, line_flops = 5.0 * cells * logn;
  static int attr_dev = -1;
  if (attr_dev != L->ctx->device) {  // n = 512: 16 columns x 545 x 8 B > 48 KB
    CMG_CUDA(cudaFuncSetAttribute(k_fft_yz<1, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    CMG_CUDA(cudaFuncSetAttribute(k_fft_yz<2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    CMG_CUDA(cudaFuncSetAttribute(k_fft_yz<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    attr_dev = L->ctx->device;
  }
  {
    LaunchScope ls(L->ctx, K_FFT, cells * (4.0 + 4.0 + 8.0), line_flops);
    k_fft_x_fwd<<<bx, kFftThreads, smx, s>>>(g.g32, g.n * 4, L->fft_map, L->fft_tw, n, logn, lines, L->fft_buf);
  }
  {
    LaunchScope ls(L->ctx, K_FFT, cells * 16.0, line_flops);
    k_fft_yz<1, 0><<<byz, kFftThreads, smyz, s>>>(L->fft_buf, L->fft_tw, n, logn, logtx);
  }
  {
    LaunchScope ls(L->ctx, K_FFT, cells * 16.0, 2.0 * line_flops + 6.0 * cells);
    k_fft_yz<2, 2><<<byz, kFftThreads, smyz, s>>>(L->fft_buf, L->fft_tw, n, logn, logtx);
  }
  {
    LaunchScope ls(L->ctx, K_FFT, cells * 16.0, line_flops);
    k_fft_yz<1, 1><<<byz, kFftThreads, smyz, s>>>(L->fft_buf, L->fft_tw, n, logn, logtx);
  }
  {
    LaunchScope ls(L->ctx, K_FFT, cells * (8.0 + 4.0 + 4.0), line_flops);
    k_fft_x_inv<<<bx, kFftThreads, smx, s>>>(L->fft_buf, L->fft_map, L->fft_tw, n, logn, lines,
                                             1.0f / ((float)n * n * n), g.phi32, g.n_alloc * 4);
  }
  CMG_CUDA(cudaGetLastError());
}

}  // namespace cmg
