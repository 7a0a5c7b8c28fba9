// brick.cu -- red-black colour passes of full periodic levels stored in
// lexicographic oct order (x fastest), with each CTA's block of octs and its
// face halo staged in shared memory (App. D.2 Eq. (gs_update); App. D.1 and
// Sec. 9.4 describe the neighbour access this replaces).
//
// A CTA owns a brick of 16 x 4 x 4 octs (one per thread).  It first copies
// the other colour of the brick and of the octs across its six faces
// (256 + 288 = 544 octs, 4 values each) into shared memory with coalesced
// 16-byte loads, each thread its own oct and one face oct (the first warp a
// second), wrapping periodically by masks, then updates its octs from shared
// memory: no neighbour-table reads (the
// neighbours of oct (x, y, z) are (x +- 1, y, z), ... modulo the grid) and no
// scattered global gathers.  Each cell forms the same six operands in the
// same order as the table kernel and sums them with nbsum6, so the two
// kernels produce the same bits.
//
// Shared memory holds the staged values slot-major ([4][box]), so that the
// 32 lanes of a warp, which own 16 consecutive x of two rows, read
// consecutive addresses of one slot (no bank conflicts).
#include "oct_ops.cuh"

namespace cmg {
namespace {

constexpr int kBX = 16, kBY = 4, kBZ = 4;
constexpr int kSX = kBX + 2, kSY = kBY + 2, kSZ = kBZ + 2;
constexpr int kBox = kSX * kSY * kSZ;
constexpr int kBrickThreads = kBX * kBY * kBZ;

__device__ __forceinline__ int box_at(int lx, int ly, int lz) { return ((lz + 1) * kSY + (ly + 1)) * kSX + (lx + 1); }

template <typename T>
struct Vec;
template <>
struct Vec<double> {
  using V = double2;
  static constexpr int per_oct = 2;
  __device__ static void put(double *sm, int si, int v, V x) {
    sm[(2 * v) * kBox + si] = x.x;
    sm[(2 * v + 1) * kBox + si] = x.y;
  }
};
template <>
struct Vec<float> {
  using V = float4;
  static constexpr int per_oct = 1;
  __device__ static void put(float *sm, int si, int, V x) {
    sm[0 * kBox + si] = x.x;
    sm[1 * kBox + si] = x.y;
    sm[2 * kBox + si] = x.z;
    sm[3 * kBox + si] = x.w;
  }
};

// Octs staged besides the brick itself: the y faces (2 x 16 x 4), the z faces
// (2 x 16 x 4) and the x faces (2 x 4 x 4), as face index f in [0, 288):
// thread t stages its own oct, face oct t, and face oct 256 + t if t < 32.
__device__ __forceinline__ void face_oct(int f, int &lx, int &ly, int &lz) {
  if (f < 128) {  // y faces
    lx = f & 15;
    lz = (f >> 4) & 3;
    ly = (f >> 6) ? kBY : -1;
  } else if (f < 256) {  // z faces
    const int r = f - 128;
    lx = r & 15;
    ly = (r >> 4) & 3;
    lz = (r >> 6) ? kBZ : -1;
  } else {  // x faces
    const int r = f - 256;
    ly = r & 3;
    lz = (r >> 2) & 3;
    lx = (r >> 4) ? kBX : -1;
  }
}

template <typename T>
__device__ __forceinline__ void stage_oct(T *sm, const T *src, int x, int y, int z, int lg, int si) {
  using VT = typename Vec<T>::V;
  const int msk = (1 << lg) - 1;
  const int64_t gi = (int64_t)(x & msk) + (((int64_t)(y & msk) + ((int64_t)(z & msk) << lg)) << lg);
#pragma unroll
  for (int v = 0; v < Vec<T>::per_oct; ++v) Vec<T>::put(sm, si, v, reinterpret_cast<const VT *>(src + gi * 4)[v]);
}

template <typename T, int P>
__global__ void __launch_bounds__(kBrickThreads) k_sweep_brick(const T *__restrict__ src, T *__restrict__ dst,
                                                               const T *__restrict__ g, int lg) {
  static_assert(kBX == 16 && kBY == 4 && kBZ == 4 && kBrickThreads == 256, "face_oct assumes a 16 x 4 x 4 brick");
  __shared__ __align__(16) T sm[4 * kBox];
  const int nbx_log = lg - 4, nby_log = lg - 2;  // bricks per axis: npd / 16, npd / 4
  const int b = blockIdx.x;
  const int x0 = (b & ((1 << nbx_log) - 1)) << 4;
  const int y0 = ((b >> nbx_log) & ((1 << nby_log) - 1)) << 2;
  const int z0 = (b >> (nbx_log + nby_log)) << 2;
  const int tx = threadIdx.x & 15, ty = (threadIdx.x >> 4) & 3, tz = threadIdx.x >> 6;
  const int64_t i = (int64_t)(x0 + tx) + (((int64_t)(y0 + ty) + ((int64_t)(z0 + tz) << lg)) << lg);
  // every read waits for the preceding kernel: on a coarse MG level it is the
  // restriction that writes this level's source
  pdl_enter();
  const int own = box_at(tx, ty, tz);
  stage_oct(sm, src, x0 + tx, y0 + ty, z0 + tz, lg, own);
  {
    int lx, ly, lz;
    face_oct(threadIdx.x, lx, ly, lz);
    stage_oct(sm, src, x0 + lx, y0 + ly, z0 + lz, lg, box_at(lx, ly, lz));
    if (threadIdx.x < 32) {
      face_oct(256 + threadIdx.x, lx, ly, lz);
      stage_oct(sm, src, x0 + lx, y0 + ly, z0 + lz, lg, box_at(lx, ly, lz));
    }
  }
  T gv[4];
  dev::load4<false>(g + i * 4, gv);
  __syncthreads();
  const T inv6 = T(1) / T(6);
  T out[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = plane_cell(P, q);
    T v[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      const int a = d >> 1, side = d & 1, c2 = c ^ (1 << a);
      int at = own;
      if (((c >> a) & 1) == side) {
        const int step = side ? 1 : -1;
        at += a == 0 ? step : a == 1 ? step * kSX : step * kSX * kSY;
      }
      v[d] = sm[(c2 >> 1) * kBox + at];
    }
    out[q] = dev::fma_t(dev::nbsum6(v), inv6, gv[q]);
  }
  dev::store4(dst + i * 4, out);
}

// keys[i] == Morton key of oct (i mod npd, (i / npd) mod npd, i / npd^2)
__global__ void k_check_lexicographic(const uint64_t *__restrict__ keys, int64_t n, int lg, int *__restrict__ bad) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t m = (1u << lg) - 1u;
  const uint64_t want = morton_encode((uint32_t)(i & m), (uint32_t)((i >> lg) & m), (uint32_t)(i >> (2 * lg)));
  if (keys[i] != want) atomicExch(bad, 1);
}

}  // namespace

template <typename T>
void brick_pass(cmg_level *L, int m, int colour) {
  MgLev &g = L->mg[m];
  const int lg = g.lex_log2;
  if (lg < 4) throw Error(CMG_ERR_INVALID_ARG, "brick pass on a level that is not a lexicographic full grid");
  T *phi = sizeof(T) == 8 ? (T *)g.phi : (T *)g.phi32;
  const T *gg = sizeof(T) == 8 ? (const T *)g.g : (const T *)g.g32;
  const int64_t st = g.n_alloc * 4;
  const unsigned grid = (unsigned)(g.n / kBrickThreads);
  // the whole 8 cells of a colour pass: other colour, source, result (the
  // neighbours are implicit: no index bytes)
  const double u = 4.0 * (double)g.n;
  LaunchScope ls(L->ctx, sizeof(T) == 8 ? K_SWEEP64 : K_SWEEP32, 3.0 * u * sizeof(T), 7.0 * u);
  if (colour == 0)
    launch_k(k_sweep_brick<T, 0>, grid, kBrickThreads, L->ctx->stream, phi + st, phi, gg, lg);
  else
    launch_k(k_sweep_brick<T, 1>, grid, kBrickThreads, L->ctx->stream, phi, phi + st, gg + g.n * 4, lg);
  CMG_CUDA(cudaGetLastError());
}
template void brick_pass<double>(cmg_level *, int, int);
template void brick_pass<float>(cmg_level *, int, int);

void mark_lexicographic(cmg_level *L) {
  for (auto &g : L->mg) g.lex_log2 = -1;
  if (!L->periodic_full || L->nx != 1) return;
  cudaStream_t s = L->ctx->stream;
  int *flag = L->mem.alloc<int>(L->mg.size(), true, s);
  for (size_t k = 0; k < L->mg.size(); ++k) {
    const MgLev &g = L->mg[k];
    const int lg = g.lev - 1;
    if (lg < 4 || lg > 20 || g.n != (int64_t(1) << (3 * lg)) || !g.all_active) continue;
    k_check_lexicographic<<<blocks_for(g.n), kThreads, 0, s>>>(g.keys, g.n, lg, flag + k);
    CMG_CUDA(cudaGetLastError());
  }
  std::vector<int> bad(L->mg.size());
  CMG_CUDA(cudaMemcpyAsync(bad.data(), flag, sizeof(int) * bad.size(), cudaMemcpyDeviceToHost, s));
  CMG_CUDA(cudaStreamSynchronize(s));
  for (size_t k = 0; k < L->mg.size(); ++k) {
    MgLev &g = L->mg[k];
    const int lg = g.lev - 1;
    if (lg < 4 || lg > 20 || g.n != (int64_t(1) << (3 * lg)) || !g.all_active) continue;
    if (!bad[k]) g.lex_log2 = lg;
  }
}

}  // namespace cmg
