// noalloc.cu -- cmg_residual_norm2_noalloc: the squared residual norm of one
// level computed from caller-provided device arrays, with no device memory
// allocated by the call.
//
// Why it exists: the level objects of this library allocate their tables and
// fields with cudaMalloc when they are built, and the library's residual norm
// reduces through a scratch buffer owned by the level.  Some callers cannot
// allocate at the moment they need a residual check: real-time solver loops
// that forbid allocation after start-up (cudaMalloc may block and synchronise
// the device), and hosts whose device memory is a fixed arena handed out by
// their own allocator.  This entry point reads arrays the caller already owns
// and reduces through a fixed-size scratch array compiled into the library
// instead.
//
// The scratch address is looked up once per device and kept for the life of
// the process; a cudaDeviceReset in the caller's process invalidates it, and
// the entry point must not be used after one.
//
// The scratch array lives in the library image: every GPU that loads the
// library holds its 512 KiB until the process exits.  All calls share it, so
// calls that overlap on the GPU (different streams, concurrent graphs) race
// and must be serialised by the caller.  Each block writes its own slot and
// the final sum reads only the slots of the current call, so nothing has to
// be cleared between calls.
#include <mutex>

#include "cmg_internal.cuh"

namespace {

constexpr int kNaThreads = 256;
constexpr int64_t kNaMaxOcts = int64_t(1) << 24;
constexpr int kNaMaxBlocks = (int)(kNaMaxOcts / kNaThreads);
constexpr int kNaMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNaMaxBlocks];

std::mutex g_na_mu;
void *g_na_scratch[kNaMaxDevices] = {};

// r = f - (sum of the 6 face neighbours - 6 phi) / h^2 per cell (Sec. 5.1.1
// item (iii)); a missing neighbour (-1 in the cache) takes the ghost value
// when ghosts are given, else 0.  Public layouts: neighbours [n][7], ghosts
// [n][6][4] (face cells in increasing child index), phi and f [n][8].
__global__ void __launch_bounds__(kNaThreads)
    k_residual_norm_public(const int32_t *__restrict__ nbr, const double *__restrict__ ghosts,
                           const double *__restrict__ phi, const double *__restrict__ f, int64_t n, double inv_h2,
                           double *__restrict__ partials) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (i < n) {
    for (int c = 0; c < 8; ++c) {
      double s = 0.0;
      for (int d = 0; d < 6; ++d) {
        const int a = d >> 1, side = d & 1, c2 = c ^ (1 << a);
        double v;
        if (((c >> a) & 1) != side) {
          v = phi[i * 8 + c2];
        } else {
          const int32_t o = nbr[i * 7 + 1 + d];
          if (o >= 0) {
            v = phi[(int64_t)o * 8 + c2];
          } else if (ghosts) {
            const int q = a == 0 ? (c >> 1) : a == 1 ? ((c & 1) | ((c >> 2) << 1)) : (c & 3);
            v = ghosts[(i * 6 + d) * 4 + q];
          } else {
            v = 0.0;
          }
        }
        s += v;
      }
      const double r = f[i * 8 + c] - (s - 6.0 * phi[i * 8 + c]) * inv_h2;
      acc = fma(r, r, acc);
    }
  }
  __shared__ double ws[kNaThreads / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < kNaThreads / 32 ? ws[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) partials[blockIdx.x] = w;
  }
}

__global__ void k_sum_partials(const double *__restrict__ partials, int nb, double *__restrict__ out) {
  __shared__ double ws[32];
  double v = 0.0;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) v += partials[t];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) *out = w;
  }
}

}  // namespace

extern "C" int cmg_residual_norm2_noalloc(const int32_t *neighbors, const double *ghosts, const double *phi,
                                          const double *f, int64_t n_octs, double h, double *norm2, void *stream) {
  if (!norm2 || n_octs < 0 || !(h > 0.0) || (n_octs > 0 && (!neighbors || !phi || !f))) return CMG_ERR_INVALID_ARG;
  if (n_octs > kNaMaxOcts) return CMG_ERR_INVALID_ARG;  // the static scratch holds 2^16 block sums
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
    cudaGetLastError();
    return CMG_ERR_CUDA;
  }
  void *scratch = nullptr;
  {
    // one-time set-up per device, with that device current: the address of
    // the static array (a host-side stand-in is not a device address)
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_scratch[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) {
        cudaGetLastError();
        return CMG_ERR_CUDA;
      }
      g_na_scratch[dev] = p;
    }
    scratch = g_na_scratch[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n_octs == 0) {
    if (cudaMemsetAsync(norm2, 0, sizeof(double), s) != cudaSuccess) {
      cudaGetLastError();
      return CMG_ERR_CUDA;
    }
    return CMG_OK;
  }
  const int nb = (int)((n_octs + kNaThreads - 1) / kNaThreads);
  k_residual_norm_public<<<nb, kNaThreads, 0, s>>>(neighbors, ghosts, phi, f, n_octs, 1.0 / (h * h),
                                                    static_cast<double *>(scratch));
  k_sum_partials<<<1, 1024, 0, s>>>(static_cast<const double *>(scratch), nb, norm2);
  if (cudaGetLastError() != cudaSuccess) return CMG_ERR_CUDA;
  return CMG_OK;
}
