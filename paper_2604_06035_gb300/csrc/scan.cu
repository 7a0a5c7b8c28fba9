// scan.cu -- exclusive prefix sum of int32 flags (deterministic numbering of
// coarse MG octs in order of first appearance).  Three passes: per-block scan,
// one-block scan of the block sums, add-back.
#include "cmg_internal.cuh"

namespace cmg {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ int32_t block_exclusive_scan(int32_t v, int32_t *total) {
  __shared__ int32_t warp_sums[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    int32_t w = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) warp_sums[lane] = w;
  }
  __syncthreads();
  const int32_t warp_prefix = wid > 0 ? warp_sums[wid - 1] : 0;
  *total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return warp_prefix + x - v;
}

__global__ void k_scan_tiles(const int32_t *__restrict__ in, int32_t *__restrict__ out, int64_t n,
                             int32_t *__restrict__ tile_sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int32_t v[kScanItems];
  int32_t local = 0;
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    v[t] = (base + t < n) ? in[base + t] : 0;
    local += v[t];
  }
  int32_t total;
  int32_t excl = block_exclusive_scan(local, &total);
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    if (base + t < n) out[base + t] = excl;
    excl += v[t];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void k_scan_sums(int32_t *__restrict__ sums, int64_t nt, int32_t *__restrict__ d_total) {
  int32_t carry = 0;
  for (int64_t base = 0; base < nt; base += kScanThreads) {
    const int64_t i = base + threadIdx.x;
    const int32_t v = i < nt ? sums[i] : 0;
    int32_t total;
    const int32_t excl = block_exclusive_scan(v, &total);
    if (i < nt) sums[i] = carry + excl;
    carry += total;
  }
  if (threadIdx.x == 0) *d_total = carry;
}

__global__ void k_scan_add(int32_t *__restrict__ out, int64_t n, const int32_t *__restrict__ sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  const int32_t add = sums[blockIdx.x];
#pragma unroll
  for (int t = 0; t < kScanItems; ++t)
    if (base + t < n) out[base + t] += add;
}

}  // namespace

int64_t scan_scratch_size(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

void scan_exclusive(const int32_t *in, int32_t *out, int64_t n, int32_t *d_total, int32_t *scratch,
                    int64_t scratch_n, cudaStream_t s) {
  const int64_t nt = (n + kScanTile - 1) / kScanTile;
  if (nt + 1 > scratch_n) throw Error(CMG_ERR_INVALID_ARG, "scan scratch too small");
  if (n == 0) {
    CMG_CUDA(cudaMemsetAsync(d_total, 0, sizeof(int32_t), s));
    return;
  }
  k_scan_tiles<<<(unsigned)nt, kScanThreads, 0, s>>>(in, out, n, scratch);
  k_scan_sums<<<1, kScanThreads, 0, s>>>(scratch, nt, d_total);
  k_scan_add<<<(unsigned)nt, kScanThreads, 0, s>>>(out, n, scratch);
  CMG_CUDA(cudaGetLastError());
}

}  // namespace cmg
