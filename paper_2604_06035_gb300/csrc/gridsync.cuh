// gridsync.cuh -- grid-wide barrier for cooperative launches, with bounded
// waits.
//
// One 32-bit word per barrier object, starting at 0.  Thread 0 of every CTA
// adds to it once per barrier: CTA 0 adds 2^31 - (CTAs - 1), every other CTA
// adds 1, so the adds of one barrier total exactly 2^31.  The top bit of the
// word therefore flips at the last arrival and at no other moment of that
// barrier (all partial sums keep it), and the low bits return to where they
// were -- no reset step.  A CTA waits until the top bit differs from the one
// its own add returned.  The add has release and the polling load acquire
// semantics at GPU scope; the block barriers around them extend the ordering
// to the CTA's other threads.  A wait longer than budget SM clock cycles
// records CMG_ERR_TIMEOUT in *err and gives up; once *err holds it, no
// barrier waits any more, so a failed launch always ends.
#pragma once

#include "cmg.h"

namespace cmg {
namespace dev {

__device__ __forceinline__ unsigned atom_add_release_gpu(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.release.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Returns false when this barrier (or an earlier one) gave up.
__device__ __forceinline__ bool grid_barrier(unsigned *word, int *err, long long budget) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1) : 1u;
    const unsigned old = atom_add_release_gpu(word, inc);
    volatile int *e = err;
    const long long t0 = clock64();
    while (((ld_acquire_gpu(word) ^ old) & 0x80000000u) == 0u) {
      if (*e == CMG_ERR_TIMEOUT) {
        ok = 0;
        break;
      }
      if (clock64() - t0 > budget) {
        atomicCAS(err, 0, (int)CMG_ERR_TIMEOUT);
        ok = 0;
        break;
      }
    }
    if (*e == CMG_ERR_TIMEOUT) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace dev
}  // namespace cmg
