// Device side of checked launches (TP_EXEC_CHECKED): before a program stores
// a tile it claims the tile's bit in the context's claim bitmap. A bit that
// is already set means a second program is about to write the same
// sub-tensor (a data race in the sense of Appendix A); the claim fails and
// the context's error word records kDevRace. Off-map tiles record kDevRace as
// well. The bitmap starts a launch all clear: every checked launch counts its
// claimants (CTAs, or the GEMM's epilogue warps) as they make their last
// claim, and the last one clears the bits the launch could have set, so the
// next launch (and every replay of a captured one) starts clear without a
// memset.
#pragma once

#include <cstdint>

#include "tp_internal.h"

namespace tp {

__device__ __forceinline__ void record_device_error(int* err, int code) { atomicCAS(err, 0, code); }

// Returns true when this call set bit `id` (the caller may store).
__device__ __forceinline__ bool claim_tile(uint32_t* bits, int64_t id, int* err) {
  const uint32_t m = 1u << (uint32_t)(id & 31);
  const uint32_t old = atomicOr(bits + (id >> 5), m);
  if (old & m) {
    record_device_error(err, kDevRace);
    return false;
  }
  return true;
}

// Called by all threads of every CTA of a checked launch after the CTA's
// last claim (block-uniform). `done` counts finished CTAs; the CTA that
// finishes last clears the first `bits` bits and resets the counter. Uses no
// shared memory (the result is broadcast through the barrier).
__device__ __forceinline__ void claims_finish(uint32_t* claims, int64_t bits, unsigned* done, unsigned ctas) {
  __syncthreads();
  int mine = 0;
  if (threadIdx.x == 0) {
    __threadfence();
    mine = atomicAdd(done, 1u) == ctas - 1u;
  }
  if (__syncthreads_or(mine)) {
    __threadfence();
    const int64_t words = (bits + 31) / 32;
    for (int64_t i = threadIdx.x; i < words; i += blockDim.x) claims[i] = 0u;
    if (threadIdx.x == 0) *done = 0u;
  }
}

}  // namespace tp
