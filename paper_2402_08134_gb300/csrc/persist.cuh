// Bounded grid barrier for the persistent cooperative kernels.
#pragma once

#include "common.cuh"

namespace symnmf {

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The arrival counter (bar[0]) and the generation word (bar[GRID_GEN]) sit in
// different 128-byte lines, so that the spinning readers of the generation do
// not contend with the arrivals.  bar must hold 2 * GRID_GEN words, zeroed
// before the launch.  Waits are bounded (1 s of %globaltimer): on expiry the
// waiting CTA sets ERR_TIMEOUT and every CTA leaves at its next barrier.
// Returns false (on every thread of the block) when the barrier gave up.
constexpr int GRID_GEN = 32;

__device__ inline bool grid_sync_bounded(unsigned* bar, unsigned* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + GRID_GEN;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    ok = 1;
    if (arrived == gridDim.x) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + GRID_GEN, 1u);
    } else {
      const uint64_t t0 = global_timer_ns();
      unsigned spins = 0;
      while (*gen == g) {
        __nanosleep(32);
        if ((++spins & 63u) == 0) {
          if (*(volatile unsigned*)err & ERR_TIMEOUT) {
            ok = 0;
            break;
          }
          if (global_timer_ns() - t0 > 1000000000ull) {
            atomicOr(err, ERR_TIMEOUT);
            ok = 0;
            break;
          }
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace symnmf
