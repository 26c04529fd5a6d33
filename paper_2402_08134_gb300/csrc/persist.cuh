// Bounded grid barrier for the persistent cooperative kernels.
#pragma once

#include "common.cuh"

namespace symnmf {

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Spin until *word >= target (acquire loads at GPU scope), for at most
// limit_ns of %globaltimer after the first 64 polls.  On expiry the waiter
// sets ERR_TIMEOUT in *err and returns false; it also gives up (false) as soon
// as it sees ERR_TIMEOUT already set by another waiter.  Every wait of the
// persistent kernels goes through here.
__device__ inline bool bounded_wait_geq(const unsigned* word, unsigned target, unsigned* err, uint64_t limit_ns) {
  uint64_t t0 = 0;
  for (unsigned spins = 1;; ++spins) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(word) : "memory");
    if (v >= target) return true;
    if (spins > 32u) __nanosleep(32);
    if ((spins & 63u) == 0) {
      if (*(volatile unsigned*)err & ERR_TIMEOUT) return false;
      const uint64_t now = global_timer_ns();
      if (t0 == 0) {
        t0 = now;
      } else if (now - t0 > limit_ns) {
        atomicOr(err, ERR_TIMEOUT);
        return false;
      }
    }
  }
}

constexpr uint64_t GRID_WAIT_LIMIT_NS = 1000000000ull;  // 1 s

// Grid barrier on a monotonic arrival counter bar[0] (zeroed before the
// launch).  Barrier number e (1, 2, ...) of the launch completes when the
// counter reaches e * gridDim.x: every CTA adds 1 (a fire-and-forget
// reduction with release semantics that publishes its writes) and thread 0 waits for
// the target with bounded_wait_geq (1 s).  `epoch` counts the barriers passed
// (thread 0's copy is the one used).  On expiry the waiting CTA sets
// ERR_TIMEOUT, and every CTA that sees that bit leaves at its next barrier.
// Returns false (on every thread of the block) when the barrier gave up.
__device__ inline bool grid_sync_bounded(unsigned* bar, unsigned* err, unsigned& epoch) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    epoch += 1u;
    const unsigned target = epoch * gridDim.x;
    // the release reduction publishes every write the CTA made before the
    // __syncthreads above (0.3 us cheaper than a full fence and an atomic)
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(bar), "r"(1u) : "memory");
    ok = bounded_wait_geq(bar, target, err, GRID_WAIT_LIMIT_NS) ? 1 : 0;
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace symnmf
