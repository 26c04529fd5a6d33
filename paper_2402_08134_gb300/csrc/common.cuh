// Shared device helpers for the sm_103a SymNMF kernels: Philox4x32-10,
// warp/block reductions, bounded-wait error reporting.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#define SYMNMF_HD __host__ __device__ __forceinline__
#define SYMNMF_D __device__ __forceinline__

namespace symnmf {

// Error bits written by kernels into the handle's device error word.
enum : unsigned {
  ERR_TIMEOUT = 1u,   // a bounded spin ran out
  ERR_NOTSPD = 2u,    // Cholesky met a non-positive pivot
  ERR_NAN = 4u,       // non-finite value produced
  ERR_BPP_ITERS = 8u  // BPP hit its iteration cap
};

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 4 x 32-bit counter,
// 2 x 32-bit key, 10 rounds of two 32x32->64 multiplies with the Weyl key
// schedule between rounds.
struct Philox4 {
  uint32_t x0, x1, x2, x3;
};

SYMNMF_HD Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)M0 * c0;
    const uint64_t p1 = (uint64_t)M1 * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  return Philox4{c0, c1, c2, c3};
}

enum : uint32_t { TAG_OMEGA = 1u, TAG_INIT = 2u, TAG_SAMPLE = 3u };

template <typename T>
SYMNMF_D T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
SYMNMF_D T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o);
    v = v > w ? v : w;
  }
  return v;
}

// Sum over a block of up to 1024 threads; every thread gets the result.
template <typename T>
SYMNMF_D T block_sum(T v, T* sh /* >= 32 entries */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  T t = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  T r = sh[0];
  __syncthreads();
  return r;
}

// Last-block-done reduction of per-block partials: no block ever waits.
template <int NV>
__device__ inline bool last_block(unsigned* counter) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

SYMNMF_D void set_error(unsigned* err, unsigned bit) {
  if (err) atomicOr(err, bit);
}

// Sum of per-block partials ws[b * stride + v] over b < nblocks for v < nv,
// by every thread of the calling block (strided over b, then a block tree):
// a fixed order, so the result is deterministic.  out[v] receives the sums.
SYMNMF_D void reduce_partials(const double* ws, int stride, int nv, unsigned nblocks, double* out,
                              double* sh /* >= 32 */) {
  for (int v = 0; v < nv; ++v) {
    double a = 0.0;
    for (unsigned b = threadIdx.x; b < nblocks; b += blockDim.x) a += __ldcg(ws + (size_t)b * stride + v);
    a = block_sum(a, sh);
    if (threadIdx.x == 0) out[v] = a;
  }
}

SYMNMF_D uint64_t mulhi_u64(uint64_t a, uint64_t b) { return __umul64hi(a, b); }

}  // namespace symnmf
