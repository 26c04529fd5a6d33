// Leverage scores of the rows of F (Alg. LvS-SymNMF): l_i = ||h_i R^-1||^2.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace symnmf {

constexpr int LEV_THREADS = 128;

// l_i = ||h_i R^-1||^2 (R^-1 upper triangular, Alg. LvS-SymNMF).  One thread
// per row: z = h R^-1 accumulated by rows of R^-1 (z_j += h_p R^-1_pj for
// j >= p), read as float4 broadcasts from shared memory (KMAX x KMAX, zero
// padded), so every load feeds four FMAs; the row of F in registers, read with
// 16-byte loads when VEC.
template <int KMAX, bool VEC>
__global__ void __launch_bounds__(LEV_THREADS) leverage_kernel(const float* __restrict__ F, int64_t n, int k,
                                                               const float* __restrict__ Rinv, double* lev) {
  __shared__ __align__(16) float Rs[KMAX * KMAX];
  for (int e = threadIdx.x; e < KMAX * KMAX; e += LEV_THREADS) {
    const int p = e / KMAX, j = e - p * KMAX;
    Rs[e] = (p < k && j < k && p <= j) ? Rinv[p * k + j] : 0.f;
  }
  __syncthreads();
  const float4* R4 = reinterpret_cast<const float4*>(Rs);
  for (int64_t r = (int64_t)blockIdx.x * LEV_THREADS + threadIdx.x; r < n; r += (int64_t)gridDim.x * LEV_THREADS) {
    const float* fr = F + r * k;
    float h[KMAX];
    if constexpr (VEC) {
#pragma unroll
      for (int q = 0; q < KMAX / 4; ++q) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (4 * q < k) v = __ldg(reinterpret_cast<const float4*>(fr) + q);
        h[4 * q] = v.x, h[4 * q + 1] = v.y, h[4 * q + 2] = v.z, h[4 * q + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int c = 0; c < KMAX; ++c) h[c] = c < k ? __ldg(fr + c) : 0.f;
    }
    float z[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) z[j] = 0.f;
#pragma unroll
    for (int p = 0; p < KMAX; ++p)
#pragma unroll
      for (int j4 = p / 4; j4 < KMAX / 4; ++j4) {
        const float4 g = R4[p * (KMAX / 4) + j4];
        z[4 * j4 + 0] = fmaf(h[p], g.x, z[4 * j4 + 0]);
        z[4 * j4 + 1] = fmaf(h[p], g.y, z[4 * j4 + 1]);
        z[4 * j4 + 2] = fmaf(h[p], g.z, z[4 * j4 + 2]);
        z[4 * j4 + 3] = fmaf(h[p], g.w, z[4 * j4 + 3]);
      }
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int j = 0; j < KMAX; j += 2) {
      s0 = fmaf(z[j], z[j], s0);
      s1 = fmaf(z[j + 1], z[j + 1], s1);
    }
    lev[r] = (double)(s0 + s1);
  }
}

template <int KMAX>
static void launch_leverage(const float* F, int64_t n, int k, const float* Rinv, double* lev, cudaStream_t st) {
  const int64_t blocks = (n + LEV_THREADS - 1) / LEV_THREADS;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)num_sms() * 8));
  if ((k % 4) == 0 && ((uintptr_t)F & 15) == 0)
    leverage_kernel<KMAX, true><<<grid, LEV_THREADS, 0, st>>>(F, n, k, Rinv, lev);
  else
    leverage_kernel<KMAX, false><<<grid, LEV_THREADS, 0, st>>>(F, n, k, Rinv, lev);
}

cudaError_t leverage_rows(const float* F, int64_t n, int k, const float* Rinv, double* lev,
                          cudaStream_t st) {
  if (k < 1 || k > 64) return cudaErrorInvalidValue;
  if (n < 1) return cudaSuccess;
  if (k <= 8)
    launch_leverage<8>(F, n, k, Rinv, lev, st);
  else if (k <= 16)
    launch_leverage<16>(F, n, k, Rinv, lev, st);
  else if (k <= 24)
    launch_leverage<24>(F, n, k, Rinv, lev, st);
  else if (k <= 32)
    launch_leverage<32>(F, n, k, Rinv, lev, st);
  else if (k <= 48)
    launch_leverage<48>(F, n, k, Rinv, lev, st);
  else
    launch_leverage<64>(F, n, k, Rinv, lev, st);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace symnmf
