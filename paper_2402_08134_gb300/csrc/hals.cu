// The full-X HALS update (Eq. symhals_update2), one kernel per padded width.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "hals_row.cuh"
#include "kernels.h"

namespace symnmf {

constexpr int HALS_THREADS = 128;

// Threads per row of the full-X HALS kernel.  A split over a lane pair (half
// the registers, twice the warps) measured slower at k = 64 (766 vs 664 us at
// n = 10^6): the shuffle joins every column's dependency chain, which is bound
// by shared-memory load latency already.
template <int KMAX>
constexpr int hals_ns() {
  return 1;
}

// Widths at which the column loop runs rolled, in rotating blocks of 16
// (hals_row_rotating): the fully unrolled 64-column body misses the
// instruction cache.
template <int KMAX>
constexpr bool hals_rot() {
  return KMAX >= 48;
}

// Full-X HALS update, Eq. symhals_update2:
//   w_i <- max(0, (Y_i + alpha h_i - sum_{j != i} w_j G_ji) / (G_ii + alpha)),
// i = 0..k-1 in order with the columns already updated.  NS = hals_ns threads
// per row, each holding its KMAX / NS columns of F_upd in registers and of Y
// in its own column of shared memory (zero padded; 16-byte loads when VEC).
// G with its diagonal zeroed and the reciprocals 1 / (G_ii + alpha) sit in
// shared memory, read as broadcasts.  With U given, the row of Y is formed as
// U_r M (LAI, M = Lambda U^T F_fix in shared memory).  Persistent grid over
// rows; F_upd . Y and ||F_upd - F_fix||^2 are kept per thread in double-float
// and reduced in FP64.
template <int KMAX, bool VEC>
__global__ void __launch_bounds__(HALS_THREADS) hals_kernel(
    float* __restrict__ Fu, const float* __restrict__ Ff, int64_t n, int k, const float* __restrict__ G, float alpha,
    const float* __restrict__ Y, int ldy, const float* __restrict__ U, int l, const float* __restrict__ M,
    double* part, double* ws, unsigned* counter, unsigned* err) {
  constexpr int NS = hals_ns<KMAX>(), KH = KMAX / NS;
  constexpr bool ROT = hals_rot<KMAX>();
  constexpr int RS = ROT ? 2 * KMAX : hals_split_stride<KMAX, NS>();
  constexpr int RPB = HALS_THREADS / NS;  // rows per block and pass
  extern __shared__ __align__(16) float sm[];
  float* Gs = sm;               // KMAX x RS, diagonal zeroed
  float* inv = Gs + KMAX * RS;  // KMAX
  float* Ys = inv + KMAX;       // KH x HALS_THREADS: each thread's row of Y, column-major
  float* Ms = Ys + KH * HALS_THREADS;  // l x KMAX (LAI only)
  const int tid = threadIdx.x;
  for (int e = tid; e < KMAX * KMAX; e += HALS_THREADS) {
    const int i = e / KMAX, j = e - i * KMAX;
    const int part = j / KH;
    const float v = (i < k && j < k && i != j) ? G[i * k + j] : 0.f;
    Gs[i * RS + part * (NS > 1 ? KH + 4 : KH) + (j - part * KH)] = v;
    if constexpr (ROT) Gs[i * RS + KMAX + j] = v;  // each row twice (rotated reads)
  }
  if (U)
    for (int e = tid; e < l * KMAX; e += HALS_THREADS) {
      const int i = e / KMAX, j = e - i * KMAX;
      Ms[e] = j < k ? M[i * k + j] : 0.f;
    }
  if (tid < KMAX) inv[tid] = tid < k ? 1.0f / (G[tid * k + tid] + alpha) : 0.f;
  __syncthreads();

  const int p = NS > 1 ? (tid & 1) : 0;            // this thread's part of its row
  const unsigned mask = NS > 1 ? 3u << (tid & 30) : 0xffffffffu;
  const int c0 = p * KH;                             // its first column
  const float4* Gp4 = reinterpret_cast<const float4*>(Gs + p * (KH + 4));
  const float4* Ms4 = reinterpret_cast<const float4*>(Ms + c0);
  float2 trv = make_float2(0.f, 0.f), ddv = make_float2(0.f, 0.f);
  bool bad = false;
  float* ys = Ys + tid;  // this thread's column: y_c at ys[c * HALS_THREADS] (no bank conflicts)
  for (int64_t r = (int64_t)blockIdx.x * RPB + tid / NS; r < n; r += (int64_t)gridDim.x * RPB) {
    float w[KH];
    float* fu = Fu + r * k + c0;
    const float* fx = Ff + r * k + c0;
    if constexpr (VEC) {
#pragma unroll
      for (int q = 0; q < KH / 4; ++q) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c0 + 4 * q < k) v = __ldg(reinterpret_cast<const float4*>(fu) + q);
        w[4 * q] = v.x, w[4 * q + 1] = v.y, w[4 * q + 2] = v.z, w[4 * q + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int c = 0; c < KH; ++c) w[c] = c0 + c < k ? __ldg(fu + c) : 0.f;
    }
    // this row of Y into shared memory (read once per column there: fewer registers)
    if (U) {  // Y_r = U_r M (LAI product fused into the update)
      float y[KH];
#pragma unroll
      for (int c = 0; c < KH; ++c) y[c] = 0.f;
      const float* ur = U + r * l;
#pragma unroll 2
      for (int pp = 0; pp < l; ++pp) {
        const float u = __ldg(ur + pp);
#pragma unroll
        for (int q = 0; q < KH / 4; ++q) {
          const float4 m = Ms4[pp * (KMAX / 4) + q];
          y[4 * q + 0] = fmaf(u, m.x, y[4 * q + 0]);
          y[4 * q + 1] = fmaf(u, m.y, y[4 * q + 1]);
          y[4 * q + 2] = fmaf(u, m.z, y[4 * q + 2]);
          y[4 * q + 3] = fmaf(u, m.w, y[4 * q + 3]);
        }
      }
#pragma unroll
      for (int c = 0; c < KH; ++c) ys[c * HALS_THREADS] = y[c];
    } else if constexpr (VEC) {
      const float* yr = Y + r * ldy + c0;
#pragma unroll
      for (int q = 0; q < KH / 4; ++q) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c0 + 4 * q < k) v = __ldg(reinterpret_cast<const float4*>(yr) + q);
        ys[(4 * q) * HALS_THREADS] = v.x, ys[(4 * q + 1) * HALS_THREADS] = v.y;
        ys[(4 * q + 2) * HALS_THREADS] = v.z, ys[(4 * q + 3) * HALS_THREADS] = v.w;
      }
    } else {
#pragma unroll
      for (int c = 0; c < KH; ++c) ys[c * HALS_THREADS] = c0 + c < k ? __ldg(Y + r * ldy + c0 + c) : 0.f;
    }
    // the fixed row is read column by column (L1 hits after the first); the
    // shared-memory column of Y is this thread's own, so no barrier is needed
    if constexpr (ROT)
      bad |= hals_row_rotating<KMAX, 16>(
          w, [&](int c) { return ys[c * HALS_THREADS]; }, alpha, k, Gs, inv, [&](int c) { return __ldg(fx + c); },
          trv, ddv);
    else
      bad |= hals_row_split<KMAX, NS>(
          w, [&](int c) { return ys[c * HALS_THREADS]; }, alpha, k, p, mask, Gp4, inv,
          [&](int c) { return __ldg(fx + c); }, trv, ddv);
    if constexpr (VEC) {
#pragma unroll
      for (int q = 0; q < KH / 4; ++q)
        if (c0 + 4 * q < k)
          reinterpret_cast<float4*>(fu)[q] = make_float4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
    } else {
#pragma unroll
      for (int c = 0; c < KH; ++c)
        if (c0 + c < k) fu[c] = w[c];
    }
  }
  if (bad) set_error(err, ERR_NAN);
  __shared__ double sh[32];
  const double tr = block_sum((double)trv.x + (double)trv.y, sh);
  const double dd = block_sum((double)ddv.x + (double)ddv.y, sh);
  if (tid == 0) {
    ws[2 * blockIdx.x] = tr;
    ws[2 * blockIdx.x + 1] = dd;
  }
  if (last_block<1>(counter)) {
    reduce_partials(ws, 2, 2, gridDim.x, part, sh);
    if (tid == 0) *counter = 0;
  }
}

template <int KMAX, bool VEC>
static cudaError_t launch_hals(float* Fu, const float* Ff, int64_t n, int k, const float* G, double alpha,
                               const float* Y, int ldy, const float* U, int l, const float* M, double* part,
                               double* ws, unsigned* counter, unsigned* err, cudaStream_t st) {
  const int rs = hals_rot<KMAX>() ? 2 * KMAX : hals_split_stride<KMAX, hals_ns<KMAX>()>();
  size_t smem = (size_t)(KMAX * rs + KMAX + (KMAX / hals_ns<KMAX>()) * HALS_THREADS) * 4;
  if (U) smem += (size_t)l * KMAX * 4;
  auto kern = hals_kernel<KMAX, VEC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, HALS_THREADS, smem);
  if (e != cudaSuccess) return e;
  const int64_t rpb = HALS_THREADS / hals_ns<KMAX>();
  const int64_t tiles = (n + rpb - 1) / rpb;
  // at most 2048 blocks: one FP64 partial pair per block in ws
  int grid = (int)std::min<int64_t>(tiles, (int64_t)num_sms() * std::min(std::max(per_sm, 1), 8));
  grid = std::max(1, std::min(grid, 2048));
  kern<<<grid, HALS_THREADS, smem, st>>>(Fu, Ff, n, k, G, (float)alpha, Y, ldy, U, l, M, part, ws, counter, err);
  count_launches(1);
  return cudaGetLastError();
}

template <int KMAX>
static cudaError_t launch_hals_v(float* Fu, const float* Ff, int64_t n, int k, const float* G, double alpha,
                                 const float* Y, int ldy, const float* U, int l, const float* M, double* part,
                                 double* ws, unsigned* counter, unsigned* err, cudaStream_t st) {
  const bool vec = (k % 4) == 0 && (ldy % 4) == 0 &&
                   (((uintptr_t)Fu | (uintptr_t)Ff | (uintptr_t)(Y ? Y : Fu)) & 15) == 0;
  return vec ? launch_hals<KMAX, true>(Fu, Ff, n, k, G, alpha, Y, ldy, U, l, M, part, ws, counter, err, st)
             : launch_hals<KMAX, false>(Fu, Ff, n, k, G, alpha, Y, ldy, U, l, M, part, ws, counter, err, st);
}

cudaError_t hals_update(float* F_upd, const float* F_fix, int64_t n, int k, const float* G, double alpha,
                        const float* Y, int ldy, const float* U, int l, const float* M, double* part, double* ws,
                        unsigned* counter, unsigned* err, cudaStream_t st) {
  if (k < 1 || n < 0) return cudaErrorInvalidValue;
#define SYMNMF_HALS(KM) \
  return launch_hals_v<KM>(F_upd, F_fix, n, k, G, alpha, Y, ldy, U, l, M, part, ws, counter, err, st)
  if (k <= 8) SYMNMF_HALS(8);
  if (k <= 16) SYMNMF_HALS(16);
  if (k <= 20) SYMNMF_HALS(20);
  if (k <= 24) SYMNMF_HALS(24);
  if (k <= 32) SYMNMF_HALS(32);
  if (k <= 48) SYMNMF_HALS(48);
  if (k <= 64) SYMNMF_HALS(64);
#undef SYMNMF_HALS
  return cudaErrorInvalidValue;
}

}  // namespace symnmf
