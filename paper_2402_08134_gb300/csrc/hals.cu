// The full-X HALS update (Eq. symhals_update2), one kernel per padded width.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "hals_row.cuh"
#include "kernels.h"

namespace symnmf {

constexpr int HALS_THREADS = 128;
// Column stride (floats) of the staged row tiles: one past the block's rows,
// so that a thread's walk down its own column and the warp's transposing
// stores both spread over the banks.
constexpr int HALS_CS = HALS_THREADS + 1;

// One thread per row.  A split of each row over a lane pair (half the
// registers, twice the warps) measured slower at k = 64 (766 vs 664 us at
// n = 10^6): the shuffle joins every column's dependency chain.

// Widths at which the column loop runs rolled, in rotating blocks of 16
// (hals_row_rotating): the fully unrolled 64-column body misses the
// instruction cache.
template <int KMAX>
constexpr bool hals_rot() {
  return KMAX >= 48;
}

template <int KMAX>
constexpr int hals_gstride() {
  return hals_rot<KMAX>() ? 2 * KMAX : KMAX;
}

// Copy the warp's 32 rows [r0, r0 + 32) of a row-major matrix (row stride ld,
// k columns) into the column-major tile T (column c of tile row t at
// T[c HALS_CS + t], tile rows wrow .. wrow + 31), zero padded past n and k.
// The lanes walk the rows' contiguous span, so each global load instruction
// covers whole cache lines (one row per thread would touch 32 lines per load).
// At 64 columns the 16-byte form is unrolled whole, so that all of a lane's
// loads are issued before its shared-memory stores: the DRAM latency is
// waited out once per tile, not once per few loads.
template <int KMAX, bool VEC>
__device__ __forceinline__ void hals_stage_in(const float* __restrict__ src, int64_t ld, int64_t r0, int64_t n,
                                              int k, float* T, int wrow, int lane) {
  if constexpr (VEC) {
    constexpr int Q = KMAX / 4;
    constexpr int U1 = KMAX == 64 ? 16 : 4;
#pragma unroll U1
    for (int e = lane; e < 32 * Q; e += 32) {
      const int rr = e / Q, c4 = e - rr * Q;
      const int64_t r = r0 + rr;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < n && 4 * c4 < k) v = __ldg(reinterpret_cast<const float4*>(src + r * ld) + c4);
      float* t = T + 4 * c4 * HALS_CS + wrow + rr;
      t[0] = v.x, t[HALS_CS] = v.y, t[2 * HALS_CS] = v.z, t[3 * HALS_CS] = v.w;
    }
  } else {
#pragma unroll 4
    for (int e = lane; e < 32 * KMAX; e += 32) {
      const int rr = e / KMAX, c = e - rr * KMAX;
      const int64_t r = r0 + rr;
      T[c * HALS_CS + wrow + rr] = (r < n && c < k) ? __ldg(src + r * ld + c) : 0.f;
    }
  }
}

// The 16-byte hals_stage_in of two matrices at once (the rows of Y and of
// F_fix): twice the loads in flight per round.
template <int KMAX>
__device__ __forceinline__ void hals_stage_in2(const float* __restrict__ sa, int64_t lda, float* Ta,
                                               const float* __restrict__ sb, int64_t ldb, float* Tb, int64_t r0,
                                               int64_t n, int k, int wrow, int lane) {
  {
    constexpr int Q = KMAX / 4;
    constexpr int U2 = KMAX == 64 ? 8 : 4;  // registers: the row of F_upd is live here
#pragma unroll U2
    for (int e = lane; e < 32 * Q; e += 32) {
      const int rr = e / Q, c4 = e - rr * Q;
      const int64_t r = r0 + rr;
      float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = va;
      if (r < n && 4 * c4 < k) {
        va = __ldg(reinterpret_cast<const float4*>(sa + r * lda) + c4);
        vb = __ldg(reinterpret_cast<const float4*>(sb + r * ldb) + c4);
      }
      float* ta = Ta + 4 * c4 * HALS_CS + wrow + rr;
      float* tb = Tb + 4 * c4 * HALS_CS + wrow + rr;
      ta[0] = va.x, ta[HALS_CS] = va.y, ta[2 * HALS_CS] = va.z, ta[3 * HALS_CS] = va.w;
      tb[0] = vb.x, tb[HALS_CS] = vb.y, tb[2 * HALS_CS] = vb.z, tb[3 * HALS_CS] = vb.w;
    }
  }
}

// The inverse of hals_stage_in: rows r0 .. min(r0 + 32, n) - 1 of the
// row-major dst (row stride k) from the tile, columns < k only.
template <int KMAX, bool VEC>
__device__ __forceinline__ void hals_stage_out(float* __restrict__ dst, int64_t r0, int64_t n, int k,
                                               const float* T, int wrow, int lane) {
  if constexpr (VEC) {
    constexpr int Q = KMAX / 4;
#pragma unroll 4
    for (int e = lane; e < 32 * Q; e += 32) {
      const int rr = e / Q, c4 = e - rr * Q;
      const int64_t r = r0 + rr;
      const float* t = T + 4 * c4 * HALS_CS + wrow + rr;
      if (r < n && 4 * c4 < k)
        reinterpret_cast<float4*>(dst + r * k)[c4] = make_float4(t[0], t[HALS_CS], t[2 * HALS_CS], t[3 * HALS_CS]);
    }
  } else {
#pragma unroll 4
    for (int e = lane; e < 32 * KMAX; e += 32) {
      const int rr = e / KMAX, c = e - rr * KMAX;
      const int64_t r = r0 + rr;
      if (r < n && c < k) dst[r * k + c] = T[c * HALS_CS + wrow + rr];
    }
  }
}

// Full-X HALS update, Eq. symhals_update2:
//   w_i <- max(0, (Y_i + alpha h_i - sum_{j != i} w_j G_ji) / (G_ii + alpha)),
// i = 0..k-1 in order with the columns already updated.  One thread per row:
// the row of F_upd in registers, its rows of Y and F_fix in the thread's own
// columns of two shared-memory tiles (zero padded).  Each warp moves its 32
// rows between global and shared memory itself, with whole-line loads and
// stores (hals_stage_in / hals_stage_out), so only warp barriers are needed.
// G with its diagonal zeroed and the reciprocals 1 / (G_ii + alpha) sit in
// shared memory, read as broadcasts.  With U given, the row of Y is formed as
// U_r M (LAI, M = Lambda U^T F_fix in shared memory).  Persistent grid over
// 128-row tiles; F_upd . Y and ||F_upd - F_fix||^2 are kept per thread in
// double-float and reduced in FP64.
template <int KMAX, bool VEC>
__global__ void __launch_bounds__(HALS_THREADS) hals_kernel(
    float* __restrict__ Fu, const float* __restrict__ Ff, int64_t n, int k, const float* __restrict__ G, float alpha,
    const float* __restrict__ Y, int ldy, const float* __restrict__ U, int l, const float* __restrict__ M,
    double* part, double* ws, unsigned* counter, unsigned* err) {
  constexpr bool ROT = hals_rot<KMAX>();
  constexpr int RS = hals_gstride<KMAX>();
  extern __shared__ __align__(16) float sm[];
  float* Gs = sm;                  // KMAX x RS, diagonal zeroed (rows twice side by side when ROT)
  float* inv = Gs + KMAX * RS;     // KMAX
  float* Ta = inv + KMAX;          // KMAX x HALS_CS: rows of F_upd, then of Y, then of F_upd again
  float* Tb = Ta + KMAX * HALS_CS;  // KMAX x HALS_CS: rows of F_fix
  float* Ms = Tb + KMAX * HALS_CS;  // l x KMAX (LAI only); 16-byte aligned as KMAX % 4 == 0
  const int tid = threadIdx.x, lane = tid & 31, wrow = tid & ~31;
  for (int e = tid; e < KMAX * KMAX; e += HALS_THREADS) {
    const int i = e / KMAX, j = e - i * KMAX;
    const float v = (i < k && j < k && i != j) ? G[i * k + j] : 0.f;
    Gs[i * RS + j] = v;
    if constexpr (ROT) Gs[i * RS + KMAX + j] = v;  // each row twice (rotated reads)
  }
  if (U)
    for (int e = tid; e < l * KMAX; e += HALS_THREADS) {
      const int i = e / KMAX, j = e - i * KMAX;
      Ms[e] = j < k ? M[i * k + j] : 0.f;
    }
  if (tid < KMAX) inv[tid] = tid < k ? 1.0f / (G[tid * k + tid] + alpha) : 0.f;
  __syncthreads();

  const float4* G4 = reinterpret_cast<const float4*>(Gs);
  const float4* Ms4 = reinterpret_cast<const float4*>(Ms);
  float2 trv = make_float2(0.f, 0.f), ddv = make_float2(0.f, 0.f);
  bool bad = false;
  float* ya = Ta + tid;  // this thread's columns: entry c at [c HALS_CS]
  const float* fb = Tb + tid;
  // uniform trip count over the block: rows past n run on zeros and are not stored
  for (int64_t t0 = (int64_t)blockIdx.x * HALS_THREADS; t0 < n; t0 += (int64_t)gridDim.x * HALS_THREADS) {
    const int64_t r0 = t0 + wrow;  // this warp's first row
    float w[KMAX];
    __syncwarp();  // the previous tile's stores have read Ta
    hals_stage_in<KMAX, VEC>(Fu, k, r0, n, k, Ta, wrow, lane);
    __syncwarp();
#pragma unroll
    for (int c = 0; c < KMAX; ++c) w[c] = ya[c * HALS_CS];
    __syncwarp();  // all lanes hold their rows before Ta takes Y
    if (U) {  // Y_r = U_r M (LAI product fused into the update)
      const int64_t r = r0 + lane;
      float y[KMAX];
#pragma unroll
      for (int c = 0; c < KMAX; ++c) y[c] = 0.f;
      if (r < n) {
        const float* ur = U + r * l;
#pragma unroll 2
        for (int pp = 0; pp < l; ++pp) {
          const float u = __ldg(ur + pp);
#pragma unroll
          for (int q = 0; q < KMAX / 4; ++q) {
            const float4 m = Ms4[pp * (KMAX / 4) + q];
            y[4 * q + 0] = fmaf(u, m.x, y[4 * q + 0]);
            y[4 * q + 1] = fmaf(u, m.y, y[4 * q + 1]);
            y[4 * q + 2] = fmaf(u, m.z, y[4 * q + 2]);
            y[4 * q + 3] = fmaf(u, m.w, y[4 * q + 3]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < KMAX; ++c) ya[c * HALS_CS] = y[c];
    } else if constexpr (VEC) {
      hals_stage_in2<KMAX>(Y, ldy, Ta, Ff, k, Tb, r0, n, k, wrow, lane);
    } else {
      hals_stage_in<KMAX, false>(Y, ldy, r0, n, k, Ta, wrow, lane);
    }
    if (U || !VEC) hals_stage_in<KMAX, VEC>(Ff, k, r0, n, k, Tb, wrow, lane);
    __syncwarp();
    if constexpr (ROT)
      bad |= hals_row_rotating<KMAX, 16>(
          w, [&](int c) { return ya[c * HALS_CS]; }, alpha, k, Gs, inv, [&](int c) { return fb[c * HALS_CS]; },
          trv, ddv);
    else
      bad |= hals_row_split<KMAX, 1>(
          w, [&](int c) { return ya[c * HALS_CS]; }, alpha, k, 0, 0xffffffffu, G4, inv,
          [&](int c) { return fb[c * HALS_CS]; }, trv, ddv);
    // the row back into this thread's columns of Ta (only its own reads of Y
    // were there), then the warp's whole-line stores
#pragma unroll
    for (int c = 0; c < KMAX; ++c) ya[c * HALS_CS] = w[c];
    __syncwarp();
    hals_stage_out<KMAX, VEC>(Fu, r0, n, k, Ta, wrow, lane);
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
  size_t smem = (size_t)(KMAX * hals_gstride<KMAX>() + KMAX + 2 * KMAX * HALS_CS) * 4;
  if (U) smem += (size_t)l * KMAX * 4;
  auto kern = hals_kernel<KMAX, VEC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, HALS_THREADS, smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (n + HALS_THREADS - 1) / HALS_THREADS;
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
