// Leverage scores of the rows of F (Alg. LvS-SymNMF): l_i = ||h_i R^-1||^2.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace symnmf {

constexpr int LEV_THREADS = 128;
constexpr int LEV_ROWS = 2 * LEV_THREADS;  // rows per block and pass: two per thread
constexpr int LEV_CS = LEV_ROWS + 1;       // column stride of the staged row tile

// l_i = ||h_i R^-1||^2 (R^-1 upper triangular, Alg. LvS-SymNMF).  Two rows per
// thread, z = h R^-1 for both accumulated by rows of R^-1 (z_j += h_p R^-1_pj
// for j >= p): each float4 broadcast of R^-1 from shared memory (KMAX x KMAX,
// zero padded) feeds eight FMAs, which halves the shared-memory wavefronts per
// row that bound the one-row form.  Each warp copies its 64 rows into a
// column-major shared tile with whole-line loads (one row per thread would
// touch 32 cache lines per load); a thread then reads h_p of its rows from its
// own two columns.
template <int KMAX, bool VEC>
__global__ void __launch_bounds__(LEV_THREADS) leverage_kernel(const float* __restrict__ F, int64_t n, int k,
                                                               const float* __restrict__ Rinv, double* lev) {
  __shared__ __align__(16) float Rs[KMAX * KMAX];
  extern __shared__ float lev_tile[];  // KMAX x LEV_CS
  for (int e = threadIdx.x; e < KMAX * KMAX; e += LEV_THREADS) {
    const int p = e / KMAX, j = e - p * KMAX;
    Rs[e] = (p < k && j < k && p <= j) ? Rinv[p * k + j] : 0.f;
  }
  __syncthreads();
  const float4* R4 = reinterpret_cast<const float4*>(Rs);
  const int lane = threadIdx.x & 31, wrow = 2 * (threadIdx.x & ~31);  // this warp's 64 tile rows
  const float* ha = lev_tile + wrow + lane;                            // rows wrow + lane and + 32
  for (int64_t t0 = (int64_t)blockIdx.x * LEV_ROWS; t0 < n; t0 += (int64_t)gridDim.x * LEV_ROWS) {
    const int64_t r0 = t0 + wrow;
    __syncwarp();  // the previous pass's reads of the tile are done
    if constexpr (VEC) {
      constexpr int Q = KMAX / 4;
      // at 64 columns 16 loads per lane in flight per round (the z registers
      // are not live yet)
      constexpr int U = KMAX == 64 ? 16 : 4;
#pragma unroll U
      for (int e = lane; e < 64 * Q; e += 32) {
        const int rr = e / Q, c4 = e - rr * Q;
        const int64_t r = r0 + rr;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < n && 4 * c4 < k) v = __ldg(reinterpret_cast<const float4*>(F + r * k) + c4);
        float* t = lev_tile + 4 * c4 * LEV_CS + wrow + rr;
        t[0] = v.x, t[LEV_CS] = v.y, t[2 * LEV_CS] = v.z, t[3 * LEV_CS] = v.w;
      }
    } else {
#pragma unroll 4
      for (int e = lane; e < 64 * KMAX; e += 32) {
        const int rr = e / KMAX, c = e - rr * KMAX;
        const int64_t r = r0 + rr;
        lev_tile[c * LEV_CS + wrow + rr] = (r < n && c < k) ? __ldg(F + r * k + c) : 0.f;
      }
    }
    __syncwarp();
    float za[KMAX], zb[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) za[j] = 0.f, zb[j] = 0.f;
#pragma unroll
    for (int p = 0; p < KMAX; ++p) {
      const float hpa = ha[p * LEV_CS], hpb = ha[p * LEV_CS + 32];
#pragma unroll
      for (int j4 = p / 4; j4 < KMAX / 4; ++j4) {
        const float4 g = R4[p * (KMAX / 4) + j4];
        za[4 * j4 + 0] = fmaf(hpa, g.x, za[4 * j4 + 0]);
        za[4 * j4 + 1] = fmaf(hpa, g.y, za[4 * j4 + 1]);
        za[4 * j4 + 2] = fmaf(hpa, g.z, za[4 * j4 + 2]);
        za[4 * j4 + 3] = fmaf(hpa, g.w, za[4 * j4 + 3]);
        zb[4 * j4 + 0] = fmaf(hpb, g.x, zb[4 * j4 + 0]);
        zb[4 * j4 + 1] = fmaf(hpb, g.y, zb[4 * j4 + 1]);
        zb[4 * j4 + 2] = fmaf(hpb, g.z, zb[4 * j4 + 2]);
        zb[4 * j4 + 3] = fmaf(hpb, g.w, zb[4 * j4 + 3]);
      }
    }
    float sa0 = 0.f, sa1 = 0.f, sb0 = 0.f, sb1 = 0.f;
#pragma unroll
    for (int j = 0; j < KMAX; j += 2) {
      sa0 = fmaf(za[j], za[j], sa0);
      sa1 = fmaf(za[j + 1], za[j + 1], sa1);
      sb0 = fmaf(zb[j], zb[j], sb0);
      sb1 = fmaf(zb[j + 1], zb[j + 1], sb1);
    }
    const int64_t ra = r0 + lane, rb = ra + 32;
    if (ra < n) lev[ra] = (double)(sa0 + sa1);
    if (rb < n) lev[rb] = (double)(sb0 + sb1);
  }
}

template <int KMAX>
static cudaError_t launch_leverage(const float* F, int64_t n, int k, const float* Rinv, double* lev,
                                   cudaStream_t st) {
  const size_t smem = (size_t)KMAX * LEV_CS * 4;
  const bool vec = (k % 4) == 0 && ((uintptr_t)F & 15) == 0;
  const void* fn = vec ? (const void*)leverage_kernel<KMAX, true> : (const void*)leverage_kernel<KMAX, false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, LEV_THREADS, smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (n + LEV_ROWS - 1) / LEV_ROWS;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms() * std::max(per_sm, 1)));
  if (vec)
    leverage_kernel<KMAX, true><<<grid, LEV_THREADS, smem, st>>>(F, n, k, Rinv, lev);
  else
    leverage_kernel<KMAX, false><<<grid, LEV_THREADS, smem, st>>>(F, n, k, Rinv, lev);
  return cudaSuccess;
}

cudaError_t leverage_rows(const float* F, int64_t n, int k, const float* Rinv, double* lev,
                          cudaStream_t st) {
  if (k < 1 || k > 64) return cudaErrorInvalidValue;
  if (n < 1) return cudaSuccess;
  cudaError_t e;
  if (k <= 8)
    e = launch_leverage<8>(F, n, k, Rinv, lev, st);
  else if (k <= 16)
    e = launch_leverage<16>(F, n, k, Rinv, lev, st);
  else if (k <= 24)
    e = launch_leverage<24>(F, n, k, Rinv, lev, st);
  else if (k <= 32)
    e = launch_leverage<32>(F, n, k, Rinv, lev, st);
  else if (k <= 48)
    e = launch_leverage<48>(F, n, k, Rinv, lev, st);
  else
    e = launch_leverage<64>(F, n, k, Rinv, lev, st);
  if (e != cudaSuccess) return e;
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace symnmf
