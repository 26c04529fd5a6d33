// Sparse and sampled products with X.
//   csr_xf          : Y = X F, a warp (half a warp for N <= 16) per CSR row,
//                     each lane owning VPL consecutive columns of F (vector
//                     loads of F rows when aligned for them, scalar loads
//                     otherwise).
//   csr_sampled_xf  : Y += X S^T S F of Alg. LvS-SymNMF: for every sampled
//                     row i (weight w) and nonzero (i, c, x): Y[c,:] += w x F[i,:]
//                     (X symmetric, so sampled columns are sampled rows).
//   dense_sampled_xf: the same product for a dense X.
#include <algorithm>

#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace symnmf {

constexpr int CSR_BATCH = 8;

// Y = X F for CSR X: LPR lanes per row (32: a warp, 16: half a warp), each
// lane owning VPL consecutive columns.  The column indices and values of up to
// LPR nonzeros are loaded at once (streaming: they are read once) and handed
// round by shuffles; CSR_BATCH gathers of F rows are in flight per lane group
// before their FMAs.
template <int LPR, int VPL, bool VEC>
__global__ void __launch_bounds__(256) csr_xf_kernel(const int64_t* __restrict__ rp,
                                                     const int32_t* __restrict__ col,
                                                     const float* __restrict__ val, int64_t n,
                                                     const float* __restrict__ F, int ldf, int N,
                                                     float* __restrict__ Y, int ldy) {
  constexpr int RPW = 32 / LPR;  // rows per warp
  const int lane = threadIdx.x & 31;
  const int li = lane % LPR;
  const unsigned mask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << (lane - li));
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int c0 = li * VPL;
  for (int64_t r = warp * RPW + lane / LPR; r < n; r += nwarps * RPW) {
    float acc[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) acc[v] = 0.f;
    const int64_t b = rp[r], e = rp[r + 1];
    for (int64_t p0 = b; p0 < e; p0 += LPR) {
      const int64_t p = p0 + li;
      int cc = 0;
      float xv = 0.f;
      if (p < e) {
        cc = __ldcs(col + p);
        xv = __ldcs(val + p);
      }
      const int cnt = (int)std::min<int64_t>(LPR, e - p0);
      for (int t0 = 0; t0 < cnt; t0 += CSR_BATCH) {
        float fv[CSR_BATCH][VPL], xs[CSR_BATCH];
#pragma unroll
        for (int u = 0; u < CSR_BATCH; ++u) {
          const int t = t0 + u;  // < LPR: t0 <= LPR - CSR_BATCH
          const int c = __shfl_sync(mask, cc, t, LPR);
          xs[u] = __shfl_sync(mask, xv, t, LPR);
          const float* fr = F + (int64_t)c * ldf + c0;
#pragma unroll
          for (int v = 0; v < VPL; ++v) fv[u][v] = 0.f;
          if (t < cnt) {
            bool done = false;
            if constexpr (VEC && VPL == 4) {
              if (c0 + 3 < N) {
                const float4 f = __ldg((const float4*)fr);
                fv[u][0] = f.x, fv[u][1] = f.y, fv[u][2] = f.z, fv[u][3] = f.w;
                done = true;
              }
            } else if constexpr (VEC && VPL == 2) {
              if (c0 + 1 < N) {
                const float2 f = __ldg((const float2*)fr);
                fv[u][0] = f.x, fv[u][1] = f.y;
                done = true;
              }
            }
            if (!done) {
#pragma unroll
              for (int v = 0; v < VPL; ++v)
                if (c0 + v < N) fv[u][v] = __ldg(fr + v);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < CSR_BATCH; ++u)
#pragma unroll
          for (int v = 0; v < VPL; ++v) acc[v] = fmaf(xs[u], fv[u][v], acc[v]);
      }
    }
    float* yr = Y + r * ldy;
#pragma unroll
    for (int v = 0; v < VPL; ++v)
      if (c0 + v < N) yr[c0 + v] = acc[v];
  }
}

cudaError_t csr_xf(const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                   const float* F, int ldf, int N, float* Y, int ldy, cudaStream_t st) {
  if (N < 1 || N > 128) return cudaErrorInvalidValue;
  const int64_t warps = n;
  int grid = (int)std::min<int64_t>((warps * 32 + 255) / 256, (int64_t)num_sms() * 16);
  if (grid < 1) grid = 1;
  if (N <= 16) {  // half a warp per row: no idle lanes
    const int grid16 = std::max(1, (int)std::min<int64_t>((n * 16 + 255) / 256, (int64_t)num_sms() * 16));
    csr_xf_kernel<16, 1, false><<<grid16, 256, 0, st>>>(row_ptr, col, val, n, F, ldf, N, Y, ldy);
    count_launches(1);
    return cudaGetLastError();
  }
  const bool vec4 = (ldf % 4 == 0) && (((uintptr_t)F & 15) == 0);
  const bool vec2 = (ldf % 2 == 0) && (((uintptr_t)F & 7) == 0);
  if (N <= 32)
    csr_xf_kernel<32, 1, false><<<grid, 256, 0, st>>>(row_ptr, col, val, n, F, ldf, N, Y, ldy);
  else if (N <= 64 && vec2)
    csr_xf_kernel<32, 2, true><<<grid, 256, 0, st>>>(row_ptr, col, val, n, F, ldf, N, Y, ldy);
  else if (N <= 64)
    csr_xf_kernel<32, 2, false><<<grid, 256, 0, st>>>(row_ptr, col, val, n, F, ldf, N, Y, ldy);
  else if (vec4)
    csr_xf_kernel<32, 4, true><<<grid, 256, 0, st>>>(row_ptr, col, val, n, F, ldf, N, Y, ldy);
  else
    csr_xf_kernel<32, 4, false><<<grid, 256, 0, st>>>(row_ptr, col, val, n, F, ldf, N, Y, ldy);
  count_launches(1);
  return cudaGetLastError();
}

// One warp per sample; lanes stride over the sampled row's nonzeros and
// columns of F.
__global__ void csr_sampled_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                   const float* __restrict__ val, const int32_t* __restrict__ idx,
                                   const float* __restrict__ wt, const int* s_tot,
                                   const float* __restrict__ F, int k, float* Y) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int S = *s_tot;
  for (int64_t j = warp; j < S; j += nwarps) {
    const int64_t i = idx[j];
    const float w = wt[j];
    const int64_t b = rp[i], e = rp[i + 1];
    for (int64_t p = b; p < e; ++p) {
      const int c = col[p];
      const float x = val[p] * w;
      for (int q = lane; q < k; q += 32) atomicAdd(Y + (int64_t)c * k + q, x * F[i * k + q]);
    }
  }
}

cudaError_t csr_sampled_xf(const int64_t* row_ptr, const int32_t* col, const float* val,
                           const int32_t* idx, const float* wt, const int* s_tot, const float* F,
                           int k, float* Y, cudaStream_t st) {
  const int grid = num_sms() * 4;
  csr_sampled_kernel<<<grid, 256, 0, st>>>(row_ptr, col, val, idx, wt, s_tot, F, k, Y);
  count_launches(1);
  return cudaGetLastError();
}

// Dense: Y[r, :] += sum_j X[i_j, r] wt_j F[i_j, :]  (row i_j of X = column i_j).
// Block = 128 consecutive r; samples processed in chunks staged in shared memory.
template <typename T>
__global__ void dense_sampled_kernel(const T* __restrict__ X, int64_t ldx, int64_t n,
                                     const int32_t* __restrict__ idx, const float* __restrict__ wt,
                                     const int* s_tot, const float* __restrict__ F, int k, float* Y) {
  __shared__ float Fs[32][64];
  __shared__ int64_t rows[32];
  const int S = *s_tot;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float acc[64];
#pragma unroll
  for (int q = 0; q < 64; ++q) acc[q] = 0.f;
  for (int j0 = 0; j0 < S; j0 += 32) {
    const int cnt = min(32, S - j0);
    for (int e = threadIdx.x; e < 32 * 64; e += blockDim.x) {
      const int jj = e / 64, q = e % 64;
      Fs[jj][q] = (jj < cnt && q < k) ? wt[j0 + jj] * F[(int64_t)idx[j0 + jj] * k + q] : 0.f;
    }
    if (threadIdx.x < 32) rows[threadIdx.x] = threadIdx.x < cnt ? (int64_t)idx[j0 + threadIdx.x] : 0;
    __syncthreads();
    if (r < n) {
      for (int jj = 0; jj < cnt; ++jj) {
        const float x = (float)X[rows[jj] * ldx + r];
#pragma unroll
        for (int q = 0; q < 64; ++q) acc[q] = fmaf(x, Fs[jj][q], acc[q]);
      }
    }
    __syncthreads();
  }
  if (r < n)
#pragma unroll
    for (int q = 0; q < 64; ++q)
      if (q < k) Y[r * k + q] += acc[q];
}

cudaError_t dense_sampled_xf(int fmt, const void* X, int64_t ldx, int64_t n, const int32_t* idx,
                             const float* wt, const int* s_tot, int s_cap, const float* F, int k,
                             float* Y, cudaStream_t st) {
  (void)s_cap;
  if (k > 64) return cudaErrorInvalidValue;
  const int grid = (int)((n + 127) / 128);
  if (fmt == 1)
    dense_sampled_kernel<float><<<grid, 128, 0, st>>>((const float*)X, ldx, n, idx, wt, s_tot, F, k, Y);
  else if (fmt == 0)
    dense_sampled_kernel<double><<<grid, 128, 0, st>>>((const double*)X, ldx, n, idx, wt, s_tot, F, k, Y);
  else if (fmt == 2)
    dense_sampled_kernel<__nv_bfloat16><<<grid, 128, 0, st>>>((const __nv_bfloat16*)X, ldx, n, idx, wt, s_tot,
                                                               F, k, Y);
  else
    return cudaErrorInvalidValue;
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace symnmf
