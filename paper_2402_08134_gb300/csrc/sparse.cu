// Sparse and sampled products with X.
//   csr_xf          : Y = X F, one warp per CSR row, each lane owning VPL
//                     consecutive columns of F (vector loads of F rows when
//                     the rows are aligned for them, scalar loads otherwise).
//   csr_sampled_xf  : Y += X S^T S F of Alg. LvS-SymNMF: for every sampled
//                     row i (weight w) and nonzero (i, c, x): Y[c,:] += w x F[i,:]
//                     (X symmetric, so sampled columns are sampled rows).
//   dense_sampled_xf: the same product for a dense X.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace symnmf {

template <int VPL, bool VEC>
__global__ void __launch_bounds__(256) csr_xf_kernel(const int64_t* __restrict__ rp,
                                                     const int32_t* __restrict__ col,
                                                     const float* __restrict__ val, int64_t n,
                                                     const float* __restrict__ F, int ldf, int N,
                                                     float* __restrict__ Y, int ldy) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int c0 = lane * VPL;
  for (int64_t r = warp; r < n; r += nwarps) {
    float acc[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) acc[v] = 0.f;
    const int64_t b = rp[r], e = rp[r + 1];
    for (int64_t p0 = b; p0 < e; p0 += 32) {
      const int64_t p = p0 + lane;
      int cc = 0;
      float xv = 0.f;
      if (p < e) {
        cc = __ldg(col + p);
        xv = __ldg(val + p);
      }
      const int cnt = (int)std::min<int64_t>(32, e - p0);
      for (int t = 0; t < cnt; ++t) {
        const int c = __shfl_sync(0xffffffffu, cc, t);
        const float x = __shfl_sync(0xffffffffu, xv, t);
        const float* fr = F + (int64_t)c * ldf;
        if (VEC && VPL == 4 && c0 + 3 < N) {
          const float4 f = __ldg((const float4*)(fr + c0));
          acc[0] = fmaf(x, f.x, acc[0]);
          acc[1] = fmaf(x, f.y, acc[1]);
          acc[2] = fmaf(x, f.z, acc[2]);
          acc[3] = fmaf(x, f.w, acc[3]);
        } else if (VEC && VPL == 2 && c0 + 1 < N) {
          const float2 f = __ldg((const float2*)(fr + c0));
          acc[0] = fmaf(x, f.x, acc[0]);
          acc[1] = fmaf(x, f.y, acc[1]);
        } else {
#pragma unroll
          for (int v = 0; v < VPL; ++v)
            if (c0 + v < N) acc[v] = fmaf(x, __ldg(fr + c0 + v), acc[v]);
        }
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
  const int64_t warps = n;
  int grid = (int)std::min<int64_t>((warps * 32 + 255) / 256, (int64_t)num_sms() * 16);
  if (grid < 1) grid = 1;
  const bool vec4 = (ldf % 4 == 0) && (((uintptr_t)F & 15) == 0);
  const bool vec2 = (ldf % 2 == 0) && (((uintptr_t)F & 7) == 0);
  if (N <= 32)
    csr_xf_kernel<1, false><<<grid, 256, 0, st>>>(row_ptr, col, val, n, F, ldf, N, Y, ldy);
  else if (N <= 64 && vec2)
    csr_xf_kernel<2, true><<<grid, 256, 0, st>>>(row_ptr, col, val, n, F, ldf, N, Y, ldy);
  else if (N <= 64)
    csr_xf_kernel<2, false><<<grid, 256, 0, st>>>(row_ptr, col, val, n, F, ldf, N, Y, ldy);
  else if (N <= 128 && vec4)
    csr_xf_kernel<4, true><<<grid, 256, 0, st>>>(row_ptr, col, val, n, F, ldf, N, Y, ldy);
  else if (N <= 128)
    csr_xf_kernel<4, false><<<grid, 256, 0, st>>>(row_ptr, col, val, n, F, ldf, N, Y, ldy);
  else
    return cudaErrorInvalidValue;
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
  else
    return cudaErrorInvalidValue;
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace symnmf
