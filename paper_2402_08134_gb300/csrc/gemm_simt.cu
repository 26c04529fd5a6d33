// Dense Y = X F on CUDA cores for float32 / float64 X (the plain FP32 form and
// the FP64 planted case).  X is streamed once per product; F (n x N, N <= 128)
// stays in L2.  Split-K over the reduction index gives enough CTAs to fill
// the 152 SMs; splits are summed in a fixed order (deterministic).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace symnmf {

constexpr int SB_M = 128, SB_K = 32, SB_THREADS = 256;

template <typename T>
struct AccT;
template <>
struct AccT<float> {
  using type = float;
};
template <>
struct AccT<double> {
  using type = double;
};

// Thread (tx, ty): columns 4tx..4tx+3, rows ty + j*RG (j < TM).
template <typename T, int NB>
__global__ void __launch_bounds__(SB_THREADS) xf_simt_kernel(const T* __restrict__ X, int64_t ldx,
                                                             int64_t n, const float* __restrict__ F,
                                                             int ldf, int N, float* out,
                                                             int64_t ldo, int64_t kchunk) {
  using A = typename AccT<T>::type;
  constexpr int CG = NB / 4;              // column groups
  constexpr int RG = SB_THREADS / CG;     // row groups
  constexpr int TM = SB_M / RG;           // rows per thread
  __shared__ T As[SB_K][SB_M + 4];
  __shared__ __align__(16) A Bs[SB_K][NB];
  const int tid = threadIdx.x;
  const int tx = tid % CG, ty = tid / CG;
  const int64_t m0 = (int64_t)blockIdx.x * SB_M;
  const int64_t kbeg = (int64_t)blockIdx.y * kchunk;
  const int64_t kend = min(n, kbeg + kchunk);
  A acc[TM][4];
#pragma unroll
  for (int j = 0; j < TM; ++j)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[j][c] = A(0);

  for (int64_t k0 = kbeg; k0 < kend; k0 += SB_K) {
    // X tile: SB_M rows x SB_K columns, stored transposed
    for (int e = tid; e < SB_M * SB_K; e += SB_THREADS) {
      const int r = e / SB_K, c = e - r * SB_K;
      const int64_t gr = m0 + r, gc = k0 + c;
      As[c][r] = (gr < n && gc < kend) ? X[gr * ldx + gc] : T(0);
    }
    for (int e = tid; e < SB_K * NB; e += SB_THREADS) {
      const int r = e / NB, c = e - r * NB;
      const int64_t gr = k0 + r;
      Bs[r][c] = (gr < kend && c < N) ? (A)F[gr * ldf + c] : A(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < SB_K; ++kk) {
      A b[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][4 * tx + c];
#pragma unroll
      for (int j = 0; j < TM; ++j) {
        const A a = (A)As[kk][ty + j * RG];
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[j][c] = fma(a, b[c], acc[j][c]);
      }
    }
    __syncthreads();
  }
  float* o = out + (int64_t)blockIdx.y * n * ldo;
#pragma unroll
  for (int j = 0; j < TM; ++j) {
    const int64_t gr = m0 + ty + j * RG;
    if (gr < n) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int gc = 4 * tx + c;
        if (gc < N) o[gr * ldo + gc] = (float)acc[j][c];
      }
    }
  }
}

__global__ void sum_splits_kernel(const float* ws, int splits, int64_t n, int N, float* Y, int ldy) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * N) return;
  const int64_t i = t / N;
  const int c = (int)(t - i * N);
  float s = 0.f;
  for (int p = 0; p < splits; ++p) s += ws[(int64_t)p * n * N + t];
  Y[i * ldy + c] = s;
}

static int simt_splits(int64_t n) {
  const int64_t mt = (n + SB_M - 1) / SB_M;
  int s = (int)((2 * num_sms() + mt - 1) / mt);
  const int64_t maxs = (n + 4 * SB_K - 1) / (4 * SB_K);
  if (s > maxs) s = (int)maxs;
  if (s > 16) s = 16;
  return s < 1 ? 1 : s;
}

size_t xf_simt_ws_floats(int64_t n, int N) {
  const int s = simt_splits(n);
  return s > 1 ? (size_t)s * n * N : 0;
}

template <typename T, int NB>
static void launch(const T* X, int64_t ldx, int64_t n, const float* F, int ldf, int N, float* out,
                   int64_t ldo, int splits, int64_t kchunk, cudaStream_t st) {
  dim3 grid((unsigned)((n + SB_M - 1) / SB_M), (unsigned)splits);
  xf_simt_kernel<T, NB><<<grid, SB_THREADS, 0, st>>>(X, ldx, n, F, ldf, N, out, ldo, kchunk);
  count_launches(1);
}

template <typename T>
static cudaError_t dispatch(const T* X, int64_t ldx, int64_t n, const float* F, int ldf, int N, float* Y,
                            int ldy, float* ws, size_t ws_floats, cudaStream_t st) {
  const int splits = simt_splits(n);
  int64_t kchunk = (n + splits - 1) / splits;
  kchunk = (kchunk + SB_K - 1) / SB_K * SB_K;
  float* out = Y;
  int64_t ldo = ldy;
  if (splits > 1) {
    if (!ws || ws_floats < (size_t)splits * n * N) return cudaErrorInvalidValue;
    out = ws;
    ldo = N;
  }
  if constexpr (sizeof(T) == 8) {
    // FP64 tiles keep NB = 32 (static shared memory); wider F goes in column chunks
    for (int c0 = 0; c0 < N; c0 += 32)
      launch<T, 32>(X, ldx, n, F + c0, ldf, min(32, N - c0), out + c0, ldo, splits, kchunk, st);
  } else if (N <= 32) {
    launch<T, 32>(X, ldx, n, F, ldf, N, out, ldo, splits, kchunk, st);
  } else if (N <= 64) {
    launch<T, 64>(X, ldx, n, F, ldf, N, out, ldo, splits, kchunk, st);
  } else if (N <= 128) {
    launch<T, 128>(X, ldx, n, F, ldf, N, out, ldo, splits, kchunk, st);
  } else {
    return cudaErrorInvalidValue;
  }
  if (splits > 1) {
    const int64_t work = n * N;
    sum_splits_kernel<<<(int)((work + 255) / 256), 256, 0, st>>>(ws, splits, n, N, Y, ldy);
    count_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t xf_simt(int fmt, const void* X, int64_t ldx, int64_t n, const float* F, int ldf, int N,
                    float* Y, int ldy, float* ws, size_t ws_floats, cudaStream_t st) {
  if (fmt == 1) return dispatch<float>((const float*)X, ldx, n, F, ldf, N, Y, ldy, ws, ws_floats, st);
  if (fmt == 0) return dispatch<double>((const double*)X, ldx, n, F, ldf, N, Y, ldy, ws, ws_floats, st);
  return cudaErrorInvalidValue;
}

}  // namespace symnmf
