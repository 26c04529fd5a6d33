// Dense Y = X F on CUDA cores for float32 / float64 X (the plain FP32 form and
// the FP64 planted case).  X is streamed once per product; F (n x N, N <= 128)
// stays in L2.  Split-K over the reduction index gives enough CTAs to fill
// the 152 SMs; splits are summed in a fixed order (deterministic).  Narrow
// FP32 products (N <= 32, 16-byte rows) take a row-streaming kernel; the
// others a shared-memory tiled one.
#include <stdint.h>

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

// Row-streaming FP32 product for narrow F (N <= 32, the plain FP32 form's
// widths): thread t of a CTA owns rows m0 + RT t .. m0 + RT t + RT - 1 and all
// N columns (RT x N4 FP32 accumulators).  Each step reads a float4 of K from
// each of its rows straight from global memory -- the 128-byte lines of the
// CTA's rows stay in L1 across the eight steps that use them, so DRAM sees
// every X byte once -- and broadcasts four rows of F from shared memory.  Per
// X element: N FMAs, no shared-memory traffic for X.  The K range is split
// over gridDim.y (partials summed in a fixed order by sum_splits_kernel).
constexpr int RS_THREADS = 256, RS_RT = 4, RS_KC = 64;

template <int NC4>
__global__ void __launch_bounds__(RS_THREADS) xf_rows_kernel(const float* __restrict__ X, int64_t ldx, int64_t n,
                                                            const float* __restrict__ F, int ldf, int N,
                                                            float* out, int64_t ldo, int64_t kchunk) {
  __shared__ __align__(16) float4 Fs[RS_KC][NC4];
  const int tid = threadIdx.x;
  const int64_t r0 = ((int64_t)blockIdx.x * RS_THREADS + tid) * RS_RT;
  const int64_t kbeg = (int64_t)blockIdx.y * kchunk;
  const int64_t kend = min(n, kbeg + kchunk);
  float4 acc[RS_RT][NC4];
#pragma unroll
  for (int i = 0; i < RS_RT; ++i)
#pragma unroll
    for (int c = 0; c < NC4; ++c) acc[i][c] = make_float4(0.f, 0.f, 0.f, 0.f);
  const float* xr[RS_RT];
#pragma unroll
  for (int i = 0; i < RS_RT; ++i) xr[i] = X + min(r0 + i, n - 1) * ldx;  // rows past n compute garbage, unstored
  for (int64_t k0 = kbeg; k0 < kend; k0 += RS_KC) {
    const int kc = (int)min((int64_t)RS_KC, kend - k0);
    __syncthreads();
    for (int e = tid; e < RS_KC * NC4 * 4; e += RS_THREADS) {
      const int kk = e / (NC4 * 4), c = e - kk * (NC4 * 4);
      reinterpret_cast<float*>(Fs)[e] = (kk < kc && c < N) ? F[(k0 + kk) * ldf + c] : 0.f;
    }
    __syncthreads();
    // the next step's X values are loaded one step ahead (registers), so that
    // their load latency overlaps the current step's FMAs
    float4 xn[RS_RT];
#pragma unroll
    for (int i = 0; i < RS_RT; ++i) xn[i] = __ldg(reinterpret_cast<const float4*>(xr[i] + k0));
    for (int kk = 0; kk < kc; kk += 4) {  // kc is a multiple of 4 (n % 4 == 0)
      if (((k0 + kk) & 31) == 0 && k0 + kk + 32 < kend)
#pragma unroll
        for (int i = 0; i < RS_RT; ++i)  // the rows' next 128-byte lines, ahead of their first use
          asm volatile("prefetch.global.L1 [%0];" ::"l"(xr[i] + k0 + kk + 32));
      float4 x[RS_RT];
#pragma unroll
      for (int i = 0; i < RS_RT; ++i) x[i] = xn[i];
      if (kk + 4 < kc)
#pragma unroll
        for (int i = 0; i < RS_RT; ++i) xn[i] = __ldg(reinterpret_cast<const float4*>(xr[i] + k0 + kk + 4));
#pragma unroll
      for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int c = 0; c < NC4; ++c) {
          const float4 f = Fs[kk + q][c];
#pragma unroll
          for (int i = 0; i < RS_RT; ++i) {
            const float xv = q == 0 ? x[i].x : q == 1 ? x[i].y : q == 2 ? x[i].z : x[i].w;
            acc[i][c].x = fmaf(xv, f.x, acc[i][c].x);
            acc[i][c].y = fmaf(xv, f.y, acc[i][c].y);
            acc[i][c].z = fmaf(xv, f.z, acc[i][c].z);
            acc[i][c].w = fmaf(xv, f.w, acc[i][c].w);
          }
        }
      }
    }
  }
  float* o = out + (int64_t)blockIdx.y * n * ldo;
#pragma unroll
  for (int i = 0; i < RS_RT; ++i) {
    const int64_t r = r0 + i;
    if (r < n) {
#pragma unroll
      for (int c = 0; c < NC4; ++c) {
        const float v[4] = {acc[i][c].x, acc[i][c].y, acc[i][c].z, acc[i][c].w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (4 * c + u < N) o[r * ldo + 4 * c + u] = v[u];
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

// The row-streaming kernel applies to FP32 X with 16-byte rows (n, ldx
// multiples of 4, aligned base) and N <= 32.
static bool rows_ok(const void* X, int64_t ldx, int64_t n, int N) {
  return N <= 32 && (n % 4) == 0 && (ldx % 4) == 0 && ((uintptr_t)X & 15) == 0;
}

// K splits of the row-streaming kernel: about two CTAs per SM.
static int rows_splits(int64_t n) {
  const int64_t rb = (n + RS_THREADS * RS_RT - 1) / (RS_THREADS * RS_RT);
  int s = (int)((2 * num_sms() + rb - 1) / rb);
  const int64_t maxs = (n + 4 * RS_KC - 1) / (4 * RS_KC);
  if (s > maxs) s = (int)maxs;
  if (s > 64) s = 64;
  return s < 1 ? 1 : s;
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
  const int s = std::max(simt_splits(n), N <= 32 ? rows_splits(n) : 1);
  return s > 1 ? (size_t)s * n * N : 0;
}

template <typename T, int NB>
static void launch(const T* X, int64_t ldx, int64_t n, const float* F, int ldf, int N, float* out,
                   int64_t ldo, int splits, int64_t kchunk, cudaStream_t st) {
  dim3 grid((unsigned)((n + SB_M - 1) / SB_M), (unsigned)splits);
  xf_simt_kernel<T, NB><<<grid, SB_THREADS, 0, st>>>(X, ldx, n, F, ldf, N, out, ldo, kchunk);
  count_launches(1);
}

template <int NC4>
static void launch_rows(const float* X, int64_t ldx, int64_t n, const float* F, int ldf, int N, float* out,
                        int64_t ldo, int splits, int64_t kchunk, cudaStream_t st) {
  dim3 grid((unsigned)((n + RS_THREADS * RS_RT - 1) / (RS_THREADS * RS_RT)), (unsigned)splits);
  xf_rows_kernel<NC4><<<grid, RS_THREADS, 0, st>>>(X, ldx, n, F, ldf, N, out, ldo, kchunk);
  count_launches(1);
}

static cudaError_t dispatch_rows(const float* X, int64_t ldx, int64_t n, const float* F, int ldf, int N, float* Y,
                                 int ldy, float* ws, size_t ws_floats, cudaStream_t st) {
  const int splits = rows_splits(n);
  int64_t kchunk = (n + splits - 1) / splits;
  kchunk = (kchunk + RS_KC - 1) / RS_KC * RS_KC;
  float* out = Y;
  int64_t ldo = ldy;
  if (splits > 1) {
    if (!ws || ws_floats < (size_t)splits * n * N) return cudaErrorInvalidValue;
    out = ws;
    ldo = N;
  }
  switch ((N + 3) / 4) {
    case 1: launch_rows<1>(X, ldx, n, F, ldf, N, out, ldo, splits, kchunk, st); break;
    case 2: launch_rows<2>(X, ldx, n, F, ldf, N, out, ldo, splits, kchunk, st); break;
    case 3: launch_rows<3>(X, ldx, n, F, ldf, N, out, ldo, splits, kchunk, st); break;
    case 4: launch_rows<4>(X, ldx, n, F, ldf, N, out, ldo, splits, kchunk, st); break;
    case 5: launch_rows<5>(X, ldx, n, F, ldf, N, out, ldo, splits, kchunk, st); break;
    case 6: launch_rows<6>(X, ldx, n, F, ldf, N, out, ldo, splits, kchunk, st); break;
    case 7: launch_rows<7>(X, ldx, n, F, ldf, N, out, ldo, splits, kchunk, st); break;
    default: launch_rows<8>(X, ldx, n, F, ldf, N, out, ldo, splits, kchunk, st); break;
  }
  if (splits > 1) {
    const int64_t work = n * N;
    sum_splits_kernel<<<(int)((work + 255) / 256), 256, 0, st>>>(ws, splits, n, N, Y, ldy);
    count_launches(1);
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t dispatch(const T* X, int64_t ldx, int64_t n, const float* F, int ldf, int N, float* Y,
                            int ldy, float* ws, size_t ws_floats, cudaStream_t st) {
  if constexpr (sizeof(T) == 4)
    if (rows_ok(X, ldx, n, N)) return dispatch_rows(X, ldx, n, F, ldf, N, Y, ldy, ws, ws_floats, st);
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
