// Row-streaming kernels of the SymNMF hot path: cross products / Grams with
// FP64 accumulation, the fused regularised HALS update (Eq. symhals_update2),
// LAI expansion Y = U (Lambda U^T F) (Alg. LAI-SymNMF), leverage-score row
// pass (Alg. LvS-SymNMF), objective and projected-gradient reductions, and
// the Philox generators.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "dfloat.cuh"
#include "kernels.h"

namespace symnmf {

// ---------------------------------------------------------------- xstats

// Last-block-done reduction of per-block partials: no block ever waits.
template <int NV>
__device__ bool last_block(unsigned* counter) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

// Element (i, j) of dense X in its storage format, as float (FP8: times the row scale).
template <int FMT>
__device__ __forceinline__ float load_xf(const void* x, int64_t ldx, float rsi, int64_t i, int64_t j) {
  if constexpr (FMT == 1) return __ldg((const float*)x + i * ldx + j);
  if constexpr (FMT == 2) return __bfloat162float(((const __nv_bfloat16*)x)[i * ldx + j]);
  if constexpr (FMT == 3) {
    __nv_fp8_e4m3 v;
    v.__x = ((const uint8_t*)x)[i * ldx + j];
    return rsi * float(v);
  }
  return 0.f;
}

// Kahan step: (s, c) holds the running sum s - c.
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// max, sum and sum of squares of X.  A block per row (strided), threads along
// the row.  ||X||^2 enters the trace-trick objective, which cancels terms of
// its size, so the sums must be accurate: FP64 input is summed in FP64; the
// narrow formats are summed per thread and row in compensated FP32 (Kahan,
// squares split exactly as v*v = p + e with one FMA) and only the per-row
// results in FP64 -- FP64 arithmetic is scarce on this part.
template <int FMT>
__global__ void xstats_dense_kernel(const void* x, int64_t ldx, const float* rs, int64_t n, double* out,
                                    double* ws, unsigned* counter) {
  __shared__ double sh[32];
  double mx = -INFINITY, sm = 0.0, sq = 0.0;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    if constexpr (FMT == 0) {
      const double* xr = (const double*)x + i * ldx;
      for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        const double v = xr[j];
        mx = fmax(mx, v);
        sm += v;
        sq += v * v;
      }
    } else {
      const float rsi = (FMT == 3) ? rs[i] : 1.f;
      float m = -INFINITY, s = 0.f, cs = 0.f, q = 0.f, cq = 0.f, eq = 0.f;
      auto add = [&](float v) {
        m = fmaxf(m, v);
        kahan_add(s, cs, v);
        const float p = v * v;
        eq += fmaf(v, v, -p);
        kahan_add(q, cq, p);
      };
      // 16-byte loads when the row start allows them (many bytes in flight per thread)
      constexpr int ES = FMT == 1 ? 4 : FMT == 2 ? 2 : 1;  // bytes per element
      constexpr int VE = 16 / ES;                          // elements per 16 bytes
      const unsigned char* rowp = (const unsigned char*)x + (size_t)i * ldx * ES;
      int64_t j0 = 0;
      if (((uintptr_t)rowp & 15) == 0) {
        const int64_t nv = n / VE;
        const uint4* r4 = reinterpret_cast<const uint4*>(rowp);
#pragma unroll 4
        for (int64_t v = threadIdx.x; v < nv; v += blockDim.x) {
          const uint4 w = __ldg(r4 + v);
          const unsigned wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if constexpr (FMT == 1) {
              add(__uint_as_float(wv[u]));
            } else if constexpr (FMT == 2) {
              add(__uint_as_float(wv[u] << 16));          // element 2u (low half)
              add(__uint_as_float(wv[u] & 0xffff0000u));  // element 2u + 1
            } else {
#pragma unroll
              for (int b = 0; b < 4; ++b) {
                __nv_fp8_e4m3 f8;
                f8.__x = (unsigned char)(wv[u] >> (8 * b));
                add(rsi * float(f8));
              }
            }
          }
        }
        j0 = nv * VE;
      }
      for (int64_t j = j0 + threadIdx.x; j < n; j += blockDim.x) add(load_xf<FMT>(x, ldx, rsi, i, j));
      mx = fmax(mx, (double)m);
      sm += (double)s - (double)cs;
      sq += ((double)q - (double)cq) + (double)eq;
    }
  }
  // block reductions
  mx = warp_max(mx);
  __shared__ double shm[32];
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? shm[threadIdx.x] : -INFINITY;
    mx = warp_max(t);
  }
  sm = block_sum(sm, sh);
  sq = block_sum(sq, sh);
  if (threadIdx.x == 0) {
    ws[3 * blockIdx.x + 0] = mx;
    ws[3 * blockIdx.x + 1] = sm;
    ws[3 * blockIdx.x + 2] = sq;
  }
  if (last_block<1>(counter)) {
    double M = -INFINITY;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) M = fmax(M, __ldcg(ws + 3 * b));
    M = warp_max(M);
    __shared__ double shx[32];
    if ((threadIdx.x & 31) == 0) shx[threadIdx.x >> 5] = M;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) M = fmax(M, shx[w]);
      out[0] = M;
    }
    reduce_partials(ws + 1, 3, 2, gridDim.x, out + 1, sh);
    if (threadIdx.x == 0) *counter = 0;
  }
}

__global__ void xstats_csr_kernel(const float* val, int64_t nnz, double* out, double* ws,
                                  unsigned* counter) {
  __shared__ double sh[32];
  double mx = -INFINITY, sm = 0.0, sq = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double v = val[e];
    mx = fmax(mx, v);
    sm += v;
    sq += v * v;
  }
  mx = warp_max(mx);
  __shared__ double shm[32];
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? shm[threadIdx.x] : -INFINITY;
    mx = warp_max(t);
  }
  sm = block_sum(sm, sh);
  sq = block_sum(sq, sh);
  if (threadIdx.x == 0) {
    ws[3 * blockIdx.x + 0] = mx;
    ws[3 * blockIdx.x + 1] = sm;
    ws[3 * blockIdx.x + 2] = sq;
  }
  if (last_block<1>(counter)) {
    double M = -INFINITY;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) M = fmax(M, __ldcg(ws + 3 * b));
    M = warp_max(M);
    __shared__ double shx[32];
    if ((threadIdx.x & 31) == 0) shx[threadIdx.x >> 5] = M;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) M = fmax(M, shx[w]);
      out[0] = M;
    }
    reduce_partials(ws + 1, 3, 2, gridDim.x, out + 1, sh);
    if (threadIdx.x == 0) *counter = 0;
  }
}

cudaError_t xstats(int fmt, const void* x, int64_t ldx, const float* row_scale, int64_t n,
                   const int64_t* row_ptr, int64_t nnz, double* out, double* ws, unsigned* counter,
                   cudaStream_t st) {
  (void)row_ptr;
  const int grid = num_sms() * 4;
  if (fmt == 4)
    xstats_csr_kernel<<<grid, 256, 0, st>>>((const float*)x, nnz, out, ws, counter);
  else if (fmt == 0)
    xstats_dense_kernel<0><<<grid, 256, 0, st>>>(x, ldx, row_scale, n, out, ws, counter);
  else if (fmt == 1)
    xstats_dense_kernel<1><<<grid, 256, 0, st>>>(x, ldx, row_scale, n, out, ws, counter);
  else if (fmt == 2)
    xstats_dense_kernel<2><<<grid, 256, 0, st>>>(x, ldx, row_scale, n, out, ws, counter);
  else
    xstats_dense_kernel<3><<<grid, 256, 0, st>>>(x, ldx, row_scale, n, out, ws, counter);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------- cross product

constexpr int XC_THREADS = 256;
constexpr int XC_CHUNK = 128;

size_t xcross_ws_doubles(int la, int lb) { return (size_t)2 * num_sms() * la * lb + 64; }

// C = A^T diag(wt) B over (gathered) rows.  Each thread keeps Kahan-
// compensated FP32 sums (error O(eps) however many rows they cover); row
// groups and block partials combine as double-float pairs (dfloat.cuh): no
// FP64 arithmetic, which is scarce on this part.  The trace-trick objective
// cancels terms of size ||X||^2, so the Grams need this accuracy.  Block
// partials are summed in block order (deterministic), by the last block or by
// a second kernel.
template <int TPT>
__global__ void __launch_bounds__(XC_THREADS) xcross_kernel(
    const float* __restrict__ A, int lda, int la, const float* __restrict__ B, int ldb, int lb,
    int64_t n, const int32_t* __restrict__ idx, const float* __restrict__ wt, const int* cnt,
    const double* __restrict__ lam, double shift, double* C, float* Cf, double* ws,
    unsigned* counter) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int la4 = (la + 3) & ~3, lb4 = (lb + 3) & ~3;
  float* As = (float*)smraw;
  float* Bs = As + XC_CHUNK * la4;
  dfl* red = (dfl*)(Bs + XC_CHUNK * lb4);
  dfl* wsd = reinterpret_cast<dfl*>(ws);  // the partials are double-float pairs
  const int ta = la4 >> 2, tb = lb4 >> 2, T = ta * tb;
  const int tid = threadIdx.x;
  const int R = T >= XC_THREADS ? 1 : XC_THREADS / T;
  const int rg = T >= XC_THREADS ? 0 : tid / T;
  const bool active = rg < R;

  const int64_t count = cnt ? (int64_t)(*cnt) : n;
  const int64_t per = (count + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = min(count, r0 + per);

  float f[TPT][16], fc[TPT][16];
#pragma unroll
  for (int t = 0; t < TPT; ++t)
#pragma unroll
    for (int e = 0; e < 16; ++e) f[t][e] = 0.f, fc[t][e] = 0.f;

  // a Gram (same operand, no weights) stages its rows once
  const bool same = (A == B) && (lda == ldb) && (la == lb) && !wt;
  const float* Bsrc = same ? As : Bs;
  // pad columns are zero once and for all
  if (la4 > la)
    for (int e = tid; e < XC_CHUNK * (la4 - la); e += XC_THREADS) As[(e / (la4 - la)) * la4 + la + e % (la4 - la)] = 0.f;
  if (!same && lb4 > lb)
    for (int e = tid; e < XC_CHUNK * (lb4 - lb); e += XC_THREADS) Bs[(e / (lb4 - lb)) * lb4 + lb + e % (lb4 - lb)] = 0.f;
  for (int64_t rb = r0; rb < r1; rb += XC_CHUNK) {
    // stage the chunk: flattened over (row, column) so that every thread's
    // loads are independent of one another (many in flight); rows past the
    // end are zero
    const int rows = (int)min((int64_t)XC_CHUNK, r1 - rb);
#pragma unroll 4
    for (int e = tid; e < XC_CHUNK * la; e += XC_THREADS) {
      const int rr = e / la, c = e - rr * la;
      float v = 0.f;
      if (rr < rows) {
        const int64_t src = idx ? (int64_t)__ldg(idx + rb + rr) : rb + rr;
        v = A[src * lda + c];
      }
      As[rr * la4 + c] = v;
    }
    if (!same) {
#pragma unroll 4
      for (int e = tid; e < XC_CHUNK * lb; e += XC_THREADS) {
        const int rr = e / lb, c = e - rr * lb;
        float v = 0.f;
        if (rr < rows) {
          const int64_t src = idx ? (int64_t)__ldg(idx + rb + rr) : rb + rr;
          v = B[src * ldb + c] * (wt ? __ldg(wt + rb + rr) : 1.f);
        }
        Bs[rr * lb4 + c] = v;
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int t = 0; t < TPT; ++t) {
        const int tile = (T >= XC_THREADS) ? tid + t * XC_THREADS : tid % T;
        if (tile < T) {
          const int ti = tile / tb, tj = tile - ti * tb;
          for (int rr = rg; rr < rows; rr += R) {
            const float4 a = *(const float4*)(As + rr * la4 + 4 * ti);
            const float4 b = *(const float4*)(Bsrc + rr * lb4 + 4 * tj);
            const float av[4] = {a.x, a.y, a.z, a.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                // Kahan step: y = a b - c; t = s + y; c = (t - s) - y; s = t
                const float y = fmaf(av[p], bv[q], -fc[t][p * 4 + q]);
                const float s2 = f[t][p * 4 + q] + y;
                fc[t][p * 4 + q] = (s2 - f[t][p * 4 + q]) - y;
                f[t][p * 4 + q] = s2;
              }
          }
        }
      }
    }
    __syncthreads();
  }

  // combine row groups (sequentially, fixed order) and write the block partial
  const int LL = la * lb;
  if (R > 1) {
    for (int g = 0; g < R; ++g) {
      if (active && rg == g) {
        const int tile = tid % T;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const dfl v{f[0][e], -fc[0][e]};
          red[tile * 16 + e] = (g == 0) ? v : df_add(red[tile * 16 + e], v);
        }
      }
      __syncthreads();
    }
    for (int e = tid; e < T * 16; e += XC_THREADS) {
      const int tile = e >> 4, w = e & 15;
      const int i = (tile / tb) * 4 + (w >> 2), j = (tile % tb) * 4 + (w & 3);
      if (i < la && j < lb) wsd[(size_t)blockIdx.x * LL + i * lb + j] = red[e];
    }
  } else {
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
      const int tile = tid + t * XC_THREADS;
      if (tile < T) {
        const int ti = tile / tb, tj = tile - ti * tb;
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int i = ti * 4 + (e >> 2), j = tj * 4 + (e & 3);
          if (i < la && j < lb) wsd[(size_t)blockIdx.x * LL + i * lb + j] = dfl{f[t][e], -fc[t][e]};
        }
      }
    }
  }
  if (counter && last_block<1>(counter)) {
    const unsigned G = gridDim.x;
    for (int e = tid; e < LL; e += XC_THREADS) {
      // four independent chains keep several L2 loads in flight (fixed order)
      dfl s0{0.f, 0.f}, s1{0.f, 0.f}, s2{0.f, 0.f}, s3{0.f, 0.f};
      unsigned b = 0;
      for (; b + 4 <= G; b += 4) {
        const float2 v0 = __ldcg(reinterpret_cast<const float2*>(wsd + (size_t)b * LL + e));
        const float2 v1 = __ldcg(reinterpret_cast<const float2*>(wsd + (size_t)(b + 1) * LL + e));
        const float2 v2 = __ldcg(reinterpret_cast<const float2*>(wsd + (size_t)(b + 2) * LL + e));
        const float2 v3 = __ldcg(reinterpret_cast<const float2*>(wsd + (size_t)(b + 3) * LL + e));
        s0 = df_add(s0, dfl{v0.x, v0.y});
        s1 = df_add(s1, dfl{v1.x, v1.y});
        s2 = df_add(s2, dfl{v2.x, v2.y});
        s3 = df_add(s3, dfl{v3.x, v3.y});
      }
      for (; b < G; ++b) {
        const float2 v0 = __ldcg(reinterpret_cast<const float2*>(wsd + (size_t)b * LL + e));
        s0 = df_add(s0, dfl{v0.x, v0.y});
      }
      double s = df_to_double(df_add(df_add(s0, s1), df_add(s2, s3)));
      const int i = e / lb, j = e - i * lb;
      if (lam) s *= lam[i];
      if (i == j) s += shift;
      if (C) C[e] = s;
      if (Cf) Cf[e] = (float)s;
    }
    if (tid == 0) *counter = 0;
  }
}

// Second stage for large reductions: one warp per entry sums the block
// partials (lanes strided over blocks, then a fixed shuffle tree; double-float).
__global__ void xcross_reduce_kernel(const double* __restrict__ ws, int G, int LL, int lb,
                                     const double* __restrict__ lam, double shift, double* C, float* Cf) {
  const int e = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= LL) return;
  const float2* wsd = reinterpret_cast<const float2*>(ws);
  dfl s{0.f, 0.f};
  for (int b = lane; b < G; b += 32) {
    const float2 v = __ldcg(wsd + (size_t)b * LL + e);
    s = df_add(s, dfl{v.x, v.y});
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const dfl t{__shfl_xor_sync(0xffffffffu, s.hi, o), __shfl_xor_sync(0xffffffffu, s.lo, o)};
    s = df_add(s, t);
  }
  if (lane == 0) {
    double v = df_to_double(s);
    const int i = e / lb, j = e - i * lb;
    if (lam) v *= lam[i];
    if (i == j) v += shift;
    if (C) C[e] = v;
    if (Cf) Cf[e] = (float)v;
  }
}

cudaError_t xcross(const float* A, int lda, int la, const float* B, int ldb, int lb, int64_t n,
                   const int32_t* idx, const float* wt, const int* cnt, const double* lam,
                   double shift, double* C, float* Cf, double* ws, unsigned* counter,
                   cudaStream_t st) {
  if (la < 1 || lb < 1 || la > 128 || lb > 128) return cudaErrorInvalidValue;
  const int la4 = (la + 3) & ~3, lb4 = (lb + 3) & ~3;
  const int T = (la4 / 4) * (lb4 / 4);
  const size_t smem = (size_t)XC_CHUNK * (la4 + lb4) * 4 + (size_t)(T < XC_THREADS ? T : 0) * 16 * 8;
  int grid = (int)((n + 255) / 256);
  const int cap = num_sms() * ((size_t)la * lb <= 4096 ? 2 : 1);
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  // many partials of many entries: reduce them with the whole GPU instead of one block
  const int LL = la * lb;
  const bool two_stage = grid >= 16 && (int64_t)grid * LL > 16384;
  unsigned* ctr = two_stage ? nullptr : counter;
  cudaError_t e;
  if (T <= XC_THREADS) {
    e = cudaFuncSetAttribute(xcross_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    xcross_kernel<1><<<grid, XC_THREADS, smem, st>>>(A, lda, la, B, ldb, lb, n, idx, wt, cnt, lam,
                                                     shift, C, Cf, ws, ctr);
  } else if (T <= 2 * XC_THREADS) {
    e = cudaFuncSetAttribute(xcross_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    xcross_kernel<2><<<grid, XC_THREADS, smem, st>>>(A, lda, la, B, ldb, lb, n, idx, wt, cnt, lam,
                                                     shift, C, Cf, ws, ctr);
  } else {
    e = cudaFuncSetAttribute(xcross_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    xcross_kernel<4><<<grid, XC_THREADS, smem, st>>>(A, lda, la, B, ldb, lb, n, idx, wt, cnt, lam,
                                                     shift, C, Cf, ws, ctr);
  }
  count_launches(1);
  if (two_stage) {
    const int warps_per_block = 8;
    xcross_reduce_kernel<<<(LL + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, st>>>(
        ws, grid, LL, lb, lam, shift, C, Cf);
    count_launches(1);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ HALS

constexpr int HALS_ROWS = 64;  // rows per tile = threads per block

// One thread per row.  Per group g (k columns, its own Gram G_g):
//   w_i <- max(0, (Y_i + alpha h_i - sum_{j != i} w_j G_ji) / (G_ii + alpha)),
// i = 0..k-1 in order with the columns already updated (Eq. symhals_update2).
template <int KMAX>
__global__ void __launch_bounds__(HALS_ROWS) hals_kernel(
    float* __restrict__ Fu, const float* __restrict__ Ff, int64_t n, int k, int ng,
    const float* __restrict__ G, float alpha, const float* __restrict__ Y, int ldy,
    const float* __restrict__ U, int l, const float* __restrict__ M, double* part, double* ws,
    unsigned* counter, unsigned* err) {
  extern __shared__ __align__(16) float sm[];
  const int RW = ng * k;         // row width
  const int P = RW + 1;          // odd smem row pitch: conflict-free per-row reads
  const int k4 = (k + 3) & ~3, k4q = k4 / 4;
  float* Gs = sm;                  // ng x k x k4, zero padded (G symmetric: row i = column i)
  float* inv = Gs + ng * k * k4;   // ng x k4
  float* Ms = inv + ng * k4;       // l x k4 (LAI only, ng == 1), zero padded
  float* Ys = Ms + (U ? l * k4 : 0);  // HALS_ROWS x P
  float* Hs = Ys + HALS_ROWS * P;
  float* Ws = Hs + HALS_ROWS * P;
  float* Us = Ws + HALS_ROWS * P;  // HALS_ROWS x (l + 1) (LAI only)
  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  for (int e = tid; e < ng * k * k4; e += HALS_ROWS) {
    const int gi = e / k4, j = e - gi * k4;  // gi = g * k + i
    Gs[e] = j < k ? G[gi * k + j] : 0.f;
  }
  if (U)
    for (int e = tid; e < l * k4; e += HALS_ROWS) {
      const int i = e / k4, j = e - i * k4;
      Ms[e] = j < k ? M[i * k + j] : 0.f;
    }
  __syncthreads();
  for (int e = tid; e < ng * k4; e += HALS_ROWS) {
    const int g = e / k4, i = e - g * k4;
    inv[e] = i < k ? 1.0f / (Gs[(g * k + i) * k4 + i] + alpha) : 0.f;
  }
  __syncthreads();
  const float4* Gs4 = reinterpret_cast<const float4*>(Gs);
  const float4* Ms4 = reinterpret_cast<const float4*>(Ms);

  double tr = 0.0, dd = 0.0;
  bool bad = false;
  const int64_t ntiles = (n + HALS_ROWS - 1) / HALS_ROWS;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t base = tile * HALS_ROWS;
    const int rows = (int)min((int64_t)HALS_ROWS, n - base);
    // coalesced staging, one warp per row (no index division)
    for (int rr = wid; rr < rows; rr += HALS_ROWS / 32) {
      const int64_t g = (base + rr);
      for (int c = lane; c < RW; c += 32) {
        Hs[rr * P + c] = Ff[g * RW + c];
        Ws[rr * P + c] = Fu[g * RW + c];
        if (!U) Ys[rr * P + c] = Y[g * (int64_t)ldy + c];
      }
      if (U)
        for (int c = lane; c < l; c += 32) Us[rr * (l + 1) + c] = U[g * (int64_t)l + c];
    }
    __syncthreads();
    if (tid < rows) {
      const float* yr = Ys + tid * P;
      const float* hr = Hs + tid * P;
      float* wr = Ws + tid * P;
      for (int g = 0; g < ng; ++g) {
        const int o = g * k;
        const float4* Gg4 = Gs4 + (size_t)g * k * k4q;
        float y[KMAX];
        if (U) {  // Y_r = U_r M (LAI product fused into the update), in registers
          const float* ur = Us + tid * (l + 1);
#pragma unroll
          for (int c = 0; c < KMAX; ++c) y[c] = 0.f;
          for (int p = 0; p < l; ++p) {
            const float u = ur[p];
#pragma unroll
            for (int c4 = 0; c4 < KMAX / 4; ++c4)
              if (c4 < k4q) {
                const float4 m = Ms4[p * k4q + c4];
                y[4 * c4 + 0] = fmaf(u, m.x, y[4 * c4 + 0]);
                y[4 * c4 + 1] = fmaf(u, m.y, y[4 * c4 + 1]);
                y[4 * c4 + 2] = fmaf(u, m.z, y[4 * c4 + 2]);
                y[4 * c4 + 3] = fmaf(u, m.w, y[4 * c4 + 3]);
              }
          }
        } else {
#pragma unroll
          for (int c = 0; c < KMAX; ++c) y[c] = c < k ? yr[o + c] : 0.f;
        }
        float w[KMAX];
#pragma unroll
        for (int j = 0; j < KMAX; ++j) w[j] = j < k ? wr[o + j] : 0.f;
#pragma unroll
        for (int i = 0; i < KMAX; ++i) {
          if (i < k) {
            // two independent chains halve the FMA latency of the column update
            float a0 = fmaf(alpha, hr[o + i], y[i]), a1 = 0.f;
#pragma unroll
            for (int j4 = 0; j4 < KMAX / 4; ++j4)
              if (j4 < k4q) {
                const float4 gq = Gg4[i * k4q + j4];
                const float gv[4] = {gq.x, gq.y, gq.z, gq.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  const int j = 4 * j4 + u;
                  if (j != i) {  // zero pads: j >= k adds nothing
                    if (u & 1)
                      a1 = fmaf(-w[j], gv[u], a1);
                    else
                      a0 = fmaf(-w[j], gv[u], a0);
                  }
                }
              }
            w[i] = fmaxf((a0 + a1) * inv[g * k4 + i], 0.f);
          }
        }
#pragma unroll
        for (int j = 0; j < KMAX; ++j)
          if (j < k) {
            if (!isfinite(w[j])) bad = true;
            wr[o + j] = w[j];
            tr += (double)w[j] * (double)y[j];
            const float d = w[j] - hr[o + j];
            dd += (double)d * (double)d;
          }
      }
    }
    __syncthreads();
    for (int rr = tid >> 5; rr < rows; rr += HALS_ROWS / 32)
      for (int c = tid & 31; c < RW; c += 32) Fu[(base + rr) * RW + c] = Ws[rr * P + c];
    __syncthreads();
  }
  if (bad) set_error(err, ERR_NAN);
  __shared__ double sh[32];
  tr = block_sum(tr, sh);
  dd = block_sum(dd, sh);
  if (tid == 0) {
    ws[2 * blockIdx.x] = tr;
    ws[2 * blockIdx.x + 1] = dd;
  }
  if (last_block<1>(counter)) {
    reduce_partials(ws, 2, 2, gridDim.x, part, sh);
    if (tid == 0) *counter = 0;
  }
}

template <int KMAX>
static cudaError_t launch_hals(float* Fu, const float* Ff, int64_t n, int k, int ng, const float* G,
                               double alpha, const float* Y, int ldy, const float* U, int l,
                               const float* M, double* part, double* ws, unsigned* counter,
                               unsigned* err, cudaStream_t st) {
  if (U && ng != 1) return cudaErrorInvalidValue;
  const int RW = ng * k, P = RW + 1, k4 = (k + 3) & ~3;
  size_t smem = (size_t)(ng * k * k4 + ng * k4 + 3 * HALS_ROWS * P) * 4;
  if (U) smem += (size_t)(HALS_ROWS * (l + 1) + l * k4) * 4;
  cudaError_t e = cudaFuncSetAttribute(hals_kernel<KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (n + HALS_ROWS - 1) / HALS_ROWS;
  int grid = (int)std::min<int64_t>(ntiles, (int64_t)num_sms() * 4);
  if (grid < 1) grid = 1;
  hals_kernel<KMAX><<<grid, HALS_ROWS, smem, st>>>(Fu, Ff, n, k, ng, G, (float)alpha, Y, ldy, U, l, M,
                                                   part, ws, counter, err);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t hals_update(float* F_upd, const float* F_fix, int64_t n, int k, int ngroups,
                        const float* G, double alpha, const float* Y, int ldy, const float* U, int l,
                        const float* M, double* part, double* ws, unsigned* counter, unsigned* err,
                        cudaStream_t st) {
  if (k <= 8)
    return launch_hals<8>(F_upd, F_fix, n, k, ngroups, G, alpha, Y, ldy, U, l, M, part, ws, counter, err, st);
  if (k <= 16)
    return launch_hals<16>(F_upd, F_fix, n, k, ngroups, G, alpha, Y, ldy, U, l, M, part, ws, counter, err, st);
  if (k <= 32)
    return launch_hals<32>(F_upd, F_fix, n, k, ngroups, G, alpha, Y, ldy, U, l, M, part, ws, counter, err, st);
  if (k <= 64)
    return launch_hals<64>(F_upd, F_fix, n, k, ngroups, G, alpha, Y, ldy, U, l, M, part, ws, counter, err, st);
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------ apply_small

__global__ void apply_small_kernel(const float* __restrict__ A, int lda, int la,
                                   const float* __restrict__ B, int lb, int64_t n, float* out,
                                   int ldo) {
  extern __shared__ float Bsh[];
  for (int e = threadIdx.x; e < la * lb; e += blockDim.x) Bsh[e] = B[e];
  __syncthreads();
  const int chunks = (lb + 15) / 16;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * chunks) return;
  const int64_t i = t / chunks;
  const int c0 = (int)(t - i * chunks) * 16;
  float acc[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j] = 0.f;
  for (int c = 0; c < la; ++c) {
    const float a = A[i * lda + c];
    const float* b = Bsh + c * lb + c0;
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (c0 + j < lb) acc[j] = fmaf(a, b[j], acc[j]);
  }
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if (c0 + j < lb) out[i * ldo + c0 + j] = acc[j];
}

cudaError_t apply_small(const float* A, int lda, int la, const float* B, int lb, int64_t n,
                        float* out, int ldo, cudaStream_t st) {
  const size_t smem = (size_t)la * lb * 4;
  cudaError_t e = cudaFuncSetAttribute(apply_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t work = n * ((lb + 15) / 16);
  const int grid = (int)((work + 255) / 256);
  apply_small_kernel<<<grid, 256, smem, st>>>(A, lda, la, B, lb, n, out, ldo);
  count_launches(1);
  return cudaGetLastError();
}

// ------------------------------------------------------------- leverage

constexpr int LEV_ROWS = 128;

// One thread per row; the block's rows are staged through shared memory with
// coalesced loads (row pitch k + 1 avoids bank conflicts).
template <int KMAX>
__global__ void __launch_bounds__(LEV_ROWS) leverage_kernel(const float* __restrict__ F, int64_t n, int k,
                                                            const float* __restrict__ Rinv, double* lev) {
  __shared__ float Rs[KMAX * KMAX];
  __shared__ float Fs[LEV_ROWS * (KMAX + 1)];
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) Rs[e] = Rinv[e];
  const int64_t base = (int64_t)blockIdx.x * LEV_ROWS;
  const int rows = (int)min((int64_t)LEV_ROWS, n - base);
  for (int e = threadIdx.x; e < rows * k; e += blockDim.x) {
    const int rr = e / k, c = e - rr * k;
    Fs[rr * (k + 1) + c] = F[base * k + e];
  }
  __syncthreads();
  if ((int)threadIdx.x >= rows) return;
  float h[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) h[j] = j < k ? Fs[threadIdx.x * (k + 1) + j] : 0.f;
  float s = 0.f;
  // z_j = sum_{p <= j} h_p Rinv[p][j]  (Rinv upper triangular)
#pragma unroll
  for (int j = 0; j < KMAX; ++j) {
    if (j < k) {
      float z0 = 0.f, z1 = 0.f;
#pragma unroll
      for (int p = 0; p <= j; ++p) {
        if (p & 1)
          z1 = fmaf(h[p], Rs[p * k + j], z1);
        else
          z0 = fmaf(h[p], Rs[p * k + j], z0);
      }
      const float z = z0 + z1;
      s = fmaf(z, z, s);
    }
  }
  lev[base + threadIdx.x] = (double)s;
}

cudaError_t leverage_rows(const float* F, int64_t n, int k, const float* Rinv, double* lev,
                          cudaStream_t st) {
  const int grid = (int)((n + LEV_ROWS - 1) / LEV_ROWS);
  if (k <= 16)
    leverage_kernel<16><<<grid, LEV_ROWS, 0, st>>>(F, n, k, Rinv, lev);
  else if (k <= 32)
    leverage_kernel<32><<<grid, LEV_ROWS, 0, st>>>(F, n, k, Rinv, lev);
  else if (k <= 64)
    leverage_kernel<64><<<grid, LEV_ROWS, 0, st>>>(F, n, k, Rinv, lev);
  else
    return cudaErrorInvalidValue;
  count_launches(1);
  return cudaGetLastError();
}

// ------------------------------------------------------------- objective

__global__ void objective_kernel(const double* normX2, const double* Ga, const double* Gb, int k,
                                 const double* part, const double* alpha, double* out, int* cnt,
                                 int cap) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) s += Ga[e] * Gb[e];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    const double v = normX2[0] + s - 2.0 * part[0] + alpha[0] * part[1];
    if (cnt) {
      const int t = *cnt;
      if (t < cap) out[t] = v;
      *cnt = t + 1;
    } else {
      out[0] = v;
    }
  }
}

cudaError_t objective(const double* normX2, const double* Ga, const double* Gb, int k,
                      const double* part, const double* alpha, double* out, int* cnt, int cap,
                      cudaStream_t st) {
  objective_kernel<<<1, 256, 0, st>>>(normX2, Ga, Gb, k, part, alpha, out, cnt, cap);
  count_launches(1);
  return cudaGetLastError();
}

// out[0] = sum a .* b, out[1] = sum (a - b)^2 over `count` entries (FP64, last block finalises).
__global__ void pair_reduce_kernel(const float* __restrict__ a, const float* __restrict__ b,
                                   int64_t count, double* out, double* ws, unsigned* counter) {
  __shared__ double sh[32];
  double s0 = 0.0, s1 = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double x = a[t], y = b[t];
    s0 += x * y;
    s1 += (x - y) * (x - y);
  }
  s0 = block_sum(s0, sh);
  s1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    ws[2 * blockIdx.x] = s0;
    ws[2 * blockIdx.x + 1] = s1;
  }
  if (last_block<1>(counter)) {
    reduce_partials(ws, 2, 2, gridDim.x, out, sh);
    if (threadIdx.x == 0) *counter = 0;
  }
}

cudaError_t pair_reduce(const float* a, const float* b, int64_t count, double* out, double* ws,
                        unsigned* counter, cudaStream_t st) {
  pair_reduce_kernel<<<num_sms() * 2, 256, 0, st>>>(a, b, count, out, ws, counter);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void sumsq_kernel(const double* v, int l, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < l; ++i) s += v[i] * v[i];
    out[0] = s;
  }
}

cudaError_t sumsq(const double* v, int l, double* out, cudaStream_t st) {
  sumsq_kernel<<<1, 32, 0, st>>>(v, l, out);
  count_launches(1);
  return cudaGetLastError();
}

// ------------------------------------------------------- projected gradient

__global__ void proj_grad_kernel(const float* __restrict__ F, const float* __restrict__ O,
                                 const float* __restrict__ Y, const float* __restrict__ Gm,
                                 int64_t n, int k, const double* alpha, double* acc) {
  extern __shared__ float Gs[];
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) Gs[e] = Gm[e];
  __syncthreads();
  const float a = (float)alpha[0];
  double s = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * k;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / k;
    const int c = (int)(t - i * k);
    float g = 0.f;
    for (int j = 0; j < k; ++j) g = fmaf(F[i * k + j], Gs[j * k + c], g);
    const float f = F[t];
    const double grad = 2.0 * ((double)g - (double)Y[t]) + 2.0 * (double)a * ((double)f - (double)O[t]);
    if (grad < 0.0 || f > 0.f) s += grad * grad;
  }
  __shared__ double sh[32];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) atomicAdd(acc, s);
}

cudaError_t proj_grad_sq(const float* F, const float* Other, const float* Y, const float* Gother,
                         int64_t n, int k, const double* alpha, double* acc, cudaStream_t st) {
  const int grid = num_sms() * 4;
  proj_grad_kernel<<<grid, 256, (size_t)k * k * 4, st>>>(F, Other, Y, Gother, n, k, alpha, acc);
  count_launches(1);
  return cudaGetLastError();
}

// ----------------------------------------------------------- generators

// Omega[i, 2p], Omega[i, 2p+1] from Philox counter (p, i lo, i hi, TAG_OMEGA):
// u1 = (x0 + 1) 2^-32, u2 = x1 2^-32, Box-Muller in double.
__global__ void gaussian_kernel(float* out, int64_t n, int l, uint32_t k0, uint32_t k1) {
  const int np = (l + 1) / 2;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * np) return;
  const int64_t i = t / np;
  const int p = (int)(t - i * np);
  const Philox4 r = philox4x32_10((uint32_t)p, (uint32_t)i, (uint32_t)(i >> 32), TAG_OMEGA, k0, k1);
  const double u1 = ((double)r.x0 + 1.0) * 0x1p-32;
  const double u2 = (double)r.x1 * 0x1p-32;
  const double rad = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  out[i * l + 2 * p] = (float)(rad * c);
  if (2 * p + 1 < l) out[i * l + 2 * p + 1] = (float)(rad * s);
}

cudaError_t philox_gaussian(float* out, int64_t n, int l, uint64_t seed, cudaStream_t st) {
  const int64_t work = n * ((l + 1) / 2);
  gaussian_kernel<<<(int)((work + 255) / 256), 256, 0, st>>>(out, n, l, (uint32_t)seed,
                                                             (uint32_t)(seed >> 32));
  count_launches(1);
  return cudaGetLastError();
}

// H[i, j] = x0 2^-32 * scale, counter (j, i lo, i hi, TAG_INIT); scale =
// scale_mul * sqrt(scale_num[0]) when scale_num != NULL, else 1.
__global__ void uniform_kernel(float* out, int64_t n, int k, uint32_t k0, uint32_t k1,
                               const double* scale_num, double scale_mul) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int64_t i = t / k;
  const int j = (int)(t - i * k);
  const Philox4 r = philox4x32_10((uint32_t)j, (uint32_t)i, (uint32_t)(i >> 32), TAG_INIT, k0, k1);
  double v = (double)r.x0 * 0x1p-32;
  if (scale_num) v *= scale_mul * sqrt(scale_num[0]);
  out[t] = (float)v;
}

cudaError_t philox_uniform(float* out, int64_t n, int k, uint64_t seed, const double* scale_num,
                           double scale_mul, cudaStream_t st) {
  const int64_t work = n * k;
  uniform_kernel<<<(int)((work + 255) / 256), 256, 0, st>>>(out, n, k, (uint32_t)seed,
                                                            (uint32_t)(seed >> 32), scale_num,
                                                            scale_mul);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void convert_bf16_kernel(const float* x, int64_t n, int64_t ldx, __nv_bfloat16* xb,
                                    int64_t ldb) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * ldb;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ldb, j = t - i * ldb;
    xb[t] = __float2bfloat16_rn(j < n ? x[i * ldx + j] : 0.f);
  }
}

cudaError_t convert_bf16(const float* x, int64_t n, int64_t ldx, uint16_t* xb, int64_t ldb,
                         cudaStream_t st) {
  convert_bf16_kernel<<<num_sms() * 8, 256, 0, st>>>(x, n, ldx, (__nv_bfloat16*)xb, ldb);
  count_launches(1);
  return cudaGetLastError();
}

// Per-row E4M3 quantisation: scale_i = max_j |X_ij| / 448 (1 for a zero row).
__global__ void quantize_fp8_kernel(const float* x, int64_t n, int64_t ldx, uint8_t* x8, int64_t ld8,
                                    float* rs) {
  __shared__ float shm[32];
  const int64_t i = blockIdx.x;
  float m = 0.f;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) m = fmaxf(m, fabsf(x[i * ldx + j]));
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = threadIdx.x < (blockDim.x >> 5) ? shm[threadIdx.x] : 0.f;
    t = warp_max(t);
    if (threadIdx.x == 0) shm[0] = t;
  }
  __syncthreads();
  const float mx = shm[0];
  const float scale = mx > 0.f ? mx / 448.0f : 1.0f;
  const float invs = 1.0f / scale;
  for (int64_t j = threadIdx.x; j < ld8; j += blockDim.x) {
    const float v = j < n ? x[i * ldx + j] * invs : 0.f;
    const __nv_fp8_e4m3 q(v);  // round to nearest, saturating to finite
    x8[i * ld8 + j] = q.__x;
  }
  if (threadIdx.x == 0) rs[i] = scale;
}

cudaError_t quantize_fp8(const float* x, int64_t n, int64_t ldx, uint8_t* x8, int64_t ld8,
                         float* row_scale, cudaStream_t st) {
  quantize_fp8_kernel<<<(unsigned)n, 256, 0, st>>>(x, n, ldx, x8, ld8, row_scale);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void check_factor_kernel(const float* F, int64_t count, unsigned* flags) {
  bool neg = false, bad = false;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float v = F[t];
    if (!isfinite(v)) bad = true;
    if (v < 0.f) neg = true;
  }
  if (neg) atomicOr(flags, 1u);
  if (bad) atomicOr(flags, 2u);
}

cudaError_t check_factor(const float* F, int64_t count, unsigned* flags, cudaStream_t st) {
  check_factor_kernel<<<num_sms() * 2, 256, 0, st>>>(F, count, flags);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void normalize_rows_kernel(const float* in, int64_t n, int l, float* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int c = 0; c < l; ++c) s += (double)in[i * l + c] * in[i * l + c];
  const float inv = s > 0.0 ? (float)(1.0 / sqrt(s)) : 0.f;
  for (int c = 0; c < l; ++c) out[i * l + c] = in[i * l + c] * inv;
}

cudaError_t normalize_rows(const float* in, int64_t n, int l, float* out, cudaStream_t st) {
  normalize_rows_kernel<<<(int)((n + 255) / 256), 256, 0, st>>>(in, n, l, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace symnmf
