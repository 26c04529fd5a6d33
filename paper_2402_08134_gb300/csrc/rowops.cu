// Row-streaming kernels of the SymNMF hot path: X statistics, cross products /
// Grams with compensated accumulation, LAI expansion Y = U (Lambda U^T F)
// (Alg. LAI-SymNMF), objective and projected-gradient reductions, and the
// Philox generators.  The full-X HALS update is in hals.cu, the leverage-score
// row pass in leverage.cu.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "dfloat.cuh"
#include "kernels.h"

namespace symnmf {

// ---------------------------------------------------------------- xstats

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

// block partials of up to XC_MAX_BLOCKS_PER_SM blocks per SM
constexpr int XC_MAX_BLOCKS_PER_SM = 4;
size_t xcross_ws_doubles(int la, int lb) { return (size_t)XC_MAX_BLOCKS_PER_SM * num_sms() * la * lb + 64; }

// C = A^T diag(wt) B over (gathered) rows.  Each thread owns 4 x 4 tiles of
// C.  It sums up to XC_SUB of its rows with plain FMAs, then adds that sum to
// a Kahan-compensated FP32 total, so the error stays at a few XC_SUB ulps
// however many rows the thread covers, at one FMA per product.  Row groups
// and block partials combine as double-float pairs (dfloat.cuh): no FP64
// arithmetic, which is scarce on this part.  The trace-trick objective cancels
// terms of size ||X||^2, so the Grams need this accuracy.  Block partials are
// summed in block order (deterministic), by the last block or by a second
// kernel.  VEC: 16-byte loads of whole rows (la, lb, lda, ldb multiples of 4,
// aligned operands).  A Gram of rows without weights, VEC and at most
// XC_PIPE_MAX columns, stages its row chunks with asynchronous 16-byte copies
// into two buffers, the next chunk in flight while the current one is summed.
constexpr int XC_SUB = 32;
constexpr int XC_PIPE_MAX = 64;

__device__ __forceinline__ void xc_cp_async16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void xc_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void xc_cp_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Tile index -> (row tile, column tile): row-major over all ta x tb tiles, or
// over the upper triangle (ti <= tj) of a symmetric product.
__device__ __forceinline__ void xc_tile(int tile, bool sym, int ta, int tb, int& ti, int& tj) {
  if (!sym) {
    ti = tile / tb;
    tj = tile - ti * tb;
    return;
  }
  ti = 0;
  while (tile >= ta - ti) {
    tile -= ta - ti;
    ++ti;
  }
  tj = ti + tile;
}

// Entry (i, j) of a block partial; a symmetric product keeps i <= j and
// writes it to both positions.
__device__ __forceinline__ void xc_emit(dfl* out, int la, int lb, bool sym, int i, int j, dfl v) {
  if (i >= la || j >= lb) return;
  if (!sym) {
    out[i * lb + j] = v;
  } else if (i <= j) {
    out[i * lb + j] = v;
    out[j * lb + i] = v;
  }
}

template <int TPT, bool VEC>
__global__ void __launch_bounds__(XC_THREADS) xcross_kernel(
    const float* __restrict__ A, int lda, int la, const float* __restrict__ B, int ldb, int lb,
    int64_t n, const int32_t* __restrict__ idx, const float* __restrict__ wt, const int* cnt,
    const double* __restrict__ lam, double shift, double* C, float* Cf, double* ws,
    unsigned* counter) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int la4 = (la + 3) & ~3, lb4 = (lb + 3) & ~3;
  float* As = (float*)smraw;
  // a Gram (same operand, no weights) stages its rows once
  const bool same = (A == B) && (lda == ldb) && (la == lb) && !wt;
  const bool pipe = VEC && same && la4 <= XC_PIPE_MAX;
  float* Bs = As + XC_CHUNK * la4;  // the second buffer of As when pipe
  // the row-group sums reuse the staging buffers after the last chunk
  dfl* red = (dfl*)smraw;
  dfl* wsd = reinterpret_cast<dfl*>(ws);  // the partials are double-float pairs
  // a symmetric product (same operand on both sides, weights allowed) covers
  // the upper tiles only and mirrors them: exactly symmetric, half the work
  const bool sym = (A == B) && (lda == ldb) && (la == lb);
  const int ta = la4 >> 2, tb = lb4 >> 2, T = sym ? ta * (ta + 1) / 2 : ta * tb;
  const int tid = threadIdx.x, nt = blockDim.x;  // nt = XC_THREADS when T > nt
  const int R = T >= nt ? 1 : nt / T;
  const int rg = T >= nt ? 0 : tid / T;
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

  const float* Bsrc = same ? As : Bs;
  // staging map: each thread copies one 4-column group of rows my_r, my_r + rpp, ...
  const int a_r = tid / ta, a_c = tid - a_r * ta, a_rpp = nt / ta;
  const int b_r = tid / tb, b_c = tid - b_r * tb, b_rpp = nt / tb;
  // each thread's tiles
  int tile_i[TPT], tile_j[TPT];
#pragma unroll
  for (int t = 0; t < TPT; ++t) {
    const int tile = (T >= nt) ? tid + t * nt : tid % T;
    xc_tile(tile < T ? tile : 0, sym, ta, tb, tile_i[t], tile_j[t]);
    if (tile >= T || !active) tile_i[t] = -1;  // idle threads own no tile
  }
  // chunk [rb, rb + XC_CHUNK) of the Gram rows into dst by asynchronous copies
  // (rows past the end are zero), as one commit group
  auto stage_async = [&](int64_t rb, float* dst) {
    if (rb < r1 && a_r < a_rpp) {
      const int rows = (int)min((int64_t)XC_CHUNK, r1 - rb);
      for (int rr = a_r; rr < XC_CHUNK; rr += a_rpp) {
        float* d = dst + rr * la4 + 4 * a_c;
        if (rr < rows) {
          const int64_t src = idx ? (int64_t)__ldg(idx + rb + rr) : rb + rr;
          xc_cp_async16(d, A + src * lda + 4 * a_c);
        } else {
          *reinterpret_cast<float4*>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    }
    xc_cp_commit();
  };
  if (pipe) stage_async(r0, As);
  int it = 0;
  for (int64_t rb = r0; rb < r1; rb += XC_CHUNK, ++it) {
    const int rows = (int)min((int64_t)XC_CHUNK, r1 - rb);
    const float* Acur = As;
    if (pipe) {
      // the other buffer was last read before the previous chunk's closing barrier
      Acur = (it & 1) ? Bs : As;
      stage_async(rb + XC_CHUNK, (it & 1) ? As : Bs);
      xc_cp_wait_prev();  // this chunk's copies (all groups but the newest) have landed
    } else if (a_r < a_rpp) {
      // stage the chunk (rows past the end and pad columns are zero)
#pragma unroll 4
      for (int rr = a_r; rr < XC_CHUNK; rr += a_rpp) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (rr < rows) {
          const int64_t src = idx ? (int64_t)__ldg(idx + rb + rr) : rb + rr;
          const float* ar = A + src * lda + 4 * a_c;
          if constexpr (VEC) {
            v = __ldg(reinterpret_cast<const float4*>(ar));
          } else {
            const int c = 4 * a_c;
            v.x = __ldg(ar);
            if (c + 1 < la) v.y = __ldg(ar + 1);
            if (c + 2 < la) v.z = __ldg(ar + 2);
            if (c + 3 < la) v.w = __ldg(ar + 3);
          }
        }
        *reinterpret_cast<float4*>(As + rr * la4 + 4 * a_c) = v;
      }
    }
    if (!same && b_r < b_rpp) {
#pragma unroll 4
      for (int rr = b_r; rr < XC_CHUNK; rr += b_rpp) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (rr < rows) {
          const int64_t src = idx ? (int64_t)__ldg(idx + rb + rr) : rb + rr;
          const float* br = B + src * ldb + 4 * b_c;
          if constexpr (VEC) {
            v = __ldg(reinterpret_cast<const float4*>(br));
          } else {
            const int c = 4 * b_c;
            v.x = __ldg(br);
            if (c + 1 < lb) v.y = __ldg(br + 1);
            if (c + 2 < lb) v.z = __ldg(br + 2);
            if (c + 3 < lb) v.w = __ldg(br + 3);
          }
          if (wt) {
            const float w = __ldg(wt + rb + rr);
            v.x *= w, v.y *= w, v.z *= w, v.w *= w;
          }
        }
        *reinterpret_cast<float4*>(Bs + rr * lb4 + 4 * b_c) = v;
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int t = 0; t < TPT; ++t) {
        if (tile_i[t] >= 0) {
          const float* ap = Acur + 4 * tile_i[t];
          const float* bp = (same ? Acur : Bsrc) + 4 * tile_j[t];
          for (int s0 = rg; s0 < rows; s0 += XC_SUB * R) {
            const int s1 = min(rows, s0 + XC_SUB * R);
            float p[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) p[e] = 0.f;
#pragma unroll 4
            for (int rr = s0; rr < s1; rr += R) {
              const float4 a = *reinterpret_cast<const float4*>(ap + rr * la4);
              const float4 b = *reinterpret_cast<const float4*>(bp + rr * lb4);
              const float av[4] = {a.x, a.y, a.z, a.w};
              const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
              for (int pp = 0; pp < 4; ++pp)
#pragma unroll
                for (int q = 0; q < 4; ++q) p[pp * 4 + q] = fmaf(av[pp], bv[q], p[pp * 4 + q]);
            }
#pragma unroll
            for (int e = 0; e < 16; ++e) kahan_add(f[t][e], fc[t][e], p[e]);
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
    for (int e = tid; e < T * 16; e += nt) {
      int ti, tj;
      xc_tile(e >> 4, sym, ta, tb, ti, tj);
      xc_emit(wsd + (size_t)blockIdx.x * LL, la, lb, sym, ti * 4 + ((e & 15) >> 2), tj * 4 + (e & 3), red[e]);
    }
  } else {
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
      if (tile_i[t] >= 0) {
#pragma unroll
        for (int e = 0; e < 16; ++e)
          xc_emit(wsd + (size_t)blockIdx.x * LL, la, lb, sym, tile_i[t] * 4 + (e >> 2), tile_j[t] * 4 + (e & 3),
                  dfl{f[t][e], -fc[t][e]});
      }
    }
  }
  if (counter && last_block<1>(counter)) {
    const unsigned G = gridDim.x;
    for (int e = tid; e < LL; e += nt) {
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
                   cudaStream_t st, int max_blocks_per_sm) {
  if (la < 1 || lb < 1 || la > 128 || lb > 128) return cudaErrorInvalidValue;
  if (max_blocks_per_sm < 1 || max_blocks_per_sm > XC_MAX_BLOCKS_PER_SM) return cudaErrorInvalidValue;
  const int la4 = (la + 3) & ~3, lb4 = (lb + 3) & ~3;
  const bool sym = (A == B) && (lda == ldb) && (la == lb);
  const bool same = sym && !wt;
  const int T = sym ? (la4 / 4) * (la4 / 4 + 1) / 2 : (la4 / 4) * (lb4 / 4);
  // as many threads as tiles x row groups use (whole warps): narrow products
  // leave room for more blocks per SM
  const int nthreads = T >= XC_THREADS ? XC_THREADS : ((XC_THREADS / T) * T + 31) / 32 * 32;
  const int tpt = T <= XC_THREADS ? 1 : T <= 2 * XC_THREADS ? 2 : 4;
  const bool vec = (la % 4) == 0 && (lb % 4) == 0 && (lda % 4) == 0 && (ldb % 4) == 0 &&
                   (((uintptr_t)A | (uintptr_t)B) & 15) == 0;
  const bool pipe = vec && same && la4 <= XC_PIPE_MAX;  // two buffers of A rows
  // the row-group sums reuse the staging space after the last chunk
  const size_t smem = std::max((size_t)XC_CHUNK * (la4 + (same ? (pipe ? la4 : 0) : lb4)) * 4,
                               (size_t)(T < XC_THREADS ? T : 0) * 16 * 8);
  const void* fn = tpt == 1 ? (vec ? (const void*)xcross_kernel<1, true> : (const void*)xcross_kernel<1, false>)
                   : tpt == 2 ? (vec ? (const void*)xcross_kernel<2, true> : (const void*)xcross_kernel<2, false>)
                              : (vec ? (const void*)xcross_kernel<4, true> : (const void*)xcross_kernel<4, false>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nthreads, smem);
  if (e != cudaSuccess) return e;
  per_sm = std::max(1, std::min(per_sm, max_blocks_per_sm));
  int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * per_sm);
  if (grid < 1) grid = 1;
  // many partials of many entries: reduce them with the whole GPU instead of one block
  const int LL = la * lb;
  const bool two_stage = grid >= 16 && (int64_t)grid * LL > 16384;
  unsigned* ctr = two_stage ? nullptr : counter;
  void* args[] = {(void*)&A, (void*)&lda, (void*)&la, (void*)&B,   (void*)&ldb, (void*)&lb, (void*)&n,   (void*)&idx,
                  (void*)&wt, (void*)&cnt, (void*)&lam, (void*)&shift, (void*)&C,   (void*)&Cf, (void*)&ws, (void*)&ctr};
  e = cudaLaunchKernel(fn, dim3(grid), dim3(nthreads), args, smem, st);
  if (e != cudaSuccess) return e;
  count_launches(1);
  if (two_stage) {
    const int warps_per_block = 8;
    xcross_reduce_kernel<<<(LL + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, st>>>(
        ws, grid, LL, lb, lam, shift, C, Cf);
    count_launches(1);
  }
  return cudaGetLastError();
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

// out[0] = sum w .* y, out[1] = sum (w - h)^2 in one pass (the residual's two sums).
__global__ void resid_reduce_kernel(const float* __restrict__ w, const float* __restrict__ h,
                                    const float* __restrict__ y, int64_t count, double* out, double* ws,
                                    unsigned* counter) {
  __shared__ double sh[32];
  double s0 = 0.0, s1 = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double x = w[t];
    const double d = x - (double)h[t];
    s0 += x * (double)y[t];
    s1 += d * d;
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

cudaError_t resid_reduce(const float* w, const float* h, const float* y, int64_t count, double* out, double* ws,
                         unsigned* counter, cudaStream_t st) {
  resid_reduce_kernel<<<num_sms() * 2, 256, 0, st>>>(w, h, y, count, out, ws, counter);
  count_launches(1);
  return cudaGetLastError();
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

// ||U diag(lam) U^T||_F^2 = sum_ij lam_i lam_j (U^T U)_ij^2 from the Gram Gu =
// U^T U (l x l, FP64), summed in FP64 in a fixed order: the exact norm of the
// operator the LAI sweeps apply, whose U is orthonormal only to FP32 rounding.
__global__ void lai_norm2_kernel(const double* Gu, const double* lam, int l, double* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int i = e / l, j = e - i * l;
    const double g = Gu[e];
    s += lam[i] * lam[j] * g * g;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[0] = s;
}

cudaError_t lai_norm2(const double* Gu, const double* lam, int l, double* out, cudaStream_t st) {
  lai_norm2_kernel<<<1, 256, 0, st>>>(Gu, lam, l, out);
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
  // the scale once per block: FP64 square roots are scarce on this part
  __shared__ double scale;
  if (threadIdx.x == 0) scale = scale_num ? scale_mul * sqrt(scale_num[0]) : 1.0;
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int64_t i = t / k;
  const int j = (int)(t - i * k);
  const Philox4 r = philox4x32_10((uint32_t)j, (uint32_t)i, (uint32_t)(i >> 32), TAG_INIT, k0, k1);
  double v = (double)r.x0 * 0x1p-32;
  if (scale_num) v *= scale;
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
