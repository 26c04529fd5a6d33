// Rank-safe orthonormalisation of the range finder's blocks (Alg. RRF:
// Q = orth(Y) after every product with X): shifted CholeskyQR3 (Fukaya,
// Kannan, Nakatsukasa, Yamamoto, Yanagisawa, SIAM J. Sci. Comput. 2020).
// Pass 1 factors Y^T Y + 1e-6 max_i (Y^T Y)_ii I, which is positive definite
// whatever the rank of Y; passes 2 and 3 are plain CholeskyQR.  Each pass:
// G = Y^T Y (FP64 sum of compensated FP32 partials), G + sI = R^T R in FP64
// (chol.cuh), then every row y of Y becomes the solution x of x R = y
// (forward substitution in FP32).  Pivots below 1e-12 (pass 1) or 1e-10
// (passes 2, 3) of the largest diagonal entry are dropped -- a zero column of
// Q -- so a rank-deficient sketch keeps exactly its numerical range.
//
// For the range finder's sizes (n = 2e4 .. 5e4, l <= 96) the three passes
// run in ONE cooperative launch: CTA c keeps rows [n c / grid, n (c+1) / grid)
// of Y in shared memory (column-major, like the LAI engine), writes FP64
// partial Grams, and after a grid barrier and a sliced fixed-order reduction
// every CTA factors the same l x l matrix itself (identical inputs and code:
// identical R everywhere) and solves its own rows.  When the rows do not fit,
// the passes run as separate kernels (cross product, single-CTA Cholesky,
// row solve) over global memory.
#include <math.h>

#include <algorithm>

#include "chol.cuh"
#include "common.cuh"
#include "kernels.h"
#include "persist.cuh"

namespace symnmf {

constexpr int CQ_THREADS = 256;

__device__ __forceinline__ void cq_kahan(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Forward substitution x R = y for one row held in registers: R strictly upper
// part in Rf (l x l4, zero on and below the diagonal and in the pads), 1 / R_ii
// in rinv (0 for a dropped pivot).
template <int LMAX>
__device__ __forceinline__ void cq_solve_row(float (&s)[LMAX], const float* Rf, const float* rinv, int l, int l4) {
#pragma unroll
  for (int i = 0; i < LMAX; ++i) {
    if (i < l) {
      const float xi = s[i] * rinv[i];
      s[i] = xi;
      const float4* Ri = reinterpret_cast<const float4*>(Rf + i * l4);
#pragma unroll
      for (int j4 = (i + 1) / 4; j4 < LMAX / 4; ++j4) {
        if (4 * j4 < l) {
          const float4 r = Ri[j4];
          s[4 * j4 + 0] = fmaf(-xi, r.x, s[4 * j4 + 0]);
          s[4 * j4 + 1] = fmaf(-xi, r.y, s[4 * j4 + 1]);
          s[4 * j4 + 2] = fmaf(-xi, r.z, s[4 * j4 + 2]);
          s[4 * j4 + 3] = fmaf(-xi, r.w, s[4 * j4 + 3]);
        }
      }
    }
  }
}

// R (FP64, upper, in A) -> Rf (FP32 strictly upper, l x l4) and rinv (l4).
__device__ __forceinline__ void cq_pack_r(const double* A, const int* dropped, int l, int l4, float* Rf,
                                          float* rinv) {
  for (int e = threadIdx.x; e < l * l4; e += blockDim.x) {
    const int i = e / l4, j = e - i * l4;
    Rf[e] = (j > i && j < l) ? (float)A[i * l + j] : 0.f;
  }
  for (int i = threadIdx.x; i < l4; i += blockDim.x) rinv[i] = (i < l && !dropped[i]) ? (float)(1.0 / A[i * l + i]) : 0.f;
}

__host__ __device__ inline int cq_tiles(int l) {
  const int b = (l + 3) / 4;
  return b * (b + 1) / 2;
}

__host__ __device__ inline int cq_row_groups(int l) {
  const int T = cq_tiles(l);
  return T >= CQ_THREADS ? 1 : std::min(4, CQ_THREADS / T);
}

// pass 0 is the shifted one
__host__ __device__ inline double cq_shift(int pass) { return pass == 0 ? -1e-6 : 0.0; }
__host__ __device__ inline double cq_drop(int pass) { return pass == 0 ? 1e-12 : 1e-10; }

// ------------------------------------------------------- one-launch engine

struct CqArgs {
  float* S;        // n x l, row-major: input Y, output Q
  int64_t n;
  int l;
  int rp;          // padded rows per CTA (multiple of 4)
  double* part;    // [grid * RG][l * l] partial Grams
  double* fin;     // [l * l]
  unsigned* bar;   // 2 * GRID_GEN words, zeroed
  unsigned* err;
};

__host__ __device__ inline size_t cq_engine_smem(int l, int rp) {
  const int l4 = (l + 3) & ~3;
  size_t b = (size_t)l * l * 8 + (size_t)2 * l * 8;  // A, piv
  b = (b + 15) & ~(size_t)15;
  b += (size_t)l4 * rp * 4;                           // Yt
  b += (size_t)l * l4 * 4 + (size_t)l4 * 4;            // Rf, rinv
  b += (size_t)l * 4 + (size_t)cq_tiles(l) * 4;        // dropped, tile table
  return b;
}

template <int LMAX>
__global__ void __launch_bounds__(CQ_THREADS, 1) cholqr_engine_kernel(CqArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int l = a.l, l4 = (l + 3) & ~3, RP = a.rp, E = l * l;
  double* A = reinterpret_cast<double*>(smraw);  // l x l
  double* piv = A + l * l;                        // 2 l
  float* Yt = reinterpret_cast<float*>(smraw + (((size_t)l * l * 8 + (size_t)2 * l * 8 + 15) & ~(size_t)15));
  float* Rf = Yt + l4 * RP;                       // l x l4
  float* rinv = Rf + l * l4;                      // l4
  int* dropped = reinterpret_cast<int*>(rinv + l4);
  int* tiles = dropped + l;                       // (bi << 16) | bj, bi <= bj

  const int tid = threadIdx.x;
  const int64_t r0 = (a.n * blockIdx.x) / gridDim.x;
  const int R = (int)((a.n * (blockIdx.x + 1)) / gridDim.x - r0);
  const int nb = l4 / 4, T = cq_tiles(l), RG = cq_row_groups(l);

  for (int e = tid; e < l4 * RP; e += CQ_THREADS) Yt[e] = 0.f;
  if (tid == 0) {
    int t = 0;
    for (int bi = 0; bi < nb; ++bi)
      for (int bj = bi; bj < nb; ++bj) tiles[t++] = (bi << 16) | bj;
  }
  __syncthreads();
  {
    const float* Sg = a.S + r0 * l;
    for (int e = tid; e < R * l; e += CQ_THREADS) {
      const int r = e / l, c = e - r * l;
      Yt[c * RP + r] = Sg[e];
    }
  }
  __syncthreads();

  for (int pass = 0; pass < 3; ++pass) {
    // partial Gram of this CTA's rows: 4x4 upper tiles, four rows per float4 step
    for (int w = tid; w < T * RG; w += CQ_THREADS) {
      const int tile = w % T, rg = w / T;
      const int bi = tiles[tile] >> 16, bj = tiles[tile] & 0xffff;
      const float* Ab = Yt + 4 * bi * RP;
      const float* Bb = Yt + 4 * bj * RP;
      float acc[16], cmp[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) acc[e] = cmp[e] = 0.f;
      for (int c = rg; c < RP / 4; c += RG) {
        float4 av[4], bv[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          av[p] = reinterpret_cast<const float4*>(Ab + p * RP)[c];
          bv[p] = reinterpret_cast<const float4*>(Bb + p * RP)[c];
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float v = av[p].x * bv[q].x;
            v = fmaf(av[p].y, bv[q].y, v);
            v = fmaf(av[p].z, bv[q].z, v);
            v = fmaf(av[p].w, bv[q].w, v);
            cq_kahan(acc[p * 4 + q], cmp[p * 4 + q], v);
          }
      }
      double* rec = a.part + ((size_t)blockIdx.x * RG + rg) * E;
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int i = 4 * bi + (e >> 2), j = 4 * bj + (e & 3);
        if (i < l && j < l) {
          const double v = (double)acc[e] - (double)cmp[e];
          rec[i * l + j] = v;
          rec[j * l + i] = v;
        }
      }
    }
    if (!grid_sync_bounded(a.bar, a.err)) return;
    // sliced fixed-order reduction of the grid * RG records into fin
    {
      const unsigned nrec = gridDim.x * RG;
      const int per = (E + gridDim.x - 1) / gridDim.x;
      const int e0 = blockIdx.x * per, e1 = min(E, e0 + per);
      const int grp = tid >> 4, sub = tid & 15;
      for (int base = e0; base < e1; base += CQ_THREADS / 16) {
        const int e = base + grp;
        double s = 0.0;
        if (e < e1) {
#pragma unroll 4
          for (unsigned q = sub; q < nrec; q += 16) s += __ldcg(a.part + (size_t)q * E + e);
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (e < e1 && sub == 0) a.fin[e] = s;
      }
    }
    if (!grid_sync_bounded(a.bar, a.err)) return;
#pragma unroll 4
    for (int e = tid; e < E; e += CQ_THREADS) A[e] = __ldcg(a.fin + e);
    __syncthreads();
    chol_upper_block(A, l, cq_shift(pass), cq_drop(pass), piv, dropped, blockIdx.x == 0 ? a.err : nullptr);
    cq_pack_r(A, dropped, l, l4, Rf, rinv);
    __syncthreads();
    for (int r = tid; r < R; r += CQ_THREADS) {
      float s[LMAX];
#pragma unroll
      for (int j = 0; j < LMAX; ++j) s[j] = j < l ? Yt[j * RP + r] : 0.f;
      cq_solve_row<LMAX>(s, Rf, rinv, l, l4);
#pragma unroll
      for (int j = 0; j < LMAX; ++j)
        if (j < l) Yt[j * RP + r] = s[j];
    }
    __syncthreads();
  }
  {
    float* Sg = a.S + r0 * l;
    for (int e = tid; e < R * l; e += CQ_THREADS) {
      const int r = e / l, c = e - r * l;
      Sg[e] = Yt[c * RP + r];
    }
  }
}

// ------------------------------------------------------ multi-kernel passes

__global__ void chol_factor_kernel(const double* G, int l, double shift, double drop_tol, float* Rf, float* rinv,
                                   unsigned* err) {
  extern __shared__ __align__(16) double Ash[];  // l x l
  __shared__ double piv[256];
  __shared__ int dropped[128];
  const int l4 = (l + 3) & ~3;
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int i = e / l, j = e - i * l;
    Ash[e] = 0.5 * (G[i * l + j] + G[j * l + i]);
  }
  __syncthreads();
  chol_upper_block(Ash, l, shift, drop_tol, piv, dropped, err);
  cq_pack_r(Ash, dropped, l, l4, Rf, rinv);
}

template <int LMAX>
__global__ void __launch_bounds__(128) trsm_rows_kernel(const float* __restrict__ Y, int64_t n, int l,
                                                        const float* __restrict__ Rf_g,
                                                        const float* __restrict__ rinv_g, float* Q) {
  extern __shared__ __align__(16) float csh[];
  const int l4 = (l + 3) & ~3;
  float* Rf = csh;
  float* rinv = csh + l * l4;
  for (int e = threadIdx.x; e < l * l4; e += blockDim.x) Rf[e] = Rf_g[e];
  for (int e = threadIdx.x; e < l4; e += blockDim.x) rinv[e] = rinv_g[e];
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  float s[LMAX];
#pragma unroll
  for (int j = 0; j < LMAX; ++j) s[j] = j < l ? Y[r * l + j] : 0.f;
  cq_solve_row<LMAX>(s, Rf, rinv, l, l4);
#pragma unroll
  for (int j = 0; j < LMAX; ++j)
    if (j < l) Q[r * l + j] = s[j];
}

size_t cholqr_part_doubles(int l) { return (size_t)num_sms() * cq_row_groups(l) * l * l; }

template <int LMAX>
static cudaError_t cholqr_run(float* S, float* T, int64_t n, int l, double* part, double* fin, double* G,
                              float* Rf, float* rinv, double* ws, unsigned* counter, unsigned* bar,
                              unsigned* err, bool allow_engine, cudaStream_t st) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  int grid = num_sms();
  if ((int64_t)grid > n) grid = (int)std::max<int64_t>(1, n);
  const int64_t rp = (((n + grid - 1) / grid) + 3) & ~3LL;
  if (allow_engine && rp <= (1 << 20) && cq_engine_smem(l, (int)rp) + 1024 <= (size_t)optin) {
    const size_t smem = cq_engine_smem(l, (int)rp);
    e = cudaFuncSetAttribute(cholqr_engine_kernel<LMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cholqr_engine_kernel<LMAX>, CQ_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm >= 1) {
      e = cudaMemsetAsync(bar, 0, 2 * GRID_GEN * sizeof(unsigned), st);
      if (e != cudaSuccess) return e;
      CqArgs a{S, n, l, (int)rp, part, fin, bar, err};
      void* params[] = {&a};
      e = cudaLaunchCooperativeKernel((const void*)cholqr_engine_kernel<LMAX>, dim3(grid), dim3(CQ_THREADS),
                                      params, smem, st);
      count_launches(1);
      return e;
    }
  }
  // separate kernels per pass; the result ends in S
  float* src = S;
  float* dst = T;
  const int l4 = (l + 3) & ~3;
  const size_t fsmem = (size_t)l * l * 8;
  e = cudaFuncSetAttribute(chol_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem);
  if (e != cudaSuccess) return e;
  const size_t tsmem = (size_t)(l * l4 + l4) * 4;
  e = cudaFuncSetAttribute(trsm_rows_kernel<LMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem);
  if (e != cudaSuccess) return e;
  for (int pass = 0; pass < 3; ++pass) {
    e = xcross(src, l, l, src, l, l, n, nullptr, nullptr, nullptr, nullptr, 0.0, G, nullptr, ws, counter, st);
    if (e != cudaSuccess) return e;
    chol_factor_kernel<<<1, 256, fsmem, st>>>(G, l, cq_shift(pass), cq_drop(pass), Rf, rinv, err);
    trsm_rows_kernel<LMAX><<<(unsigned)((n + 127) / 128), 128, tsmem, st>>>(src, n, l, Rf, rinv, dst);
    count_launches(2);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    std::swap(src, dst);
  }
  // three passes leave the result in T
  return cudaMemcpyAsync(S, src, (size_t)n * l * sizeof(float), cudaMemcpyDeviceToDevice, st);
}

cudaError_t cholqr3(float* S, float* T, int64_t n, int l, double* part, double* fin, double* G, float* Rf,
                    float* rinv, double* ws, unsigned* counter, unsigned* bar, unsigned* err, bool allow_engine,
                    cudaStream_t st) {
  if (n < 1 || l < 1 || l > 128) return cudaErrorInvalidValue;
  if (l <= 32)
    return cholqr_run<32>(S, T, n, l, part, fin, G, Rf, rinv, ws, counter, bar, err, allow_engine, st);
  if (l <= 64)
    return cholqr_run<64>(S, T, n, l, part, fin, G, Rf, rinv, ws, counter, bar, err, allow_engine, st);
  if (l <= 96)
    return cholqr_run<96>(S, T, n, l, part, fin, G, Rf, rinv, ws, counter, bar, err, allow_engine, st);
  return cholqr_run<128>(S, T, n, l, part, fin, G, Rf, rinv, ws, counter, bar, err, allow_engine, st);
}

}  // namespace symnmf
