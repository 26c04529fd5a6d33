// Rank-safe orthonormalisation of the range finder's blocks (Alg. RRF:
// Q = orth(Y) after every product with X): shifted CholeskyQR3 (Fukaya,
// Kannan, Nakatsukasa, Yamamoto, Yanagisawa, SIAM J. Sci. Comput. 2020).
// Pass 1 factors Y^T Y + 1e-6 max_i (Y^T Y)_ii I, which is positive definite
// whatever the rank of Y; passes 2 and 3 are plain CholeskyQR.  Each pass:
// G = Y^T Y (compensated FP32 partials summed in double-float, then taken to
// FP64), G + sI = R^T R in FP64 (chol.cuh), then every row y of Y becomes the
// solution x of x R = y (forward substitution in FP32).  Pivots below 1e-12 (pass 1) or 1e-10
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
#include "dfloat.cuh"
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
  for (int i = threadIdx.x; i < l4; i += blockDim.x)
    rinv[i] = (i < l && !dropped[i]) ? (float)(1.0 / A[i * l + i]) : 0.f;
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
  int pitch;       // column pitch of Y in shared memory (rp padded to 8, plus 32)
  dfl* part;       // [grid * RG][l * l] partial Grams
  dfl* fin;        // [l * l]
  unsigned* bar;   // barrier counter, zeroed
  unsigned* err;
  int npass;       // 3: shifted CholeskyQR3; 2: the shifted pass and one plain pass
};

constexpr int CQ_BATCH = 16;

__host__ __device__ inline size_t cq_engine_smem(int l, int rp) {
  const int l4 = (l + 3) & ~3;
  size_t b = (size_t)l * l * 8 + (size_t)2 * l * 8;  // A, piv, 1 / pivot (FP64)
  b = (b + 15) & ~(size_t)15;
  b += (size_t)CQ_THREADS * 8;                         // reduction partials (double-float)
  b += (size_t)l4 * (((rp + 7) & ~7) + 32) * 4;       // Yt (skewed columns)
  b += (size_t)l * l4 * 4 + (size_t)l4 * 4;            // Rf, rinv
  b += (size_t)l * 4 + (size_t)cq_tiles(l) * 4;        // dropped, tile table
  b += (size_t)l * (l + 1) / 2 * 4;                    // triangle entries of the Cholesky
  return b;
}

// Double-float sum of N values by a balanced tree (depth log2 N).
template <int N>
__device__ __forceinline__ dfl cq_tree_sum(dfl (&v)[N]) {
#pragma unroll
  for (int w = N / 2; w >= 1; w >>= 1)
#pragma unroll
    for (int u = 0; u < w; ++u) v[u] = df_add(v[u], v[u + w]);
  return v[0];
}

template <int LMAX>
__global__ void __launch_bounds__(CQ_THREADS, 1) cholqr_engine_kernel(CqArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int l = a.l, l4 = (l + 3) & ~3, RP = a.rp, P = a.pitch, E = l * l;
  // column c of Y starts at c P + 4 ((c / 4) mod 8): the 4-column blocks read
  // together by the Gram tiles fall in different bank groups
  auto col = [P](int c) { return c * P + ((c >> 2) & 7) * 4; };
  double* A = reinterpret_cast<double*>(smraw);  // l x l
  double* piv = A + l * l;                        // l
  double* invd = piv + l;                         // l
  dfl* red = reinterpret_cast<dfl*>(smraw + (((size_t)l * l * 8 + (size_t)2 * l * 8 + 15) & ~(size_t)15));
  float* Yt = reinterpret_cast<float*>(red + CQ_THREADS);
  float* Rf = Yt + l4 * P;                        // l x l4
  float* rinv = Rf + l * l4;                      // l4
  int* dropped = reinterpret_cast<int*>(rinv + l4);
  int* tiles = dropped + l;                       // (bi << 16) | bj, bi <= bj
  ushort2* tri = reinterpret_cast<ushort2*>(tiles + cq_tiles(l));

  const int tid = threadIdx.x;
  const int64_t r0 = (a.n * blockIdx.x) / gridDim.x;
  const int R = (int)((a.n * (blockIdx.x + 1)) / gridDim.x - r0);
  const int nb = l4 / 4, T = cq_tiles(l), RG = cq_row_groups(l);

  for (int e = tid; e < l4 * P; e += CQ_THREADS) Yt[e] = 0.f;
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
      Yt[col(c) + r] = Sg[e];
    }
  }
  __syncthreads();

  unsigned epoch = 0;
  for (int pass = 0; pass < a.npass; ++pass) {
    // partial Gram of this CTA's rows: 4x4 upper tiles, four rows per float4 step
    for (int w = tid; w < T * RG; w += CQ_THREADS) {
      const int tile = w % T, rg = w / T;
      const int bi = tiles[tile] >> 16, bj = tiles[tile] & 0xffff;
      const float4* Ap[4];
      const float4* Bp[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        Ap[p] = reinterpret_cast<const float4*>(Yt + col(4 * bi + p));
        Bp[p] = reinterpret_cast<const float4*>(Yt + col(4 * bj + p));
      }
      float acc[16], cmp[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) acc[e] = cmp[e] = 0.f;
#pragma unroll 1
      for (int c = rg; c < RP / 4; c += RG) {
        float4 av[4], bv[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          av[p] = Ap[p][c];
          bv[p] = Bp[p][c];
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
      dfl* rec = a.part + ((size_t)blockIdx.x * RG + rg) * E;
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int i = 4 * bi + (e >> 2), j = 4 * bj + (e & 3);
        if (i < l && j < l) {
          const dfl v{acc[e], -cmp[e]};  // Kahan pair: sum = acc - cmp
          rec[i * l + j] = v;
          rec[j * l + i] = v;
        }
      }
    }
    if (!grid_sync_bounded(a.bar, a.err, epoch)) return;
    // sliced fixed-order reduction of the grid * RG records into fin: CTA c
    // owns a contiguous run of entries, read coalesced (consecutive threads,
    // consecutive entries of one record); each thread sums every S-th record,
    // and the S partial sums of an entry are added in a fixed order
    {
      const unsigned nrec = gridDim.x * RG;
      const int per = (E + gridDim.x - 1) / gridDim.x;
      const int c0 = blockIdx.x * per, c1 = min(E, c0 + per);
      for (int i0 = c0; i0 < c1; i0 += CQ_THREADS) {
        const int np = min(CQ_THREADS, c1 - i0), S = CQ_THREADS / np;
        const int pos = tid % np, g = tid / np;
        if (g < S) {
          dfl acc{0.f, 0.f};
          for (unsigned q0 = g; q0 < nrec; q0 += (unsigned)S * CQ_BATCH) {
            dfl v[CQ_BATCH];
#pragma unroll
            for (int u = 0; u < CQ_BATCH; ++u) {
              const unsigned q = q0 + (unsigned)S * u;
              if (q < nrec) {
                const float2 f = __ldcg(reinterpret_cast<const float2*>(a.part + (size_t)q * E + i0 + pos));
                v[u] = dfl{f.x, f.y};
              } else {
                v[u] = dfl{0.f, 0.f};
              }
            }
            acc = df_add(acc, cq_tree_sum<CQ_BATCH>(v));
          }
          red[g * np + pos] = acc;
        }
        __syncthreads();
        if (tid < np) {
          dfl s{0.f, 0.f};
          for (int gg = 0; gg < S; ++gg) s = df_add(s, red[gg * np + tid]);
          a.fin[i0 + tid] = s;
        }
        __syncthreads();
      }
    }
    if (!grid_sync_bounded(a.bar, a.err, epoch)) return;
#pragma unroll 4
    for (int e = tid; e < E; e += CQ_THREADS) {
      const float2 f = __ldcg(reinterpret_cast<const float2*>(a.fin + e));
      A[e] = (double)f.x + (double)f.y;
    }
    __syncthreads();
    chol_upper_block(A, l, cq_shift(pass), cq_drop(pass), piv, invd, dropped, tri, nullptr);
    cq_pack_r(A, dropped, l, l4, Rf, rinv);
    __syncthreads();
    for (int r = tid; r < R; r += CQ_THREADS) {
      float s[LMAX];
#pragma unroll
      for (int j = 0; j < LMAX; ++j) s[j] = j < l ? Yt[col(j) + r] : 0.f;
      cq_solve_row<LMAX>(s, Rf, rinv, l, l4);
#pragma unroll
      for (int j = 0; j < LMAX; ++j)
        if (j < l) Yt[col(j) + r] = s[j];
    }
    __syncthreads();
  }
  {
    float* Sg = a.S + r0 * l;
    for (int e = tid; e < R * l; e += CQ_THREADS) {
      const int r = e / l, c = e - r * l;
      Sg[e] = Yt[col(c) + r];
    }
  }
}

// ------------------------------------------------------ multi-kernel passes

__global__ void chol_factor_kernel(const double* G, int l, double shift, double drop_tol, float* Rf, float* rinv) {
  extern __shared__ __align__(16) double Ash[];  // l x l, then the triangle entries
  __shared__ double piv[128], invd[128];
  __shared__ int dropped[128];
  const int l4 = (l + 3) & ~3;
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int i = e / l, j = e - i * l;
    Ash[e] = 0.5 * (G[i * l + j] + G[j * l + i]);
  }
  __syncthreads();
  chol_upper_block(Ash, l, shift, drop_tol, piv, invd, dropped, reinterpret_cast<ushort2*>(Ash + l * l), nullptr);
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
static cudaError_t cholqr_run(int npass, float* S, float* T, int64_t n, int l, double* part, double* fin, double* G,
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
      e = cudaMemsetAsync(bar, 0, sizeof(unsigned), st);
      if (e != cudaSuccess) return e;
      // the double-typed buffers hold double-float pairs (same size)
      CqArgs a{S, n, l, (int)rp, (int)(((rp + 7) & ~7LL) + 32), reinterpret_cast<dfl*>(part),
               reinterpret_cast<dfl*>(fin), bar, err, npass};
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
  const size_t fsmem = (size_t)l * l * 8 + (size_t)l * (l + 1) / 2 * 4;
  e = cudaFuncSetAttribute(chol_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem);
  if (e != cudaSuccess) return e;
  const size_t tsmem = (size_t)(l * l4 + l4) * 4;
  e = cudaFuncSetAttribute(trsm_rows_kernel<LMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem);
  if (e != cudaSuccess) return e;
  for (int pass = 0; pass < npass; ++pass) {
    e = xcross(src, l, l, src, l, l, n, nullptr, nullptr, nullptr, nullptr, 0.0, G, nullptr, ws, counter, st);
    if (e != cudaSuccess) return e;
    chol_factor_kernel<<<1, 256, fsmem, st>>>(G, l, cq_shift(pass), cq_drop(pass), Rf, rinv);
    trsm_rows_kernel<LMAX><<<(unsigned)((n + 127) / 128), 128, tsmem, st>>>(src, n, l, Rf, rinv, dst);
    count_launches(2);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    std::swap(src, dst);
  }
  // an odd pass count leaves the result in T
  if (src == S) return cudaSuccess;
  return cudaMemcpyAsync(S, src, (size_t)n * l * sizeof(float), cudaMemcpyDeviceToDevice, st);
}

cudaError_t cholqr3(float* S, float* T, int64_t n, int l, double* part, double* fin, double* G, float* Rf,
                    float* rinv, double* ws, unsigned* counter, unsigned* bar, unsigned* err, bool allow_engine,
                    cudaStream_t st, int npass) {
  if (n < 1 || l < 1 || l > 96 || npass < 2 || npass > 3) return cudaErrorInvalidValue;
  if (l <= 32)
    return cholqr_run<32>(npass, S, T, n, l, part, fin, G, Rf, rinv, ws, counter, bar, err, allow_engine, st);
  if (l <= 64)
    return cholqr_run<64>(npass, S, T, n, l, part, fin, G, Rf, rinv, ws, counter, bar, err, allow_engine, st);
  if (l <= 80)
    return cholqr_run<80>(npass, S, T, n, l, part, fin, G, Rf, rinv, ws, counter, bar, err, allow_engine, st);
  return cholqr_run<96>(npass, S, T, n, l, part, fin, G, Rf, rinv, ws, counter, bar, err, allow_engine, st);
}

}  // namespace symnmf
