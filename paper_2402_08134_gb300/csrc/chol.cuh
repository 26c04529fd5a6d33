// Block-wide FP64 Cholesky of a small symmetric matrix in shared memory.
#pragma once

#include "common.cuh"
#include "dfloat.cuh"

namespace symnmf {

// A + s I = R^T R with R upper triangular, computed in place by all threads
// of the block (right-looking, one __syncthreads per column).  A (m x m,
// row-major, shared memory) holds the symmetric input (upper triangle read)
// and receives R, zero below the diagonal.  piv holds 2 m doubles, dropped m
// ints (shared memory).  s = shift when shift >= 0, else -shift times the
// largest diagonal entry of A.  A pivot d <= drop_tol * (largest diagonal of
// A) or not > 0 is dropped: row j of R is zero and column j takes no part in
// the trailing update.  With drop_tol <= 0 (strict mode) a dropped pivot
// also raises ERR_NOTSPD.
//
// Step j subtracts row j's outer product from the trailing rows and scales
// row j - 1 (no longer read) into R.  The pivot of column j + 1 is formed by
// the thread that applies the last update to A[j+1][j+1], right after that
// update, so pivot j is visible to every thread after the barrier that closes
// step j - 1.
__device__ __forceinline__ void chol_pivot(double* A, int m, int j, double tol, bool strict, double* piv,
                                           int* dropped, unsigned* err) {
  const double d = A[j * m + j];
  if (d <= tol || !(d > 0.0)) {
    dropped[j] = 1;
    piv[2 * j] = 0.0;
    piv[2 * j + 1] = 0.0;
    if (strict) set_error(err, ERR_NOTSPD);
  } else {
    dropped[j] = 0;
    piv[2 * j] = 1.0 / sqrt(d);  // scale of row j of R
    piv[2 * j + 1] = 1.0 / d;    // factor of the trailing update
  }
}

__device__ inline void chol_upper_block(double* A, int m, double shift, double drop_tol, double* piv, int* dropped,
                                 unsigned* err) {
  __shared__ double s_maxdiag;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  if (tid == 0) {
    double mx = 0.0;
    for (int i = 0; i < m; ++i) mx = fmax(mx, A[i * m + i]);
    s_maxdiag = mx;
  }
  __syncthreads();
  const double maxdiag = s_maxdiag;
  const double s = shift >= 0.0 ? shift : -shift * maxdiag;
  const double tol = drop_tol > 0.0 ? drop_tol * maxdiag : 0.0;
  const bool strict = drop_tol <= 0.0;
  if (s != 0.0)
    for (int i = tid; i < m; i += nt) A[i * m + i] += s;
  __syncthreads();
  if (tid == 0) chol_pivot(A, m, 0, tol, strict, piv, dropped, err);
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    if (j > 0) {
      const double rs = piv[2 * (j - 1)];
      for (int c = j - 1 + tid; c < m; c += nt) A[(j - 1) * m + c] *= rs;
    }
    const double inv_d = piv[2 * j + 1];
    const double* aj = A + j * m;
    // trailing update of the upper triangle: rows r > j by warps, columns c >= r by lanes
    for (int r = j + 1 + wid; r < m; r += nw) {
      const double t = aj[r] * inv_d;
      double* ar = A + r * m;
      for (int c = r + lane; c < m; c += 32) {
        ar[c] = fma(-t, aj[c], ar[c]);
        if (c == j + 1) chol_pivot(A, m, j + 1, tol, strict, piv, dropped, err);  // r == c == j + 1
      }
    }
    __syncthreads();
  }
  if (tid == 0) A[(m - 1) * m + (m - 1)] *= piv[2 * (m - 1)];
  for (int e = tid; e < m * m; e += nt)
    if (e % m < e / m) A[e] = 0.0;
  __syncthreads();
}

// The same factorisation in double-float (dfloat.cuh), for the CholeskyQR
// passes of the range finder: A (m x m, row-major, shared memory) as hi/lo
// pairs receives R; piv and invd hold m pairs (1 / sqrt of each pivot and
// 1 / pivot), dropped m ints, tri the m (m + 1) / 2 entries (r, c), c >= r,
// of the upper triangle in row-major order (built here).  The input is scaled
// by a power of two so that its largest diagonal entry is near 1 (the
// double-float range is FP32's), and R is scaled back exactly.  Pivots are
// dropped as in chol_upper_block (never strict).
//
// Step j updates the trailing triangle (rows > j), which is the suffix of tri
// starting at row j + 1 with (j + 1, j + 1) first.  Warp 0 is the pivot warp:
// its lane 0 updates (j + 1, j + 1) and forms the next pivot, with no other
// work to wait for; the other warps walk the rest of the suffix with a common
// stride, so their work is balanced.
__device__ __forceinline__ void chol_pivot_df(dfl* A, int m, int j, float tol, dfl* piv, dfl* invd, int* dropped) {
  const dfl d = A[j * m + j];
  if (!(d.hi + d.lo > tol)) {
    dropped[j] = 1;
    piv[j] = dfl{0.f, 0.f};
    invd[j] = dfl{0.f, 0.f};
  } else {
    dropped[j] = 0;
    const dfl r = df_rsqrt(d);
    piv[j] = r;
    invd[j] = df_mul(r, r);
  }
}

__device__ __forceinline__ int chol_tri_offset(int r, int m) { return r * m - r * (r - 1) / 2; }

__device__ inline void chol_upper_block_df(dfl* A, int m, double shift, double drop_tol, dfl* piv, dfl* invd,
                                           int* dropped, ushort2* tri) {
  // needs blockDim.x > 32 (a pivot warp and at least one other)
  __shared__ double s_maxdiag;
  __shared__ float s_scale, s_unscale;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int total = m * (m + 1) / 2;
  if (tid == 0) {
    double mx = 0.0;
    for (int i = 0; i < m; ++i) mx = fmax(mx, df_to_double(A[i * m + i]));
    s_maxdiag = mx;
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);
    e = max(-120, min(120, e)) & ~1;  // even: the factor's scale is then an exact power of two as well
    s_scale = ldexpf(1.f, -e);
    s_unscale = ldexpf(1.f, e / 2);
  }
  for (int r = tid; r < m; r += nt) {
    const int o = chol_tri_offset(r, m);
    for (int c = r; c < m; ++c) tri[o + c - r] = make_ushort2((unsigned short)r, (unsigned short)c);
  }
  __syncthreads();
  const float sc = s_scale;
  const double maxdiag = s_maxdiag * (double)sc;
  const double s = shift >= 0.0 ? shift * (double)sc : -shift * maxdiag;
  const float tol = drop_tol > 0.0 ? (float)(drop_tol * maxdiag) : 0.f;
  const dfl sd = df_from_double(s);
  for (int e = tid; e < m * m; e += nt) {
    dfl v = A[e];
    v.hi *= sc;
    v.lo *= sc;
    if (s != 0.0 && e % (m + 1) == 0) v = df_add(v, sd);
    A[e] = v;
  }
  __syncthreads();
  if (tid == 0) chol_pivot_df(A, m, 0, tol, piv, invd, dropped);
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    if (j > 0) {  // row j - 1 is final: scale it into R
      const dfl rs = piv[j - 1];
      for (int c = j - 1 + tid; c < m; c += nt) A[(j - 1) * m + c] = df_mul(A[(j - 1) * m + c], rs);
    }
    const dfl id = invd[j];
    const dfl* aj = A + j * m;
    const int e0 = chol_tri_offset(j + 1, m);
    if (tid < 32) {
      if (tid == 0 && e0 < total) {  // (j + 1, j + 1), then the next pivot
        const int r = j + 1;
        A[r * m + r] = df_fms(A[r * m + r], df_mul(aj[r], id), aj[r]);
        chol_pivot_df(A, m, r, tol, piv, invd, dropped);
      }
    } else {
      for (int e = e0 + 1 + (tid - 32); e < total; e += nt - 32) {
        const ushort2 rc = tri[e];
        const int r = rc.x, c = rc.y;
        A[r * m + c] = df_fms(A[r * m + c], df_mul(aj[r], id), aj[c]);
      }
    }
    __syncthreads();
  }
  if (tid == 0) A[(m - 1) * m + (m - 1)] = df_mul(A[(m - 1) * m + (m - 1)], piv[m - 1]);
  __syncthreads();
  const float us = s_unscale;
  for (int e = tid; e < m * m; e += nt) {
    if (e % m < e / m) {
      A[e] = dfl{0.f, 0.f};
    } else {
      A[e].hi *= us;
      A[e].lo *= us;
    }
  }
  __syncthreads();
}

}  // namespace symnmf
