// Block-wide FP64 Cholesky of a small symmetric matrix in shared memory.
#pragma once

#include "common.cuh"

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

}  // namespace symnmf
