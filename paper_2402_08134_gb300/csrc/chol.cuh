// Block-wide FP64 Cholesky of a small symmetric matrix in shared memory.
#pragma once

#include "common.cuh"

namespace symnmf {

// A + s I = R^T R with R upper triangular, in FP64, computed in place by all
// threads of the block (right-looking, one __syncthreads per column).  A
// (m x m, row-major, shared memory) holds the symmetric input (upper triangle
// read) and receives R, zero below the diagonal.  piv and invd hold m doubles
// (1 / sqrt of each pivot and 1 / pivot), dropped m ints, tri the
// m (m + 1) / 2 entries (r, c), c >= r, of the upper triangle in row-major
// order (built here); all in shared memory.  s = shift when shift >= 0, else
// -shift times the largest diagonal entry of A.  A pivot d <= drop_tol *
// (largest diagonal of A) or not > 0 is dropped: row j of R is zero and
// column j takes no part in the trailing update.  With drop_tol <= 0 (strict
// mode) a dropped pivot also raises ERR_NOTSPD.
//
// Step j updates the trailing triangle (rows > j), which is the suffix of tri
// starting at row j + 1 with (j + 1, j + 1) first, and scales row j - 1 (no
// longer read) into R.  Warp 0 is the pivot warp: its lane 0 updates
// (j + 1, j + 1) and forms the next pivot right away, so pivot j + 1 is
// visible to every thread after the barrier that closes step j; the other
// warps walk the rest of the suffix with a common stride, so their work is
// balanced.  1 / sqrt(d) is the FP64 reciprocal square root; 1 / d is its
// square.  Needs blockDim.x > 32.
__device__ __forceinline__ void chol_pivot_f64(const double* A, int m, int j, double tol, bool strict, double* piv,
                                               double* invd, int* dropped, unsigned* err) {
  const double d = A[j * m + j];
  if (!(d > tol)) {
    dropped[j] = 1;
    piv[j] = 0.0;
    invd[j] = 0.0;
    if (strict && err) set_error(err, ERR_NOTSPD);
  } else {
    dropped[j] = 0;
    const double r = rsqrt(d);
    piv[j] = r;
    invd[j] = r * r;
  }
}

__device__ __forceinline__ int chol_tri_offset(int r, int m) { return r * m - r * (r - 1) / 2; }

__device__ inline void chol_upper_block(double* A, int m, double shift, double drop_tol, double* piv, double* invd,
                                        int* dropped, ushort2* tri, unsigned* err) {
  __shared__ double s_maxdiag;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int total = m * (m + 1) / 2;
  if (tid == 0) {
    double mx = 0.0;
    for (int i = 0; i < m; ++i) mx = fmax(mx, A[i * m + i]);
    s_maxdiag = mx;
  }
  for (int r = tid; r < m; r += nt) {
    const int o = chol_tri_offset(r, m);
    for (int c = r; c < m; ++c) tri[o + c - r] = make_ushort2((unsigned short)r, (unsigned short)c);
  }
  __syncthreads();
  const double maxdiag = s_maxdiag;
  const double s = shift >= 0.0 ? shift : -shift * maxdiag;
  const double tol = drop_tol > 0.0 ? drop_tol * maxdiag : 0.0;
  const bool strict = drop_tol <= 0.0;
  if (s != 0.0)
    for (int i = tid; i < m; i += nt) A[i * m + i] += s;
  __syncthreads();
  if (tid == 0) chol_pivot_f64(A, m, 0, tol, strict, piv, invd, dropped, err);
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    if (j > 0) {  // row j - 1 is final: scale it into R
      const double rs = piv[j - 1];
      for (int c = j - 1 + tid; c < m; c += nt) A[(j - 1) * m + c] *= rs;
    }
    const double id = invd[j];
    const double* aj = A + j * m;
    const int e0 = chol_tri_offset(j + 1, m);
    if (tid < 32) {
      if (tid == 0 && e0 < total) {  // (j + 1, j + 1), then the next pivot
        const int r = j + 1;
        A[r * m + r] = fma(-(aj[r] * id), aj[r], A[r * m + r]);
        chol_pivot_f64(A, m, r, tol, strict, piv, invd, dropped, err);
      }
    } else {
      for (int e = e0 + 1 + (tid - 32); e < total; e += nt - 32) {
        const ushort2 rc = tri[e];
        const int r = rc.x, c = rc.y;
        A[r * m + c] = fma(-(aj[r] * id), aj[c], A[r * m + c]);
      }
    }
    __syncthreads();
  }
  if (tid == 0) A[(m - 1) * m + (m - 1)] *= piv[m - 1];
  __syncthreads();
  for (int e = tid; e < m * m; e += nt)
    if (e % m < e / m) A[e] = 0.0;
  __syncthreads();
}

}  // namespace symnmf
