// Single-CTA FP64 kernels on k x k / l x l matrices: Cholesky with explicit
// triangular inverse (CholeskyQR of the LvS section, second CholeskyQR2 pass
// of the range finder) and cyclic Jacobi eigen-decomposition (Alg. Apx-EVD,
// T = Q_T Lambda Q_T^T, and the rank-safe first orthonormalisation pass).
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "chol.cuh"
#include "kernels.h"

namespace symnmf {

// A = G + shift I = R^T R (R upper, chol.cuh), then Rinv = R^{-1}.  A
// dropped pivot gives a zero row/column of Rinv; in strict mode
// (drop_tol <= 0) a pivot <= 0 also raises ERR_NOTSPD.
__global__ void chol_inverse_kernel(const double* G, int k, double shift, double drop_tol,
                                    double* Rinv, float* Rinv_f, unsigned* err) {
  extern __shared__ double A[];  // k*k (becomes R), then X = R^{-1} k*k
  double* X = A + k * k;
  __shared__ int dropped[128];
  __shared__ double piv[256];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < k * k; e += nt) {
    const int i = e / k, j = e - i * k;
    A[e] = 0.5 * (G[i * k + j] + G[j * k + i]);
    X[e] = 0.0;
  }
  __syncthreads();
  chol_upper_block(A, k, shift, drop_tol, piv, dropped, err);
  // R^{-1} column by column (back substitution), one column per thread
  for (int c = tid; c < k; c += nt) {
    for (int i = c; i >= 0; --i) {
      if (dropped[i]) {
        X[i * k + c] = 0.0;
        continue;
      }
      double s = (i == c) ? 1.0 : 0.0;
      for (int j = i + 1; j <= c; ++j) s -= A[i * k + j] * X[j * k + c];
      X[i * k + c] = s / A[i * k + i];
    }
  }
  __syncthreads();
  for (int e = tid; e < k * k; e += nt) {
    const int i = e / k, j = e - i * k;
    const double v = (j >= i) ? X[e] : 0.0;
    if (Rinv) Rinv[e] = v;
    if (Rinv_f) Rinv_f[e] = (float)v;
  }
}

cudaError_t chol_inverse(const double* G, int k, double shift, double drop_tol, double* Rinv,
                         float* Rinv_f, unsigned* err, cudaStream_t st) {
  if (k < 1 || k > 112) return cudaErrorInvalidValue;  // 2 k^2 doubles of shared memory
  const size_t smem = (size_t)2 * k * k * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(chol_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  chol_inverse_kernel<<<1, 256, smem, st>>>(G, k, shift, drop_tol, Rinv, Rinv_f, err);
  count_launches(1);
  return cudaGetLastError();
}

// Cyclic two-sided Jacobi with the round-robin (circle) ordering: each round
// rotates l/2 disjoint pairs at once (Golub & Van Loan, symmetric Schur 2x2).
// Rotations run in FP32 (GB300's FP64 rate is ~1/64 of FP32 and T is only
// l x l); the convergence sums are FP64.  Eigenvectors come out orthonormal
// to ~1e-7, far below the precision of the products that formed T.
__global__ void jacobi_kernel(const double* Ain, int l, double* Vout, double* lam) {
  extern __shared__ float smf[];
  const int L = (l + 1) & ~1;  // padded to even; index l is a dummy when l is odd
  float* A = smf;              // l*l
  float* V = A + l * l;        // l*l
  float* cs = V + l * l;       // 2 * (L/2)
  int* pp = (int*)(cs + L);    // L/2
  int* qq = pp + L / 2;
  __shared__ double off, tot;
  __shared__ double shr[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < l * l; e += nt) {
    const int i = e / l, j = e - i * l;
    A[e] = (float)(0.5 * (Ain[i * l + j] + Ain[j * l + i]));
    V[e] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  const int m = L / 2;
  for (int sweep = 0; sweep < 30; ++sweep) {
    double o = 0.0, t = 0.0;
    for (int e = tid; e < l * l; e += nt) {
      const double v = (double)A[e] * (double)A[e];
      t += v;
      if (e / l != e % l) o += v;
    }
    o = block_sum(o, shr);
    t = block_sum(t, shr);
    if (tid == 0) {
      off = o;
      tot = t;
    }
    __syncthreads();
    if (off <= 1e-13 * tot || off == 0.0) break;
    for (int round = 0; round < L - 1; ++round) {
      // pairs of the circle method: slot 0 fixed, slots 1..L-1 rotate
      for (int i = tid; i < m; i += nt) {
        const int a = (i == 0) ? 0 : ((i - 1 + round) % (L - 1)) + 1;
        const int bslot = L - 1 - i;
        const int b = ((bslot - 1 + round) % (L - 1)) + 1;
        int p = min(a, b), q = max(a, b);
        float c = 1.f, s = 0.f;
        if (q < l) {
          const float apq = A[p * l + q];
          if (apq != 0.f) {
            const float tau = (A[q * l + q] - A[p * l + p]) / (2.f * apq);
            const float tt = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            c = 1.f / sqrtf(1.f + tt * tt);
            s = tt * c;
          }
        } else {
          p = -1;
        }
        pp[i] = p;
        qq[i] = q;
        cs[2 * i] = c;
        cs[2 * i + 1] = s;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int e = tid; e < m * l; e += nt) {
        const int i = e / l, col = e - i * l;
        const int p = pp[i], q = qq[i];
        if (p < 0) continue;
        const float c = cs[2 * i], s = cs[2 * i + 1];
        const float ap = A[p * l + col], aq = A[q * l + col];
        A[p * l + col] = c * ap - s * aq;
        A[q * l + col] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J and V <- V J
      for (int e = tid; e < m * l; e += nt) {
        const int i = e / l, row = e - i * l;
        const int p = pp[i], q = qq[i];
        if (p < 0) continue;
        const float c = cs[2 * i], s = cs[2 * i + 1];
        const float ap = A[row * l + p], aq = A[row * l + q];
        A[row * l + p] = c * ap - s * aq;
        A[row * l + q] = s * ap + c * aq;
        const float vp = V[row * l + p], vq = V[row * l + q];
        V[row * l + p] = c * vp - s * vq;
        V[row * l + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  for (int e = tid; e < l * l; e += nt) Vout[e] = (double)V[e];
  for (int i = tid; i < l; i += nt) lam[i] = (double)A[i * l + i];
}

cudaError_t jacobi_evd(const double* A, int l, double* V, double* lam, cudaStream_t st) {
  if (l < 1 || l > 96) return cudaErrorInvalidValue;
  const int L = (l + 1) & ~1;
  const size_t smem = (size_t)2 * l * l * 4 + (size_t)L * 4 + (size_t)L * 4 + 16;
  cudaError_t e = cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  jacobi_kernel<<<1, 512, smem, st>>>(A, l, V, lam);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void svqb_kernel(const double* V, const double* lam, int l, double tol, float* B) {
  __shared__ double mx;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < l; ++i) m = fmax(m, lam[i]);
    mx = m;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int j = e % l;
    const double s = lam[j];
    B[e] = (s > tol * mx && s > 0.0) ? (float)(V[e] / sqrt(s)) : 0.f;
  }
}

cudaError_t svqb_matrix(const double* V, const double* lam, int l, double tol, float* B,
                        cudaStream_t st) {
  svqb_kernel<<<1, 256, 0, st>>>(V, lam, l, tol, B);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void to_float_scaled_kernel(const double* C, int la, int lb, const double* lam, float* out) {
  for (int e = threadIdx.x + blockIdx.x * blockDim.x; e < la * lb; e += blockDim.x * gridDim.x) {
    const int i = e / lb;
    out[e] = (float)(lam ? lam[i] * C[e] : C[e]);
  }
}

cudaError_t to_float_scaled(const double* C, int la, int lb, const double* lam, float* out,
                            cudaStream_t st) {
  to_float_scaled_kernel<<<(la * lb + 255) / 256, 256, 0, st>>>(C, la, lb, lam, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace symnmf
