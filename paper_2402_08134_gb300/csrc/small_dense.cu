// Single-CTA kernels on k x k / l x l matrices: FP64 Cholesky with explicit
// triangular inverse (the leverage scores' CholeskyQR of the LvS section) and
// cyclic Jacobi eigen-decomposition (Alg. Apx-EVD, T = Q_T Lambda Q_T^T).
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "chol.cuh"
#include "kernels.h"

namespace symnmf {

constexpr int CI_KMAX = 96;  // chol_inverse: 2 k^2 doubles of shared memory

// A = G + shift I = R^T R (R upper), then Rinv = R^{-1}, both in FP64.  The
// Cholesky is chol_upper_block (chol.cuh); the inverse goes row by row from
// the bottom,
//   Rinv[i][c] = -(sum_{i < j <= c} R[i][j] Rinv[j][c]) / R[i][i],
// each row's entries in parallel, TPC threads per entry (a shuffle tree).  A
// dropped pivot gives a zero row/column of Rinv; in strict mode
// (drop_tol <= 0) it also raises ERR_NOTSPD.
__global__ void chol_inverse_kernel(const double* G, int k, double shift, double drop_tol, double* Rinv,
                                    float* Rinv_f, unsigned* err, double* Rout) {
  extern __shared__ __align__(16) unsigned char ci_raw[];
  double* A = reinterpret_cast<double*>(ci_raw);  // k x k, becomes R
  double* X = A + k * k;                          // k x k, becomes R^{-1}
  ushort2* tri = reinterpret_cast<ushort2*>(X + k * k);
  __shared__ double piv[CI_KMAX], invd[CI_KMAX];
  __shared__ int dropped[CI_KMAX];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < k * k; e += nt) {
    const int i = e / k, j = e - i * k;
    A[e] = 0.5 * (G[i * k + j] + G[j * k + i]);
    X[e] = 0.0;
  }
  __syncthreads();
  chol_upper_block(A, k, shift, drop_tol, piv, invd, dropped, tri, err);
  const int tpc = k <= nt / 8 ? 8 : k <= nt / 4 ? 4 : k <= nt / 2 ? 2 : 1;  // threads per entry
  const int c = tid / tpc, part = tid - c * tpc;
  for (int i = k - 1; i >= 0; --i) {
    // 1 / R_ii = sqrt(1 / pivot) = piv[i] (0 for a dropped pivot)
    const double rinv = dropped[i] ? 0.0 : piv[i];
    double acc = 0.0;
    if (c < k && c > i)
      for (int j = i + 1 + part; j <= c; j += tpc) acc = fma(-A[i * k + j], X[j * k + c], acc);
    for (int o = 1; o < tpc; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (part == 0 && c < k && c >= i) X[i * k + c] = c == i ? rinv : acc * rinv;
    __syncthreads();
  }
  for (int e = tid; e < k * k; e += nt) {
    const int i = e / k, j = e - i * k;
    const double v = (j >= i) ? X[e] : 0.0;
    if (Rinv) Rinv[e] = v;
    if (Rinv_f) Rinv_f[e] = (float)v;
    if (Rout) Rout[e] = A[e];
  }
}

cudaError_t chol_inverse(const double* G, int k, double shift, double drop_tol, double* Rinv,
                         float* Rinv_f, unsigned* err, cudaStream_t st, double* R) {
  if (k < 1 || k > CI_KMAX) return cudaErrorInvalidValue;
  // two k x k FP64 matrices and the triangle's index table
  const size_t smem = (size_t)2 * k * k * sizeof(double) + (size_t)k * (k + 1) / 2 * sizeof(ushort2);
  cudaError_t e = cudaFuncSetAttribute(chol_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  chol_inverse_kernel<<<1, 256, smem, st>>>(G, k, shift, drop_tol, Rinv, Rinv_f, err, R);
  count_launches(1);
  return cudaGetLastError();
}

// Cyclic two-sided Jacobi with the round-robin (circle) ordering: each round
// rotates l/2 disjoint pairs at once (Golub & Van Loan, symmetric Schur 2x2),
// applying J^T A J block by block (2 x 2 blocks of two pairs) in one pass.
// Rotations run in FP32 (GB300's FP64 rate is ~1/64 of FP32 and T is only
// l x l); the convergence sums are FP64.  Sweeps stop once the off-diagonal
// mass is at the FP32 rounding level, off <= (8 l eps32)^2 ||T||_F^2: then
// ||T - V Lambda V^T||_F <= 8 l eps32 ||T||_F (about 2e-5 for l = 50), and the
// eigenvectors are orthonormal to ~1e-7, far below the precision of the
// products that formed T.
//
// One barrier per round: A is double-buffered (a round reads one buffer and
// writes the other), every thread forms the rotations of the pairs its blocks
// need from the round's input, and the pairs of every round are tabulated
// once at the start (they do not depend on A).

// The Schur rotation (c, s) of pair (p, q) of A (p = -1: the pair holds the
// dummy index, no rotation).
__device__ __forceinline__ void jac_rotation(const float* A, int l, int p, int q, float& c, float& sn) {
  c = 1.f;
  sn = 0.f;
  if (p < 0) return;
  const float apq = A[p * l + q];
  if (apq != 0.f) {
    const float tau = (A[q * l + q] - A[p * l + p]) / (2.f * apq);
    const float tt = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
    c = rsqrtf(1.f + tt * tt);
    sn = tt * c;
  }
}

__global__ void jacobi_kernel(const double* Ain, int l, double* Vout, double* lam) {
  extern __shared__ float smf[];
  const int L = (l + 1) & ~1;  // padded to even; index l is a dummy when l is odd
  const int m = L / 2;         // disjoint pairs per round
  // smf: two l*l buffers of A (a round's input and output), then V (l*l)
  float* V = smf + 2 * l * l;
  short2* pq = reinterpret_cast<short2*>(V + l * l);  // (L - 1) rounds x m pairs: (p, q), p = -1 for the dummy
  __shared__ double off, tot;
  __shared__ double shr[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < l * l; e += nt) {
    const int i = e / l, j = e - i * l;
    smf[e] = (float)(0.5 * (Ain[i * l + j] + Ain[j * l + i]));
    V[e] = (i == j) ? 1.f : 0.f;
  }
  // pairs of the circle method: slot 0 fixed, slots 1..L-1 rotate; a pair with
  // the dummy index keeps its real index q = l-1.. unrotated (p = -1)
  for (int e = tid; e < (L - 1) * m; e += nt) {
    const int round = e / m, i = e - round * m;
    const int a = (i == 0) ? 0 : ((i - 1 + round) % (L - 1)) + 1;
    const int bslot = L - 1 - i;
    const int b = ((bslot - 1 + round) % (L - 1)) + 1;
    int p = min(a, b), q = max(a, b);
    if (q >= l) {
      q = p;  // the only real index of the pair
      p = -1;
    }
    pq[e] = make_short2((short)p, (short)q);
  }
  __syncthreads();
  int cur = 0;
  const double lim = 8.0 * l * 5.9604644775390625e-8;  // 8 l 2^-24
  for (int sweep = 0; sweep < 30; ++sweep) {
    const float* A = smf + cur * l * l;
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
    if (off <= lim * lim * tot || off == 0.0) break;
    for (int round = 0; round < L - 1; ++round) {
      const float* Ai = smf + cur * l * l;
      float* Ao = smf + (cur ^ 1) * l * l;
      const short2* pr = pq + round * m;
      // Ao <- J^T Ai J on every 2x2 block (rows of pair u, columns of pair v)
      // at once, and V <- V J (rows i, columns of pair v)
      for (int e = tid; e < m * m + l * m; e += nt) {
        if (e < m * m) {
          const int u = e / m, v = e - u * m;
          const short2 su2 = pr[u], sv2 = pr[v];
          const int pu = su2.x, qu = su2.y, pv = sv2.x, qv = sv2.y;
          float cu, su, cv, sv;
          jac_rotation(Ai, l, pu, qu, cu, su);
          jac_rotation(Ai, l, pv, qv, cv, sv);
          // rows pu (may be -1), qu; columns pv (may be -1), qv
          const float x = (pu >= 0 && pv >= 0) ? Ai[pu * l + pv] : 0.f;
          const float y = (pu >= 0) ? Ai[pu * l + qv] : 0.f;
          const float z = (pv >= 0) ? Ai[qu * l + pv] : 0.f;
          const float w = Ai[qu * l + qv];
          const float x1 = cu * x - su * z, z1 = su * x + cu * z;
          const float y1 = cu * y - su * w, w1 = su * y + cu * w;
          if (pu >= 0 && pv >= 0) Ao[pu * l + pv] = cv * x1 - sv * y1;
          if (pu >= 0) Ao[pu * l + qv] = sv * x1 + cv * y1;
          if (pv >= 0) Ao[qu * l + pv] = cv * z1 - sv * w1;
          Ao[qu * l + qv] = sv * z1 + cv * w1;
        } else {
          const int f = e - m * m, row = f / m, v = f - row * m;
          const short2 sv2 = pr[v];
          const int pv = sv2.x, qv = sv2.y;
          if (pv >= 0) {
            float cv, sv;
            jac_rotation(Ai, l, pv, qv, cv, sv);
            const float a0 = V[row * l + pv], a1 = V[row * l + qv];
            V[row * l + pv] = cv * a0 - sv * a1;
            V[row * l + qv] = sv * a0 + cv * a1;
          }
        }
      }
      cur ^= 1;
      __syncthreads();
    }
  }
  const float* A = smf + cur * l * l;
  for (int e = tid; e < l * l; e += nt) Vout[e] = (double)V[e];
  for (int i = tid; i < l; i += nt) lam[i] = (double)A[i * l + i];
}

cudaError_t jacobi_evd(const double* A, int l, double* V, double* lam, cudaStream_t st) {
  if (l < 1 || l > 96) return cudaErrorInvalidValue;
  const int L = (l + 1) & ~1;
  // two buffers of A, V, and the (p, q) table of all L - 1 rounds
  const size_t smem = (size_t)3 * l * l * 4 + (size_t)(L - 1) * (L / 2) * sizeof(short2) + 16;
  cudaError_t e = cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  jacobi_kernel<<<1, 1024, smem, st>>>(A, l, V, lam);
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
