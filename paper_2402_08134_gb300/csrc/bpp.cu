// Row NLS update for the ANLS form of the surrogate (Eq. ANLS4symNMF; the
// per-row QPs of the Update() appendix):
//     x_r = argmin_{x >= 0} 1/2 x^T (G + alpha I) x - (y_r + alpha f_r)^T x
// solved by block principal pivoting (Kim & Park, SIAM J. Sci. Comput. 2011):
// full exchange of all infeasible variables while their count drops, three
// further full exchanges as backup, then Murty's single-variable rule, which
// terminates finitely.  One thread per row, FP64, k <= 16, warm-started from
// the support of the current row.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace symnmf {

constexpr int BPP_K = 16;

// Solve Gp[F,F] x_F = b_F by Cholesky on the passive set (bitmask).
__device__ static bool solve_passive(const double* Gp, int k, unsigned F, const double* b, double* x) {
  int id[BPP_K];
  int m = 0;
  for (int i = 0; i < k; ++i)
    if (F >> i & 1u) id[m++] = i;
  double L[BPP_K * BPP_K];
  double z[BPP_K];
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = Gp[id[i] * k + id[j]];
      for (int p = 0; p < j; ++p) s -= L[i * BPP_K + p] * L[j * BPP_K + p];
      if (i == j) {
        if (!(s > 0.0)) return false;
        L[i * BPP_K + i] = sqrt(s);
      } else {
        L[i * BPP_K + j] = s / L[j * BPP_K + j];
      }
    }
  }
  for (int i = 0; i < m; ++i) {
    double s = b[id[i]];
    for (int p = 0; p < i; ++p) s -= L[i * BPP_K + p] * z[p];
    z[i] = s / L[i * BPP_K + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = z[i];
    for (int p = i + 1; p < m; ++p) s -= L[p * BPP_K + i] * z[p];
    z[i] = s / L[i * BPP_K + i];
  }
  for (int i = 0; i < k; ++i) x[i] = 0.0;
  for (int i = 0; i < m; ++i) x[id[i]] = z[i];
  return true;
}

__global__ void __launch_bounds__(128) bpp_kernel(float* __restrict__ Fu, const float* __restrict__ Ff,
                                                  int64_t n, int k, const double* __restrict__ G,
                                                  double alpha, const float* __restrict__ Y, int ldy,
                                                  const float* __restrict__ U, int l,
                                                  const float* __restrict__ M, double* part,
                                                  double* ws, unsigned* counter, unsigned* err) {
  __shared__ double Gp[BPP_K * BPP_K];
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e / k, j = e - i * k;
    Gp[e] = G[e] + (i == j ? alpha : 0.0);
  }
  __syncthreads();
  double tr = 0.0, dd = 0.0;
  bool capped = false;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    double b[BPP_K], y[BPP_K], x[BPP_K];
    for (int i = 0; i < k; ++i) {
      double yi;
      if (U) {
        float s = 0.f;
        for (int p = 0; p < l; ++p) s = fmaf(U[r * l + p], M[p * k + i], s);
        yi = s;
      } else {
        yi = Y[r * ldy + i];
      }
      y[i] = yi;
      b[i] = yi + alpha * (double)Ff[r * k + i];
    }
    double bmax = 0.0;
    for (int i = 0; i < k; ++i) bmax = fmax(bmax, fabs(b[i]));
    const double eps = 1e-13 * (bmax + 1e-300);
    unsigned F = 0;
    for (int i = 0; i < k; ++i)
      if (Fu[r * k + i] > 0.f) F |= 1u << i;
    int ninf = k + 1, backup = 3;
    bool done = false;
    for (int it = 0; it < 8 * k + 20; ++it) {
      if (!solve_passive(Gp, k, F, b, x)) {
        F = 0;  // cannot happen for SPD Gp; restart from the empty set
        solve_passive(Gp, k, F, b, x);
      }
      unsigned V = 0;
      int cnt = 0, last = -1;
      for (int i = 0; i < k; ++i) {
        bool inf;
        if (F >> i & 1u) {
          inf = x[i] < -eps;
        } else {
          double g = -b[i];
          for (int j = 0; j < k; ++j) g += Gp[i * k + j] * x[j];
          inf = g < -eps;
        }
        if (inf) {
          V |= 1u << i;
          ++cnt;
          last = i;
        }
      }
      if (cnt == 0) {
        done = true;
        break;
      }
      if (cnt < ninf) {
        ninf = cnt;
        backup = 3;
        F ^= V;
      } else if (backup > 0) {
        --backup;
        F ^= V;
      } else {
        F ^= 1u << last;  // Murty's rule: the largest infeasible index
      }
    }
    if (!done) capped = true;
    for (int i = 0; i < k; ++i) {
      const double xi = x[i] > 0.0 ? x[i] : 0.0;
      const float xf = (float)xi;
      Fu[r * k + i] = xf;
      tr += (double)xf * y[i];
      const double d = (double)xf - (double)Ff[r * k + i];
      dd += d * d;
    }
  }
  if (capped) set_error(err, ERR_BPP_ITERS);
  __shared__ double sh[32];
  tr = block_sum(tr, sh);
  dd = block_sum(dd, sh);
  if (threadIdx.x == 0) {
    ws[2 * blockIdx.x] = tr;
    ws[2 * blockIdx.x + 1] = dd;
  }
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (am_last) {
    __threadfence();
    reduce_partials(ws, 2, 2, gridDim.x, part, sh);
    if (threadIdx.x == 0) *counter = 0;
  }
}

cudaError_t bpp_rows(float* F_upd, const float* F_fix, int64_t n, int k, const double* G, double alpha,
                     const float* Y, int ldy, const float* U, int l, const float* M, double* part,
                     double* ws, unsigned* counter, unsigned* err, cudaStream_t st) {
  if (k > BPP_K) return cudaErrorInvalidValue;
  int grid = (int)std::min<int64_t>((n + 127) / 128, (int64_t)num_sms() * 8);
  if (grid < 1) grid = 1;
  bpp_kernel<<<grid, 128, 0, st>>>(F_upd, F_fix, n, k, G, alpha, Y, ldy, U, l, M, part, ws, counter, err);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace symnmf
