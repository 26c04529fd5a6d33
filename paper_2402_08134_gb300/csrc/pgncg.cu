// Row kernels of PGNCG-SymNMF and LAI-PGNCG-SymNMF (section "Projected
// Gauss-Newton with Conjugate Gradients for SymNMF"; appendix Alg.
// LAI-PGNCG-SymNMF): an all-at-once update of H for ||X - H H^T||_F^2.
//
// Per iteration, with Y = X H (or U Lambda U^T H) and G = H^T H:
//   R = J^T r = 2 (H G - Y), P = R, Z = 0, e = ||R||^2
//   s_max times:  Yc = J^T J P = 2 (P G + H (P^T H))
//                 alpha = e / <P, Yc>,  Z += alpha P,  R -= alpha Yc
//                 e' = ||R||^2,  beta = e' / e,  P = R + beta P,  e = e'
//   H = max(H - Z, 0)
// (standard conjugate gradients on the Gauss-Newton normal equations; the
// printed loop never updates P).  CG stops early -- alpha = beta = 0 from then
// on -- once ||R|| <= 1e-6 ||R_0||, the FP32 rounding level, where the
// recurrence would only divide rounding noise.
//
// Rows are independent: one thread per row, G and P^T H (k x k, FP32) in
// shared memory.  The scalars (e, e_0, alpha, beta, the stop flag) stay on
// the device, each computed by the last block of the kernel that produces
// its sum (partials summed in a fixed order: deterministic); no host
// synchronisation inside an iteration.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace symnmf {

constexpr int GN_THREADS = 128;

__device__ __forceinline__ void gn_load_small(const float* A, int count, float* As) {
  for (int e = threadIdx.x; e < count; e += blockDim.x) As[e] = A[e];
  __syncthreads();
}

// Reduce this block's double partial into ws[blockIdx] and, in the last
// block, the total into *out (fixed order).  Returns true in the last block.
__device__ __forceinline__ bool gn_block_total(double v, double* ws, unsigned* counter, double* out, double* sh) {
  v = block_sum(v, sh);
  if (threadIdx.x == 0) ws[blockIdx.x] = v;
  if (last_block<1>(counter)) {
    reduce_partials(ws, 1, 1, gridDim.x, out, sh);
    __syncthreads();
    if (threadIdx.x == 0) *counter = 0;
    return true;
  }
  return false;
}

// R = 2 (H G - Y), P = R, Z = 0; cg[GN_E] = cg[GN_E0] = ||R||^2, stop flag cleared.
template <int KMAX>
__global__ void __launch_bounds__(GN_THREADS) gn_grad_kernel(const float* __restrict__ H, const float* __restrict__ Y,
                                                            const float* __restrict__ G, int64_t n, int k, float* R,
                                                            float* P, float* Z, double* ws, unsigned* counter,
                                                            double* cg) {
  extern __shared__ float gsm[];
  __shared__ double sh[32];
  gn_load_small(G, k * k, gsm);
  double e = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    float h[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) h[j] = j < k ? H[r * k + j] : 0.f;
    for (int c = 0; c < k; ++c) {
      float acc = -Y[r * k + c];
#pragma unroll
      for (int j = 0; j < KMAX; ++j)
        if (j < k) acc = fmaf(h[j], gsm[j * k + c], acc);
      const float v = 2.f * acc;
      R[r * k + c] = v;
      P[r * k + c] = v;
      Z[r * k + c] = 0.f;
      e += (double)v * (double)v;
    }
  }
  if (gn_block_total(e, ws, counter, cg + GN_E, sh) && threadIdx.x == 0) {
    cg[GN_E0] = cg[GN_E];
    cg[GN_STOP] = 0.0;
  }
}

// Yc = 2 (P G + H PtH); alpha = e / <P, Yc> (0 once CG has stopped).
template <int KMAX>
__global__ void __launch_bounds__(GN_THREADS) gn_hvp_kernel(const float* __restrict__ H, const float* __restrict__ P,
                                                           const float* __restrict__ G, const float* __restrict__ PtH,
                                                           int64_t n, int k, float* Yc, double* ws, unsigned* counter,
                                                           double* cg) {
  extern __shared__ float gsm[];
  __shared__ double sh[32];
  float* Gs = gsm;
  float* Ps = gsm + k * k;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    Gs[e] = G[e];
    Ps[e] = PtH[e];
  }
  __syncthreads();
  double pq = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    float p[KMAX], h[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
      p[j] = j < k ? P[r * k + j] : 0.f;
      h[j] = j < k ? H[r * k + j] : 0.f;
    }
    for (int c = 0; c < k; ++c) {
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < KMAX; ++j)
        if (j < k) acc = fmaf(p[j], Gs[j * k + c], fmaf(h[j], Ps[j * k + c], acc));
      const float v = 2.f * acc;
      Yc[r * k + c] = v;
      pq += (double)P[r * k + c] * (double)v;
    }
  }
  double tot = 0.0;
  if (gn_block_total(pq, ws, counter, &tot, sh) && threadIdx.x == 0) {
    const bool stop = cg[GN_STOP] != 0.0 || !(tot > 0.0);
    cg[GN_ALPHA] = stop ? 0.0 : cg[GN_E] / tot;
    if (stop) cg[GN_STOP] = 1.0;
  }
}

// Z += alpha P, R -= alpha Yc; e' = ||R||^2, beta = e' / e (0 once stopped), e = e'.
__global__ void __launch_bounds__(GN_THREADS) gn_update_kernel(const float* __restrict__ P,
                                                              const float* __restrict__ Yc, int64_t count, float* R,
                                                              float* Z, double* ws, unsigned* counter, double* cg) {
  __shared__ double sh[32];
  const float a = (float)cg[GN_ALPHA];
  double e = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
    Z[t] = fmaf(a, P[t], Z[t]);
    const float rv = fmaf(-a, Yc[t], R[t]);
    R[t] = rv;
    e += (double)rv * (double)rv;
  }
  double tot = 0.0;
  if (gn_block_total(e, ws, counter, &tot, sh) && threadIdx.x == 0) {
    const bool stop = cg[GN_STOP] != 0.0 || tot <= 1e-12 * cg[GN_E0] || !(cg[GN_E] > 0.0);
    cg[GN_BETA] = stop ? 0.0 : tot / cg[GN_E];
    cg[GN_E] = tot;
    if (stop) cg[GN_STOP] = 1.0;
  }
}

// P = R + beta P.
__global__ void gn_dir_kernel(const float* __restrict__ R, int64_t count, float* P, const double* cg) {
  const float b = (float)cg[GN_BETA];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    P[t] = fmaf(b, P[t], R[t]);
}

// H = max(H - Z, 0) (the projection of the Gauss-Newton step), W = H; a
// non-finite entry sets ERR_NAN.
__global__ void gn_project_kernel(const float* __restrict__ Z, int64_t count, float* H, float* W, unsigned* err) {
  bool bad = false;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x) {
    const float v = H[t] - Z[t];
    bad |= !isfinite(v);
    const float h = fmaxf(v, 0.f);
    H[t] = h;
    W[t] = h;
  }
  if (bad) set_error(err, ERR_NAN);
}

// ||X - H H^T||^2 = ||X||^2 - 2 tr(H^T X H) + sum_ij G_ij^2; tr from part[0]
// (sum H .* Y).  The value goes to out[*cnt] (if < cap) and *cnt advances.
__global__ void gn_objective_kernel(const double* normX2, const double* Gd, int k, const double* part, double* out,
                                    int* cnt, int cap) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) s += Gd[e] * Gd[e];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    const int i = *cnt;
    if (i < cap) out[i] = normX2[0] - 2.0 * part[0] + s;
    *cnt = i + 1;
  }
}

static int gn_grid(int64_t rows) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((rows + GN_THREADS - 1) / GN_THREADS, (int64_t)num_sms() * 4));
}

template <int KMAX>
static cudaError_t gn_grad_t(const float* H, const float* Y, const float* G, int64_t n, int k, float* R, float* P,
                             float* Z, double* ws, unsigned* counter, double* cg, cudaStream_t st) {
  gn_grad_kernel<KMAX><<<gn_grid(n), GN_THREADS, (size_t)k * k * 4, st>>>(H, Y, G, n, k, R, P, Z, ws, counter, cg);
  count_launches(1);
  return cudaGetLastError();
}

template <int KMAX>
static cudaError_t gn_hvp_t(const float* H, const float* P, const float* G, const float* PtH, int64_t n, int k,
                            float* Yc, double* ws, unsigned* counter, double* cg, cudaStream_t st) {
  gn_hvp_kernel<KMAX><<<gn_grid(n), GN_THREADS, (size_t)2 * k * k * 4, st>>>(H, P, G, PtH, n, k, Yc, ws, counter,
                                                                              cg);
  count_launches(1);
  return cudaGetLastError();
}

size_t gn_ws_doubles() { return (size_t)num_sms() * 4 + 8; }

cudaError_t gn_grad(const float* H, const float* Y, const float* G, int64_t n, int k, float* R, float* P, float* Z,
                    double* ws, unsigned* counter, double* cg, cudaStream_t st) {
  if (k <= 16) return gn_grad_t<16>(H, Y, G, n, k, R, P, Z, ws, counter, cg, st);
  if (k <= 32) return gn_grad_t<32>(H, Y, G, n, k, R, P, Z, ws, counter, cg, st);
  if (k <= 64) return gn_grad_t<64>(H, Y, G, n, k, R, P, Z, ws, counter, cg, st);
  return cudaErrorInvalidValue;
}

cudaError_t gn_hvp(const float* H, const float* P, const float* G, const float* PtH, int64_t n, int k, float* Yc,
                   double* ws, unsigned* counter, double* cg, cudaStream_t st) {
  if (k <= 16) return gn_hvp_t<16>(H, P, G, PtH, n, k, Yc, ws, counter, cg, st);
  if (k <= 32) return gn_hvp_t<32>(H, P, G, PtH, n, k, Yc, ws, counter, cg, st);
  if (k <= 64) return gn_hvp_t<64>(H, P, G, PtH, n, k, Yc, ws, counter, cg, st);
  return cudaErrorInvalidValue;
}

cudaError_t gn_update(const float* P, const float* Yc, int64_t count, float* R, float* Z, double* ws,
                      unsigned* counter, double* cg, cudaStream_t st) {
  gn_update_kernel<<<gn_grid(count), GN_THREADS, 0, st>>>(P, Yc, count, R, Z, ws, counter, cg);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t gn_dir(const float* R, int64_t count, float* P, const double* cg, cudaStream_t st) {
  gn_dir_kernel<<<gn_grid(count), GN_THREADS, 0, st>>>(R, count, P, cg);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t gn_project(const float* Z, int64_t count, float* H, float* W, unsigned* err, cudaStream_t st) {
  gn_project_kernel<<<gn_grid(count), GN_THREADS, 0, st>>>(Z, count, H, W, err);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t gn_objective(const double* normX2, const double* Gd, int k, const double* part, double* out, int* cnt,
                         int cap, cudaStream_t st) {
  gn_objective_kernel<<<1, 128, 0, st>>>(normX2, Gd, k, part, out, cnt, cap);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace symnmf
