// Learned warm start: a 3-layer network maps a node's normalised sketch row
// x_i = (X Omega)_i / ||(X Omega)_i|| (Omega of Alg. RRF) to a nonnegative
// starting row of H:  a1 = relu(x W1 + b1), a2 = relu(a1 W2 + b2),
// H0 = softplus(a2 W3 + b3).  It is trained on converged factors H* that the
// solver itself produces, with the column-permutation-invariant loss
//   L = ||H^ H^^T - H* H*^T||_F^2 / ||H* H*^T||_F^2
// evaluated through k x k Grams.  The paper starts from a scaled uniform
// random H (experiments section); this network is an addition, with that
// random start as the fallback.
//
// Kernels: a tiled FP32 CUDA-core GEMM with optional transposes, fused
// bias + activation epilogue and split-K (weight gradients reduce over all
// rows); column sums for bias gradients; activation derivatives; the Gram
// loss and its gradient; Adam.  At the sizes of the warm-start workload
// (50000 x 74 -> 256 -> 256 -> 32, 9.3 GFLOP per forward pass) these run in
// well under a millisecond per instance.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/symnmf.h"
#include "common.cuh"
#include "handle.h"
#include "kernels.h"

namespace symnmf {

constexpr int MG_TM = 64, MG_TN = 64, MG_TK = 16;

enum { ACT_NONE = 0, ACT_RELU = 1, ACT_SOFTPLUS = 2 };

// C[m, n] (+)= sum_k A(m, k) B(k, n) over k in this block's K range.
// A(m, k) = TA ? A[k * lda + m] : A[m * lda + k]; B(k, n) = TB ? B[n * ldb + k] : B[k * ldb + n].
// Epilogue (single K split only): + bias[n], activation; with split-K the
// partial sums are added atomically into C (which must be zeroed).
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) mlp_gemm_kernel(const float* __restrict__ A, int lda,
                                                       const float* __restrict__ B, int ldb, float* C,
                                                       int ldc, int M, int N, int64_t K, int64_t kchunk,
                                                       const float* __restrict__ bias, int act, float* Zout) {
  __shared__ float As[MG_TK][MG_TM + 4];
  __shared__ float Bs[MG_TK][MG_TN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * MG_TM, n0 = blockIdx.x * MG_TN;
  const int64_t kb = (int64_t)blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  float acc[4][4] = {};
  for (int64_t k0 = kb; k0 < ke; k0 += MG_TK) {
    for (int e = tid; e < MG_TK * MG_TM; e += 256) {
      int kk, mm;
      if (TA) {  // contiguous in m
        kk = e / MG_TM;
        mm = e % MG_TM;
      } else {  // contiguous in k
        mm = e / MG_TK;
        kk = e % MG_TK;
      }
      const int64_t gk = k0 + kk;
      const int gm = m0 + mm;
      float v = 0.f;
      if (gk < ke && gm < M) v = TA ? A[gk * lda + gm] : A[(int64_t)gm * lda + gk];
      As[kk][mm] = v;
    }
    for (int e = tid; e < MG_TK * MG_TN; e += 256) {
      int kk, nn;
      if (TB) {
        nn = e / MG_TK;
        kk = e % MG_TK;
      } else {
        kk = e / MG_TN;
        nn = e % MG_TN;
      }
      const int64_t gk = k0 + kk;
      const int gn = n0 + nn;
      float v = 0.f;
      if (gk < ke && gn < N) v = TB ? B[(int64_t)gn * ldb + gk] : B[gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < MG_TK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  const bool split = gridDim.z > 1;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      float v = acc[i][j];
      if (split) {
        atomicAdd(C + (int64_t)gm * ldc + gn, v);
        continue;
      }
      if (bias) v += bias[gn];
      if (Zout) Zout[(int64_t)gm * ldc + gn] = v;
      if (act == ACT_RELU) v = fmaxf(v, 0.f);
      else if (act == ACT_SOFTPLUS) v = v > 20.f ? v : log1pf(expf(v));
      C[(int64_t)gm * ldc + gn] = v;
    }
  }
}

template <bool TA, bool TB>
static cudaError_t mlp_gemm(const float* A, int lda, const float* B, int ldb, float* C, int ldc, int M, int N,
                            int64_t K, const float* bias, int act, float* Zout, int splits, cudaStream_t st) {
  int64_t kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + MG_TK - 1) / MG_TK * MG_TK;
  dim3 grid((N + MG_TN - 1) / MG_TN, (M + MG_TM - 1) / MG_TM, (unsigned)splits);
  mlp_gemm_kernel<TA, TB><<<grid, 256, 0, st>>>(A, lda, B, ldb, C, ldc, M, N, K, kchunk, bias, act, Zout);
  count_launches(1);
  return cudaGetLastError();
}

// out[j] = sum_i X[i, j] (bias gradients), atomically over row blocks.
__global__ void colsum_kernel(const float* X, int64_t rows, int cols, float* out) {
  const int j = blockIdx.x * 32 + (threadIdx.x & 31);
  const int64_t r0 = (int64_t)blockIdx.y * 1024;
  float s = 0.f;
  if (j < cols)
    for (int64_t r = r0 + (threadIdx.x >> 5); r < min(rows, r0 + 1024); r += blockDim.x >> 5) s += X[r * cols + j];
  __shared__ float sh[8][33];
  sh[threadIdx.x >> 5][threadIdx.x & 31] = s;
  __syncthreads();
  if (threadIdx.x < 32 && j < cols) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w][threadIdx.x];
    atomicAdd(out + j, t);
  }
}

// d <- d * f'(z): relu' = (z > 0), softplus' = sigmoid(z)
__global__ void act_grad_kernel(float* d, const float* z, int64_t count, int act) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float zz = z[t];
    if (act == ACT_RELU) d[t] = zz > 0.f ? d[t] : 0.f;
    else d[t] = d[t] / (1.0f + expf(-zz));
  }
}

// loss = (||A||^2 - 2 ||B||^2 + ||C||^2) / ||C||^2, A = H^T H^, B = H^^T H*, C = H*^T H*.
__global__ void gram_loss_kernel(const double* A, const double* B, const double* Cm, int k, double* loss,
                                 float* coef) {
  __shared__ double sh[32];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    a += A[e] * A[e];
    b += B[e] * B[e];
    c += Cm[e] * Cm[e];
  }
  a = block_sum(a, sh);
  b = block_sum(b, sh);
  c = block_sum(c, sh);
  if (threadIdx.x == 0) {
    loss[0] = (a - 2.0 * b + c) / c;
    coef[0] = (float)(4.0 / c);
  }
}

// dH^ = coef * (H^ A - H* B^T), A = H^^T H^, B = H^^T H*  (k x k FP32 copies)
__global__ void gram_loss_grad_kernel(const float* Hh, const float* Hs, const float* Af, const float* Bf,
                                      const float* coef, int64_t rows, int k, float* dH) {
  __shared__ float As[64 * 64], Bs[64 * 64];
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    As[e] = Af[e];
    Bs[e] = Bf[e];
  }
  __syncthreads();
  const float cf = coef[0];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < rows * k;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / k;
    const int j = (int)(t - i * k);
    float s = 0.f;
    for (int p = 0; p < k; ++p) s += Hh[i * k + p] * As[p * k + j] - Hs[i * k + p] * Bs[j * k + p];
    dH[t] = cf * s;
  }
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int64_t count, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x) {
    const float gg = g[t];
    const float mm = b1 * m[t] + (1.f - b1) * gg;
    const float vv = b2 * v[t] + (1.f - b2) * gg * gg;
    m[t] = mm;
    v[t] = vv;
    p[t] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  }
}

// He-uniform init from Philox: counter (index lo, index hi, layer, 4), key seed.
__global__ void mlp_init_kernel(float* p, int64_t count, float lim, uint32_t layer, uint32_t k0, uint32_t k1) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const Philox4 r = philox4x32_10((uint32_t)t, (uint32_t)(t >> 32), layer, 4u, k0, k1);
  const double u = (double)r.x0 * 0x1p-32;
  p[t] = (float)((2.0 * u - 1.0) * lim);
}

}  // namespace symnmf

using namespace symnmf;

struct symnmf_mlp_ctx {
  int d[4];
  int64_t off[7];  // W1, b1, W2, b2, W3, b3, end
  cudaStream_t st;
  float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
  // activations for `cap` rows
  int64_t cap = 0;
  float *z1 = nullptr, *a1 = nullptr, *z2 = nullptr, *a2 = nullptr, *z3 = nullptr, *out = nullptr, *dout = nullptr,
        *da2 = nullptr, *da1 = nullptr;
  double *G = nullptr, *ws = nullptr, *loss = nullptr;
  float *Gf = nullptr, *coef = nullptr;
  unsigned* counter = nullptr;
  std::vector<void*> allocs;
};

static cudaError_t malloc_m(symnmf_mlp_t m, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) m->allocs.push_back(*p);
  return e;
}

static symnmf_status ensure_rows(symnmf_mlp_t m, int64_t rows) {
  if (rows <= m->cap) return SYMNMF_OK;
  for (float** p : {&m->z1, &m->a1, &m->z2, &m->a2, &m->z3, &m->out, &m->dout, &m->da2, &m->da1}) {
    if (*p) {
      cudaFree(*p);
      m->allocs.erase(std::remove(m->allocs.begin(), m->allocs.end(), (void*)*p), m->allocs.end());
      *p = nullptr;
    }
  }
  const int h1 = m->d[1], h2 = m->d[2], o = m->d[3];
  struct {
    float** p;
    int w;
  } bufs[] = {{&m->z1, h1}, {&m->a1, h1}, {&m->z2, h2}, {&m->a2, h2}, {&m->z3, o},
              {&m->out, o}, {&m->dout, o}, {&m->da2, h2}, {&m->da1, h1}};
  for (auto& b : bufs)
    if (malloc_m(m, (void**)b.p, (size_t)rows * b.w * 4) != cudaSuccess) return SYMNMF_ENOMEM;
  m->cap = rows;
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_mlp_create(int in, int h1, int h2, int out, uint64_t seed, void* stream,
                                           symnmf_mlp_t* out_net) {
  if (!out_net || in < 1 || h1 < 1 || h2 < 1 || out < 1 || out > 64) return SYMNMF_EINVAL;
  *out_net = nullptr;
  symnmf_mlp_t m = new symnmf_mlp_ctx();
  m->d[0] = in;
  m->d[1] = h1;
  m->d[2] = h2;
  m->d[3] = out;
  m->st = (cudaStream_t)stream;
  int64_t o = 0;
  for (int l = 0; l < 3; ++l) {
    m->off[2 * l] = o;
    o += (int64_t)m->d[l] * m->d[l + 1];
    m->off[2 * l + 1] = o;
    o += m->d[l + 1];
  }
  m->off[6] = o;
  const size_t bytes = (size_t)o * 4;
  if (malloc_m(m, (void**)&m->params, bytes) != cudaSuccess || malloc_m(m, (void**)&m->grads, bytes) != cudaSuccess ||
      malloc_m(m, (void**)&m->m, bytes) != cudaSuccess || malloc_m(m, (void**)&m->v, bytes) != cudaSuccess ||
      malloc_m(m, (void**)&m->G, 3 * 64 * 64 * 8) != cudaSuccess ||
      malloc_m(m, (void**)&m->ws, xcross_ws_doubles(64, 64) * 8) != cudaSuccess ||
      malloc_m(m, (void**)&m->loss, 8) != cudaSuccess || malloc_m(m, (void**)&m->Gf, 3 * 64 * 64 * 4) != cudaSuccess ||
      malloc_m(m, (void**)&m->coef, 4) != cudaSuccess || malloc_m(m, (void**)&m->counter, 4) != cudaSuccess) {
    symnmf_mlp_destroy(m);
    return SYMNMF_ENOMEM;
  }
  cudaStream_t st = m->st;
  cudaMemsetAsync(m->params, 0, bytes, st);
  cudaMemsetAsync(m->m, 0, bytes, st);
  cudaMemsetAsync(m->v, 0, bytes, st);
  cudaMemsetAsync(m->counter, 0, 4, st);
  for (int l = 0; l < 3; ++l) {
    const int64_t cnt = (int64_t)m->d[l] * m->d[l + 1];
    const float lim = sqrtf(6.0f / (float)m->d[l]);
    mlp_init_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(m->params + m->off[2 * l], cnt, lim, l,
                                                                    (uint32_t)seed, (uint32_t)(seed >> 32));
    count_launches(1);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    symnmf_mlp_destroy(m);
    return SYMNMF_ECUDA;
  }
  *out_net = m;
  return SYMNMF_OK;
}

extern "C" void symnmf_mlp_destroy(symnmf_mlp_t m) {
  if (!m) return;
  for (void* p : m->allocs) cudaFree(p);
  delete m;
}

extern "C" int64_t symnmf_mlp_param_count(symnmf_mlp_t m) { return m ? m->off[6] : 0; }

extern "C" symnmf_status symnmf_mlp_get_params(symnmf_mlp_t m, float* host_out, int64_t count) {
  if (!m || !host_out || count != m->off[6]) return SYMNMF_EINVAL;
  if (cudaMemcpyAsync(host_out, m->params, count * 4, cudaMemcpyDeviceToHost, m->st) != cudaSuccess ||
      cudaStreamSynchronize(m->st) != cudaSuccess)
    return SYMNMF_ECUDA;
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_mlp_set_params(symnmf_mlp_t m, const float* host_in, int64_t count) {
  if (!m || !host_in || count != m->off[6]) return SYMNMF_EINVAL;
  if (cudaMemcpyAsync(m->params, host_in, count * 4, cudaMemcpyHostToDevice, m->st) != cudaSuccess ||
      cudaStreamSynchronize(m->st) != cudaSuccess)
    return SYMNMF_ECUDA;
  return SYMNMF_OK;
}

static symnmf_status forward(symnmf_mlp_t m, const float* x, int64_t rows, float* out) {
  const int in = m->d[0], h1 = m->d[1], h2 = m->d[2], o = m->d[3];
  const float* P = m->params;
  cudaStream_t st = m->st;
  if (mlp_gemm<false, false>(x, in, P + m->off[0], h1, m->a1, h1, (int)rows, h1, in, P + m->off[1], ACT_RELU,
                             m->z1, 1, st) != cudaSuccess ||
      mlp_gemm<false, false>(m->a1, h1, P + m->off[2], h2, m->a2, h2, (int)rows, h2, h1, P + m->off[3], ACT_RELU,
                             m->z2, 1, st) != cudaSuccess ||
      mlp_gemm<false, false>(m->a2, h2, P + m->off[4], o, out, o, (int)rows, o, h2, P + m->off[5], ACT_SOFTPLUS,
                             m->z3, 1, st) != cudaSuccess)
    return SYMNMF_ECUDA;
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_mlp_forward(symnmf_mlp_t m, const float* x, int64_t rows, float* out) {
  if (!m || !x || !out || rows < 1 || rows > (int64_t)1 << 30) return SYMNMF_EINVAL;
  symnmf_status s = ensure_rows(m, rows);
  if (s != SYMNMF_OK) return s;
  return forward(m, x, rows, out);
}

static int splits_for(int64_t rows) {
  int s = (int)std::min<int64_t>(64, (rows + 1023) / 1024);
  return s < 1 ? 1 : s;
}

extern "C" symnmf_status symnmf_mlp_loss_grad(symnmf_mlp_t m, const float* x, const float* Hstar, int64_t rows,
                                              float* grads, double* loss_host) {
  if (!m || !x || !Hstar || rows < 1 || rows > (int64_t)1 << 30) return SYMNMF_EINVAL;
  symnmf_status s = ensure_rows(m, rows);
  if (s != SYMNMF_OK) return s;
  s = forward(m, x, rows, m->out);
  if (s != SYMNMF_OK) return s;
  const int in = m->d[0], h1 = m->d[1], h2 = m->d[2], k = m->d[3];
  cudaStream_t st = m->st;
  double* A = m->G;
  double* B = m->G + 64 * 64;
  double* Cm = m->G + 2 * 64 * 64;
  float* Af = m->Gf;
  float* Bf = m->Gf + 64 * 64;
  cudaError_t e;
  // k x k Grams (FP64 accumulation) and the loss
  if ((e = xcross(m->out, k, k, m->out, k, k, rows, nullptr, nullptr, nullptr, nullptr, 0.0, A, Af, m->ws,
                  m->counter, st)) != cudaSuccess ||
      (e = xcross(m->out, k, k, Hstar, k, k, rows, nullptr, nullptr, nullptr, nullptr, 0.0, B, Bf, m->ws,
                  m->counter, st)) != cudaSuccess ||
      (e = xcross(Hstar, k, k, Hstar, k, k, rows, nullptr, nullptr, nullptr, nullptr, 0.0, Cm, nullptr, m->ws,
                  m->counter, st)) != cudaSuccess)
    return to_status(e);
  gram_loss_kernel<<<1, 256, 0, st>>>(A, B, Cm, k, m->loss, m->coef);
  gram_loss_grad_kernel<<<num_sms() * 4, 256, 0, st>>>(m->out, Hstar, Af, Bf, m->coef, rows, k, m->dout);
  count_launches(2);
  // backward through softplus, relu, relu
  float* g = m->grads;
  const float* P = m->params;
  cudaMemsetAsync(g, 0, (size_t)m->off[6] * 4, st);
  const int sp = splits_for(rows);
  const int64_t ak = rows * k;
  act_grad_kernel<<<num_sms() * 4, 256, 0, st>>>(m->dout, m->z3, ak, ACT_SOFTPLUS);
  count_launches(1);
  if (mlp_gemm<true, false>(m->a2, h2, m->dout, k, g + m->off[4], k, h2, k, rows, nullptr, 0, nullptr, sp, st) !=
      cudaSuccess)
    return SYMNMF_ECUDA;
  colsum_kernel<<<dim3((k + 31) / 32, (unsigned)((rows + 1023) / 1024)), 256, 0, st>>>(m->dout, rows, k,
                                                                                       g + m->off[5]);
  count_launches(1);
  if (mlp_gemm<false, true>(m->dout, k, P + m->off[4], k, m->da2, h2, (int)rows, h2, k, nullptr, 0, nullptr, 1,
                            st) != cudaSuccess)
    return SYMNMF_ECUDA;
  act_grad_kernel<<<num_sms() * 4, 256, 0, st>>>(m->da2, m->z2, rows * h2, ACT_RELU);
  count_launches(1);
  if (mlp_gemm<true, false>(m->a1, h1, m->da2, h2, g + m->off[2], h2, h1, h2, rows, nullptr, 0, nullptr, sp, st) !=
      cudaSuccess)
    return SYMNMF_ECUDA;
  colsum_kernel<<<dim3((h2 + 31) / 32, (unsigned)((rows + 1023) / 1024)), 256, 0, st>>>(m->da2, rows, h2,
                                                                                        g + m->off[3]);
  count_launches(1);
  if (mlp_gemm<false, true>(m->da2, h2, P + m->off[2], h2, m->da1, h1, (int)rows, h1, h2, nullptr, 0, nullptr, 1,
                            st) != cudaSuccess)
    return SYMNMF_ECUDA;
  act_grad_kernel<<<num_sms() * 4, 256, 0, st>>>(m->da1, m->z1, rows * h1, ACT_RELU);
  count_launches(1);
  if (mlp_gemm<true, false>(x, in, m->da1, h1, g + m->off[0], h1, in, h1, rows, nullptr, 0, nullptr, sp, st) !=
      cudaSuccess)
    return SYMNMF_ECUDA;
  colsum_kernel<<<dim3((h1 + 31) / 32, (unsigned)((rows + 1023) / 1024)), 256, 0, st>>>(m->da1, rows, h1,
                                                                                        g + m->off[1]);
  count_launches(1);
  if (grads && cudaMemcpyAsync(grads, g, (size_t)m->off[6] * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return SYMNMF_ECUDA;
  if (loss_host) {
    if (cudaMemcpyAsync(loss_host, m->loss, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return SYMNMF_ECUDA;
  }
  return cudaGetLastError() == cudaSuccess ? SYMNMF_OK : SYMNMF_ECUDA;
}

extern "C" symnmf_status symnmf_mlp_adam(symnmf_mlp_t m, float lr, int t) {
  if (!m || t < 1) return SYMNMF_EINVAL;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  adam_kernel<<<num_sms() * 2, 256, 0, m->st>>>(m->params, m->grads, m->m, m->v, m->off[6], lr, b1, b2, 1e-8f, c1,
                                                 c2);
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? SYMNMF_OK : SYMNMF_ECUDA;
}

extern "C" symnmf_status symnmf_warm_start(symnmf_t h, symnmf_mlp_t m, const float* features) {
  if (!h || !m) return SYMNMF_EINVAL;
  if (m->d[3] != h->k) return SYMNMF_EINVAL;
  const float* f = features;
  float* buf = nullptr;
  if (!f) {
    if (!h->lai_ready || h->l != m->d[0]) return SYMNMF_ESTATE;
    if (cudaMallocAsync((void**)&buf, (size_t)h->n * h->l * 4, h->st) != cudaSuccess) return SYMNMF_ENOMEM;
    symnmf_status s = symnmf_sketch_features(h, buf);
    if (s != SYMNMF_OK) {
      cudaFreeAsync(buf, h->st);
      return s;
    }
    f = buf;
  }
  float* H0 = nullptr;
  if (cudaMallocAsync((void**)&H0, (size_t)h->n * h->k * 4, h->st) != cudaSuccess) {
    if (buf) cudaFreeAsync(buf, h->st);
    return SYMNMF_ENOMEM;
  }
  cudaStream_t saved = m->st;
  m->st = h->st;
  symnmf_status s = ensure_rows(m, h->n);
  if (s == SYMNMF_OK) s = forward(m, f, h->n, H0);
  m->st = saved;
  if (buf) cudaFreeAsync(buf, h->st);
  if (s == SYMNMF_OK) s = symnmf_set_factors(h, H0, nullptr);
  cudaFreeAsync(H0, h->st);
  return s;
}
