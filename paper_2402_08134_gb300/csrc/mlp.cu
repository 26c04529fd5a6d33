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
// Mixed precision: every product -- the three of the forward pass and the
// five of the backward pass (three weight gradients, two activation
// gradients) -- is a BF16 x BF16 tcgen05 GEMM with FP32 accumulation
// (tc_gemm, gemm_tc.cu); weights, biases, activations, pre-activations and
// Adam's state stay FP32 (master weights), converted to BF16 only as GEMM
// operands.  Weight gradients reduce over all rows inside the GEMM's
// stream-K split, whose partials are summed in a fixed order; bias gradients
// are column sums in a fixed order: training is deterministic.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "../../include/symnmf.h"
#include "common.cuh"
#include "handle.h"
#include "kernels.h"

namespace symnmf {

enum { ACT_NONE = 0, ACT_RELU = 1, ACT_SOFTPLUS = 2 };

__host__ __device__ inline int64_t mlp_pad(int64_t v, int64_t to) { return (v + to - 1) / to * to; }

// dst (Rpad x ldd, BF16) = src (R x C, ld lds) rounded to nearest, zero elsewhere.
__global__ void to_bf16_rows_kernel(const float* __restrict__ src, int64_t R, int C, int64_t lds,
                                    __nv_bfloat16* dst, int64_t Rpad, int64_t ldd) {
  const int64_t total = Rpad * ldd;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / ldd;
    const int64_t c = t - r * ldd;
    dst[t] = __float2bfloat16_rn((r < R && c < C) ? src[r * lds + c] : 0.f);
  }
}

// In place: z = Y + b (kept for the backward pass); a = act(z), and when Ab is
// given its BF16 copy (rows of ld ldb), the next layer's GEMM operand.
__global__ void bias_act_kernel(float* Z, const float* __restrict__ b, int64_t rows, int N, int act, float* A,
                                __nv_bfloat16* Ab, int64_t ldb) {
  const int64_t total = rows * N;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / N;
    const int c = (int)(t - r * N);
    const float z = Z[t] + b[c];
    Z[t] = z;
    const float a = act == ACT_RELU ? fmaxf(z, 0.f) : act == ACT_SOFTPLUS ? (z > 20.f ? z : log1pf(expf(z))) : z;
    A[t] = a;
    if (Ab) Ab[r * ldb + c] = __float2bfloat16_rn(a);
  }
}

// Column sums in a fixed order: block b sums rows [b R, (b + 1) R) of every
// column (threads over columns, coalesced), then one pass adds the blocks'
// sums in block order.
constexpr int CS_ROWS = 2048;
__global__ void colsum_part_kernel(const float* __restrict__ X, int64_t rows, int cols, double* ws) {
  const int64_t r0 = (int64_t)blockIdx.x * CS_ROWS, r1 = min(rows, r0 + CS_ROWS);
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    double s = 0.0;
    for (int64_t r = r0; r < r1; ++r) s += X[r * cols + c];
    ws[(int64_t)blockIdx.x * cols + c] = s;
  }
}
__global__ void colsum_final_kernel(const double* __restrict__ ws, int nb, int cols, float* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += ws[(int64_t)b * cols + c];
  out[c] = (float)s;
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
  bool packed = false;  // BF16 weight copies follow params
  // BF16 weight operands: forward W_L^T packed (BN(out) x pad16(in)); backward W3, W2 rows
  __nv_bfloat16 *W1P = nullptr, *W2P = nullptr, *W3P = nullptr, *W3b = nullptr, *W2b = nullptr;
  // activations for `cap` rows
  int64_t cap = 0;
  float *z1 = nullptr, *a1 = nullptr, *z2 = nullptr, *a2 = nullptr, *z3 = nullptr, *out = nullptr, *dout = nullptr,
        *da2 = nullptr, *da1 = nullptr;
  __nv_bfloat16 *xb = nullptr, *a1b = nullptr, *a2b = nullptr, *dz3b = nullptr, *dz2b = nullptr;  // GEMM A rows
  __nv_bfloat16 *xT = nullptr, *a1T = nullptr, *a2T = nullptr;                                      // transposed
  __nv_bfloat16 *dz1P = nullptr, *dz2P = nullptr, *dz3P = nullptr;  // dZ packed as the B operand of dW
  float* gws = nullptr;
  size_t gws_floats = 0;
  double* cws = nullptr;  // column-sum partials
  double *G = nullptr, *ws = nullptr, *loss = nullptr;
  float *Gf = nullptr, *coef = nullptr;
  unsigned* counter = nullptr;
  unsigned* err = nullptr;
  std::vector<void*> allocs;
  std::vector<void*> row_allocs;  // freed when the row capacity grows
};

static int bn_of(int N) { return tc_block_n(N); }
static int64_t p8(int64_t v) { return mlp_pad(v, 8); }
static int64_t p16(int64_t v) { return mlp_pad(v, 16); }

static cudaError_t malloc_m(symnmf_mlp_t m, void** p, size_t bytes, bool per_rows = false) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) (per_rows ? m->row_allocs : m->allocs).push_back(*p);
  return e;
}

static cudaError_t to_bf16_rows(const float* src, int64_t R, int C, int64_t lds, __nv_bfloat16* dst, int64_t Rpad,
                                int64_t ldd, cudaStream_t st) {
  const int64_t total = Rpad * ldd;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 8));
  to_bf16_rows_kernel<<<grid, 256, 0, st>>>(src, R, C, lds, dst, Rpad, ldd);
  count_launches(1);
  return cudaGetLastError();
}

// Y (rows x N, ld ldy) = A (rows x kdim, BF16, ld lda) times the right factor whose columns are the
// rows of Bp (BN(N) x ldb, BF16): one tcgen05 GEMM with a deterministic stream-K reduction.
static cudaError_t mgemm(symnmf_mlp_t m, const void* A, int64_t lda, int64_t rows, int64_t kdim, const void* Bp,
                         int64_t ldb, int N, float* Y, int ldy) {
  return tc_gemm(SYMNMF_X_DENSE_BF16, A, lda, rows, kdim, nullptr, Bp, ldb, nullptr, N, Y, ldy, m->gws,
                 m->gws_floats, m->err, m->st);
}

static cudaError_t colsum(symnmf_mlp_t m, const float* X, int64_t rows, int cols, float* out) {
  const int nb = (int)((rows + CS_ROWS - 1) / CS_ROWS);
  colsum_part_kernel<<<nb, 256, 0, m->st>>>(X, rows, cols, m->cws);
  colsum_final_kernel<<<(cols + 255) / 256, 256, 0, m->st>>>(m->cws, nb, cols, out);
  count_launches(2);
  return cudaGetLastError();
}

// BF16 copies of the weights (after create, set_params or an Adam step).
static cudaError_t pack_weights(symnmf_mlp_t m) {
  if (m->packed) return cudaSuccess;
  const int in = m->d[0], h1 = m->d[1], h2 = m->d[2], o = m->d[3];
  const float* P = m->params;
  cudaStream_t st = m->st;
  cudaError_t e;
  if ((e = pack_ft_bf16(P + m->off[0], in, h1, h1, bn_of(h1), m->W1P, p16(in), st)) != cudaSuccess) return e;
  if ((e = pack_ft_bf16(P + m->off[2], h1, h2, h2, bn_of(h2), m->W2P, p16(h1), st)) != cudaSuccess) return e;
  if ((e = pack_ft_bf16(P + m->off[4], h2, o, o, bn_of(o), m->W3P, p16(h2), st)) != cudaSuccess) return e;
  if ((e = to_bf16_rows(P + m->off[4], h2, o, o, m->W3b, bn_of(h2), p16(o), st)) != cudaSuccess) return e;
  if ((e = to_bf16_rows(P + m->off[2], h1, h2, h2, m->W2b, bn_of(h1), p16(h2), st)) != cudaSuccess) return e;
  m->packed = true;
  return cudaSuccess;
}

static symnmf_status ensure_rows(symnmf_mlp_t m, int64_t rows) {
  if (rows <= m->cap) return SYMNMF_OK;
  for (void* p : m->row_allocs) cudaFree(p);
  m->row_allocs.clear();
  const int in = m->d[0], h1 = m->d[1], h2 = m->d[2], o = m->d[3];
  const int64_t rp = p16(rows);
  struct F32 {
    float** p;
    int w;
  } f32[] = {{&m->z1, h1}, {&m->a1, h1}, {&m->z2, h2}, {&m->a2, h2}, {&m->z3, o},
             {&m->out, o}, {&m->dout, o}, {&m->da2, h2}, {&m->da1, h1}};
  for (auto& b : f32)
    if (malloc_m(m, (void**)b.p, (size_t)rows * b.w * 4, true) != cudaSuccess) return SYMNMF_ENOMEM;
  struct B16 {
    __nv_bfloat16** p;
    size_t count;
  } b16[] = {{&m->xb, (size_t)rows * p8(in)},      {&m->a1b, (size_t)rows * p8(h1)}, {&m->a2b, (size_t)rows * p8(h2)},
             {&m->dz3b, (size_t)rows * p8(o)},     {&m->dz2b, (size_t)rows * p8(h2)}, {&m->xT, (size_t)in * rp},
             {&m->a1T, (size_t)h1 * rp},           {&m->a2T, (size_t)h2 * rp},       {&m->dz1P, (size_t)bn_of(h1) * rp},
             {&m->dz2P, (size_t)bn_of(h2) * rp},   {&m->dz3P, (size_t)bn_of(o) * rp}};
  for (auto& b : b16)
    if (malloc_m(m, (void**)b.p, b.count * 2, true) != cudaSuccess) return SYMNMF_ENOMEM;
  const int64_t nb = (rows + CS_ROWS - 1) / CS_ROWS;
  if (malloc_m(m, (void**)&m->cws, (size_t)nb * std::max(std::max(h1, h2), o) * 8, true) != cudaSuccess)
    return SYMNMF_ENOMEM;
  m->cap = rows;
  return SYMNMF_OK;
}

// Row buffers for `rows` and GEMM scratch for the largest of the eight
// products' plans at this row count.
static symnmf_status prepare(symnmf_mlp_t m, int64_t rows) {
  symnmf_status s = ensure_rows(m, rows);
  if (s != SYMNMF_OK) return s;
  const int in = m->d[0], h1 = m->d[1], h2 = m->d[2], o = m->d[3];
  const int64_t shapes[8][3] = {{rows, in, h1}, {rows, h1, h2}, {rows, h2, o},  {h2, rows, o},
                                {rows, o, h2},  {h1, rows, h2}, {rows, h2, h1}, {in, rows, h1}};
  size_t need = 0;
  for (auto& sh : shapes) need = std::max(need, tc_gemm_ws_floats(sh[0], sh[1], bn_of((int)sh[2])));
  if (need > m->gws_floats) {
    if (m->gws) {
      cudaFree(m->gws);
      m->allocs.erase(std::remove(m->allocs.begin(), m->allocs.end(), (void*)m->gws), m->allocs.end());
      m->gws = nullptr;
      m->gws_floats = 0;
    }
    if (malloc_m(m, (void**)&m->gws, need * 4) != cudaSuccess) return SYMNMF_ENOMEM;
    m->gws_floats = need;
  }
  return SYMNMF_OK;
}

// The bounded waits of the tensor-core products record a timeout in the error
// word; read it at the calls that synchronise.
static symnmf_status read_err(symnmf_mlp_t m) {
  unsigned e = 0;
  if (cudaMemcpyAsync(&e, m->err, 4, cudaMemcpyDeviceToHost, m->st) != cudaSuccess ||
      cudaStreamSynchronize(m->st) != cudaSuccess)
    return SYMNMF_ECUDA;
  if (!e) return SYMNMF_OK;
  cudaMemsetAsync(m->err, 0, 4, m->st);
  return SYMNMF_ETIMEOUT;
}

extern "C" symnmf_status symnmf_mlp_create(int in, int h1, int h2, int out, uint64_t seed, void* stream,
                                           symnmf_mlp_t* out_net) {
  // widths: the tensor-core products take up to 512 output columns; the loss's
  // k x k Grams up to 64
  if (!out_net || in < 1 || in > (1 << 20) || h1 < 1 || h1 > 512 || h2 < 1 || h2 > 512 || out < 1 || out > 64)
    return SYMNMF_EINVAL;
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
  const size_t bf = 2;
  if (malloc_m(m, (void**)&m->params, bytes) != cudaSuccess || malloc_m(m, (void**)&m->grads, bytes) != cudaSuccess ||
      malloc_m(m, (void**)&m->m, bytes) != cudaSuccess || malloc_m(m, (void**)&m->v, bytes) != cudaSuccess ||
      malloc_m(m, (void**)&m->G, 3 * 64 * 64 * 8) != cudaSuccess ||
      malloc_m(m, (void**)&m->ws, xcross_ws_doubles(64, 64) * 8) != cudaSuccess ||
      malloc_m(m, (void**)&m->loss, 8) != cudaSuccess || malloc_m(m, (void**)&m->Gf, 3 * 64 * 64 * 4) != cudaSuccess ||
      malloc_m(m, (void**)&m->coef, 4) != cudaSuccess || malloc_m(m, (void**)&m->counter, 4) != cudaSuccess ||
      malloc_m(m, (void**)&m->err, 4) != cudaSuccess ||
      malloc_m(m, (void**)&m->W1P, bf * bn_of(h1) * p16(in)) != cudaSuccess ||
      malloc_m(m, (void**)&m->W2P, bf * bn_of(h2) * p16(h1)) != cudaSuccess ||
      malloc_m(m, (void**)&m->W3P, bf * bn_of(out) * p16(h2)) != cudaSuccess ||
      malloc_m(m, (void**)&m->W3b, bf * bn_of(h2) * p16(out)) != cudaSuccess ||
      malloc_m(m, (void**)&m->W2b, bf * bn_of(h1) * p16(h2)) != cudaSuccess) {
    symnmf_mlp_destroy(m);
    return SYMNMF_ENOMEM;
  }
  cudaStream_t st = m->st;
  cudaMemsetAsync(m->params, 0, bytes, st);
  cudaMemsetAsync(m->m, 0, bytes, st);
  cudaMemsetAsync(m->v, 0, bytes, st);
  cudaMemsetAsync(m->counter, 0, 4, st);
  cudaMemsetAsync(m->err, 0, 4, st);
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
  for (void* p : m->row_allocs) cudaFree(p);
  for (void* p : m->allocs) cudaFree(p);
  delete m;
}

extern "C" int64_t symnmf_mlp_param_count(symnmf_mlp_t m) { return m ? m->off[6] : 0; }

extern "C" symnmf_status symnmf_mlp_get_params(symnmf_mlp_t m, float* host_out, int64_t count) {
  if (!m || !host_out || count != m->off[6]) return SYMNMF_EINVAL;
  if (cudaMemcpyAsync(host_out, m->params, count * 4, cudaMemcpyDeviceToHost, m->st) != cudaSuccess)
    return SYMNMF_ECUDA;
  return read_err(m);
}

extern "C" symnmf_status symnmf_mlp_set_params(symnmf_mlp_t m, const float* host_in, int64_t count) {
  if (!m || !host_in || count != m->off[6]) return SYMNMF_EINVAL;
  if (cudaMemcpyAsync(m->params, host_in, count * 4, cudaMemcpyHostToDevice, m->st) != cudaSuccess ||
      cudaStreamSynchronize(m->st) != cudaSuccess)
    return SYMNMF_ECUDA;
  m->packed = false;
  return SYMNMF_OK;
}

// Three BF16 tensor-core products, each followed by one kernel that adds the
// bias, applies the activation and writes the next product's BF16 operand.
static symnmf_status forward(symnmf_mlp_t m, const float* x, int64_t rows, float* out) {
  const int in = m->d[0], h1 = m->d[1], h2 = m->d[2], o = m->d[3];
  const float* P = m->params;
  cudaStream_t st = m->st;
  const int grid = num_sms() * 4;
  cudaError_t e;
  if ((e = pack_weights(m)) != cudaSuccess || (e = to_bf16_rows(x, rows, in, in, m->xb, rows, p8(in), st)) != cudaSuccess ||
      (e = mgemm(m, m->xb, p8(in), rows, in, m->W1P, p16(in), h1, m->z1, h1)) != cudaSuccess)
    return to_status(e);
  bias_act_kernel<<<grid, 256, 0, st>>>(m->z1, P + m->off[1], rows, h1, ACT_RELU, m->a1, m->a1b, p8(h1));
  count_launches(1);
  if ((e = mgemm(m, m->a1b, p8(h1), rows, h1, m->W2P, p16(h1), h2, m->z2, h2)) != cudaSuccess) return to_status(e);
  bias_act_kernel<<<grid, 256, 0, st>>>(m->z2, P + m->off[3], rows, h2, ACT_RELU, m->a2, m->a2b, p8(h2));
  count_launches(1);
  if ((e = mgemm(m, m->a2b, p8(h2), rows, h2, m->W3P, p16(h2), o, m->z3, o)) != cudaSuccess) return to_status(e);
  bias_act_kernel<<<grid, 256, 0, st>>>(m->z3, P + m->off[5], rows, o, ACT_SOFTPLUS, out, nullptr, 0);
  count_launches(1);
  return to_status(cudaGetLastError());
}

extern "C" symnmf_status symnmf_mlp_forward(symnmf_mlp_t m, const float* x, int64_t rows, float* out) {
  if (!m || !x || !out || rows < 1 || rows > (int64_t)1 << 30) return SYMNMF_EINVAL;
  symnmf_status s = prepare(m, rows);
  if (s != SYMNMF_OK) return s;
  return forward(m, x, rows, out);
}

// Backward pass.  For each layer L (from the last): dW_L = A_{L-1}^T dZ_L is one
// tensor-core product over all rows (A^T and dZ^T packed K-major along the
// rows), db_L a fixed-order column sum, and dA_{L-1} = dZ_L W_L^T a product
// with the BF16 rows of W_L as the packed operand.
extern "C" symnmf_status symnmf_mlp_loss_grad(symnmf_mlp_t m, const float* x, const float* Hstar, int64_t rows,
                                              float* grads, double* loss_host) {
  if (!m || !x || !Hstar || rows < 1 || rows > (int64_t)1 << 30) return SYMNMF_EINVAL;
  symnmf_status s = prepare(m, rows);
  if (s != SYMNMF_OK) return s;
  s = forward(m, x, rows, m->out);
  if (s != SYMNMF_OK) return s;
  const int in = m->d[0], h1 = m->d[1], h2 = m->d[2], k = m->d[3];
  const int64_t rp = p16(rows);
  cudaStream_t st = m->st;
  const int grid = num_sms() * 4;
  double* A = m->G;
  double* B = m->G + 64 * 64;
  double* Cm = m->G + 2 * 64 * 64;
  float* Af = m->Gf;
  float* Bf = m->Gf + 64 * 64;
  cudaError_t e;
  // k x k Grams (FP64 accumulation), the loss and dL/dH^
  if ((e = xcross(m->out, k, k, m->out, k, k, rows, nullptr, nullptr, nullptr, nullptr, 0.0, A, Af, m->ws,
                  m->counter, st)) != cudaSuccess ||
      (e = xcross(m->out, k, k, Hstar, k, k, rows, nullptr, nullptr, nullptr, nullptr, 0.0, B, Bf, m->ws,
                  m->counter, st)) != cudaSuccess ||
      (e = xcross(Hstar, k, k, Hstar, k, k, rows, nullptr, nullptr, nullptr, nullptr, 0.0, Cm, nullptr, m->ws,
                  m->counter, st)) != cudaSuccess)
    return to_status(e);
  gram_loss_kernel<<<1, 256, 0, st>>>(A, B, Cm, k, m->loss, m->coef);
  gram_loss_grad_kernel<<<grid, 256, 0, st>>>(m->out, Hstar, Af, Bf, m->coef, rows, k, m->dout);
  act_grad_kernel<<<grid, 256, 0, st>>>(m->dout, m->z3, rows * k, ACT_SOFTPLUS);  // dZ3
  count_launches(3);
  float* g = m->grads;
  // layer 3
  if ((e = pack_ft_bf16(m->a2, rows, h2, h2, h2, m->a2T, rp, st)) != cudaSuccess ||
      (e = pack_ft_bf16(m->dout, rows, k, k, bn_of(k), m->dz3P, rp, st)) != cudaSuccess ||
      (e = mgemm(m, m->a2T, rp, h2, rows, m->dz3P, rp, k, g + m->off[4], k)) != cudaSuccess ||
      (e = colsum(m, m->dout, rows, k, g + m->off[5])) != cudaSuccess ||
      (e = to_bf16_rows(m->dout, rows, k, k, m->dz3b, rows, p8(k), st)) != cudaSuccess ||
      (e = mgemm(m, m->dz3b, p8(k), rows, k, m->W3b, p16(k), h2, m->da2, h2)) != cudaSuccess)
    return to_status(e);
  act_grad_kernel<<<grid, 256, 0, st>>>(m->da2, m->z2, rows * h2, ACT_RELU);  // dZ2
  count_launches(1);
  // layer 2
  if ((e = pack_ft_bf16(m->a1, rows, h1, h1, h1, m->a1T, rp, st)) != cudaSuccess ||
      (e = pack_ft_bf16(m->da2, rows, h2, h2, bn_of(h2), m->dz2P, rp, st)) != cudaSuccess ||
      (e = mgemm(m, m->a1T, rp, h1, rows, m->dz2P, rp, h2, g + m->off[2], h2)) != cudaSuccess ||
      (e = colsum(m, m->da2, rows, h2, g + m->off[3])) != cudaSuccess ||
      (e = to_bf16_rows(m->da2, rows, h2, h2, m->dz2b, rows, p8(h2), st)) != cudaSuccess ||
      (e = mgemm(m, m->dz2b, p8(h2), rows, h2, m->W2b, p16(h2), h1, m->da1, h1)) != cudaSuccess)
    return to_status(e);
  act_grad_kernel<<<grid, 256, 0, st>>>(m->da1, m->z1, rows * h1, ACT_RELU);  // dZ1
  count_launches(1);
  // layer 1
  if ((e = pack_ft_bf16(x, rows, in, in, in, m->xT, rp, st)) != cudaSuccess ||
      (e = pack_ft_bf16(m->da1, rows, h1, h1, bn_of(h1), m->dz1P, rp, st)) != cudaSuccess ||
      (e = mgemm(m, m->xT, rp, in, rows, m->dz1P, rp, h1, g + m->off[0], h1)) != cudaSuccess ||
      (e = colsum(m, m->da1, rows, h1, g + m->off[1])) != cudaSuccess)
    return to_status(e);
  if (grads && cudaMemcpyAsync(grads, g, (size_t)m->off[6] * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return SYMNMF_ECUDA;
  if (loss_host) {
    if (cudaMemcpyAsync(loss_host, m->loss, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) return SYMNMF_ECUDA;
    return read_err(m);
  }
  return to_status(cudaGetLastError());
}

extern "C" symnmf_status symnmf_mlp_adam(symnmf_mlp_t m, float lr, int t) {
  if (!m || t < 1) return SYMNMF_EINVAL;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  adam_kernel<<<num_sms() * 2, 256, 0, m->st>>>(m->params, m->grads, m->m, m->v, m->off[6], lr, b1, b2, 1e-8f, c1,
                                                 c2);
  count_launches(1);
  m->packed = false;
  return to_status(cudaGetLastError());
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
  symnmf_status s = prepare(m, h->n);
  if (s == SYMNMF_OK) s = forward(m, f, h->n, H0);
  if (s == SYMNMF_OK) s = read_err(m);
  m->st = saved;
  if (buf) cudaFreeAsync(buf, h->st);
  if (s == SYMNMF_OK) s = symnmf_set_factors(h, H0, nullptr);
  cudaFreeAsync(H0, h->st);
  return s;
}
