// C ABI of the SymNMF library: the solver handle and the driver of the hot
// path.  Every numerical step runs in this library's kernels; this file only
// sequences them on the handle's stream, records sweep bodies as CUDA graphs,
// and maps errors to status codes.
#include <math.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/symnmf.h"
#include "common.cuh"
#include "handle.h"
#include "kernels.h"
#include "persist.cuh"

namespace symnmf {

static std::atomic<uint64_t> g_launches{0};
void count_launches(uint64_t n) { g_launches += n; }

// SM count of the current device, looked up once per device (grids and
// workspaces are sized for the device a call runs on).
int num_sms() {
  constexpr int MAXDEV = 64;
  static std::atomic<int> cached[MAXDEV];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
    cudaGetLastError();
    dev = 0;
  }
  const int slot = dev < MAXDEV ? dev : MAXDEV - 1;
  int v = dev < MAXDEV ? cached[slot].load(std::memory_order_relaxed) : 0;
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
    cudaGetLastError();
    v = 148;
  }
  if (dev < MAXDEV) cached[slot].store(v, std::memory_order_relaxed);
  return v;
}

symnmf_status to_status(cudaError_t e) {
  switch (e) {
    case cudaSuccess: return SYMNMF_OK;
    case cudaErrorMemoryAllocation: return SYMNMF_ENOMEM;
    case cudaErrorInvalidValue: return SYMNMF_EINVAL;
    default: return SYMNMF_ECUDA;
  }
}

}  // namespace symnmf

using namespace symnmf;

// ------------------------------------------------------------------ helpers

static symnmf_status fail(symnmf_t h, symnmf_status s, const std::string& msg) {
  if (h) h->msg = msg;
  return s;
}

static symnmf_status cuda_fail(symnmf_t h, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return SYMNMF_OK;
  cudaGetLastError();
  return fail(h, to_status(e), std::string(where) + ": " + cudaGetErrorString(e));
}

#define TRY(call)                                        \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) return cuda_fail(h, _e, #call); \
  } while (0)

#define TRYS(call)                       \
  do {                                   \
    symnmf_status _s = (call);           \
    if (_s != SYMNMF_OK) return _s;      \
  } while (0)

// Handle memory comes from a library-owned stream-ordered pool per device:
// creating and destroying handles then neither maps fresh memory nor
// synchronises the device (cudaFree does), and up to 1 GiB of freed handle
// memory stays cached for the next handle.  Without a pool, the device's
// default pool is used.
static cudaMemPool_t handle_pool() {
  constexpr int MAXDEV = 64;
  static std::mutex mu;
  static cudaMemPool_t pools[MAXDEV] = {};
  static bool tried[MAXDEV] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!tried[dev]) {
    tried[dev] = true;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&pools[dev], &props) == cudaSuccess) {
      uint64_t keep = (uint64_t)1 << 30;
      cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
      pools[dev] = nullptr;
      cudaGetLastError();
    }
  }
  return pools[dev];
}

// Device memory owned by the handle: stream-ordered on the handle's stream,
// except while a sweep is being captured into a graph (an allocation there
// would become a graph node), where plain cudaMalloc is used.
template <typename T>
static cudaError_t dalloc(symnmf_t h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  const size_t bytes = count * sizeof(T);
  cudaError_t e;
  if (h->capturing) {
    e = cudaMalloc((void**)p, bytes);
    if (e == cudaSuccess) h->allocs_sync.push_back((void*)*p);
    return e;
  }
  cudaMemPool_t pool = handle_pool();
  e = pool ? cudaMallocFromPoolAsync((void**)p, bytes, pool, h->st) : cudaMallocAsync((void**)p, bytes, h->st);
  if (e == cudaSuccess) h->allocs.push_back((void*)*p);
  return e;
}

// Read and clear the device error word (synchronises the stream).
static symnmf_status check_device_error(symnmf_t h) {
  TRY(cudaStreamSynchronize(h->st));
  unsigned e = 0;
  TRY(cudaMemcpy(&e, h->err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (e) TRY(cudaMemset(h->err, 0, sizeof(unsigned)));
  if (e & (ERR_TIMEOUT | ERR_NAN)) h->eng_resume_ok = false;  // the engine's saved state is not trusted
  if (e & ERR_TIMEOUT) return fail(h, SYMNMF_ETIMEOUT, "a bounded device wait ran out");
  if (e & ERR_NOTSPD) return fail(h, SYMNMF_ENOTSPD, "Gram matrix is not positive definite");
  if (e & ERR_NAN) return fail(h, SYMNMF_ENAN, "non-finite value in a factor");
  if (e & ERR_BPP_ITERS) h->msg = "BPP reached its iteration cap on some rows (result kept)";
  return SYMNMF_OK;
}

// Recorded objectives (host, after a synchronising copy): a non-finite one
// means a NaN or Inf reached the operator or the factors.
static symnmf_status check_objectives(symnmf_t h, const double* obj, int count) {
  for (int i = 0; i < count; ++i)
    if (!isfinite(obj[i])) return fail(h, SYMNMF_ENAN, "non-finite objective");
  return SYMNMF_OK;
}

static bool is_dense(int fmt) { return fmt >= SYMNMF_X_DENSE_F64 && fmt <= SYMNMF_X_DENSE_FP8; }

// Workspace for a dense / sparse product of width N.
static symnmf_status ensure_gemm_ws(symnmf_t h, int N) {
  size_t need = 0;
  const int fmt = h->p.fmt;
  if (fmt == SYMNMF_X_DENSE_F32 || fmt == SYMNMF_X_DENSE_F64 || h->p.x_hi)
    need = xf_simt_ws_floats(h->n, N);
  if (fmt == SYMNMF_X_DENSE_BF16 || fmt == SYMNMF_X_DENSE_FP8) {
    const int BN = tc_block_n(N);
    const size_t t = xf_tc_ws_floats(h->n, BN);
    if (t > need) need = t;
    const size_t pack = (size_t)BN * h->ldp * (fmt == SYMNMF_X_DENSE_BF16 ? 2 : 1);
    if (pack > h->fpack_bytes) {
      if (h->capturing) return fail(h, SYMNMF_ESTATE, "allocation during graph capture");
      void* p;
      TRY(dalloc(h, (char**)&p, pack));
      h->fpack = p;
      h->fpack_bytes = pack;
    }
    if (!h->colscale) TRY(dalloc(h, &h->colscale, 512));  // one scale per packed column (BN <= 512)
  }
  if (need > h->gemm_ws_floats) {
    if (h->capturing) return fail(h, SYMNMF_ESTATE, "allocation during graph capture");
    TRY(dalloc(h, &h->gemm_ws, need));
    h->gemm_ws_floats = need;
  }
  return SYMNMF_OK;
}

// Y (n x N, ld ldy) = X F for the operator `src` (SRC_X or SRC_XHI).
symnmf_status product(symnmf_t h, int src, const float* F, int N, int ldf, float* Y, int ldy) {
  TRYS(ensure_gemm_ws(h, N));
  if (src == SYMNMF_SRC_XHI) {
    TRY(xf_simt(SYMNMF_X_DENSE_F32, h->p.x_hi, h->ldx_hi, h->n, F, ldf, N, Y, ldy, h->gemm_ws,
                h->gemm_ws_floats, h->st));
    return SYMNMF_OK;
  }
  const int fmt = h->p.fmt;
  switch (fmt) {
    case SYMNMF_X_DENSE_F64:
    case SYMNMF_X_DENSE_F32:
      if (h->o.gemm == SYMNMF_GEMM_TC) return fail(h, SYMNMF_EUNSUPPORTED, "tcgen05 path needs BF16/FP8 X");
      TRY(xf_simt(fmt, h->p.x, h->ldx, h->n, F, ldf, N, Y, ldy, h->gemm_ws, h->gemm_ws_floats, h->st));
      return SYMNMF_OK;
    case SYMNMF_X_DENSE_BF16:
    case SYMNMF_X_DENSE_FP8: {
      if (h->o.gemm == SYMNMF_GEMM_SIMT) return fail(h, SYMNMF_EUNSUPPORTED, "SIMT path needs F32/F64 X");
      const int BN = tc_block_n(N);
      if (fmt == SYMNMF_X_DENSE_BF16)
        TRY(pack_ft_bf16(F, h->n, ldf, N, BN, h->fpack, h->ldp, h->st));
      else
        TRY(pack_ft_fp8(F, h->n, ldf, N, BN, h->fpack, h->ldp, h->colscale, h->st));
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      if (h->profiling && !h->capturing) {
        if (h->prof_used == h->prof_events.size()) {
          cudaEvent_t a, b;
          TRY(cudaEventCreate(&a));
          TRY(cudaEventCreate(&b));
          h->prof_events.push_back({a, b});
          h->prof_bytes.push_back(0.0);
        }
        e0 = h->prof_events[h->prof_used].first;
        e1 = h->prof_events[h->prof_used].second;
        const double es = fmt == SYMNMF_X_DENSE_BF16 ? 2.0 : 1.0;
        h->prof_bytes[h->prof_used] = (double)h->n * h->n * es + (double)h->n * N * (es + 4.0);
        h->prof_used++;
      }
      TRY(xf_tc(fmt, h->p.x, h->ldx, h->p.row_scale, h->n, h->fpack, h->ldp, h->colscale, N, Y, ldy,
                h->gemm_ws, h->gemm_ws_floats, h->err, h->st, e0, e1));
      return SYMNMF_OK;
    }
    case SYMNMF_X_CSR_F32:
      TRY(csr_xf(h->p.row_ptr, h->p.col, (const float*)h->p.x, h->n, F, ldf, N, Y, ldy, h->st));
      return SYMNMF_OK;
  }
  return fail(h, SYMNMF_EINVAL, "unknown X format");
}

static const double* normx_for(symnmf_t h, int src) {
  if (src == SYMNMF_SRC_LAI) return h->scal + S_LAI_NORM2;
  if (src == SYMNMF_SRC_COMP) return h->scal + S_COMP_NORM2;
  if (src == SYMNMF_SRC_XHI) return h->scal + S_XHI_NORM2;
  return h->scal + S_NORM2;
}

// One half sweep: update F_upd (side 0: W, side 1: H) from the fixed factor.
static symnmf_status half_sweep(symnmf_t h, int side, int src, int rule) {
  h->fac_version++;
  h->grams_fresh = true;  // the updated factor's Gram follows below, the other is current
  const int64_t n = h->n;
  const int k = h->k;
  float* Fu = side ? h->H : h->W;
  const float* Ff = side ? h->W : h->H;
  const int gfix = side ? 1 : 0;  // Gd[0] = H^T H, Gd[1] = W^T W
  const int gupd = side ? 0 : 1;
  const float* Y = nullptr;
  const float* U = nullptr;
  const float* M = nullptr;
  const float* Gf_use = h->Gf[gfix];
  const double* Gd_use = h->Gd[gfix];
  if (src == SYMNMF_SRC_LAI) {
    // M = Lambda (U^T F) (l x k), Y_r = U_r M fused into the update
    TRY(xcross(h->U, h->l, h->l, Ff, k, k, n, nullptr, nullptr, nullptr, h->lam, 0.0, nullptr, h->Mf,
               h->ws, h->counters + 0, h->st));
    U = h->U;
    M = h->Mf;
  } else if (src == SYMNMF_SRC_COMP) {
    // Compressed-NMF: M = Q^T F (l x k), G_c = M^T M, Y_r = (X Q)_r M fused into the update
    TRY(xcross(h->Qk, h->l, h->l, Ff, k, k, n, nullptr, nullptr, nullptr, nullptr, 0.0, nullptr, h->Mf, h->ws,
               h->counters + 0, h->st));
    TRY(xcross(h->Mf, k, k, h->Mf, k, k, h->l, nullptr, nullptr, nullptr, nullptr, 0.0, h->Gs_d, h->Gs_f, h->ws,
               h->counters + 0, h->st));
    U = h->Bk;
    M = h->Mf;
    Gf_use = h->Gs_f;
    Gd_use = h->Gs_d;
  } else {
    TRYS(product(h, src, Ff, k, k, h->Y, k));
    Y = h->Y;
  }
  if (rule == SYMNMF_RULE_HALS)
    TRY(hals_update(Fu, Ff, n, k, Gf_use, h->alpha, Y, k, U, h->l, M, h->scal + S_PART, h->ws,
                    h->counters + 1, h->err, h->st));
  else
    TRY(bpp_rows(Fu, Ff, n, k, Gd_use, h->alpha, Y, k, U, h->l, M, h->scal + S_PART, h->ws,
                 h->counters + 1, h->err, h->st));
  TRY(xcross(Fu, k, k, Fu, k, k, n, nullptr, nullptr, nullptr, nullptr, 0.0, h->Gd[gupd], h->Gf[gupd],
             h->ws, h->counters + 2, h->st));
  // after the H half: the surrogate objective of the operator; for the compressed
  // problem ||Q^T (W H^T - X)||^2 + alpha ||W - H||^2, whose Gram is G_c
  if (side == 1)
    TRY(objective(normx_for(h, src), src == SYMNMF_SRC_COMP ? Gd_use : h->Gd[1], h->Gd[0], k, h->scal + S_PART,
                  h->scal + S_ALPHA, h->obj_ring, h->obj_cnt, OBJ_RING, h->st));
  return SYMNMF_OK;
}

static symnmf_status sweep_body(symnmf_t h, int src, int rule) {
  TRYS(half_sweep(h, 0, src, rule));
  TRYS(half_sweep(h, 1, src, rule));
  return SYMNMF_OK;
}

static symnmf_status refresh_grams(symnmf_t h) {
  h->grams_fresh = true;
  const int k = h->k;
  TRY(xcross(h->H, k, k, h->H, k, k, h->n, nullptr, nullptr, nullptr, nullptr, 0.0, h->Gd[0], h->Gf[0],
             h->ws, h->counters + 2, h->st));
  TRY(xcross(h->W, k, k, h->W, k, k, h->n, nullptr, nullptr, nullptr, nullptr, 0.0, h->Gd[1], h->Gf[1],
             h->ws, h->counters + 2, h->st));
  return SYMNMF_OK;
}

// One thread waits, through the persistent kernels' bounded wait, for a
// word that nothing ever sets; the wait runs out after limit_ns and records
// ERR_TIMEOUT in the handle's error word.
__global__ void wait_unset_flag_kernel(const unsigned* flag, unsigned* err, uint64_t limit_ns) {
  if (threadIdx.x == 0 && blockIdx.x == 0) bounded_wait_geq(flag, 1u, err, limit_ns);
}

// ---------------------------------------------------------------- create

extern "C" symnmf_status symnmf_create(const symnmf_problem* prob, const symnmf_options* opt, void* stream,
                                       symnmf_t* out) {
  if (!out || !prob) return SYMNMF_EINVAL;
  *out = nullptr;
  const symnmf_problem& p = *prob;
  if (p.n < 1 || p.k < 1 || p.k > 64 || !p.x) return SYMNMF_EINVAL;
  if (p.fmt < SYMNMF_X_DENSE_F64 || p.fmt > SYMNMF_X_CSR_F32) return SYMNMF_EINVAL;
  if (p.fmt == SYMNMF_X_CSR_F32 && (!p.row_ptr || !p.col || p.nnz < 0)) return SYMNMF_EINVAL;
  if (p.fmt == SYMNMF_X_DENSE_FP8 && !p.row_scale) return SYMNMF_EINVAL;
  const int64_t ldx = p.ldx > 0 ? p.ldx : p.n;
  if (is_dense(p.fmt) && ldx < p.n) return SYMNMF_EINVAL;
  if (p.fmt == SYMNMF_X_DENSE_BF16 && ((ldx % 8) || ((uintptr_t)p.x & 15))) return SYMNMF_EINVAL;
  if (p.fmt == SYMNMF_X_DENSE_FP8 && ((ldx % 16) || ((uintptr_t)p.x & 15))) return SYMNMF_EINVAL;
  const int64_t ldx_hi = p.ldx_hi > 0 ? p.ldx_hi : p.n;
  if (p.x_hi && ldx_hi < p.n) return SYMNMF_EINVAL;

  symnmf_t h = new symnmf_ctx();
  h->p = p;
  if (opt) h->o = *opt;
  if (h->o.max_width <= 0) h->o.max_width = 2 * p.k + 10;
  if (h->o.max_width > 96) h->o.max_width = 96;
  h->st = (cudaStream_t)stream;
  h->n = p.n;
  h->k = p.k;
  h->ldx = ldx;
  h->ldx_hi = ldx_hi;
  h->ldp = (p.n + 15) / 16 * 16;
  const int64_t n = p.n;
  const int k = p.k;
  auto bail = [&](cudaError_t e) {
    symnmf_status s = to_status(e);
    symnmf_destroy(h);
    return s;
  };
#define CALLOC(ptr, cnt)                          \
  do {                                            \
    cudaError_t _e = dalloc(h, &(ptr), (cnt));    \
    if (_e != cudaSuccess) return bail(_e);       \
  } while (0)
  CALLOC(h->H, (size_t)n * k);
  CALLOC(h->W, (size_t)n * k);
  CALLOC(h->Y, (size_t)n * k);
  for (int i = 0; i < 2; ++i) {
    CALLOC(h->Gd[i], (size_t)k * k);
    CALLOC(h->Gf[i], (size_t)k * k);
  }
  CALLOC(h->Gs_d, (size_t)k * k);
  CALLOC(h->Gs_f, (size_t)k * k);
  CALLOC(h->scal, (size_t)S_COUNT);
  CALLOC(h->obj_ring, (size_t)OBJ_RING);
  CALLOC(h->obj_cnt, 4);
  h->ws_doubles = xcross_ws_doubles(96, 96);
  if (h->ws_doubles < 3 * 4096) h->ws_doubles = 3 * 4096;
  CALLOC(h->ws, h->ws_doubles);
  CALLOC(h->counters, 16);
  CALLOC(h->err, 4);
  CALLOC(h->Rinv_d, (size_t)k * k);
  CALLOC(h->Rinv_f, (size_t)k * k);
#undef CALLOC
  cudaError_t e;
  if ((e = cudaMemsetAsync(h->counters, 0, 16 * sizeof(unsigned), h->st)) != cudaSuccess) return bail(e);
  if ((e = cudaMemsetAsync(h->err, 0, 4 * sizeof(unsigned), h->st)) != cudaSuccess) return bail(e);
  if ((e = cudaMemsetAsync(h->scal, 0, S_COUNT * sizeof(double), h->st)) != cudaSuccess) return bail(e);
  if ((e = cudaMemsetAsync(h->H, 0, (size_t)n * k * 4, h->st)) != cudaSuccess) return bail(e);
  if ((e = cudaMemsetAsync(h->W, 0, (size_t)n * k * 4, h->st)) != cudaSuccess) return bail(e);
  // ||X||^2, max(X), mean(X)
  if ((e = xstats(p.fmt, p.x, ldx, p.row_scale, n, p.row_ptr, p.nnz, h->scal + S_MAX, h->ws,
                  h->counters + 3, h->st)) != cudaSuccess)
    return bail(e);
  if (p.x_hi &&
      (e = xstats(SYMNMF_X_DENSE_F32, p.x_hi, ldx_hi, nullptr, n, nullptr, 0, h->scal + S_XHI_MAX, h->ws,
                  h->counters + 3, h->st)) != cudaSuccess)
    return bail(e);
  if ((e = cudaStreamSynchronize(h->st)) != cudaSuccess) return bail(e);
  double st3[3];
  if ((e = cudaMemcpy(st3, h->scal + S_MAX, 3 * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return bail(e);
  if (!isfinite(st3[0]) || !isfinite(st3[1]) || !isfinite(st3[2])) {
    symnmf_destroy(h);
    return SYMNMF_ENAN;  // X holds a non-finite entry
  }
  double mx = st3[0];
  if (p.fmt == SYMNMF_X_CSR_F32 && p.nnz < n * n) mx = fmax(mx, 0.0);  // implicit zeros
  h->alpha = p.alpha > 0 ? p.alpha : mx;
  h->normX2 = st3[2];
  if (!(h->alpha > 0.0)) {
    symnmf_destroy(h);
    return SYMNMF_EINVAL;  // alpha must be positive (X has no positive entry)
  }
  double host_scal[S_COUNT];
  if ((e = cudaMemcpy(host_scal, h->scal, sizeof(host_scal), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return bail(e);
  if (p.x_hi && (!isfinite(host_scal[S_XHI_MAX]) || !isfinite(host_scal[S_XHI_MAX + 2]))) {
    symnmf_destroy(h);
    return SYMNMF_ENAN;  // the float32 copy holds a non-finite entry
  }
  host_scal[S_ALPHA] = h->alpha;
  host_scal[S_NORM2] = st3[2];
  host_scal[S_MEAN] = st3[1] / ((double)n * (double)n);
  if (!p.x_hi) host_scal[S_XHI_NORM2] = host_scal[S_NORM2];
  if ((e = cudaMemcpy(h->scal, host_scal, sizeof(host_scal), cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(e);
  symnmf_status s = ensure_gemm_ws(h, k);
  if (s != SYMNMF_OK) {
    symnmf_destroy(h);
    return s;
  }
  *out = h;
  return SYMNMF_OK;
}

extern "C" void symnmf_destroy(symnmf_t h) {
  if (!h) return;
  for (auto& g : h->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (h->loop.exec) cudaGraphExecDestroy(h->loop.exec);
  if (h->cap_st) cudaStreamDestroy(h->cap_st);
  for (auto& pr : h->prof_events) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  for (auto& pr : h->eprof_events) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  for (cudaEvent_t e : h->lprof_events) cudaEventDestroy(e);
  for (void* p : h->allocs) cudaFreeAsync(p, h->st);  // after the handle's work on its stream
  for (void* p : h->allocs_sync) cudaFree(p);
  delete h;
}

extern "C" const char* symnmf_last_error(symnmf_t h) { return h ? h->msg.c_str() : "null handle"; }

extern "C" symnmf_status symnmf_info(symnmf_t h, double* alpha, double* normX2) {
  if (!h) return SYMNMF_EINVAL;
  if (alpha) *alpha = h->alpha;
  if (normX2) *normX2 = h->normX2;
  return SYMNMF_OK;
}

extern "C" uint64_t symnmf_launch_count(void) { return g_launches.load(); }

extern "C" symnmf_status symnmf_debug_wait_timeout(symnmf_t h, int64_t limit_ns) {
  if (!h || limit_ns < 1000 || limit_ns > 1000000000) return SYMNMF_EINVAL;
  // counters[15] is zeroed at create and written by no kernel
  wait_unset_flag_kernel<<<1, 32, 0, h->st>>>(h->counters + 15, h->err, (uint64_t)limit_ns);
  count_launches(1);
  TRY(cudaGetLastError());
  return check_device_error(h);
}

// --------------------------------------------------------------- factors

extern "C" symnmf_status symnmf_set_factors(symnmf_t h, const float* H0, const float* W0) {
  if (!h || !H0) return SYMNMF_EINVAL;
  h->fac_version++;
  const size_t bytes = (size_t)h->n * h->k * sizeof(float);
  TRY(cudaMemcpyAsync(h->H, H0, bytes, cudaMemcpyDeviceToDevice, h->st));
  TRY(cudaMemcpyAsync(h->W, W0 ? W0 : H0, bytes, cudaMemcpyDeviceToDevice, h->st));
  TRY(cudaMemsetAsync(h->counters + 8, 0, sizeof(unsigned), h->st));
  TRY(check_factor(h->H, (int64_t)h->n * h->k, h->counters + 8, h->st));
  TRY(check_factor(h->W, (int64_t)h->n * h->k, h->counters + 8, h->st));
  unsigned flags = 0;
  TRY(cudaMemcpyAsync(&flags, h->counters + 8, sizeof(unsigned), cudaMemcpyDeviceToHost, h->st));
  TRY(cudaStreamSynchronize(h->st));
  TRY(cudaMemsetAsync(h->counters + 8, 0, sizeof(unsigned), h->st));
  if (flags) return fail(h, SYMNMF_EINVAL, "starting factors must be finite and nonnegative");
  TRYS(refresh_grams(h));
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_init_random(symnmf_t h, int scaled) {
  if (!h) return SYMNMF_EINVAL;
  h->fac_version++;
  TRY(philox_uniform(h->H, h->n, h->k, h->p.seed, scaled ? h->scal + S_MEAN : nullptr,
                     2.0 / sqrt((double)h->k), h->st));
  TRY(cudaMemcpyAsync(h->W, h->H, (size_t)h->n * h->k * 4, cudaMemcpyDeviceToDevice, h->st));
  TRYS(refresh_grams(h));
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_get_factors(symnmf_t h, float* H_out, float* W_out) {
  if (!h) return SYMNMF_EINVAL;
  const size_t bytes = (size_t)h->n * h->k * sizeof(float);
  if (H_out) TRY(cudaMemcpyAsync(H_out, h->H, bytes, cudaMemcpyDeviceToDevice, h->st));
  if (W_out) TRY(cudaMemcpyAsync(W_out, h->W, bytes, cudaMemcpyDeviceToDevice, h->st));
  return SYMNMF_OK;
}

// ------------------------------------------------------------------- LAI

static symnmf_status ensure_lai(symnmf_t h, int l) {
  if (h->lai_cap >= l) return SYMNMF_OK;
  const int L = h->o.max_width;
  const size_t nl = (size_t)h->n * L;
  TRY(dalloc(h, &h->Om, nl));
  TRY(dalloc(h, &h->Qa, nl));
  TRY(dalloc(h, &h->Qb, nl));
  TRY(dalloc(h, &h->U, nl));
  TRY(dalloc(h, &h->Qk, nl));
  TRY(dalloc(h, &h->Bk, nl));
  TRY(dalloc(h, &h->Mf, (size_t)L * 64));
  TRY(dalloc(h, &h->Sm_d, (size_t)L * L));
  TRY(dalloc(h, &h->V_d, (size_t)L * L));
  TRY(dalloc(h, &h->lam, (size_t)L));
  TRY(dalloc(h, &h->ev, (size_t)L));
  TRY(dalloc(h, &h->Sm_f, (size_t)L * L));
  TRY(dalloc(h, &h->Rl_f, (size_t)L * L));
  TRY(dalloc(h, &h->eng_ws, lai_engine_ws_bytes(L, h->k, OBJ_RING)));
  TRY(dalloc(h, &h->eng_G, (size_t)2 * h->k * h->k));
  TRY(dalloc(h, &h->eng_bar, 64));  // barrier counter of the CholeskyQR3 launch
  TRY(dalloc(h, &h->cq_part, cholqr_part_doubles(L)));
  TRY(dalloc(h, &h->cq_fin, (size_t)L * L));
  TRY(dalloc(h, &h->cq_Rf, (size_t)L * (L + 3)));
  TRY(dalloc(h, &h->cq_rinv, (size_t)L + 3));
  h->lai_cap = L;
  TRYS(ensure_gemm_ws(h, L));
  return SYMNMF_OK;
}

// Rank-safe orthonormalisation of S (n x l) in place, T scratch (n x l):
// shifted CholeskyQR3 (cholqr.cu), one cooperative launch unless the handle
// asks for separate kernels per step.  The range finder's intermediate bases
// only carry the span to the next product with X, so they stop after two
// passes (well conditioned, orthonormal to ~1e-4); the final basis, which
// Apx-EVD rotates into U, takes all three.
static symnmf_status orth(symnmf_t h, float* S, float* T, int l, bool final_basis) {
  TRY(cholqr3(S, T, h->n, l, h->cq_part, h->cq_fin, h->Sm_d, h->cq_Rf, h->cq_rinv, h->ws, h->counters + 0,
              h->eng_bar, h->err, h->o.lai_mode != 1, h->st, final_basis ? 3 : 2));
  return SYMNMF_OK;
}

// ||U Lambda U^T||_F^2 of the stored operator, for the trace-trick objective of
// the LAI sweeps: sum_ij lambda_i lambda_j (U^T U)_ij^2 with U^T U from the
// compensated cross product.  It equals sum lambda^2 for an exactly
// orthonormal U; the FP32 U is orthonormal only to rounding, and the
// objective's other terms use that U, so the norm must too.
static symnmf_status lai_operator_norm(symnmf_t h, int l) {
  TRY(xcross(h->U, l, l, h->U, l, l, h->n, nullptr, nullptr, nullptr, nullptr, 0.0, h->Sm_d, nullptr, h->ws,
             h->counters + 0, h->st));
  TRY(lai_norm2(h->Sm_d, h->lam, l, h->scal + S_LAI_NORM2, h->st));
  return SYMNMF_OK;
}

// Alg. Apx-EVD on the orthonormal basis in Qb (n x l): T = Q^T X Q, T = V Lambda V^T, U = Q V.
// Q and X Q are kept (Qk, Bk) for the compressed problem, with ||Q^T X||_F^2.
static symnmf_status apx_evd_from_basis(symnmf_t h, const float* Qb, float* Ts, int l) {
  (void)Ts;
  const int64_t n = h->n;
  TRYS(product(h, SYMNMF_SRC_X, Qb, l, l, h->Bk, l));
  TRY(cudaMemcpyAsync(h->Qk, Qb, (size_t)n * l * sizeof(float), cudaMemcpyDeviceToDevice, h->st));
  TRY(pair_reduce(h->Bk, h->Bk, n * l, h->scal + S_COMP_NORM2, h->ws, h->counters + 6, h->st));
  TRY(xcross(Qb, l, l, h->Bk, l, l, n, nullptr, nullptr, nullptr, nullptr, 0.0, h->Sm_d, nullptr, h->ws,
             h->counters + 0, h->st));
  TRY(jacobi_evd(h->Sm_d, l, h->V_d, h->lam, h->st));
  TRY(to_float_scaled(h->V_d, l, l, nullptr, h->Sm_f, h->st));
  TRY(apply_small(Qb, l, l, h->Sm_f, l, n, h->U, l, h->st));
  TRYS(lai_operator_norm(h, l));
  h->l = l;
  h->lai_ready = true;
  h->lai_from_user = false;
  h->lai_version++;
  return SYMNMF_OK;
}

static symnmf_status sketch_setup(symnmf_t h, int l, const float* omega) {
  if (l < h->k || l > h->o.max_width) return fail(h, SYMNMF_EINVAL, "need k <= l <= max_width");
  if (h->p.fmt == SYMNMF_X_CSR_F32 && l > 128) return SYMNMF_EINVAL;
  TRYS(ensure_lai(h, l));
  if (omega)
    TRY(cudaMemcpyAsync(h->Om, omega, (size_t)h->n * l * 4, cudaMemcpyDeviceToDevice, h->st));
  else
    TRY(philox_gaussian(h->Om, h->n, l, h->p.seed, h->st));
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_lai_sketch(symnmf_t h, int l, int q, const float* omega) {
  if (!h) return SYMNMF_EINVAL;
  if (q < 0) return fail(h, SYMNMF_EINVAL, "need q >= 0");
  TRYS(sketch_setup(h, l, omega));
  float* A = h->Qa;
  float* B = h->Qb;
  TRYS(product(h, SYMNMF_SRC_X, h->Om, l, l, A, l));  // Y = X Omega
  TRYS(orth(h, A, B, l, q == 0));
  for (int j = 0; j < q; ++j) {
    TRYS(product(h, SYMNMF_SRC_X, A, l, l, B, l));  // X^T Q (= X Q)
    TRYS(orth(h, B, A, l, false));
    TRYS(product(h, SYMNMF_SRC_X, B, l, l, A, l));  // X Q
    TRYS(orth(h, A, B, l, j == q - 1));
  }
  return apx_evd_from_basis(h, A, B, l);
}

extern "C" symnmf_status symnmf_lai_sketch_ada(symnmf_t h, int l, int q_max, double tol, const float* omega,
                                               int* checks_out, int* passes_out, double* nr_hist) {
  if (!h) return SYMNMF_EINVAL;
  if (q_max < 0) return fail(h, SYMNMF_EINVAL, "need q_max >= 0");
  TRYS(sketch_setup(h, l, omega));
  const int64_t n = h->n;
  float* Q = h->Qa;  // the current basis
  float* S = h->Qb;  // the other buffer
  // every basis whose residual is checked takes all three CholeskyQR passes
  // (orthonormal to FP32 rounding, which the ||X||^2 - ||B||^2 identity needs);
  // Q = orth(B^T) only carries the span to the next product unless it is final
  TRYS(product(h, SYMNMF_SRC_X, h->Om, l, l, Q, l));  // Y = X Omega
  TRYS(orth(h, Q, S, l, true));
  int passes = 1, checks = 0;
  double prev = 0.0;
  for (int j = 0; j < q_max; ++j) {
    TRYS(product(h, SYMNMF_SRC_X, Q, l, l, S, l));  // B^T = X^T Q (= X Q)
    ++passes;
    // ||Q B - X||_F^2 = ||X||_F^2 - ||B||_F^2: sum of squares of B^T in FP64
    TRY(pair_reduce(S, S, n * l, h->scal + S_ADA, h->ws, h->counters + 6, h->st));
    double bb[2], nx2 = 0.0;
    TRY(cudaMemcpyAsync(bb, h->scal + S_ADA, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    TRY(cudaMemcpyAsync(&nx2, h->scal + S_NORM2, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    TRYS(check_device_error(h));
    const double nr = sqrt(fmax(nx2 - bb[0], 0.0) / nx2);
    if (nr_hist) nr_hist[checks] = nr;
    ++checks;
    const bool stop = checks >= 2 && prev - nr < tol;
    prev = nr;
    TRYS(orth(h, S, Q, l, stop));  // Q = qr(B^T), now in S
    std::swap(Q, S);
    if (stop) break;
    TRYS(product(h, SYMNMF_SRC_X, Q, l, l, S, l));  // Y = X Q
    ++passes;
    TRYS(orth(h, S, Q, l, true));  // Q = qr(Y), now in S
    std::swap(Q, S);
  }
  if (checks_out) *checks_out = checks;
  if (passes_out) *passes_out = passes + 1;  // with the product for T
  return apx_evd_from_basis(h, Q, S, l);
}

extern "C" symnmf_status symnmf_set_lai(symnmf_t h, const float* U, const double* lam_host, int l) {
  if (!h || !U || !lam_host) return SYMNMF_EINVAL;
  if (l < h->k || l > h->o.max_width) return fail(h, SYMNMF_EINVAL, "need k <= l <= max_width");
  TRYS(ensure_lai(h, l));
  TRY(cudaMemcpyAsync(h->U, U, (size_t)h->n * l * sizeof(float), cudaMemcpyDeviceToDevice, h->st));
  TRY(cudaMemcpyAsync(h->lam, lam_host, (size_t)l * sizeof(double), cudaMemcpyHostToDevice, h->st));
  TRYS(lai_operator_norm(h, l));
  TRY(cudaStreamSynchronize(h->st));  // lam_host may be released on return
  h->l = l;
  h->lai_ready = true;
  h->lai_from_user = true;
  h->lai_version++;
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_get_lai(symnmf_t h, float* U_out, double* lam_out, int* l_out) {
  if (!h) return SYMNMF_EINVAL;
  if (!h->lai_ready) return fail(h, SYMNMF_ESTATE, "no sketch yet");
  if (U_out) TRY(cudaMemcpyAsync(U_out, h->U, (size_t)h->n * h->l * 4, cudaMemcpyDeviceToDevice, h->st));
  if (lam_out) {
    TRY(cudaMemcpyAsync(lam_out, h->lam, (size_t)h->l * 8, cudaMemcpyDeviceToHost, h->st));
    TRY(cudaStreamSynchronize(h->st));
  }
  if (l_out) *l_out = h->l;
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_sketch_features(symnmf_t h, float* out) {
  if (!h || !out) return SYMNMF_EINVAL;
  if (!h->lai_ready) return fail(h, SYMNMF_ESTATE, "no sketch yet");
  // X Omega of the fixed Omega, row-normalised (the warm-start network input)
  TRYS(product(h, SYMNMF_SRC_X, h->Om, h->l, h->l, h->Qb, h->l));
  TRY(normalize_rows(h->Qb, h->n, h->l, out, h->st));
  return SYMNMF_OK;
}

// ---------------------------------------------------------------- sweeps

static symnmf_status validate_sweep(symnmf_t h, int src, int rule) {
  if (src < 0 || src > 3) return fail(h, SYMNMF_EINVAL, "bad source");
  if ((src == SYMNMF_SRC_LAI || src == SYMNMF_SRC_COMP) && !h->lai_ready)
    return fail(h, SYMNMF_ESTATE, "LAI / compressed sweep before lai_sketch");
  if (src == SYMNMF_SRC_COMP && h->lai_from_user)
    return fail(h, SYMNMF_ESTATE, "the compressed problem needs a sketch, not set_lai");
  if (src == SYMNMF_SRC_XHI && !h->p.x_hi) return fail(h, SYMNMF_ESTATE, "no float32 copy of X given");
  if (rule == SYMNMF_RULE_BPP && h->k > 16) return fail(h, SYMNMF_EUNSUPPORTED, "BPP rule needs k <= 16");
  if (rule != SYMNMF_RULE_HALS && rule != SYMNMF_RULE_BPP) return fail(h, SYMNMF_EINVAL, "bad rule");
  return SYMNMF_OK;
}

// A captured sweep graph for (src, rule) at the current sketch, or nullptr.
static symnmf_ctx::Graph* cached_graph(symnmf_t h, int src, int rule) {
  for (auto& g : h->graphs)
    if (g.exec && g.src == src && g.rule == rule && g.lai_version == h->lai_version) return &g;
  return nullptr;
}

// Capturing and instantiating a graph costs about as much as a few eager
// sweeps: a new graph is made only when at least this many replays follow.
constexpr int GRAPH_MIN_REPLAYS = 4;

static symnmf_status get_graph(symnmf_t h, int src, int rule, symnmf_ctx::Graph** out) {
  for (auto& g : h->graphs)
    if (g.exec && g.src == src && g.rule == rule && g.lai_version == h->lai_version) {
      *out = &g;
      return SYMNMF_OK;
    }
  // one eager sweep first sizes every workspace, so capture allocates nothing
  symnmf_ctx::Graph* slot = nullptr;
  for (auto& g : h->graphs)
    if (!g.exec) {
      slot = &g;
      break;
    }
  if (!slot) {
    slot = &h->graphs[0];
    cudaGraphExecDestroy(slot->exec);
    slot->exec = nullptr;
  }
  // record on a private stream (the caller's stream may be the legacy NULL
  // stream, which cannot be captured); the graph is launched on the caller's
  if (!h->cap_st) TRY(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
  cudaGraph_t graph;
  cudaStream_t saved = h->st;
  h->st = h->cap_st;
  cudaError_t eb = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal);
  if (eb != cudaSuccess) {
    h->st = saved;
    return cuda_fail(h, eb, "cudaStreamBeginCapture");
  }
  h->capturing = true;
  const uint64_t before = g_launches.load();
  symnmf_status s = sweep_body(h, src, rule);
  h->capturing = false;
  cudaError_t e = cudaStreamEndCapture(h->st, &graph);
  h->st = saved;
  if (s != SYMNMF_OK) {
    if (e == cudaSuccess) cudaGraphDestroy(graph);
    return s;
  }
  TRY(e);
  cudaError_t ei = cudaGraphInstantiate(&slot->exec, graph, 0);
  cudaGraphDestroy(graph);
  TRY(ei);
  slot->nkernels = g_launches.load() - before;
  g_launches -= slot->nkernels;  // captured, not launched
  slot->src = src;
  slot->rule = rule;
  slot->lai_version = h->lai_version;
  *out = slot;
  return SYMNMF_OK;
}

// LAI-HALS sweeps in one cooperative launch per chunk of sweeps.
static symnmf_status lai_engine_sweeps(symnmf_t h, int nsweeps, double* obj_host) {
  const int k = h->k;
  int done = 0;
  while (done < nsweeps) {
    const int chunk = (nsweeps - done) < OBJ_RING ? (nsweeps - done) : OBJ_RING;
    // resume from the engine's saved state when nothing else touched W, H or the operator
    const bool resume = h->eng_resume_ok && h->eng_fac_version == h->fac_version &&
                        h->eng_lai_version == h->lai_version;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->profiling && !h->capturing) {
      if (h->eprof_used == h->eprof_events.size()) {
        cudaEvent_t a, b;
        TRY(cudaEventCreate(&a));
        TRY(cudaEventCreate(&b));
        h->eprof_events.push_back({a, b});
        h->eprof_flops.push_back(0.0);
      }
      e0 = h->eprof_events[h->eprof_used].first;
      e1 = h->eprof_events[h->eprof_used].second;
      h->eprof_flops[h->eprof_used] = lai_engine_flops(h->n, k, h->l, chunk, !resume);
      h->eprof_used++;
    }
    TRY(lai_engine(h->U, h->lam, h->W, h->H, h->n, k, h->l, chunk, h->alpha, h->scal + S_LAI_NORM2, h->eng_ws,
                   h->obj_ring, OBJ_RING, h->eng_G, h->err, h->o.lai_mode != 2, h->st, e0, e1, resume, h->Gd[0],
                   h->Gd[1], h->Gf[0], h->Gf[1]));
    h->eng_resume_ok = true;
    h->eng_fac_version = h->fac_version;
    h->eng_lai_version = h->lai_version;
    if (obj_host) {
      TRY(cudaMemcpyAsync(obj_host + done, h->obj_ring, (size_t)chunk * sizeof(double), cudaMemcpyDeviceToHost,
                          h->st));
      TRYS(check_device_error(h));
      TRYS(check_objectives(h, obj_host + done, chunk));
    }
    done += chunk;
  }
  if (nsweeps > 0) h->grams_fresh = true;  // the engine wrote the handle's Grams of its final factors
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_hals_sweep(symnmf_t h, int nsweeps, int source, int rule, double* obj_host) {
  if (!h || nsweeps < 0) return SYMNMF_EINVAL;
  TRYS(validate_sweep(h, source, rule));
  if (source == SYMNMF_SRC_LAI && rule == SYMNMF_RULE_HALS && h->o.lai_mode != 1)
    return lai_engine_sweeps(h, nsweeps, obj_host);
  int done = 0;
  bool warmed = false;
  while (done < nsweeps) {
    const int chunk = (nsweeps - done) < OBJ_RING ? (nsweeps - done) : OBJ_RING;
    TRY(cudaMemsetAsync(h->obj_cnt, 0, sizeof(int), h->st));
    int t = 0;
    if (h->o.use_graph && (chunk >= 1 + GRAPH_MIN_REPLAYS || cached_graph(h, source, rule))) {
      if (!warmed) {
        // first sweep eagerly: workspaces get sized outside capture
        TRYS(sweep_body(h, source, rule));
        ++t;
        warmed = true;
      }
      symnmf_ctx::Graph* g = nullptr;
      if (t < chunk) TRYS(get_graph(h, source, rule, &g));
      for (; t < chunk; ++t) {
        TRY(cudaGraphLaunch(g->exec, h->st));
        count_launches(g->nkernels);
      }
    } else {
      for (; t < chunk; ++t) TRYS(sweep_body(h, source, rule));
    }
    if (obj_host) {
      TRY(cudaMemcpyAsync(obj_host + done, h->obj_ring, (size_t)chunk * sizeof(double),
                          cudaMemcpyDeviceToHost, h->st));
      TRYS(check_device_error(h));
      TRYS(check_objectives(h, obj_host + done, chunk));
    }
    done += chunk;
  }
  return SYMNMF_OK;
}

// ---------------------------------------------------------------- LvS

static symnmf_status ensure_sampler(symnmf_t h, int s) {
  const int cap = (int)((h->n > s ? h->n : s));
  if (h->sb.cap >= cap) return SYMNMF_OK;
  SampleBufs& b = h->sb;
  const int nblk = sampler_blocks(h->n);
  TRY(dalloc(h, &b.lev, (size_t)h->n));
  TRY(dalloc(h, &b.cdf, (size_t)h->n));
  TRY(dalloc(h, &b.idx, (size_t)cap));
  TRY(dalloc(h, &b.wt, (size_t)cap));
  TRY(dalloc(h, &b.counts, 4));
  TRY(dalloc(h, &b.sums, 4));
  TRY(dalloc(h, &b.total, 1));
  TRY(dalloc(h, &b.blk_cnt, (size_t)nblk));
  TRY(dalloc(h, &b.blk_q, (size_t)nblk));
  TRY(dalloc(h, &b.blk_theta, (size_t)nblk));
  TRY(dalloc(h, &b.blk_mass, (size_t)nblk));
  b.nblk_cap = nblk;
  b.cap = cap;
  return SYMNMF_OK;
}

// Leverage scores of the fixed factor of `side` into sb.lev.
static symnmf_status leverage_dev(symnmf_t h, int side) {
  const float* F = side ? h->W : h->H;
  const int k = h->k;
  TRY(xcross(F, k, k, F, k, k, h->n, nullptr, nullptr, nullptr, nullptr, 0.0, h->Gs_d, nullptr, h->ws,
             h->counters + 4, h->st));
  TRY(chol_inverse(h->Gs_d, k, 0.0, 0.0, h->Rinv_d, h->Rinv_f, h->err, h->st));
  TRY(leverage_rows(F, h->n, k, h->Rinv_f, h->sb.lev, h->st));
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_leverage(symnmf_t h, int side, double* lev_out) {
  if (!h || (side != 0 && side != 1)) return SYMNMF_EINVAL;
  TRYS(ensure_sampler(h, 0));
  TRYS(leverage_dev(h, side));
  if (lev_out) TRY(cudaMemcpyAsync(lev_out, h->sb.lev, (size_t)h->n * 8, cudaMemcpyDeviceToDevice, h->st));
  return check_device_error(h);
}

static symnmf_status sample_dev(symnmf_t h, int side, int iter, double tau, int s) {
  TRY(hybrid_sample(h->sb, h->n, h->k, tau, s, h->p.seed, (uint32_t)iter, (uint32_t)side, h->st));
  h->sample_side = side;
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_lvs_sample(symnmf_t h, int side, int iter, double tau, int s,
                                           const double* lev_in, int32_t* idx_out, float* wt_out, int cap,
                                           int* s_det, int* s_tot, double* theta) {
  if (!h || (side != 0 && side != 1) || s < 0 || !(tau >= 0.0)) return SYMNMF_EINVAL;
  TRYS(ensure_sampler(h, s));
  if (lev_in)
    TRY(cudaMemcpyAsync(h->sb.lev, lev_in, (size_t)h->n * 8, cudaMemcpyHostToDevice, h->st));
  else
    TRYS(leverage_dev(h, side));
  TRYS(sample_dev(h, side, iter, tau, s));
  int counts[4];
  double sums[4];
  TRY(cudaMemcpyAsync(counts, h->sb.counts, 3 * sizeof(int), cudaMemcpyDeviceToHost, h->st));
  TRY(cudaMemcpyAsync(sums, h->sb.sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  TRYS(check_device_error(h));
  const int tot = counts[2];
  const int m = cap < tot ? cap : tot;
  if (idx_out && m > 0) TRY(cudaMemcpy(idx_out, h->sb.idx, (size_t)m * 4, cudaMemcpyDeviceToHost));
  if (wt_out && m > 0) TRY(cudaMemcpy(wt_out, h->sb.wt, (size_t)m * 4, cudaMemcpyDeviceToHost));
  if (s_det) *s_det = counts[0];
  if (s_tot) *s_tot = tot;
  if (theta) *theta = sums[0];
  return SYMNMF_OK;
}

static symnmf_status lvs_update_dev(symnmf_t h, int side, int rule, cudaEvent_t ev_products = nullptr) {
  h->fac_version++;
  h->grams_fresh = false;
  const int k = h->k;
  const int64_t n = h->n;
  const float* Ff = side ? h->W : h->H;
  float* Fu = side ? h->H : h->W;
  // Y = X S^T S F (the HALS / BPP kernels add alpha F themselves)
  TRY(cudaMemsetAsync(h->Y, 0, (size_t)n * k * 4, h->st));
  if (h->p.fmt == SYMNMF_X_CSR_F32)
    TRY(csr_sampled_xf(h->p.row_ptr, h->p.col, (const float*)h->p.x, h->sb.idx, h->sb.wt, h->sb.counts + 2,
                       Ff, k, h->Y, h->st));
  else
    TRY(dense_sampled_xf(h->p.fmt, h->p.x, h->ldx, n, h->sb.idx, h->sb.wt, h->sb.counts + 2, h->sb.cap, Ff,
                         k, h->Y, h->st));
  // G = F^T S^T S F
  TRY(xcross(Ff, k, k, Ff, k, k, h->sb.cap, h->sb.idx, h->sb.wt, h->sb.counts + 2, nullptr, 0.0, h->Gs_d,
             h->Gs_f, h->ws, h->counters + 5, h->st));
  if (ev_products) TRY(cudaEventRecord(ev_products, h->st));
  if (rule == SYMNMF_RULE_HALS)
    TRY(hals_update(Fu, Ff, n, k, h->Gs_f, h->alpha, h->Y, k, nullptr, 0, nullptr, h->scal + S_PART,
                    h->ws, h->counters + 1, h->err, h->st));
  else
    TRY(bpp_rows(Fu, Ff, n, k, h->Gs_d, h->alpha, h->Y, k, nullptr, 0, nullptr, h->scal + S_PART, h->ws,
                 h->counters + 1, h->err, h->st));
  return SYMNMF_OK;
}

static symnmf_status check_lvs(symnmf_t h, int rule) {
  if (h->p.fmt == SYMNMF_X_DENSE_FP8)
    return fail(h, SYMNMF_EUNSUPPORTED, "LvS needs CSR or dense F32/F64/BF16 X");
  if (rule == SYMNMF_RULE_BPP && h->k > 16) return fail(h, SYMNMF_EUNSUPPORTED, "BPP rule needs k <= 16");
  if (h->p.fmt != SYMNMF_X_CSR_F32 && h->k > 64) return SYMNMF_EUNSUPPORTED;
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_lvs_update(symnmf_t h, int side, int rule) {
  if (!h || (side != 0 && side != 1)) return SYMNMF_EINVAL;
  TRYS(check_lvs(h, rule));
  if (h->sample_side != side) return fail(h, SYMNMF_ESTATE, "lvs_update without a sample of that side");
  TRYS(lvs_update_dev(h, side, rule));
  return SYMNMF_OK;
}

// While profiling, the next LvS half's four events (before the leverage
// scores, after the sample, after the sampled products, after the update).
static symnmf_status lvs_events(symnmf_t h, cudaEvent_t* ev) {
  if (!h->profiling || h->capturing) {
    ev[0] = ev[1] = ev[2] = ev[3] = nullptr;
    return SYMNMF_OK;
  }
  while (h->lprof_events.size() < 4 * (h->lprof_used + 1)) {
    cudaEvent_t e;
    TRY(cudaEventCreate(&e));
    h->lprof_events.push_back(e);
  }
  for (int i = 0; i < 4; ++i) ev[i] = h->lprof_events[4 * h->lprof_used + i];
  h->lprof_used++;
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_lvs_iterate(symnmf_t h, int iter0, int iters, double tau, int s, int rule) {
  if (!h || iters < 0 || s < 0) return SYMNMF_EINVAL;
  TRYS(check_lvs(h, rule));
  TRYS(ensure_sampler(h, s));
  for (int it = iter0; it < iter0 + iters; ++it) {
    for (int side = 0; side < 2; ++side) {
      cudaEvent_t ev[4];
      TRYS(lvs_events(h, ev));
      if (ev[0]) TRY(cudaEventRecord(ev[0], h->st));
      TRYS(leverage_dev(h, side));
      TRYS(sample_dev(h, side, it, tau, s));
      if (ev[1]) TRY(cudaEventRecord(ev[1], h->st));
      TRYS(lvs_update_dev(h, side, rule, ev[2]));
      if (ev[3]) TRY(cudaEventRecord(ev[3], h->st));
    }
  }
  TRYS(refresh_grams(h));
  return SYMNMF_OK;
}

// ----------------------------------------------------------------- PGNCG

static symnmf_status ensure_pgncg(symnmf_t h) {
  if (h->cgR) return SYMNMF_OK;
  const size_t nk = (size_t)h->n * h->k;
  TRY(dalloc(h, &h->cgR, nk));
  TRY(dalloc(h, &h->cgP, nk));
  TRY(dalloc(h, &h->cgZ, nk));
  TRY(dalloc(h, &h->cgY, nk));
  TRY(dalloc(h, &h->cgPtH, (size_t)h->k * h->k));
  TRY(dalloc(h, &h->cgPtH_d, (size_t)h->k * h->k));
  TRY(dalloc(h, &h->cg_ws, gn_ws_doubles()));
  return SYMNMF_OK;
}

// Y (n x k) = X F for `source` (the LAI operator as U (Lambda (U^T F))).
static symnmf_status apply_source(symnmf_t h, int source, const float* F, float* Yo) {
  const int k = h->k;
  if (source == SYMNMF_SRC_LAI) {
    TRY(xcross(h->U, h->l, h->l, F, k, k, h->n, nullptr, nullptr, nullptr, h->lam, 0.0, nullptr, h->Mf, h->ws,
               h->counters + 0, h->st));
    TRY(apply_small(h->U, h->l, h->l, h->Mf, k, h->n, Yo, k, h->st));
    return SYMNMF_OK;
  }
  return product(h, source, F, k, k, Yo, k);
}

// Y = X H and G = H^T H (FP64 Gd[0], FP32 Gf[0]); with `record`, the SymNMF
// objective of H appended to the objective ring.
static symnmf_status gn_products(symnmf_t h, int source, bool record) {
  const int k = h->k;
  TRYS(apply_source(h, source, h->H, h->Y));
  TRY(xcross(h->H, k, k, h->H, k, k, h->n, nullptr, nullptr, nullptr, nullptr, 0.0, h->Gd[0], h->Gf[0], h->ws,
             h->counters + 2, h->st));
  if (record) {
    TRY(pair_reduce(h->H, h->Y, h->n * k, h->scal + S_PART2, h->ws, h->counters + 6, h->st));
    TRY(gn_objective(normx_for(h, source), h->Gd[0], k, h->scal + S_PART2, h->obj_ring, h->obj_cnt, OBJ_RING,
                     h->st));
  }
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_pgncg(symnmf_t h, int iters, int source, int s_max, double* obj_host) {
  if (!h || iters < 0 || s_max < 1 || s_max > 1000 || source == SYMNMF_SRC_COMP) return SYMNMF_EINVAL;
  TRYS(validate_sweep(h, source, SYMNMF_RULE_HALS));
  if (iters > OBJ_RING) return fail(h, SYMNMF_EINVAL, "at most 4096 iterations per call");
  TRYS(ensure_pgncg(h));
  const int k = h->k;
  const int64_t nk = h->n * k;
  double* cg = h->scal + S_CG;
  TRY(cudaMemsetAsync(h->obj_cnt, 0, sizeof(int), h->st));
  for (int t = 0; t < iters; ++t) {
    // the objective of the previous iterate comes with this iteration's product
    TRYS(gn_products(h, source, obj_host != nullptr && t > 0));
    TRY(gn_grad(h->H, h->Y, h->Gf[0], h->n, k, h->cgR, h->cgP, h->cgZ, h->cg_ws, h->counters + 7, cg, h->st));
    for (int s = 0; s < s_max; ++s) {
      TRY(xcross(h->cgP, k, k, h->H, k, k, h->n, nullptr, nullptr, nullptr, nullptr, 0.0, h->cgPtH_d, h->cgPtH,
                 h->ws, h->counters + 2, h->st));
      TRY(gn_hvp(h->H, h->cgP, h->Gf[0], h->cgPtH, h->n, k, h->cgY, h->cg_ws, h->counters + 7, cg, h->st));
      TRY(gn_update(h->cgP, h->cgY, nk, h->cgR, h->cgZ, h->cg_ws, h->counters + 7, cg, h->st));
      if (s + 1 < s_max) TRY(gn_dir(h->cgR, nk, h->cgP, cg, h->st));
    }
    h->fac_version++;
    h->grams_fresh = false;
    TRY(gn_project(h->cgZ, nk, h->H, h->W, h->err, h->st));
  }
  if (obj_host && iters > 0) {
    TRYS(gn_products(h, source, true));  // the last iterate's objective
    TRY(cudaMemcpyAsync(obj_host, h->obj_ring, (size_t)iters * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    TRYS(check_device_error(h));
    TRYS(check_objectives(h, obj_host, iters));
  }
  TRYS(refresh_grams(h));
  return SYMNMF_OK;
}

// ------------------------------------------------------------ schedule

// One iteration on `src` (a sweep, or a PGNCG iteration), returning the
// normalized residual of that operator from the recorded objective.
static symnmf_status schedule_step(symnmf_t h, const symnmf_schedule* sc, int src, double* nr) {
  double obj = 0.0;
  if (sc->algo == 1)
    TRYS(symnmf_pgncg(h, 1, src, sc->s_max, &obj));
  else
    TRYS(symnmf_hals_sweep(h, 1, src, sc->rule, &obj));
  double nx2 = 0.0;
  TRY(cudaMemcpy(&nx2, normx_for(h, src), sizeof(double), cudaMemcpyDeviceToHost));
  *nr = sqrt(fmax(obj, 0.0) / nx2);
  return SYMNMF_OK;
}

// Iterations on `src` until the residual has fallen by less than stop_tol in
// stop_count consecutive iterations, or `cap`.  Returns the iterations run.
static symnmf_status schedule_phase(symnmf_t h, const symnmf_schedule* sc, int src, int cap, int* iters,
                                    double* nr_last) {
  double prev = 0.0, nr = 0.0;
  int small = 0, t = 0;
  while (t < cap) {
    TRYS(schedule_step(h, sc, src, &nr));
    ++t;
    if (t > 1) small = (prev - nr < sc->stop_tol) ? small + 1 : 0;
    prev = nr;
    if (small >= sc->stop_count) break;
  }
  *iters = t;
  *nr_last = nr;
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_solve(symnmf_t h, const symnmf_schedule* sc, symnmf_report* rep) {
  if (!h || !sc) return SYMNMF_EINVAL;
  const int m = sc->method;
  if (m != SYMNMF_SRC_X && m != SYMNMF_SRC_LAI && m != SYMNMF_SRC_COMP) return fail(h, SYMNMF_EINVAL, "method");
  if (sc->algo == 1 && m == SYMNMF_SRC_COMP) return fail(h, SYMNMF_EINVAL, "PGNCG with X or LAI");
  if (sc->stop_count < 1 || sc->max_iters < 0 || sc->max_refine < 0 || sc->q_max < 0)
    return fail(h, SYMNMF_EINVAL, "schedule limits");
  symnmf_report r{};
  if (m != SYMNMF_SRC_X)
    TRYS(symnmf_lai_sketch_ada(h, sc->l, sc->q_max, sc->ada_tol, nullptr, &r.checks, &r.passes, nullptr));
  TRYS(schedule_phase(h, sc, m, sc->max_iters, &r.iters, &r.nr_phase));
  const int truth = h->p.x_hi ? SYMNMF_SRC_XHI : SYMNMF_SRC_X;
  if (sc->refine && m != SYMNMF_SRC_X) {
    double nr_ir = 0.0;
    TRYS(schedule_phase(h, sc, truth, sc->max_refine, &r.refine_iters, &nr_ir));
  }
  // PGNCG keeps W = H, so this is ||X - H H^T|| / ||X|| for it
  TRYS(symnmf_residual(h, truth, &r.nr_final, nullptr, nullptr));
  if (rep) *rep = r;
  return SYMNMF_OK;
}

// -------------------------------------------------------------- residual

// Y = X F for the operator `source` (X, its float32 copy, or the LAI).
static symnmf_status apply_operator(symnmf_t h, int source, const float* F, float* Yo) {
  const int k = h->k;
  if (source == SYMNMF_SRC_LAI) {
    TRY(xcross(h->U, h->l, h->l, F, k, k, h->n, nullptr, nullptr, nullptr, h->lam, 0.0, nullptr, h->Mf, h->ws,
               h->counters + 0, h->st));
    TRY(apply_small(h->U, h->l, h->l, h->Mf, k, h->n, Yo, k, h->st));
    return SYMNMF_OK;
  }
  return product(h, source, F, k, k, Yo, k);
}

// The device part of a residual evaluation (Grams current): scal[S_OBJ] =
// ||X - W H^T||^2 by the trace trick, scal[S_RES + 1] = ||W - H||^2.  No sync.
static symnmf_status residual_dev(symnmf_t h, int source) {
  const int k = h->k;
  TRYS(apply_operator(h, source, h->H, h->Y));  // Y = X H
  // (sum W .* XH, ||W - H||^2) in one pass
  TRY(resid_reduce(h->W, h->H, h->Y, h->n * k, h->scal + S_RES, h->ws, h->counters + 6, h->st));
  TRY(objective(normx_for(h, source), h->Gd[1], h->Gd[0], k, h->scal + S_RES, h->scal + S_ZERO,
                h->scal + S_OBJ, nullptr, 0, h->st));
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_residual(symnmf_t h, int source, double* norm_resid, double* surrogate,
                                         double* proj_grad) {
  if (!h) return SYMNMF_EINVAL;
  if (source == SYMNMF_SRC_COMP) return fail(h, SYMNMF_EINVAL, "residual of X, the LAI or the float32 copy");
  TRYS(validate_sweep(h, source, SYMNMF_RULE_HALS));
  const int k = h->k;
  const int64_t n = h->n;
  if (!h->grams_fresh) TRYS(refresh_grams(h));
  auto apply_op = [&](const float* F, float* Yo) -> symnmf_status { return apply_operator(h, source, F, Yo); };
  TRYS(residual_dev(h, source));
  double pg2 = 0.0;
  if (proj_grad) {
    TRY(cudaMemsetAsync(h->scal + S_PG, 0, sizeof(double), h->st));
    TRY(proj_grad_sq(h->W, h->H, h->Y, h->Gf[0], n, k, h->scal + S_ALPHA, h->scal + S_PG, h->st));
    TRYS(apply_op(h->W, h->Y));  // Y = X W
    TRY(proj_grad_sq(h->H, h->W, h->Y, h->Gf[1], n, k, h->scal + S_ALPHA, h->scal + S_PG, h->st));
  }
  double hs[S_COUNT];
  TRY(cudaMemcpyAsync(hs, h->scal, sizeof(hs), cudaMemcpyDeviceToHost, h->st));
  TRYS(check_device_error(h));
  const double r2 = hs[S_OBJ];
  const double nx2 = source == SYMNMF_SRC_LAI ? hs[S_LAI_NORM2]
                     : source == SYMNMF_SRC_XHI ? hs[S_XHI_NORM2]
                                                : hs[S_NORM2];
  pg2 = hs[S_PG];
  if (norm_resid) *norm_resid = sqrt(fmax(r2, 0.0) / nx2);
  if (surrogate) *surrogate = r2 + h->alpha * hs[S_RES + 1];
  if (proj_grad) *proj_grad = sqrt(pg2);
  return SYMNMF_OK;
}

// ------------------------------------------------ sweeps to a residual target

// One residual check's decision: NR = sqrt(max(r2, 0) / ||X||^2) into the log,
// one more check counted, and the loop continues while NR > target and fewer
// than max_checks checks were made (a NaN NR stops it).  With a handle, the
// decision also sets the enclosing WHILE node's condition.
__global__ void loop_decide_kernel(const double* r2, const double* nx2, double target, int max_checks, int* li,
                                   double* nr_log, cudaGraphConditionalHandle cond, int use_cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int c = li[0];
  const double nr = sqrt(fmax(*r2, 0.0) / *nx2);
  if (c < LOOP_MAX) nr_log[c] = nr;
  li[0] = c + 1;
  const unsigned go = (nr > target && c + 1 < max_checks) ? 1u : 0u;
  li[1] = (int)go;
  if (use_cond) cudaGraphSetConditional(cond, go);
}

// The WHILE node's condition from the first check's decision.
__global__ void loop_seed_kernel(const int* li, cudaGraphConditionalHandle cond) {
  if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(cond, li[1] ? 1u : 0u);
}

// One pass of the loop body: `chunk` LAI sweeps in one engine launch resumed
// from the previous launch's state, the Grams, the residual of `check`, the
// decision.
static symnmf_status loop_body(symnmf_t h, int check, int chunk, double target, int max_checks,
                               cudaGraphConditionalHandle cond) {
  TRY(lai_engine(h->U, h->lam, h->W, h->H, h->n, h->k, h->l, chunk, h->alpha, h->scal + S_LAI_NORM2, h->eng_ws,
                 h->obj_ring, OBJ_RING, h->eng_G, h->err, h->o.lai_mode != 2, h->st, nullptr, nullptr, true,
                 h->Gd[0], h->Gd[1], h->Gf[0], h->Gf[1]));
  TRYS(residual_dev(h, check));
  loop_decide_kernel<<<1, 32, 0, h->st>>>(h->scal + S_OBJ, normx_for(h, check), target, max_checks, h->loop_i,
                                          h->loop_nr, cond, 1);
  count_launches(1);
  return SYMNMF_OK;
}

// The loop graph for these parameters: [seed] -> WHILE(cond) { loop_body }.
// Recorded on the private stream; everything it touches was sized by the
// eager first pass, so recording allocates nothing.
static symnmf_status get_loop_graph(symnmf_t h, int check, int chunk, double target, int max_checks) {
  const void* bufs[5] = {h->U, h->eng_ws, h->fpack, h->gemm_ws, h->loop_i};
  auto& L = h->loop;
  if (L.exec && L.check == check && L.chunk == chunk && L.max_checks == max_checks && L.l == h->l &&
      L.target == target && std::equal(bufs, bufs + 5, L.bufs))
    return SYMNMF_OK;
  if (L.exec) {
    cudaGraphExecDestroy(L.exec);  // one instantiation of a graph with a conditional node at a time
    L.exec = nullptr;
  }
  if (!h->cap_st) TRY(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  TRY(cudaGraphCreate(&g, 0));
  cudaStream_t saved = h->st;
  h->st = h->cap_st;
  uint64_t body_kernels = 0;
  auto record = [&]() -> symnmf_status {
    cudaGraphConditionalHandle cond;
    TRY(cudaGraphConditionalHandleCreate(&cond, g, 0, 0));
    TRY(cudaStreamBeginCaptureToGraph(h->st, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    loop_seed_kernel<<<1, 32, 0, h->st>>>(h->loop_i, cond);
    cudaError_t e = cudaGetLastError();
    cudaGraph_t got = nullptr;
    cudaError_t ee = cudaStreamEndCapture(h->st, &got);
    TRY(e);
    TRY(ee);
    cudaGraphNode_t seed = nullptr;
    size_t nn = 1;
    TRY(cudaGraphGetNodes(g, &seed, &nn));
    if (nn != 1) return fail(h, SYMNMF_ECUDA, "loop graph: expected one seed node");
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    TRY(cudaGraphAddNode(&node, g, &seed, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    TRY(cudaStreamBeginCaptureToGraph(h->st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    const uint64_t before = g_launches.load();
    symnmf_status s = loop_body(h, check, chunk, target, max_checks, cond);
    h->capturing = false;
    body_kernels = g_launches.load() - before;
    g_launches -= body_kernels;  // recorded, not launched
    ee = cudaStreamEndCapture(h->st, &got);
    if (s != SYMNMF_OK) return s;
    TRY(ee);
    TRY(cudaGraphInstantiate(&L.exec, g, 0));
    return SYMNMF_OK;
  };
  symnmf_status s = record();
  h->st = saved;
  h->capturing = false;
  cudaGraphDestroy(g);
  if (s != SYMNMF_OK) {
    cudaGetLastError();
    L.exec = nullptr;
    return s;
  }
  L.check = check;
  L.chunk = chunk;
  L.max_checks = max_checks;
  L.l = h->l;
  L.target = target;
  std::copy(bufs, bufs + 5, L.bufs);
  L.nkernels = body_kernels;
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_sweep_to_target(symnmf_t h, int source, int check, int chunk, int max_sweeps,
                                                double target, int* sweeps_out, int* checks_out, double* nr_out) {
  if (!h || chunk < 1 || max_sweeps < 1 || !(target == target)) return SYMNMF_EINVAL;
  if (check == SYMNMF_SRC_COMP) return fail(h, SYMNMF_EINVAL, "residual of X, the LAI or the float32 copy");
  TRYS(validate_sweep(h, source, SYMNMF_RULE_HALS));
  TRYS(validate_sweep(h, check, SYMNMF_RULE_HALS));
  const int max_checks = (max_sweeps + chunk - 1) / chunk;
  if (max_checks > LOOP_MAX) return fail(h, SYMNMF_EINVAL, "more residual checks than the loop records");
  if (!h->loop_i) {
    TRY(dalloc(h, &h->loop_i, 2));
    TRY(dalloc(h, &h->loop_nr, (size_t)LOOP_MAX));
  }
  TRY(cudaMemsetAsync(h->loop_i, 0, 2 * sizeof(int), h->st));
  const bool engine = source == SYMNMF_SRC_LAI && h->o.lai_mode != 1 && chunk <= OBJ_RING;
  // the device loop needs whole chunks and is recorded once a call repeats
  // the previous call's parameters; otherwise (and for the other sweep
  // kernels) the host checks after each chunk
  auto& L = h->loop;
  const bool repeat = L.prev_check == check && L.prev_chunk == chunk && L.prev_max_checks == max_checks &&
                      L.prev_l == h->l && L.prev_target == target;
  L.prev_check = check;
  L.prev_chunk = chunk;
  L.prev_max_checks = max_checks;
  L.prev_l = h->l;
  L.prev_target = target;
  const bool device_loop = engine && h->o.use_graph && max_sweeps % chunk == 0 && max_checks > 1 && repeat;
  int checks = 0;
  if (device_loop) {
    // first pass eagerly: the engine's prologue, and every workspace sized
    TRYS(lai_engine_sweeps(h, chunk, nullptr));
    TRYS(residual_dev(h, check));
    loop_decide_kernel<<<1, 32, 0, h->st>>>(h->scal + S_OBJ, normx_for(h, check), target, max_checks, h->loop_i,
                                            h->loop_nr, 0, 0);
    count_launches(1);
    TRY(cudaGetLastError());
    TRYS(get_loop_graph(h, check, chunk, target, max_checks));
    TRY(cudaGraphLaunch(L.exec, h->st));
    int li[2] = {0, 0};
    TRY(cudaMemcpyAsync(li, h->loop_i, sizeof(li), cudaMemcpyDeviceToHost, h->st));
    TRYS(check_device_error(h));
    checks = li[0];
    count_launches(1 + (uint64_t)(checks - 1) * L.nkernels);
  } else {
    int done = 0;
    while (done < max_sweeps) {
      const int m = (max_sweeps - done) < chunk ? (max_sweeps - done) : chunk;
      TRYS(symnmf_hals_sweep(h, m, source, SYMNMF_RULE_HALS, nullptr));
      done += m;
      if (!h->grams_fresh) TRYS(refresh_grams(h));
      TRYS(residual_dev(h, check));
      loop_decide_kernel<<<1, 32, 0, h->st>>>(h->scal + S_OBJ, normx_for(h, check), target, max_checks,
                                              h->loop_i, h->loop_nr, 0, 0);
      count_launches(1);
      int li[2] = {0, 0};
      TRY(cudaMemcpyAsync(li, h->loop_i, sizeof(li), cudaMemcpyDeviceToHost, h->st));
      TRYS(check_device_error(h));
      checks = li[0];
      if (!li[1]) break;
    }
  }
  if (checks < 1 || checks > max_checks) return fail(h, SYMNMF_ECUDA, "residual check loop count");
  double nr = 0.0;
  TRY(cudaMemcpy(&nr, h->loop_nr + (checks - 1), sizeof(double), cudaMemcpyDeviceToHost));
  if (sweeps_out) *sweeps_out = checks * chunk < max_sweeps ? checks * chunk : max_sweeps;
  if (checks_out) *checks_out = checks;
  if (nr_out) *nr_out = nr;
  return SYMNMF_OK;
}

// ------------------------------------------------------- standalone kernels

// Process-wide event timing of standalone tensor-core products (symnmf_dense_xf).
namespace {
std::mutex g_sprof_mu;
bool g_sprof_on = false;
size_t g_sprof_used = 0;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_sprof_ev;
std::vector<double> g_sprof_flops, g_sprof_bytes;
}  // namespace

// Events for the next standalone product when profiling is on (nullptr otherwise).
static cudaError_t standalone_events(cudaEvent_t* e0, cudaEvent_t* e1, double flops, double bytes) {
  std::lock_guard<std::mutex> lock(g_sprof_mu);
  *e0 = *e1 = nullptr;
  if (!g_sprof_on) return cudaSuccess;
  if (g_sprof_used == g_sprof_ev.size()) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&b)) != cudaSuccess) return e;
    g_sprof_ev.push_back({a, b});
    g_sprof_flops.push_back(0.0);
    g_sprof_bytes.push_back(0.0);
  }
  *e0 = g_sprof_ev[g_sprof_used].first;
  *e1 = g_sprof_ev[g_sprof_used].second;
  g_sprof_flops[g_sprof_used] = flops;
  g_sprof_bytes[g_sprof_used] = bytes;
  g_sprof_used++;
  return cudaSuccess;
}

extern "C" symnmf_status symnmf_profile_standalone(int enable) {
  std::lock_guard<std::mutex> lock(g_sprof_mu);
  g_sprof_on = enable != 0;
  g_sprof_used = 0;
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_profile_standalone_read(double* total_ms, int64_t* launches, double* flops,
                                                        double* bytes) {
  std::lock_guard<std::mutex> lock(g_sprof_mu);
  double t = 0.0, fl = 0.0, by = 0.0;
  for (size_t i = 0; i < g_sprof_used; ++i) {
    cudaError_t e = cudaEventSynchronize(g_sprof_ev[i].second);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, g_sprof_ev[i].first, g_sprof_ev[i].second);
    if (e != cudaSuccess) return to_status(e);
    t += ms;
    fl += g_sprof_flops[i];
    by += g_sprof_bytes[i];
  }
  if (total_ms) *total_ms = t;
  if (launches) *launches = (int64_t)g_sprof_used;
  if (flops) *flops = fl;
  if (bytes) *bytes = by;
  g_sprof_used = 0;
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_dense_xf(int fmt, const void* x, int64_t ldx, const float* row_scale,
                                         int64_t n, const float* F, int ldf, int N, float* Y, int ldy,
                                         int gemm, void* stream) {
  if (!x || !F || !Y || n < 1 || N < 1 || N > 512 || ldx < n || ldf < N || ldy < N) return SYMNMF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const bool tc = fmt == SYMNMF_X_DENSE_BF16 || fmt == SYMNMF_X_DENSE_FP8;
  if (tc && gemm == SYMNMF_GEMM_SIMT) return SYMNMF_EUNSUPPORTED;
  if (!tc && gemm == SYMNMF_GEMM_TC) return SYMNMF_EUNSUPPORTED;
  if (!tc && N > 128) return SYMNMF_EINVAL;
  if (fmt == SYMNMF_X_DENSE_FP8 && !row_scale) return SYMNMF_EINVAL;
  cudaError_t e;
  if (!tc) {
    const size_t wsf = xf_simt_ws_floats(n, N);
    float* ws = nullptr;
    if (wsf && (e = cudaMallocAsync((void**)&ws, wsf * 4, st)) != cudaSuccess) return to_status(e);
    e = xf_simt(fmt, x, ldx, n, F, ldf, N, Y, ldy, ws, wsf, st);
    if (ws) cudaFreeAsync(ws, st);
    return to_status(e);
  }
  const int BN = tc_block_n(N);
  const int64_t ldp = (n + 15) / 16 * 16;
  const size_t es = fmt == SYMNMF_X_DENSE_FP8 ? 1 : 2;
  const size_t wsf = xf_tc_ws_floats(n, BN);
  void* pack = nullptr;
  float* ws = nullptr;
  float* cs = nullptr;
  unsigned* err = nullptr;
  e = cudaMallocAsync(&pack, (size_t)BN * ldp * es, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&ws, wsf * 4, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&cs, (size_t)BN * 4, st);  // one scale per packed column
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&err, 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 4, st);
  if (e == cudaSuccess)
    e = fmt == SYMNMF_X_DENSE_BF16 ? pack_ft_bf16(F, n, ldf, N, BN, pack, ldp, st)
                                   : pack_ft_fp8(F, n, ldf, N, BN, pack, ldp, cs, st);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = standalone_events(&e0, &e1, 2.0 * n * n * N, (double)n * n * es + (double)n * N * (es + 4.0));
  if (e == cudaSuccess)
    e = xf_tc(fmt, x, ldx, row_scale, n, pack, ldp, cs, N, Y, ldy, ws, wsf, err, st, e0, e1);
  unsigned herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  for (void* p : {pack, (void*)ws, (void*)cs, (void*)err})
    if (p) cudaFreeAsync(p, st);
  if (e != cudaSuccess) return to_status(e);
  return herr ? SYMNMF_ETIMEOUT : SYMNMF_OK;
}

extern "C" symnmf_status symnmf_csr_xf(const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                                       const float* F, int N, float* Y, void* stream) {
  if (!row_ptr || !col || !val || !F || !Y || n < 1 || N < 1 || N > 128) return SYMNMF_EINVAL;
  return to_status(csr_xf(row_ptr, col, val, n, F, N, N, Y, N, (cudaStream_t)stream));
}

extern "C" symnmf_status symnmf_gram(const float* F, int64_t n, int N, double* G, void* stream) {
  if (!F || !G || n < 1 || N < 1 || N > 128) return SYMNMF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  double* ws = nullptr;
  unsigned* cnt = nullptr;
  const size_t wsd = xcross_ws_doubles(N, N);
  cudaError_t e;
  if ((e = cudaMallocAsync((void**)&ws, wsd * 8, st)) != cudaSuccess) return to_status(e);
  if ((e = cudaMallocAsync((void**)&cnt, 4, st)) != cudaSuccess) {
    cudaFreeAsync(ws, st);
    return to_status(e);
  }
  e = cudaMemsetAsync(cnt, 0, 4, st);
  // two blocks per SM, as symnmf_gram_noalloc: both entry points sum in the same order
  if (e == cudaSuccess)
    e = xcross(F, N, N, F, N, N, n, nullptr, nullptr, nullptr, nullptr, 0.0, G, nullptr, ws, cnt, st, 2);
  cudaFreeAsync(ws, st);
  cudaFreeAsync(cnt, st);
  return to_status(e);
}

extern "C" symnmf_status symnmf_cholesky(const double* G, int k, double shift, double* R, double* Rinv,
                                         void* stream) {
  if (!G || k < 1 || k > 96 || !(shift >= 0.0)) return SYMNMF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* err = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&err, sizeof(unsigned), st);
  if (e != cudaSuccess) return to_status(e);
  e = cudaMemsetAsync(err, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = chol_inverse(G, k, shift, 0.0, Rinv, nullptr, err, st, R);
  unsigned herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(err, st);
  if (e != cudaSuccess) return to_status(e);
  return (herr & ERR_NOTSPD) ? SYMNMF_ENOTSPD : SYMNMF_OK;
}

extern "C" symnmf_status symnmf_gaussian(float* out, int64_t n, int l, uint64_t seed, void* stream) {
  if (!out || n < 1 || l < 1) return SYMNMF_EINVAL;
  return to_status(philox_gaussian(out, n, l, seed, (cudaStream_t)stream));
}

extern "C" symnmf_status symnmf_quantize_fp8(const float* x, int64_t n, int64_t ldx, uint8_t* x8, int64_t ld8,
                                             float* row_scale, void* stream) {
  if (!x || !x8 || !row_scale || n < 1 || ldx < n || ld8 < n) return SYMNMF_EINVAL;
  return to_status(quantize_fp8(x, n, ldx, x8, ld8, row_scale, (cudaStream_t)stream));
}

extern "C" symnmf_status symnmf_convert_bf16(const float* x, int64_t n, int64_t ldx, uint16_t* xb, int64_t ldb,
                                             void* stream) {
  if (!x || !xb || n < 1 || ldx < n || ldb < n) return SYMNMF_EINVAL;
  return to_status(convert_bf16(x, n, ldx, xb, ldb, (cudaStream_t)stream));
}

// ------------------------------------------------------------- profiling

extern "C" symnmf_status symnmf_profile(symnmf_t h, int enable) {
  if (!h) return SYMNMF_EINVAL;
  h->profiling = enable != 0;
  h->prof_used = 0;
  h->eprof_used = 0;
  h->lprof_used = 0;
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_profile_read_lvs(symnmf_t h, double* sampling_ms, double* products_ms,
                                                 double* update_ms, int64_t* halves) {
  if (!h) return SYMNMF_EINVAL;
  TRY(cudaStreamSynchronize(h->st));
  double t[3] = {0.0, 0.0, 0.0};
  for (size_t i = 0; i < h->lprof_used; ++i)
    for (int b = 0; b < 3; ++b) {
      float ms = 0.f;
      TRY(cudaEventElapsedTime(&ms, h->lprof_events[4 * i + b], h->lprof_events[4 * i + b + 1]));
      t[b] += ms;
    }
  if (sampling_ms) *sampling_ms = t[0];
  if (products_ms) *products_ms = t[1];
  if (update_ms) *update_ms = t[2];
  if (halves) *halves = (int64_t)h->lprof_used;
  h->lprof_used = 0;
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_profile_read(symnmf_t h, double* total_ms, int64_t* launches, double* bytes) {
  if (!h) return SYMNMF_EINVAL;
  TRY(cudaStreamSynchronize(h->st));
  double t = 0.0, by = 0.0;
  for (size_t i = 0; i < h->prof_used; ++i) {
    float ms = 0.f;
    TRY(cudaEventElapsedTime(&ms, h->prof_events[i].first, h->prof_events[i].second));
    t += ms;
    by += h->prof_bytes[i];
  }
  if (total_ms) *total_ms = t;
  if (launches) *launches = (int64_t)h->prof_used;
  if (bytes) *bytes = by;
  h->prof_used = 0;
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_profile_read_engine(symnmf_t h, double* total_ms, int64_t* launches,
                                                    double* flops) {
  if (!h) return SYMNMF_EINVAL;
  TRY(cudaStreamSynchronize(h->st));
  double t = 0.0, fl = 0.0;
  for (size_t i = 0; i < h->eprof_used; ++i) {
    float ms = 0.f;
    TRY(cudaEventElapsedTime(&ms, h->eprof_events[i].first, h->eprof_events[i].second));
    t += ms;
    fl += h->eprof_flops[i];
  }
  if (total_ms) *total_ms = t;
  if (launches) *launches = (int64_t)h->eprof_used;
  if (flops) *flops = fl;
  h->eprof_used = 0;
  return SYMNMF_OK;
}
