// Persistent LAI sweep engine (Alg. LAI-SymNMF loop body, HALS rule).
//
// With X ~ U Lambda U^T, a half sweep needs only M = Lambda U^T F_fix (l x k)
// and G = F_fix^T F_fix (k x k): every row r of the updated factor then
// follows from Y_r = U_r M (Eq. symhals_update2).  Both M and G are sums
// over all n rows, so on a GPU a half sweep is "row work, then a global
// reduction".  For the sizes of the LAI workload (n = 2e4 .. 5e4, k <= 64,
// l <= 96) separate kernels per step are launch- and latency-bound, so this
// engine runs every sweep in ONE cooperative launch (one CTA per SM):
//
//   per half sweep
//     1. each CTA updates its rows (tiles of 128 rows staged in shared
//        memory; Y_r = U_r M in registers; columns in order, each using the
//        ones already updated) and accumulates, over its rows, FP32 partials
//        of U^T F_upd, F_upd^T F_upd, and FP64 sum F_upd .* Y, ||F_upd - F_fix||^2;
//     2. grid barrier;
//     3. CTA c sums slice c of the entries over all CTA partials in FP64
//        (fixed order: deterministic) into a global "final" buffer;
//     4. grid barrier;
//     5. every CTA loads the new M (rows scaled by lambda) and G; CTA 0 writes
//        the surrogate objective after the H half (trace trick, FP64).
//
// The barrier is an arrival counter plus a generation word in global memory.
// Its waits are bounded (%globaltimer, 1 s): on expiry the waiting CTA sets
// ERR_TIMEOUT and every CTA leaves at its next barrier, so the host reads an
// error status instead of a hung launch.  Co-residency of all CTAs comes
// from the cooperative launch.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace symnmf {

constexpr int LE_THREADS = 256;
constexpr int LE_ROWS = 128;  // rows per staged tile (one updating thread per row)

__device__ __forceinline__ uint64_t le_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Returns false (on every thread of the block) when the barrier gave up.
__device__ bool le_grid_sync(unsigned* bar, unsigned* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    ok = 1;
    if (arrived == gridDim.x) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const uint64_t t0 = le_timer();
      unsigned spins = 0;
      while (*gen == g) {
        if ((++spins & 63u) == 0) {
          if (*(volatile unsigned*)err & ERR_TIMEOUT) {
            ok = 0;
            break;
          }
          if (le_timer() - t0 > 1000000000ull) {
            atomicOr(err, ERR_TIMEOUT);
            ok = 0;
            break;
          }
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

struct LaiArgs {
  const float* U;      // n x l
  const double* lam;   // l
  float* W;            // n x k
  float* H;            // n x k
  int64_t n;
  int k, l, nsweeps;
  float alpha;
  double alpha_d;
  const double* normX2;  // sum lambda^2
  double* part;          // [gridDim][E]
  double* fin;           // [2][E]: final sums, slot 0 = W side, slot 1 = H side
  double* obj;           // [nsweeps] (ring, capacity cap)
  int obj_cap;
  double* Gout;          // [2][k*k] FP64 Grams after the last sweep: [0] H^T H, [1] W^T W
  unsigned* bar;
  unsigned* err;
};

// Layout of one partial / final record: l*k entries of U^T F, k*k of F^T F, then tr, dd.
__host__ __device__ inline int le_entries(int l, int k) { return l * k + k * k + 2; }

template <int KMAX>
__global__ void __launch_bounds__(LE_THREADS, 1) lai_engine_kernel(LaiArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int k = a.k, l = a.l;
  const int E = le_entries(l, k);
  const int l4 = (l + 3) & ~3, k4 = (k + 3) & ~3;
  float* Ms = sm;                       // l x k  (lambda-scaled)
  float* Gs = Ms + l * k;               // k x k
  float* inv = Gs + k * k;              // k
  float* Us = inv + k4;                 // LE_ROWS x (l4 + 1)
  float* Fx = Us + LE_ROWS * (l4 + 1);  // LE_ROWS x (k4 + 1): fixed factor rows
  float* Fu = Fx + LE_ROWS * (k4 + 1);  // LE_ROWS x (k4 + 1): updated factor rows
  float* red = Fu + LE_ROWS * (k4 + 1); // 256 * 16 floats: row-group combine
  __shared__ double shd[32];

  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int64_t r0 = (a.n * blockIdx.x) / gridDim.x;
  const int64_t r1 = (a.n * (blockIdx.x + 1)) / gridDim.x;

  // 4x4 tiles over [U^T F (l4/4 x k4/4 tiles) | F^T F (k4/4 x k4/4 tiles)]
  const int tm = (l4 / 4) * (k4 / 4), tg = (k4 / 4) * (k4 / 4), T = tm + tg;
  const int RG = T >= LE_THREADS ? 1 : LE_THREADS / T;  // row groups
  const int my_rg = tid / T;
  const int TPT = (T + LE_THREADS - 1) / LE_THREADS;  // tiles per thread when T > threads

  // ---- partials of (U^T F, F^T F) over this CTA's rows of F (F in global) ----
  // also used for the prologue; tr / dd are passed in.
  auto partials = [&](const float* F, const float* Fsmem_unused, double tr, double dd, double* dst) {
    (void)Fsmem_unused;
    float acc[4][16];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int e = 0; e < 16; ++e) acc[t][e] = 0.f;
    for (int64_t b = r0; b < r1; b += LE_ROWS) {
      const int rows = (int)min((int64_t)LE_ROWS, r1 - b);
      for (int rr = wid; rr < LE_ROWS; rr += LE_THREADS / 32) {
        const bool live = rr < rows;
        for (int c = lane; c < l4; c += 32) Us[rr * (l4 + 1) + c] = (live && c < l) ? a.U[(b + rr) * l + c] : 0.f;
        for (int c = lane; c < k4; c += 32) Fu[rr * (k4 + 1) + c] = (live && c < k) ? F[(b + rr) * k + c] : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (t >= TPT) break;
        const int tile = (T >= LE_THREADS) ? tid + t * LE_THREADS : tid % T;
        if (tile < T && my_rg < RG) {
          const float* A;
          int ai, strideA, bj;
          if (tile < tm) {
            ai = (tile / (k4 / 4)) * 4;
            bj = (tile % (k4 / 4)) * 4;
            A = Us;
            strideA = l4 + 1;
          } else {
            const int g = tile - tm;
            ai = (g / (k4 / 4)) * 4;
            bj = (g % (k4 / 4)) * 4;
            A = Fu;
            strideA = k4 + 1;
          }
          for (int rr = my_rg; rr < rows; rr += RG) {
            float av[4], bv[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
              av[p] = A[rr * strideA + ai + p];
              bv[p] = Fu[rr * (k4 + 1) + bj + p];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
              for (int q = 0; q < 4; ++q) acc[t][p * 4 + q] = fmaf(av[p], bv[q], acc[t][p * 4 + q]);
          }
        }
      }
      __syncthreads();
    }
    // combine row groups in shared memory (fixed order), write FP64 record
    double* rec = dst + (size_t)blockIdx.x * E;
    for (int t = 0; t < TPT && t < 4; ++t) {
      const int tile = (T >= LE_THREADS) ? tid + t * LE_THREADS : tid % T;
      for (int g = 0; g < RG; ++g) {
        if (tile < T && my_rg == g)
#pragma unroll
          for (int e = 0; e < 16; ++e) red[(tile % LE_THREADS) * 16 + e] = (g == 0 ? 0.f : red[(tile % LE_THREADS) * 16 + e]) + acc[t][e];
        __syncthreads();
      }
      if (tile < T && my_rg == 0) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int p = e >> 2, q = e & 3;
          if (tile < tm) {
            const int i = (tile / (k4 / 4)) * 4 + p, j = (tile % (k4 / 4)) * 4 + q;
            if (i < l && j < k) rec[i * k + j] = (double)red[(tile % LE_THREADS) * 16 + e];
          } else {
            const int g2 = tile - tm;
            const int i = (g2 / (k4 / 4)) * 4 + p, j = (g2 % (k4 / 4)) * 4 + q;
            if (i < k && j < k) rec[l * k + i * k + j] = (double)red[(tile % LE_THREADS) * 16 + e];
          }
        }
      }
      __syncthreads();
    }
    double t2 = block_sum(tr, shd);
    double d2 = block_sum(dd, shd);
    if (tid == 0) {
      rec[l * k + k * k] = t2;
      rec[l * k + k * k + 1] = d2;
    }
  };

  // ---- sliced reduction of all CTA records into fin[slot] ----
  auto reduce_slice = [&](double* fin) {
    const int per = (E + gridDim.x - 1) / gridDim.x;
    const int e0 = blockIdx.x * per, e1 = min(E, e0 + per);
    for (int e = e0 + wid; e < e1; e += LE_THREADS / 32) {
      double s = 0.0;
      for (unsigned q = lane; q < gridDim.x; q += 32) s += __ldcg(a.part + (size_t)q * E + e);
      s = warp_sum(s);
      if (lane == 0) fin[e] = s;
    }
  };

  // ---- load M (lambda-scaled), G, inv from fin ----
  auto load_state = [&](const double* fin) {
    for (int e = tid; e < l * k; e += LE_THREADS) Ms[e] = (float)(a.lam[e / k] * __ldcg(fin + e));
    for (int e = tid; e < k * k; e += LE_THREADS) Gs[e] = (float)__ldcg(fin + l * k + e);
    __syncthreads();
    for (int i = tid; i < k; i += LE_THREADS) inv[i] = 1.0f / (Gs[i * k + i] + a.alpha);
    __syncthreads();
  };

  // prologue: state of the H side (W-update uses M = Lambda U^T H, G = H^T H)
  partials(a.H, nullptr, 0.0, 0.0, a.part);
  if (!le_grid_sync(a.bar, a.err)) return;
  reduce_slice(a.fin + E);
  if (!le_grid_sync(a.bar, a.err)) return;
  load_state(a.fin + E);

  for (int t = 0; t < a.nsweeps; ++t) {
    for (int side = 0; side < 2; ++side) {
      float* Fupd = side ? a.H : a.W;
      const float* Ffix = side ? a.W : a.H;
      double tr = 0.0, dd = 0.0;
      bool bad = false;
      // 1. row updates (threads 0..LE_ROWS-1 own one row of each tile)
      for (int64_t b = r0; b < r1; b += LE_ROWS) {
        const int rows = (int)min((int64_t)LE_ROWS, r1 - b);
        for (int rr = wid; rr < rows; rr += LE_THREADS / 32) {
          for (int c = lane; c < l; c += 32) Us[rr * (l4 + 1) + c] = a.U[(b + rr) * l + c];
          for (int c = lane; c < k; c += 32) {
            Fx[rr * (k4 + 1) + c] = Ffix[(b + rr) * k + c];
            Fu[rr * (k4 + 1) + c] = Fupd[(b + rr) * k + c];
          }
        }
        __syncthreads();
        if (tid < rows) {
          const float* ur = Us + tid * (l4 + 1);
          const float* hr = Fx + tid * (k4 + 1);
          float* wr = Fu + tid * (k4 + 1);
          float y[KMAX], w[KMAX];
#pragma unroll
          for (int c = 0; c < KMAX; ++c) y[c] = 0.f;
          for (int p = 0; p < l; ++p) {
            const float u = ur[p];
#pragma unroll
            for (int c = 0; c < KMAX; ++c)
              if (c < k) y[c] = fmaf(u, Ms[p * k + c], y[c]);
          }
#pragma unroll
          for (int j = 0; j < KMAX; ++j) w[j] = j < k ? wr[j] : 0.f;
#pragma unroll
          for (int i = 0; i < KMAX; ++i) {
            if (i < k) {
              float a0 = fmaf(a.alpha, hr[i], y[i]), a1 = 0.f;
#pragma unroll
              for (int j = 0; j < KMAX; ++j)
                if (j != i && j < k) {
                  if (j & 1)
                    a1 = fmaf(-w[j], Gs[j * k + i], a1);
                  else
                    a0 = fmaf(-w[j], Gs[j * k + i], a0);
                }
              w[i] = fmaxf((a0 + a1) * inv[i], 0.f);
            }
          }
#pragma unroll
          for (int j = 0; j < KMAX; ++j)
            if (j < k) {
              if (!isfinite(w[j])) bad = true;
              wr[j] = w[j];
              tr += (double)w[j] * (double)y[j];
              const float d = w[j] - hr[j];
              dd += (double)d * (double)d;
            }
        }
        __syncthreads();
        for (int rr = wid; rr < rows; rr += LE_THREADS / 32)
          for (int c = lane; c < k; c += 32) Fupd[(b + rr) * k + c] = Fu[rr * (k4 + 1) + c];
        __syncthreads();
      }
      if (bad) set_error(a.err, ERR_NAN);
      // 1b. partials over the updated rows (re-read: the tiles above are overwritten)
      partials(Fupd, nullptr, tr, dd, a.part);
      if (!le_grid_sync(a.bar, a.err)) return;
      double* fin = a.fin + (side == 0 ? 0 : E);
      reduce_slice(fin);
      if (!le_grid_sync(a.bar, a.err)) return;
      load_state(fin);
      if (side == 1 && blockIdx.x == 0) {
        // objective after the sweep: sum lambda^2 + sum GW .* GH - 2 tr + alpha dd
        const double* fw = a.fin;
        const double* fh = a.fin + E;
        double s = 0.0;
        for (int e = tid; e < k * k; e += LE_THREADS) s += __ldcg(fw + l * k + e) * __ldcg(fh + l * k + e);
        s = block_sum(s, shd);
        if (tid == 0 && t < a.obj_cap)
          a.obj[t] = a.normX2[0] + s - 2.0 * __ldcg(fh + l * k + k * k) + a.alpha_d * __ldcg(fh + l * k + k * k + 1);
      }
    }
  }
  // Grams after the last sweep for the handle's state: [0] = H^T H, [1] = W^T W
  if (blockIdx.x == 0)
    for (int e = tid; e < k * k; e += LE_THREADS) {
      a.Gout[e] = __ldcg(a.fin + E + l * k + e);
      a.Gout[k * k + e] = __ldcg(a.fin + l * k + e);
    }
}

size_t lai_engine_part_doubles(int l, int k) { return (size_t)num_sms() * le_entries(l, k); }
size_t lai_engine_fin_doubles(int l, int k) { return (size_t)2 * le_entries(l, k); }

template <int KMAX>
static cudaError_t launch_engine(const LaiArgs& a, cudaStream_t st) {
  const int l4 = (a.l + 3) & ~3, k4 = (a.k + 3) & ~3;
  const size_t smem = (size_t)(a.l * a.k + a.k * a.k + k4 + LE_ROWS * (l4 + 1) + 2 * LE_ROWS * (k4 + 1) +
                               LE_THREADS * 16) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(lai_engine_kernel<KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lai_engine_kernel<KMAX>, LE_THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int grid = num_sms();
  if ((int64_t)grid > a.n) grid = (int)std::max<int64_t>(1, a.n);
  LaiArgs args = a;
  void* params[] = {&args};
  e = cudaLaunchCooperativeKernel((const void*)lai_engine_kernel<KMAX>, dim3(grid), dim3(LE_THREADS), params,
                                  smem, st);
  count_launches(1);
  return e;
}

cudaError_t lai_engine(const float* U, const double* lam, float* W, float* H, int64_t n, int k, int l,
                       int nsweeps, double alpha, const double* normX2, double* part, double* fin, double* obj,
                       int obj_cap, double* Gout, unsigned* bar, unsigned* err, cudaStream_t st) {
  if (k < 1 || k > 64 || l < 1 || l > 96 || n < 1) return cudaErrorInvalidValue;
  LaiArgs a{U, lam, W, H, n, k, l, nsweeps, (float)alpha, alpha, normX2, part, fin, obj, obj_cap, Gout, bar, err};
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  if (k <= 16) return launch_engine<16>(a, st);
  if (k <= 32) return launch_engine<32>(a, st);
  return launch_engine<64>(a, st);
}

}  // namespace symnmf
