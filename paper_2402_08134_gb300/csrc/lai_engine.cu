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
//     1. each CTA updates its rows (tiles of up to 256 rows staged once in
//        shared memory; Y_r = U_r M in registers; columns in order, each using the
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

__device__ __forceinline__ uint64_t le_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The arrival counter (bar[0]) and the generation word (bar[LE_GEN]) sit in
// different 128-byte lines, so that the spinning readers of the generation do
// not contend with the arrivals.  Returns false (on every thread of the
// block) when the barrier gave up.
constexpr int LE_GEN = 32;

__device__ bool le_grid_sync(unsigned* bar, unsigned* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + LE_GEN;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    ok = 1;
    if (arrived == gridDim.x) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + LE_GEN, 1u);
    } else {
      const uint64_t t0 = le_timer();
      unsigned spins = 0;
      while (*gen == g) {
        __nanosleep(32);
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
  int tile_rows;
};

// Layout of one partial / final record: l*k entries of U^T F, k*k of F^T F, then tr, dd.
__host__ __device__ inline int le_entries(int l, int k) { return l * k + k * k + 2; }

template <int KMAX>
__global__ void __launch_bounds__(LE_THREADS, 1) lai_engine_kernel(LaiArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int k = a.k, l = a.l, TR = a.tile_rows;
  const int E = le_entries(l, k);
  const int l4 = (l + 3) & ~3, k4 = (k + 3) & ~3;
  const int us = l4 + 1, fs = k4 + 1;   // odd row pitches: conflict-free per-row reads
  float* Ms = sm;                        // l x k4, lambda-scaled, zero padded (float4 rows)
  float* Gs = Ms + l * k4;               // k x k4, zero padded (symmetric: row i = column i)
  float* inv = Gs + k * k4;              // k4
  float* Us = inv + k4;                  // TR x us: U rows of the tile
  float* Fx = Us + TR * us;              // TR x fs: fixed factor rows
  float* Fu = Fx + TR * fs;              // TR x fs: rows being updated
  float* red = Fu + TR * fs;             // LE_THREADS x 16: row-group combine
  __shared__ double shd[32];

  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int64_t r0 = (a.n * blockIdx.x) / gridDim.x;
  const int64_t r1 = (a.n * (blockIdx.x + 1)) / gridDim.x;

  // 4x4 tiles over [U^T F (l4/4 x k4/4 tiles) | F^T F (k4/4 x k4/4 tiles)]
  const int kt = k4 / 4;
  const int tm = (l4 / 4) * kt, tg = kt * kt, T = tm + tg;
  const int RG = T >= LE_THREADS ? 1 : LE_THREADS / T;  // row groups
  const int my_rg = T >= LE_THREADS ? 0 : tid / T;
  const int TPT = (T + LE_THREADS - 1) / LE_THREADS;     // tiles per thread (<= 4)
  float acc[4][16];

  auto clear_acc = [&]() {
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int e = 0; e < 16; ++e) acc[t][e] = 0.f;
  };

  // stage U rows (and optionally the fixed rows) of tile [b, b + rows); pads are zero
  auto stage = [&](int64_t b, int rows, const float* Ffix, const float* Fupd) {
    for (int rr = wid; rr < TR; rr += LE_THREADS / 32) {
      const bool live = rr < rows;
      const int64_t g = b + rr;
      for (int c = lane; c < l4; c += 32) Us[rr * us + c] = (live && c < l) ? a.U[g * l + c] : 0.f;
      for (int c = lane; c < k4; c += 32) {
        if (Ffix) Fx[rr * fs + c] = (live && c < k) ? Ffix[g * k + c] : 0.f;
        Fu[rr * fs + c] = (live && c < k) ? Fupd[g * k + c] : 0.f;
      }
    }
  };

  // accumulate this tile's rows of U^T Fu and Fu^T Fu into acc (FP32)
  auto accumulate = [&](int rows) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (t >= TPT) break;
      const int tile = (T >= LE_THREADS) ? tid + t * LE_THREADS : tid % T;
      if (tile < T && my_rg < RG) {
        const float* A;
        int ai, sa, bj;
        if (tile < tm) {
          ai = (tile / kt) * 4;
          bj = (tile % kt) * 4;
          A = Us;
          sa = us;
        } else {
          const int g = tile - tm;
          ai = (g / kt) * 4;
          bj = (g % kt) * 4;
          A = Fu;
          sa = fs;
        }
        for (int rr = my_rg; rr < rows; rr += RG) {
          float av[4], bv[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            av[p] = A[rr * sa + ai + p];
            bv[p] = Fu[rr * fs + bj + p];
          }
#pragma unroll
          for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[t][p * 4 + q] = fmaf(av[p], bv[q], acc[t][p * 4 + q]);
        }
      }
    }
  };

  // combine row groups (fixed order) and write this CTA's FP64 record
  auto finish = [&](double tr, double dd) {
    double* rec = a.part + (size_t)blockIdx.x * E;
    for (int t = 0; t < TPT; ++t) {
      const int tile = (T >= LE_THREADS) ? tid + t * LE_THREADS : tid % T;
      const int slot = (tile % LE_THREADS) * 16;
      for (int g = 0; g < RG; ++g) {
        if (tile < T && my_rg == g) {
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            float v = 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (u == t) v = acc[u][e];
            red[slot + e] = (g == 0 ? 0.f : red[slot + e]) + v;
          }
        }
        __syncthreads();
      }
      if (tile < T && my_rg == 0) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int p = e >> 2, q = e & 3;
          if (tile < tm) {
            const int i = (tile / kt) * 4 + p, j = (tile % kt) * 4 + q;
            if (i < l && j < k) rec[i * k + j] = (double)red[slot + e];
          } else {
            const int g2 = tile - tm;
            const int i = (g2 / kt) * 4 + p, j = (g2 % kt) * 4 + q;
            if (i < k && j < k) rec[l * k + i * k + j] = (double)red[slot + e];
          }
        }
      }
      __syncthreads();
    }
    const double t2 = block_sum(tr, shd);
    const double d2 = block_sum(dd, shd);
    if (tid == 0) {
      rec[l * k + k * k] = t2;
      rec[l * k + k * k + 1] = d2;
    }
  };

  // sliced reduction of all CTA records into fin (one warp per entry)
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

  // M (lambda-scaled), G, 1 / (G_ii + alpha) from fin
  auto load_state = [&](const double* fin) {
    for (int e = tid; e < l * k4; e += LE_THREADS) {
      const int i = e / k4, j = e - i * k4;
      Ms[e] = j < k ? (float)(a.lam[i] * __ldcg(fin + i * k + j)) : 0.f;
    }
    for (int e = tid; e < k * k4; e += LE_THREADS) {
      const int i = e / k4, j = e - i * k4;
      Gs[e] = j < k ? (float)__ldcg(fin + l * k + i * k + j) : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < k4; i += LE_THREADS) inv[i] = i < k ? 1.0f / (Gs[i * k4 + i] + a.alpha) : 0.f;
    __syncthreads();
  };

  // prologue: state of the H side (the W-update uses M = Lambda U^T H, G = H^T H)
  clear_acc();
  for (int64_t b = r0; b < r1; b += TR) {
    const int rows = (int)min((int64_t)TR, r1 - b);
    stage(b, rows, nullptr, a.H);
    __syncthreads();
    accumulate(rows);
    __syncthreads();
  }
  finish(0.0, 0.0);
  if (!le_grid_sync(a.bar, a.err)) return;
  reduce_slice(a.fin + E);
  if (!le_grid_sync(a.bar, a.err)) return;
  load_state(a.fin + E);

  const float4* Ms4 = reinterpret_cast<const float4*>(Ms);
  const float4* Gs4 = reinterpret_cast<const float4*>(Gs);
  const int k4q = k4 / 4;
  for (int t = 0; t < a.nsweeps; ++t) {
    for (int side = 0; side < 2; ++side) {
      float* Fupd = side ? a.H : a.W;
      const float* Ffix = side ? a.W : a.H;
      double tr = 0.0, dd = 0.0;
      bool bad = false;
      clear_acc();
      for (int64_t b = r0; b < r1; b += TR) {
        const int rows = (int)min((int64_t)TR, r1 - b);
        stage(b, rows, Ffix, Fupd);
        __syncthreads();
        if (tid < rows) {
          const float* ur = Us + tid * us;
          const float* hr = Fx + tid * fs;
          float* wr = Fu + tid * fs;
          float y[KMAX], w[KMAX];
#pragma unroll
          for (int c = 0; c < KMAX; ++c) y[c] = 0.f;
          // Y_r = U_r M  (LAI product), float4 broadcast reads of M's rows
          for (int p = 0; p < l; ++p) {
            const float u = ur[p];
#pragma unroll
            for (int c4 = 0; c4 < KMAX / 4; ++c4) {
              if (c4 < k4q) {
                const float4 m = Ms4[p * k4q + c4];
                y[4 * c4 + 0] = fmaf(u, m.x, y[4 * c4 + 0]);
                y[4 * c4 + 1] = fmaf(u, m.y, y[4 * c4 + 1]);
                y[4 * c4 + 2] = fmaf(u, m.z, y[4 * c4 + 2]);
                y[4 * c4 + 3] = fmaf(u, m.w, y[4 * c4 + 3]);
              }
            }
          }
#pragma unroll
          for (int j = 0; j < KMAX; ++j) w[j] = j < k ? wr[j] : 0.f;
          // columns in order, each using the columns already updated (G symmetric: row i)
#pragma unroll
          for (int i = 0; i < KMAX; ++i) {
            if (i < k) {
              float a0 = fmaf(a.alpha, hr[i], y[i]), a1 = 0.f;
#pragma unroll
              for (int j4 = 0; j4 < KMAX / 4; ++j4) {
                if (j4 < k4q) {
                  const float4 g = Gs4[i * k4q + j4];
                  const float gv[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
                  for (int u = 0; u < 4; ++u) {
                    const int j = 4 * j4 + u;
                    if (j != i) {  // pads of G are zero, so j >= k adds nothing
                      if (u & 1)
                        a1 = fmaf(-w[j], gv[u], a1);
                      else
                        a0 = fmaf(-w[j], gv[u], a0);
                    }
                  }
                }
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
          for (int c = lane; c < k; c += 32) Fupd[(b + rr) * k + c] = Fu[rr * fs + c];
        accumulate(rows);  // partials of the next half straight from shared memory
        __syncthreads();
      }
      if (bad) set_error(a.err, ERR_NAN);
      finish(tr, dd);
      if (!le_grid_sync(a.bar, a.err)) return;
      double* fin = a.fin + (side == 0 ? 0 : E);
      reduce_slice(fin);
      if (!le_grid_sync(a.bar, a.err)) return;
      load_state(fin);
      if (side == 1 && blockIdx.x == 0) {
        // objective after the sweep: sum lambda^2 + sum GW .* GH - 2 tr + alpha dd
        const double* fw = a.fin;
        const double* fh = a.fin + E;
        double s2 = 0.0;
        for (int e = tid; e < k * k; e += LE_THREADS) s2 += __ldcg(fw + l * k + e) * __ldcg(fh + l * k + e);
        s2 = block_sum(s2, shd);
        if (tid == 0 && t < a.obj_cap)
          a.obj[t] = a.normX2[0] + s2 - 2.0 * __ldcg(fh + l * k + k * k) + a.alpha_d * __ldcg(fh + l * k + k * k + 1);
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

static size_t engine_smem(int l, int k, int tr) {
  const int l4 = (l + 3) & ~3, k4 = (k + 3) & ~3;
  return (size_t)(l * k4 + k * k4 + k4 + tr * (l4 + 1) + 2 * tr * (k4 + 1) + LE_THREADS * 16) * sizeof(float);
}

template <int KMAX>
static cudaError_t launch_engine(LaiArgs a, cudaStream_t st) {
  // one tile per CTA when it fits (n = 2e4 gives ~132 rows per CTA)
  a.tile_rows = engine_smem(a.l, a.k, 256) <= 200 * 1024 ? 256 : 128;
  const size_t smem = engine_smem(a.l, a.k, a.tile_rows);
  cudaError_t e = cudaFuncSetAttribute(lai_engine_kernel<KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lai_engine_kernel<KMAX>, LE_THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int grid = num_sms();
  if ((int64_t)grid > a.n) grid = (int)std::max<int64_t>(1, a.n);
  void* params[] = {&a};
  e = cudaLaunchCooperativeKernel((const void*)lai_engine_kernel<KMAX>, dim3(grid), dim3(LE_THREADS), params,
                                  smem, st);
  count_launches(1);
  return e;
}

cudaError_t lai_engine(const float* U, const double* lam, float* W, float* H, int64_t n, int k, int l,
                       int nsweeps, double alpha, const double* normX2, double* part, double* fin, double* obj,
                       int obj_cap, double* Gout, unsigned* bar, unsigned* err, cudaStream_t st) {
  if (k < 1 || k > 64 || l < 1 || l > 96 || n < 1) return cudaErrorInvalidValue;
  LaiArgs a{U, lam, W, H, n, k, l, nsweeps, (float)alpha, alpha, normX2, part, fin, obj, obj_cap, Gout, bar, err, 256};
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * LE_GEN * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  if (k <= 8) return launch_engine<8>(a, st);
  if (k <= 16) return launch_engine<16>(a, st);
  if (k <= 24) return launch_engine<24>(a, st);
  if (k <= 32) return launch_engine<32>(a, st);
  if (k <= 48) return launch_engine<48>(a, st);
  return launch_engine<64>(a, st);
}

}  // namespace symnmf
