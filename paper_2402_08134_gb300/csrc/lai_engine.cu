// Persistent LAI sweep engine (Alg. LAI-SymNMF loop body, HALS rule).
//
// With X ~ U Lambda U^T, a half sweep needs only M = Lambda U^T F_fix (l x k)
// and G = F_fix^T F_fix (k x k): every row r of the updated factor then
// follows from Y_r = U_r M (Eq. symhals_update2).  Both M and G are sums
// over all n rows, so on a GPU a half sweep is "row work, then a global
// reduction".  For the sizes of the LAI workload (n = 2e4 .. 5e4, k <= 64,
// l <= 96) separate kernels per step are launch- and latency-bound, so this
// engine runs every sweep in ONE cooperative launch (one CTA per SM).  CTA c
// owns the contiguous rows [n c / grid, n (c + 1) / grid) of U, W and H.
//
//   per half sweep
//     1. each CTA updates its rows (Y_r = U_r M in registers; columns in
//        order, each using the ones already updated) and accumulates, over its
//        rows, FP32 partials of U^T F_upd, F_upd^T F_upd, and FP64 sums of
//        per-row F_upd . Y and ||F_upd - F_fix||^2;
//     2. grid barrier;
//     3. CTA c sums slice c of the entries over all CTA partials in FP64
//        (fixed order: deterministic) into a global "final" buffer;
//     4. grid barrier;
//     5. every CTA loads the new M (rows scaled by lambda) and G; CTA 0 writes
//        the surrogate objective after the H half (trace trick, FP64).
//
// Two variants of the row work:
//   resident  the CTA's rows of U, W and H stay in shared memory for the whole
//             launch, stored column-major (entry (r, c) at c * RP + r, RP = the
//             row count padded to 4): per-row reads by thread r are
//             conflict-free and the cross-product partials read float4 runs of
//             four rows.  W and H reach global memory once, at the end.  Used
//             whenever the rows fit (n = 5e4, k = 32, l = 74 takes 216 KB).
//   streamed  rows pass through shared memory in tiles of up to 256, staged
//             from and written back to global memory every half sweep.
//
// The grid barrier (persist.cuh) is bounded: on expiry the host reads an
// error status instead of a hung launch.  Co-residency of all CTAs comes
// from the cooperative launch.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "persist.cuh"

namespace symnmf {

constexpr int LE_THREADS = 256;

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
  int tile_rows;         // streamed: rows per tile; resident: padded rows per CTA (RP)
};

// Layout of one partial / final record: l*k entries of U^T F, k*k of F^T F, then tr, dd.
__host__ __device__ inline int le_entries(int l, int k) { return l * k + k * k + 2; }

// 4x4 tiles over [U^T F (l4/4 x k4/4 tiles) | F^T F (k4/4 x k4/4 tiles)], spread
// over the block's threads; with fewer tiles than threads, RG row groups of
// threads split the rows and are combined in a fixed order.
struct LeTiles {
  int kt, tm, T, RG, my_rg, TPT;
};

__device__ __forceinline__ LeTiles le_tiles(int l4, int k4) {
  LeTiles t;
  t.kt = k4 / 4;
  t.tm = (l4 / 4) * t.kt;
  t.T = t.tm + t.kt * t.kt;
  t.RG = t.T >= LE_THREADS ? 1 : LE_THREADS / t.T;
  t.my_rg = t.T >= LE_THREADS ? 0 : (int)threadIdx.x / t.T;
  t.TPT = (t.T + LE_THREADS - 1) / LE_THREADS;  // <= 4 for l <= 96, k <= 64
  return t;
}

__device__ __forceinline__ int le_tile_of(const LeTiles& tl, int t) {
  return (tl.T >= LE_THREADS) ? (int)threadIdx.x + t * LE_THREADS : (int)threadIdx.x % tl.T;
}

__device__ __forceinline__ void le_clear(float (&acc)[4][16]) {
#pragma unroll
  for (int t = 0; t < 4; ++t)
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[t][e] = 0.f;
}

// Combine row groups (fixed order) and write this CTA's FP64 record.
__device__ __forceinline__ void le_finish(const LaiArgs& a, const LeTiles& tl, const float (&acc)[4][16],
                                          float* red, double* shd, double tr, double dd) {
  const int k = a.k, l = a.l, E = le_entries(l, k);
  double* rec = a.part + (size_t)blockIdx.x * E;
  for (int t = 0; t < tl.TPT; ++t) {
    const int tile = le_tile_of(tl, t);
    const int slot = (tile % LE_THREADS) * 16;
    for (int g = 0; g < tl.RG; ++g) {
      if (tile < tl.T && tl.my_rg == g) {
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
    if (tile < tl.T && tl.my_rg == 0) {
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int p = e >> 2, q = e & 3;
        if (tile < tl.tm) {
          const int i = (tile / tl.kt) * 4 + p, j = (tile % tl.kt) * 4 + q;
          if (i < l && j < k) rec[i * k + j] = (double)red[slot + e];
        } else {
          const int g2 = tile - tl.tm;
          const int i = (g2 / tl.kt) * 4 + p, j = (g2 % tl.kt) * 4 + q;
          if (i < k && j < k) rec[l * k + i * k + j] = (double)red[slot + e];
        }
      }
    }
    __syncthreads();
  }
  const double t2 = block_sum(tr, shd);
  const double d2 = block_sum(dd, shd);
  if (threadIdx.x == 0) {
    rec[l * k + k * k] = t2;
    rec[l * k + k * k + 1] = d2;
  }
}

// Sliced reduction of all CTA records into fin: 16 lanes per entry, the
// lanes' strided sums combined by a fixed xor tree (deterministic).
__device__ __forceinline__ void le_reduce_slice(const LaiArgs& a, double* fin) {
  const int E = le_entries(a.l, a.k);
  const int per = (E + gridDim.x - 1) / gridDim.x;
  const int e0 = blockIdx.x * per, e1 = min(E, e0 + per);
  const int grp = threadIdx.x >> 4, sub = threadIdx.x & 15;
  for (int base = e0; base < e1; base += LE_THREADS / 16) {
    const int e = base + grp;
    double s = 0.0;
    if (e < e1) {
#pragma unroll 4
      for (unsigned q = sub; q < gridDim.x; q += 16) s += __ldcg(a.part + (size_t)q * E + e);
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (e < e1 && sub == 0) fin[e] = s;
  }
}

// M (lambda-scaled), G, 1 / (G_ii + alpha) from fin.
__device__ __forceinline__ void le_load_state(const LaiArgs& a, const double* fin, float* Ms, float* Gs,
                                              float* inv) {
  const int k = a.k, l = a.l, k4 = (k + 3) & ~3;
#pragma unroll 4
  for (int e = threadIdx.x; e < l * k4; e += LE_THREADS) {
    const int i = e / k4, j = e - i * k4;
    Ms[e] = j < k ? (float)(__ldg(a.lam + i) * __ldcg(fin + i * k + j)) : 0.f;
  }
#pragma unroll 4
  for (int e = threadIdx.x; e < k * k4; e += LE_THREADS) {
    const int i = e / k4, j = e - i * k4;
    Gs[e] = j < k ? (float)__ldcg(fin + l * k + i * k + j) : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k4; i += LE_THREADS) inv[i] = i < k ? 1.0f / (Gs[i * k4 + i] + a.alpha) : 0.f;
  __syncthreads();
}

// Objective after a full sweep (CTA 0): sum lambda^2 + sum GW .* GH - 2 tr + alpha dd.
__device__ __forceinline__ void le_objective(const LaiArgs& a, int t, double* shd) {
  const int k = a.k, l = a.l, E = le_entries(l, k);
  const double* fw = a.fin;
  const double* fh = a.fin + E;
  double s2 = 0.0;
  for (int e = threadIdx.x; e < k * k; e += LE_THREADS) s2 += __ldcg(fw + l * k + e) * __ldcg(fh + l * k + e);
  s2 = block_sum(s2, shd);
  if (threadIdx.x == 0 && t < a.obj_cap)
    a.obj[t] = a.normX2[0] + s2 - 2.0 * __ldcg(fh + l * k + k * k) + a.alpha_d * __ldcg(fh + l * k + k * k + 1);
}

// HALS update of one row (Eq. symhals_update2): y = U_r M with U_r read
// through `u_at(p)`, the fixed row through `fx_at(i)`, the row being updated
// through the reference `fu_ref(j)`.  Gives the row's F_upd . Y and
// ||F_upd - F_fix||^2 in FP32 (the caller sums rows in FP64); returns true
// when a non-finite value appeared.
template <int KMAX, class UA, class FXA, class FUA>
__device__ __forceinline__ bool le_row_update(float alpha, int l, int k, int k4q, const float4* Ms4,
                                              const float4* Gs4, const float* inv, UA u_at, FXA fx_at, FUA fu_ref,
                                              float& trow, float& drow) {
  float y[KMAX], w[KMAX];
#pragma unroll
  for (int c = 0; c < KMAX; ++c) y[c] = 0.f;
  // Y_r = U_r M  (LAI product), float4 broadcast reads of M's rows
  for (int p = 0; p < l; ++p) {
    const float u = u_at(p);
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
  for (int j = 0; j < KMAX; ++j) w[j] = j < k ? fu_ref(j) : 0.f;
  // columns in order, each using the columns already updated (G symmetric: row i)
#pragma unroll
  for (int i = 0; i < KMAX; ++i) {
    if (i < k) {
      float a0 = fmaf(alpha, fx_at(i), y[i]), a1 = 0.f;
#pragma unroll
      for (int j4 = 0; j4 < KMAX / 4; ++j4) {
        if (j4 < k4q) {
          const float4 g = Gs4[i * k4q + j4];
          const float gv[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int j = 4 * j4 + q;
            if (j != i) {  // pads of G are zero, so j >= k adds nothing
              if (q & 1)
                a1 = fmaf(-w[j], gv[q], a1);
              else
                a0 = fmaf(-w[j], gv[q], a0);
            }
          }
        }
      }
      w[i] = fmaxf((a0 + a1) * inv[i], 0.f);
    }
  }
  bool bad = false;
  float t0 = 0.f, t1 = 0.f, d0 = 0.f, d1 = 0.f;
#pragma unroll
  for (int j = 0; j < KMAX; ++j)
    if (j < k) {
      if (!isfinite(w[j])) bad = true;
      fu_ref(j) = w[j];
      const float d = w[j] - fx_at(j);
      if (j & 1) {
        t1 = fmaf(w[j], y[j], t1);
        d1 = fmaf(d, d, d1);
      } else {
        t0 = fmaf(w[j], y[j], t0);
        d0 = fmaf(d, d, d0);
      }
    }
  trow = t0 + t1;
  drow = d0 + d1;
  return bad;
}

// ------------------------------------------------------------ resident rows

template <int KMAX>
__global__ void __launch_bounds__(LE_THREADS, 1) lai_resident_kernel(LaiArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int k = a.k, l = a.l, RP = a.tile_rows;
  const int l4 = (l + 3) & ~3, k4 = (k + 3) & ~3, k4q = k4 / 4;
  const int E = le_entries(l, k);
  float* Ms = sm;             // l x k4, lambda-scaled, zero padded (float4 rows)
  float* Gs = Ms + l * k4;    // k x k4, zero padded (symmetric: row i = column i)
  float* inv = Gs + k * k4;   // k4
  float* Ut = inv + k4;       // l4 x RP: column c of the CTA's U rows at Ut + c * RP
  float* Wt = Ut + l4 * RP;   // k4 x RP
  float* Ht = Wt + k4 * RP;   // k4 x RP
  float* red = Ht + k4 * RP;  // LE_THREADS x 16: row-group combine
  __shared__ double shd[32];

  const int tid = threadIdx.x;
  const int64_t r0 = (a.n * blockIdx.x) / gridDim.x;
  const int R = (int)((a.n * (blockIdx.x + 1)) / gridDim.x - r0);
  const LeTiles tl = le_tiles(l4, k4);
  float acc[4][16];

  // prologue: the CTA's rows, transposed into shared memory (pads stay zero)
  for (int e = tid; e < (l4 + 2 * k4) * RP; e += LE_THREADS) Ut[e] = 0.f;
  __syncthreads();
  {
    const float* Ug = a.U + r0 * l;
    for (int e = tid; e < R * l; e += LE_THREADS) {
      const int r = e / l, c = e - r * l;
      Ut[c * RP + r] = __ldg(Ug + e);
    }
    const float* Wg = a.W + r0 * k;
    const float* Hg = a.H + r0 * k;
    for (int e = tid; e < R * k; e += LE_THREADS) {
      const int r = e / k, c = e - r * k;
      Wt[c * RP + r] = Wg[e];
      Ht[c * RP + r] = Hg[e];
    }
  }
  __syncthreads();

  // U^T F and F^T F over the CTA's rows, four rows per float4 step
  auto accumulate = [&](const float* Fu) {
    const int rq = RP / 4;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (t >= tl.TPT) break;
      const int tile = le_tile_of(tl, t);
      if (tile < tl.T && tl.my_rg < tl.RG) {
        const float* A;
        int bj;
        if (tile < tl.tm) {
          A = Ut + (tile / tl.kt) * 4 * RP;
          bj = (tile % tl.kt) * 4;
        } else {
          const int g = tile - tl.tm;
          A = Fu + (g / tl.kt) * 4 * RP;
          bj = (g % tl.kt) * 4;
        }
        const float* B = Fu + bj * RP;
        for (int c = tl.my_rg; c < rq; c += tl.RG) {
          float4 av[4], bv[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            av[p] = reinterpret_cast<const float4*>(A + p * RP)[c];
            bv[p] = reinterpret_cast<const float4*>(B + p * RP)[c];
          }
#pragma unroll
          for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              float s = acc[t][p * 4 + q];
              s = fmaf(av[p].x, bv[q].x, s);
              s = fmaf(av[p].y, bv[q].y, s);
              s = fmaf(av[p].z, bv[q].z, s);
              s = fmaf(av[p].w, bv[q].w, s);
              acc[t][p * 4 + q] = s;
            }
        }
      }
    }
  };

  // prologue: state of the H side (the W-update uses M = Lambda U^T H, G = H^T H)
  le_clear(acc);
  accumulate(Ht);
  le_finish(a, tl, acc, red, shd, 0.0, 0.0);
  if (!grid_sync_bounded(a.bar, a.err)) return;
  le_reduce_slice(a, a.fin + E);
  if (!grid_sync_bounded(a.bar, a.err)) return;
  le_load_state(a, a.fin + E, Ms, Gs, inv);

  const float4* Ms4 = reinterpret_cast<const float4*>(Ms);
  const float4* Gs4 = reinterpret_cast<const float4*>(Gs);
  for (int t = 0; t < a.nsweeps; ++t) {
    for (int side = 0; side < 2; ++side) {
      float* Fu = side ? Ht : Wt;
      const float* Fx = side ? Wt : Ht;
      double tr = 0.0, dd = 0.0;
      bool bad = false;
      for (int r = tid; r < R; r += LE_THREADS) {
        float trow, drow;
        bad |= le_row_update<KMAX>(
            a.alpha, l, k, k4q, Ms4, Gs4, inv, [&](int p) { return Ut[p * RP + r]; },
            [&](int i) { return Fx[i * RP + r]; }, [&](int j) -> float& { return Fu[j * RP + r]; }, trow, drow);
        tr += (double)trow;
        dd += (double)drow;
      }
      if (bad) set_error(a.err, ERR_NAN);
      __syncthreads();
      le_clear(acc);
      accumulate(Fu);
      le_finish(a, tl, acc, red, shd, tr, dd);
      if (!grid_sync_bounded(a.bar, a.err)) return;
      double* fin = a.fin + (side == 0 ? 0 : E);
      le_reduce_slice(a, fin);
      if (!grid_sync_bounded(a.bar, a.err)) return;
      le_load_state(a, fin, Ms, Gs, inv);
      if (side == 1 && blockIdx.x == 0) le_objective(a, t, shd);
    }
  }
  // epilogue: the CTA's rows of W and H back to global memory
  {
    float* Wg = a.W + r0 * k;
    float* Hg = a.H + r0 * k;
    for (int e = tid; e < R * k; e += LE_THREADS) {
      const int r = e / k, c = e - r * k;
      Wg[e] = Wt[c * RP + r];
      Hg[e] = Ht[c * RP + r];
    }
  }
  // Grams after the last sweep for the handle's state: [0] = H^T H, [1] = W^T W
  if (blockIdx.x == 0)
    for (int e = tid; e < k * k; e += LE_THREADS) {
      a.Gout[e] = __ldcg(a.fin + E + l * k + e);
      a.Gout[k * k + e] = __ldcg(a.fin + l * k + e);
    }
}

// ------------------------------------------------------------- streamed rows

template <int KMAX>
__global__ void __launch_bounds__(LE_THREADS, 1) lai_streamed_kernel(LaiArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int k = a.k, l = a.l, TR = a.tile_rows;
  const int l4 = (l + 3) & ~3, k4 = (k + 3) & ~3, k4q = k4 / 4;
  const int E = le_entries(l, k);
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
  const int64_t r0 = (a.n * blockIdx.x) / gridDim.x;
  const int64_t r1 = (a.n * (blockIdx.x + 1)) / gridDim.x;
  const LeTiles tl = le_tiles(l4, k4);
  float acc[4][16];

  // pad columns (c >= l of U, c >= k of the factors) are zero once and for all;
  // rows past a tile's end are never read
  for (int e = tid; e < TR * (us + 2 * fs); e += LE_THREADS) Us[e] = 0.f;
  __syncthreads();

  // stage U rows (and optionally the fixed rows) of tile [b, b + rows): the
  // tile is one contiguous run of each array, read with independent loads
  auto stage = [&](int64_t b, int rows, const float* Ffix, const float* Fupd) {
    const float* Ug = a.U + b * l;
#pragma unroll 4
    for (int e = tid; e < rows * l; e += LE_THREADS) {
      const int r = e / l, c = e - r * l;
      Us[r * us + c] = __ldg(Ug + e);
    }
#pragma unroll 4
    for (int e = tid; e < rows * k; e += LE_THREADS) {
      const int r = e / k, c = e - r * k;
      if (Ffix) Fx[r * fs + c] = Ffix[b * k + e];
      Fu[r * fs + c] = Fupd[b * k + e];
    }
  };

  // accumulate this tile's rows of U^T Fu and Fu^T Fu into acc (FP32)
  auto accumulate = [&](int rows) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (t >= tl.TPT) break;
      const int tile = le_tile_of(tl, t);
      if (tile < tl.T && tl.my_rg < tl.RG) {
        const float* A;
        int ai, sa, bj;
        if (tile < tl.tm) {
          ai = (tile / tl.kt) * 4;
          bj = (tile % tl.kt) * 4;
          A = Us;
          sa = us;
        } else {
          const int g = tile - tl.tm;
          ai = (g / tl.kt) * 4;
          bj = (g % tl.kt) * 4;
          A = Fu;
          sa = fs;
        }
        for (int rr = tl.my_rg; rr < rows; rr += tl.RG) {
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

  // prologue: state of the H side (the W-update uses M = Lambda U^T H, G = H^T H)
  le_clear(acc);
  for (int64_t b = r0; b < r1; b += TR) {
    const int rows = (int)min((int64_t)TR, r1 - b);
    stage(b, rows, nullptr, a.H);
    __syncthreads();
    accumulate(rows);
    __syncthreads();
  }
  le_finish(a, tl, acc, red, shd, 0.0, 0.0);
  if (!grid_sync_bounded(a.bar, a.err)) return;
  le_reduce_slice(a, a.fin + E);
  if (!grid_sync_bounded(a.bar, a.err)) return;
  le_load_state(a, a.fin + E, Ms, Gs, inv);

  const float4* Ms4 = reinterpret_cast<const float4*>(Ms);
  const float4* Gs4 = reinterpret_cast<const float4*>(Gs);
  for (int t = 0; t < a.nsweeps; ++t) {
    for (int side = 0; side < 2; ++side) {
      float* Fupd = side ? a.H : a.W;
      const float* Ffix = side ? a.W : a.H;
      double tr = 0.0, dd = 0.0;
      bool bad = false;
      le_clear(acc);
      for (int64_t b = r0; b < r1; b += TR) {
        const int rows = (int)min((int64_t)TR, r1 - b);
        stage(b, rows, Ffix, Fupd);
        __syncthreads();
        if (tid < rows) {
          const float* ur = Us + tid * us;
          const float* hr = Fx + tid * fs;
          float* wr = Fu + tid * fs;
          float trow, drow;
          bad |= le_row_update<KMAX>(
              a.alpha, l, k, k4q, Ms4, Gs4, inv, [&](int p) { return ur[p]; }, [&](int i) { return hr[i]; },
              [&](int j) -> float& { return wr[j]; }, trow, drow);
          tr += (double)trow;
          dd += (double)drow;
        }
        __syncthreads();
#pragma unroll 4
        for (int e = tid; e < rows * k; e += LE_THREADS) {
          const int r = e / k, c = e - r * k;
          Fupd[b * k + e] = Fu[r * fs + c];
        }
        accumulate(rows);  // partials of the next half straight from shared memory
        __syncthreads();
      }
      if (bad) set_error(a.err, ERR_NAN);
      le_finish(a, tl, acc, red, shd, tr, dd);
      if (!grid_sync_bounded(a.bar, a.err)) return;
      double* fin = a.fin + (side == 0 ? 0 : E);
      le_reduce_slice(a, fin);
      if (!grid_sync_bounded(a.bar, a.err)) return;
      le_load_state(a, fin, Ms, Gs, inv);
      if (side == 1 && blockIdx.x == 0) le_objective(a, t, shd);
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

static size_t streamed_smem(int l, int k, int tr) {
  const int l4 = (l + 3) & ~3, k4 = (k + 3) & ~3;
  return (size_t)(l * k4 + k * k4 + k4 + tr * (l4 + 1) + 2 * tr * (k4 + 1) + LE_THREADS * 16) * sizeof(float);
}

static size_t resident_smem(int l, int k, int rp) {
  const int l4 = (l + 3) & ~3, k4 = (k + 3) & ~3;
  return (size_t)((l + k + 1) * k4 + (l4 + 2 * k4) * rp + LE_THREADS * 16) * sizeof(float);
}

static size_t smem_optin_limit() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  return v > 1024 ? (size_t)(v - 1024) : 0;  // room for the kernels' static shared memory
}

template <int KMAX>
static cudaError_t launch_engine(LaiArgs a, bool allow_resident, cudaStream_t st) {
  int grid = num_sms();
  if ((int64_t)grid > a.n) grid = (int)std::max<int64_t>(1, a.n);
  const int64_t rmax = (a.n + grid - 1) / grid;
  const int64_t rp = (rmax + 3) & ~3LL;
  const void* fn;
  size_t smem;
  if (allow_resident && rp <= (1 << 20) && resident_smem(a.l, a.k, (int)rp) <= smem_optin_limit()) {
    fn = (const void*)lai_resident_kernel<KMAX>;
    a.tile_rows = (int)rp;
    smem = resident_smem(a.l, a.k, (int)rp);
  } else {
    fn = (const void*)lai_streamed_kernel<KMAX>;
    // one tile per CTA when it fits (n = 2e4 gives ~132 rows per CTA)
    a.tile_rows = streamed_smem(a.l, a.k, 256) <= 200 * 1024 ? 256 : 128;
    smem = streamed_smem(a.l, a.k, a.tile_rows);
  }
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, LE_THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  void* params[] = {&a};
  e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(LE_THREADS), params, smem, st);
  count_launches(1);
  return e;
}

cudaError_t lai_engine(const float* U, const double* lam, float* W, float* H, int64_t n, int k, int l,
                       int nsweeps, double alpha, const double* normX2, double* part, double* fin, double* obj,
                       int obj_cap, double* Gout, unsigned* bar, unsigned* err, bool allow_resident,
                       cudaStream_t st) {
  if (k < 1 || k > 64 || l < 1 || l > 96 || n < 1) return cudaErrorInvalidValue;
  LaiArgs a{U, lam, W, H, n, k, l, nsweeps, (float)alpha, alpha, normX2, part, fin, obj, obj_cap, Gout, bar, err, 256};
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * GRID_GEN * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  if (k <= 8) return launch_engine<8>(a, allow_resident, st);
  if (k <= 16) return launch_engine<16>(a, allow_resident, st);
  if (k <= 24) return launch_engine<24>(a, allow_resident, st);
  if (k <= 32) return launch_engine<32>(a, allow_resident, st);
  if (k <= 48) return launch_engine<48>(a, allow_resident, st);
  return launch_engine<64>(a, allow_resident, st);
}

}  // namespace symnmf
