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
//     1. each CTA updates its rows (Y = U M for its rows, then per row the
//        columns in order, each using the ones already updated) and writes
//        one FP32 record (its row groups added) of its partial sums over its rows: U^T F_upd,
//        F_upd^T F_upd (upper 4x4 tiles; FMA sums over four rows folded into
//        Kahan-compensated totals, each rounded once), and (as hi/lo float
//        pairs of FP64 sums) F_upd . Y and ||F_upd - F_fix||^2;
//     2. grid barrier;
//     3. CTA c sums slice c of the entries over all records in double-float
//        (Dekker's two-sum; a warp per float4 column, lanes over records, a
//        fixed shuffle tree: deterministic) and writes the FP64
//        sums, plus the next half's state in FP32 -- lambda-scaled M, G and
//        1 / (G_ii + alpha) laid out as the CTAs hold them in shared memory --
//        and, after the H half, its share of the surrogate objective (trace
//        trick, FP64);
//     4. grid barrier;
//     5. every CTA copies the state into shared memory (float4 loads).
//   After the last sweep the CTAs sum the objective shares of every sweep.
//
// Two variants of the row work:
//   resident  the CTA's rows of U, W and H stay in shared memory for the whole
//             launch, stored column-major: column c starts at c P + 4 ((c / 4)
//             mod 8), P = the row count padded to 8 plus 32, a skew that puts
//             the four-column blocks read together by the cross products in
//             different bank groups.  Y = U M is a CTA-wide product with 4x4
//             register tiles into shared memory; the per-row column updates
//             (one thread per row) read Y from there; the cross products read
//             float4 runs of four rows.  W and H reach global memory once, at
//             the end.  Used whenever the rows fit.
//   streamed  rows pass through shared memory in tiles of up to 256, staged
//             from and written back to global memory every half sweep; each
//             thread forms its row of Y itself.
//
// The grid barrier (persist.cuh) is bounded: on expiry the host reads an
// error status instead of a hung launch.  Co-residency of all CTAs comes
// from the cooperative launch.
#pragma once

#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "persist.cuh"
#include "hals_row.cuh"

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
  float* part;           // [gridDim * RG][EP] partial records
  double* fin;           // [2][E]: final sums, slot 0 = W side, slot 1 = H side
  float* state;          // [2][SL]: M (lambda-scaled, l x k4), G (gp x gp), 1 / (G_ii + alpha) (gp)
  double* objp;          // [obj_cap][gridDim]: objective shares
  double* obj;           // [nsweeps] (ring, capacity cap)
  int obj_cap;
  double* Gout;          // [2][k*k] FP64 Grams after the last sweep: [0] H^T H, [1] W^T W
  unsigned* bar;
  unsigned* err;
  int tile_rows;         // streamed: rows per tile; resident: rows per CTA padded to 4 (RP)
  int gp;                // G held as gp x gp (gp = KMAX of the kernel), zero padded
  int pitch;             // resident: column pitch (RP padded to 8)
  int resume;            // 1: the H-side state saved by the previous launch is current (no prologue)
  // optional copies of the final Grams for the caller (nullptr: none): H^T H and W^T W in FP64
  // and rounded to FP32
  double* Gd_h;
  double* Gd_w;
  float* Gf_h;
  float* Gf_w;
};

// Final sums: l*k entries of U^T F, k*k of F^T F, then tr, dd.
__host__ __device__ inline int le_entries(int l, int k) { return l * k + k * k + 2; }
// State of a half: M (l x k4, lambda-scaled), G (gp x gp), 1 / (G_ii + alpha) (gp), zero padded.
__host__ __device__ inline int le_state_floats(int l, int k, int gp) { return l * ((k + 3) & ~3) + gp * gp + gp; }
__host__ __device__ inline int le_gp(int k) {
  return k <= 8 ? 8 : k <= 16 ? 16 : k <= 20 ? 20 : k <= 24 ? 24 : k <= 32 ? 32 : k <= 48 ? 48 : 64;
}

// 4x4 tiles: (l4/4) x (k4/4) tiles of U^T F, then the upper-triangular tiles
// (bi <= bj, row-major) of F^T F.  A partial record stores tile t's 16
// entries at [16 t, 16 t + 16) and then tr, tr_lo, dd, dd_lo.
__host__ __device__ inline int le_tile_count(int l, int k) {
  const int kt = ((k + 3) & ~3) / 4, lt = ((l + 3) & ~3) / 4;
  return lt * kt + kt * (kt + 1) / 2;
}
__host__ __device__ inline int le_rec_entries(int l, int k) { return 16 * le_tile_count(l, k) + 4; }
__host__ __device__ inline int le_tri_index(int bi, int bj, int kt) { return bi * kt - bi * (bi - 1) / 2 + (bj - bi); }

__device__ __forceinline__ void le_tri(int g, int kt, int& bi, int& bj) {
  int b = 0;
  while (g >= kt - b) {
    g -= kt - b;
    ++b;
  }
  bi = b;
  bj = b + g;
}

// Double-float accumulation (Dekker 1971, two-sum): (hi, lo) holds hi + lo.
__device__ __forceinline__ void df_add(float& hi, float& lo, float h2, float l2) {
  const float s = hi + h2;
  const float bb = s - hi;
  const float t = ((hi - (s - bb)) + (h2 - bb)) + lo + l2;
  hi = s + t;
  lo = t - (hi - s);
}

// Kahan-compensated FP32 accumulation: the total is s - c.
__device__ __forceinline__ void le_kahan(float& s, float& c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Tiles spread over the block's threads; with fewer tiles than threads, up
// to LE_MAXRG row groups of threads split the rows, each group writing its
// own record.
constexpr int LE_MAXRG = 4;
__host__ __device__ inline int le_row_groups(int l, int k) {
  const int T = le_tile_count(l, k);
  return T >= LE_THREADS ? 1 : (LE_THREADS / T < LE_MAXRG ? LE_THREADS / T : LE_MAXRG);
}
struct LeTiles {
  int kt, tm, T, RG, my_rg, TPT;
};

__device__ __forceinline__ LeTiles le_tiles(int l4, int k4) {
  LeTiles t;
  t.kt = k4 / 4;
  t.tm = (l4 / 4) * t.kt;
  t.T = t.tm + t.kt * (t.kt + 1) / 2;
  t.RG = t.T >= LE_THREADS ? 1 : min(LE_MAXRG, LE_THREADS / t.T);
  t.my_rg = t.T >= LE_THREADS ? 0 : (int)threadIdx.x / t.T;
  t.TPT = (t.T + LE_THREADS - 1) / LE_THREADS;  // <= 3 for l <= 96, k <= 64
  return t;
}

__device__ __forceinline__ int le_tile_of(const LeTiles& tl, int t) {
  return (tl.T >= LE_THREADS) ? (int)threadIdx.x + t * LE_THREADS : (int)threadIdx.x % tl.T;
}

// Operand block rows of tile `tile`: A (U columns or F columns) and B (F columns).
__device__ __forceinline__ void le_tile_rows(const LeTiles& tl, int tile, int& a_blk, int& b_blk, bool& a_is_u) {
  if (tile < tl.tm) {
    a_is_u = true;
    a_blk = tile / tl.kt;
    b_blk = tile % tl.kt;
  } else {
    a_is_u = false;
    le_tri(tile - tl.tm, tl.kt, a_blk, b_blk);
  }
}

__device__ __forceinline__ void le_clear(float (&acc)[3][16], float (&cmp)[3][16]) {
#pragma unroll
  for (int t = 0; t < 3; ++t)
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[t][e] = cmp[t][e] = 0.f;
}

// Compensated totals -> plain totals (s - c, rounded once) before the record is written.
__device__ __forceinline__ void le_settle(float (&acc)[3][16], const float (&cmp)[3][16]) {
#pragma unroll
  for (int t = 0; t < 3; ++t)
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[t][e] -= cmp[t][e];
}

// Write this CTA's record: the row groups' tile sums (Kahan-settled FP32) are
// staged in shared memory and added in row-group order, then stored as float4
// runs; the CTA's tr, dd (double-float, reduced over the block) fill the last
// four floats.  One record per CTA.
__device__ __forceinline__ void le_finish(const LaiArgs& a, const LeTiles& tl, const float (&acc)[3][16],
                                          float* red, float2 trv, float2 ddv) {
  const int EP = le_rec_entries(a.l, a.k);
  float* rec = a.part + (size_t)blockIdx.x * EP;
  if (tl.RG == 1) {
    for (int t = 0; t < tl.TPT; ++t) {
      const int tile = le_tile_of(tl, t);
      if (tile < tl.T && tl.my_rg == 0) {  // threads past the row groups hold no sums
        float4* rec4 = reinterpret_cast<float4*>(rec);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float v[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            v[e] = 0.f;
#pragma unroll
            for (int w = 0; w < 3; ++w)
              if (w == t) v[e] = acc[w][4 * u + e];
          }
          rec4[tile * 4 + u] = make_float4(v[0], v[1], v[2], v[3]);
        }
      }
    }
  } else {
    // TPT == 1: thread (rg, tile) holds acc[0]; RG * T * 16 <= 16 * LE_THREADS floats fit red
    const int tile = le_tile_of(tl, 0);
    if (tile < tl.T && tl.my_rg < tl.RG) {
      float4* dst = reinterpret_cast<float4*>(red + ((size_t)tl.my_rg * tl.T + tile) * 16);
#pragma unroll
      for (int u = 0; u < 4; ++u) dst[u] = make_float4(acc[0][4 * u], acc[0][4 * u + 1], acc[0][4 * u + 2],
                                                       acc[0][4 * u + 3]);
    }
    __syncthreads();
    const int nq = tl.T * 4;  // float4 runs of the record's tiles
    for (int q = threadIdx.x; q < nq; q += LE_THREADS) {
      float4 s4 = reinterpret_cast<const float4*>(red)[q];
      for (int g = 1; g < tl.RG; ++g) {
        const float4 v = reinterpret_cast<const float4*>(red)[(size_t)g * nq + q];
        s4.x += v.x;
        s4.y += v.y;
        s4.z += v.z;
        s4.w += v.w;
      }
      reinterpret_cast<float4*>(rec)[q] = s4;
    }
    __syncthreads();  // red is reused below
  }
  // tr, dd: warp xor trees, then one barrier and warp 0
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    df_add(trv.x, trv.y, __shfl_xor_sync(0xffffffffu, trv.x, o), __shfl_xor_sync(0xffffffffu, trv.y, o));
    df_add(ddv.x, ddv.y, __shfl_xor_sync(0xffffffffu, ddv.x, o), __shfl_xor_sync(0xffffffffu, ddv.y, o));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[4 * wid + 0] = trv.x;
    red[4 * wid + 1] = trv.y;
    red[4 * wid + 2] = ddv.x;
    red[4 * wid + 3] = ddv.y;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = LE_THREADS / 32;
    float th = lane < nw ? red[4 * lane + 0] : 0.f, tl2 = lane < nw ? red[4 * lane + 1] : 0.f;
    float dh = lane < nw ? red[4 * lane + 2] : 0.f, dl = lane < nw ? red[4 * lane + 3] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      df_add(th, tl2, __shfl_xor_sync(0xffffffffu, th, o), __shfl_xor_sync(0xffffffffu, tl2, o));
      df_add(dh, dl, __shfl_xor_sync(0xffffffffu, dh, o), __shfl_xor_sync(0xffffffffu, dl, o));
    }
    if (lane == 0) reinterpret_cast<float4*>(rec + EP - 4)[0] = make_float4(th, tl2, dh, dl);
  }
  __syncthreads();  // red is reused by the caller
}

// Sliced reduction of all records (one per CTA).  CTA c owns a contiguous run
// of record positions (whole float4 columns); each warp reduces one column at
// a time: lane j sums the column's float4 in records j, j + 32, ... in
// double-float (all its loads in flight together), then a fixed xor tree over
// the lanes adds the 32 partial sums (deterministic).  Each position is mapped
// back to its entry: the FP64 sums go to fin[side] (both (i, j) and (j, i) for
// F^T F), the FP32 state of the next half to state[side], and after the H half
// of sweep t >= 0 this CTA's objective share to objp[t].
constexpr int LE_BATCH = 8;
constexpr int LE_STASH = 512;  // slice positions whose W-half sums stay in shared memory

// stash: this CTA's W-half sums of its slice (positions c0 + i), written by the
// side-0 reduction and read by the side-1 one (same slicing), when the slice
// fits LE_STASH; lam_s: lambda in shared memory.  Both keep the H half's
// objective terms off dependent global loads.
__device__ __forceinline__ void le_reduce_slice(const LaiArgs& a, int side, int t, double* shd, double* stash,
                                                const double* lam_s) {
  const int k = a.k, l = a.l, k4 = (k + 3) & ~3, gp = a.gp;
  const int E = le_entries(l, k), EP = le_rec_entries(l, k), SL = le_state_floats(l, k, gp);
  const int lk = l * k, kt = k4 / 4, tm = (((l + 3) & ~3) / 4) * kt;
  const unsigned nrec = gridDim.x;
  double* fin = a.fin + side * E;
  float* st = a.state + side * SL;
  // positions per CTA, a multiple of 4: the float4 columns and the hi/lo pairs of
  // tr and dd (the last column, EP a multiple of 4) never straddle two CTAs
  const int per = ((EP + gridDim.x - 1) / gridDim.x + 3) & ~3;
  const int c0 = blockIdx.x * per, c1 = min(EP, c0 + per);
  const bool stashed = per <= LE_STASH;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double share = 0.0;
  for (int col = c0 + 4 * wid; col < c1; col += 4 * (LE_THREADS / 32)) {
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    const float* src = a.part + col;
    for (unsigned q0 = lane; q0 < nrec; q0 += 32u * LE_BATCH) {
      float4 v[LE_BATCH];
#pragma unroll
      for (int u = 0; u < LE_BATCH; ++u) {
        const unsigned q = q0 + 32u * u;
        v[u] = q < nrec ? __ldcg(reinterpret_cast<const float4*>(src + (size_t)q * EP))
                        : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < LE_BATCH; ++u) {
        df_add(hi[0], lo[0], v[u].x, 0.f);
        df_add(hi[1], lo[1], v[u].y, 0.f);
        df_add(hi[2], lo[2], v[u].z, 0.f);
        df_add(hi[3], lo[3], v[u].w, 0.f);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int e = 0; e < 4; ++e)
        df_add(hi[e], lo[e], __shfl_xor_sync(0xffffffffu, hi[e], o), __shfl_xor_sync(0xffffffffu, lo[e], o));
    // every lane holds the column's sums after the xor tree: lanes 0..3 map one
    // position each (FP64 is a narrow pipe on this part: four short chains in
    // parallel instead of one long one)
    if (lane >= 4) continue;
    if (col == EP - 4) {
      // tr and dd: hi/lo pairs of double-float sums
      if (lane != 0) continue;
      const double tr = (double)hi[0] + (double)lo[0] + (double)hi[1] + (double)lo[1];
      const double dd = (double)hi[2] + (double)lo[2] + (double)hi[3] + (double)lo[3];
      fin[lk + k * k] = tr;
      fin[lk + k * k + 1] = dd;
      if (side == 1 && t >= 0) share += -2.0 * tr + a.alpha_d * dd;
      continue;
    }
    {
      const int e = lane;
      const float he = e == 0 ? hi[0] : e == 1 ? hi[1] : e == 2 ? hi[2] : hi[3];
      const float le = e == 0 ? lo[0] : e == 1 ? lo[1] : e == 2 ? lo[2] : lo[3];
      const int idx = col + e;
      const double v = (double)he + (double)le;
      double v_w = 0.0;  // the W half's sum at this position (side 1)
      if (stashed) {
        if (side == 0) stash[idx - c0] = v;
        else v_w = stash[idx - c0];
      }
      const int tile = idx >> 4, p = (idx >> 2) & 3, q = idx & 3;
      if (tile < tm) {
        const int i = 4 * (tile / kt) + p, j = 4 * (tile % kt) + q;
        if (i < l && j < k) {
          fin[i * k + j] = v;
          st[i * k4 + j] = (float)(lam_s[i] * v);
          // the H half's rows used M~ = fl32(lambda U^T W), rounded once and shared by
          // every row, so tr(H^T U M~) misses the exact tr by sum (U^T H) .* (M~ - M):
          // added back here, where U^T H (this sum, v) and U^T W are in FP64
          if (side == 1 && t >= 0) {
            const double m = lam_s[i] * (stashed ? v_w : __ldcg(a.fin + i * k + j));
            share += 2.0 * v * ((double)(float)m - m);
          }
        }
      } else {
        int bi, bj;
        le_tri(tile - tm, kt, bi, bj);
        const int i = 4 * bi + p, j = 4 * bj + q;
        if (i < k && j < k) {
          fin[lk + i * k + j] = v;
          fin[lk + j * k + i] = v;
          st[l * k4 + i * gp + j] = (float)v;
          st[l * k4 + j * gp + i] = (float)v;
          if (i == j) st[l * k4 + gp * gp + i] = 1.0f / ((float)v + a.alpha);
          // (W^T W)_ij (H^T H)_ij over all (i, j): an off-diagonal tile holds each pair once
          if (side == 1 && t >= 0)
            share += (bi == bj ? 1.0 : 2.0) * (stashed ? v_w : __ldcg(a.fin + lk + i * k + j)) * v;
        }
      }
    }
  }
  if (side == 1 && t >= 0) {
    share = block_sum(share, shd);
    if (threadIdx.x == 0 && t < a.obj_cap)
      a.objp[(size_t)t * gridDim.x + blockIdx.x] = share + (blockIdx.x == 0 ? a.normX2[0] : 0.0);
  }
}

// The state written by le_reduce_slice for `side`, into shared memory [Ms | Gs | inv].
__device__ __forceinline__ void le_load_state(const LaiArgs& a, int side, float* Ms) {
  const int SL = le_state_floats(a.l, a.k, a.gp), SL4 = SL / 4;
  const float4* src = reinterpret_cast<const float4*>(a.state + side * SL);
  float4* dst = reinterpret_cast<float4*>(Ms);
#pragma unroll 4
  for (int e = threadIdx.x; e < SL4; e += LE_THREADS) dst[e] = __ldcg(src + e);
  __syncthreads();
}

// After the last sweep: obj[t] = sum of the CTAs' shares (CTA c takes sweeps c, c + grid, ...).
__device__ __forceinline__ void le_objective_sums(const LaiArgs& a, double* shd) {
  for (int t = blockIdx.x; t < a.nsweeps && t < a.obj_cap; t += gridDim.x) {
    double s = 0.0;
    for (unsigned q = threadIdx.x; q < gridDim.x; q += LE_THREADS) s += __ldcg(a.objp + (size_t)t * gridDim.x + q);
    s = block_sum(s, shd);
    if (threadIdx.x == 0) a.obj[t] = s;
  }
}

// ------------------------------------------------------------ resident rows

// Column pitch: a multiple of 8 with 32 floats to spare, so that a column
// shifted by its skew (up to 28 floats) never reaches the next one.
__host__ __device__ inline int le_pitch(int rp) { return ((rp + 7) & ~7) + 32; }
__host__ __device__ inline size_t le_resident_floats(int l, int k, int rp) {
  const int l4 = (l + 3) & ~3, k4 = (k + 3) & ~3;
  return (size_t)le_state_floats(l, k, le_gp(k)) + (size_t)(l4 + 3 * k4) * le_pitch(rp) + (size_t)16 * LE_THREADS;
}

template <int KMAX>
__global__ void __launch_bounds__(LE_THREADS, 1) lai_resident_kernel(LaiArgs a) {
  extern __shared__ __align__(16) float sm[];
  const int k = a.k, l = a.l, RP = a.tile_rows, rq = RP / 4, P = a.pitch;
  const int l4 = (l + 3) & ~3, k4 = (k + 3) & ~3, k4q = k4 / 4;
  const int E = le_entries(l, k);
  float* Ms = sm;               // l x k4, lambda-scaled, zero padded (float4 rows)
  float* Gs = Ms + l * k4;      // KMAX x KMAX, zero padded (symmetric: row i = column i)
  float* inv = Gs + KMAX * KMAX;  // KMAX
  float* Ut = inv + KMAX;      // l4 columns: the CTA's rows of U
  float* Wt = Ut + l4 * P;     // k4 columns
  float* Ht = Wt + k4 * P;     // k4 columns
  float* Yt = Ht + k4 * P;     // k4 columns: Y = U M of the current half
  float* red = Yt + k4 * P;    // 16 x LE_THREADS
  auto col = [P](int c) { return c * P + ((c >> 2) & 7) * 4; };  // start of column c
  __shared__ double shd[32];
  __shared__ double stash[LE_STASH];
  __shared__ double lam_s[96];
  for (int i = threadIdx.x; i < a.l; i += LE_THREADS) lam_s[i] = a.lam[i];

  const int tid = threadIdx.x;
  const int64_t r0 = (a.n * blockIdx.x) / gridDim.x;
  const int R = (int)((a.n * (blockIdx.x + 1)) / gridDim.x - r0);
  const LeTiles tl = le_tiles(l4, k4);
  float acc[3][16], cmp[3][16];

  // prologue: the CTA's rows, transposed into shared memory (pads stay zero)
  for (int e = tid; e < (l4 + 3 * k4) * P; e += LE_THREADS) Ut[e] = 0.f;
  __syncthreads();
  {
    const float* Ug = a.U + r0 * l;
    for (int e = tid; e < R * l; e += LE_THREADS) {
      const int r = e / l, c = e - r * l;
      Ut[col(c) + r] = __ldg(Ug + e);
    }
    const float* Wg = a.W + r0 * k;
    const float* Hg = a.H + r0 * k;
    for (int e = tid; e < R * k; e += LE_THREADS) {
      const int r = e / k, c = e - r * k;
      Wt[col(c) + r] = Wg[e];
      Ht[col(c) + r] = Hg[e];
    }
  }
  __syncthreads();

  // U^T F and F^T F over the CTA's rows, four rows per float4 step
  auto accumulate = [&](const float* Fu) {
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      if (t >= tl.TPT) break;
      const int tile = le_tile_of(tl, t);
      if (tile < tl.T && tl.my_rg < tl.RG) {
        int ab, bb;
        bool au;
        le_tile_rows(tl, tile, ab, bb, au);
        const float* A = au ? Ut : Fu;
        const float4* Ap[4];
        const float4* Bp[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          Ap[p] = reinterpret_cast<const float4*>(A + col(4 * ab + p));
          Bp[p] = reinterpret_cast<const float4*>(Fu + col(4 * bb + p));
        }
#pragma unroll 2
        for (int c = tl.my_rg; c < rq; c += tl.RG) {
          float4 av[4], bv[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            av[p] = Ap[p][c];
            bv[p] = Bp[p][c];
          }
#pragma unroll
          for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              float s = av[p].x * bv[q].x;
              s = fmaf(av[p].y, bv[q].y, s);
              s = fmaf(av[p].z, bv[q].z, s);
              s = fmaf(av[p].w, bv[q].w, s);
              le_kahan(acc[t][p * 4 + q], cmp[t][p * 4 + q], s);
            }
        }
      }
    }
  };

  // prologue: state of the H side (the W-update uses M = Lambda U^T H, G = H^T H),
  // unless the previous launch saved it
  unsigned epoch = 0;
  if (!a.resume) {
    le_clear(acc, cmp);
    accumulate(Ht);
    le_settle(acc, cmp);
    le_finish(a, tl, acc, red, make_float2(0.f, 0.f), make_float2(0.f, 0.f));
    if (!grid_sync_bounded(a.bar, a.err, epoch)) return;
    le_reduce_slice(a, 1, -1, shd, stash, lam_s);
    if (!grid_sync_bounded(a.bar, a.err, epoch)) return;
  }
  le_load_state(a, 1, Ms);

  const float4* Ms4 = reinterpret_cast<const float4*>(Ms);
  const float4* Gs4 = reinterpret_cast<const float4*>(Gs);

  for (int t = 0; t < a.nsweeps; ++t) {
    for (int side = 0; side < 2; ++side) {
      float* Fu = side ? Ht : Wt;
      const float* Fx = side ? Wt : Ht;
      // Y = U M for the CTA's rows: 4 rows x 4 columns per thread (float4 of U
      // down a column, broadcast float4 of a row of M)
      for (int q = tid; q < rq * k4q; q += LE_THREADS) {
        const int rb = q % rq, cb = q / rq;
        float y[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) y[e] = 0.f;
#pragma unroll 2
        for (int p = 0; p < l; ++p) {
          const float4 u = reinterpret_cast<const float4*>(Ut + col(p))[rb];
          const float4 m = Ms4[p * k4q + cb];
          const float uv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            y[i * 4 + 0] = fmaf(uv[i], m.x, y[i * 4 + 0]);
            y[i * 4 + 1] = fmaf(uv[i], m.y, y[i * 4 + 1]);
            y[i * 4 + 2] = fmaf(uv[i], m.z, y[i * 4 + 2]);
            y[i * 4 + 3] = fmaf(uv[i], m.w, y[i * 4 + 3]);
          }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
          reinterpret_cast<float4*>(Yt + col(4 * cb + j))[rb] = make_float4(y[j], y[4 + j], y[8 + j], y[12 + j]);
      }
      __syncthreads();
      float2 trv = make_float2(0.f, 0.f), ddv = make_float2(0.f, 0.f);
      bool bad = false;
      for (int r = tid; r < R; r += LE_THREADS) {
        float y[KMAX];
#pragma unroll
        for (int c = 0; c < KMAX; ++c) y[c] = c < k ? Yt[col(c) + r] : 0.f;
        bad |= hals_row_update<KMAX>(
            y, a.alpha, k, Gs4, inv, [&](int i) { return Fx[col(i) + r]; },
            [&](int j) -> float& { return Fu[col(j) + r]; }, trv, ddv);
      }
      if (bad) set_error(a.err, ERR_NAN);
      __syncthreads();
      le_clear(acc, cmp);
      accumulate(Fu);
      le_settle(acc, cmp);
      le_finish(a, tl, acc, red, trv, ddv);
      if (!grid_sync_bounded(a.bar, a.err, epoch)) return;
      le_reduce_slice(a, side, t, shd, stash, lam_s);
      if (!grid_sync_bounded(a.bar, a.err, epoch)) return;
      le_load_state(a, side, Ms);
    }
  }
  // epilogue: the CTA's rows of W and H back to global memory
  {
    float* Wg = a.W + r0 * k;
    float* Hg = a.H + r0 * k;
    for (int e = tid; e < R * k; e += LE_THREADS) {
      const int r = e / k, c = e - r * k;
      Wg[e] = Wt[col(c) + r];
      Hg[e] = Ht[col(c) + r];
    }
  }
  // Grams after the last sweep for the handle's state: [0] = H^T H, [1] = W^T W
  if (blockIdx.x == 0)
    for (int e = tid; e < k * k; e += LE_THREADS) {
      const double gh = __ldcg(a.fin + E + l * k + e), gw = __ldcg(a.fin + l * k + e);
      a.Gout[e] = gh;
      a.Gout[k * k + e] = gw;
      if (a.Gd_h) {
        a.Gd_h[e] = gh;
        a.Gd_w[e] = gw;
        a.Gf_h[e] = (float)gh;
        a.Gf_w[e] = (float)gw;
      }
    }
  le_objective_sums(a, shd);
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
  float* Gs = Ms + l * k4;               // KMAX x KMAX, zero padded (symmetric: row i = column i)
  float* inv = Gs + KMAX * KMAX;         // KMAX
  float* Us = inv + KMAX;                // TR x us: U rows of the tile
  float* Fx = Us + TR * us;              // TR x fs: fixed factor rows
  float* Fu = Fx + TR * fs;              // TR x fs: rows being updated
  float* red = Fu + TR * fs;             // 16 x LE_THREADS: row-group combine
  __shared__ double shd[32];
  __shared__ double stash[LE_STASH];
  __shared__ double lam_s[96];
  for (int i = threadIdx.x; i < a.l; i += LE_THREADS) lam_s[i] = a.lam[i];

  const int tid = threadIdx.x;
  const int64_t r0 = (a.n * blockIdx.x) / gridDim.x;
  const int64_t r1 = (a.n * (blockIdx.x + 1)) / gridDim.x;
  const LeTiles tl = le_tiles(l4, k4);
  float acc[3][16], cmp[3][16];

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
    for (int t = 0; t < 3; ++t) {
      if (t >= tl.TPT) break;
      const int tile = le_tile_of(tl, t);
      if (tile < tl.T && tl.my_rg < tl.RG) {
        int ab, bb;
        bool au;
        le_tile_rows(tl, tile, ab, bb, au);
        const float* A = au ? Us : Fu;
        const int sa = au ? us : fs, ai = 4 * ab, bj = 4 * bb;
        // FMA sums over up to four of the group's rows, folded into the Kahan totals
        for (int r4 = tl.my_rg; r4 < rows; r4 += 4 * tl.RG) {
          float part[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) part[e] = 0.f;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int rr = r4 + u * tl.RG;
            if (rr < rows) {
              float av[4], bv[4];
#pragma unroll
              for (int p = 0; p < 4; ++p) {
                av[p] = A[rr * sa + ai + p];
                bv[p] = Fu[rr * fs + bj + p];
              }
#pragma unroll
              for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) part[p * 4 + q] = fmaf(av[p], bv[q], part[p * 4 + q]);
            }
          }
#pragma unroll
          for (int e = 0; e < 16; ++e) le_kahan(acc[t][e], cmp[t][e], part[e]);
        }
      }
    }
  };

  // prologue: state of the H side (the W-update uses M = Lambda U^T H, G = H^T H),
  // unless the previous launch saved it
  unsigned epoch = 0;
  if (!a.resume) {
    le_clear(acc, cmp);
    for (int64_t b = r0; b < r1; b += TR) {
      const int rows = (int)min((int64_t)TR, r1 - b);
      stage(b, rows, nullptr, a.H);
      __syncthreads();
      accumulate(rows);
      __syncthreads();
    }
    le_settle(acc, cmp);
    le_finish(a, tl, acc, red, make_float2(0.f, 0.f), make_float2(0.f, 0.f));
    if (!grid_sync_bounded(a.bar, a.err, epoch)) return;
    le_reduce_slice(a, 1, -1, shd, stash, lam_s);
    if (!grid_sync_bounded(a.bar, a.err, epoch)) return;
  }
  le_load_state(a, 1, Ms);

  const float4* Ms4 = reinterpret_cast<const float4*>(Ms);
  const float4* Gs4 = reinterpret_cast<const float4*>(Gs);
  for (int t = 0; t < a.nsweeps; ++t) {
    for (int side = 0; side < 2; ++side) {
      float* Fupd = side ? a.H : a.W;
      const float* Ffix = side ? a.W : a.H;
      float2 trv = make_float2(0.f, 0.f), ddv = make_float2(0.f, 0.f);
      bool bad = false;
      le_clear(acc, cmp);
      for (int64_t b = r0; b < r1; b += TR) {
        const int rows = (int)min((int64_t)TR, r1 - b);
        stage(b, rows, Ffix, Fupd);
        __syncthreads();
        if (tid < rows) {
          const float* ur = Us + tid * us;
          const float* hr = Fx + tid * fs;
          float* wr = Fu + tid * fs;
          // Y_r = U_r M, float4 broadcast reads of M's rows
          float y[KMAX];
#pragma unroll
          for (int c = 0; c < KMAX; ++c) y[c] = 0.f;
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
          bad |= hals_row_update<KMAX>(
              y, a.alpha, k, Gs4, inv, [&](int i) { return hr[i]; }, [&](int j) -> float& { return wr[j]; }, trv,
              ddv);
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
      le_settle(acc, cmp);
      le_finish(a, tl, acc, red, trv, ddv);
      if (!grid_sync_bounded(a.bar, a.err, epoch)) return;
      le_reduce_slice(a, side, t, shd, stash, lam_s);
      if (!grid_sync_bounded(a.bar, a.err, epoch)) return;
      le_load_state(a, side, Ms);
    }
  }
  // Grams after the last sweep for the handle's state: [0] = H^T H, [1] = W^T W
  if (blockIdx.x == 0)
    for (int e = tid; e < k * k; e += LE_THREADS) {
      const double gh = __ldcg(a.fin + E + l * k + e), gw = __ldcg(a.fin + l * k + e);
      a.Gout[e] = gh;
      a.Gout[k * k + e] = gw;
      if (a.Gd_h) {
        a.Gd_h[e] = gh;
        a.Gd_w[e] = gw;
        a.Gf_h[e] = (float)gh;
        a.Gf_w[e] = (float)gw;
      }
    }
  le_objective_sums(a, shd);
}

// Workspace layout (each piece 256-byte aligned): barrier counter, fin, objective
// shares, records, state.
inline size_t le_align(size_t b) { return (b + 255) & ~(size_t)255; }

inline size_t streamed_smem(int l, int k, int tr) {
  const int l4 = (l + 3) & ~3, k4 = (k + 3) & ~3;
  return ((size_t)le_state_floats(l, k, le_gp(k)) + (size_t)tr * (l4 + 1) + (size_t)2 * tr * (k4 + 1) +
          (size_t)LE_THREADS * 16) * sizeof(float);
}

inline size_t smem_optin_limit() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  return v > 8192 ? (size_t)(v - 8192) : 0;  // room for the kernels' static shared memory (~5.2 KB)
}

template <int KMAX>
cudaError_t launch_engine(LaiArgs a, bool allow_resident, cudaStream_t st, cudaEvent_t ev0,
                                 cudaEvent_t ev1) {
  int grid = num_sms();
  if ((int64_t)grid > a.n) grid = (int)std::max<int64_t>(1, a.n);
  const int64_t rmax = (a.n + grid - 1) / grid;
  const int64_t rp = (rmax + 3) & ~3LL;
  const void* fn;
  size_t smem;
  if (allow_resident && rp <= (1 << 20) && le_resident_floats(a.l, a.k, (int)rp) * 4 <= smem_optin_limit()) {
    fn = (const void*)lai_resident_kernel<KMAX>;
    a.tile_rows = (int)rp;
    a.pitch = le_pitch((int)rp);
    smem = le_resident_floats(a.l, a.k, (int)rp) * 4;
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
  if (ev0 && (e = cudaEventRecord(ev0, st)) != cudaSuccess) return e;
  e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(LE_THREADS), params, smem, st);
  count_launches(1);
  if (e == cudaSuccess && ev1) e = cudaEventRecord(ev1, st);
  return e;
}

// Launchers of the kernels for G held as gp x gp (gp = le_gp(k)), one
// translation unit per group of widths so that they compile in parallel:
// gp in {8, 16, 20, 24} (lai_engine_narrow.cu) and {32, 48, 64}
// (lai_engine_wide.cu).
cudaError_t lai_engine_launch_narrow(int gp, const LaiArgs& a, bool allow_resident, cudaStream_t st,
                                     cudaEvent_t ev0, cudaEvent_t ev1);
cudaError_t lai_engine_launch_wide(int gp, const LaiArgs& a, bool allow_resident, cudaStream_t st,
                                   cudaEvent_t ev0, cudaEvent_t ev1);

}  // namespace symnmf
