// Column updates of one row of the regularized HALS rule (Eq. symhals_update2),
// shared by the full-X sweep kernel and the LAI sweep engine.
#pragma once

#include "common.cuh"

namespace symnmf {

// (hi, lo) += x by Dekker's two-sum (the running sum is hi + lo).
__device__ __forceinline__ void hr_df_add(float2& a, float x) {
  const float s = a.x + x;
  const float bb = s - a.x;
  a.y += (a.x - (s - bb)) + (x - bb);
  a.x = s;
}

// Column updates of one row (Eq. symhals_update2): `w` holds the row being
// updated and `y` its row of X F, both zero padded past k; the fixed row is
// read through `fx_at(i)` (called for i < k only).  G is KMAX x KMAX and
// 1 / (G_ii + alpha) KMAX long, zero padded: columns i >= k come out 0 and
// the loop has no data-dependent branches.  Four FMA chains per column.
// `done(i, h_i)` runs after column i is final.
template <int KMAX, class FXA, class DONE>
__device__ __forceinline__ void hals_row_columns(float (&w)[KMAX], const float (&y)[KMAX], float alpha, int k,
                                                 const float4* Gs4, const float* inv, FXA fx_at, DONE done) {
  // columns in order, each using the columns already updated (G symmetric: row i)
#pragma unroll
  for (int i = 0; i < KMAX; ++i) {
    const float hi = i < k ? fx_at(i) : 0.f;
    float ac[4] = {fmaf(alpha, hi, y[i]), 0.f, 0.f, 0.f};
#pragma unroll
    for (int j4 = 0; j4 < KMAX / 4; ++j4) {
      const float4 g = Gs4[i * (KMAX / 4) + j4];
      const float gv[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = 4 * j4 + q;
        if (j != i) ac[q] = fmaf(-w[j], gv[q], ac[q]);
      }
    }
    w[i] = fmaxf(((ac[0] + ac[1]) + (ac[2] + ac[3])) * inv[i], 0.f);
    done(i, hi);
  }
}

// One row with the row being updated read and written through the reference
// `fu_ref(j)` (shared memory in the LAI engine).  Adds the row's F_upd . Y and
// ||F_upd - F_fix||^2 to the double-float accumulators after the columns;
// returns true when a non-finite value appeared.
template <int KMAX, class FXA, class FUA>
__device__ __forceinline__ bool hals_row_update(const float (&y)[KMAX], float alpha, int k, const float4* Gs4,
                                                const float* inv, FXA fx_at, FUA fu_ref, float2& trv, float2& ddv) {
  float w[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; ++j) w[j] = j < k ? fu_ref(j) : 0.f;
  hals_row_columns<KMAX>(w, y, alpha, k, Gs4, inv, fx_at, [](int, float) {});
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
  hr_df_add(trv, t0 + t1);
  hr_df_add(ddv, d0 + d1);
  return bad;
}

// Shared-memory row stride (floats) of G for rows split over NS threads: each
// thread's KMAX / NS columns start 4 floats further on, so that the two halves
// read in one instruction sit in different banks.
template <int KMAX, int NS>
constexpr int hals_split_stride() {
  return NS > 1 ? NS * (KMAX / NS + 4) : KMAX;
}

// One row split over NS adjacent lanes (the lane pair `mask`), part p owning
// columns [p KMAX/NS, (p+1) KMAX/NS) of w in registers (zero padded past k)
// and reading its row of X F through `y_at(own index)` (zero past k).  Gp4 points at this part's columns of G with the diagonal zeroed (row
// stride hals_split_stride), so every lane sums -w_j G_ij over its own j and
// the parts' sums meet by one shuffle; the owner of column i then forms
// w_i = max(0, (y_i + alpha h_i - sum_{j != i} w_j G_ij) / (G_ii + alpha))
// (Eq. symhals_update2) with the fixed row's h_i from `fx_at(own index)`,
// called for i < k only.  Adds the part's F_upd . Y and ||F_upd - F_fix||^2
// to the double-float accumulators; returns true on a non-finite value.
template <int KMAX, int NS, class YA, class FXA>
__device__ __forceinline__ bool hals_row_split(float (&w)[KMAX / NS], YA y_at, float alpha, int k, int p,
                                               unsigned mask, const float4* Gp4, const float* inv, FXA fx_at,
                                               float2& trv, float2& ddv) {
  constexpr int KH = KMAX / NS;
  constexpr int RS4 = hals_split_stride<KMAX, NS>() / 4;
  bool bad = false;
  float t[2] = {0.f, 0.f}, d2[2] = {0.f, 0.f};
#pragma unroll
  for (int i = 0; i < KMAX; ++i) {
    float ac[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j4 = 0; j4 < KH / 4; ++j4) {
      const float4 g = Gp4[i * RS4 + j4];
      ac[0] = fmaf(-w[4 * j4 + 0], g.x, ac[0]);
      ac[1] = fmaf(-w[4 * j4 + 1], g.y, ac[1]);
      ac[2] = fmaf(-w[4 * j4 + 2], g.z, ac[2]);
      ac[3] = fmaf(-w[4 * j4 + 3], g.w, ac[3]);
    }
    float s = (ac[0] + ac[1]) + (ac[2] + ac[3]);
    if constexpr (NS > 1) s += __shfl_xor_sync(mask, s, 1);
    if (p == i / KH) {
      const int ii = i % KH;
      const float hi = i < k ? fx_at(ii) : 0.f;
      const float yi = y_at(ii);
      const float wi = fmaxf((yi + fmaf(alpha, hi, s)) * inv[i], 0.f);  // padded columns: inv = 0
      w[ii] = wi;
      if (!isfinite(wi)) bad = true;
      const float d = wi - hi;
      t[i & 1] = fmaf(wi, yi, t[i & 1]);
      d2[i & 1] = fmaf(d, d, d2[i & 1]);
    }
  }
  hr_df_add(trv, t[0] + t[1]);
  hr_df_add(ddv, d2[0] + d2[1]);
  return bad;
}

// The same rule for one row held by one thread, with the column loop rolled in
// blocks of BB columns so that the code stays small at large widths (the fully
// unrolled 64-column body overflows the instruction cache): before block b the
// registers w hold the row rotated left by b BB columns, so the block's columns
// are always w[0..BB) (static register indices); G is read from rows stored
// twice side by side (row stride 2 KMAX, diagonal zeroed), starting at column
// b BB, which lines G up with the rotated w.  After the last block w is back in
// order.  Same arithmetic per column as hals_row_split with NS = 1 (four FMA
// chains), summed in the rotated order.
template <int KMAX, int BB, class YA, class FXA>
__device__ __forceinline__ bool hals_row_rotating(float (&w)[KMAX], YA y_at, float alpha, int k, const float* Gd,
                                                  const float* inv, FXA fx_at, float2& trv, float2& ddv) {
  static_assert(KMAX % BB == 0 && BB % 4 == 0 && BB % 2 == 0, "blocks of whole float4 runs");
  bool bad = false;
  float t[2] = {0.f, 0.f}, d2[2] = {0.f, 0.f};
#pragma unroll 1
  for (int b = 0; b < KMAX / BB; ++b) {
#pragma unroll
    for (int ii = 0; ii < BB; ++ii) {
      const int i = b * BB + ii;
      const float4* g4 = reinterpret_cast<const float4*>(Gd + (size_t)i * 2 * KMAX + b * BB);
      float ac[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int j4 = 0; j4 < KMAX / 4; ++j4) {
        const float4 g = g4[j4];
        ac[0] = fmaf(-w[4 * j4 + 0], g.x, ac[0]);
        ac[1] = fmaf(-w[4 * j4 + 1], g.y, ac[1]);
        ac[2] = fmaf(-w[4 * j4 + 2], g.z, ac[2]);
        ac[3] = fmaf(-w[4 * j4 + 3], g.w, ac[3]);
      }
      const float s = (ac[0] + ac[1]) + (ac[2] + ac[3]);
      const float hi = i < k ? fx_at(i) : 0.f;
      const float yi = y_at(i);
      const float wi = fmaxf((yi + fmaf(alpha, hi, s)) * inv[i], 0.f);  // padded columns: inv = 0
      w[ii] = wi;
      if (!isfinite(wi)) bad = true;
      const float d = wi - hi;
      t[ii & 1] = fmaf(wi, yi, t[ii & 1]);
      d2[ii & 1] = fmaf(d, d, d2[ii & 1]);
    }
    float head[BB];
#pragma unroll
    for (int q = 0; q < BB; ++q) head[q] = w[q];
#pragma unroll
    for (int j = 0; j < KMAX - BB; ++j) w[j] = w[j + BB];
#pragma unroll
    for (int q = 0; q < BB; ++q) w[KMAX - BB + q] = head[q];
  }
  hr_df_add(trv, t[0] + t[1]);
  hr_df_add(ddv, d2[0] + d2[1]);
  return bad;
}

}  // namespace symnmf
