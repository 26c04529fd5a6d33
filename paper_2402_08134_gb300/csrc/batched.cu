// Batched grouped SymNMF: many independent problems, each with R random
// restarts stacked as extra factor columns (F_p = [F_p^(1) ... F_p^(R)],
// n_p x R k_p), so that one pass over X_p serves every restart.
//
// One sweep = per half: one grouped tcgen05 product launch over the
// concatenated (problem, row tile, k block) iteration space of all problems,
// one grouped reduction, one grouped HALS launch (per-restart Grams), one
// grouped Gram launch, and (H half) one objective launch.  The sweep body is
// recorded once as a CUDA graph and replayed.  The grouped product's pipeline
// depth and CTAs per SM are chosen at the first sweep by timing the
// candidates (the library's own autotuner).
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/symnmf.h"
#include "common.cuh"
#include "hals_row.cuh"
#include "handle.h"
#include "kernels.h"
#include "tc_common.cuh"

namespace symnmf {

constexpr int GB_BN = 128;  // widest stacked factor (restarts x k)
constexpr int GB_MAXR = 8;  // most restarts per problem

struct __align__(64) GroupProb {
  CUtensorMap tmA;
  CUtensorMap tmB;
  long long it_off;
  long long tile_off;
  int kblocks, mtiles, bn, pad;
};

struct HalsProb {
  long long f_off;     // factor / Y offset (floats)
  long long g_off;     // Gram offset (R*k*k per problem)
  long long row_off;   // first global row
  long long tile_off;  // first 64-row tile (HALS) / 256-row chunk (Gram) handled below
  long long chunk_off;
  long long gp_off;    // padded FP32 Grams and inverses: R (KM^2 + KM), KM = k padded to 8/16/24/32
  int n, k, R, pr_off;  // pr_off: first (problem, restart) slot
  double alpha;
};

// ------------------------------------------------------- grouped product

template <int STAGES>
__global__ void __launch_bounds__(TC_THREADS, 1)
    grouped_tc_kernel(const GroupProb* __restrict__ probs, int nprob, long long total_iters,
                      float* __restrict__ partials, int max_segs, unsigned* err) {
  constexpr int A_BYTES = TC_BM * TC_ROW_BYTES;
  constexpr int B_BYTES = GB_BN * TC_ROW_BYTES;
  constexpr uint32_t TMEM_COLS = 2 * GB_BN;
  constexpr uint32_t IDESC0 = make_idesc<false>(TC_BM, 8) & ~(0x3Fu << 17);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_BYTES;
  uint64_t* full = (uint64_t*)(sB + STAGES * B_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* done = tempty + 2;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long it0 = ((long long)blockIdx.x * total_iters) / gridDim.x;
  const long long it1 = ((long long)(blockIdx.x + 1) * total_iters) / gridDim.x;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 4);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  // problem containing iteration it0
  int p0 = 0;
  while (p0 + 1 < nprob && probs[p0 + 1].it_off <= it0) ++p0;

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, issued_mask = 0, last_parity = 0;
      int p = p0, acquired = -1;
      for (long long it = it0; it < it1; ++it) {
        while (p + 1 < nprob && it >= probs[p + 1].it_off) ++p;
        const GroupProb* P = probs + p;
        if (acquired != p) {
          tensormap_acquire(&P->tmA);
          tensormap_acquire(&P->tmB);
          acquired = p;
        }
        const int kb_n = P->kblocks;
        const long long local = it - P->it_off;
        const int tile = (int)(local / kb_n);
        const int kb = (int)(local - (long long)tile * kb_n);
        if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag)) {
          *abort_flag = 1;
          set_error(err, ERR_TIMEOUT);
          break;
        }
        mbar_expect_tx(&full[stage], A_BYTES + P->bn * TC_ROW_BYTES);
        tma_load_2d(sA + stage * A_BYTES, &P->tmA, kb * 64, tile * TC_BM, &full[stage]);
        tma_load_2d(sB + stage * B_BYTES, &P->tmB, kb * 64, 0, &full[stage]);
        issued_mask |= 1u << stage;
        last_parity = (last_parity & ~(1u << stage)) | (phase << stage);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
      for (int s = 0; s < STAGES; ++s)
        if (issued_mask >> s & 1u) {
          volatile int no_abort = 0;
          mbar_wait(&full[s], (last_parity >> s) & 1u, &no_abort);
        }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int stage = 0, seg = 0, p = p0;
      uint32_t phase = 0;
      bool ok = true;
      long long it = it0;
      while (ok && it < it1) {
        while (p + 1 < nprob && it >= probs[p + 1].it_off) ++p;
        const GroupProb* P = probs + p;
        const long long local = it - P->it_off;
        const long long tile = local / P->kblocks;
        const long long seg_end = min(it1, P->it_off + (tile + 1) * P->kblocks);
        const uint32_t idesc = IDESC0 | ((uint32_t)(P->bn >> 3) << 17);
        const int a = seg & 1;
        const uint32_t use = (uint32_t)(seg >> 1);
        if (!mbar_wait(&tempty[a], (use & 1u) ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(a * GB_BN);
        const long long seg_begin = it;
        for (; it < seg_end; ++it) {
          if (!mbar_wait(&full[stage], phase, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sA + stage * A_BYTES);
          const uint32_t b0 = smem_u32(sB + stage * B_BYTES);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            umma<false>(d, sw128_desc(a0 + ks * 32), sw128_desc(b0 + ks * 32), idesc,
                        (it > seg_begin || ks > 0) ? 1u : 0u);
          umma_commit(&empty[stage]);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        umma_commit(&tfull[a]);
        ++seg;
      }
      if (!ok) {
        *abort_flag = 1;
        set_error(err, ERR_TIMEOUT);
      }
      umma_commit(done);
      volatile int no_abort = 0;
      mbar_wait(done, 0, &no_abort);
    }
  } else {
    const int ew = warp & 3;
    const int row = ew * 32 + lane;
    int seg = 0, p = p0;
    long long it = it0;
    while (it < it1) {
      while (p + 1 < nprob && it >= probs[p + 1].it_off) ++p;
      const GroupProb* P = probs + p;
      const long long local = it - P->it_off;
      const long long tile = local / P->kblocks;
      const long long seg_end = min(it1, P->it_off + (tile + 1) * P->kblocks);
      const int bn = P->bn;
      const int a = seg & 1;
      const uint32_t use = (uint32_t)(seg >> 1);
      if (!mbar_wait(&tfull[a], use & 1u, abort_flag)) {
        *abort_flag = 1;
        set_error(err, ERR_TIMEOUT);
        break;
      }
      tc_fence_after();
      float* dst = partials + (((size_t)blockIdx.x * max_segs + seg) * TC_BM + row) * GB_BN;
      const uint32_t taddr = tmem_base + ((uint32_t)(ew * 32) << 16) + (uint32_t)(a * GB_BN);
#pragma unroll 1
      for (int c = 0; c < bn; c += 16) {
        float v[16];
        tmem_ld16(taddr + (uint32_t)c, v);
#pragma unroll
        for (int q = 0; q < 16; q += 4) *(float4*)(dst + c + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[a]);
      it = seg_end;
      ++seg;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                 : "memory");
}

struct ReduceTab {
  const long long* it_off;    // [nprob]
  const long long* tile_off;  // [nprob]
  const int* kblocks;         // [nprob]
  const long long* row_off;   // [nprob + 1]
  const long long* f_off;     // [nprob]
  const int* width;           // [nprob]
};

__device__ __forceinline__ int find_le(const long long* off, int count, long long x) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One block per global 128-row tile: the CTAs whose k ranges covered the tile
// (and the segment each stored it in) are found once, then the block sums
// their partial tiles in CTA order (deterministic) with float4 loads and
// writes the tile's rows of Y.
constexpr int GR_TABLE = 512;  // covering CTAs held in shared memory

__global__ void __launch_bounds__(256) grouped_reduce_kernel(ReduceTab tab, int nprob,
                                                             const float* __restrict__ partials, int max_segs,
                                                             long long total, int G, float* Y_all) {
  __shared__ int qs[GR_TABLE], segs[GR_TABLE];
  const long long gt = blockIdx.x;  // global tile
  const int p = find_le(tab.tile_off, nprob, gt);
  const long long tile = gt - tab.tile_off[p];
  const int kb = tab.kblocks[p], w = tab.width[p];
  const long long f_it = tab.it_off[p] + tile * kb, l_it = f_it + kb - 1;
  const long long c0 = ((f_it + 1) * G - 1) / total, c1 = ((l_it + 1) * G - 1) / total;
  const int nq = (int)(c1 - c0 + 1);
  auto seg_of = [&](long long q) {
    const long long itb = (q * total) / G;
    const int pb = find_le(tab.it_off, nprob, itb);
    return (int)(gt - (tab.tile_off[pb] + (itb - tab.it_off[pb]) / tab.kblocks[pb]));
  };
  for (int e = threadIdx.x; e < nq && e < GR_TABLE; e += blockDim.x) {
    qs[e] = (int)(c0 + e);
    segs[e] = seg_of(c0 + e);
  }
  __syncthreads();
  const long long r0 = tab.row_off[p] + tile * TC_BM;
  const int rows = (int)min((long long)TC_BM, tab.row_off[p + 1] - r0);
  float* Y = Y_all + tab.f_off[p] + tile * TC_BM * w;
  const bool vec = (w % 4) == 0 && (tab.f_off[p] % 4) == 0;
  const int w4 = (w + 3) / 4;
  for (int e = threadIdx.x; e < rows * w4; e += blockDim.x) {
    const int rr = e / w4, c = 4 * (e - rr * w4);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = 0; i < nq; ++i) {
      const long long q = i < GR_TABLE ? qs[i] : c0 + i;
      const int seg = i < GR_TABLE ? segs[i] : seg_of(c0 + i);
      const float4 v =
          __ldcs(reinterpret_cast<const float4*>(partials + ((q * max_segs + seg) * TC_BM + rr) * GB_BN + c));
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
    float* yr = Y + (long long)rr * w + c;
    if (vec) {
      *reinterpret_cast<float4*>(yr) = acc;
    } else {
      const float a4[4] = {acc.x, acc.y, acc.z, acc.w};
      for (int u = 0; u < 4 && c + u < w; ++u) yr[u] = a4[u];
    }
  }
}

// F^T of every problem packed as BF16, bn_p rows of ldp_p (zero padded): one
// block per 64-row tile (the HALS tiles), staged through shared memory so that
// both the reads of F rows and the writes of packed rows coalesce.
constexpr int GP_ROWS = 64, GP_PITCH = 128 + 1;

__global__ void __launch_bounds__(256) grouped_pack_kernel(const HalsProb* __restrict__ hp,
                                                           const long long* tile_off, int nprob,
                                                           const long long* pack_off, const int* bn,
                                                           const long long* ldp, const float* F_all,
                                                           __nv_bfloat16* out) {
  __shared__ float Fs[GP_ROWS * GP_PITCH];
  const int p = find_le(tile_off, nprob, (long long)blockIdx.x);
  const HalsProb P = hp[p];
  const int w = P.R * P.k;
  const long long base = (blockIdx.x - tile_off[p]) * GP_ROWS;
  const int rows = (int)min((long long)GP_ROWS, (long long)P.n - base);
  const float* F = F_all + P.f_off + base * w;
  for (int e = threadIdx.x; e < GP_ROWS * w; e += blockDim.x) {
    const int rr = e / w, c = e - rr * w;
    Fs[rr * GP_PITCH + c] = rr < rows ? F[e] : 0.f;
  }
  __syncthreads();
  const long long L = ldp[p];
  const int bnp = bn[p];
  __nv_bfloat16* o = out + pack_off[p];
  for (int e = threadIdx.x; e < bnp * GP_ROWS; e += blockDim.x) {
    const int c = e / GP_ROWS, rr = e - c * GP_ROWS;
    const long long i = base + rr;
    if (i < L) o[c * L + i] = __float2bfloat16_rn(c < w ? Fs[rr * GP_PITCH + c] : 0.f);
  }
}

// ----------------------------------------------------------- grouped HALS

constexpr int GH_ROWS = 64;

// (hi, lo) += (h2, l2), double-float (Dekker's two-sum)
__device__ __forceinline__ void gb_df_add(float& hi, float& lo, float h2, float l2) {
  const float s = hi + h2;
  const float bb = s - hi;
  lo += ((hi - (s - bb)) + (h2 - bb)) + l2;
  hi = s;
}

// The row work of one thread for a problem of width k <= KMAX (G rows padded to KMAX).
template <int KMAX>
__device__ __forceinline__ void grouped_hals_row(const HalsProb& P, int g, long long row, float* __restrict__ Fu_all,
                                                 const float* __restrict__ Ff_all, const float* __restrict__ Y_all,
                                                 const float* Gs, const float* inv, float alpha, unsigned* err,
                                                 float2& trv, float2& ddv) {
  const int k = P.k, RW = P.R * k;
  const long long o = P.f_off + row * RW + (long long)g * k;
  // z = Y + alpha F_fix (as the row routine forms it), so that only w and z
  // stay in registers; Y and F_fix are read again (cache hits) for the sums
  float w[KMAX], z[KMAX];
  if ((k & 3) == 0 && (o & 3) == 0) {  // 16-byte row segments
#pragma unroll
    for (int q = 0; q < KMAX / 4; ++q) {
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f), h = a, y = a;
      if (4 * q < k) {
        a = *reinterpret_cast<const float4*>(Fu_all + o + 4 * q);
        h = *reinterpret_cast<const float4*>(Ff_all + o + 4 * q);
        y = *reinterpret_cast<const float4*>(Y_all + o + 4 * q);
      }
      w[4 * q] = a.x, w[4 * q + 1] = a.y, w[4 * q + 2] = a.z, w[4 * q + 3] = a.w;
      z[4 * q] = fmaf(alpha, h.x, y.x), z[4 * q + 1] = fmaf(alpha, h.y, y.y);
      z[4 * q + 2] = fmaf(alpha, h.z, y.z), z[4 * q + 3] = fmaf(alpha, h.w, y.w);
    }
  } else {
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
      w[j] = j < k ? Fu_all[o + j] : 0.f;
      z[j] = j < k ? fmaf(alpha, Ff_all[o + j], Y_all[o + j]) : 0.f;
    }
  }
  hals_row_columns<KMAX>(w, z, 0.f, k, reinterpret_cast<const float4*>(Gs + g * KMAX * KMAX), inv + g * KMAX,
                         [](int) { return 0.f; }, [](int, float) {});
  bool bad = false;
  float t0 = 0.f, t1 = 0.f, d0 = 0.f, d1 = 0.f;
  if ((k & 3) == 0 && (o & 3) == 0) {  // 16-byte row segments
#pragma unroll
    for (int q = 0; q < KMAX / 4; ++q)
      if (4 * q < k) {
        const float4 y = *reinterpret_cast<const float4*>(Y_all + o + 4 * q);
        const float4 h = *reinterpret_cast<const float4*>(Ff_all + o + 4 * q);
        const float4 wq = make_float4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        *reinterpret_cast<float4*>(Fu_all + o + 4 * q) = wq;
        if (!isfinite(wq.x) || !isfinite(wq.y) || !isfinite(wq.z) || !isfinite(wq.w)) bad = true;
        t0 = fmaf(wq.x, y.x, t0);
        t1 = fmaf(wq.y, y.y, t1);
        t0 = fmaf(wq.z, y.z, t0);
        t1 = fmaf(wq.w, y.w, t1);
        const float4 d = make_float4(wq.x - h.x, wq.y - h.y, wq.z - h.z, wq.w - h.w);
        d0 = fmaf(d.x, d.x, d0);
        d1 = fmaf(d.y, d.y, d1);
        d0 = fmaf(d.z, d.z, d0);
        d1 = fmaf(d.w, d.w, d1);
      }
    if (bad) set_error(err, ERR_NAN);
    trv.x = t0 + t1;
    ddv.x = d0 + d1;
    return;
  }
  // Y and F_fix again (cache hits; restrict pointers let the loads run ahead of the stores)
#pragma unroll
  for (int j = 0; j < KMAX; ++j)
    if (j < k) {
      if (!isfinite(w[j])) bad = true;
      Fu_all[o + j] = w[j];
      const float yj = Y_all[o + j];
      const float d = w[j] - Ff_all[o + j];
      if (j & 1) {
        t1 = fmaf(w[j], yj, t1);
        d1 = fmaf(d, d, d1);
      } else {
        t0 = fmaf(w[j], yj, t0);
        d0 = fmaf(d, d, d0);
      }
    }
  if (bad) set_error(err, ERR_NAN);
  trv.x = t0 + t1;
  ddv.x = d0 + d1;
}

// The fixed factor's Grams as the HALS blocks read them: per problem R zero-padded
// KM x KM FP32 matrices with the diagonal zeroed, then R x KM values
// 1 / (G_ii + alpha) (0 past k).  One block per problem.
__device__ __forceinline__ int gh_km(int k) { return k <= 8 ? 8 : k <= 16 ? 16 : k <= 24 ? 24 : 32; }

__global__ void __launch_bounds__(256) grouped_gram_prep_kernel(const HalsProb* __restrict__ hp,
                                                                const double* __restrict__ Gd_all, float* Gp_all) {
  const HalsProb P = hp[blockIdx.x];
  const int k = P.k, R = P.R, KM = gh_km(k);
  float* Gp = Gp_all + P.gp_off;
  for (int e = threadIdx.x; e < R * (KM * KM + KM); e += blockDim.x) {
    float v;
    if (e < R * KM * KM) {
      const int g = e / (KM * KM), rem = e - g * KM * KM;
      const int i = rem / KM, j = rem - i * KM;
      v = (i < k && j < k && i != j) ? (float)Gd_all[P.g_off + (long long)g * k * k + i * k + j] : 0.f;
    } else {
      const int e2 = e - R * KM * KM, g = e2 / KM, i = e2 - g * KM;
      v = i < k ? 1.0f / ((float)Gd_all[P.g_off + (long long)g * k * k + i * k + i] + (float)P.alpha) : 0.f;
    }
    Gp[e] = v;
  }
}

// One thread per (row, restart): threads [g 64, g 64 + 64) of a block update
// restart g of the block's 64 rows (Eq. symhals_update2, columns in order, the
// shared row routine of the full-X kernel), instantiated for the block's
// problem width padded to 8, 16, 24 or 32.  The restart's prepared Gram is
// copied into shared memory (float4 broadcasts in the column loop).
// F_upd . Y and ||F_upd - F_fix||^2 are summed per row in FP32 and across rows
// in double-float (warp xor trees), one FP64 atomic per restart and block.
__global__ void __launch_bounds__(GH_ROWS * GB_MAXR) grouped_hals_kernel(const HalsProb* __restrict__ hp,
                                                                         const long long* tile_off, int nprob,
                                                                         float* Fu_all, const float* Ff_all,
                                                                         const float* Y_all, const float* Gp_all,
                                                                         double* part, unsigned* err) {
  extern __shared__ __align__(16) float sm[];
  __shared__ float2 wsum[2 * GB_MAXR * (GH_ROWS / 32)];
  const int p = find_le(tile_off, nprob, (long long)blockIdx.x);
  const HalsProb P = hp[p];
  const int k = P.k, R = P.R;
  const int KM = gh_km(k);
  const long long tile = blockIdx.x - tile_off[p];
  float* Gs = sm;                 // [R][KM][KM]
  float* inv = Gs + R * KM * KM;  // [R][KM]
  const float alpha = (float)P.alpha;
  const int tid = threadIdx.x;
  {
    const float4* src = reinterpret_cast<const float4*>(Gp_all + P.gp_off);
    float4* dst = reinterpret_cast<float4*>(sm);
    for (int e = tid; e < R * (KM * KM + KM) / 4; e += blockDim.x) dst[e] = src[e];
  }
  __syncthreads();
  const int g = tid / GH_ROWS, rr = tid - g * GH_ROWS;
  const long long row = tile * GH_ROWS + rr;
  float2 trv = make_float2(0.f, 0.f), ddv = make_float2(0.f, 0.f);
  if (g < R && row < P.n) {
    switch (KM) {
      case 8: grouped_hals_row<8>(P, g, row, Fu_all, Ff_all, Y_all, Gs, inv, alpha, err, trv, ddv); break;
      case 16: grouped_hals_row<16>(P, g, row, Fu_all, Ff_all, Y_all, Gs, inv, alpha, err, trv, ddv); break;
      case 24: grouped_hals_row<24>(P, g, row, Fu_all, Ff_all, Y_all, Gs, inv, alpha, err, trv, ddv); break;
      default: grouped_hals_row<32>(P, g, row, Fu_all, Ff_all, Y_all, Gs, inv, alpha, err, trv, ddv); break;
    }
  }
  // per restart: xor trees over the warp's 32 rows, then the block's row warps
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    gb_df_add(trv.x, trv.y, __shfl_xor_sync(0xffffffffu, trv.x, off), __shfl_xor_sync(0xffffffffu, trv.y, off));
    gb_df_add(ddv.x, ddv.y, __shfl_xor_sync(0xffffffffu, ddv.x, off), __shfl_xor_sync(0xffffffffu, ddv.y, off));
  }
  constexpr int WPR = GH_ROWS / 32;  // warps per restart
  const int wid = tid >> 5;
  if ((tid & 31) == 0) {
    wsum[2 * wid] = trv;
    wsum[2 * wid + 1] = ddv;
  }
  __syncthreads();
  if (tid < R) {
    float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
    for (int q = 0; q < WPR; ++q) {
      gb_df_add(a.x, a.y, wsum[2 * (tid * WPR + q)].x, wsum[2 * (tid * WPR + q)].y);
      gb_df_add(b.x, b.y, wsum[2 * (tid * WPR + q) + 1].x, wsum[2 * (tid * WPR + q) + 1].y);
    }
    atomicAdd(part + 2 * (P.pr_off + tid), (double)a.x + (double)a.y);
    atomicAdd(part + 2 * (P.pr_off + tid) + 1, (double)b.x + (double)b.y);
  }
}

// Per-restart Grams of every problem: blocks own 512-row chunks; upper 4x4
// tiles only; FP32 over 32-row sub-chunks, double-float (FP32 pairs) per
// thread across them, one FP64 atomic per entry per block (mirrored tiles
// added to both halves).
constexpr int GG_CHUNK = 512, GG_SUB = 32, GG_THREADS = 256;

// Upper 4x4 tile number u (row-major over ti <= tj) of a kt x kt tile grid.
__device__ __forceinline__ void gg_tri(int u, int kt, int& ti, int& tj) {
  int b = 0;
  while (u >= kt - b) {
    u -= kt - b;
    ++b;
  }
  ti = b;
  tj = b + u;
}

__global__ void __launch_bounds__(GG_THREADS) grouped_gram_kernel(const HalsProb* __restrict__ hp,
                                                                  const long long* chunk_off, int nprob,
                                                                  const float* F_all, double* Gd_all) {
  __shared__ __align__(16) float Fs[GG_SUB * GB_BN];
  __shared__ float2 red[GG_THREADS * 16];
  const int p = find_le(chunk_off, nprob, (long long)blockIdx.x);
  const HalsProb P = hp[p];
  const int k = P.k, R = P.R, RW = R * k;
  const int k4 = (k + 3) & ~3, tk = k4 >> 2;
  const int tt = tk * (tk + 1) / 2;  // upper 4x4 tiles of one restart
  const int T = R * tt;              // over all restarts
  const int RG = T >= GG_THREADS ? 1 : GG_THREADS / T;
  const int tid = threadIdx.x;
  const int rg = tid / T;
  const long long r0 = (blockIdx.x - chunk_off[p]) * (long long)GG_CHUNK;
  const long long r1 = min((long long)P.n, r0 + GG_CHUNK);
  const float* F = F_all + P.f_off;
  float2 acc[2][16];
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[t][e] = make_float2(0.f, 0.f);
  // rows staged compactly (pitch RW); 16-byte copies and loads when the widths allow
  const bool vec = (RW & 3) == 0 && (P.f_off & 3) == 0 && (k & 3) == 0;
  for (long long rb = r0; rb < r1; rb += GG_SUB) {
    const int rows = (int)min((long long)GG_SUB, r1 - rb);
    if (vec) {
      const int nv = rows * RW / 4, nz = GG_SUB * RW / 4;
      const float4* src = reinterpret_cast<const float4*>(F + rb * RW);
      float4* dst = reinterpret_cast<float4*>(Fs);
      for (int e = tid; e < nz; e += GG_THREADS) dst[e] = e < nv ? src[e] : make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      for (int e = tid; e < GG_SUB * RW; e += GG_THREADS) {
        const int rr = e / RW;
        Fs[e] = rr < rows ? F[rb * RW + e] : 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int tile = T >= GG_THREADS ? tid + t * GG_THREADS : (t == 0 ? tid % T : T);
      if (tile < T && rg < RG) {
        const int g = tile / tt;
        int ti, tj;
        gg_tri(tile - g * tt, tk, ti, tj);
        float f[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) f[e] = 0.f;
        for (int rr = rg; rr < GG_SUB; rr += RG) {
          const float* row = Fs + rr * RW + g * k;
          float av[4], bv[4];
          if (vec) {
            const float4 a4 = *reinterpret_cast<const float4*>(row + ti * 4);
            const float4 b4 = *reinterpret_cast<const float4*>(row + tj * 4);
            av[0] = a4.x, av[1] = a4.y, av[2] = a4.z, av[3] = a4.w;
            bv[0] = b4.x, bv[1] = b4.y, bv[2] = b4.z, bv[3] = b4.w;
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              av[q] = (ti * 4 + q < k) ? row[ti * 4 + q] : 0.f;
              bv[q] = (tj * 4 + q < k) ? row[tj * 4 + q] : 0.f;
            }
          }
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) f[a * 4 + b] = fmaf(av[a], bv[b], f[a * 4 + b]);
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) gb_df_add(acc[t][e].x, acc[t][e].y, f[e], 0.f);
      }
    }
    __syncthreads();
  }
  // combine row groups in shared memory, then one atomic per entry
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int tile = T >= GG_THREADS ? tid + t * GG_THREADS : (t == 0 ? tid % T : T);
    const bool mine = tile < T && rg < RG && (T >= GG_THREADS || t == 0);
    for (int g2 = 0; g2 < RG; ++g2) {
      if (mine && rg == g2)
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          float2 v = g2 == 0 ? make_float2(0.f, 0.f) : red[(tile % GG_THREADS) * 16 + e];
          gb_df_add(v.x, v.y, acc[t][e].x, acc[t][e].y);
          red[(tile % GG_THREADS) * 16 + e] = v;
        }
      __syncthreads();
    }
    if (mine && rg == 0) {
      const int g = tile / tt;
      int ti, tj;
      gg_tri(tile - g * tt, tk, ti, tj);
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int i = ti * 4 + (e >> 2), j = tj * 4 + (e & 3);
        if (i < k && j < k) {
          const float2 v = red[(tile % GG_THREADS) * 16 + e];
          const double dv = (double)v.x + (double)v.y;
          double* Gg = Gd_all + P.g_off + (long long)g * k * k;
          atomicAdd(Gg + i * k + j, dv);
          if (ti != tj) atomicAdd(Gg + j * k + i, dv);  // the mirrored tile
        }
      }
    }
    __syncthreads();
  }
}

// Surrogate objective of every (problem, restart) by the trace trick, one warp
// each: sum (W^T W) .* (H^T H) over the lanes (FP64, fixed xor tree), plus
// ||X||^2 - 2 tr + alpha dd.  cnt[0] is the ring slot; the last block to
// finish (cnt[1] counts the blocks) advances it.
__global__ void __launch_bounds__(256) grouped_objective_kernel(const HalsProb* hp, int R, const double* normX2,
                                                                const double* GW, const double* GH,
                                                                const double* part, double* ring, int* cnt, int cap,
                                                                int PR) {
  const int t = cnt[0];
  const int lane = threadIdx.x & 31;
  const int pr = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (pr < PR) {
    const int p = pr / R, g = pr - p * R;  // restarts are uniform over the batch
    const HalsProb& P = hp[p];
    const int k = P.k;
    const long long o = P.g_off + (long long)g * k * k;
    double s = 0.0;
    for (int e = lane; e < k * k; e += 32) s = fma(GW[o + e], GH[o + e], s);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0 && t < cap)
      ring[(long long)t * PR + pr] = normX2[p] + s - 2.0 * part[2 * pr] + P.alpha * part[2 * pr + 1];
  }
  if (last_block<1>(reinterpret_cast<unsigned*>(cnt + 1)) && threadIdx.x == 0) {
    cnt[1] = 0;
    cnt[0] = t + 1;
  }
}

// Restart r of problem p: Philox counter (j, i lo, i hi, TAG_INIT), key seed_p + r;
// identical to the single-problem start with seed = seed_p + r.
__global__ void grouped_init_kernel(const HalsProb* hp, const long long* row_off, int nprob,
                                    long long total_rows, const unsigned long long* seeds,
                                    const double* means, int scaled, float* H_all, float* W_all) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total_rows * GB_BN) return;
  const long long gr = t / GB_BN;
  const int c = (int)(t - gr * GB_BN);
  const int p = find_le(row_off, nprob, gr);
  const HalsProb& P = hp[p];
  const int w = P.R * P.k;
  if (c >= w) return;
  const long long i = gr - row_off[p];
  const int r = c / P.k, j = c - r * P.k;
  const unsigned long long key = seeds[p] + (unsigned long long)r;
  const Philox4 x = philox4x32_10((uint32_t)j, (uint32_t)i, (uint32_t)(i >> 32), TAG_INIT, (uint32_t)key,
                                  (uint32_t)(key >> 32));
  double v = (double)x.x0 * 0x1p-32;
  if (scaled) v *= 2.0 / sqrt((double)P.k) * sqrt(means[p]);
  const long long o = P.f_off + i * w + c;
  H_all[o] = (float)v;
  W_all[o] = (float)v;
}

}  // namespace symnmf

using namespace symnmf;

// ----------------------------------------------------------------- handle

struct symnmf_batch_ctx {
  cudaStream_t st = nullptr, cap_st = nullptr;
  std::string msg;
  std::vector<void*> allocs;
  int nprob = 0, R = 1, PR = 0;
  bool bf16 = true;
  std::vector<symnmf_problem> probs;
  std::vector<HalsProb> hp;
  std::vector<long long> ldp, pack_off;
  long long total_rows = 0, total_f = 0, total_g = 0, total_pack = 0, hals_tiles = 0, gram_chunks = 0;
  long long total_tiles = 0;  // 128-row tiles of the grouped product
  long long total_iters = 0;
  float *H = nullptr, *W = nullptr, *Y = nullptr;
  double* Gd[2] = {nullptr, nullptr};
  float* Gp = nullptr;  // padded FP32 Grams of the fixed factor for the HALS blocks
  double *part = nullptr, *normX2 = nullptr, *means = nullptr, *ring = nullptr, *scratch = nullptr;
  int* cnt = nullptr;
  unsigned *err = nullptr, *counter = nullptr;
  HalsProb* d_hp = nullptr;
  GroupProb* d_gp = nullptr;
  long long *d_tile_off = nullptr, *d_chunk_off = nullptr, *d_row_off = nullptr, *d_it_off = nullptr,
            *d_gtile_off = nullptr, *d_f_off = nullptr, *d_pack_off = nullptr, *d_ldp = nullptr;
  int *d_kb = nullptr, *d_width = nullptr, *d_bn = nullptr;
  unsigned long long* d_seeds = nullptr;
  void* pack = nullptr;
  float* partials = nullptr;
  size_t partial_floats = 0;
  // tuned product configuration
  int stages = 6, ctas_per_sm = 1, G = 0, max_segs = 1;
  size_t hals_smem = 0;  // dynamic shared memory of the grouped HALS kernel
  bool tuned = false;
  double tuned_ms = 0.0;
  cudaGraphExec_t graph = nullptr;
  uint64_t graph_kernels = 0;
  std::vector<float*> Fscratch;  // F32 path: per-problem Y pointers are inside Y
};

template <typename T>
static cudaError_t balloc(symnmf_batch_t b, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e == cudaSuccess) b->allocs.push_back((void*)*p);
  return e;
}

static symnmf_status bfail(symnmf_batch_t b, symnmf_status s, const std::string& m) {
  if (b) b->msg = m;
  return s;
}

#define BTRY(call)                                                                              \
  do {                                                                                          \
    cudaError_t _e = (call);                                                                    \
    if (_e != cudaSuccess) {                                                                    \
      cudaGetLastError();                                                                       \
      return bfail(b, to_status(_e), std::string(#call) + ": " + cudaGetErrorString(_e));       \
    }                                                                                           \
  } while (0)
#define BTRYS(call)                  \
  do {                               \
    symnmf_status _s = (call);       \
    if (_s != SYMNMF_OK) return _s;  \
  } while (0)

static int max_segs_for(long long total, int G, const std::vector<HalsProb>& hp,
                        const std::vector<long long>& it_off, const std::vector<long long>& gtile,
                        const std::vector<int>& kb) {
  auto gtile_of = [&](long long it) {
    int p = (int)(std::upper_bound(it_off.begin(), it_off.end(), it) - it_off.begin()) - 1;
    return gtile[p] + (it - it_off[p]) / kb[p];
  };
  int best = 1;
  for (int c = 0; c < G; ++c) {
    const long long a = ((long long)c * total) / G, e = ((long long)(c + 1) * total) / G;
    if (e <= a) continue;
    const long long segs = gtile_of(e - 1) - gtile_of(a) + 1;
    if (segs > best) best = (int)segs;
  }
  (void)hp;
  return best;
}

static size_t grouped_smem(int stages) { return (size_t)stages * (TC_BM + GB_BN) * TC_ROW_BYTES + 1024 + 256; }

static cudaError_t launch_grouped(symnmf_batch_t b, int stages, int G, int max_segs) {
  const size_t smem = grouped_smem(stages);
  cudaError_t e;
  switch (stages) {
    case 3:
      e = cudaFuncSetAttribute(grouped_tc_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      grouped_tc_kernel<3><<<G, TC_THREADS, smem, b->st>>>(b->d_gp, b->nprob, b->total_iters, b->partials,
                                                           max_segs, b->err);
      break;
    case 4:
      e = cudaFuncSetAttribute(grouped_tc_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      grouped_tc_kernel<4><<<G, TC_THREADS, smem, b->st>>>(b->d_gp, b->nprob, b->total_iters, b->partials,
                                                           max_segs, b->err);
      break;
    default:
      e = cudaFuncSetAttribute(grouped_tc_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      grouped_tc_kernel<6><<<G, TC_THREADS, smem, b->st>>>(b->d_gp, b->nprob, b->total_iters, b->partials,
                                                           max_segs, b->err);
      break;
  }
  count_launches(1);
  return cudaGetLastError();
}

// All products Y_p = X_p F_p of one half sweep.
static symnmf_status batched_product(symnmf_batch_t b, const float* F_all) {
  if (b->bf16) {
    grouped_pack_kernel<<<(unsigned)b->hals_tiles, 256, 0, b->st>>>(b->d_hp, b->d_tile_off, b->nprob, b->d_pack_off,
                                                                   b->d_bn, b->d_ldp, F_all, (__nv_bfloat16*)b->pack);
    count_launches(1);
    BTRY(cudaGetLastError());
    BTRY(launch_grouped(b, b->stages, b->G, b->max_segs));
    ReduceTab tab{b->d_it_off, b->d_gtile_off, b->d_kb, b->d_row_off, b->d_f_off, b->d_width};
    grouped_reduce_kernel<<<(unsigned)b->total_tiles, 256, 0, b->st>>>(tab, b->nprob, b->partials, b->max_segs,
                                                                       b->total_iters, b->G, b->Y);
    count_launches(1);
    BTRY(cudaGetLastError());
    return SYMNMF_OK;
  }
  for (int p = 0; p < b->nprob; ++p) {
    const HalsProb& P = b->hp[p];
    const int w = P.R * P.k;
    const size_t wsf = xf_simt_ws_floats(P.n, w);
    BTRY(xf_simt(SYMNMF_X_DENSE_F32, b->probs[p].x, b->probs[p].ldx > 0 ? b->probs[p].ldx : P.n, P.n,
                 F_all + P.f_off, w, w, b->Y + P.f_off, w, b->partials, wsf <= b->partial_floats ? b->partial_floats : 0,
                 b->st));
  }
  return SYMNMF_OK;
}

static symnmf_status batched_half(symnmf_batch_t b, int side) {
  float* Fu = side ? b->H : b->W;
  const float* Ff = side ? b->W : b->H;
  const int gfix = side ? 1 : 0, gupd = side ? 0 : 1;
  BTRYS(batched_product(b, Ff));
  BTRY(cudaMemsetAsync(b->part, 0, (size_t)2 * b->PR * sizeof(double), b->st));
  grouped_gram_prep_kernel<<<(unsigned)b->nprob, 256, 0, b->st>>>(b->d_hp, b->Gd[gfix], b->Gp);
  grouped_hals_kernel<<<(unsigned)b->hals_tiles, GH_ROWS * b->R, b->hals_smem, b->st>>>(
      b->d_hp, b->d_tile_off, b->nprob, Fu, Ff, b->Y, b->Gp, b->part, b->err);
  count_launches(2);
  BTRY(cudaGetLastError());
  BTRY(cudaMemsetAsync(b->Gd[gupd], 0, (size_t)b->total_g * sizeof(double), b->st));
  grouped_gram_kernel<<<(unsigned)b->gram_chunks, GG_THREADS, 0, b->st>>>(b->d_hp, b->d_chunk_off, b->nprob,
                                                                          Fu, b->Gd[gupd]);
  count_launches(1);
  BTRY(cudaGetLastError());
  if (side == 1) {
    grouped_objective_kernel<<<(unsigned)((b->PR * 32 + 255) / 256), 256, 0, b->st>>>(
        b->d_hp, b->R, b->normX2, b->Gd[1], b->Gd[0], b->part, b->ring, b->cnt, OBJ_RING, b->PR);
    count_launches(1);
    BTRY(cudaGetLastError());
  }
  return SYMNMF_OK;
}

static symnmf_status batched_body(symnmf_batch_t b) {
  BTRYS(batched_half(b, 0));
  BTRYS(batched_half(b, 1));
  return SYMNMF_OK;
}

static symnmf_status batched_grams(symnmf_batch_t b) {
  for (int s = 0; s < 2; ++s) {
    BTRY(cudaMemsetAsync(b->Gd[s], 0, (size_t)b->total_g * sizeof(double), b->st));
    grouped_gram_kernel<<<(unsigned)b->gram_chunks, GG_THREADS, 0, b->st>>>(b->d_hp, b->d_chunk_off, b->nprob,
                                                                            s ? b->W : b->H, b->Gd[s]);
    count_launches(1);
    BTRY(cudaGetLastError());
  }
  return SYMNMF_OK;
}

// Timing autotuner for the grouped product: pipeline depth x CTAs per SM.
static symnmf_status autotune(symnmf_batch_t b) {
  if (b->tuned || !b->bf16) return SYMNMF_OK;
  struct Cand {
    int stages, per_sm;
  } cands[3] = {{6, 1}, {4, 1}, {3, 2}};
  cudaEvent_t e0, e1;
  BTRY(cudaEventCreate(&e0));
  BTRY(cudaEventCreate(&e1));
  double best = 1e30;
  int bi = 0;
  // pack H once so that the product has valid operands
  grouped_pack_kernel<<<(unsigned)b->hals_tiles, 256, 0, b->st>>>(b->d_hp, b->d_tile_off, b->nprob, b->d_pack_off,
                                                                 b->d_bn, b->d_ldp, b->H, (__nv_bfloat16*)b->pack);
  count_launches(1);
  for (int c = 0; c < 3; ++c) {
    const int G = (int)std::min<long long>((long long)num_sms() * cands[c].per_sm, b->total_iters);
    std::vector<long long> it_off(b->nprob), gt(b->nprob);
    std::vector<int> kb(b->nprob);
    // host copies of the tables
    cudaMemcpy(it_off.data(), b->d_it_off, b->nprob * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(gt.data(), b->d_gtile_off, b->nprob * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(kb.data(), b->d_kb, b->nprob * 4, cudaMemcpyDeviceToHost);
    const int ms = max_segs_for(b->total_iters, G, b->hp, it_off, gt, kb);
    if ((size_t)G * ms * TC_BM * GB_BN > b->partial_floats) continue;
    BTRY(launch_grouped(b, cands[c].stages, G, ms));  // warm
    BTRY(cudaEventRecord(e0, b->st));
    for (int r = 0; r < 3; ++r) BTRY(launch_grouped(b, cands[c].stages, G, ms));
    BTRY(cudaEventRecord(e1, b->st));
    BTRY(cudaEventSynchronize(e1));
    float ms_t = 0.f;
    BTRY(cudaEventElapsedTime(&ms_t, e0, e1));
    if (ms_t / 3 < best) {
      best = ms_t / 3;
      bi = c;
      b->G = G;
      b->max_segs = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->stages = cands[bi].stages;
  b->ctas_per_sm = cands[bi].per_sm;
  b->tuned_ms = best;
  b->tuned = true;
  unsigned herr = 0;
  BTRY(cudaMemcpy(&herr, b->err, 4, cudaMemcpyDeviceToHost));
  if (herr) return bfail(b, SYMNMF_ETIMEOUT, "grouped product wait ran out while tuning");
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_batched_create(const symnmf_problem* probs, int nprob, int restarts,
                                               const symnmf_options* opt, void* stream, symnmf_batch_t* out) {
  if (!out || !probs || nprob < 1 || restarts < 1 || restarts > GB_MAXR) return SYMNMF_EINVAL;
  *out = nullptr;
  const int fmt0 = probs[0].fmt;
  if (fmt0 != SYMNMF_X_DENSE_BF16 && fmt0 != SYMNMF_X_DENSE_F32) return SYMNMF_EINVAL;
  for (int p = 0; p < nprob; ++p) {
    const symnmf_problem& q = probs[p];
    const int64_t ldx = q.ldx > 0 ? q.ldx : q.n;
    if (q.fmt != fmt0 || q.n < 1 || q.k < 1 || q.k > 32 || q.k * restarts > GB_BN || !q.x || ldx < q.n)
      return SYMNMF_EINVAL;
    if (fmt0 == SYMNMF_X_DENSE_BF16 && ((ldx % 8) || ((uintptr_t)q.x & 15))) return SYMNMF_EINVAL;
  }
  symnmf_batch_t b = new symnmf_batch_ctx();
  b->st = (cudaStream_t)stream;
  b->nprob = nprob;
  b->R = restarts;
  b->bf16 = fmt0 == SYMNMF_X_DENSE_BF16;
  b->probs.assign(probs, probs + nprob);
  (void)opt;
  auto bail = [&](symnmf_status s) {
    symnmf_batched_destroy(b);
    return s;
  };
  // layout tables
  std::vector<long long> tile_off(nprob), chunk_off(nprob), row_off(nprob + 1), it_off(nprob), gtile(nprob),
      f_off(nprob);
  std::vector<int> kb(nprob), width(nprob), bn(nprob);
  long long f = 0, g = 0, gp = 0, rows = 0, tiles = 0, chunks = 0, its = 0, gt = 0, pk = 0;
  int pr = 0;
  b->ldp.resize(nprob);
  b->pack_off.resize(nprob);
  for (int p = 0; p < nprob; ++p) {
    const symnmf_problem& q = probs[p];
    HalsProb h{};
    h.n = (int)q.n;
    h.k = q.k;
    h.R = restarts;
    h.f_off = f;
    h.g_off = g;
    h.gp_off = gp;
    h.row_off = rows;
    h.pr_off = pr;
    f_off[p] = f;
    width[p] = q.k * restarts;
    bn[p] = tc_block_n(width[p]);
    row_off[p] = rows;
    tile_off[p] = tiles;
    chunk_off[p] = chunks;
    it_off[p] = its;
    gtile[p] = gt;
    kb[p] = (int)((q.n + 63) / 64);
    const long long mt = (q.n + TC_BM - 1) / TC_BM;
    b->ldp[p] = (q.n + 15) / 16 * 16;
    b->pack_off[p] = pk;
    pk += (long long)bn[p] * b->ldp[p];
    its += mt * kb[p];
    gt += mt;
    f += (long long)q.n * width[p];
    g += (long long)restarts * q.k * q.k;
    {
      const int km = q.k <= 8 ? 8 : q.k <= 16 ? 16 : q.k <= 24 ? 24 : 32;
      gp += (long long)restarts * (km * km + km);
    }
    rows += q.n;
    tiles += (q.n + GH_ROWS - 1) / GH_ROWS;
    chunks += (q.n + GG_CHUNK - 1) / GG_CHUNK;
    pr += restarts;
    b->hp.push_back(h);
  }
  row_off[nprob] = rows;
  // grouped HALS: R zero-padded (at most 32 x 32) Grams and R x 32 inverses
  b->hals_smem = (size_t)restarts * (32 * 32 + 32) * sizeof(float);
  if (cudaFuncSetAttribute(grouped_hals_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)b->hals_smem) != cudaSuccess)
    return bail(SYMNMF_ECUDA);
  b->PR = pr;
  b->total_f = f;
  b->total_g = g;
  b->total_rows = rows;
  b->hals_tiles = tiles;
  b->gram_chunks = chunks;
  b->total_iters = its;
  b->total_tiles = gt;
  b->total_pack = pk;
#define BA(ptr, cnt)                                           \
  do {                                                         \
    if (balloc(b, &(ptr), (cnt)) != cudaSuccess) return bail(SYMNMF_ENOMEM); \
  } while (0)
  BA(b->H, f);
  BA(b->W, f);
  BA(b->Y, f);
  BA(b->Gd[0], g);
  BA(b->Gd[1], g);
  BA(b->Gp, gp);
  BA(b->part, 2 * pr);
  BA(b->normX2, nprob);
  BA(b->means, nprob);
  BA(b->ring, (size_t)OBJ_RING * pr);
  BA(b->cnt, 4);
  BA(b->err, 4);
  BA(b->counter, 4);
  BA(b->scratch, 3 * 4096);
  BA(b->d_hp, nprob);
  BA(b->d_tile_off, nprob);
  BA(b->d_chunk_off, nprob);
  BA(b->d_row_off, nprob + 1);
  BA(b->d_it_off, nprob);
  BA(b->d_gtile_off, nprob);
  BA(b->d_f_off, nprob);
  BA(b->d_pack_off, nprob);
  BA(b->d_ldp, nprob);
  BA(b->d_kb, nprob);
  BA(b->d_width, nprob);
  BA(b->d_bn, nprob);
  BA(b->d_seeds, nprob);
  cudaStream_t st = b->st;
  cudaMemsetAsync(b->err, 0, 4, st);
  cudaMemsetAsync(b->counter, 0, 4, st);
  cudaMemsetAsync(b->H, 0, f * 4, st);
  cudaMemsetAsync(b->W, 0, f * 4, st);
  // per-problem alpha (max X), ||X||^2 and mean
  std::vector<double> nx(nprob), mean(nprob);
  std::vector<unsigned long long> seeds(nprob);
  for (int p = 0; p < nprob; ++p) {
    const symnmf_problem& q = probs[p];
    const int64_t ldx = q.ldx > 0 ? q.ldx : q.n;
    if (xstats(q.fmt, q.x, ldx, nullptr, q.n, nullptr, 0, b->scratch + 3 * 4000, b->scratch, b->counter, st) !=
        cudaSuccess)
      return bail(SYMNMF_ECUDA);
    double s3[3];
    if (cudaMemcpyAsync(s3, b->scratch + 3 * 4000, 24, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return bail(SYMNMF_ECUDA);
    b->hp[p].alpha = q.alpha > 0 ? q.alpha : s3[0];
    if (!(b->hp[p].alpha > 0)) return bail(SYMNMF_EINVAL);
    nx[p] = s3[2];
    mean[p] = s3[1] / ((double)q.n * q.n);
    seeds[p] = q.seed;
  }
  if (b->bf16) {
    if (balloc(b, (uint16_t**)&b->pack, (size_t)pk) != cudaSuccess) return bail(SYMNMF_ENOMEM);
    std::vector<GroupProb> gp(nprob);
    for (int p = 0; p < nprob; ++p) {
      const symnmf_problem& q = probs[p];
      const int64_t ldx = q.ldx > 0 ? q.ldx : q.n;
      const uint16_t* pk_p = (const uint16_t*)b->pack + b->pack_off[p];
      if (!tc_make_map(&gp[p].tmA, q.x, false, q.n, q.n, ldx * 2, 64, TC_BM) ||
          !tc_make_map(&gp[p].tmB, pk_p, false, q.n, bn[p], b->ldp[p] * 2, 64, bn[p]))
        return bail(SYMNMF_EINVAL);
      gp[p].it_off = it_off[p];
      gp[p].tile_off = gtile[p];
      gp[p].kblocks = kb[p];
      gp[p].mtiles = (int)((q.n + TC_BM - 1) / TC_BM);
      gp[p].bn = bn[p];
    }
    if (balloc(b, &b->d_gp, nprob) != cudaSuccess) return bail(SYMNMF_ENOMEM);
    cudaMemcpy(b->d_gp, gp.data(), sizeof(GroupProb) * nprob, cudaMemcpyHostToDevice);
    // partials sized for the widest candidate grid
    size_t need = 0;
    for (int per_sm = 1; per_sm <= 2; ++per_sm) {
      const int G = (int)std::min<long long>((long long)num_sms() * per_sm, its);
      const int ms = max_segs_for(its, G, b->hp, it_off, gtile, kb);
      need = std::max(need, (size_t)G * ms * TC_BM * GB_BN);
    }
    b->G = (int)std::min<long long>(num_sms(), its);
    b->max_segs = max_segs_for(its, b->G, b->hp, it_off, gtile, kb);
    b->partial_floats = need;
    if (balloc(b, &b->partials, need) != cudaSuccess) return bail(SYMNMF_ENOMEM);
  } else {
    size_t need = 0;
    for (int p = 0; p < nprob; ++p) need = std::max(need, xf_simt_ws_floats(probs[p].n, width[p]));
    b->partial_floats = need;
    if (balloc(b, &b->partials, need) != cudaSuccess) return bail(SYMNMF_ENOMEM);
  }
  cudaMemcpy(b->d_hp, b->hp.data(), sizeof(HalsProb) * nprob, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_tile_off, tile_off.data(), 8 * nprob, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_chunk_off, chunk_off.data(), 8 * nprob, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_row_off, row_off.data(), 8 * (nprob + 1), cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_it_off, it_off.data(), 8 * nprob, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_gtile_off, gtile.data(), 8 * nprob, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_f_off, f_off.data(), 8 * nprob, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_pack_off, b->pack_off.data(), 8 * nprob, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_ldp, b->ldp.data(), 8 * nprob, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_kb, kb.data(), 4 * nprob, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_width, width.data(), 4 * nprob, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_bn, bn.data(), 4 * nprob, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_seeds, seeds.data(), 8 * nprob, cudaMemcpyHostToDevice);
  cudaMemcpy(b->normX2, nx.data(), 8 * nprob, cudaMemcpyHostToDevice);
  cudaMemcpy(b->means, mean.data(), 8 * nprob, cudaMemcpyHostToDevice);
  if (cudaDeviceSynchronize() != cudaSuccess) return bail(SYMNMF_ECUDA);
#undef BA
  *out = b;
  return SYMNMF_OK;
}

extern "C" void symnmf_batched_destroy(symnmf_batch_t b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap_st) cudaStreamDestroy(b->cap_st);
  for (void* p : b->allocs) cudaFree(p);
  delete b;
}

extern "C" const char* symnmf_batched_last_error(symnmf_batch_t b) { return b ? b->msg.c_str() : "null handle"; }

extern "C" symnmf_status symnmf_batched_init_random(symnmf_batch_t b, int scaled) {
  if (!b) return SYMNMF_EINVAL;
  const long long work = b->total_rows * GB_BN;
  grouped_init_kernel<<<(unsigned)((work + 255) / 256), 256, 0, b->st>>>(
      b->d_hp, b->d_row_off, b->nprob, b->total_rows, b->d_seeds, b->means, scaled, b->H, b->W);
  count_launches(1);
  BTRY(cudaGetLastError());
  return batched_grams(b);
}

extern "C" symnmf_status symnmf_batched_set_factors(symnmf_batch_t b, int p, const float* H0, const float* W0) {
  if (!b || p < 0 || p >= b->nprob || !H0) return SYMNMF_EINVAL;
  const HalsProb& P = b->hp[p];
  const size_t bytes = (size_t)P.n * P.R * P.k * 4;
  BTRY(cudaMemcpyAsync(b->H + P.f_off, H0, bytes, cudaMemcpyDeviceToDevice, b->st));
  BTRY(cudaMemcpyAsync(b->W + P.f_off, W0 ? W0 : H0, bytes, cudaMemcpyDeviceToDevice, b->st));
  return batched_grams(b);
}

extern "C" symnmf_status symnmf_batched_get_factors(symnmf_batch_t b, int p, float* H_out, float* W_out) {
  if (!b || p < 0 || p >= b->nprob) return SYMNMF_EINVAL;
  const HalsProb& P = b->hp[p];
  const size_t bytes = (size_t)P.n * P.R * P.k * 4;
  if (H_out) BTRY(cudaMemcpyAsync(H_out, b->H + P.f_off, bytes, cudaMemcpyDeviceToDevice, b->st));
  if (W_out) BTRY(cudaMemcpyAsync(W_out, b->W + P.f_off, bytes, cudaMemcpyDeviceToDevice, b->st));
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_batched_info(symnmf_batch_t b, int* stages, int* ctas_per_sm, double* product_ms) {
  if (!b) return SYMNMF_EINVAL;
  if (stages) *stages = b->stages;
  if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
  if (product_ms) *product_ms = b->tuned_ms;
  return SYMNMF_OK;
}

extern "C" symnmf_status symnmf_batched_sweep(symnmf_batch_t b, int nsweeps, double* obj_host) {
  if (!b || nsweeps < 0) return SYMNMF_EINVAL;
  BTRYS(autotune(b));
  int done = 0;
  bool warmed = false;
  while (done < nsweeps) {
    const int chunk = std::min(nsweeps - done, OBJ_RING);
    BTRY(cudaMemsetAsync(b->cnt, 0, 8, b->st));  // ring slot, finished-block count
    int t = 0;
    if (!warmed) {
      BTRYS(batched_body(b));
      ++t;
      warmed = true;
    }
    if (t < chunk && !b->graph) {
      if (!b->cap_st) BTRY(cudaStreamCreateWithFlags(&b->cap_st, cudaStreamNonBlocking));
      cudaStream_t saved = b->st;
      b->st = b->cap_st;
      cudaGraph_t g;
      BTRY(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
      const uint64_t before = symnmf_launch_count();
      symnmf_status s = batched_body(b);
      cudaError_t e = cudaStreamEndCapture(b->st, &g);
      b->st = saved;
      if (s != SYMNMF_OK) return s;
      BTRY(e);
      cudaError_t ei = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      BTRY(ei);
      b->graph_kernels = symnmf_launch_count() - before;
      count_launches((uint64_t)0 - b->graph_kernels);  // recorded, not launched
    }
    for (; t < chunk; ++t) {
      BTRY(cudaGraphLaunch(b->graph, b->st));
      count_launches(b->graph_kernels);
    }
    if (obj_host) {
      BTRY(cudaMemcpyAsync(obj_host + (size_t)done * b->PR, b->ring, (size_t)chunk * b->PR * 8,
                           cudaMemcpyDeviceToHost, b->st));
      BTRY(cudaStreamSynchronize(b->st));
      unsigned herr = 0;
      BTRY(cudaMemcpy(&herr, b->err, 4, cudaMemcpyDeviceToHost));
      if (herr) {
        cudaMemset(b->err, 0, 4);
        return bfail(b, (herr & ERR_TIMEOUT) ? SYMNMF_ETIMEOUT : SYMNMF_ENAN, "device error word set");
      }
    }
    done += chunk;
  }
  return SYMNMF_OK;
}
