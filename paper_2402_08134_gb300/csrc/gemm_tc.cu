// Dense Y = X F on the 5th-generation tensor cores (tcgen05) for BF16 or FP8
// (E4M3, per-row scales of X and per-column scales of F) X, FP32 accumulation
// in tensor memory.  This is the product whose O(n^2 k) cost dominates a
// SymNMF sweep (the complexity discussion of the LvS section) and the range
// finder of Alg. RRF.
//
// Layout: A = X (n x n, K-major rows, TMA tiles 128 x 128 bytes, 128-byte
// swizzle), B = F^T packed (BN x n, K-major, same swizzle), D = 128 x BN FP32
// in TMEM.  Warp roles per CTA (224 threads, one CTA per SM):
//   warp 0      : TMA producer of A (one thread) into its own smem ring;
//   warp 6      : TMA producer of B (one thread) into a second, shallower ring
//                 (F is re-read by every CTA and comes from L2; X streams from
//                 HBM and needs the deeper buffering);
//   warp 1      : TMEM allocator + MMA issuer (one thread);
//   warps 2..5  : epilogue, tcgen05.ld of the accumulator -> FP32 partials.
// Up to 128 columns, four TMEM accumulators alternate so that the epilogue of
// one accumulation overlaps the MMAs of the next ones; an accumulation covers
// at most 8 k blocks and the epilogue adds a row tile's accumulations in FP32
// registers (round to nearest), which keeps the tensor core's per-MMA
// accumulation drift (~2e-8 relative, low) from building up over long K.
// Wider products (more than 128 columns) run on CTA pairs (xf_tc2_kernel):
// they fill TMEM with one accumulator per segment and keep that drift
// (~6e-5 at K = 20000).
//
// Work split (stream-K): the (row tile, k block) iteration space is cut into
// gridDim.x equal contiguous ranges, one per CTA, so every SM streams the
// same number of X bytes.  A CTA writes one partial tile per row tile it
// touches; a second kernel sums the partials of each row tile in CTA order
// (deterministic) and applies the FP8 scales.
//
// Every mbarrier wait is bounded (%globaltimer, 2 s): on expiry the CTA sets
// ERR_TIMEOUT, stops issuing work, drains its own copies and MMAs (again
// bounded), frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

#ifndef XF_TC_CHUNK
#define XF_TC_CHUNK 8  // k blocks per TMEM accumulation (128-row tiles)
#endif

namespace symnmf {

constexpr int XF_THREADS = 224;  // warps 0..6: A producer, MMA, 4 epilogue warps, B producer

// One CTA per 128-row tile, up to 128 columns (wider products run on CTA
// pairs: xf_tc2_kernel).
template <int BN>
struct TcCfg {
  static_assert(BN <= 128, "wider products run on CTA pairs");
  static constexpr int BM = TC_BM;
  static constexpr int MMA_N = BN;                  // columns per MMA
  static constexpr int NB_MMA = 1;                  // MMAs per k step
  static constexpr bool REGACC = true;              // epilogue adds accumulations in registers
  static constexpr int A_BYTES = BM * TC_ROW_BYTES;
  static constexpr int B_BYTES = BN * TC_ROW_BYTES;
  static constexpr int B_STAGES = 4;
  // X stages fill what the F^T stages leave of 200 KB (at most 10).
  static constexpr int A_FIT = (200 * 1024 - B_STAGES * B_BYTES) / A_BYTES;
  static constexpr int A_STAGES = A_FIT > 10 ? 10 : A_FIT;
  // accumulator buffers in TMEM: four alternate, so that the epilogue's drains
  // of short accumulations never hold up the MMAs
  static constexpr int NBUF = 4;
  // k blocks accumulated in TMEM before the epilogue adds them into FP32
  // registers (round to nearest): the tensor core's accumulation drifts low by
  // a fraction of an FP32 ulp per MMA, which over a whole 20000-long K range
  // biased X F by ~7e-5 relative.
  static constexpr int64_t CHUNK = XF_TC_CHUNK;
  static constexpr uint32_t TMEM_COLS = NBUF * BN < 32 ? 32 : NBUF * BN;
  static_assert(TMEM_COLS <= 512, "TMEM holds 512 columns");
  static constexpr int SMEM = A_STAGES * A_BYTES + B_STAGES * B_BYTES + 1024 + 512;
  static_assert(SMEM <= 227 * 1024, "dynamic shared memory above the opt-in limit");
};

template <int BN, bool FP8>
__global__ void __launch_bounds__(XF_THREADS, 1)
    xf_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 int kblocks, int64_t total_iters, float* __restrict__ partials, int max_segs,
                 unsigned* err) {
  using C = TcCfg<BN>;
  constexpr int BM = C::BM, NBUF = C::NBUF;
  constexpr int SA = C::A_STAGES, SB = C::B_STAGES;
  constexpr int KSTEPS = TC_ROW_BYTES / 32;  // 32 bytes of K per MMA (16 bf16 / 32 e4m3)
  constexpr int KELEMS = FP8 ? 128 : 64;     // elements of K per k block
  constexpr uint32_t IDESC = make_idesc<FP8>(TC_BM, C::MMA_N);

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + SA * C::A_BYTES;
  uint64_t* fullA = (uint64_t*)(sB + SB * C::B_BYTES);
  uint64_t* emptyA = fullA + SA;
  uint64_t* fullB = emptyA + SA;
  uint64_t* emptyB = fullB + SB;
  uint64_t* tfull = emptyB + SB;
  uint64_t* tempty = tfull + 4;
  uint64_t* done = tempty + 4;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t it0 = ((int64_t)blockIdx.x * total_iters) / gridDim.x;
  const int64_t it1 = ((int64_t)(blockIdx.x + 1) * total_iters) / gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < SA; ++s) {
      mbar_init(&fullA[s], 1);
      mbar_init(&emptyA[s], 1);
    }
    for (int s = 0; s < SB; ++s) {
      mbar_init(&fullB[s], 1);
      mbar_init(&emptyB[s], 1);
    }
    for (int a = 0; a < 4; ++a) {
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
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 || warp == 6) {
    if (lane == 0) {
      // ---------------- producers: warp 0 streams A (X row tiles), warp 6 streams B (F^T)
      const bool isA = warp == 0;
      const int S = isA ? SA : SB;
      uint64_t* fullR = isA ? fullA : fullB;
      uint64_t* emptyR = isA ? emptyA : emptyB;
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_mask = 0;   // stages used at least once
      uint32_t last_parity = 0;   // bit s: parity of the last fill of stage s
      for (int64_t it = it0; it < it1; ++it) {
        const int tile = (int)(it / kblocks);
        const int kb = (int)(it - (int64_t)tile * kblocks);
        if (!mbar_wait(&emptyR[stage], phase ^ 1u, abort_flag)) {
          *abort_flag = 1;
          set_error(err, ERR_TIMEOUT);
          break;
        }
        if (isA) {
          mbar_expect_tx(&fullR[stage], C::A_BYTES);
#pragma unroll
          for (int h = 0; h < BM / TC_BM; ++h)
            tma_load_2d(sA + stage * C::A_BYTES + h * TC_BM * TC_ROW_BYTES, &tmA, kb * KELEMS,
                        tile * BM + h * TC_BM, &fullR[stage]);
        } else {
          mbar_expect_tx(&fullR[stage], C::B_BYTES);
#pragma unroll
          for (int j = 0; j < C::NB_MMA; ++j)
            tma_load_2d(sB + stage * C::B_BYTES + j * C::MMA_N * TC_ROW_BYTES, &tmB, kb * KELEMS, j * C::MMA_N,
                        &fullR[stage]);
        }
        issued_mask |= 1u << stage;
        last_parity = (last_parity & ~(1u << stage)) | (phase << stage);
        if (++stage == S) {
          stage = 0;
          phase ^= 1u;
        }
      }
      // drain: every copy this thread issued has landed before the CTA exits
      for (int s = 0; s < S; ++s)
        if (issued_mask >> s & 1u) {
          volatile int no_abort = 0;
          mbar_wait(&fullR[s], (last_parity >> s) & 1u, &no_abort);
        }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int sa = 0, sb = 0;
      uint32_t pa = 0, pb = 0;
      int dr = 0;  // accumulations handed to the epilogue
      bool ok = true;
      int64_t it = it0;
      while (ok && it < it1) {
        const int64_t tile = it / kblocks;
        const int64_t seg_end = min(it1, (tile + 1) * kblocks);
        const int64_t chunk_end = min(seg_end, it + C::CHUNK);
        const int a = dr % NBUF;
        const uint32_t use = (uint32_t)(dr / NBUF);
        if (!mbar_wait(&tempty[a], (use & 1u) ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(a * BN);
        const int64_t seg_begin = it;
        for (; it < chunk_end; ++it) {
          if (!mbar_wait(&fullA[sa], pa, abort_flag) || !mbar_wait(&fullB[sb], pb, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sA + sa * C::A_BYTES);
          const uint32_t b0 = smem_u32(sB + sb * C::B_BYTES);
#pragma unroll
          for (int h = 0; h < BM / TC_BM; ++h)
#pragma unroll
            for (int ks = 0; ks < KSTEPS; ++ks)
#pragma unroll
              for (int j = 0; j < C::NB_MMA; ++j)
                umma<FP8>(d + (uint32_t)(h * BN + j * C::MMA_N),
                          sw128_desc(a0 + h * TC_BM * TC_ROW_BYTES + ks * 32),
                          sw128_desc(b0 + j * C::MMA_N * TC_ROW_BYTES + ks * 32), IDESC,
                          (it > seg_begin || ks > 0) ? 1u : 0u);
          umma_commit(&emptyA[sa]);
          umma_commit(&emptyB[sb]);
          if (++sa == SA) {
            sa = 0;
            pa ^= 1u;
          }
          if (++sb == SB) {
            sb = 0;
            pb ^= 1u;
          }
        }
        if (!ok) break;
        umma_commit(&tfull[a]);
        ++dr;
      }
      if (!ok) {
        *abort_flag = 1;
        set_error(err, ERR_TIMEOUT);
      }
      // all MMAs issued by this thread complete before TMEM is released
      umma_commit(done);
      volatile int no_abort = 0;
      mbar_wait(done, 0, &no_abort);
    }
  } else {
    // ---------------- epilogue (warps 2..5)
    const int ew = warp & 3;
    int seg = 0;
    int64_t it = it0;
    if constexpr (C::REGACC) {
      // one thread per row of the 128-row tile: the chunks' accumulators are
      // added in registers (round to nearest) and the segment's sum written once
      int dr = 0;
      while (it < it1) {
        const int64_t tile = it / kblocks;
        const int64_t seg_end = min(it1, (tile + 1) * kblocks);
        float acc[BN];
#pragma unroll
        for (int c = 0; c < BN; ++c) acc[c] = 0.f;
        bool ok = true;
        while (it < seg_end) {
          const int a = dr % NBUF;
          const uint32_t use = (uint32_t)(dr / NBUF);
          if (!mbar_wait(&tfull[a], use & 1u, abort_flag)) {
            *abort_flag = 1;
            set_error(err, ERR_TIMEOUT);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t taddr = tmem_base + ((uint32_t)(ew * 32) << 16) + (uint32_t)(a * BN);
#pragma unroll
          for (int c = 0; c < BN; c += 16) {
            float v[16];
            tmem_ld16(taddr + (uint32_t)c, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) acc[c + q] += v[q];
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[a]);
          ++dr;
          it = min(seg_end, it + C::CHUNK);
        }
        if (!ok) break;
        float* dst = partials + (((size_t)blockIdx.x * max_segs + seg) * BM + ew * 32 + lane) * BN;
#pragma unroll
        for (int c = 0; c < BN; c += 4) *(float4*)(dst + c) = make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
        ++seg;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(C::TMEM_COLS)
                 : "memory");
}

// 512 columns on CTA pairs (cta_group::2).  A pair of CTAs on two SMs (a
// cluster of 2) shares each 256-row X tile: CTA r holds rows [128 r, 128 r +
// 128) of the tile and, of each of the two N = 256 MMAs per k step, F^T rows
// [256 j + 128 r, 256 j + 128 r + 128); the leader (rank 0) issues the pair's
// MMAs (M = 256), which read both CTAs' shared memory and leave each CTA's 128
// rows x 512 columns in its own TMEM.  Per CTA and k block that is 16 KB of X
// and 32 KB of F^T against 4.2 M MACs, where one CTA alone on a 128-row tile
// needs 64 KB of F^T for the same work: the L2 stream of F^T that bounds the
// single-CTA tile halves.  Both CTAs' TMA copies complete on the leader's
// stage barrier; the leader's commits arrive on both CTAs' "stage free" and
// "accumulator full" barriers; both CTAs' epilogue warps arrive on the
// leader's "accumulator free" barrier.  Waits are bounded as in xf_tc_kernel;
// every thread of both CTAs reaches the final cluster barrier.
constexpr int TC2_THREADS = 192;  // warp 0 TMA producer, warp 1 MMA issuer (leader), warps 2..5 epilogue

// NB N = 256 MMAs per k step: 256 (NB = 1) or 512 (NB = 2) columns.
template <int NB>
struct Tc2Cfg {
  static constexpr int BN = 256 * NB;
  static constexpr int A_BYTES = TC_BM * TC_ROW_BYTES;        // this CTA's 128 rows of X
  static constexpr int B_BYTES = NB * TC_BM * TC_ROW_BYTES;   // this CTA's half of each MMA's F^T
  static constexpr int STAGE = A_BYTES + B_BYTES;             // 32 or 48 KB
  static constexpr int STAGES = (192 * 1024) / STAGE;         // 6 or 4
  static constexpr int SMEM = STAGES * STAGE + 1024 + 512;
  static_assert(SMEM <= 227 * 1024, "dynamic shared memory above the opt-in limit");
};

template <bool FP8, int NB>
__global__ void __launch_bounds__(TC2_THREADS, 1)
    xf_tc2_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int kblocks,
                  int64_t total_iters, float* __restrict__ partials, int max_segs, unsigned* err) {
  using C = Tc2Cfg<NB>;
  constexpr int TC2_BN = C::BN, TC2_A_BYTES = C::A_BYTES, TC2_STAGE = C::STAGE, TC2_STAGES = C::STAGES;
  constexpr int KELEMS = FP8 ? 128 : 64;  // elements of K per k block
  constexpr int KSTEPS = TC_ROW_BYTES / 32;
  constexpr uint32_t IDESC = make_idesc<FP8>(2 * TC_BM, 256);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + TC2_STAGES * TC2_STAGE);
  uint64_t* empty = full + TC2_STAGES;
  uint64_t* tfull = empty + TC2_STAGES;
  uint64_t* tempty = tfull + 1;
  uint64_t* done = tempty + 1;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
  const int64_t it0 = ((int64_t)pair * total_iters) / npairs;
  const int64_t it1 = ((int64_t)(pair + 1) * total_iters) / npairs;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TC2_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 8);  // 4 epilogue warps in each CTA (the leader's barrier is the one used)
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {  // both CTAs take part in the pair's allocation
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC2_BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_mask = 0, last_parity = 0;
      for (int64_t it = it0; it < it1; ++it) {
        const int64_t tile = it / kblocks;
        const int kb = (int)(it - tile * kblocks);
        if (!mbar_wait_cl(&empty[stage], phase ^ 1u, abort_flag)) {
          *abort_flag = 1;
          set_error(err, ERR_TIMEOUT);
          break;
        }
        if (rank == 0) mbar_expect_tx(&full[stage], 2 * TC2_STAGE);  // both CTAs' copies
        const uint32_t bar_cl = map_to_rank(smem_u32(&full[stage]), 0);
        uint8_t* sA = smem + stage * TC2_STAGE;
        uint8_t* sB = sA + TC2_A_BYTES;
        tma_load_2d_pair(sA, &tmA, kb * KELEMS, (int)(tile * 2 * TC_BM + rank * TC_BM), bar_cl);
#pragma unroll
        for (int j = 0; j < NB; ++j)
          tma_load_2d_pair(sB + j * TC_BM * TC_ROW_BYTES, &tmB, kb * KELEMS, (int)(256 * j + rank * TC_BM), bar_cl);
        issued_mask |= 1u << stage;
        last_parity = (last_parity & ~(1u << stage)) | (phase << stage);
        if (++stage == TC2_STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
      // the leader's stage barriers count both CTAs' copies: every copy issued
      // has landed once they complete
      if (rank == 0)
        for (int s = 0; s < TC2_STAGES; ++s)
          if (issued_mask >> s & 1u) {
            volatile int no_abort = 0;
            mbar_wait_cl(&full[s], (last_parity >> s) & 1u, &no_abort);
          }
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      int sa = 0, seg = 0;
      uint32_t pa = 0;
      bool ok = true;
      int64_t it = it0;
      while (ok && it < it1) {
        const int64_t tile = it / kblocks;
        const int64_t seg_end = min(it1, (tile + 1) * kblocks);
        if (!mbar_wait_cl(tempty, ((uint32_t)seg & 1u) ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int64_t seg_begin = it;
        for (; it < seg_end; ++it) {
          if (!mbar_wait_cl(&full[sa], pa, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(smem + sa * TC2_STAGE);
          const uint32_t b0 = a0 + TC2_A_BYTES;
#pragma unroll
          for (int ks = 0; ks < KSTEPS; ++ks)
#pragma unroll
            for (int j = 0; j < NB; ++j)
              umma_pair<FP8>(tmem_base + (uint32_t)(j * 256), sw128_desc(a0 + ks * 32),
                             sw128_desc(b0 + j * TC_BM * TC_ROW_BYTES + ks * 32), IDESC,
                             (it > seg_begin || ks > 0) ? 1u : 0u);
          umma_commit_pair(&empty[sa], 3);
          if (++sa == TC2_STAGES) {
            sa = 0;
            pa ^= 1u;
          }
        }
        if (!ok) break;
        umma_commit_pair(tfull, 3);
        ++seg;
      }
      if (!ok) {
        *abort_flag = 1;
        set_error(err, ERR_TIMEOUT);
      }
      // all MMAs of the pair complete before either CTA releases its TMEM
      asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(done))
                   : "memory");
      volatile int no_abort = 0;
      mbar_wait_cl(done, 0, &no_abort);
    }
  } else {
    // epilogue: this CTA's 128 rows (its TMEM lanes) x 512 columns per segment
    const int ew = warp & 3;
    int seg = 0;
    int64_t it = it0;
    const uint32_t tempty_leader = map_to_rank(smem_u32(tempty), 0);
    while (it < it1) {
      const int64_t tile = it / kblocks;
      const int64_t seg_end = min(it1, (tile + 1) * kblocks);
      if (!mbar_wait_cl(tfull, (uint32_t)seg & 1u, abort_flag)) {
        *abort_flag = 1;
        set_error(err, ERR_TIMEOUT);
        break;
      }
      tc_fence_after();
      const int row = (int)rank * TC_BM + ew * 32 + lane;
      float* dst = partials + (((size_t)pair * max_segs + seg) * 2 * TC_BM + row) * TC2_BN;
      const uint32_t taddr = tmem_base + ((uint32_t)(ew * 32) << 16);
#pragma unroll 1
      for (int c = 0; c < TC2_BN; c += 16) {
        float v[16];
        tmem_ld16(taddr + (uint32_t)c, v);
#pragma unroll
        for (int q = 0; q < 16; q += 4) *(float4*)(dst + c + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_remote(tempty_leader);
      it = seg_end;
      ++seg;
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TC2_BN) : "memory");
}

// Y[r, c] = (sum over the CTAs that covered row tile r / 128 of their partial)
//           * row_scale[r] * col_scale[c]  (scales for FP8 only).
__global__ void tc_reduce_kernel(const float* __restrict__ partials, int max_segs, int BN, int BM, int kblocks,
                                 int64_t total, int G, int64_t n, int N, float* Y, int ldy,
                                 const float* __restrict__ rs, const float* __restrict__ cs) {
  // one thread per (row, 4 columns); the CTAs that covered the row's tile are
  // c0..c1 (stream-K ranges are contiguous), CTA q's segment index for the tile
  // is tile - (first tile of q)
  const int nq = (N + 3) >> 2;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nq) return;
  const int64_t r = t / nq;
  const int c = (int)(t - r * nq) * 4;
  const int64_t tile = r / BM;
  const int rr = (int)(r - tile * BM);
  const int64_t f_it = tile * kblocks, l_it = (tile + 1) * kblocks - 1;
  const int64_t c0 = ((f_it + 1) * G - 1) / total;
  const int64_t c1 = ((l_it + 1) * G - 1) / total;
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t q = c0; q <= c1; ++q) {
    const int64_t first_tile = ((q * total) / G) / kblocks;
    const int seg = (int)(tile - first_tile);
    const float4 v = *reinterpret_cast<const float4*>(partials + (((q * max_segs + seg) * BM + rr) * BN + c));
    s.x += v.x;
    s.y += v.y;
    s.z += v.z;
    s.w += v.w;
  }
  const float sv[4] = {s.x, s.y, s.z, s.w};
  const float rsr = rs ? rs[r] : 1.f;
#pragma unroll
  for (int u = 0; u < 4; ++u)
    if (c + u < N) Y[r * ldy + c + u] = rs ? sv[u] * rsr * cs[c + u] : sv[u];
}

// ------------------------------------------------------------ host side

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

bool tc_make_map(CUtensorMap* m, const void* base, bool fp8, uint64_t inner, uint64_t outer,
                     uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  const CUresult r = fn(m, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                        const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int tc_block_n(int N) {
  if (N <= 32) return 32;
  if (N <= 64) return 64;
  if (N <= 128) return 128;
  if (N <= 256) return 256;
  return 512;
}

struct TcPlan {
  int G, kblocks, mtiles, max_segs, bm;
  int64_t total;
};


// More than 128 columns: CTA pairs on 256-row tiles (G counts pairs).  At
// 256 columns the pairs measured 5 % (BF16) and 12 % (E4M3) faster than one
// CTA on a 256-row tile; at 512 they lift the product from 0.63 to 0.94 of
// the tensor peak.
static bool tc_pair(int N) { return N > 128; }

static TcPlan tc_plan(int64_t m, int64_t kdim, bool fp8, int bm = TC_BM, bool pairs = false) {
  TcPlan p;
  const int kel = fp8 ? 128 : 64;
  p.bm = bm;
  p.kblocks = (int)((kdim + kel - 1) / kel);
  p.mtiles = (int)((m + bm - 1) / bm);
  p.total = (int64_t)p.kblocks * p.mtiles;
  p.G = (int)std::min<int64_t>(pairs ? num_sms() / 2 : num_sms(), p.total);
  p.max_segs = 1;
  for (int c = 0; c < p.G; ++c) {
    const int64_t a = ((int64_t)c * p.total) / p.G, b = ((int64_t)(c + 1) * p.total) / p.G;
    const int segs = (int)((b - 1) / p.kblocks - a / p.kblocks + 1);
    if (segs > p.max_segs) p.max_segs = segs;
  }
  return p;
}

size_t tc_gemm_ws_floats(int64_t m, int64_t kdim, int BN) {
  // largest of the plans a product of this width can use
  const bool pairs = tc_pair(BN);
  const int bm = pairs ? 2 * TC_BM : TC_BM;
  size_t need = 0;
  for (int f = 0; f < 2; ++f) {
    const TcPlan p = tc_plan(m, kdim, f != 0, bm, pairs);
    need = std::max(need, (size_t)p.G * p.max_segs * bm * BN);
  }
  return need;
}

size_t xf_tc_ws_floats(int64_t n, int BN) { return tc_gemm_ws_floats(n, n, BN); }

// Fpack[c, i] = F[i, c] (zero padded to Npad x ldp) through 32 x 32 tiles in
// shared memory: both the reads of F rows and the writes of Fpack rows coalesce.
__global__ void pack_ft_bf16_kernel(const float* F, int64_t n, int ldf, int N, int Npad,
                                    __nv_bfloat16* out, int64_t ldp) {
  __shared__ float tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int64_t i = i0 + y;
    const int c = c0 + threadIdx.x;
    tile[y][threadIdx.x] = (i < n && c < N) ? F[i * ldf + c] : 0.f;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int c = c0 + y;
    const int64_t i = i0 + threadIdx.x;
    if (c < Npad && i < ldp) out[(int64_t)c * ldp + i] = __float2bfloat16_rn(tile[threadIdx.x][y]);
  }
}

cudaError_t pack_ft_bf16(const float* F, int64_t n, int ldf, int N, int Npad, void* out, int64_t ldp,
                         cudaStream_t st) {
  const dim3 grid((unsigned)((ldp + 31) / 32), (unsigned)((Npad + 31) / 32));
  pack_ft_bf16_kernel<<<grid, dim3(32, 8), 0, st>>>(F, n, ldf, N, Npad, (__nv_bfloat16*)out, ldp);
  count_launches(1);
  return cudaGetLastError();
}

__global__ void colmax_kernel(const float* F, int64_t n, int ldf, int N, float* cs) {
  __shared__ float sh[32];
  const int c = blockIdx.x;
  float m = 0.f;
  if (c < N)
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, fabsf(F[i * ldf + c]));
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, sh[w]);
    cs[c] = t > 0.f ? t / 448.0f : 1.0f;
  }
}

__global__ void pack_ft_fp8_kernel(const float* F, int64_t n, int ldf, int N, int Npad, uint8_t* out,
                                   int64_t ldp, const float* cs) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)Npad * ldp) return;
  const int64_t c = t / ldp, i = t - c * ldp;
  const float v = (c < N && i < n) ? F[i * ldf + c] / cs[c] : 0.f;
  const __nv_fp8_e4m3 q(v);
  out[t] = q.__x;
}

cudaError_t pack_ft_fp8(const float* F, int64_t n, int ldf, int N, int Npad, void* out, int64_t ldp,
                        float* col_scale, cudaStream_t st) {
  colmax_kernel<<<Npad, 256, 0, st>>>(F, n, ldf, N, col_scale);
  const int64_t work = (int64_t)Npad * ldp;
  pack_ft_fp8_kernel<<<(int)((work + 255) / 256), 256, 0, st>>>(F, n, ldf, N, Npad, (uint8_t*)out, ldp,
                                                                col_scale);
  count_launches(2);
  return cudaGetLastError();
}

template <bool FP8, int NB>
static cudaError_t launch_tc2(const CUtensorMap& ma, const CUtensorMap& mb, const TcPlan& p, float* ws,
                              unsigned* err, cudaStream_t st) {
  using C = Tc2Cfg<NB>;
  cudaError_t e =
      cudaFuncSetAttribute(xf_tc2_kernel<FP8, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * p.G));
  cfg.blockDim = dim3(TC2_THREADS);
  cfg.dynamicSmemBytes = C::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, xf_tc2_kernel<FP8, NB>, ma, mb, p.kblocks, p.total, ws, p.max_segs, err);
  count_launches(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int BN, bool FP8>
static cudaError_t launch_tc(const CUtensorMap& ma, const CUtensorMap& mb, const TcPlan& p, float* ws,
                             unsigned* err, cudaStream_t st) {
  using C = TcCfg<BN>;
  cudaError_t e = cudaFuncSetAttribute(xf_tc_kernel<BN, FP8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       C::SMEM);
  if (e != cudaSuccess) return e;
  xf_tc_kernel<BN, FP8><<<p.G, XF_THREADS, C::SMEM, st>>>(ma, mb, p.kblocks, p.total, ws, p.max_segs, err);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t xf_tc(int fmt, const void* X, int64_t ldx, const float* row_scale, int64_t n,
                  const void* Fpack, int64_t ldp, const float* col_scale, int N, float* Y, int ldy,
                  float* ws, size_t ws_floats, unsigned* err, cudaStream_t st, cudaEvent_t ev_begin,
                  cudaEvent_t ev_end) {
  return tc_gemm(fmt, X, ldx, n, n, row_scale, Fpack, ldp, col_scale, N, Y, ldy, ws, ws_floats, err, st, ev_begin,
                 ev_end);
}

cudaError_t tc_gemm(int fmt, const void* X, int64_t ldx, int64_t m, int64_t n, const float* row_scale,
                    const void* Fpack, int64_t ldp, const float* col_scale, int N, float* Y, int ldy, float* ws,
                    size_t ws_floats, unsigned* err, cudaStream_t st, cudaEvent_t ev_begin, cudaEvent_t ev_end) {
  const bool fp8 = fmt == 3;
  if (!fp8 && fmt != 2) return cudaErrorInvalidValue;
  const int BN = tc_block_n(N);
  if (N > 512) return cudaErrorInvalidValue;
  const size_t es = fp8 ? 1 : 2;
  // TMA: 16-byte aligned bases and row pitches
  if (((uintptr_t)X & 15) || ((uintptr_t)Fpack & 15) || (ldx * es) % 16 || (ldp * es) % 16)
    return cudaErrorInvalidValue;
  const bool pairs = tc_pair(N);
  const TcPlan p = tc_plan(m, n, fp8, pairs ? 2 * TC_BM : TC_BM, pairs);
  if (ws_floats < (size_t)p.G * p.max_segs * p.bm * BN) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  const uint32_t kel = fp8 ? 128 : 64;
  if (!tc_make_map(&ma, X, fp8, (uint64_t)n, (uint64_t)m, (uint64_t)ldx * es, kel, TC_BM))
    return cudaErrorInvalidValue;
  if (!tc_make_map(&mb, Fpack, fp8, (uint64_t)n, (uint64_t)BN, (uint64_t)ldp * es, kel,
                   (uint32_t)(pairs ? TC_BM : BN)))
    return cudaErrorInvalidValue;
  cudaError_t e;
  if (ev_begin) cudaEventRecord(ev_begin, st);
  if (fp8) {
    switch (BN) {
      case 32: e = launch_tc<32, true>(ma, mb, p, ws, err, st); break;
      case 64: e = launch_tc<64, true>(ma, mb, p, ws, err, st); break;
      case 128: e = launch_tc<128, true>(ma, mb, p, ws, err, st); break;
      case 256: e = launch_tc2<true, 1>(ma, mb, p, ws, err, st); break;
      default: e = launch_tc2<true, 2>(ma, mb, p, ws, err, st); break;
    }
  } else {
    switch (BN) {
      case 32: e = launch_tc<32, false>(ma, mb, p, ws, err, st); break;
      case 64: e = launch_tc<64, false>(ma, mb, p, ws, err, st); break;
      case 128: e = launch_tc<128, false>(ma, mb, p, ws, err, st); break;
      case 256: e = launch_tc2<false, 1>(ma, mb, p, ws, err, st); break;
      default: e = launch_tc2<false, 2>(ma, mb, p, ws, err, st); break;
    }
  }
  if (ev_end) cudaEventRecord(ev_end, st);
  if (e != cudaSuccess) return e;
  const int64_t work = m * ((N + 3) / 4);
  tc_reduce_kernel<<<(int)((work + 255) / 256), 256, 0, st>>>(
      ws, p.max_segs, BN, p.bm, p.kblocks, p.total, p.G, m, N, Y, ldy, fp8 ? row_scale : nullptr,
      fp8 ? col_scale : nullptr);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace symnmf
