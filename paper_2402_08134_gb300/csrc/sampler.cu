// Hybrid leverage-score sampling (Section "Practical Considerations for
// LvS-SymNMF"): rows with l_i / k >= tau are kept deterministically (weight 1,
// ascending order); s_R = max(s - s_D, 0) rows are drawn with replacement from
// the rest with probability proportional to l_i.
//
// The draw map is exact integer arithmetic so that any summation order gives
// the same indices: q_i = floor(l_i 2^40) (0 for kept rows), C = inclusive
// prefix of q, T = C[n-1]; draw j uses Philox counter (j, iter, side, 3),
// u = x0 2^32 + x1, r = floor(u T / 2^64) and takes the first i with C_i > r.
// Weights on S^T S: mass_R / (s_R l_i), mass_R = sum over non-kept rows of l.
//
// Three passes, no inter-block waiting: per-block totals, a one-block scan
// of the block totals, then per-block compaction + prefix writes; finally
// one thread per draw.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace symnmf {

constexpr int SP_THREADS = 256, SP_ITEMS = 4, SP_TILE = SP_THREADS * SP_ITEMS;

int sampler_blocks(int64_t n) { return (int)((n + SP_TILE - 1) / SP_TILE); }

__device__ __forceinline__ void classify(const double* lev, int64_t i, int64_t n, double thr, bool& det,
                                         uint64_t& q, double& l) {
  det = false;
  q = 0;
  l = 0.0;
  if (i < n) {
    l = lev[i];
    det = l >= thr;
    q = det ? 0ull : (uint64_t)floor(l * 1099511627776.0);  // 2^40
  }
}

__global__ void __launch_bounds__(SP_THREADS) sample_pass1(const double* __restrict__ lev, int64_t n,
                                                           double thr, int* blk_cnt,
                                                           unsigned long long* blk_q,
                                                           double* blk_theta, double* blk_mass) {
  __shared__ double shd[32];
  __shared__ unsigned long long shq[32];
  __shared__ int shc[32];
  const int64_t base = (int64_t)blockIdx.x * SP_TILE;
  int c = 0;
  uint64_t qs = 0;
  double th = 0.0, ms = 0.0;
#pragma unroll
  for (int e = 0; e < SP_ITEMS; ++e) {
    const int64_t i = base + e * SP_THREADS + threadIdx.x;
    bool det;
    uint64_t q;
    double l;
    classify(lev, i, n, thr, det, q, l);
    c += det;
    qs += q;
    if (det) th += l; else ms += l;
  }
  c = block_sum(c, shc);
  qs = block_sum((unsigned long long)qs, shq);
  th = block_sum(th, shd);
  ms = block_sum(ms, shd);
  if (threadIdx.x == 0) {
    blk_cnt[blockIdx.x] = c;
    blk_q[blockIdx.x] = qs;
    blk_theta[blockIdx.x] = th;
    blk_mass[blockIdx.x] = ms;
  }
}

// One block: exclusive scans of the block counts / weights (in place),
// totals, s_D, s_R, s_tot.
__global__ void __launch_bounds__(1024) sample_scan(int nblk, int* blk_cnt, unsigned long long* blk_q,
                                                    const double* blk_theta, const double* blk_mass,
                                                    int s, int cap, int* counts, double* sums,
                                                    unsigned long long* total) {
  __shared__ int sc[1024];
  __shared__ unsigned long long sq[1024];
  const int t = threadIdx.x;
  const int per = (nblk + 1023) / 1024;
  const int b0 = min(nblk, t * per), b1 = min(nblk, b0 + per);
  int c = 0;
  unsigned long long q = 0;
  for (int b = b0; b < b1; ++b) {
    c += blk_cnt[b];
    q += blk_q[b];
  }
  sc[t] = c;
  sq[t] = q;
  __syncthreads();
  // Hillis-Steele inclusive scan over the 1024 thread totals
  for (int o = 1; o < 1024; o <<= 1) {
    const int vc = t >= o ? sc[t - o] : 0;
    const unsigned long long vq = t >= o ? sq[t - o] : 0ull;
    __syncthreads();
    sc[t] += vc;
    sq[t] += vq;
    __syncthreads();
  }
  int oc = t > 0 ? sc[t - 1] : 0;
  unsigned long long oq = t > 0 ? sq[t - 1] : 0ull;
  for (int b = b0; b < b1; ++b) {
    const int vc = blk_cnt[b];
    const unsigned long long vq = blk_q[b];
    blk_cnt[b] = oc;
    blk_q[b] = oq;
    oc += vc;
    oq += vq;
  }
  // theta and the non-kept mass: each thread's blocks in order, then a fixed
  // tree (deterministic; a serial FP64 loop over all blocks was slow here)
  __shared__ double sh[32];
  double th = 0.0, ms = 0.0;
  for (int b = b0; b < b1; ++b) {
    th += blk_theta[b];
    ms += blk_mass[b];
  }
  th = block_sum(th, sh);
  ms = block_sum(ms, sh);
  if (t == 0) {
    const int sD = sc[1023];
    const unsigned long long T = sq[1023];
    int sR = (T > 0ull) ? max(s - sD, 0) : 0;
    int stot = sD + sR;
    if (stot > cap) {  // cannot happen with cap >= max(n, s); clamp defensively
      stot = cap;
      sR = max(0, cap - sD);
    }
    counts[0] = min(sD, cap);
    counts[1] = sR;
    counts[2] = stot;
    sums[0] = th;
    sums[1] = ms;
    *total = T;
  }
}

__global__ void __launch_bounds__(SP_THREADS) sample_pass2(const double* __restrict__ lev, int64_t n,
                                                           double thr, const int* blk_cnt,
                                                           const unsigned long long* blk_q,
                                                           unsigned long long* cdf, int32_t* idx,
                                                           float* wt, int cap) {
  __shared__ int wc[SP_THREADS / 32];
  __shared__ unsigned long long wq[SP_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * SP_TILE;
  int carry_c = blk_cnt[blockIdx.x];
  unsigned long long carry_q = blk_q[blockIdx.x];
  for (int e = 0; e < SP_ITEMS; ++e) {
    const int64_t i = base + e * SP_THREADS + threadIdx.x;
    bool det;
    uint64_t q;
    double l;
    classify(lev, i, n, thr, det, q, l);
    // inclusive warp scans
    int c = det ? 1 : 0;
    unsigned long long qq = q;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int vc = __shfl_up_sync(0xffffffffu, c, o);
      const unsigned long long vq = __shfl_up_sync(0xffffffffu, qq, o);
      if (lane >= o) {
        c += vc;
        qq += vq;
      }
    }
    if (lane == 31) {
      wc[wid] = c;
      wq[wid] = qq;
    }
    __syncthreads();
    int offc = carry_c;
    unsigned long long offq = carry_q;
    for (int w = 0; w < wid; ++w) {
      offc += wc[w];
      offq += wq[w];
    }
    if (i < n) {
      cdf[i] = offq + qq;  // inclusive prefix of q
      if (det) {
        const int pos = offc + c - 1;
        if (pos < cap) {
          idx[pos] = (int32_t)i;
          wt[pos] = 1.0f;
        }
      }
    }
    int totc = 0;
    unsigned long long totq = 0;
    for (int w = 0; w < SP_THREADS / 32; ++w) {
      totc += wc[w];
      totq += wq[w];
    }
    carry_c += totc;
    carry_q += totq;
    __syncthreads();
  }
}

__global__ void sample_draw(const double* __restrict__ lev, int64_t n,
                            const unsigned long long* __restrict__ cdf, const int* counts,
                            const double* sums, const unsigned long long* total, uint32_t iter,
                            uint32_t side, uint32_t k0, uint32_t k1, int32_t* idx, float* wt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int sD = counts[0], sR = counts[1];
  if (j >= sR) return;
  const Philox4 r = philox4x32_10((uint32_t)j, iter, side, TAG_SAMPLE, k0, k1);
  const uint64_t u = ((uint64_t)r.x0 << 32) | (uint64_t)r.x1;
  const uint64_t target = mulhi_u64(u, *total);
  // first i with cdf[i] > target
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (cdf[mid] > target) hi = mid; else lo = mid + 1;
  }
  idx[sD + j] = (int32_t)lo;
  wt[sD + j] = (float)(sums[1] / ((double)sR * lev[lo]));
}

cudaError_t hybrid_sample(SampleBufs& b, int64_t n, int k, double tau, int s, uint64_t seed,
                          uint32_t iter, uint32_t side, cudaStream_t st) {
  const int nblk = sampler_blocks(n);
  if (nblk > b.nblk_cap) return cudaErrorInvalidValue;
  const double thr = tau * (double)k;
  sample_pass1<<<nblk, SP_THREADS, 0, st>>>(b.lev, n, thr, b.blk_cnt, b.blk_q, b.blk_theta, b.blk_mass);
  sample_scan<<<1, 1024, 0, st>>>(nblk, b.blk_cnt, b.blk_q, b.blk_theta, b.blk_mass, s, b.cap, b.counts,
                                  b.sums, b.total);
  sample_pass2<<<nblk, SP_THREADS, 0, st>>>(b.lev, n, thr, b.blk_cnt, b.blk_q, b.cdf, b.idx, b.wt,
                                            b.cap);
  const int dgrid = (s + 255) / 256;
  if (dgrid > 0)
    sample_draw<<<dgrid, 256, 0, st>>>(b.lev, n, b.cdf, b.counts, b.sums, b.total, iter, side,
                                       (uint32_t)seed, (uint32_t)(seed >> 32), b.idx, b.wt);
  count_launches(dgrid > 0 ? 4 : 3);
  return cudaGetLastError();
}

}  // namespace symnmf
