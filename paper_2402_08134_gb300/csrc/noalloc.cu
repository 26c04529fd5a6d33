// Gram matrix without any allocation, for callers that must not allocate
// device memory (see symnmf_gram_noalloc in include/symnmf.h).
//
// The cross-product kernel needs scratch for its per-block partial sums.
// symnmf_gram gets that scratch from cudaMallocAsync on every call; here it
// lives in a file-scope device array instead, which every GPU that loads this
// library holds until the process exits.  The array's device address is
// looked up once per device with cudaGetSymbolAddress (in host code the
// symbol is only a host-side stand-in, not a device address).
#include <mutex>

#include "../../include/symnmf.h"
#include "common.cuh"
#include "handle.h"
#include "kernels.h"

namespace {

constexpr int NA_MAX_WIDTH = 64;    // widest F accepted (G is at most 64 x 64)
constexpr int NA_BLOCKS_PER_SM = 2;  // cross-product blocks per SM asked for
constexpr int NA_MAX_BLOCKS = 512;   // block partials the array can hold (2 per SM, up to 256 SMs)
constexpr size_t NA_SCRATCH_DOUBLES = (size_t)NA_MAX_BLOCKS * NA_MAX_WIDTH * NA_MAX_WIDTH + 64;

// 16 MiB of block partials plus the kernel's arrival counter (a separate line).
__device__ __align__(256) double g_gram_scratch[NA_SCRATCH_DOUBLES];
__device__ __align__(256) unsigned g_gram_counter[64];

constexpr int NA_MAX_DEVICES = 64;
struct DevScratch {
  double* ws = nullptr;
  unsigned* counter = nullptr;
};
DevScratch g_dev[NA_MAX_DEVICES];
std::mutex g_mu;

// Device addresses of the two arrays for the current device (set up once per device).
cudaError_t scratch_for_current_device(DevScratch* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  DevScratch& d = g_dev[dev];
  if (!d.ws) {
    void* ws = nullptr;
    void* ctr = nullptr;
    e = cudaGetSymbolAddress(&ws, g_gram_scratch);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress(&ctr, g_gram_counter);
    if (e != cudaSuccess) return e;
    d.ws = static_cast<double*>(ws);
    d.counter = static_cast<unsigned*>(ctr);
  }
  *out = d;
  return cudaSuccess;
}

}  // namespace

extern "C" symnmf_status symnmf_gram_noalloc(const float* F, int64_t n, int N, double* G, void* stream) {
  if (!F || !G || n < 1 || N < 1) return SYMNMF_EINVAL;
  if (N > NA_MAX_WIDTH) return SYMNMF_EINVAL;  // beyond the static scratch: at most 64 columns
  // at most NA_BLOCKS_PER_SM cross-product blocks per SM: their partials fit the array
  if (NA_BLOCKS_PER_SM * symnmf::num_sms() > NA_MAX_BLOCKS) return SYMNMF_EUNSUPPORTED;
  DevScratch s;
  cudaError_t e = scratch_for_current_device(&s);
  if (e != cudaSuccess) return symnmf::to_status(e);
  cudaStream_t st = (cudaStream_t)stream;
  // the counter must start at zero; the partials are overwritten before they are read
  e = cudaMemsetAsync(s.counter, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return symnmf::to_status(e);
  e = symnmf::xcross(F, N, N, F, N, N, n, nullptr, nullptr, nullptr, nullptr, 0.0, G, nullptr, s.ws, s.counter,
                     st, NA_BLOCKS_PER_SM);
  return symnmf::to_status(e);
}
