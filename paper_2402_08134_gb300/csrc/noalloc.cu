// Gram matrix without any allocation, for callers that must not allocate
// device memory (see symnmf_gram_noalloc in include/symnmf.h).
//
// The cross-product kernel needs scratch for its per-block partial sums.
// symnmf_gram gets that scratch from cudaMallocAsync on every call; here it
// lives in a file-scope device array instead, which every GPU that loads this
// library holds until the process exits.  In host code the array's name is
// only a host-side stand-in, not a device address, so every call looks up
// the array's address on the current device with cudaGetSymbolAddress (no
// allocation; the first call on a device also loads the library's device
// symbols there).  Looking it up on every call, rather than caching it,
// keeps the address right after a cudaDeviceReset, which unloads the module
// and may place the array elsewhere when it is loaded again.
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

// Device addresses of the two arrays on the current device.
cudaError_t scratch_for_current_device(double** ws, unsigned** counter) {
  void* w = nullptr;
  void* c = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&w, g_gram_scratch);
  if (e != cudaSuccess) return e;
  e = cudaGetSymbolAddress(&c, g_gram_counter);
  if (e != cudaSuccess) return e;
  *ws = static_cast<double*>(w);
  *counter = static_cast<unsigned*>(c);
  return cudaSuccess;
}

}  // namespace

extern "C" symnmf_status symnmf_gram_noalloc(const float* F, int64_t n, int N, double* G, void* stream) {
  if (!F || !G || n < 1 || N < 1) return SYMNMF_EINVAL;
  if (N > NA_MAX_WIDTH) return SYMNMF_EINVAL;  // beyond the static scratch: at most 64 columns
  // at most NA_BLOCKS_PER_SM cross-product blocks per SM: their partials fit the array
  if (NA_BLOCKS_PER_SM * symnmf::num_sms() > NA_MAX_BLOCKS) return SYMNMF_EUNSUPPORTED;
  double* ws = nullptr;
  unsigned* counter = nullptr;
  cudaError_t e = scratch_for_current_device(&ws, &counter);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return symnmf::to_status(e);
  }
  cudaStream_t st = (cudaStream_t)stream;
  // the counter must start at zero; the partials are overwritten before they are read
  e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return symnmf::to_status(e);
  e = symnmf::xcross(F, N, N, F, N, N, n, nullptr, nullptr, nullptr, nullptr, 0.0, G, nullptr, ws, counter, st,
                     NA_BLOCKS_PER_SM);
  return symnmf::to_status(e);
}
