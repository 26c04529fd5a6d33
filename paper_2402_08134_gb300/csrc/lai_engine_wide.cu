// Engine launches for G held as 32, 48 or 64 square (24 < k <= 64).
#include "lai_engine.cuh"

namespace symnmf {

cudaError_t lai_engine_launch_wide(int gp, const LaiArgs& a, bool allow_resident, cudaStream_t st,
                                   cudaEvent_t ev0, cudaEvent_t ev1) {
  switch (gp) {
    case 32:
      return launch_engine<32>(a, allow_resident, st, ev0, ev1);
    case 48:
      return launch_engine<48>(a, allow_resident, st, ev0, ev1);
    case 64:
      return launch_engine<64>(a, allow_resident, st, ev0, ev1);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace symnmf
