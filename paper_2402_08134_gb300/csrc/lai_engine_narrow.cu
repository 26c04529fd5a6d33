// Engine launches for G held as 8, 16, 20 or 24 square (k <= 24).
#include "lai_engine.cuh"

namespace symnmf {

cudaError_t lai_engine_launch_narrow(int gp, const LaiArgs& a, bool allow_resident, cudaStream_t st,
                                     cudaEvent_t ev0, cudaEvent_t ev1) {
  switch (gp) {
    case 8:
      return launch_engine<8>(a, allow_resident, st, ev0, ev1);
    case 16:
      return launch_engine<16>(a, allow_resident, st, ev0, ev1);
    case 20:
      return launch_engine<20>(a, allow_resident, st, ev0, ev1);
    case 24:
      return launch_engine<24>(a, allow_resident, st, ev0, ev1);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace symnmf
