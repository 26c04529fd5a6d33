// Warm-start network (filled in below the core path).
#include "../../include/symnmf.h"

extern "C" symnmf_status symnmf_mlp_create(int, int, int, int, uint64_t, void*, symnmf_mlp_t* out) {
  if (out) *out = nullptr;
  return SYMNMF_EUNSUPPORTED;
}
extern "C" void symnmf_mlp_destroy(symnmf_mlp_t) {}
extern "C" symnmf_status symnmf_mlp_get_params(symnmf_mlp_t, float*, int64_t) { return SYMNMF_EUNSUPPORTED; }
extern "C" symnmf_status symnmf_mlp_set_params(symnmf_mlp_t, const float*, int64_t) { return SYMNMF_EUNSUPPORTED; }
extern "C" int64_t symnmf_mlp_param_count(symnmf_mlp_t) { return 0; }
extern "C" symnmf_status symnmf_mlp_forward(symnmf_mlp_t, const float*, int64_t, float*) { return SYMNMF_EUNSUPPORTED; }
extern "C" symnmf_status symnmf_mlp_loss_grad(symnmf_mlp_t, const float*, const float*, int64_t, float*, double*) {
  return SYMNMF_EUNSUPPORTED;
}
extern "C" symnmf_status symnmf_mlp_adam(symnmf_mlp_t, float, int) { return SYMNMF_EUNSUPPORTED; }
extern "C" symnmf_status symnmf_warm_start(symnmf_t, symnmf_mlp_t, const float*) { return SYMNMF_EUNSUPPORTED; }
