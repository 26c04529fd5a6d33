// Host side of the persistent LAI sweep engine (the kernels and their design
// are in lai_engine.cuh): workspace size, FLOP count, and the launch.
#include "lai_engine.cuh"

namespace symnmf {

size_t lai_engine_ws_bytes(int l, int k, int obj_cap) {
  const size_t grid = (size_t)num_sms();
  return le_align(256) + le_align((size_t)2 * le_entries(l, k) * 8) + le_align((size_t)obj_cap * grid * 8) +
         le_align(grid * le_rec_entries(l, k) * 4) +
         le_align((size_t)2 * le_state_floats(l, k, le_gp(k)) * 4);
}

double lai_engine_flops(int64_t n, int k, int l, int nsweeps, bool prologue) {
  const double half = (double)n * ((double)l * k + (double)k * k + (double)l * k + 0.5 * k * (k + 1));
  const double pro = prologue ? (double)n * ((double)l * k + 0.5 * k * (k + 1)) : 0.0;
  return 2.0 * (pro + 2.0 * nsweeps * half);
}

cudaError_t lai_engine(const float* U, const double* lam, float* W, float* H, int64_t n, int k, int l,
                       int nsweeps, double alpha, const double* normX2, void* ws, double* obj, int obj_cap,
                       double* Gout, unsigned* err, bool allow_resident, cudaStream_t st, cudaEvent_t ev0,
                       cudaEvent_t ev1, bool resume, double* Gd_h, double* Gd_w, float* Gf_h, float* Gf_w) {
  if (k < 1 || k > 64 || l < 1 || l > 96 || n < 1 || nsweeps > obj_cap) return cudaErrorInvalidValue;
  char* b = static_cast<char*>(ws);
  const size_t grid = (size_t)num_sms();
  unsigned* bar = reinterpret_cast<unsigned*>(b);
  b += le_align(256);
  double* fin = reinterpret_cast<double*>(b);
  b += le_align((size_t)2 * le_entries(l, k) * 8);
  double* objp = reinterpret_cast<double*>(b);
  b += le_align((size_t)obj_cap * grid * 8);
  float* part = reinterpret_cast<float*>(b);
  b += le_align(grid * le_rec_entries(l, k) * 4);
  float* state = reinterpret_cast<float*>(b);
  const int gp = le_gp(k);
  LaiArgs a{U,    lam,   W,    H,   n,       k,    l,   nsweeps, (float)alpha, alpha, normX2, part,
            fin,  state, objp, obj, obj_cap, Gout, bar, err,     256,          gp,    0,     resume ? 1 : 0,
            Gd_h, Gd_w,  Gf_h, Gf_w};
  if (!Gd_h || !Gd_w || !Gf_h || !Gf_w) a.Gd_h = a.Gd_w = nullptr, a.Gf_h = a.Gf_w = nullptr;
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  // the state's pad entries are never written by the kernel (a resumed launch
  // keeps the state the previous one saved)
  if (!resume) {
    e = cudaMemsetAsync(state, 0, (size_t)2 * le_state_floats(l, k, gp) * sizeof(float), st);
    if (e != cudaSuccess) return e;
  }
  return gp <= 24 ? lai_engine_launch_narrow(gp, a, allow_resident, st, ev0, ev1)
                  : lai_engine_launch_wide(gp, a, allow_resident, st, ev0, ev1);
}

}  // namespace symnmf
