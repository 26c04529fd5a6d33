// Solver handle layout (internal).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/symnmf.h"
#include "kernels.h"

namespace symnmf {

// Slots of the per-handle device scalar array.
enum {
  S_ALPHA = 0,
  S_NORM2 = 1,      // ||X||_F^2
  S_LAI_NORM2 = 2,  // sum lambda^2 = ||U Lambda U^T||_F^2
  S_MAX = 3,        // xstats: max, sum, sum of squares (S_MAX .. S_MAX + 2)
  S_MEAN = 6,
  S_PART = 7,       // 2 slots: sum F_new .* Y, ||F_new - F_fix||^2
  S_PART2 = 9,      // 2 slots
  S_PART3 = 11,     // 2 slots
  S_PG = 13,
  S_OBJ = 14,
  S_ZERO = 15,      // stays 0
  S_XHI_MAX = 16,   // 3 slots for the float32 copy
  S_XHI_NORM2 = 18,
  S_ADA = 20,       // 2 slots: ||B||_F^2 of the adaptive range finder's check
  S_COMP_NORM2 = 22,  // 2 slots: ||Q^T X||_F^2 of the compressed problem
  S_CG = 24,        // GN_COUNT slots: scalars of the PGNCG conjugate-gradient loop
  S_RES = 32,       // 2 slots: sum W .* (X H), ||W - H||^2 of a residual evaluation
  S_COUNT = 40
};
constexpr int OBJ_RING = 4096;
constexpr int LOOP_MAX = 1024;  // residual checks one symnmf_sweep_to_target call records

symnmf_status to_status(cudaError_t e);

}  // namespace symnmf

struct symnmf_ctx {
  symnmf_problem p{};
  symnmf_options o{};
  cudaStream_t st = nullptr;
  int64_t n = 0, ldx = 0, ldx_hi = 0, ldp = 0;
  int k = 0;
  double alpha = 0.0, normX2 = 0.0;
  std::string msg;
  std::vector<void*> allocs;       // stream-ordered (pool) allocations, freed on st
  std::vector<void*> allocs_sync;  // plain cudaMalloc (made while capturing)

  float *H = nullptr, *W = nullptr, *Y = nullptr;
  double* Gd[2] = {nullptr, nullptr};  // [0] H^T H, [1] W^T W (FP64)
  float* Gf[2] = {nullptr, nullptr};
  double* Gs_d = nullptr;  // sampled / scratch Gram
  float* Gs_f = nullptr;
  double* scal = nullptr;
  double* obj_ring = nullptr;
  int* obj_cnt = nullptr;
  double* ws = nullptr;
  size_t ws_doubles = 0;
  unsigned* counters = nullptr;  // last-block counters, one per launch site family
  unsigned* err = nullptr;       // device error word
  float* gemm_ws = nullptr;
  size_t gemm_ws_floats = 0;
  void* fpack = nullptr;
  size_t fpack_bytes = 0;
  float* colscale = nullptr;

  // LAI
  int l = 0, lai_cap = 0, lai_version = 0;
  bool lai_ready = false;
  bool lai_from_user = false;  // U, Lambda given by symnmf_set_lai (no basis Q kept)
  float *Om = nullptr, *Qa = nullptr, *Qb = nullptr, *U = nullptr, *Mf = nullptr;
  double *Sm_d = nullptr, *V_d = nullptr, *lam = nullptr, *ev = nullptr;
  float *Sm_f = nullptr, *Rl_f = nullptr;
  float *Qk = nullptr, *Bk = nullptr;  // the sketch's final basis Q and X Q (n x l each)
  char* eng_ws = nullptr;    // LAI engine workspace
  double* eng_G = nullptr;   // Grams after the engine's last sweep
  unsigned* eng_bar = nullptr;
  double *cq_part = nullptr, *cq_fin = nullptr;  // CholeskyQR engine buffers
  float *cq_Rf = nullptr, *cq_rinv = nullptr;

  // PGNCG: residual R, direction P, step Z, J^T J P (n x k each), P^T H (k x k)
  float *cgR = nullptr, *cgP = nullptr, *cgZ = nullptr, *cgY = nullptr, *cgPtH = nullptr;
  double* cgPtH_d = nullptr;
  double* cg_ws = nullptr;

  // LvS
  symnmf::SampleBufs sb{};
  double* Rinv_d = nullptr;
  float* Rinv_f = nullptr;
  int sample_side = -1;

  // recorded sweep bodies
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    int src = -1, rule = -1, lai_version = -1;
    uint64_t nkernels = 0;
  } graphs[6];
  bool capturing = false;
  // factor bookkeeping: fac_version counts writes of W / H by anything but the
  // LAI engine; the engine may resume from its own saved state (skipping its
  // prologue) while nothing else has written the factors or the operator since
  uint64_t fac_version = 0;
  bool eng_resume_ok = false;
  uint64_t eng_fac_version = 0;
  int eng_lai_version = -1;
  bool grams_fresh = false;  // Gd / Gf hold H^T H and W^T W of the current factors
  cudaStream_t cap_st = nullptr;

  // the device-side check loop of symnmf_sweep_to_target: one graph (a WHILE
  // node around chunk, check and decision), keyed by its parameters and by the
  // buffers it was recorded with
  struct Loop {
    cudaGraphExec_t exec = nullptr;
    int check = -1, chunk = 0, max_checks = 0, l = 0;
    double target = 0.0;
    const void* bufs[5] = {};
    uint64_t nkernels = 0;  // kernels per body pass
    // parameters of the previous call: a loop is recorded only when a call
    // repeats them (recording costs more than the host round trips it saves
    // in one solve)
    int prev_check = -1, prev_chunk = 0, prev_max_checks = 0, prev_l = 0;
    double prev_target = 0.0;
  } loop;
  int* loop_i = nullptr;        // [0] checks made, [1] continue flag
  double* loop_nr = nullptr;    // normalized residual of each check (LOOP_MAX)

  // live timing of the tensor-core product kernel (eager calls only)
  bool profiling = false;
  size_t prof_used = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
  std::vector<double> prof_bytes;
  size_t lprof_used = 0;  // LvS halves timed while profiling: 4 events each
  std::vector<cudaEvent_t> lprof_events;
  size_t eprof_used = 0;  // LAI sweep engine launches timed while profiling
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> eprof_events;
  std::vector<double> eprof_flops;
};
