// Host-side launchers of the sm_103a kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace symnmf {

// Counts kernel launches for symnmf_launch_count().
void count_launches(uint64_t n);
int num_sms();

// ----------------------------------------------------------------- reductions
// Over a dense X (fmt as symnmf_xfmt, FP8 with row scales) or CSR values:
// out[0] = max, out[1] = sum, out[2] = sum of squares (FP64).
// ws: >= 3 * 1024 doubles + 1 uint scratch (counter) ; counter must be zero.
cudaError_t xstats(int fmt, const void* x, int64_t ldx, const float* row_scale, int64_t n,
                   const int64_t* row_ptr, int64_t nnz, double* out, double* ws, unsigned* counter,
                   cudaStream_t st);

// ------------------------------------------------------------- dense products
size_t xf_simt_ws_floats(int64_t n, int N);
cudaError_t xf_simt(int fmt /*F32 or F64*/, const void* X, int64_t ldx, int64_t n, const float* F,
                    int ldf, int N, float* Y, int ldy, float* ws, size_t ws_floats, cudaStream_t st);

// tcgen05 path: operands are a packed K-major copy of F^T (Npad x ldp).
int tc_block_n(int N);  // 32, 64, 128, 256 or 512
size_t xf_tc_ws_floats(int64_t n, int BN);
cudaError_t pack_ft_bf16(const float* F, int64_t n, int ldf, int N, int Npad, void* out, int64_t ldp,
                         cudaStream_t st);
cudaError_t pack_ft_fp8(const float* F, int64_t n, int ldf, int N, int Npad, void* out, int64_t ldp,
                        float* col_scale, cudaStream_t st);
cudaError_t xf_tc(int fmt /*BF16 or FP8*/, const void* X, int64_t ldx, const float* row_scale,
                  int64_t n, const void* Fpack, int64_t ldp, const float* col_scale, int N, float* Y,
                  int ldy, float* ws, size_t ws_floats, unsigned* err, cudaStream_t st,
                  cudaEvent_t ev_begin = nullptr, cudaEvent_t ev_end = nullptr);

// Rectangular form: Y (m x N) = A (m x kdim, row-major, ld lda, BF16 or E4M3
// with row scales) times F, F^T packed as for xf_tc (N x ldp, ldp >= kdim).
// Rows of A past m and columns past kdim read as zero (TMA fill).
size_t tc_gemm_ws_floats(int64_t m, int64_t kdim, int BN);
cudaError_t tc_gemm(int fmt, const void* A, int64_t lda, int64_t m, int64_t kdim, const float* row_scale,
                    const void* Fpack, int64_t ldp, const float* col_scale, int N, float* Y, int ldy, float* ws,
                    size_t ws_floats, unsigned* err, cudaStream_t st, cudaEvent_t ev_begin = nullptr,
                    cudaEvent_t ev_end = nullptr);

// ------------------------------------------------------------------ sparse
cudaError_t csr_xf(const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                   const float* F, int ldf, int N, float* Y, int ldy, cudaStream_t st);
// Y[c, :] += wt[j] * x_{i_j c} * F[i_j, :] over the stored sample (Y must be zeroed first).
cudaError_t csr_sampled_xf(const int64_t* row_ptr, const int32_t* col, const float* val,
                           const int32_t* idx, const float* wt, const int* s_tot, const float* F,
                           int k, float* Y, cudaStream_t st);
// Dense version (fmt F64 / F32 / BF16): Y[r, :] += sum_j X[r, i_j] wt_j F[i_j, :]
// (X symmetric: reads rows i_j, coalesced).
cudaError_t dense_sampled_xf(int fmt, const void* X, int64_t ldx, int64_t n, const int32_t* idx,
                             const float* wt, const int* s_tot, int s_cap, const float* F, int k,
                             float* Y, cudaStream_t st);

// ------------------------------------------------------------- row kernels
// C (la x lb, FP64, and optionally FP32 Cf) = scale_row(A)^T B over n rows, with
// optional row gather idx/wt (count from *cnt when cnt != NULL), optional row
// scaling of the result by lam (C[i, :] *= lam[i]), and optional + shift*I.
// ws: xcross_ws_doubles() doubles (max_blocks_per_sm x SMs x la x lb block
// partials); counter: one zeroed unsigned.
size_t xcross_ws_doubles(int la, int lb);
cudaError_t xcross(const float* A, int lda, int la, const float* B, int ldb, int lb, int64_t n,
                   const int32_t* idx, const float* wt, const int* cnt, const double* lam,
                   double shift, double* C, float* Cf, double* ws, unsigned* counter,
                   cudaStream_t st, int max_blocks_per_sm = 4);

// HALS update of F_upd rows (Eq. symhals_update2) with Y either given (Y != NULL)
// or computed as U M (U n x l, M l x k FP32).  G FP32 k x k (no alpha),
// F_fix the fixed factor, k <= 64.  Accumulates FP64 partials: part[0] = sum
// F_new .* Y, part[1] = ||F_new - F_fix||^2 (reduced into part[0..1] by the
// last block; ws >= 2 * 2048 doubles, counter zeroed).
cudaError_t hals_update(float* F_upd, const float* F_fix, int64_t n, int k, const float* G, double alpha,
                        const float* Y, int ldy, const float* U, int l, const float* M, double* part, double* ws,
                        unsigned* counter, unsigned* err, cudaStream_t st);

// out[i, j] = sum_c A[i, c] B[c, j], A n x la (lda), B la x lb (FP32 small, row-major).
cudaError_t apply_small(const float* A, int lda, int la, const float* B, int lb, int64_t n,
                        float* out, int ldo, cudaStream_t st);

// lev[i] = || F[i, :] Rinv ||^2 (Rinv upper k x k FP32).
cudaError_t leverage_rows(const float* F, int64_t n, int k, const float* Rinv, double* lev,
                          cudaStream_t st);

// Objective after a half sweep: obj = normX2 + sum(Ga .* Gb) - 2 part[0] + alpha part[1].
// With cnt != NULL the value goes to out[*cnt] (if < cap) and *cnt is incremented,
// so a recorded graph can append one value per replay.
cudaError_t objective(const double* normX2, const double* Ga, const double* Gb, int k,
                      const double* part, const double* alpha, double* out, int* cnt, int cap,
                      cudaStream_t st);
// out[0] = sum a .* b, out[1] = sum (a - b)^2 (FP64); ws >= 2 * 2 * num_sms() doubles.
cudaError_t pair_reduce(const float* a, const float* b, int64_t count, double* out, double* ws,
                        unsigned* counter, cudaStream_t st);
// out[0] = sum w .* y, out[1] = sum (w - h)^2 (FP64; ws >= 2 * 2 * num_sms() doubles).
cudaError_t resid_reduce(const float* w, const float* h, const float* y, int64_t count, double* out, double* ws,
                         unsigned* counter, cudaStream_t st);
cudaError_t sumsq(const double* v, int l, double* out, cudaStream_t st);
// out = ||U diag(lam) U^T||_F^2 = sum_ij lam_i lam_j Gu_ij^2 with Gu = U^T U (l x l FP64).
cudaError_t lai_norm2(const double* Gu, const double* lam, int l, double* out, cudaStream_t st);

// Projected gradient partial: sum over entries of (grad)^2 where grad < 0 or F > 0,
// grad = 2 (F Gother - Y) + 2 alpha (F - Other).  Adds into acc[0] (FP64 atomics).
cudaError_t proj_grad_sq(const float* F, const float* Other, const float* Y, const float* Gother,
                         int64_t n, int k, const double* alpha, double* acc, cudaStream_t st);

// Generators.
cudaError_t philox_gaussian(float* out, int64_t n, int l, uint64_t seed, cudaStream_t st);
cudaError_t philox_uniform(float* out, int64_t n, int k, uint64_t seed, const double* scale_num,
                           double scale_mul, cudaStream_t st);
cudaError_t convert_bf16(const float* x, int64_t n, int64_t ldx, uint16_t* xb, int64_t ldb,
                         cudaStream_t st);
cudaError_t quantize_fp8(const float* x, int64_t n, int64_t ldx, uint8_t* x8, int64_t ld8,
                         float* row_scale, cudaStream_t st);
// Non-finite / negative check of a factor: sets err bits.
cudaError_t check_factor(const float* F, int64_t count, unsigned* flags, cudaStream_t st);
// Row normalisation: out[i, :] = in[i, :] / ||in[i, :]||.
cudaError_t normalize_rows(const float* in, int64_t n, int l, float* out, cudaStream_t st);

// --------------------------------------------------------- small dense
// Cholesky of G + shift I (k <= 96) in FP64: R upper (optional FP64 copy in
// R), Rinv (FP64 and FP32 copies, each optional).
// drop_tol > 0: pivots <= drop_tol * max_diag give zero rows/cols in Rinv
// (rank-safe mode); else such a pivot sets ERR_NOTSPD.
cudaError_t chol_inverse(const double* G, int k, double shift, double drop_tol, double* Rinv,
                         float* Rinv_f, unsigned* err, cudaStream_t st, double* R = nullptr);
// Symmetric Jacobi eigen-decomposition of A (l <= 128): V (columns = vectors), lam.
cudaError_t jacobi_evd(const double* A, int l, double* V, double* lam, cudaStream_t st);
// B = V diag(lam_j^{-1/2}) for lam_j > tol * max(lam) else 0 (FP32 out, l x l).
cudaError_t svqb_matrix(const double* V, const double* lam, int l, double tol, float* B,
                        cudaStream_t st);
// Small FP32 copies / scalings: Mf = diag(lam) C (la x lb), FP32.
cudaError_t to_float_scaled(const double* C, int la, int lb, const double* lam, float* out,
                            cudaStream_t st);

// ----------------------------------------------------------------- sampler
struct SampleBufs {
  double* lev;        // [n]
  unsigned long long* cdf;  // [n] inclusive prefix of q
  int32_t* idx;       // [cap]
  float* wt;          // [cap]
  int* counts;        // device: [0] s_D, [1] s_R, [2] s_tot
  double* sums;       // device: [0] theta, [1] mass_R
  unsigned long long* total;  // device: T
  // block scratch
  int* blk_cnt;
  unsigned long long* blk_q;
  double* blk_theta;
  double* blk_mass;
  int nblk_cap;
  int cap;
};
int sampler_blocks(int64_t n);
cudaError_t hybrid_sample(SampleBufs& b, int64_t n, int k, double tau, int s, uint64_t seed,
                          uint32_t iter, uint32_t side, cudaStream_t st);

// ------------------------------------------------------------- LAI engine
// All `nsweeps` LAI-HALS sweeps in one cooperative launch (see lai_engine.cu);
// `allow_resident` lets the CTAs keep their rows in shared memory when they fit.
// `resume`: W, H and the workspace are as the previous launch on this
// workspace left them, so its saved state replaces the prologue.
size_t lai_engine_ws_bytes(int l, int k, int obj_cap);
// ev_begin / ev_end (optional) are recorded right around the kernel launch.
// Gd_h, Gd_w, Gf_h, Gf_w (optional, all or none): the final H^T H and W^T W
// also written there, in FP64 and rounded to FP32.
cudaError_t lai_engine(const float* U, const double* lam, float* W, float* H, int64_t n, int k, int l,
                       int nsweeps, double alpha, const double* normX2, void* ws, double* obj, int obj_cap,
                       double* Gout, unsigned* err, bool allow_resident, cudaStream_t st,
                       cudaEvent_t ev_begin = nullptr, cudaEvent_t ev_end = nullptr, bool resume = false,
                       double* Gd_h = nullptr, double* Gd_w = nullptr, float* Gf_h = nullptr,
                       float* Gf_w = nullptr);
// Algorithmic FLOPs of one engine launch: per half sweep n (l k [Y = U M] +
// k^2 [column updates] + l k [U^T F] + k (k + 1) / 2 [F^T F]) FMAs, plus the
// prologue's n (l k + k (k + 1) / 2) (not run by a resumed launch); two FLOPs per FMA.
double lai_engine_flops(int64_t n, int k, int l, int nsweeps, bool prologue = true);

// -------------------------------------------------------------- CholeskyQR3
// Shifted CholeskyQR3 of S (n x l, l <= 96) in place; T is n x l scratch for
// the multi-kernel form (see cholqr.cu).  part: cholqr_part_doubles(l);
// fin, G: l * l doubles; Rf: l * (l + 3) floats; rinv: l + 3 floats.
// npass = 2 stops after the shifted pass and one plain pass: a basis of the
// same span that is well conditioned but orthonormal only to ~1e-4.
size_t cholqr_part_doubles(int l);
cudaError_t cholqr3(float* S, float* T, int64_t n, int l, double* part, double* fin, double* G, float* Rf,
                    float* rinv, double* ws, unsigned* counter, unsigned* bar, unsigned* err, bool allow_engine,
                    cudaStream_t st, int npass = 3);

// ------------------------------------------------------------------ PGNCG
// Device scalars of the conjugate-gradient loop (double cg[GN_COUNT]).
enum { GN_E = 0, GN_E0 = 1, GN_ALPHA = 2, GN_BETA = 3, GN_STOP = 4, GN_COUNT = 8 };
size_t gn_ws_doubles();
// R = 2 (H G - Y), P = R, Z = 0, cg[GN_E] = cg[GN_E0] = ||R||^2 (G = H^T H FP32, k <= 64).
cudaError_t gn_grad(const float* H, const float* Y, const float* G, int64_t n, int k, float* R, float* P, float* Z,
                    double* ws, unsigned* counter, double* cg, cudaStream_t st);
// Yc = 2 (P G + H PtH), cg[GN_ALPHA] = cg[GN_E] / <P, Yc> (0 once stopped).
cudaError_t gn_hvp(const float* H, const float* P, const float* G, const float* PtH, int64_t n, int k, float* Yc,
                   double* ws, unsigned* counter, double* cg, cudaStream_t st);
// Z += alpha P, R -= alpha Yc, cg[GN_BETA] = ||R||^2 / cg[GN_E], cg[GN_E] = ||R||^2.
cudaError_t gn_update(const float* P, const float* Yc, int64_t count, float* R, float* Z, double* ws,
                      unsigned* counter, double* cg, cudaStream_t st);
// P = R + beta P.
cudaError_t gn_dir(const float* R, int64_t count, float* P, const double* cg, cudaStream_t st);
// H = W = max(H - Z, 0).
cudaError_t gn_project(const float* Z, int64_t count, float* H, float* W, unsigned* err, cudaStream_t st);
// out[*cnt] = normX2 - 2 part[0] + sum Gd^2 (the SymNMF objective by the trace trick), *cnt += 1.
cudaError_t gn_objective(const double* normX2, const double* Gd, int k, const double* part, double* out, int* cnt,
                         int cap, cudaStream_t st);

// -------------------------------------------------------------------- BPP
cudaError_t bpp_rows(float* F_upd, const float* F_fix, int64_t n, int k, const double* G,
                     double alpha, const float* Y, int ldy, const float* U, int l, const float* M,
                     double* part, double* ws, unsigned* counter, unsigned* err, cudaStream_t st);

}  // namespace symnmf
