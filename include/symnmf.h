/*
 * symnmf.h - C ABI of the GB300 (sm_103a) randomized SymNMF library.
 *
 * Method: Hayashi, Aksoy, Ballard, Park, "Randomized Algorithms for Symmetric
 * Nonnegative Matrix Factorization" (arXiv 2402.08134).  The library solves the
 * regularised surrogate (Eq. surrogate_symnmf_obj)
 *
 *     min_{W, H >= 0} ||X - W H^T||_F^2 + alpha ||W - H||_F^2
 *
 * by alternating W- and H-updates (HALS, Eq. symhals_update2; or the exact
 * row NLS / BPP form of Eq. ANLS4symNMF), with the products X.H replaced
 *   - by U (Lambda (U^T H)) after a randomized range finder (Alg. RRF,
 *     Alg. Apx-EVD, Alg. LAI-SymNMF), or
 *   - by the leverage-score-sampled product X S^T S H (Alg. LvS-SymNMF,
 *     hybrid sampling of Section "Practical Considerations for LvS-SymNMF").
 *
 * Conventions for every call:
 *   - Matrices are row-major.  X is n x n and symmetric (not checked).
 *     W, H are n x k float32 with leading dimension k.
 *   - Pointers documented "device" must be CUDA device memory of the current
 *     device; "host" pointers are ordinary CPU memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls on a handle are ordered on the handle's stream; a call
 *     returns before its GPU work ends unless it returns host values, in
 *     which case it synchronises that stream.
 *   - Borrowed memory (X, CSR arrays, scales, caller buffers) stays owned by
 *     the caller and must outlive the handle / the call.  The handle owns its
 *     factors, sketch and workspaces (allocated at create, stream-ordered on the
 *     handle's stream from a library-owned memory pool; freed in stream order at
 *     destroy, so the handle's stream must outlive the handle).
 *   - Errors are returned as symnmf_status; no call throws or aborts.  A
 *     failing call leaves a message in symnmf_last_error(handle).  Kernel
 *     waits are bounded: a wait that runs out sets a device error word that
 *     the next synchronising call reports as SYMNMF_ETIMEOUT.
 */
#ifndef SYMNMF_GB300_H
#define SYMNMF_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct symnmf_ctx* symnmf_t;
typedef struct symnmf_batch_ctx* symnmf_batch_t;
typedef struct symnmf_mlp_ctx* symnmf_mlp_t;

typedef enum {
  SYMNMF_OK = 0,
  SYMNMF_EINVAL = 1,      /* bad argument (size, pointer, format, alignment) */
  SYMNMF_ENOMEM = 2,      /* a device allocation failed */
  SYMNMF_ENOTSPD = 3,     /* a Gram matrix that must be positive definite is not */
  SYMNMF_ETIMEOUT = 4,    /* a bounded device wait ran out */
  SYMNMF_ENAN = 5,        /* a non-finite value reached a factor or objective */
  SYMNMF_ECUDA = 6,       /* a CUDA runtime call failed (see last_error) */
  SYMNMF_ESTATE = 7,      /* call out of order (e.g. LAI sweep before lai_sketch) */
  SYMNMF_EUNSUPPORTED = 8 /* combination not built (e.g. BPP with k > 16) */
} symnmf_status;

/* Storage of X. */
typedef enum {
  SYMNMF_X_DENSE_F64 = 0,  /* double, n rows of ldx */
  SYMNMF_X_DENSE_F32 = 1,  /* float,  n rows of ldx */
  SYMNMF_X_DENSE_BF16 = 2, /* bfloat16, n rows of ldx, ldx % 8 == 0 (16-byte rows for TMA) */
  SYMNMF_X_DENSE_FP8 = 3,  /* e4m3 codes x8 with X_ij ~= row_scale[i] * x8_ij; ldx % 16 == 0 */
  SYMNMF_X_CSR_F32 = 4     /* CSR: row_ptr[n+1] int64, col[nnz] int32, x = float val[nnz] */
} symnmf_xfmt;

/* Which operator stands for X in a sweep or a residual. */
enum {
  SYMNMF_SRC_X = 0,   /* the problem's X in its own format */
  SYMNMF_SRC_LAI = 1, /* U Lambda U^T from symnmf_lai_sketch (Alg. LAI-SymNMF) */
  SYMNMF_SRC_XHI = 2, /* the optional float32 copy x_hi (correction / refinement sweeps) */
  SYMNMF_SRC_COMP = 3 /* Compressed-NMF (appendix "Comparison between LAI-NMF and
                         Compressed-NMF"): each half solves the compressed problem
                         min ||Q^T (F_fix F^T - X)||^2 + alpha ||F - F_fix||^2 on the
                         last sketch's basis Q, i.e. Update(G_c + alpha I, Y_c + alpha
                         F_fix) with M = Q^T F_fix, G_c = M^T M, Y_c = (X Q) M; sweeps
                         only (not a residual or PGNCG source) */
};

/* Update rule: Update(G, Y) of the paper's appendix. */
enum { SYMNMF_RULE_HALS = 0, SYMNMF_RULE_BPP = 1 };

/* Dense product kernel. */
enum {
  SYMNMF_GEMM_AUTO = 0, /* tensor cores for BF16/FP8 X, SIMT for F32/F64 X */
  SYMNMF_GEMM_SIMT = 1, /* CUDA-core kernel (F32/F64 X only) */
  SYMNMF_GEMM_TC = 2    /* tcgen05 + TMA kernel (BF16/FP8 X only) */
};

typedef struct {
  int64_t n;              /* order of X, >= 1 */
  int32_t k;              /* rank, 1..64 (HALS); 1..16 for the BPP rule */
  int32_t fmt;            /* symnmf_xfmt */
  const void* x;          /* device: dense X or CSR values */
  int64_t ldx;            /* dense leading dimension in elements; 0 means n */
  const float* row_scale; /* device [n], FP8 only */
  const int64_t* row_ptr; /* device [n+1], CSR only */
  const int32_t* col;     /* device [nnz], CSR only */
  int64_t nnz;            /* CSR only */
  const float* x_hi;      /* device, optional float32 dense X (row-major, ld = ldx_hi) */
  int64_t ldx_hi;         /* 0 means n */
  double alpha;           /* > 0: the regulariser; <= 0: alpha = max(X) (experiments section) */
  uint64_t seed;          /* Philox4x32-10 key for init, Omega and sample draws */
} symnmf_problem;

typedef struct {
  int32_t gemm;       /* SYMNMF_GEMM_* */
  int32_t use_graph;  /* 1: record sweep bodies (and the check loop of symnmf_sweep_to_target) as CUDA
                        graphs once and replay them; 0: launch every kernel from the host */
  int32_t max_width;  /* largest sketch width l to be requested (0: 2k + 10); values
                         above 96 are lowered to 96 */
  int32_t max_samples;/* largest sample count s for LvS calls (0: n) */
  int32_t lai_mode;   /* LAI steps: 0 = persistent cooperative launches (all
                         LAI-HALS sweeps in one, each CholeskyQR3 of the range
                         finder in one), rows kept in shared memory when they
                         fit (default); 1 = separate kernels per step; 2 = as
                         0 but the sweep launch streams its rows from global
                         memory every half sweep */
  int32_t reserved[3];
} symnmf_options;

/* ------------------------------------------------------------------ handle */

/* Create a solver for one problem.  Validates sizes and alignment (EINVAL),
 * allocates W, H and workspaces (ENOMEM), computes ||X||_F^2 and, when
 * prob->alpha <= 0, alpha = max_ij X_ij on `stream` (ENAN when X or x_hi
 * holds a non-finite entry).  W and H start at zero: call symnmf_set_factors
 * or symnmf_init_random before sweeping. */
symnmf_status symnmf_create(const symnmf_problem* prob, const symnmf_options* opt, void* stream,
                            symnmf_t* out);
void symnmf_destroy(symnmf_t h);
const char* symnmf_last_error(symnmf_t h);
/* alpha in use and ||X||_F^2 (host values; synchronises). */
symnmf_status symnmf_info(symnmf_t h, double* alpha, double* normX2);

/* Copy starting factors in (device n x k each).  W0 == NULL means W0 := H0
 * (the paper initialises H only).  Negative entries are rejected (EINVAL). */
symnmf_status symnmf_set_factors(symnmf_t h, const float* H0, const float* W0);
/* H0_ij = u_ij * scale with u from Philox4x32-10 (counter (j, i lo, i hi, 2),
 * key = seed); scale = 2 sqrt(mean(X) / k) when `scaled` (experiments
 * section), else 1.  W0 := H0. */
symnmf_status symnmf_init_random(symnmf_t h, int scaled);
/* Copy the current factors out (device n x k each; either may be NULL). */
symnmf_status symnmf_get_factors(symnmf_t h, float* H_out, float* W_out);

/* ------------------------------------------------------------ LAI (Alg. 1) */

/* Alg. RRF + Alg. Apx-EVD: Y = X Omega, Q = orth(Y), q times
 * { Q = orth(X Q); Q = orth(X Q) }, T = Q^T X Q, T = V Lambda V^T,
 * U = Q V.  orth() is a rank-safe shifted CholeskyQR3 (Fukaya et al. 2020):
 * the Gram Y^T Y from FP32 products folded into Kahan-compensated FP32 sums
 * and combined in double-float (about 44 significant bits), the Cholesky in
 * FP64, pivots below 1e-12 (shifted pass) / 1e-10 (plain passes) of the
 * largest dropped, and the rows solved in FP32; intermediate bases stop after
 * two passes, the final basis takes three.  T is formed like the Gram; its
 * eigen-decomposition is a cyclic Jacobi with FP32 rotations, stopped at FP32
 * rounding (||T - V Lambda V^T||_F <= 8 l 2^-24 ||T||_F), Lambda returned in
 * FP64.  `omega` (device n x l float32) or NULL for the Philox Gaussian
 * stream (counter (p, i lo, i hi, 1)).  l in [k, max_width], q >= 0.
 * X passes use the problem's X (BF16/FP8 on tensor cores when so stored).
 * ||U Lambda U^T||_F^2 (the LAI objective's ||X||^2 term) is formed from
 * U^T U, so that it matches the stored FP32 U exactly. */
symnmf_status symnmf_lai_sketch(symnmf_t h, int l, int q, const float* omega);
/* The same sketch with the basis from the adaptive range finder (appendix,
 * Alg. Ada-RRF): Q = orth(X Omega); then at most q_max times: B^T = X Q,
 * residual r = sqrt(||X||^2 - ||B||^2) / ||X|| (the appendix's QB identity,
 * ||B||^2 summed in FP64), Q = orth(B^T); stop when r fell by less than `tol`
 * since the previous check (the experiments use 1e-3); otherwise Q =
 * orth(X Q).  Then T = Q^T X Q and U, Lambda as in symnmf_lai_sketch.  Host
 * outputs (each may be NULL): checks_out = number of residual checks,
 * passes_out = products with X including the one for T, nr_hist[checks] =
 * the residuals (room for q_max values).  Synchronises once per check. */
symnmf_status symnmf_lai_sketch_ada(symnmf_t h, int l, int q_max, double tol, const float* omega,
                                    int* checks_out, int* passes_out, double* nr_hist);
/* Use a given low-rank approximation X ~ U Lambda U^T instead of a sketch
 * (U device n x l float32 with orthonormal columns, Lambda host double[l]),
 * e.g. a truncated EVD computed elsewhere.  Copies both; synchronises. */
symnmf_status symnmf_set_lai(symnmf_t h, const float* U, const double* lam_host, int l);
/* U (device n x l float32, may be NULL) and Lambda (host double[l], may be NULL). */
symnmf_status symnmf_get_lai(symnmf_t h, float* U_out, double* lam_out, int* l_out);

/* -------------------------------------------------------------- sweeps */

/* `nsweeps` sweeps (W-update then H-update) with X given by `source`
 * (SYMNMF_SRC_*) and `rule`.  obj_host (host, may be NULL) receives after
 * each sweep the surrogate objective ||X - W H^T||^2 + alpha ||W - H||^2 of
 * that operator, by the trace trick of the "Fast Residual Evaluation"
 * appendix with FP64 accumulation; for SRC_LAI, ||X||^2 is
 * ||U Lambda U^T||_F^2 (sum lambda^2 up to the FP32 orthonormality of U);
 * for SRC_COMP the value is the H half's compressed objective
 * ||Q^T (W H^T - X)||^2 + alpha ||W - H||^2.
 * Synchronises only when obj_host != NULL (once, at the end); a non-finite
 * recorded objective returns SYMNMF_ENAN. */
symnmf_status symnmf_hals_sweep(symnmf_t h, int nsweeps, int source, int rule, double* obj_host);

/* `iters` iterations of PGNCG-SymNMF on the SymNMF objective ||X - H H^T||_F^2
 * (section "Projected Gauss-Newton with Conjugate Gradients for SymNMF";
 * with source = SYMNMF_SRC_LAI the appendix's LAI-PGNCG-SymNMF, X H replaced
 * by U (Lambda (U^T H))).  Per iteration: R = 2 (H H^T H - X H); s_max steps
 * of conjugate gradients on the Gauss-Newton normal equations
 * 2 (Z H^T H + H Z^T H) = R from Z = 0 (stopped early once ||R|| falls
 * below 1e-6 of its start); H = max(H - Z, 0).  Row work in FP32, CG
 * scalars and reductions in FP64, all on the device.  W follows H (W := H).
 * obj_host (host, may be NULL): ||X - H H^T||_F^2 after each iteration, by the
 * trace trick with FP64 accumulation (one extra product with X in all);
 * synchronises only then.  iters <= 4096, 1 <= s_max <= 1000. */
symnmf_status symnmf_pgncg(symnmf_t h, int iters, int source, int s_max, double* obj_host);

/* The experiments' schedule (section "Experimental Results", WoS setup), run
 * end to end on the device:
 *   1. with method SYMNMF_SRC_LAI or SYMNMF_SRC_COMP, the sketch by the
 *      adaptive range finder (symnmf_lai_sketch_ada with l, q_max, ada_tol);
 *   2. iterations on `method`'s operator (HALS / BPP sweeps by `rule`, or
 *      PGNCG iterations when algo = 1) until the normalized residual
 *      sqrt(objective / ||operator||^2), read after every iteration, has
 *      fallen by less than stop_tol in each of stop_count consecutive
 *      iterations (the experiments use 1e-4 and 4), or max_iters;
 *   3. with refine != 0 and a sketched method, Iterative Refinement: the
 *      same iterations and stopping rule on X itself (its float32 copy when
 *      the problem has one), at most max_refine.
 * The start is the handle's current factors.  The report gives the
 * sketch's checks and passes, the iterations of each phase, and the true
 * normalized residual ||X - W H^T|| / ||X|| at the end (||X - H H^T|| / ||X||
 * for PGNCG) against X (or its float32 copy).  Synchronises every iteration. */
typedef struct {
  int32_t method;      /* SYMNMF_SRC_X, SYMNMF_SRC_LAI or SYMNMF_SRC_COMP */
  int32_t algo;        /* 0: alternating updates by `rule`; 1: PGNCG (X or LAI only) */
  int32_t rule;        /* SYMNMF_RULE_HALS or SYMNMF_RULE_BPP */
  int32_t l;           /* sketch width */
  int32_t q_max;       /* at most this many power iterations (Ada-RRF) */
  int32_t stop_count;  /* consecutive small decreases that stop a phase (>= 1) */
  int32_t max_iters;   /* cap of the first phase */
  int32_t refine;      /* 1: Iterative Refinement after a sketched phase */
  int32_t max_refine;  /* cap of the refinement phase */
  int32_t s_max;       /* CG steps per PGNCG iteration */
  double ada_tol;      /* Ada-RRF: stop when the QB residual falls by less */
  double stop_tol;     /* per-iteration decrease of the normalized residual */
} symnmf_schedule;

typedef struct {
  int32_t checks, passes;    /* the adaptive range finder's residual checks and X passes */
  int32_t iters, refine_iters;
  double nr_phase;           /* normalized residual of the operator when phase 2 stopped */
  double nr_final;           /* true-X normalized residual at the end */
} symnmf_report;

symnmf_status symnmf_solve(symnmf_t h, const symnmf_schedule* sched, symnmf_report* report);

/* ------------------------------------------------------------ LvS (Alg. 2) */

/* Leverage scores of the fixed factor (side 0: H, used to update W; side 1:
 * W) by CholeskyQR: F^T F from compensated FP32 sums combined in
 * double-float, R = chol(F^T F) and R^{-1} in FP64, then l_i = ||f_i R^{-1}||^2
 * with R^{-1} rounded to FP32 (FP32 row pass; device double[n] out).
 * ENOTSPD when F^T F is singular (a pivot <= 0). */
symnmf_status symnmf_leverage(symnmf_t h, int side, double* lev_out);

/* Hybrid sample of the fixed factor for iteration `iter`:
 * I_D = {i : l_i / k >= tau} (ascending), s_D = |I_D|, s_R = max(s - s_D, 0)
 * draws with replacement over I_R with probability q_i / T,
 * q_i = floor(l_i 2^40), drawn by Philox counter (j, iter, side, 3):
 * u = x0 2^32 + x1, row = first i with C_i > floor(u T / 2^64), C the
 * inclusive prefix sum of q.  Weights (on S^T S): 1 for I_D, 1 / (s_R p~_i)
 * for draws, p~_i = l_i / sum_{I_R} l.  lev_in (host double[n]) replaces the
 * device scores when not NULL.  Outputs (host, may be NULL): idx/wt (cap
 * entries: I_D first, then draws in draw order), s_det, s_tot = s_D + s_R,
 * theta = sum_{I_D} l_i.  The sample stays in the handle for lvs_update.
 * Synchronises. */
symnmf_status symnmf_lvs_sample(symnmf_t h, int side, int iter, double tau, int s, const double* lev_in,
                                int32_t* idx_out, float* wt_out, int cap, int* s_det, int* s_tot,
                                double* theta);
/* Update W (side 0) or H (side 1) from the stored sample: Y = X S^T S F,
 * G = F^T S^T S F, then Update(G + alpha I, Y + alpha F) by `rule`.  X must
 * be CSR or dense F64/F32/BF16: the sampled columns of X are read as the
 * sampled rows (X is symmetric), contiguous in memory. */
symnmf_status symnmf_lvs_update(symnmf_t h, int side, int rule);
/* `iters` full LvS iterations entirely on the device (leverage, sample,
 * sampled products, update; both halves), counters iter0 .. iter0+iters-1.
 * No host synchronisation. */
symnmf_status symnmf_lvs_iterate(symnmf_t h, int iter0, int iters, double tau, int s, int rule);

/* ----------------------------------------------------------- residuals */

/* With X given by `source`: norm_resid = ||X - W H^T||_F / ||X||_F (trace
 * trick, FP64 accumulation), surrogate = ||X - W H^T||^2 + alpha ||W - H||^2,
 * proj_grad = sqrt(||grad^P_W||^2 + ||grad^P_H||^2) of the surrogate
 * ("Projected Gradients" appendix, with the 2 alpha (W - H) terms).  Each
 * output may be NULL; proj_grad costs two products with X.  Synchronises. */
symnmf_status symnmf_residual(symnmf_t h, int source, double* norm_resid, double* surrogate_obj,
                              double* proj_grad);

/* Sweeps of `source` (rule HALS) in chunks of `chunk`, each chunk followed by
 * the normalized residual ||X - W H^T||_F / ||X||_F of the operator `check`
 * (as symnmf_residual computes it); stops after the first check at or below
 * `target`, or after max_sweeps sweeps.  The residual-check schedule of the
 * experiments (a check every few iterations, stop once the residual is
 * reached), with the decision taken on the device: for SRC_LAI sweeps of the
 * persistent engine with max_sweeps a multiple of chunk and use_graph set, once a call repeats
 * the previous call's check, chunk, max_sweeps / chunk, target and sketch
 * width, the first chunk and check run eagerly and the rest in one CUDA graph
 * (recorded on that call, replayed by later ones) whose WHILE node repeats
 * chunk, check and decision until the decision stops it, so no host round
 * trip separates the checks.  Otherwise the host checks after each chunk.
 * Both give the same results to the last bit.  Outputs (host, each may be
 * NULL): the sweeps run, the checks made (at most LOOP_MAX = 1024, else
 * SYMNMF_EINVAL) and the last check's residual.  Synchronises once at the end
 * (device loop) or once per chunk. */
symnmf_status symnmf_sweep_to_target(symnmf_t h, int source, int check, int chunk, int max_sweeps, double target,
                                     int* sweeps_out, int* checks_out, double* nr_out);

/* -------------------------------------------------- standalone kernels */

/* Y = X F for a dense X (fmt F64/F32/BF16/FP8, ld ldx, FP8 with row_scale),
 * F device float [n x N] (ld ldf), Y device float [n x N] (ld ldy); N <= 512
 * for BF16 / FP8 X (tcgen05: 128-row tiles up to 128 columns, 256-row tiles
 * at 256, two N = 256 MMAs per k step at 512), N <= 128 for F32 / F64 X.
 * Up to 128 columns the tensor-core accumulation is flushed to FP32 every 8
 * k blocks; wider products accumulate a whole K segment in TMEM, which the
 * tensor core rounds low by about 2e-8 relative per MMA (~6e-5 at n = 20000).
 * gemm = SYMNMF_GEMM_*.  Synchronises the stream (BF16 / FP8). */
symnmf_status symnmf_dense_xf(int fmt, const void* x, int64_t ldx, const float* row_scale, int64_t n,
                              const float* F, int ldf, int N, float* Y, int ldy, int gemm, void* stream);
/* Y = X F for CSR X (row_ptr int64[n+1], col int32[nnz], val float[nnz]); F, Y device
 * float [n x N] with leading dimension N; N <= 128. */
symnmf_status symnmf_csr_xf(const int64_t* row_ptr, const int32_t* col, const float* val, int64_t n,
                            const float* F, int N, float* Y, void* stream);
/* G = F^T F (device double[N x N] out; F device float [n x N], N <= 128):
 * FP32 products summed over at most 32 rows, folded into Kahan-compensated
 * FP32 totals, and the block totals combined in double-float in a fixed
 * order (deterministic; about 44 significant bits). */
symnmf_status symnmf_gram(const float* F, int64_t n, int N, double* G, void* stream);
/* The same Gram matrix as symnmf_gram, computed without allocating any memory.
 * The paper has no counterpart: this entry point exists for callers that must
 * not call cudaMalloc or an allocating library, e.g. code that runs where the
 * device memory is owned by someone else (a host application's fixed pool or
 * a real-time loop that forbids allocation).  The kernel's scratch for block
 * partials lives in a static device array of 16 MiB (plus one counter) that
 * every GPU that loads this library holds until the process exits.  Limits:
 * N <= 64 (SYMNMF_EINVAL beyond) and at most 256 SMs (SYMNMF_EUNSUPPORTED).
 * Every call looks up the array's address on the current device
 * (cudaGetSymbolAddress, which allocates nothing); the first call on a device
 * also loads the library's device symbols there, so make that first call
 * before any stream capture.  All calls share the array and each leaves its
 * partials there: calls that overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller.  The result is
 * bit-identical to symnmf_gram's.  Stream-ordered, no synchronisation. */
symnmf_status symnmf_gram_noalloc(const float* F, int64_t n, int N, double* G, void* stream);
/* FP64 Cholesky G + shift I = R^T R (R upper) and R^{-1}, as used for the
 * leverage scores (Alg. LvS-SymNMF, thin QR of the fixed factor by
 * CholeskyQR) and, with its pivot-dropping rule, for each CholeskyQR pass of
 * the range finder.  G device double [k x k] (symmetrised as (G + G^T) / 2),
 * 1 <= k <= 96, shift >= 0; R and Rinv device double [k x k] row-major, upper
 * triangular (either may be NULL).  SYMNMF_ENOTSPD when a pivot is not
 * positive (G + shift I not positive definite); R and Rinv then hold zero rows
 * for the failed pivots.  Synchronises the stream. */
symnmf_status symnmf_cholesky(const double* G, int k, double shift, double* R, double* Rinv, void* stream);
/* Philox Gaussian Omega (device float [n x l]) as in symnmf_lai_sketch. */
symnmf_status symnmf_gaussian(float* out, int64_t n, int l, uint64_t seed, void* stream);
/* FP8 copy of a dense float X: row_scale_i = max_j |X_ij| / 448, x8 = e4m3(X / row_scale). */
symnmf_status symnmf_quantize_fp8(const float* x, int64_t n, int64_t ldx, uint8_t* x8, int64_t ld8,
                                  float* row_scale, void* stream);
/* BF16 copy of a dense float X (round to nearest even). */
symnmf_status symnmf_convert_bf16(const float* x, int64_t n, int64_t ldx, uint16_t* xb, int64_t ldb,
                                  void* stream);

/* Live timing of the dense tensor-core product kernel.  While enabled, every
 * eager (not graph-recorded) product launch on the handle is bracketed by
 * CUDA events on the handle's stream.  profile_read synchronises and returns
 * the summed kernel time (ms), the number of launches and their algorithmic
 * bytes (X once, F and Y once each), then resets the record. */
symnmf_status symnmf_profile(symnmf_t h, int enable);
symnmf_status symnmf_profile_read(symnmf_t h, double* total_ms, int64_t* launches, double* bytes);
/* Process-wide timing of the standalone tensor-core products (symnmf_dense_xf
 * with X in BF16 or FP8): while enabled, the product kernel of every call is
 * bracketed by CUDA events; the read returns the summed kernel time (ms), the
 * number of launches, their FLOPs (2 n^2 N each) and algorithmic bytes (X
 * once, F and Y once), then resets the record.  Thread-safe. */
symnmf_status symnmf_profile_standalone(int enable);
symnmf_status symnmf_profile_standalone_read(double* total_ms, int64_t* launches, double* flops, double* bytes);
/* The same for the persistent LAI-HALS sweep launches (Alg. LAI-SymNMF loop):
 * summed kernel time (ms), number of launches and their algorithmic FLOPs --
 * per half sweep n (l k + k^2 + l k + k (k + 1) / 2) FMAs (Y = U M, the column
 * updates, U^T F, upper F^T F), plus a prologue of n (l k + k (k + 1) / 2),
 * two FLOPs each.  Resets the record. */
symnmf_status symnmf_profile_read_engine(symnmf_t h, double* total_ms, int64_t* launches, double* flops);

/* The LvS iterations' time split (the buckets of the paper's per-iteration
 * breakdown, section "Microsoft Open Academic Graph"): while symnmf_profile is
 * enabled, every half of symnmf_lvs_iterate is bracketed by CUDA events on the
 * handle's stream.  Read (synchronises; resets the record): sampling_ms =
 * leverage scores (Gram, FP64 Cholesky and inverse, row pass) and the hybrid
 * sampler; products_ms = the sampled products Y = X S^T S F and
 * G = F^T S^T S F ("MM"); update_ms = the Update() rule ("Solve"); halves =
 * the halves recorded. */
symnmf_status symnmf_profile_read_lvs(symnmf_t h, double* sampling_ms, double* products_ms, double* update_ms,
                                      int64_t* halves);

/* Number of kernels this library has launched in this process (graph replays
 * count each kernel node). */
uint64_t symnmf_launch_count(void);

/* Test of the bounded-wait error path: one kernel waits, through the same
 * bounded wait as the persistent kernels' grid barriers, for a handle word
 * that nothing sets, gives up after limit_ns (1e3 .. 1e9 ns) and records a
 * timeout in the handle's device error word; the call then synchronises and
 * returns SYMNMF_ETIMEOUT.  The handle stays usable (the word is cleared). */
symnmf_status symnmf_debug_wait_timeout(symnmf_t h, int64_t limit_ns);

/* ------------------------------------------------------------- batched */

/* One grouped solver over `nprob` independent problems (dense BF16 or F32 X),
 * each with `restarts` random restarts stacked as extra columns of its
 * factors (width restarts * k_p <= 128).  A sweep runs all problems in one
 * persistent grouped product launch plus one grouped update launch per half;
 * with use_graph the whole sweep sequence is recorded once and replayed.
 * Tile shapes come from the library's own timing-based autotuner. */
symnmf_status symnmf_batched_create(const symnmf_problem* probs, int nprob, int restarts,
                                    const symnmf_options* opt, void* stream, symnmf_batch_t* out);
void symnmf_batched_destroy(symnmf_batch_t b);
const char* symnmf_batched_last_error(symnmf_batch_t b);
/* Philox start for every problem and restart (restart r uses key seed_p + r). */
symnmf_status symnmf_batched_init_random(symnmf_batch_t b, int scaled);
/* Device factors of problem p: H0 (n_p x restarts*k_p), W0 nullable -> H0. */
symnmf_status symnmf_batched_set_factors(symnmf_batch_t b, int p, const float* H0, const float* W0);
symnmf_status symnmf_batched_get_factors(symnmf_batch_t b, int p, float* H_out, float* W_out);
/* `nsweeps` sweeps of every problem.  obj_host (may be NULL): double
 * [nsweeps][nprob * restarts] surrogate objectives, problem-major. */
symnmf_status symnmf_batched_sweep(symnmf_batch_t b, int nsweeps, double* obj_host);
/* Configuration the autotuner chose for the grouped product at the first
 * sweep (pipeline stages, CTAs per SM) and its measured time in ms (0 before
 * the first sweep). */
symnmf_status symnmf_batched_info(symnmf_batch_t b, int* stages, int* ctas_per_sm, double* product_ms);

/* ------------------------------------------------- learned warm start */

/* Network x -> softplus(relu(relu(x W1 + b1) W2 + b2) W3 + b3), dims
 * (in, h1, h2, out); float32 master weights, He-uniform init from Philox. */
symnmf_status symnmf_mlp_create(int in, int h1, int h2, int out, uint64_t seed, void* stream,
                                symnmf_mlp_t* out_net);
void symnmf_mlp_destroy(symnmf_mlp_t m);
/* Parameters as one float array: W1 (in x h1), b1, W2 (h1 x h2), b2, W3 (h2 x out), b3. */
symnmf_status symnmf_mlp_get_params(symnmf_mlp_t m, float* host_out, int64_t count);
symnmf_status symnmf_mlp_set_params(symnmf_mlp_t m, const float* host_in, int64_t count);
int64_t symnmf_mlp_param_count(symnmf_mlp_t m);
/* out (device rows x out_dim) = network(x) for x device rows x in. */
symnmf_status symnmf_mlp_forward(symnmf_mlp_t m, const float* x, int64_t rows, float* out);
/* Loss and parameter gradients for one instance: Hhat = network(x),
 * L = ||Hhat Hhat^T - Hs Hs^T||^2 / ||Hs Hs^T||^2 evaluated with k x k Grams.
 * grads (device float[param_count]) may be NULL; loss_host may be NULL. */
symnmf_status symnmf_mlp_loss_grad(symnmf_mlp_t m, const float* x, const float* Hstar, int64_t rows,
                                   float* grads, double* loss_host);
/* One Adam step (t counts from 1) with the gradients of the last loss_grad. */
symnmf_status symnmf_mlp_adam(symnmf_mlp_t m, float lr, int t);
/* H0 for a problem handle from sketch features: rows of X Omega, normalised,
 * through the network; W0 := H0.  Requires lai_sketch or an explicit
 * features array (device n x in, may be NULL to use X Omega of the handle). */
symnmf_status symnmf_warm_start(symnmf_t h, symnmf_mlp_t m, const float* features);
/* Row-normalised X Omega of the last lai_sketch (device n x l out). */
symnmf_status symnmf_sketch_features(symnmf_t h, float* out);

#ifdef __cplusplus
}
#endif
#endif /* SYMNMF_GB300_H */
