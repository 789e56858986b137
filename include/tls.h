/*
 * tls.h -- C ABI of the GB300 (sm_103a) RQI-PCGTLS library.
 *
 * Method: Rayleigh quotient iteration for the smallest singular value sigma_{n+1} of [A, b]
 * and the total-least-squares solution x_TLS = -v(1:n, n+1) / v(n+1, n+1) (Oktay & Carson,
 * arXiv 2305.19028, Sec. 1), with every RQI step solving the two shifted systems
 * (A^T A - sigma_k^2 I) w = f by preconditioned conjugate gradients, PCGTLS (Alg. 3), in the
 * three-precision form of Alg. 4:
 *   u_f  the precision of the preconditioner R (the paper's u_q): FP16 / BF16 / FP32 / FP64;
 *   u    the PCGTLS working precision (the paper's u_p): FP32 or FP64;
 *   u_r  the precision of the residuals, the Rayleigh quotient and the stop test (the paper's
 *        u): always FP64.
 * R is the Cholesky factor of the column-scaled Gram matrix H = D^{-1} A^T A D^{-1},
 * D = diag(||a_j||) (Sec. 3.1, two-sided diagonal scaling), so R = R_H D.
 *
 * Conventions for every entry point:
 *  - Nothing throws across the ABI. Each call returns a tls_status; a per-context message
 *    with details is available from tls_last_error().
 *  - All work runs on the context's CUDA stream (the stream passed at creation, or a
 *    stream the context creates when NULL is passed). tls_solve synchronises that stream only
 *    to return x and sigma.
 *  - Matrices are row-major. Sizes are int64_t. Pointers are either host pointers or device
 *    pointers as stated per argument.
 *  - A context is not thread-safe; distinct contexts may be used from distinct threads.
 */
#ifndef TLS_H_
#define TLS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TLS_OK = 0,
  TLS_ERR_ARG = 1,               /* invalid argument (sizes, NULL, NaN/Inf in the data) */
  TLS_ERR_CUDA = 2,              /* a CUDA runtime call failed */
  TLS_ERR_OOM = 3,               /* device allocation failed */
  TLS_ERR_STATE = 4,             /* call out of order (e.g. tls_solve before tls_factor) */
  TLS_ERR_FACTOR_BREAKDOWN = 5,  /* Cholesky met a non-positive pivot on every rung */
  TLS_ERR_NOT_SPD = 6,           /* PCGTLS met delta_j <= 0: A^T A - sigma^2 I not SPD (Sec. 3) */
  TLS_ERR_NOT_UNIQUE = 7,        /* sigma_{n+1} >= sigma'_n estimate: x_TLS not unique (Sec. 3) */
  TLS_ERR_NO_CONVERGENCE = 8,    /* max_rqi reached with psi above the acceptance level */
  TLS_ERR_TIMEOUT = 9            /* a bounded device wait gave up */
} tls_status;

typedef enum {
  TLS_FP16 = 0,
  TLS_BF16 = 1,
  TLS_FP32 = 2,
  TLS_FP64 = 3,
  TLS_AUTO = 4   /* the selector network picks u_f (tls_set_selector / tls_batch_set_selector) */
} tls_prec;

/* Stop reasons reported in tls_info.stop_reason. */
enum {
  TLS_STOP_TOL = 1,       /* psi_k <= tol * (||A||_F^2 + ||b||^2), tested from k = 2 on       */
  TLS_STOP_PSI_UP = 2,    /* psi_k > psi_{k-1} (or >= with psi_rule_ge), Sec. 3 after Eq. (4) */
  TLS_STOP_MAX_RQI = 3,   /* k reached max_rqi                                              */
  TLS_STOP_STALL = 4      /* a PCGTLS solve stalled or met delta_j <= 0 before psi reached  */
                          /* the attainable level: the solve ended early for the precision  */
                          /* fallback (tls_options.stall_fallback)                          */
};

/* Why the precision fallback of tls_solve refactored (tls_info.fallback_trigger). */
enum {
  TLS_TRIGGER_NONE = 0,
  TLS_TRIGGER_MAX_RQI = 1,     /* the RQI loop ended on max_rqi                              */
  TLS_TRIGGER_STALL = 2,       /* a PCGTLS solve reduced ||s|| by less than stall_ratio      */
  TLS_TRIGGER_NOT_SPD = 3,     /* delta_j <= 0: the preconditioned operator lost positive    */
                               /* definiteness (the requirement behind Eq. (9), Sec. 3.1)    */
  TLS_TRIGGER_CONSTRAINT = 4   /* tls_factor: u_f above constr_guard x constraint 2 of the   */
                               /* column-scaled matrix (Eq. (9) with sigma_{n+1} = 0)         */
};

typedef struct {
  tls_prec u;          /* PCGTLS precision u_p: TLS_FP32 (mixed) or TLS_FP64 (plain)          */
  int mode_A;          /* 1: operator with A, delta = ||A q||^2 - sigma^2 ||q||^2 (default);    */
                       /* 0: Alg. 3 as printed, delta = ||p||^2 - sigma^2 ||q||^2 (no pass over */
                       /* A: the operator is I - sigma^2 R^{-T} R^{-1}); 2: hybrid, the printed */
                       /* form while psi falls by at least hybrid_ratio per RQI step, then the  */
                       /* operator with A (dense contexts)                                      */
  int cg_fixed;        /* 1: k+1 PCGTLS steps in RQI step k (Alg. 4, default);                 */
                       /* 0: up to cg_max steps, stopping when ||s_j|| <= cg_tol ||s_0||        */
  double cg_tol;
  int cg_max;
  int psi_rule_ge;     /* 1: stop on psi_k >= psi_{k-1} (the rule of Sec. 4.2)                 */
  int ls_iters;        /* PCG steps (sigma^2 = 0) that produce the LS start x_0 (default 6)    */
  int max_shifts;      /* Cholesky retries with H + s I, s = 2^-10 * 4^i before escalating u_f */
  int gram_simt;       /* 1: form H with the CUDA-core kernel even for FP16/BF16 (default 0:   */
                       /* tensor cores, tcgen05)                                             */
  double psi_accept;   /* an increase psi_k > psi_{k-1} stops only once psi_{k-1} <=           */
                       /* psi_accept * (||A||_F^2 + ||b||^2); above it the increase is taken   */
                       /* as a transient of the inexact inner solves (default 1e-15, near the */
                       /* FP64 rounding level of psi; a very large value gives the paper's    */
                       /* rule exactly)                                                        */
  int shift_first;     /* 1 (default): FP16/BF16 factors start from H + 2 u_f I, the diagonal  */
                       /* perturbation of low-precision Cholesky; 0: start unshifted and shift */
                       /* only after a breakdown                                              */
  int fallback;        /* 1 (default): when the RQI loop ends on max_rqi (not converged), refactor */
                       /* one precision up (FP16/BF16 -> FP32 -> FP64) and solve again, at most  */
                       /* twice -- the precision fallback for a factor that violates the         */
                       /* stability constraints of Sec. 3.1; 0: return the max_rqi result       */
  double constr_guard; /* > 0: tls_factor checks constraint 2 (Eq. (9), Sec. 3.1) on the column-  */
                       /* scaled matrix the factor is built from, kappa_F(A D^{-1})^{-1} =      */
                       /* 1 / (sqrt(n) ||R_H^{-1}||_F) (sigma_{n+1} taken as 0), and escalates  */
                       /* an FP16/BF16 factor to the next precision when u_f > constr_guard x    */
                       /* that bound (1: the paper's heuristic as printed); 0 (default): off     */
  int stall_fallback;  /* 1 (default, with fallback): end the RQI loop early (TLS_STOP_STALL) and */
                       /* fall back one precision when, at RQI step k >= 2 and psi still above   */
                       /* the acceptance level, a PCGTLS solve reduced ||s_j|| / ||s_0|| by less  */
                       /* than stall_ratio, met delta_j <= 0, or (tolerance mode) used cg_max    */
                       /* steps without reaching cg_tol                                           */
  double stall_ratio;  /* default 0.9                                                          */
  int constraint_iters;/* > 0: tls_solve also estimates constraints 1 and 2 (Eq. (5), Eq. (9))   */
                       /* as tls_condition does, with this many power iterations, into        */
                       /* tls_info.constr1 / constr2; 0 (default): those fields are NaN         */
  double hybrid_ratio; /* mode_A = 2: switch to the operator with A at the first RQI step whose  */
                       /* psi exceeds hybrid_ratio x the previous psi, or whose solves met       */
                       /* delta_j <= 0 (default 0.1)                                            */
  int reproducible;    /* 1 (default): bitwise reproducible results (every reduction in a fixed  */
                       /* order); 0: the one-launch PCGTLS solve sums A^T t with float atomics  */
                       /* (one grid barrier less per step; results may differ in the last bits  */
                       /* from run to run)                                                       */
  int factor;          /* how R-hat is formed (dense contexts): 0 (default) the Cholesky factor */
                       /* of the column-scaled Gram matrix (Sec. 3, on tensor cores); 1 the     */
                       /* Householder QR of the column-scaled A in u_q = u_f (Alg. 4's         */
                       /* "A = Q[R 0]^T", the paper's default; its constraint is kappa^-1 rather */
                       /* than kappa^-2). With 1 no Gram matrix is formed, so tls_condition is   */
                       /* unavailable (TLS_ERR_STATE) and tls_info.constr1/constr2 stay NaN;     */
                       /* m is limited by the panel kernel (rows of a 32-column FP32 panel, or a */
                       /* 16-column FP64 one, in the shared memory of one 16-CTA cluster)        */
} tls_options;

typedef struct {
  int stop_reason;       /* TLS_STOP_* */
  int rqi_steps;         /* residual evaluations in the RQI loop (k of the last one)         */
  int best_k;            /* k of the returned iterate (the one with the smallest psi)        */
  int cg_iters;          /* PCGTLS steps summed over both solves of every RQI step           */
  int shifts;            /* diagonal shifts applied to H before the factorisation succeeded  */
  int not_spd;           /* 1 if some PCGTLS solve stopped on delta_j <= 0                   */
  tls_prec u_f_used;     /* precision of the factor that was used                            */
  double psi_final;      /* psi of the returned iterate                                      */
  double sigma2;         /* sigma^2 of the returned iterate                                  */
  double shift;          /* the shift s of H + s I that was used (0 if none)                 */
  double t_factor_ms;    /* device time of the last tls_factor (CUDA events)                 */
  double t_solve_ms;     /* device time of this tls_solve                                    */
  int fail_pivot;        /* pivot index of the last Cholesky breakdown before success (-1)   */
  int pass_variant[2];   /* autotuned kernel of the pass over A: [FP64 residual, PCGTLS];    */
                         /* 0 register kernel, 1 staged 256 threads, 2 staged 512 threads,   */
                         /* 3 pipelined, 4 (residual) double-FP32 arithmetic on A32 + Alo;   */
                         /* small FP64 problems solved in one launch: {-1, 1}                */
                         /* for the one-CTA solve, {-2, R} for the solve on a cluster of R   */
  int n_psi;             /* entries of psi_hist filled                                       */
  double psi_hist[24];   /* psi_k of the RQI loop, k = 1, 2, ... (first 24)                  */
  int fallbacks;         /* precision fallbacks taken (tls_options.fallback); the other       */
                         /* fields describe the final factor and solve                        */
  int fallback_trigger;  /* TLS_TRIGGER_* of the last fallback or factor escalation           */
  int escalations;       /* factor precisions skipped by the constraint guard                 */
  double constr1;        /* constraint 1, kappa(A)^{-1} (Eq. (5)); NaN unless constraint_iters */
  double constr2;        /* constraint 2, kappa_F(A)^{-1} (1 - sigma_{n+1}^2 / sigma'_n^2)     */
                         /* (Eq. (9)) with this solve's sigma; NaN unless constraint_iters     */
  double constr2_scaled; /* constraint 2 of the column-scaled matrix with sigma_{n+1} = 0 (the */
                         /* guard's bound); NaN unless the guard or constraint_iters ran       */
  int mode_switch_k;     /* mode_A = 2: the RQI step k from which the operator with A was used */
                         /* (0: never switched); -1 for the other modes                         */
} tls_info;

typedef struct tls_ctx tls_ctx;

/* Default options: u = FP32, mode A, k+1 PCGTLS steps, strict psi rule, 12 LS steps,
 * 3 shifts, tensor-core Gram. */
void tls_default_options(tls_options* opt);

/* NULL when every field of *opt is in its range, else a static string saying which is not
 * (switches 0 or 1; cg_max in [1, 100000], ls_iters and constraint_iters in [0, 100000],
 * max_shifts in [0, 30]; cg_tol, constr_guard, stall_ratio, hybrid_ratio finite and >= 0;
 * psi_accept >= 0). tls_factor and tls_batch_factor apply the same check (TLS_ERR_ARG) plus the
 * rules that depend on the context. Host only: needs no GPU. */
const char* tls_options_check(const tls_options* opt);

/*
 * tls_create_dense -- a TLS problem [A, b] with dense A (Sec. 1: min ||[E, r]||_F subject to
 * (A + E) x = b + r).
 *   m, n      rows and columns of A, m >= n >= 1.
 *   A         m x n, row-major with leading dimension lda >= n (elements); FP64.
 *   b         m FP64 values.
 *   on_device 0: A and b are host pointers; 1: they are device pointers of the current device.
 *   stream    a cudaStream_t (as void*) for all the context's work, or NULL to create one.
 * The context copies A and b into device memory it owns (the caller keeps its buffers).
 * The copy is checked for NaN/Inf on the device (TLS_ERR_ARG; one read of the data, host or
 * device pointers alike). *out is NULL on error.
 */
tls_status tls_create_dense(tls_ctx** out, int64_t m, int64_t n, const double* A, int64_t lda,
                            const double* b, int on_device, void* stream);

/*
 * tls_create_csr -- as tls_create_dense with A in CSR form:
 *   row_ptr   m + 1 int64 offsets, row_ptr[0] = 0, non-decreasing, row_ptr[m] = nnz;
 *   col_idx   nnz int32 column indices in [0, n), strictly increasing within each row;
 *   val       nnz FP64 values.
 * Host pointers only (on_device must be 0). row_ptr[0] and row_ptr[m] are checked on the host;
 * after the upload one kernel checks the rest of the structure and that val and b are finite
 * (TLS_ERR_ARG), before anything indexes with col_idx. The column (CSC) index the A^T products
 * gather through is then built on the device (a stable counting sort by column; entries of a
 * column in increasing row order). n <= 51200 (TLS_ERR_ARG above: the per-warp column counters
 * of that sort live in shared memory).
 */
tls_status tls_create_csr(tls_ctx** out, int64_t m, int64_t n, int64_t nnz,
                          const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                          const double* b, int on_device, void* stream);

/*
 * tls_factor -- build the preconditioner R in precision u_f (Alg. 4, the factorisation step;
 * Sec. 3.1): column scaling D, the Gram matrix H = (A D^{-1})^T (A D^{-1}) from A D^{-1}
 * rounded to u_f (tensor cores, FP32 accumulation, for FP16/BF16), Cholesky H + s I = R_H^T R_H
 * with R_H rounded to u_f, and R = R_H D. The shift ladder is s = 0 or (shift_first, FP16/BF16)
 * s = 2 u_f, then s = 2 u_f 4^i (i <= max_shifts) after each non-positive pivot; past the
 * ladder it escalates u_f (FP16/BF16 -> FP32 -> FP64);
 * TLS_ERR_FACTOR_BREAKDOWN if FP64 fails too. opt may be NULL (defaults).
 */
tls_status tls_factor(tls_ctx* ctx, tls_prec u_f, const tls_options* opt);

/*
 * tls_solve -- run RQI-PCGTLS (Alg. 2 with the solves of Alg. 3, precisions as in Alg. 4)
 * from the LS start and return the iterate with the smallest psi_k (Eq. (4)).
 *   tol      stop when psi_k <= tol * (||A||_F^2 + ||b||^2) (a normwise backward error of
 *            the eigenpair of Eq. (1)); 0 leaves only the psi-increase rule and max_rqi.
 *   max_rqi  maximum number of RQI updates, 0 ... 1000 (RQI step k runs k + 1 PCGTLS steps
 *            per solve, so the cap bounds the work of one call; TLS_ERR_ARG above it).
 *   x        n FP64 values, host memory, written on success.
 *   sigma    host, sigma = sqrt(sigma_k^2) of the returned iterate.
 *   info     host, may be NULL.
 * Requires a successful tls_factor (else TLS_ERR_STATE).
 */
tls_status tls_solve(tls_ctx* ctx, double tol, int max_rqi, double* x, double* sigma,
                     tls_info* info);

/* x on the device instead of the host (n FP64 values, device pointer on the context's
 * device; the library cannot check its size); sigma and info on the host as in tls_solve. The
 * copy into x_dev is issued on the context's stream and complete when the call returns. */
tls_status tls_solve_device(tls_ctx* ctx, double tol, int max_rqi, double* x_dev,
                            double* sigma, tls_info* info);

/*
 * tls_factor_batched / tls_solve_batched -- `count` independent problems (contexts of any sizes,
 * each created with its own stream, i.e. stream NULL at creation, for the work to overlap).
 * Up to 16 host worker threads drive the contexts; the kernels of different problems run
 * concurrently on the GPU. per_problem[i] receives each status (may be NULL); x[i] (host, n_i
 * FP64), sigma[i] and infos[i] (may be NULL) the results. Returns the first non-OK status in
 * index order, or TLS_OK. Contexts must be distinct.
 */
tls_status tls_factor_batched(int count, tls_ctx* const* ctxs, tls_prec u_f,
                              const tls_options* opt, tls_status* per_problem);
tls_status tls_solve_batched(int count, tls_ctx* const* ctxs, double tol, int max_rqi,
                             double* const* x, double* sigma, tls_info* infos,
                             tls_status* per_problem);

/*
 * Packed batch -- many small dense problems (n <= TLS_BATCH_MAX_N, any m >= n) packed into
 * shared device arrays and solved together: every phase of RQI-PCGTLS (Alg. 2, with the
 * PCGTLS solves of Alg. 3 in the precisions of Alg. 4) is one kernel launch for the whole
 * batch -- passes over A tiled across all problems, one CTA per problem for the n-sized work.
 * The problems advance in lock step (same RQI step, same PCGTLS step); a problem that stops
 * is skipped by later launches.
 *
 * tls_batch_create_dense -- count >= 1 problems; problem i has A[i] (m[i] x n[i], row-major,
 *   leading dimension lda[i] >= n[i], FP64) and b[i] (m[i] FP64), host pointers (on_device 0)
 *   or device pointers (on_device 1); the copies are checked for NaN/Inf on the device (one
 *   read of the data). The batch copies the data; stream
 *   as in tls_create_dense. Computes the column norms and the FP32 working copy. Errors:
 *   TLS_ERR_ARG (sizes, n > TLS_BATCH_MAX_N, m >= 2^31, non-finite data), TLS_ERR_OOM.
 * tls_batch_factor -- Gram, Cholesky and W = R_H^{-1} of every problem at factor precision
 *   u_f, with the shift ladder of tls_factor per problem and, for a problem whose every shift
 *   breaks down, the next precision (FP16/BF16 -> FP32 -> FP64). opt as in tls_factor (NULL:
 *   defaults); the packed batch requires mode_A = 1 and u = TLS_FP32 or TLS_FP64.
 *   TLS_ERR_FACTOR_BREAKDOWN if some problem broke down at FP64 as well.
 * tls_batch_solve -- RQI-PCGTLS for every problem, same stopping rules as tls_solve and the
 *   same precision fallback (tls_options.fallback) applied per problem. x[i] (host, n[i]
 *   doubles; a NULL entry skips the copy), sigma[i], infos[i] (NULL: none), per_problem[i]
 *   (NULL: none). t_factor_ms / t_solve_ms of every info are the batch's times. max_rqi
 *   0 ... 100 (the captured graph holds every RQI step; TLS_ERR_ARG above it).
 *   Returns TLS_ERR_STATE before a successful factor, else the first non-OK per-problem status.
 */
#define TLS_BATCH_MAX_N 512
typedef struct tls_batch tls_batch;
tls_status tls_batch_create_dense(tls_batch** out, int count, const int64_t* m, const int64_t* n,
                                  const double* const* A, const int64_t* lda,
                                  const double* const* b, int on_device, void* stream);
tls_status tls_batch_factor(tls_batch* bt, tls_prec u_f, const tls_options* opt);
tls_status tls_batch_set_selector(tls_batch* bt, const float* params, const float* mean,
                                  const float* scale);
tls_status tls_batch_features(tls_batch* bt, float* F_host);
tls_status tls_batch_solve(tls_batch* bt, double tol, int max_rqi, double* const* x,
                           double* sigma, tls_info* infos, tls_status* per_problem);
void tls_batch_destroy(tls_batch* bt);
const char* tls_batch_last_error(const tls_batch* bt);

/*
 * Selector network for the packed batch (a learned choice of the factor precision, Sec. 3.1's
 * constraints as its hand-rule baseline): a 16 -> 64 -> 64 -> 4 MLP (ReLU) on 16 features of
 * each problem. tls_batch_factor(bt, TLS_AUTO, opt) factors every problem at FP16, computes the
 * features from A, b and that factor, runs the network, and refactors each problem at the
 * precision it picks (logits for FP16 / BF16 / FP32); with opt->cg_fixed = 0 the fourth output
 * (log10 of the inner tolerance) sets each problem's PCGTLS tolerance. The fallback of
 * tls_batch_solve still guards every problem.
 *
 * tls_batch_set_selector -- params: TLS_MLP_PARAMS FP32 values (W1[64][16], b1[64], W2[64][64],
 *   b2[64], W3[4][64], b3[4]; used rounded to FP16), mean / scale: the feature normalisation
 *   (16 each). Host pointers, copied. Without a selector, TLS_AUTO means FP16.
 * tls_batch_features -- the 16 raw features of every problem from its current factor, into
 *   F_host (count x 16, row-major). TLS_ERR_STATE before a successful tls_batch_factor.
 *
 * Training entry points (device pointers, the caller's stream; FP32 master parameters):
 * tls_mlp_forward -- out (nsamp x 4) for X (nsamp x 16, normalised features).
 * tls_mlp_grad    -- mean loss and gradient over the samples idx[0..nsamp) of X (idx NULL: the
 *   first nsamp rows): cross-entropy of the logits against ycls plus
 *   lambda * ymask * (out[3] - ytol)^2; scratch holds nsamp * (TLS_MLP_PARAMS + 1) floats.
 *   The caller guarantees that every idx value indexes a row of X (and of ycls, ytol, ymask)
 *   and that every ycls value is 0, 1 or 2; the Python trainer checks both.
 * tls_mlp_adam    -- one Adam step (step >= 1) of params with gradient grad and moments m, v.
 */
#define TLS_MLP_PARAMS 5508
#define TLS_SELECTOR_FEATURES 16
tls_status tls_mlp_forward(const float* params, int nsamp, const float* X, float* out,
                           void* stream);
tls_status tls_mlp_grad(const float* params, int nsamp, const float* X, const int* idx,
                        const int* ycls, const float* ytol, const float* ymask, float lambda,
                        float* scratch, float* grad, float* loss_mean, void* stream);
tls_status tls_mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr,
                        float beta1, float beta2, float eps, void* stream);

/*
 * tls_condition -- estimates behind the two constraints on the factor precision (Sec. 3.1):
 * constraint 1, u_q <~ kappa(A)^{-1} (Eq. (5)), and constraint 2,
 * u_q <~ kappa_F(A)^{-1} (1 - sigma_{n+1}^2 / sigma'_n^2) (Eq. (9)).
 * Power iterations (iters steps each, 1 ... 100000) give sigma'_1 (on A^T A through the Gram matrix) and
 * sigma'_n (on (R^T R)^{-1} through the factor's triangular products, so the estimate is that
 * of the computed factor, shift included); ||A^+||_F is taken as ||R^{-1}||_F.
 * out (host, 9 values): sigma'_1, sigma'_n, kappa(A), ||A||_F, ||A^+||_F, kappa_F(A),
 * sigma_{n+1} (of the last tls_solve; NaN before one), constraint 1, constraint 2.
 * Requires a successful tls_factor (TLS_ERR_STATE otherwise).
 */
tls_status tls_condition(tls_ctx* ctx, int iters, double* out);

/*
 * tls_set_selector -- install the selector network for tls_factor(ctx, TLS_AUTO, opt), which
 * then factors at FP16, computes the 16 features of that factor, runs the network and, when it
 * picks BF16 or FP32, refactors at that precision; the network's PCGTLS tolerance is used by
 * tls_solve in tolerance mode (cg_fixed = 0). params: TLS_MLP_PARAMS FP32 values; mean, scale:
 * the feature normalisation (TLS_SELECTOR_FEATURES each). Host pointers, copied. Without a
 * selector, TLS_AUTO means FP16. Same network and features as tls_batch_set_selector.
 */
tls_status tls_set_selector(tls_ctx* ctx, const float* params, const float* mean,
                            const float* scale);

/*
 * tls_features -- the TLS_SELECTOR_FEATURES raw selector features of the current factor
 * (host out), defined as for tls_batch_features. TLS_ERR_STATE before a successful tls_factor.
 */
tls_status tls_features(tls_ctx* ctx, float* F_host);

void tls_destroy(tls_ctx* ctx);
const char* tls_status_str(tls_status s);
const char* tls_last_error(const tls_ctx* ctx);

/* Problem sizes of a context (m, n; nnz = -1 for dense). */
void tls_shape(const tls_ctx* ctx, int64_t* m, int64_t* n, int64_t* nnz);

/*
 * tls_set_allocator -- route the library's device allocations through caller functions
 * (e.g. a framework's caching allocator). alloc(bytes, stream, user) returns a device pointer
 * or NULL; release(ptr, bytes, stream, user) frees it. Pass NULLs to go back to the library's
 * own block cache (tls_pool_enable). Affects allocations made afterwards; every block is
 * returned to the allocator that made it, whatever is set when it is freed.
 */
typedef void* (*tls_alloc_fn)(uint64_t bytes, void* stream, void* user);
typedef void (*tls_free_fn)(void* ptr, uint64_t bytes, void* stream, void* user);
void tls_set_allocator(tls_alloc_fn alloc, tls_free_fn release, void* user);

/*
 * Block cache. Without a caller allocator, the device buffers of contexts and batches, and
 * their small pinned host buffers, come from a process-wide cache: a destroyed context's
 * blocks stay allocated (per device, in size classes of 512 B up to 1 MiB and 2 MiB above)
 * and serve the next context, so that a create / factor / solve / destroy cycle per problem
 * makes no cudaMalloc, cudaFree (which synchronises the device), cudaMallocHost or
 * cudaFreeHost call once the cache is warm. Cached blocks are not cleared: the library never
 * reads a buffer before writing it. A failed cudaMalloc releases the device's cached blocks and
 * is retried once. Thread-safe.
 *   tls_pool_enable(on)  on = 1 (default) caches freed blocks; on = 0 releases the cache and
 *                        frees blocks with cudaFree / cudaFreeHost from then on.
 *   tls_pool_trim()      releases every cached (unused) block; returns the bytes released.
 *                        Blocks held by live contexts are untouched.
 *   tls_pool_stats(...)  bytes cached on devices, cached pinned host bytes, and bytes held by
 *                        live contexts and batches through the cache or cudaMalloc (all
 *                        devices); any pointer may be NULL.
 */
void tls_pool_enable(int on);
uint64_t tls_pool_trim(void);
void tls_pool_stats(uint64_t* cached_device, uint64_t* cached_host, uint64_t* live_device);

/*
 * tls_residual_noalloc -- the FP64 residual block of one RQI step, r = b - A x,
 * sigma^2 = r^T r / (1 + x^T x), f = -A^T r - sigma^2 x, g = -b^T r + sigma^2 and
 * psi = sqrt((||f||^2 + g^2) / (||x||^2 + 1)), for callers that may not allocate device memory.
 * The paper has no counterpart to this entry point: it exists for callers such as an
 * application whose framework allocator already owns the GPU's memory and must account for
 * every byte, a latency-critical loop in which cudaMalloc / cudaFree (which can synchronise the
 * device) are not acceptable, or a plug-in that is handed its buffers and may create nothing.
 * It performs no device allocation at all: its scratch lives in one file-scope device array of
 * TLS_NOALLOC_SCRATCH_BYTES bytes that every GPU loading this library holds until the process
 * exits.
 *   m, n    sizes, m >= 1, 1 <= n <= TLS_NOALLOC_MAX_N (larger n: TLS_ERR_ARG).
 *   A       device, m x n FP64, row-major, leading dimension lda >= n.
 *   b, x    device, m and n FP64 values.
 *   f       device output, n FP64 values.
 *   scal    device output, 5 FP64 values: sigma^2, g, psi, r^T r, b^T r.
 *   stream  cudaStream_t (as void*) the work runs on (NULL: the default stream); the call
 *           returns without synchronising.
 * The first call on a device looks up the scratch array's device address for that device
 * (cudaGetSymbolAddress with the device current); make that first call before any stream
 * capture. Every call shares the one array and keeps the last call's contents in it (the call
 * clears what must start at zero itself), so calls whose work overlaps on the GPU -- on
 * different streams, or from different threads -- race and give wrong results: order them.
 */
#define TLS_NOALLOC_MAX_N 4096
#define TLS_NOALLOC_SCRATCH_BYTES (2u * 1024u * 1024u + 4096u)
tls_status tls_residual_noalloc(int64_t m, int64_t n, const double* A, int64_t lda,
                                const double* b, const double* x, double* f, double* scal,
                                void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TLS_H_ */
