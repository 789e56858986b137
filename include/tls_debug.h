/*
 * tls_debug.h -- inspection entry points of the RQI-PCGTLS library: each runs one step of
 * the solve path on a factored context with host inputs/outputs, so that a caller (or a
 * test) can check the kernels in isolation. Same conventions as tls.h.
 */
#ifndef TLS_DEBUG_H_
#define TLS_DEBUG_H_

#include <stdint.h>
#include "tls.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * tls_export_factor -- copy the factor the solve uses (Sec. 3.1): R_host (n x n, row-major)
 * receives R_H, the Cholesky factor of the column-scaled Gram matrix rounded to u_f (upper
 * triangular; R = R_H diag(d)); d_host (n) the column norms d_j = ||a_j||; H_host (n x n) the
 * scaled Gram matrix H = (A D^{-1})^T (A D^{-1}) as formed from the u_f-rounded data.
 * Any output may be NULL. TLS_ERR_STATE before a successful tls_factor.
 */
tls_status tls_export_factor(tls_ctx* ctx, double* R_host, double* d_host, double* H_host);

/*
 * tls_batch_export_factor -- as tls_export_factor for problem i of a packed batch: R_host and
 * H_host (n_i x n_i), d_host (n_i); any may be NULL. TLS_ERR_ARG for i out of range,
 * TLS_ERR_STATE before a successful tls_batch_factor.
 */
tls_status tls_batch_export_factor(tls_batch* bt, int i, double* R_host, double* d_host,
                                   double* H_host);

/*
 * tls_export_working_copy -- the FP32 working copy of A (m x n, row-major) that the PCGTLS
 * passes read when u = FP32: each entry is A rounded to nearest (even) FP32. A32_host: m*n
 * floats (host). TLS_ERR_STATE before a successful tls_factor with u = FP32.
 */
tls_status tls_export_working_copy(tls_ctx* ctx, float* A32_host);

/*
 * tls_residual -- one RQI residual block in FP64 at x (Alg. 2 lines r_k..g_k, Eq. (2), Eq. (4)):
 * f_host (n) = -A^T r - sigma^2 x with r = b - A x; scal_host[0..4] = sigma^2 = r^T r/(1+x^T x),
 * g = -b^T r + sigma^2, psi = sqrt((||f||^2 + g^2)/(||x||^2 + 1)), r^T r, b^T r.
 * Needs no factor. x_host: n values (host).
 */
tls_status tls_residual(tls_ctx* ctx, const double* x_host, double* f_host, double* scal_host);

/*
 * tls_pcgtls -- PCGTLS (Alg. 3) for (A^T A - sigma2 I) w = f in the context's precision u, for
 * nr = 1 or 2 right-hand sides f0 (and f1) sharing each pass over A: `steps` steps (0 ...
 * 100000), or fewer when ||s_j|| <= cg_tol ||s_0|| (cg_tol > 0; NaN is refused) or
 * delta_j <= 0. w0 (and w1): n values each.
 * iters[2], not_spd[2] (may be NULL): per right-hand side. Host pointers.
 */
tls_status tls_pcgtls(tls_ctx* ctx, int nr, double sigma2, const double* f0, const double* f1,
                      int steps, double cg_tol, double* w0, double* w1, int* iters,
                      int* not_spd);

/*
 * tls_precond -- the preconditioner products in precision u: s0 = R^{-T} y (Alg. 3
 * initialisation) and u = R^{-1} R^{-T} y (the solve with A^T A ~ R^T R of Alg. 2, line 4).
 * y, s0, u: n values (host); s0 or u may be NULL.
 */
tls_status tls_precond(tls_ctx* ctx, const double* y, double* s0, double* u);
/*
 * tls_precond_trsv -- the same two quantities by triangular solves with the factor itself
 * (Alg. 3's R^{-T} and R^{-1}, R = R_H D): blocked substitution on R_H in precision u, one CTA,
 * the reference for the products with the explicit inverse that the solve uses. n_pad is
 * limited by one CTA's shared memory (8192 FP32, 4096 FP64 columns: TLS_ERR_ARG above).
 */
tls_status tls_precond_trsv(tls_ctx* ctx, const double* y, double* s0, double* u);

/* Kernel classes timed by the profiler. */
enum {
  TLS_PROF_SCALE = 0,        /* column norms, FP32 copy, scaled cast of A       */
  TLS_PROF_GRAM = 1,         /* H = A_s^T A_s                                   */
  TLS_PROF_CHOL = 2,         /* blocked Cholesky (each attempt)                 */
  TLS_PROF_TRTRI = 3,        /* rounding of R_H, W = R_H^{-1}, W^T, (R^T R)^{-1} */
  TLS_PROF_RESID_PASS = 4,   /* FP64 pass over A of the RQI residual           */
  TLS_PROF_RESID_REDUCE = 5, /* its reduction: f, sigma^2, g, psi               */
  TLS_PROF_PCG_PASS2 = 6,    /* PCGTLS pass over A, two right-hand sides        */
  TLS_PROF_PCG_PASS1 = 7,    /* PCGTLS pass over A, one right-hand side (LS)    */
  TLS_PROF_PCG_REDUCE = 8,   /* PCGTLS partial reduction and w, y updates       */
  TLS_PROF_PCG_GEMV = 9,     /* products with W and W^T, s and p recurrences    */
  TLS_PROF_VEC = 10,         /* FP64 RQI vector updates                          */
  TLS_PROF_PCG_SOLVE2 = 11,  /* a whole paired PCGTLS solve in one launch (passes, */
                             /* reductions, W and W^T products of every step)    */
  TLS_PROF_PCG_SOLVE1 = 12,  /* the same for one right-hand side (the LS start)  */
  TLS_PROF_NCLASSES = 13
};

/*
 * tls_profile_enable -- when on, every kernel (group) the context launches is bracketed by
 * CUDA events on its stream; times are summed per class after each tls_factor / tls_solve.
 * Enabling (or disabling) resets the sums.
 */
tls_status tls_profile_enable(tls_ctx* ctx, int on);

/*
 * tls_set_pass_variant -- replace the autotuned kernel of the dense passes over A (until the
 * next tls_factor): 0 register kernel, 1 / 2 bulk-copy-staged with 256 / 512 threads (only
 * where the staging fits: TLS_ERR_ARG otherwise), 3 pipelined register kernel, for the
 * residual pass (in FP64) and the PCGTLS pass respectively; variant_fp64 = 4: the residual pass
 * in double-FP32 arithmetic on the pair A32 + Alo (the default for FP32 working precision;
 * TLS_ERR_ARG for FP64 working precision). The FP64 residual passes stop at n_pad = 4096
 * (TLS_ERR_ARG above). TLS_ERR_STATE before tls_factor or for CSR.
 */
tls_status tls_set_pass_variant(tls_ctx* ctx, int variant_fp64, int variant_u);

/*
 * tls_set_small_path -- the solver used for a dense problem small enough to be solved in one
 * launch (u = FP64, n <= 64, mode A, fixed PCGTLS step counts, its rows of A and W in shared
 * memory): 0 automatic (a thread-block cluster of up to 16 CTAs where one fits, else one CTA),
 * 1 one CTA, 2 a cluster (tls_solve returns TLS_ERR_ARG when no cluster shape fits), 3 neither
 * (the multi-kernel path of larger problems). Kept until changed. TLS_ERR_ARG for another
 * value.
 */
tls_status tls_set_small_path(tls_ctx* ctx, int path);
/* Launch count and summed device milliseconds of one class (TLS_PROF_*). */
tls_status tls_profile_get(const tls_ctx* ctx, int cls, int64_t* count, double* ms);
/* Units of work behind the timed launches of class cls: for TLS_PROF_PCG_SOLVE2 / SOLVE1 the
 * PCGTLS steps (passes over A) those launches ran; 0 for the other classes. */
tls_status tls_profile_units(const tls_ctx* ctx, int cls, int64_t* units);
/*
 * tls_set_pcg_fused -- how dense FP32 PCGTLS solves (A-explicit operator) run: 0 automatic (one
 * persistent cooperative launch per solve where the shape fits, else the multi-launch path),
 * 1 the one-launch solve (TLS_ERR_ARG when the shape does not fit it), 2 the multi-launch path
 * (a pass launch and a cooperative step-tail launch per step); 3, 4, 5: the one-launch solve
 * with tiles of A loaded by one bulk copy (TMA) per tile, one bulk copy per row, or 16-byte
 * asynchronous copies by every thread (3 is the default loading, as in 0 and 1; 5 runs the
 * pass of 6); 6: the one-launch solve with one CTA barrier per tile of A and the tile held in
 * registers across it (the default pass has no CTA barrier: each warp waits only for the row
 * values it needs, and a tile stays in shared memory until every warp is done with it); 7: the
 * default pass with smaller tiles and more stages. Kept until changed.
 */
tls_status tls_set_pcg_fused(tls_ctx* ctx, int mode);
/*
 * tls_set_pcg_l2_keep -- bytes of the FP32 copy of A that the one-launch PCGTLS solve loads with
 * an L2 evict-last policy (the first tiles of every CTA's row block), so that they stay in L2
 * from one step's pass to the next; the rest is loaded evict-first. 0 keeps none.
 */
tls_status tls_set_pcg_l2_keep(tls_ctx* ctx, int64_t bytes);
/*
 * tls_set_factor_chain -- c = 1 .. 4 (default 2): the block steps of an FP32 Cholesky factor
 * whose trailing matrix fits run in one persistent cooperative launch of up to c CTAs per SM (a
 * grid barrier between steps); 0: one launch per block step. The arithmetic is the same in
 * all. Kept until changed.
 */
tls_status tls_set_factor_chain(tls_ctx* ctx, int on);
/*
 * tls_set_factor_tc -- 1 (default): for FP16 / BF16 factors, the trailing updates of the block
 * steps that run before the persistent chain (trailing matrices of more than about four 64 x 64
 * tiles per SM, i.e. n above about 2200) go to the tensor cores: the panel rows rounded to u_f
 * (the rows of R-hat the factor keeps), tcgen05 MMAs with FP32 accumulation, the next diagonal
 * block factored by the CTA of the first tile. 0: FP32 updates on the CUDA cores. Kept until
 * changed.
 */
tls_status tls_set_factor_tc(tls_ctx* ctx, int on);
/*
 * tls_trace_enable / tls_trace_get -- phase timestamps (global timer, ns) of the one-launch
 * PCGTLS solve, recorded by CTA 0 into a device buffer of the context when on (the last solve
 * overwrites them): out[0] the launch's start, out[1] the end of the initialisation, then ten
 * words per step j (up to 64 steps) at 2 + 10 j: pass start, pass end, and the ends of
 * grid barrier 1, the update of r and w, the same again (word 4 equals word 3), the
 * M = (R^T R)^{-1} product, grid barrier 2, the new scalars, the next search direction, and the
 * nanoseconds CTA 0 waited for tiles of A in that pass; then, for grid barrier b (0: the first,
 * 2: the second) of step j < 8 (i = 3 j + b), the time CTA c arrived at it (642 + 256 i + c) and
 * the time its arrival was counted (6786 + 256 i + c), and the times CTA 0 saw the last arrival
 * and finished its acquire fence (12930 + 2 i, + 1). Unused words are 0. *count receives the
 * number of words (0 before tls_trace_enable). Host buffer of cap words.
 */
tls_status tls_trace_enable(tls_ctx* ctx, int on);
tls_status tls_trace_get(tls_ctx* ctx, uint64_t* out, int cap, int* count);
/* The same per-class timing for a packed batch (classes as above; PCG_REDUCE covers the
 * per-problem PCGTLS step including its W / W^T products; VEC the small per-problem kernels). */
tls_status tls_batch_profile_enable(tls_batch* bt, int on);
tls_status tls_batch_profile_get(const tls_batch* bt, int cls, int64_t* count, double* ms);
/* Entries of A (sum of m n over the problems still active) that the pass launches of class
 * cls read while profiling was on: the algorithmic work behind the timed launches. */
tls_status tls_batch_profile_elems(const tls_batch* bt, int cls, int64_t* elems);
/* Kernels launched by the library since it was loaded (all contexts). */
uint64_t tls_kernel_launches(void);

/*
 * tls_pool_poison -- fill every block the library allocates from then on (device blocks from
 * the cache or from cudaMalloc, with cudaMemsetAsync on the allocating stream; pinned host
 * blocks with memset) with the byte `value` (0..255; 0xFF makes every FP32 / FP64 word a NaN),
 * so that a test can show that no result depends on a buffer's previous contents. value < 0
 * turns it off (the default). Blocks from a caller allocator (tls_set_allocator) are not filled.
 */
void tls_pool_poison(int value);

#ifdef __cplusplus
}
#endif
#endif /* TLS_DEBUG_H_ */
