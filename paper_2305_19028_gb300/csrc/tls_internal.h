// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>
#include <atomic>

namespace tls {

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// Every n-indexed dimension (columns of A, H, R, W and the n-vectors) is padded to a multiple
// of kPad. The padding is zero in A and in vectors and the identity in H / R / W, so padded
// entries never contribute and no kernel needs a ragged edge along n.
constexpr int kPad = 64;

// Number of kernels this library has launched (all contexts), for launch accounting.
extern std::atomic<unsigned long long> g_launches;
inline void count_launch(int k = 1) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }

enum class Prec : int { FP16 = 0, BF16 = 1, FP32 = 2, FP64 = 3 };

namespace mlp {
// selector network forward pass: out (nsamp x 4) for normalised features X (nsamp x 16)
void launch_mlp_forward(const float* P, int nsamp, const float* X, float* out, cudaStream_t s);
}

// Device allocation through the caller's allocator (tls_set_allocator), the library's block
// cache or cudaMalloc; hook_free returns a block to where it came from (pool.cu).
void* hook_alloc(size_t bytes, cudaStream_t s);
void hook_free(void* p, size_t bytes, cudaStream_t s);
// Pinned host blocks (cached like the device blocks).
void* host_alloc(size_t bytes);
void host_free(void* p);

// Device scalars of one paired PCGTLS solve (Alg. 3), per right-hand side r in {0, 1}.
struct PcgScalars {
  double eta[2];      // eta_j = ||s_j||^2
  double eta0[2];     // eta_0
  double qq[2];       // ||q_j||^2
  double pp[2];       // ||p_j||^2 (Alg. 3 as printed)
  double tt[2];       // ||A q_j||^2 (A-explicit operator)
  double alpha[2];    // alpha_j
  double beta[2];     // beta_{j-1}: p_j = s_j + beta_{j-1} p_{j-1}
  double delta[2];    // delta_j
  double sigma2;      // shift of the system
  double cg_tol2;     // relative tolerance squared on eta_j / eta_0 (0: off)
  int done[2];        // RHS finished (eta = 0, delta <= 0 or tolerance met)
  int not_spd[2];     // stopped on delta_j < 0
  int iters[2];       // completed steps
  int nr;             // number of right-hand sides (1 or 2)
  int passes;         // passes over A run by the last one-launch solve
  unsigned int counter[4];   // last-block counters, always 0 between kernels
};

// Device scalars of one RQI residual step (Alg. 2 lines r_k .. g_k, Eq. (4)).
struct RqiScalars {
  double rr;          // ||r||^2
  double br;          // b^T r
  double xx;          // ||x||^2
  double sigma2;      // rr / (1 + xx)
  double g;           // -b^T r + sigma2
  double ff;          // ||f||^2
  double psi;         // sqrt((ff + g^2) / (xx + 1))
  double zf, zx;      // z^T f, z^T x
  double betak;       // beta_k
  unsigned int counter[4];
};

// One-CTA solve of a small dense problem in FP64 (k_small.cu).
struct SmallParams {
  double tol, psi_accept;
  int max_rqi, ls_iters, psi_rule_ge, pad_;
};
struct SmallResult {
  double sigma2, psi_final;
  int stop, rqi_steps, best_k, cg_iters, not_spd, n_psi;
  double psi_hist[24];
};
constexpr size_t kSmallSmemMax = 200 * 1024;
// Shared memory the small solve needs for m x n (0 when n is outside 1..64).
size_t small_solve_smem(int m, int n);
// A: m x n of an m x lda FP64 array; W: n x n of an ldw-strided upper-triangular inverse of
// R_H; dinv: 1 / d; scale = ||A||_F^2 + ||b||^2. Returns false (nothing launched) when the
// problem does not fit.
bool launch_small_solve(const double* A, int64_t lda, int m, int n, const double* b,
                        const double* dinv, const double* W, int64_t ldw, double scale,
                        const SmallParams& prm, double* x_out, SmallResult* res, cudaStream_t s);
// The same solve on a thread-block cluster (rows of A spread over up to 16 CTAs, one per SM);
// returns the cluster size launched, or 0 when no cluster shape fits (nothing launched).
// cluster_solve_fits: some cluster shape holds the problem (at least 16 rows per CTA).
bool cluster_solve_fits(int m, int n);
int launch_cluster_solve(const double* A, int64_t lda, int m, int n, const double* b,
                         const double* dinv, const double* W, int64_t ldw, double scale,
                         const SmallParams& prm, double* x_out, SmallResult* res,
                         cudaStream_t s);

// ---------------------------------------------------------------------------------------
// Factorisation kernels (k_factor.cu)
// ---------------------------------------------------------------------------------------
// *flag |= 1 when one of the `count` FP64 values at p (device, 16-byte aligned) is NaN or
// infinite (the input check of the create calls, on the device copy).
void launch_nonfinite(const double* p, int64_t count, int* flag, int num_sms, cudaStream_t s);
// Column squared norms of A (m x n, row-major, lda) with an optional FP32 copy A32 (ld ldo)
// and, with it, the optional low parts Alo = fl32(A - A32) (so A32 + Alo carries A to 2^-48).
// d_out[j] = sqrt(sum_i a_ij^2) (FP64 out). part: scratch of grid x ld doubles.
void launch_colnorm(const double* A, int64_t lda, int64_t m, int64_t n, int64_t npad,
                    float* A32, float* Alo, int64_t ldo, double* d_out, float* dinv32,
                    double* dinv64, double* part, cudaStream_t s);
// AsT[j][i] = fl_prec(A[i][j] / d[j]) (transposed, n x mpad, zero padded). A is FP32 (A32)
// or FP64 (A64) row-major; prec selects the output element type.
void launch_scale_cast_T(const void* A, bool a_is_fp64, int64_t lda, int64_t m, int64_t n,
                         int64_t npad, int64_t mpad, const double* dinv, const float* dinv32,
                         void* AsT, Prec prec, cudaStream_t s);
// H (npad x npad, type T = float for FP16/BF16/FP32 input, double for FP64) = AsT AsT^T,
// identity on the padded diagonal.
// work (may be NULL): for an FP64 Gram of npad <= 128, `chunks` (gram_split_chunks) partial
// npad x npad FP64 matrices (the rows are split over that many CTA sets, summed in fixed order).
void launch_gram_simt(const void* AsT, Prec prec, int64_t n, int64_t npad, int64_t mpad,
                      void* H, cudaStream_t s, void* work = nullptr, int chunks = 1);
// Row chunks of the split FP64 Gram: at least 8 rows each, at most one per SM (num_sms, the
// device's multiprocessor count) and at most 32 MB of partials in all; 1 when npad > 128.
int gram_split_chunks(int64_t npad, int64_t mpad, int num_sms);
// tcgen05 (UMMA) Gram for FP16/BF16 input into FP32 H. Returns false if the shape is not
// supported (falls back to nothing: the caller decides). part (optional, npad^2 floats): the
// 128 x 256-tile form with the K range in two halves (npad a multiple of 256).
bool launch_gram_tc(const void* AsT, Prec prec, int64_t n, int64_t npad, int64_t mpad,
                    float* H, int* err, cudaStream_t s, float* part = nullptr);
// 1 if the tensor-core path can run on the current device (sm_103 and a tensor-map encoder).
bool gram_tc_available();
// Error code recorded in *err by a bounded wait of the tensor-core kernel (0: none); resets it.
int gram_tc_error(int* err, cudaStream_t s);
// Blocked upper Cholesky in place on M (npad x npad, T), with shift added to the first n
// diagonal entries first; the rows of R are rounded to prec block by block and the inverses
// of the 64 x 64 diagonal blocks are written to Wd (npad x npad, other entries untouched);
// info[0] = first failing global pivot + 1 (0: success). gbar (192 words, the first two zero,
// and zero again afterwards unless a bounded wait expired, which records code 31 in *err; the
// others are cleared before use): with it, the
// FP32 block steps whose trailing matrix fits run in one persistent cooperative launch of
// chain_per_sm x num_sms CTAs instead of one launch per step. trace (optional, 256 zeroed words): per block
// step s < 64 of that launch, at 4 s: CTA 0's start, its tile done, its diagonal block done,
// the last tile worker done (global-timer ns).
// ptbuf (optional, npad x 64 halves): FP16 / BF16 factors run the trailing updates of the block
// steps before the chain on the tensor cores (the panel rounded to u_f, FP32 accumulation).
template <typename T>
void launch_cholesky(T* M, int64_t n, int64_t npad, double shift, int* info, T* Wd, Prec prec,
                     cudaStream_t s, unsigned int* gbar = nullptr, int* err = nullptr,
                     int num_sms = 0, unsigned long long* trace = nullptr,
                     int chain_per_sm = 2, void* ptbuf = nullptr);
// Round the upper triangle of R (T) to prec in place (FP16/BF16); no-op for FP32/FP64.
template <typename T>
void launch_round_to(T* R, int64_t npad, Prec prec, cudaStream_t s);
// W = R^{-1} (upper, npad x npad) and WT = W^T (row-major), both T. work: npad x npad T.
// have_diag: W already holds the inverses of the 64 x 64 diagonal blocks and zeros elsewhere.
// part (optional, FP32 only: 3 npad^2 elements): the top levels' long products split in k.
template <typename T>
void launch_trtri(const T* R, T* W, T* WT, T* work, int64_t npad, bool have_diag,
                  cudaStream_t s, T* part = nullptr);
// Convert FP32 <-> FP64 square matrices (used for escalation / export).
void launch_f2d(const float* in, double* out, int64_t count, cudaStream_t s);
void launch_d2f(const double* in, float* out, int64_t count, cudaStream_t s);
void launch_set_identity_pad(void* M, bool fp64, int64_t n, int64_t npad, cudaStream_t s);

// Triangular solves with R = R_H D by blocked substitution on R_H (k_trsv.cu): s = R^{-T} y,
// u = R^{-1} s (y: FP64 on the device, n values; s, u: npad values of T). One CTA; false when
// the right-hand side does not fit its shared memory.
template <typename T>
bool launch_trsv(const T* R, int64_t npad, int64_t n, const T* dinv, const double* y, T* s_out,
                 T* u_out, cudaStream_t s);

// ---------------------------------------------------------------------------------------
// Householder QR preconditioner (k_qr.cu)
// ---------------------------------------------------------------------------------------
// Panel width the cluster panel kernel can hold for m rows (32, 16 or 8; 0: m too large).
template <typename T>
int qr_panel_width(int64_t m);
// Elements of T the QR's work buffer needs (T of a panel and the partial products V^T A).
template <typename T>
size_t qr_work_elems(int64_t m, int64_t n, int num_sms);
// Aq (m x n, row stride ldq, T) = A D^{-1} rounded to prec, from the FP64 master or the FP32
// working copy (row stride lda_src).
template <typename T>
int launch_qr_scale(const void* Asrc, bool from64, int64_t lda_src, int64_t m, int64_t n,
                    const double* dinv, const float* dinv32, Prec prec, T* Aq, int64_t ldq,
                    cudaStream_t s);
// Blocked Householder QR of the m x n row-major A (lda), m >= n, in place: R in the upper
// triangle of rows 0 .. n-1, the reflectors below; tau (n) their scalars. work: qr_work_elems.
// *info = j + 1 for the first reflector whose diagonal entry is zero or not finite. Returns 0,
// or < 0 when the problem does not fit the panel kernel (nothing launched).
template <typename T>
int launch_qr_r(T* A, int64_t lda, int64_t m, int64_t n, T* tau, T* work, int* info,
                int num_sms, cudaStream_t s);
// M (npad x npad) = R with a positive diagonal (rows scaled by sign(R_ii)), zero below, the
// identity on the padding.
template <typename T, typename Tout>
void launch_qr_extract(const T* Aq, int64_t lda, int64_t n, int64_t npad, Tout* M,
                       cudaStream_t s);

// ---------------------------------------------------------------------------------------
// Solve kernels (k_solve.cu)
// ---------------------------------------------------------------------------------------
struct ApassPlan {
  int grid;           // CTAs of the fused pass (= number of partials P)
  int vpt;            // vectors per thread
  bool tma;           // rows staged through shared memory by bulk async copies
  size_t smem;        // dynamic shared memory of the staged kernel
  int threads;        // CTA size of the staged kernel
  int variant;        // 0: register kernel, 1: staged 256 threads, 2: staged 512 threads,
                      // 3: pipelined register kernel
};
constexpr int kApassVariants = 4;
template <typename T>
ApassPlan plan_apass(int64_t m, int64_t npad, int nr, int num_sms, int variant);

// Fused pass over dense A: for every row i, c_r = (resid ? b_i - A_i.v_r : A_i.v_r);
// part[cta][r][:] = sum over the CTA's rows of c_r A_i; sout[r][0] = sum c_r^2,
// sout[r][1] = sum b_i c_r. v: nr vectors of stride ldv.
template <typename T>
void launch_apass(const ApassPlan& plan, const T* A, int64_t lda, int64_t m, int64_t npad,
                  int nr, bool resid, const T* v, int64_t ldv, const double* b, T* part,
                  double* spart, double* sout, unsigned int* counter, const int* done, int* err,
                  cudaStream_t s);

// PCGTLS (Alg. 3) building blocks, T = float or double (the precision u_p).
// prep: y[r] = fin[r] / d (fin FP64, r < nr), w = p = 0, scalars reset.
template <typename T>
void launch_pcg_prep(const double* fin0, double fin0_scale, const double* fin1, int nr,
                     int64_t n, int64_t npad, const double* dinv, T* y, T* w, T* p0, T* p1,
                     PcgScalars* sc, double sigma2, double cg_tol, cudaStream_t s);
// s = W^T y (init) or the s update of step j, partial ||s||^2, last CTA finalises eta/beta.
template <typename T>
void launch_gemv_wt(const T* WT, int64_t npad, const T* y, T* s, const T* p, T* sbuf_part,
                    double* part, PcgScalars* sc, bool init, bool modeA, int nr,
                    cudaStream_t s_);
// p_j = s + beta p_prev (written to p_out), q = D^{-1} W p_j, partial ||q||^2 (and ||p||^2).
template <typename T>
void launch_gemv_w(const T* W, int64_t npad, const T* s, const T* p_prev, T* p_out,
                   const T* dinv, T* q, double* part, PcgScalars* sc, int nr,
                   cudaStream_t s_);
// The rest of PCGTLS step j after its pass over A (reduction of the pass partials, w and y,
// v = W^T y and s, eta and beta) and, when `next`, the head of step j + 1 (p and q = D^{-1} W p),
// in one cooperative launch. bar: 19 zero-initialised words (grid barrier and arrival
// counters, zero again after every launch); err: the bounded waits record code 3 there.
// Returns false when the cooperative launch is not possible.
template <typename T>
bool launch_pcg_step(const T* part, int P, int nr, int64_t npad, T* q, T* w, T* y,
                     const T* dinv, PcgScalars* sc, const double* tt, const T* WT, const T* W,
                     T* s, const T* p_cur, T* p_next, double* gpart, bool next,
                     unsigned int* bar, int* err, int num_sms, cudaStream_t st);
// The RQI residual pass in double-FP32 arithmetic on A = A32 + Alo (k_solve.cu): x, b FP64;
// FP64 per-CTA partials of A^T r in part (grid x npad) and of (||r||^2, b^T r) in spart, their
// totals in sout[0..1]; the same outputs as the FP64 pass. Returns the grid, 0 when npad is
// outside its range (then nothing was launched).
int launch_resid_df(const float* Ahi, const float* Alo, int64_t m, int64_t npad,
                    const double* x, const double* b, double* part, double* spart, double* sout,
                    unsigned int* counter, int* err, int num_sms, cudaStream_t s,
                    RqiScalars* rs = nullptr, double* f = nullptr, double* fpart = nullptr,
                    unsigned int* gbar = nullptr, bool* fused = nullptr);
// A whole PCGTLS solve (A-explicit operator, FP32, nr right-hand sides fin0 * fin0_scale and
// fin1, `steps` steps or fewer on the stop flags) in one persistent cooperative launch of
// num_sms CTAs (k_pcg_fused.cu), preconditioned by M = (R^T R)^{-1} (npad x npad, FP32).
// w, z: nr x npad floats; atd: 2 x nr x npad floats (scratch); part: (num_sms + 1) x nr x npad
// floats (scratch). det = 1: A^T t reduced in CTA order with one more grid barrier per step
// (bitwise reproducible); det = 0: summed with float atomics (the order can change from run
// to run). bar: 96 zero-initialised words (zero again after the launch unless a bounded wait
// expired, which records a code in *err; the caller then clears them). Writes w and the
// scalars in sc. keep_bytes of A (leading tiles of every CTA's rows) are kept in L2. pass_kind:
// 0 warps decoupled, tiles of A held in shared memory until every warp's axpy (the largest
// tiles that leave three stages), 1 one CTA barrier per tile with the tile held in registers
// across it (the only kind for load_mode 2), 2 as 0 with smaller tiles and five stages or more.
bool pcg_fused_supported(int64_t npad, int nr, int num_sms);
cudaError_t launch_pcg_fused(const float* A, int64_t m, int64_t n, int64_t npad, int nr,
                             const double* fin0, double fin0_scale, const double* fin1,
                             const float* M, float* w, float* z, float* atd, float* part,
                             int det, PcgScalars* sc,
                             double sigma2, double cg_tol, int steps, unsigned int* bar, int* err,
                             int num_sms, cudaStream_t st, unsigned long long* trace = nullptr,
                             int load_mode = 0, int64_t keep_bytes = 0, int pass_kind = 0);
// M = D^{-1} W W^T D^{-1} (npad x npad, FP32) from W = R_H^{-1} (upper) and dinv = 1 / d.
// part (optional, 3 npad^2 floats): the k sums split into up to four chunks over more CTAs.
void launch_precond_matrix(const float* W, const float* dinv, int64_t npad, float* M,
                           cudaStream_t s, float* part = nullptr);
// Words of the optional phase trace of the one-launch PCGTLS solve (see k_pcg_fused.cu).
int pcg_fused_trace_words();
// Reduction of the fused pass partials and the update w += alpha q, y = D^{-1}(A^T t - s2 q).
template <typename T>
void launch_pcg_reduce(const T* part, int P, int64_t npad, const T* q, T* w, T* y,
                       const T* dinv, PcgScalars* sc, const double* tt, int nr,
                       cudaStream_t s);
// Alg. 3 as printed: w += alpha q, y = D^{-1} q (no pass over A).
template <typename T>
void launch_pcg_update_R(const T* q, T* w, T* y, const T* dinv, PcgScalars* sc, int nr,
                         int64_t npad, cudaStream_t s);
// RQI residual reduction (FP64): f = -A^T r - sigma2 x, psi etc.
void launch_resid_reduce(const double* part, int P, int64_t npad, const double* x, double* f,
                         const double* sout, RqiScalars* rs, double* fpart, cudaStream_t s);
// x_{k+1} = z + beta_k u with z = x + w (Alg. 2), xx = ||x_{k+1}||^2.
template <typename T>
void launch_rqi_update(double* x, const T* w, const T* u, const double* f, RqiScalars* rs,
                       int64_t n, cudaStream_t s, double* part = nullptr);
// x = x + sigma2 * u (Alg. 2 line 5), xx updated.
template <typename T>
void launch_inverse_step(double* x, const T* u, RqiScalars* rs, int64_t n, cudaStream_t s,
                         double* part = nullptr);
// x = (double) w, xx updated.
template <typename T>
void launch_copy_to_x(double* x, const T* w, RqiScalars* rs, int64_t n, cudaStream_t s,
                      double* part = nullptr);
// Down-convert an FP64 vector (n) to T into a buffer of npad (zero padded).
template <typename T>
void launch_vec_convert(const double* in, T* out, int64_t n, int64_t npad, cudaStream_t s);
// (part: optional scratch of 96 doubles; with it these x kernels run on several CTAs and add
// their partials in CTA order)
void launch_xx(const double* x, RqiScalars* rs, int64_t n, cudaStream_t s, double* part = nullptr);

// ---------------------------------------------------------------------------------------
// Condition estimates (k_cond.cu)
// ---------------------------------------------------------------------------------------
template <typename T>
void launch_dhd(const T* H, int64_t npad, const T* dinv, const T* x, T* y, cudaStream_t s);
template <typename T>
void launch_power_finish(T* x, const T* y, int64_t n, double* lam, cudaStream_t s);
template <typename T>
void launch_power_init(T* x, int64_t n, int64_t npad, cudaStream_t s);
template <typename T>
int launch_frob_dw(const T* W, int64_t n, int64_t npad, const T* dinv, double* part,
                   cudaStream_t s);
template <typename T>
void launch_vec_to_double(const T* x, double* y, int64_t n, int64_t npad, cudaStream_t s);
void launch_feature_normalise(float* F, const float* mean, const float* scale, cudaStream_t s);
// The 16 selector features of one factored problem into F (device, 16 floats); x, y: npad
// scratch vectors; scratch: 1 + ceil(n/8) doubles.
template <typename T>
void launch_features(const double* d, const T* R, const T* W, const T* WT, int64_t n, int64_t npad,
                     int64_t m, double norm2_A, double norm2_b, int nshift, double shift,
                     int fail_pivot, double log10_uf, T* x, T* y, double* scratch, float* F,
                     cudaStream_t s);

// ---------------------------------------------------------------------------------------
// Sparse (CSR + CSC) kernels (k_sparse.cu)
// ---------------------------------------------------------------------------------------
void sparse_to_f32(const double* v64, float* v32, int64_t nnz, cudaStream_t s);
void sparse_colnorm(const int* cp, const double* cv64, const float* cv32, int64_t n, int64_t npad,
                    double* d, double* dinv, float* dinv32, cudaStream_t s);
template <typename T>
void sparse_gram(const int* rp, const int* ci, const float* v32, const double* v64,
                 const int* cp, const int* ri, const float* cv32, const double* cv64,
                 const float* dinv32, const double* dinv, int64_t n, int64_t npad, int64_t nnz,
                 Prec prec, T* as, T* cas, T* H, cudaStream_t s);
void sparse_resid(const int* rp, const int* ci, const double* v64, const int* cp, const int* ri,
                  const double* cv64, const double* b, const double* x, int64_t m, int64_t n,
                  int64_t npad, double* r, double* f, double* spart, double* sout,
                  unsigned int* counter, RqiScalars* rs, double* fpart, cudaStream_t s);
template <typename T>
void sparse_pcg_pass(const int* rp, const int* ci, const T* val, const int* cp, const int* ri,
                     const T* cval, int64_t m, int64_t n, int64_t npad, int nr, const T* q, T* t,
                     T* w, T* y, const T* dinv, PcgScalars* sc, double* spart, double* sout,
                     unsigned int* counter, const int* done, cudaStream_t s);
int sparse_grid_rows(int64_t m);
// CSR check on the device: rp64 (m + 1 int64) non-decreasing from 0 to nnz, ci in [0, n) and
// strictly increasing per row, v64 and b finite; writes rp32; *bad |= 1 on a violation.
void csr_check(const int64_t* rp64, const int* ci, const double* v64, const double* b, int64_t m,
               int64_t n, int64_t nnz, int* rp32, int* bad, cudaStream_t s);
// CSC index of a checked CSR matrix (stable counting sort by column): cp (npad + 1), ri and cv
// (nnz). G CTAs; scratch cnt and off (G x npad ints each), tot (npad ints). Needs
// csc_build_warps(npad) >= 1 (npad <= 51200).
int csc_build_warps(int64_t npad);
void csc_build(const int* rp32, const int* ci, const double* v64, int64_t m, int64_t npad,
               int64_t nnz, int G, int* cnt, int* off, int* tot, int* cp, int* ri, double* cv,
               cudaStream_t s);

}  // namespace tls
