// Internal declarations of the packed batched path (not part of the ABI).
//
// A batch holds `count` independent dense TLS problems of uneven sizes (n <= kMaxN) packed into
// shared device arrays. Every phase of RQI-PCGTLS (Alg. 2 with the PCGTLS solves of Alg. 3 / 4)
// runs for all problems of the batch in one launch: the passes over A are split into row tiles
// of every problem (one tile table, one grid), the n-sized work (partial-sum reduction, Rayleigh
// quotient, the PCGTLS scalars, the products with W = R^{-1}) runs one CTA per problem. The
// problems advance in lock step (same RQI step k, same PCGTLS step j); a problem that stopped
// is skipped by every later launch.
#pragma once
#include "tls_internal.h"

namespace tls {
namespace bat {

constexpr int kMaxN = 512;   // columns of one problem in a packed batch
constexpr int kNB = 64;      // Cholesky / Gram block; matrices and n-vectors are padded to it
constexpr int kPT = 256;     // threads of the pass kernels (row tiles)
constexpr int kCT = 512;     // threads of the per-problem kernels
constexpr int kNumCfg = 5;   // lane layouts of the pass kernels (by row length)

// Lane layout of the pass over one problem's rows: `lr` lanes share a row, each lane holds
// `ch` chunks of 4 consecutive columns (columns 4 (lane + lr c) .. +3, c < ch).
struct PassCfg { int lr, ch; };
constexpr PassCfg kCfg[kNumCfg] = {{8, 1}, {16, 1}, {32, 1}, {32, 2}, {32, 4}};
inline int cfg_for(int64_t lda) {
  for (int c = 0; c < kNumCfg; ++c)
    if (lda <= 4 * kCfg[c].lr * kCfg[c].ch) return c;
  return -1;
}

// Per-problem layout (element offsets into the packed arrays).
struct BProb {
  int64_t m, n;
  int64_t lda;    // row stride of A64 / A32: n rounded up to 4 (16-byte rows in FP32)
  int64_t npb;    // n rounded up to kNB: length of the n-vectors, order of H, R, W
  int64_t offA;   // A64 / A32 (m x lda, zero beyond column n)
  int64_t offB;   // b (m)
  int64_t offV;   // n-vectors (npb); pairs of vectors at 2 offV
  int64_t offM;   // npb x npb matrices
  int64_t poff;   // pass partials: tile i of the problem owns elements (poff + i lda) NR ..
  int tile0, ntiles;
  int cfg;        // PassCfg index
  int prec;       // factor precision (Prec) of the current factor
};

struct BTile { int prob, row0, rows, pad_; };

// One CTA of the batched Gram: the 64 x 64 tile (bi, bj) of problem `prob` over rows [r0, r1);
// slot >= 0: a partial tile written to workspace slot `slot` (rows split over several CTAs).
// For the reduction list the same struct names a split tile: its slots are slot .. slot +
// (r1 - r0) - 1.
struct GTile { int prob, bi, bj, r0, r1, slot, pad0_, pad1_; };

// One CTA of the blocked Cholesky / inverse task lists: problem `prob`, block step `s`, block
// (bi, bj). Cholesky step s: the diagonal block (s, s), the panel blocks (s, bj) and the
// trailing blocks (bi, bj), s < bi <= bj, in three launches. Inverse: level bj - bi.
struct CTask { int prob, s, bi, bj; };

// Device state of one problem (host reads it back at the end of a solve).
struct BState {
  // factor
  double shift;
  int info;          // Cholesky breakdown: pivot + 1 (0: success)
  int shifts;        // breakdowns before the factor succeeded
  int fail_pivot;
  int pad0_;
  // RQI (Alg. 2, Eq. (2), Eq. (4))
  double rr, br, xx, sigma2, g, ff, psi;
  double prev_psi, best_psi, best_s2, scale, betak;
  double norm2_A, norm2_b;
  int k, best_k, stop, active;
  int cg_total, not_spd_any, n_psi, pad1_;
  double psi_hist[24];
  // PCGTLS, two right-hand sides (Alg. 3)
  double eta[2], eta0[2], alpha[2], beta[2], delta[2], qq[2], pp[2];
  double cg_sigma2, cg_tol2;
  int done[2], not_spd[2], iters[2], nr, pad2_;
};

// Pointers of the packed arrays (device).
struct BArrays {
  const BProb* probs;
  const BTile* tiles;
  BState* st;
  const double* A64;
  float* A32;
  float* Alo;           // A - A32 rounded to FP32 (the low parts for the double-FP32 residual)
  const double* b;
  double *d, *dinv;
  float* dinv32;
  void* H;              // Gram (FP32, or FP64 for an FP64 factor), upper triangle used
  void* R;              // the factor R_H (same type as H), upper, rounded to u_f
  void *W, *WT;         // W = R_H^{-1} and W^T in the u type
  double *x, *xbest, *f;
  void *vw, *vs, *vp, *vq;   // u-type vector pairs (w, s, p, q)
  void* partU;          // pass partials in the u type (two right-hand sides)
  double* part64;       // pass partials in FP64 (one right-hand side)
  double* spart;        // per-tile scalar partials (4 per tile)
  const double* cg_tol; // per-problem PCGTLS tolerance (selector), or NULL: the solve's own
};

enum PassMode : int { kColnorm = 0, kResid = 1, kPcg = 2, kResidDf = 3 };
enum ResidMode : int { kResidLs = 0, kResidStart = 1, kResidRqi = 2 };

struct SolveParams {
  double tol, psi_accept;
  int max_rqi, psi_rule_ge, cg_fixed, cg_max;
  double cg_tol;
};

// One problem's rows to place into A64: m x n FP64 at src (device, row stride src_ld) to
// A64 + dst (row stride lda).
struct RepackJob {
  const double* src;
  int64_t src_ld, dst, m, n, lda;
};

// ---- launchers (k_batch.cu) --------------------------------------------------------------
// Copies the rows of each job into the padded layout of A64 (one pass; columns n .. lda-1 are
// left as they are) and sets *bad = 1 if a copied value is NaN or infinite.
void launch_repack(double* A64, const RepackJob* jobs, int njobs, int* bad, int num_sms,
                   cudaStream_t s);
void launch_pass_colnorm(const BArrays& a, int ntiles, cudaStream_t s);
void launch_colnorm_post(const BArrays& a, const int* list, int cnt, cudaStream_t s);
// Pass and per-problem kernels take a work list and its length: a device count with a
// persistent grid that loops over the list (graph-capturable: no host knowledge of the count),
// or NULL with one list entry per CTA (grid = the list length).
// The residual pass in double-FP32 arithmetic on A32 + Alo (FP32 working precision; the same
// FP64 outputs as launch_pass_resid).
void launch_pass_resid_df(const BArrays& a, const int* tlist, const int* ntile, int grid,
                          cudaStream_t s);
void launch_pass_resid(const BArrays& a, const int* tlist, const int* ntile, int grid,
                       cudaStream_t s);
template <typename T>
void launch_pass_pcg(const BArrays& a, const int* tlist, const int* ntile, int grid, int nr,
                     cudaStream_t s);
template <typename C>
void launch_gram(const BArrays& a, const GTile* gtiles, int ngt, const GTile* groups, int ngr,
                 void* work, cudaStream_t s);
// tasks: device task list; off (host): starts of the diagonal, panel and trailing lists of each
// step (3 steps + 1 entries)
template <typename C>
void launch_chol(const BArrays& a, const int* list, int cnt, const double* shift, int* info,
                 const CTask* tasks, const int* off, int steps, cudaStream_t s);
// tasks: device task list; off (host): starts of the levels (levels + 1 entries)
template <typename C, typename T>
void launch_trtri(const BArrays& a, const CTask* tasks, const int* off, int levels,
                  cudaStream_t s);
template <typename T>
void launch_solve_init(const BArrays& a, const int* list, int cnt, cudaStream_t s);
template <typename T>
void launch_resid_post(const BArrays& a, const int* list, const int* cnt, int grid, int mode,
                       const SolveParams& sp, cudaStream_t s);
template <typename T>
void launch_pcg_post(const BArrays& a, const int* list, const int* cnt, int grid, cudaStream_t s);
template <typename T>
void launch_ls_finish(const BArrays& a, const int* list, const int* cnt, int grid,
                      cudaStream_t s);
template <typename T>
void launch_rqi_update(const BArrays& a, const int* list, const int* cnt, int grid,
                       cudaStream_t s);
template <typename C, typename T>
void launch_features(const BArrays& a, const int* list, int cnt, const int* nshift,
                     const int* fpiv, const int* prec, const double* shift, const float* mean,
                     const float* scale, float* F, cudaStream_t s);
void launch_count_active(const BArrays& a, const int* list, int cnt, int* out, int* act_probs,
                         int* act_tiles, cudaStream_t s);

}  // namespace bat
}  // namespace tls
