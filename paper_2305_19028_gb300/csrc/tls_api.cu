// C ABI of the library (include/tls.h, include/tls_debug.h): contexts, the factorisation
// ladder and the RQI-PCGTLS driver (Alg. 2 / Alg. 4 of Oktay & Carson, arXiv 2305.19028).
#include "../../include/tls.h"
#include "../../include/tls_debug.h"
#include "tls_internal.h"
#include "tls_options.h"

#include <cmath>
#include <map>
#include <mutex>
#include <thread>
#include <atomic>
#include <tuple>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace tls {
std::atomic<unsigned long long> g_launches{0};
}

using tls::Prec;
using tls::PcgScalars;
using tls::RqiScalars;

namespace {

struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace

constexpr int kBarWords = 640;   // the one-launch solve: [0, 128); the factor chain: [128, 576);
                                 // the cooperative residual pass: [576, 578)

struct tls_ctx {
  int64_t m = 0, n = 0, npad = 0, mpad = 0, nnz = -1;
  int device = 0, num_sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  std::vector<DevBuf> bufs;
  // persistent work buffers, reused by every factor / solve while they are large enough (no
  // cudaMalloc / cudaFree, which synchronise the device, between repeated calls)
  DevBuf slots[24];
  int small_path = 0;      // tls_set_small_path
  int pcg_fused = 0;       // tls_set_pcg_fused
  int fused_load = 0;      // how the one-launch solve loads tiles of A (tls_set_pcg_fused)
  int fused_pass = 0;      // how its pass holds the tiles (tls_set_pcg_fused)
  int64_t l2_keep = 0;     // bytes of A the one-launch solve keeps resident in L2
  unsigned int* fbar = nullptr;   // kBarWords barrier words: [0], [64] the one-launch solve's
                                  // counter and abort word; from [128] the persistent Cholesky's
  int chol_tc = 1;                // trailing updates before the chain on the tensor cores
  int chol_chain = 2;             // block steps of the FP32 factor in one persistent launch
                                  // (up to this many CTAs per SM; 0: one launch per step)
  RqiScalars* h_norm = nullptr;   // pinned: ||A||_F^2 (xx) and ||b||^2 read back after the factor

  // problem data (device)
  bool sparse = false;     // A held as CSR + CSC instead of dense
  int* rp = nullptr;       // CSR row offsets (m + 1)
  int* ci = nullptr;       // CSR column indices (nnz)
  double* v64 = nullptr;   // CSR values (nnz)
  float* v32 = nullptr;    // CSR values rounded to FP32
  int* cp = nullptr;       // CSC column offsets (npad + 1)
  int* ri = nullptr;       // CSC row indices (nnz)
  double* cv64 = nullptr;  // CSC values (nnz)
  float* cv32 = nullptr;   // CSC values rounded to FP32
  double* rbuf = nullptr;  // residual r (m, sparse path)
  void* tbuf = nullptr;    // t = A q, two right-hand sides (2 m, u type, sparse path)
  double* A64 = nullptr;   // m x npad, zero padded columns
  double* b = nullptr;     // m
  float* A32 = nullptr;    // m x npad, made by tls_factor when u = FP32
  float* Alo = nullptr;    // m x npad, fl32(A - A32): A32 + Alo is A to 2^-48 (residual pass)
  double norm2_A = 0.0, norm2_b = 0.0;

  // factor
  bool factored = false;
  bool colnorm_done = false;   // D (and A_u in FP32 when a32_done) depend on A alone: computed once
  bool a32_done = false;
  Prec u = Prec::FP32;
  tls_prec uf_used = TLS_FP16;
  tls_options opt{};
  double* d = nullptr;       // column norms (npad)
  double* dinv = nullptr;    // 1 / d
  float* dinv32 = nullptr;   // 1 / d in FP32 (for the FP32 PCGTLS kernels)
  void* H = nullptr;         // scaled Gram (npad^2, float or double, see H_fp64)
  bool H_fp64 = false;
  bool gram_tc_used = false;
  void* R = nullptr;         // R_H rounded to u_f, stored in the u type (npad^2)
  void* W = nullptr;         // R_H^{-1} (u type)
  void* WT = nullptr;        // W^T (u type)
  float* PM = nullptr;       // (R^T R)^{-1} = D^{-1} W W^T D^{-1} (FP32, for the one-launch solve)
  bool pm_ready = false;     // PM belongs to the current factor
  int shifts = 0;
  double shift = 0.0;
  int64_t fail_pivot = -1;   // pivot index of the last breakdown (-1: none)
  double last_sigma2 = -1.0; // sigma^2 of the last successful tls_solve (-1: none yet)
  double constr2_scaled = NAN;   // constraint 2 of A D^{-1} (sigma_{n+1} = 0) of the factor
  int escalations = 0;       // factor precisions skipped by the constraint guard
  int stall_trigger = 0;     // TLS_TRIGGER_* of the last TLS_STOP_STALL
  double t_factor_ms = 0.0;
  // selector network (tls_factor with TLS_AUTO)
  bool has_sel = false;
  float* dsel = nullptr;     // parameters, then feature mean and scale
  bool use_sel_tol = false;  // the last factor was chosen by the network: its PCGTLS tolerance
  double sel_cg_tol = 0.0;
  int sel_class = -1;

  // solve workspace
  double* x = nullptr;       // npad
  double* x_best = nullptr;  // npad
  double* f = nullptr;       // npad
  void* vbuf = nullptr;      // u-type vectors: y, w, s, p0, p1, q (each 2 x npad)
  void* part = nullptr;      // pass partials, u type: P x 2 x npad
  double* part64 = nullptr;  // FP64 residual pass partials: P x npad
  double* spart = nullptr;   // P x 2 x 2
  double* sout = nullptr;    // 4 (residual) + 4 (PCGTLS)
  double* gpart = nullptr;   // gemv / reduction partials (1024 x 4)
  unsigned int* counter = nullptr;  // 4
  int* derr = nullptr;       // error word of bounded device waits (0: none)
  PcgScalars* sc = nullptr;
  RqiScalars* rs = nullptr;
  int P64 = 0, PU = 0;
  bool resid_df = true;      // the residual pass in double-FP32 arithmetic where it applies
  tls::ApassPlan plan64{}, planU{};
  // pinned host mirrors
  RqiScalars* h_rs = nullptr;
  PcgScalars* h_sc = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t evf0 = nullptr, evf1 = nullptr;   // the last factor's start and end
  bool factor_time_pending = false;
  // per-kernel-class CUDA-event timing (tls_profile_enable)
  bool prof_on = false;
  std::vector<cudaEvent_t> pev;
  std::vector<int> pcls;
  int pused = 0;
  double prof_ms[TLS_PROF_NCLASSES] = {};
  int64_t prof_cnt[TLS_PROF_NCLASSES] = {};
  int64_t prof_units[TLS_PROF_NCLASSES] = {};
  bool last_pcg_fused = false;     // the last PCGTLS solve ran as one launch
  bool trace_on = false;           // tls_trace_enable
  unsigned long long* trace = nullptr;   // phase timestamps of the last one-launch solve
};

namespace {

void set_err(tls_ctx* c, const std::string& s) {
  if (c) c->err = s;
}

tls_status cuda_status(tls_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return TLS_OK;
  set_err(c, std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? TLS_ERR_OOM : TLS_ERR_CUDA;
}

#define TLS_CK(call)                                                  \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) return cuda_status(ctx, e_, #call);       \
  } while (0)

#define TLS_CK_LAUNCH(what)                                           \
  do {                                                                \
    cudaError_t e_ = cudaGetLastError();                              \
    if (e_ != cudaSuccess) return cuda_status(ctx, e_, what);        \
  } while (0)

}  // namespace


namespace {

void* dev_alloc(tls_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = tls::hook_alloc(bytes, c->stream);
  if (p) c->bufs.push_back({p, bytes});
  return p;
}

void dev_free(tls_ctx* c, void* p) {
  if (!p) return;
  for (size_t i = 0; i < c->bufs.size(); ++i) {
    if (c->bufs[i].ptr == p) {
      tls::hook_free(p, c->bufs[i].bytes, c->stream);
      c->bufs.erase(c->bufs.begin() + (long)i);
      return;
    }
  }
}

enum Slot : int {
  kSlotCpart, kSlotInfo, kSlotAsT, kSlotH, kSlotM, kSlotWc, kSlotR, kSlotW, kSlotWT, kSlotWork,
  kSlotVbuf, kSlotPart, kSlotTbuf, kSlotCond, kSlotNorm, kSlotFeat, kSlotGsplit, kSlotPM,
  kSlotQR, kSlotQRwork, kSlotPMpart, kSlotPT, kSlotCount
};
static_assert(kSlotCount <= 24, "slots");

// A persistent buffer of at least `bytes` for slot `id` (contents not kept when it grows).
void* slot(tls_ctx* c, int id, size_t bytes) {
  if (bytes == 0) bytes = 16;
  DevBuf& sl = c->slots[id];
  if (sl.ptr && sl.bytes >= bytes) return sl.ptr;
  if (sl.ptr) dev_free(c, sl.ptr);
  sl.ptr = dev_alloc(c, bytes);
  sl.bytes = sl.ptr ? bytes : 0;
  return sl.ptr;
}

template <typename T>
T* alloc_t(tls_ctx* c, int64_t count) {
  return static_cast<T*>(dev_alloc(c, sizeof(T) * (size_t)count));
}


tls_status ctx_common_init(tls_ctx* ctx, int64_t m, int64_t n, void* stream) {
  ctx->m = m;
  ctx->n = n;
  ctx->npad = tls::round_up(n, tls::kPad);
  ctx->mpad = tls::round_up(m, tls::kPad);
  TLS_CK(cudaGetDevice(&ctx->device));
  TLS_CK(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device));
  if (stream) {
    ctx->stream = static_cast<cudaStream_t>(stream);
  } else {
    TLS_CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
    ctx->own_stream = true;
  }
  TLS_CK(cudaEventCreate(&ctx->ev0));
  TLS_CK(cudaEventCreate(&ctx->ev1));
  TLS_CK(cudaEventCreate(&ctx->evf0));
  TLS_CK(cudaEventCreate(&ctx->evf1));
  ctx->h_rs = static_cast<RqiScalars*>(tls::host_alloc(sizeof(RqiScalars)));
  ctx->h_sc = static_cast<PcgScalars*>(tls::host_alloc(sizeof(PcgScalars)));
  ctx->h_norm = static_cast<RqiScalars*>(tls::host_alloc(2 * sizeof(RqiScalars)));
  if (!ctx->h_rs || !ctx->h_sc || !ctx->h_norm) {
    set_err(ctx, "pinned host allocation failed");
    return TLS_ERR_OOM;
  }
  const int64_t npad = ctx->npad;
  ctx->b = alloc_t<double>(ctx, m);
  ctx->x = alloc_t<double>(ctx, npad);
  ctx->x_best = alloc_t<double>(ctx, npad);
  ctx->f = alloc_t<double>(ctx, npad);
  ctx->d = alloc_t<double>(ctx, npad);
  ctx->dinv = alloc_t<double>(ctx, npad);
  ctx->dinv32 = alloc_t<float>(ctx, npad);
  ctx->sout = alloc_t<double>(ctx, 8);
  ctx->gpart = alloc_t<double>(ctx, 4096);
  ctx->counter = alloc_t<unsigned int>(ctx, 32);   // last-CTA counters; [4..22] PCGTLS step
  ctx->fbar = alloc_t<unsigned int>(ctx, kBarWords);
  ctx->derr = alloc_t<int>(ctx, 1);
  ctx->sc = alloc_t<PcgScalars>(ctx, 1);
  ctx->rs = alloc_t<RqiScalars>(ctx, 1);
  if (!ctx->b || !ctx->x || !ctx->x_best || !ctx->f || !ctx->d || !ctx->dinv || !ctx->sout ||
      !ctx->gpart || !ctx->counter || !ctx->sc || !ctx->rs || !ctx->derr || !ctx->dinv32 ||
      !ctx->fbar) {
    set_err(ctx, "device allocation failed");
    return TLS_ERR_OOM;
  }
  TLS_CK(cudaMemsetAsync(ctx->counter, 0, 32 * sizeof(unsigned int), ctx->stream));
  TLS_CK(cudaMemsetAsync(ctx->fbar, 0, kBarWords * sizeof(unsigned int), ctx->stream));
  TLS_CK(cudaMemsetAsync(ctx->derr, 0, sizeof(int), ctx->stream));
  TLS_CK(cudaMemsetAsync(ctx->sc, 0, sizeof(PcgScalars), ctx->stream));
  TLS_CK(cudaMemsetAsync(ctx->rs, 0, sizeof(RqiScalars), ctx->stream));
  TLS_CK(cudaMemsetAsync(ctx->x, 0, sizeof(double) * npad, ctx->stream));
  TLS_CK(cudaMemsetAsync(ctx->x_best, 0, sizeof(double) * npad, ctx->stream));
  TLS_CK(cudaMemsetAsync(ctx->f, 0, sizeof(double) * npad, ctx->stream));
  // FP64 residual pass plan and partials
  ctx->plan64 = tls::plan_apass<double>(m, npad, 1, ctx->num_sms, 1);
  ctx->P64 = ctx->plan64.grid;
  // partials sized for the largest grid of any pass variant (2 CTAs per SM)
  ctx->part64 = alloc_t<double>(ctx, (int64_t)2 * ctx->num_sms * npad);
  // pass partials: dense passes use <= 2 CTAs per SM; the sparse row kernels one CTA per 256 rows
  const int64_t nsp = std::max<int64_t>((int64_t)2 * ctx->num_sms * 2 * 2,
                                        4 * (int64_t)tls::sparse_grid_rows(m)) + 16;
  ctx->spart = alloc_t<double>(ctx, nsp);
  if (!ctx->part64 || !ctx->spart) {
    set_err(ctx, "device allocation failed");
    return TLS_ERR_OOM;
  }
  return TLS_OK;
}

void destroy_ctx(tls_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  while (!ctx->bufs.empty()) dev_free(ctx, ctx->bufs.back().ptr);
  tls::host_free(ctx->h_rs);
  tls::host_free(ctx->h_norm);
  tls::host_free(ctx->h_sc);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  if (ctx->evf0) cudaEventDestroy(ctx->evf0);
  if (ctx->evf1) cudaEventDestroy(ctx->evf1);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

size_t u_size(Prec u) { return u == Prec::FP64 ? 8 : 4; }

// Brackets one kernel (or kernel group) with CUDA events on the context stream when
// profiling is on; the times are collected after the next synchronisation.
struct Prof {
  tls_ctx* c;
  int idx = -1;
  Prof(tls_ctx* ctx, int cls) : c(ctx) {
    if (!c->prof_on) return;
    if ((size_t)(2 * c->pused + 2) > c->pev.size()) {
      for (int k = 0; k < 2; ++k) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        c->pev.push_back(e);
      }
      c->pcls.push_back(0);
    }
    idx = c->pused++;
    c->pcls[idx] = cls;
    cudaEventRecord(c->pev[2 * idx], c->stream);
  }
  ~Prof() {
    if (idx >= 0) cudaEventRecord(c->pev[2 * idx + 1], c->stream);
  }
};

void prof_collect(tls_ctx* c) {
  for (int i = 0; i < c->pused; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->pev[2 * i], c->pev[2 * i + 1]) == cudaSuccess) {
      c->prof_ms[c->pcls[i]] += ms;
      c->prof_cnt[c->pcls[i]] += 1;
    }
  }
  c->pused = 0;
}

// ---------------------------------------------------------------------------------------
// RQI residual block (FP64 pass over A): r, sigma^2, f, g, psi at ctx->x.
// ---------------------------------------------------------------------------------------
// The residual pass runs in double-FP32 arithmetic on A32 + Alo (k_solve.cu, resid_df_kernel)
// for FP32 working precision once the pair exists and n_pad is in the kernel's range; the FP64
// kernels otherwise (plain FP64 solves, CSR, or when turned off by tls_set_pass_variant).
bool resid_df_active(const tls_ctx* ctx) {
  return ctx->resid_df && !ctx->sparse && ctx->u == Prec::FP32 && ctx->A32 != nullptr &&
         ctx->Alo != nullptr && ctx->a32_done && ctx->npad <= 8192 && ctx->npad % 64 == 0;
}

tls_status residual_pass(tls_ctx* ctx) {
  if (ctx->sparse) {
    Prof pr(ctx, TLS_PROF_RESID_PASS);
    tls::sparse_resid(ctx->rp, ctx->ci, ctx->v64, ctx->cp, ctx->ri, ctx->cv64, ctx->b, ctx->x,
                      ctx->m, ctx->n, ctx->npad, ctx->rbuf, ctx->f, ctx->spart, ctx->sout,
                      ctx->counter, ctx->rs, ctx->gpart, ctx->stream);
    TLS_CK_LAUNCH("sparse residual pass");
    return TLS_OK;
  }
  int P = 0;
  bool reduced = false;
  {
    Prof pr(ctx, TLS_PROF_RESID_PASS);
    if (resid_df_active(ctx))
      // (the reduction to f, sigma^2, g, psi in the same cooperative launch, barrier words at
      // fbar[576], clear of the one-launch solve's and the factor chain's)
      P = tls::launch_resid_df(ctx->A32, ctx->Alo, ctx->m, ctx->npad, ctx->x, ctx->b,
                               ctx->part64, ctx->spart, ctx->sout, ctx->counter, ctx->derr,
                               ctx->num_sms, ctx->stream, ctx->rs, ctx->f, ctx->gpart,
                               ctx->fbar + 576, &reduced);
    if (P == 0) {
      if (ctx->npad > 4096) {
        set_err(ctx, "the FP64 residual pass supports n_pad <= 4096");
        return TLS_ERR_ARG;
      }
      tls::launch_apass<double>(ctx->plan64, ctx->A64, ctx->npad, ctx->m, ctx->npad, 1, true,
                                ctx->x, ctx->npad, ctx->b, ctx->part64, ctx->spart, ctx->sout,
                                ctx->counter, nullptr, ctx->derr, ctx->stream);
      P = ctx->P64;
    }
  }
  if (!reduced) {
    Prof pr(ctx, TLS_PROF_RESID_REDUCE);
    tls::launch_resid_reduce(ctx->part64, P, ctx->npad, ctx->x, ctx->f, ctx->sout, ctx->rs,
                             ctx->gpart, ctx->stream);
  }
  TLS_CK_LAUNCH("residual pass");
  return TLS_OK;
}

// ---------------------------------------------------------------------------------------
// Paired PCGTLS (Alg. 3) in the u type T: nr right-hand sides fin0 * s0 and fin1.
// ---------------------------------------------------------------------------------------
// device address of the PCGTLS termination flags (no host dereference of the device pointer)
const int* done_ptr(tls_ctx* ctx) {
  return reinterpret_cast<const int*>(reinterpret_cast<const char*>(ctx->sc) +
                                      offsetof(PcgScalars, done));
}

template <typename T>
const T* dinv_t(tls_ctx* ctx);
template <>
const float* dinv_t<float>(tls_ctx* ctx) { return ctx->dinv32; }
template <>
const double* dinv_t<double>(tls_ctx* ctx) { return ctx->dinv; }

template <typename T>
struct UVecs {
  T *y, *w, *s, *p0, *p1, *q;
};

template <typename T>
UVecs<T> uvecs(tls_ctx* ctx) {
  T* base = static_cast<T*>(ctx->vbuf);
  const int64_t k = 2 * ctx->npad;
  return {base, base + k, base + 2 * k, base + 3 * k, base + 4 * k, base + 5 * k};
}

template <typename T>
tls_status run_pcg(tls_ctx* ctx, int nr, const double* fin0, double s0, const double* fin1,
                   double sigma2, int steps, double cg_tol, bool modeA) {
  UVecs<T> v = uvecs<T>(ctx);
  const int64_t npad = ctx->npad;
  const T* Au = (ctx->u == Prec::FP64) ? reinterpret_cast<const T*>(ctx->A64)
                                       : reinterpret_cast<const T*>(ctx->A32);
  const T* W = static_cast<const T*>(ctx->W);
  const T* WT = static_cast<const T*>(ctx->WT);
  if constexpr (std::is_same<T, float>::value) {
  if (modeA && !ctx->sparse && steps > 0 && ctx->pcg_fused != 2 &&
      tls::pcg_fused_supported(npad, nr, ctx->num_sms)) {
    // the whole solve in one persistent cooperative launch, preconditioned by the matrix
    // (R^T R)^{-1} formed once per factor
    cudaError_t e = cudaSuccess;
    if (!ctx->pm_ready) {
      ctx->PM = static_cast<float*>(slot(ctx, kSlotPM, sizeof(float) * (size_t)npad * npad));
      if (!ctx->PM) {
        set_err(ctx, "device allocation failed (preconditioner matrix)");
        return TLS_ERR_OOM;
      }
      float* mpart = static_cast<float*>(slot(ctx, kSlotPMpart, sizeof(float) * 3 * (size_t)npad * npad));
      Prof pr(ctx, TLS_PROF_TRTRI);
      tls::launch_precond_matrix(reinterpret_cast<const float*>(W), ctx->dinv32, npad, ctx->PM,
                                 ctx->stream, mpart);
      e = cudaGetLastError();
      ctx->pm_ready = (e == cudaSuccess);
    }
    if (e == cudaSuccess) {
      Prof pr(ctx, nr == 2 ? TLS_PROF_PCG_SOLVE2 : TLS_PROF_PCG_SOLVE1);
      e = tls::launch_pcg_fused(
          reinterpret_cast<const float*>(ctx->A32), ctx->m, ctx->n, npad, nr, fin0, s0, fin1,
          ctx->PM, reinterpret_cast<float*>(v.w), reinterpret_cast<float*>(v.s),
          reinterpret_cast<float*>(v.p0), static_cast<float*>(ctx->part),
          ctx->opt.reproducible != 0 ? 1 : 0, ctx->sc, sigma2, cg_tol, steps, ctx->fbar,
          ctx->derr,
          ctx->num_sms,
          ctx->stream, ctx->trace_on ? ctx->trace : nullptr, ctx->fused_load, ctx->l2_keep,
          ctx->fused_pass);
    }
    if (e == cudaSuccess) {
      ctx->last_pcg_fused = true;
      if (ctx->prof_on && nr == 1) ctx->prof_units[TLS_PROF_PCG_SOLVE1] += steps;
      return TLS_OK;
    }
    (void)cudaGetLastError();
    if (ctx->pcg_fused == 1) {
      set_err(ctx, std::string("one-launch PCGTLS solve failed: ") + cudaGetErrorString(e));
      return TLS_ERR_CUDA;
    }
    ctx->pcg_fused = 2;   // not launchable here (e.g. no cooperative residency): multi-launch
  }
  }
  ctx->last_pcg_fused = false;
  {
    Prof pr(ctx, TLS_PROF_PCG_GEMV);
    tls::launch_pcg_prep<T>(fin0, s0, fin1, nr, ctx->n, npad, ctx->dinv, v.y, v.w, v.p0, v.p1,
                            ctx->sc, sigma2, cg_tol, ctx->stream);
    tls::launch_gemv_wt<T>(WT, npad, v.y, v.s, nullptr, nullptr, ctx->gpart, ctx->sc, true,
                           modeA, nr, ctx->stream);
  }
  T* pb[2] = {v.p0, v.p1};
  if (modeA && !ctx->sparse && steps > 0) {
    // pass over A, then the rest of the step and the head of the next in one cooperative
    // launch (pcg_step)
    {
      Prof pr(ctx, TLS_PROF_PCG_GEMV);
      tls::launch_gemv_w<T>(W, npad, v.s, pb[1], pb[0], dinv_t<T>(ctx), v.q, ctx->gpart, ctx->sc,
                            nr, ctx->stream);
    }
    for (int j = 0; j < steps; ++j) {
      T* pcur = pb[j & 1];
      T* pnext = pb[(j + 1) & 1];
      {
        Prof pr(ctx, nr == 2 ? TLS_PROF_PCG_PASS2 : TLS_PROF_PCG_PASS1);
        tls::launch_apass<T>(ctx->planU, Au, npad, ctx->m, npad, nr, false, v.q, npad, nullptr,
                             static_cast<T*>(ctx->part), ctx->spart, ctx->sout + 4,
                             ctx->counter + 1, done_ptr(ctx), ctx->derr, ctx->stream);
      }
      Prof pr(ctx, TLS_PROF_PCG_REDUCE);
      if (!tls::launch_pcg_step<T>(static_cast<const T*>(ctx->part), ctx->PU, nr, npad, v.q, v.w,
                                   v.y, dinv_t<T>(ctx), ctx->sc, ctx->sout + 4, WT, W, v.s, pcur,
                                   pnext, ctx->gpart, j + 1 < steps, ctx->counter + 4, ctx->derr,
                                   ctx->num_sms, ctx->stream)) {
        set_err(ctx, "cooperative launch of the PCGTLS step failed");
        return TLS_ERR_CUDA;
      }
    }
    TLS_CK_LAUNCH("pcgtls");
    return TLS_OK;
  }
  for (int j = 0; j < steps; ++j) {
    T* pcur = pb[j & 1];
    T* pprev = pb[(j + 1) & 1];
    {
      Prof pr(ctx, TLS_PROF_PCG_GEMV);
      tls::launch_gemv_w<T>(W, npad, v.s, pprev, pcur, dinv_t<T>(ctx), v.q, ctx->gpart, ctx->sc,
                            nr, ctx->stream);
    }
    if (modeA && ctx->sparse) {
      Prof pr(ctx, nr == 2 ? TLS_PROF_PCG_PASS2 : TLS_PROF_PCG_PASS1);
      const bool f32 = sizeof(T) == 4;
      const T* val = f32 ? reinterpret_cast<const T*>(ctx->v32) : reinterpret_cast<const T*>(ctx->v64);
      const T* cval = f32 ? reinterpret_cast<const T*>(ctx->cv32) : reinterpret_cast<const T*>(ctx->cv64);
      tls::sparse_pcg_pass<T>(ctx->rp, ctx->ci, val, ctx->cp, ctx->ri, cval, ctx->m, ctx->n, npad, nr,
                              v.q, static_cast<T*>(ctx->tbuf), v.w, v.y, dinv_t<T>(ctx), ctx->sc,
                              ctx->spart, ctx->sout + 4, ctx->counter + 1, done_ptr(ctx),
                              ctx->stream);
    } else if (modeA) {
      {
        Prof pr(ctx, nr == 2 ? TLS_PROF_PCG_PASS2 : TLS_PROF_PCG_PASS1);
        tls::launch_apass<T>(ctx->planU, Au, npad, ctx->m, npad, nr, false, v.q, npad, nullptr,
                             static_cast<T*>(ctx->part), ctx->spart, ctx->sout + 4,
                             ctx->counter + 1, done_ptr(ctx), ctx->derr, ctx->stream);
      }
      Prof pr(ctx, TLS_PROF_PCG_REDUCE);
      tls::launch_pcg_reduce<T>(static_cast<const T*>(ctx->part), ctx->PU, npad, v.q, v.w, v.y,
                                dinv_t<T>(ctx), ctx->sc, ctx->sout + 4, nr, ctx->stream);
    } else {
      Prof pr(ctx, TLS_PROF_PCG_REDUCE);
      tls::launch_pcg_update_R<T>(v.q, v.w, v.y, dinv_t<T>(ctx), ctx->sc, nr, npad, ctx->stream);
    }
    {
      Prof pr(ctx, TLS_PROF_PCG_GEMV);
      tls::launch_gemv_wt<T>(WT, npad, v.y, v.s, pcur, nullptr, ctx->gpart, ctx->sc, false,
                             modeA, nr, ctx->stream);
    }
  }
  TLS_CK_LAUNCH("pcgtls");
  return TLS_OK;
}

template <typename T>
tls_status precond_apply(tls_ctx* ctx, const double* y) {
  // q = R^{-1} R^{-T} y via one init step (s_0 = R^{-T} y) and one W product (beta = 0)
  UVecs<T> v = uvecs<T>(ctx);
  tls::launch_pcg_prep<T>(y, 1.0, nullptr, 1, ctx->n, ctx->npad, ctx->dinv, v.y, v.w, v.p0, v.p1,
                          ctx->sc, 0.0, 0.0, ctx->stream);
  tls::launch_gemv_wt<T>(static_cast<const T*>(ctx->WT), ctx->npad, v.y, v.s, nullptr, nullptr,
                         ctx->gpart, ctx->sc, true, true, 1, ctx->stream);
  tls::launch_gemv_w<T>(static_cast<const T*>(ctx->W), ctx->npad, v.s, v.p1, v.p0,
                        dinv_t<T>(ctx), v.q, ctx->gpart, ctx->sc, 1, ctx->stream);
  TLS_CK_LAUNCH("precond");
  return TLS_OK;
}

// A small dense problem in FP64 (n <= 64 and A, b, W and the vectors within one SM's shared
// memory) with the default PCGTLS schedule: the whole solve in one CTA (k_small.cu).
bool small_eligible(const tls_ctx* ctx) {
  const tls_options& o = ctx->opt;
  if (ctx->small_path == 3 || ctx->sparse || ctx->u != Prec::FP64 || ctx->n > 64 ||
      o.mode_A != 1 || o.cg_fixed == 0 || ctx->use_sel_tol)
    return false;
  const size_t one = tls::small_solve_smem((int)ctx->m, (int)ctx->n);
  const bool one_fits = one > 0 && one <= tls::kSmallSmemMax;
  const bool cluster_fits = tls::cluster_solve_fits((int)ctx->m, (int)ctx->n);
  if (ctx->small_path == 1) return one_fits;
  if (ctx->small_path == 2) return true;   // tls_solve reports when no cluster shape fits
  return one_fits || cluster_fits;
}

tls_status small_solve(tls_ctx* ctx, double tol, int max_rqi, tls_info* info, double* sigma_out,
                       bool* handled) {
  *handled = true;
  const tls_options& o = ctx->opt;
  cudaStream_t st = ctx->stream;
  TLS_CK(cudaEventRecord(ctx->ev0, st));
  tls::SmallParams prm{};
  prm.tol = tol;
  prm.psi_accept = o.psi_accept;
  prm.max_rqi = max_rqi;
  prm.ls_iters = std::max(1, o.ls_iters);
  prm.psi_rule_ge = o.psi_rule_ge;
  auto* dres = reinterpret_cast<tls::SmallResult*>(ctx->gpart);
  int cluster = 0;   // cluster size of the launch, 0 for the one-CTA solve
  {
    Prof pr(ctx, TLS_PROF_VEC);
    const double scale = ctx->norm2_A + ctx->norm2_b;
    const double* W = static_cast<const double*>(ctx->W);
    if (ctx->small_path != 1)
      cluster = tls::launch_cluster_solve(ctx->A64, ctx->npad, (int)ctx->m, (int)ctx->n, ctx->b,
                                          ctx->dinv, W, ctx->npad, scale, prm, ctx->x_best,
                                          dres, st);
    if (cluster == 0) {
      if (ctx->small_path == 2) {
        set_err(ctx, "no thread-block cluster shape fits this problem");
        return TLS_ERR_ARG;
      }
      if (!tls::launch_small_solve(ctx->A64, ctx->npad, (int)ctx->m, (int)ctx->n, ctx->b,
                                   ctx->dinv, W, ctx->npad, scale, prm, ctx->x_best, dres, st)) {
        *handled = false;   // neither fits (no cluster could be launched): multi-kernel path
        return TLS_OK;
      }
    }
  }
  TLS_CK_LAUNCH("small solve");
  tls::SmallResult r{};
  TLS_CK(cudaMemcpyAsync(&r, dres, sizeof(r), cudaMemcpyDeviceToHost, st));
  TLS_CK(cudaEventRecord(ctx->ev1, st));
  TLS_CK(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
  prof_collect(ctx);
  if (ctx->factor_time_pending) {
    float fms = 0.f;
    if (cudaEventElapsedTime(&fms, ctx->evf0, ctx->evf1) == cudaSuccess) ctx->t_factor_ms = fms;
    ctx->factor_time_pending = false;
  }
  *sigma_out = std::sqrt(std::max(r.sigma2, 0.0));
  ctx->last_sigma2 = r.sigma2;
  if (info) {
    info->stop_reason = r.stop;
    info->rqi_steps = r.rqi_steps;
    info->best_k = r.best_k;
    info->cg_iters = r.cg_iters;
    info->shifts = ctx->shifts;
    info->not_spd = r.not_spd;
    info->u_f_used = ctx->uf_used;
    info->psi_final = r.psi_final;
    info->sigma2 = r.sigma2;
    info->shift = ctx->shift;
    info->t_factor_ms = ctx->t_factor_ms;
    info->t_solve_ms = ms;
    info->fail_pivot = (int)ctx->fail_pivot;
    info->pass_variant[0] = cluster ? -2 : -1;   // no pass kernels: the one-launch solve
    info->pass_variant[1] = cluster ? cluster : 1;
    info->n_psi = r.n_psi;
    for (int i = 0; i < r.n_psi; ++i) info->psi_hist[i] = r.psi_hist[i];
    info->escalations = ctx->escalations;
    info->constr2_scaled = ctx->constr2_scaled;
    info->mode_switch_k = -1;
  }
  return TLS_OK;
}

template <typename T>
tls_status solve_impl(tls_ctx* ctx, double tol, int max_rqi, tls_info* info, double* sigma_out) {
  if constexpr (std::is_same<T, double>::value) {
    if (small_eligible(ctx)) {
      bool handled = true;
      const tls_status ss = small_solve(ctx, tol, max_rqi, info, sigma_out, &handled);
      if (handled) return ss;
    }
  }
  const tls_options& o = ctx->opt;
  // mode_A: 1 the A-explicit operator, 0 Alg. 3 as printed (operator R^T R), 2 the hybrid:
  // the printed form while psi falls fast, the A-explicit operator from the first RQI step on
  // whose psi is above hybrid_ratio times the previous one, or whose solves met delta_j <= 0
  const bool hybrid = o.mode_A == 2;
  bool modeA = o.mode_A == 1;
  int switch_k = hybrid ? 0 : -1;
  UVecs<T> v = uvecs<T>(ctx);
  cudaStream_t st = ctx->stream;
  TLS_CK(cudaEventRecord(ctx->ev0, st));
  // Alg. 2 line 1: LS start. Residual at x = 0 gives f = -A^T b; PCG with sigma^2 = 0.
  TLS_CK(cudaMemsetAsync(ctx->x, 0, sizeof(double) * ctx->npad, st));
  tls::launch_xx(ctx->x, ctx->rs, ctx->n, st, ctx->gpart + 2048);
  tls_status stt = residual_pass(ctx);
  if (stt != TLS_OK) return stt;
  stt = run_pcg<T>(ctx, 1, ctx->f, -1.0, nullptr, 0.0, std::max(1, o.ls_iters), 0.0, modeA);
  if (stt != TLS_OK) return stt;
  {
    Prof pr(ctx, TLS_PROF_VEC);
    tls::launch_copy_to_x<T>(ctx->x, v.w, ctx->rs, ctx->n, st, ctx->gpart + 2048);
  }
  // lines 2-5: r_0, sigma_0^2, u_0 = (R^T R)^{-1} x_0, x_1 = x_0 + sigma_0^2 u_0
  stt = residual_pass(ctx);
  if (stt != TLS_OK) return stt;
  stt = precond_apply<T>(ctx, ctx->x);
  if (stt != TLS_OK) return stt;
  {
    Prof pr(ctx, TLS_PROF_VEC);
    tls::launch_inverse_step<T>(ctx->x, v.q, ctx->rs, ctx->n, st, ctx->gpart + 2048);
  }
  TLS_CK_LAUNCH("inverse step");

  const double scale = ctx->norm2_A + ctx->norm2_b;
  double prev_psi = INFINITY;
  int stop = TLS_STOP_MAX_RQI;
  int best_k = 0, k = 0, cg_total = 0, not_spd = 0, last_steps = 0;
  bool continue_after_switch = false, save_best = false;
  double best_psi = INFINITY, best_s2 = 0.0;
  double psi_hist[24];
  int n_psi = 0;
  for (;;) {
    ++k;
    stt = residual_pass(ctx);
    if (stt != TLS_OK) return stt;
    TLS_CK(cudaMemcpyAsync(ctx->h_rs, ctx->rs, sizeof(RqiScalars), cudaMemcpyDeviceToHost, st));
    if (k > 1)
      TLS_CK(cudaMemcpyAsync(ctx->h_sc, ctx->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st));
    TLS_CK(cudaStreamSynchronize(st));
    if (k > 1) {
      if (ctx->prof_on && ctx->last_pcg_fused)
        ctx->prof_units[TLS_PROF_PCG_SOLVE2] += ctx->h_sc->passes;
      cg_total += ctx->h_sc->iters[0] + ctx->h_sc->iters[1];
      not_spd |= ctx->h_sc->not_spd[0] | ctx->h_sc->not_spd[1];
    }
    const double psi = ctx->h_rs->psi, s2 = ctx->h_rs->sigma2;
    if (n_psi < 24) psi_hist[n_psi++] = psi;
    if (!std::isfinite(psi) || !std::isfinite(s2)) {
      stop = TLS_STOP_PSI_UP;
      break;
    }
    // Sec. 3 after Eq. (4): stop when psi increases -- unless psi is still far above the
    // attainable level (psi_accept), where an increase is a transient of the inexact solves
    const bool up = o.psi_rule_ge ? (psi >= prev_psi) : (psi > prev_psi);
    if (up && best_psi <= o.psi_accept * scale) {
      stop = TLS_STOP_PSI_UP;
      break;
    }
    if (psi < best_psi) {
      best_k = k;
      best_psi = psi;
      best_s2 = s2;
      // x_k is copied to x_best after the next solves are queued (they only read x), so
      // the copy is not between the host's decision and the GPU's next launch
      save_best = true;
    }
    // the tolerance test from the second RQI step on: psi_1 is taken at the inverse-iteration
    // start x_1, whose error is only first order in psi_1
    if (!up && k >= 2 && psi <= tol * scale) {
      stop = TLS_STOP_TOL;
      break;
    }
    if (k > max_rqi) {
      stop = TLS_STOP_MAX_RQI;
      break;
    }
    // the hybrid's switch to the A-explicit operator (the printed form stopped paying)
    if (hybrid && !modeA && k > 1 &&
        (psi > o.hybrid_ratio * prev_psi || (ctx->h_sc->not_spd[0] | ctx->h_sc->not_spd[1]))) {
      modeA = true;
      switch_k = k;
      prev_psi = psi;
      continue_after_switch = true;
    }
    // the precision fallback before max_rqi: the last pair of PCGTLS solves stalled or lost
    // positive definiteness while psi is still above the attainable level
    if (k > 1 && !continue_after_switch && o.fallback && o.stall_fallback &&
        ctx->uf_used != TLS_FP64 && best_psi > o.psi_accept * scale) {
      const PcgScalars& h = *ctx->h_sc;
      const double rel = (h.eta0[0] > 0.0) ? std::sqrt(h.eta[0] / h.eta0[0]) : 0.0;
      int trig = TLS_TRIGGER_NONE;
      if (h.not_spd[0] | h.not_spd[1]) trig = TLS_TRIGGER_NOT_SPD;
      else if (o.cg_fixed && last_steps >= 3 && rel >= o.stall_ratio) trig = TLS_TRIGGER_STALL;
      else if (!o.cg_fixed && !h.done[0] && h.iters[0] >= last_steps) trig = TLS_TRIGGER_STALL;
      if (trig != TLS_TRIGGER_NONE) {
        ctx->stall_trigger = trig;
        stop = TLS_STOP_STALL;
        break;
      }
    }
    continue_after_switch = false;
    prev_psi = psi;
    // two shifted solves (Alg. 4, PCGTLS with k+1 steps) and the x update
    const int steps = o.cg_fixed ? (k + 1) : std::max(1, o.cg_max);
    last_steps = steps;
    const double cgt = ctx->use_sel_tol ? ctx->sel_cg_tol : o.cg_tol;
    stt = run_pcg<T>(ctx, 2, ctx->f, -1.0, ctx->x, s2, steps, o.cg_fixed ? 0.0 : cgt, modeA);
    if (stt != TLS_OK) return stt;
    if (save_best) {
      TLS_CK(cudaMemcpyAsync(ctx->x_best, ctx->x, sizeof(double) * ctx->npad,
                             cudaMemcpyDeviceToDevice, st));
      save_best = false;
    }
    {
      Prof pr(ctx, TLS_PROF_VEC);
      tls::launch_rqi_update<T>(ctx->x, v.w, v.w + ctx->npad, ctx->f, ctx->rs, ctx->n, st,
                                ctx->gpart + 2048);
    }
    TLS_CK_LAUNCH("rqi update");
  }
  if (save_best)
    TLS_CK(cudaMemcpyAsync(ctx->x_best, ctx->x, sizeof(double) * ctx->npad,
                           cudaMemcpyDeviceToDevice, st));
  TLS_CK(cudaEventRecord(ctx->ev1, st));
  int herr = 0;
  TLS_CK(cudaMemcpyAsync(&herr, ctx->derr, sizeof(int), cudaMemcpyDeviceToHost, st));
  TLS_CK(cudaEventSynchronize(ctx->ev1));
  TLS_CK(cudaStreamSynchronize(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
  prof_collect(ctx);
  if (ctx->factor_time_pending) {
    float fms = 0.f;
    if (cudaEventElapsedTime(&fms, ctx->evf0, ctx->evf1) == cudaSuccess) ctx->t_factor_ms = fms;
    ctx->factor_time_pending = false;
  }
  if (herr != 0) {
    TLS_CK(cudaMemsetAsync(ctx->derr, 0, sizeof(int), st));
    TLS_CK(cudaMemsetAsync(ctx->fbar, 0, kBarWords * sizeof(unsigned int), st));
    set_err(ctx, "a bounded device wait expired (code " + std::to_string(herr) + ")");
    return TLS_ERR_TIMEOUT;
  }
  *sigma_out = std::sqrt(std::max(best_s2, 0.0));
  ctx->last_sigma2 = best_s2;
  if (info) {
    info->stop_reason = stop;
    info->rqi_steps = k;
    info->best_k = best_k;
    info->cg_iters = cg_total;
    info->shifts = ctx->shifts;
    info->not_spd = not_spd;
    info->u_f_used = ctx->uf_used;
    info->psi_final = best_psi;
    info->sigma2 = best_s2;
    info->shift = ctx->shift;
    info->t_factor_ms = ctx->t_factor_ms;
    info->t_solve_ms = ms;
    info->fail_pivot = (int)ctx->fail_pivot;
    info->pass_variant[0] = resid_df_active(ctx) ? 4 : ctx->plan64.variant;
    info->pass_variant[1] = ctx->planU.variant;
    info->n_psi = n_psi;
    for (int i = 0; i < n_psi; ++i) info->psi_hist[i] = psi_hist[i];
    info->escalations = ctx->escalations;
    info->constr2_scaled = ctx->constr2_scaled;
    info->mode_switch_k = switch_k;
  }
  return TLS_OK;
}

// ---------------------------------------------------------------------------------------
// Factorisation ladder
// ---------------------------------------------------------------------------------------
Prec to_prec(tls_prec p) { return static_cast<Prec>((int)p); }

// ---------------------------------------------------------------------------------------
// Autotuner for the fused pass over A: each variant (register kernel; bulk-copy-staged with 256
// or 512 threads; pipelined register kernel) is timed on the context's own matrix (one warm-up and three launches, CUDA
// events) and the fastest is cached per (type, right-hand sides, m, n_pad) for the process.
// ---------------------------------------------------------------------------------------
std::map<std::tuple<int, int, int, int64_t, int64_t, int>, int> g_tune;
std::mutex g_tune_mu;

template <typename T>
tls::ApassPlan tune_apass(tls_ctx* ctx, const T* A, int nr, bool resid, const T* v,
                          const double* b, T* part, double* sout, unsigned int* counter) {
  const auto key = std::make_tuple((int)sizeof(T), nr, resid ? 1 : 0, ctx->m, ctx->npad,
                                   ctx->device);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end())
      return tls::plan_apass<T>(ctx->m, ctx->npad, nr, ctx->num_sms, it->second);
  }
  int best_v = 1;
  float best_ms = 1e30f;
  for (int var = 0; var < tls::kApassVariants; ++var) {
    tls::ApassPlan pl = tls::plan_apass<T>(ctx->m, ctx->npad, nr, ctx->num_sms, var);
    if ((var == 1 || var == 2) && !pl.tma) continue;   // staging does not fit: not a candidate
    auto go = [&]() {
      tls::launch_apass<T>(pl, A, ctx->npad, ctx->m, ctx->npad, nr, resid, v, ctx->npad, b, part,
                           ctx->spart, sout, counter, nullptr, ctx->derr, ctx->stream);
    };
    go();
    cudaEventRecord(ctx->ev0, ctx->stream);
    for (int r = 0; r < 3; ++r) go();
    cudaEventRecord(ctx->ev1, ctx->stream);
    if (cudaEventSynchronize(ctx->ev1) != cudaSuccess) {
      (void)cudaGetLastError();
      continue;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    if (ms < best_ms) {
      best_ms = ms;
      best_v = var;
    }
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best_v;
  }
  return tls::plan_apass<T>(ctx->m, ctx->npad, nr, ctx->num_sms, best_v);
}

void tune_passes(tls_ctx* ctx) {
  // the FP64 residual pass (1 RHS) and the PCGTLS pass (2 RHS) in the u type
  ctx->plan64 = tune_apass<double>(ctx, ctx->A64, 1, true, ctx->x, ctx->b, ctx->part64, ctx->sout,
                                   ctx->counter);
  ctx->P64 = ctx->plan64.grid;
  if (ctx->u == Prec::FP64) {
    ctx->planU = tune_apass<double>(ctx, ctx->A64, 2, false, static_cast<double*>(ctx->vbuf),
                                    nullptr, static_cast<double*>(ctx->part), ctx->sout + 4,
                                    ctx->counter + 1);
  } else {
    ctx->planU = tune_apass<float>(ctx, ctx->A32, 2, false, static_cast<float*>(ctx->vbuf),
                                   nullptr, static_cast<float*>(ctx->part), ctx->sout + 4,
                                   ctx->counter + 1);
  }
  ctx->PU = ctx->planU.grid;
}

tls_status ensure_solve_buffers(tls_ctx* ctx) {
  const int64_t npad = ctx->npad;
  const size_t us = u_size(ctx->u);
  ctx->vbuf = slot(ctx, kSlotVbuf, us * 12 * (size_t)npad);
  if (ctx->u == Prec::FP64) ctx->planU = tls::plan_apass<double>(ctx->m, npad, 2, ctx->num_sms, 1);
  else ctx->planU = tls::plan_apass<float>(ctx->m, npad, 2, ctx->num_sms, 1);
  ctx->PU = ctx->planU.grid;
  ctx->part = slot(ctx, kSlotPart, us * (size_t)2 * ctx->num_sms * 2 * (size_t)npad);
  if (!ctx->vbuf || !ctx->part) {
    set_err(ctx, "device allocation failed (solve buffers)");
    return TLS_ERR_OOM;
  }
  TLS_CK(cudaMemsetAsync(ctx->vbuf, 0, us * 12 * (size_t)npad, ctx->stream));
  if (ctx->sparse) {
    ctx->tbuf = slot(ctx, kSlotTbuf, us * 2 * (size_t)ctx->m);
    if (!ctx->tbuf) {
      set_err(ctx, "device allocation failed (sparse solve buffers)");
      return TLS_ERR_OOM;
    }
  } else {
    tune_passes(ctx);
  }
  TLS_CK(cudaMemsetAsync(ctx->derr, 0, sizeof(int), ctx->stream));
  return TLS_OK;
}

// 1 / (sqrt(n) ||W||_F) with W = R_H^{-1} of the current factor (in the u type): constraint 2
// of the column-scaled matrix with sigma_{n+1} = 0. Synchronises the stream.
tls_status scaled_constraint2(tls_ctx* ctx, double* out) {
  cudaStream_t st = ctx->stream;
  int g;
  if (ctx->u == Prec::FP64)
    g = tls::launch_frob_dw<double>(static_cast<const double*>(ctx->W), ctx->n, ctx->npad,
                                    nullptr, ctx->gpart, st);
  else
    g = tls::launch_frob_dw<float>(static_cast<const float*>(ctx->W), ctx->n, ctx->npad,
                                   nullptr, ctx->gpart, st);
  TLS_CK_LAUNCH("scaled constraint");
  std::vector<double> h((size_t)g);
  TLS_CK(cudaMemcpyAsync(h.data(), ctx->gpart, sizeof(double) * g, cudaMemcpyDeviceToHost, st));
  TLS_CK(cudaStreamSynchronize(st));
  double frob = 0.0;
  for (double v : h) frob += v;
  *out = (frob > 0.0) ? 1.0 / (std::sqrt((double)ctx->n) * std::sqrt(frob)) : 0.0;
  return TLS_OK;
}

tls_status factor_impl(tls_ctx* ctx, tls_prec uf_req) {
  cudaStream_t st = ctx->stream;
  ctx->resid_df = true;
  const int64_t m = ctx->m, n = ctx->n, npad = ctx->npad, mpad = ctx->mpad;
  TLS_CK(cudaEventRecord(ctx->evf0, st));
  ctx->factored = false;
  if (!ctx->sparse && ctx->u == Prec::FP32 && ctx->A32 == nullptr) {
    ctx->A32 = alloc_t<float>(ctx, m * npad);
    ctx->Alo = alloc_t<float>(ctx, m * npad);
    if (!ctx->A32 || !ctx->Alo) {
      set_err(ctx, "device allocation failed (FP32 copy of A)");
      return TLS_ERR_OOM;
    }
  }
  // column scaling D (Sec. 3.1); the FP32 copy of A for u = FP32 is written in the same pass
  double* cpart = static_cast<double*>(slot(ctx, kSlotCpart, sizeof(double) * 64 * npad));
  RqiScalars* dnorm = static_cast<RqiScalars*>(slot(ctx, kSlotNorm, 2 * sizeof(RqiScalars)));
  if (!cpart || !dnorm) {
    set_err(ctx, "device allocation failed");
    return TLS_ERR_OOM;
  }
  // (the completion counters of the norm kernels below start at zero)
  TLS_CK(cudaMemsetAsync(dnorm, 0, 2 * sizeof(RqiScalars), st));
  const bool want32 = ctx->u == Prec::FP32;
  if (!ctx->colnorm_done || (want32 && !ctx->a32_done)) {
    Prof pr(ctx, TLS_PROF_SCALE);
    if (ctx->sparse)
      tls::sparse_colnorm(ctx->cp, ctx->cv64, want32 ? ctx->cv32 : nullptr, n, npad, ctx->d,
                          ctx->dinv, ctx->dinv32, st);
    else
      tls::launch_colnorm(ctx->A64, npad, m, n, npad, want32 ? ctx->A32 : nullptr, ctx->Alo,
                          npad, ctx->d, ctx->dinv32, ctx->dinv, cpart, st);
    TLS_CK_LAUNCH("column norms");
    ctx->colnorm_done = true;
    ctx->a32_done = ctx->a32_done || want32;
  }
  // ||A||_F^2 = sum of d_j^2 and ||b||^2 on the device; read back with the factor's first
  // synchronisation (no extra host round trip)
  TLS_CK(cudaMemsetAsync(ctx->x, 0, sizeof(double) * npad, st));
  tls::launch_xx(ctx->d, dnorm, n, st, ctx->gpart + 2048);
  tls::launch_xx(ctx->b, dnorm + 1, m, st, ctx->gpart + 2048);
  TLS_CK(cudaMemcpyAsync(ctx->h_norm, dnorm, 2 * sizeof(RqiScalars), cudaMemcpyDeviceToHost, st));
  bool norms_read = false;
  auto read_norms = [&]() {
    if (norms_read) return;
    norms_read = true;
    ctx->norm2_A = ctx->h_norm[0].xx;
    ctx->norm2_b = ctx->h_norm[1].xx;
  };

  // the ladder of factor precisions (Sec. 3.1 constraints, escalation on breakdown)
  std::vector<tls_prec> ladder;
  ladder.push_back(uf_req);
  if (uf_req == TLS_FP16 || uf_req == TLS_BF16) ladder.push_back(TLS_FP32);
  if (uf_req != TLS_FP64) ladder.push_back(TLS_FP64);
  int* dinfo = static_cast<int*>(slot(ctx, kSlotInfo, sizeof(int)));
  if (!dinfo) return TLS_ERR_OOM;
  ctx->shifts = 0;
  ctx->shift = 0.0;
  ctx->fail_pivot = -1;
  ctx->escalations = 0;
  ctx->constr2_scaled = NAN;
  bool ok = false;
  const bool qr = (ctx->opt.factor == 1) && !ctx->sparse;
  for (tls_prec uf : ladder) {
    const Prec pf = to_prec(uf);
    const bool chol64 = (pf == Prec::FP64);
    const size_t ce = chol64 ? 8 : 4;
    const bool from64 = (ctx->u != Prec::FP32) || (pf == Prec::FP64);
    // unit roundoff of the factor precision (Table 2; bf16: 2^-8)
    const double uf_round = (pf == Prec::FP16) ? std::ldexp(1.0, -11)
                            : (pf == Prec::BF16) ? std::ldexp(1.0, -8)
                            : (pf == Prec::FP32) ? std::ldexp(1.0, -24) : std::ldexp(1.0, -53);
    const bool low = (pf == Prec::FP16 || pf == Prec::BF16);
    void* Wc = nullptr;
    void* M = nullptr;
    if (qr) {
      // Alg. 4: R-hat from the Householder QR of A D^{-1} rounded to u_q (the same column
      // scaling as the Cholesky route, so R-hat plays the part of R_H); no Gram matrix
      ctx->H = nullptr;
      M = slot(ctx, kSlotM, ce * (size_t)npad * (size_t)npad);
      void* Aq = slot(ctx, kSlotQR, ce * (size_t)m * (size_t)npad);
      const size_t qwe = (size_t)npad + (chol64 ? tls::qr_work_elems<double>(m, n, ctx->num_sms)
                                                : tls::qr_work_elems<float>(m, n, ctx->num_sms));
      void* qw = slot(ctx, kSlotQRwork, ce * qwe);
      if (!M || !Aq || !qw) {
        set_err(ctx, "device allocation failed (QR workspace)");
        return TLS_ERR_OOM;
      }
      TLS_CK(cudaMemsetAsync(dinfo, 0, sizeof(int), st));
      const void* src = from64 ? (const void*)ctx->A64 : (const void*)ctx->A32;
      {
        Prof pr(ctx, TLS_PROF_SCALE);
        if (chol64)
          tls::launch_qr_scale<double>(src, from64, npad, m, n, ctx->dinv, ctx->dinv32, pf,
                                       static_cast<double*>(Aq), npad, st);
        else
          tls::launch_qr_scale<float>(src, from64, npad, m, n, ctx->dinv, ctx->dinv32, pf,
                                      static_cast<float*>(Aq), npad, st);
      }
      int qrc;
      {
        Prof pr(ctx, TLS_PROF_CHOL);
        if (chol64) {
          double* q = static_cast<double*>(qw);
          qrc = tls::launch_qr_r<double>(static_cast<double*>(Aq), npad, m, n, q, q + npad, dinfo,
                                         ctx->num_sms, st);
          if (qrc == 0)
            tls::launch_qr_extract<double, double>(static_cast<double*>(Aq), npad, n, npad,
                                                   static_cast<double*>(M), st);
        } else {
          float* q = static_cast<float*>(qw);
          qrc = tls::launch_qr_r<float>(static_cast<float*>(Aq), npad, m, n, q, q + npad, dinfo,
                                        ctx->num_sms, st);
          if (qrc == 0)
            tls::launch_qr_extract<float, float>(static_cast<float*>(Aq), npad, n, npad,
                                                 static_cast<float*>(M), st);
        }
      }
      if (qrc != 0) {
        set_err(ctx, qrc == -3 ? "Householder QR: the panel kernel's cluster launch failed"
                               : "Householder QR: m too large for the panel kernel (rows of a "
                                 "panel are held in the shared memory of one 16-CTA cluster)");
        return TLS_ERR_ARG;
      }
      TLS_CK_LAUNCH("householder qr");
      int hinfo = 0;
      TLS_CK(cudaMemcpyAsync(&hinfo, dinfo, sizeof(int), cudaMemcpyDeviceToHost, st));
      TLS_CK(cudaStreamSynchronize(st));
      read_norms();
      if (hinfo != 0) {
        // a zero (or non-finite) diagonal entry of R-hat: rank deficient in u_q, escalate
        ctx->fail_pivot = hinfo - 1;
        continue;
      }
      ok = true;
    } else {
    const size_t ae = (pf == Prec::FP64) ? 8 : (pf == Prec::FP32 ? 4 : 2);
    // dense: the scaled, rounded, transposed A_s; sparse: its values in CSR and CSC order
    void* AsT = ctx->sparse
                    ? slot(ctx, kSlotAsT, 2 * ce * (size_t)std::max<int64_t>(ctx->nnz, 1))
                    : slot(ctx, kSlotAsT, ae * (size_t)npad * (size_t)mpad);
    ctx->H = slot(ctx, kSlotH, ce * (size_t)npad * (size_t)npad);
    M = slot(ctx, kSlotM, ce * (size_t)npad * (size_t)npad);
    if (!AsT || !ctx->H || !M) {
      set_err(ctx, "device allocation failed (factor workspace)");
      return TLS_ERR_OOM;
    }
    if (ctx->sparse) {
      Prof pr(ctx, TLS_PROF_GRAM);
      const int64_t nz = std::max<int64_t>(ctx->nnz, 1);
      if (chol64)
        tls::sparse_gram<double>(ctx->rp, ctx->ci, ctx->v32, ctx->v64, ctx->cp, ctx->ri, ctx->cv32,
                                 ctx->cv64, ctx->dinv32, ctx->dinv, n, npad, ctx->nnz, pf,
                                 static_cast<double*>(AsT), static_cast<double*>(AsT) + nz,
                                 static_cast<double*>(ctx->H), st);
      else
        tls::sparse_gram<float>(ctx->rp, ctx->ci, ctx->v32, ctx->v64, ctx->cp, ctx->ri, ctx->cv32,
                                ctx->cv64, ctx->dinv32, ctx->dinv, n, npad, ctx->nnz, pf,
                                static_cast<float*>(AsT), static_cast<float*>(AsT) + nz,
                                static_cast<float*>(ctx->H), st);
      ctx->gram_tc_used = false;
    } else {
    {
      Prof pr(ctx, TLS_PROF_SCALE);
      tls::launch_scale_cast_T(from64 ? (const void*)ctx->A64 : (const void*)ctx->A32, from64,
                               npad, m, n, npad, mpad, ctx->dinv, ctx->dinv32, AsT, pf, st);
    }
    {
      Prof pr(ctx, TLS_PROF_GRAM);
      bool tc = false;
      if ((pf == Prec::FP16 || pf == Prec::BF16) && !ctx->opt.gram_simt) {
        // (the partial sums use the buffer of the preconditioner matrix's split products,
        // free until the inverse)
        float* gpart = static_cast<float*>(
            slot(ctx, kSlotPMpart, sizeof(float) * 3 * (size_t)npad * (size_t)npad));
        tc = tls::launch_gram_tc(AsT, pf, n, npad, mpad, static_cast<float*>(ctx->H), ctx->derr,
                                 st, gpart);
      }
      if (tc) {
        const int terr = tls::gram_tc_error(ctx->derr, st);   // synchronises the stream
        if (terr != 0) {
          // a bounded wait in the tensor-core kernel gave up: recompute on CUDA cores
          set_err(ctx, "tensor-core Gram wait expired (code " + std::to_string(terr) +
                           "); recomputed on CUDA cores");
          tc = false;
        }
      }
      if (!tc) {
        void* gw = nullptr;
        const int chunks = tls::gram_split_chunks(npad, mpad, ctx->num_sms);
        if (pf == Prec::FP64 && chunks > 1)
          gw = slot(ctx, kSlotGsplit, sizeof(double) * (size_t)chunks * npad * npad);
        tls::launch_gram_simt(AsT, pf, n, npad, mpad, ctx->H, st, gw, gw ? chunks : 1);
      }
      ctx->gram_tc_used = tc;
    }
    }
    TLS_CK_LAUNCH("gram");
    Wc = slot(ctx, kSlotWc, ce * (size_t)npad * (size_t)npad);   // diagonal-block inverses
    if (!Wc) {
      set_err(ctx, "device allocation failed (factor workspace)");
      return TLS_ERR_OOM;
    }
    const int max_shift = std::max(0, ctx->opt.max_shifts);
    const int first = (low && ctx->opt.shift_first) ? 1 : 0;
    for (int sh = first; sh <= max_shift + first; ++sh) {
      const double shift = (sh == 0) ? 0.0 : 2.0 * uf_round * std::pow(4.0, sh - 1);
      TLS_CK(cudaMemcpyAsync(M, ctx->H, ce * (size_t)npad * (size_t)npad,
                             cudaMemcpyDeviceToDevice, st));
      TLS_CK(cudaMemsetAsync(Wc, 0, ce * (size_t)npad * (size_t)npad, st));
      TLS_CK(cudaMemsetAsync(dinfo, 0, sizeof(int), st));
      {
        Prof pr(ctx, TLS_PROF_CHOL);
        if (chol64)
          tls::launch_cholesky<double>(static_cast<double*>(M), n, npad, shift, dinfo,
                                       static_cast<double*>(Wc), pf, st);
        else
          tls::launch_cholesky<float>(static_cast<float*>(M), n, npad, shift, dinfo,
                                      static_cast<float*>(Wc), pf, st,
                                      ctx->chol_chain ? ctx->fbar + 128 : nullptr, ctx->derr,
                                      ctx->num_sms, ctx->trace_on ? ctx->trace : nullptr,
                                      ctx->chol_chain,
                                      ctx->chol_tc ? slot(ctx, kSlotPT, 2 * 64 * (size_t)npad)
                                                   : nullptr);
      }
      TLS_CK_LAUNCH("cholesky");
      int hinfo = 0, herr = 0;
      TLS_CK(cudaMemcpyAsync(&hinfo, dinfo, sizeof(int), cudaMemcpyDeviceToHost, st));
      TLS_CK(cudaMemcpyAsync(&herr, ctx->derr, sizeof(int), cudaMemcpyDeviceToHost, st));
      TLS_CK(cudaStreamSynchronize(st));
      if (herr != 0) {
        TLS_CK(cudaMemsetAsync(ctx->derr, 0, sizeof(int), st));
        TLS_CK(cudaMemsetAsync(ctx->fbar, 0, kBarWords * sizeof(unsigned int), st));
        set_err(ctx, "a bounded device wait expired in the factor (code " +
                         std::to_string(herr) + ")");
        return TLS_ERR_TIMEOUT;
      }
      read_norms();
      if (hinfo == 0) {
        ok = true;
        ctx->shift = shift;
        break;
      }
      ctx->shifts += 1;
      ctx->fail_pivot = hinfo - 1;
    }
    }   // Cholesky route
    if (!ok) continue;
    // R_H rounded to u_f (the computed factor R-hat), then carried in the u type
    if (chol64) tls::launch_round_to<double>(static_cast<double*>(M), npad, pf, st);
    else tls::launch_round_to<float>(static_cast<float*>(M), npad, pf, st);
    const size_t us = u_size(ctx->u);
    ctx->R = slot(ctx, kSlotR, us * (size_t)npad * (size_t)npad);
    ctx->W = slot(ctx, kSlotW, us * (size_t)npad * (size_t)npad);
    ctx->WT = slot(ctx, kSlotWT, us * (size_t)npad * (size_t)npad);
    ctx->pm_ready = false;
    void* work = slot(ctx, kSlotWork, us * (size_t)npad * (size_t)npad);
    if (!ctx->R || !ctx->W || !ctx->WT || !work) {
      set_err(ctx, "device allocation failed (inverse factor)");
      return TLS_ERR_OOM;
    }
    const int64_t cnt = npad * npad;
    Prof pr(ctx, TLS_PROF_TRTRI);
    // (the Cholesky route has the inverses of R-hat's 64 x 64 diagonal blocks in Wc already;
    // the QR route leaves them to the triangular inverse)
    const bool have_diag = (Wc != nullptr);
    if (ctx->u == Prec::FP64) {
      if (chol64) {
        TLS_CK(cudaMemcpyAsync(ctx->R, M, 8 * cnt, cudaMemcpyDeviceToDevice, st));
        if (have_diag) TLS_CK(cudaMemcpyAsync(ctx->W, Wc, 8 * cnt, cudaMemcpyDeviceToDevice, st));
      } else {
        tls::launch_f2d(static_cast<float*>(M), static_cast<double*>(ctx->R), cnt, st);
        if (have_diag) tls::launch_f2d(static_cast<float*>(Wc), static_cast<double*>(ctx->W), cnt, st);
      }
      tls::launch_trtri<double>(static_cast<double*>(ctx->R), static_cast<double*>(ctx->W),
                                static_cast<double*>(ctx->WT), static_cast<double*>(work), npad,
                                have_diag, st);
    } else {
      if (chol64) {
        tls::launch_d2f(static_cast<double*>(M), static_cast<float*>(ctx->R), cnt, st);
        if (have_diag) tls::launch_d2f(static_cast<double*>(Wc), static_cast<float*>(ctx->W), cnt, st);
      } else {
        TLS_CK(cudaMemcpyAsync(ctx->R, M, 4 * cnt, cudaMemcpyDeviceToDevice, st));
        if (have_diag) TLS_CK(cudaMemcpyAsync(ctx->W, Wc, 4 * cnt, cudaMemcpyDeviceToDevice, st));
      }
      float* tpart = static_cast<float*>(
          slot(ctx, kSlotPMpart, sizeof(float) * 3 * (size_t)npad * (size_t)npad));
      tls::launch_trtri<float>(static_cast<float*>(ctx->R), static_cast<float*>(ctx->W),
                               static_cast<float*>(ctx->WT), static_cast<float*>(work), npad,
                               have_diag, st, tpart);
    }
    TLS_CK_LAUNCH("triangular inverse");
    ctx->uf_used = uf;
    ctx->H_fp64 = chol64;
    if (low && ctx->opt.constr_guard > 0.0 && uf != ladder.back()) {
      // constraint 2 (Eq. (9), Sec. 3.1) of the column-scaled matrix A D^{-1} the factor is
      // built from: kappa_F(A D^{-1}) = ||A D^{-1}||_F ||R_H^{-1}||_F = sqrt(n) ||W||_F (unit
      // columns), with sigma_{n+1} = 0 before the solve
      const tls_status gs = scaled_constraint2(ctx, &ctx->constr2_scaled);
      if (gs != TLS_OK) return gs;
      if (uf_round > ctx->opt.constr_guard * ctx->constr2_scaled) {
        ctx->escalations += 1;
        ok = false;
        continue;
      }
    }
    break;
  }
  if (!ok) {
    set_err(ctx, qr ? "Householder QR: a zero diagonal entry of R at every precision"
                    : "Cholesky breakdown at every shift and precision");
    return TLS_ERR_FACTOR_BREAKDOWN;
  }
  tls_status s2 = ensure_solve_buffers(ctx);
  if (s2 != TLS_OK) return s2;
  // the triangular inverse may still run: the next call on the stream orders after it, and
  // the factor's device time is read once it is known to be complete
  TLS_CK(cudaEventRecord(ctx->evf1, st));
  ctx->factor_time_pending = true;
  if (ctx->prof_on) {
    TLS_CK(cudaEventSynchronize(ctx->evf1));
    prof_collect(ctx);
  }
  ctx->factored = true;
  return TLS_OK;
}

template <typename T>
static tls_status pcgtls_host(tls_ctx* ctx, int nr, double sigma2, const double* f0,
                              const double* f1, int steps, double cg_tol, double* w0, double* w1,
                              int* iters, int* not_spd) {
  cudaStream_t st = ctx->stream;
  const int64_t n = ctx->n, npad = ctx->npad;
  // stage the right-hand sides in f (RHS 0) and x_best (RHS 1) of the context
  TLS_CK(cudaMemsetAsync(ctx->f, 0, sizeof(double) * npad, st));
  TLS_CK(cudaMemcpyAsync(ctx->f, f0, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  if (nr > 1) {
    TLS_CK(cudaMemsetAsync(ctx->x_best, 0, sizeof(double) * npad, st));
    TLS_CK(cudaMemcpyAsync(ctx->x_best, f1, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  }
  tls_status s = run_pcg<T>(ctx, nr, ctx->f, 1.0, ctx->x_best, sigma2, steps, cg_tol,
                            ctx->opt.mode_A != 0);
  if (s != TLS_OK) return s;
  UVecs<T> v = uvecs<T>(ctx);
  std::vector<T> hw((size_t)2 * npad);
  int herr = 0;
  TLS_CK(cudaMemcpyAsync(hw.data(), v.w, sizeof(T) * 2 * npad, cudaMemcpyDeviceToHost, st));
  TLS_CK(cudaMemcpyAsync(ctx->h_sc, ctx->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st));
  TLS_CK(cudaMemcpyAsync(&herr, ctx->derr, sizeof(int), cudaMemcpyDeviceToHost, st));
  TLS_CK(cudaStreamSynchronize(st));
  prof_collect(ctx);
  if (herr != 0) {
    TLS_CK(cudaMemsetAsync(ctx->derr, 0, sizeof(int), st));
    TLS_CK(cudaMemsetAsync(ctx->fbar, 0, kBarWords * sizeof(unsigned int), st));
    set_err(ctx, "a bounded device wait expired (code " + std::to_string(herr) + ")");
    return TLS_ERR_TIMEOUT;
  }
  for (int64_t j = 0; j < n; ++j) {
    w0[j] = (double)hw[j];
    if (nr > 1 && w1) w1[j] = (double)hw[npad + j];
  }
  if (iters) { iters[0] = ctx->h_sc->iters[0]; iters[1] = ctx->h_sc->iters[1]; }
  if (not_spd) { not_spd[0] = ctx->h_sc->not_spd[0]; not_spd[1] = ctx->h_sc->not_spd[1]; }
  return TLS_OK;
}

template <typename T>
static tls_status precond_host(tls_ctx* ctx, const double* y, double* s0, double* u) {
  cudaStream_t st = ctx->stream;
  const int64_t n = ctx->n, npad = ctx->npad;
  TLS_CK(cudaMemsetAsync(ctx->f, 0, sizeof(double) * npad, st));
  TLS_CK(cudaMemcpyAsync(ctx->f, y, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  tls_status s = precond_apply<T>(ctx, ctx->f);
  if (s != TLS_OK) return s;
  UVecs<T> v = uvecs<T>(ctx);
  std::vector<T> hs(npad), hq(npad);
  TLS_CK(cudaMemcpyAsync(hs.data(), v.s, sizeof(T) * npad, cudaMemcpyDeviceToHost, st));
  TLS_CK(cudaMemcpyAsync(hq.data(), v.q, sizeof(T) * npad, cudaMemcpyDeviceToHost, st));
  TLS_CK(cudaStreamSynchronize(st));
  for (int64_t j = 0; j < n; ++j) {
    if (s0) s0[j] = (double)hs[j];
    if (u) u[j] = (double)hq[j];
  }
  return TLS_OK;
}

template <typename T>
static tls_status precond_trsv_host(tls_ctx* ctx, const double* y, double* s0, double* u) {
  cudaStream_t st = ctx->stream;
  const int64_t n = ctx->n, npad = ctx->npad;
  TLS_CK(cudaMemsetAsync(ctx->f, 0, sizeof(double) * npad, st));
  TLS_CK(cudaMemcpyAsync(ctx->f, y, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  UVecs<T> v = uvecs<T>(ctx);
  const T* dinvT = reinterpret_cast<const T*>(sizeof(T) == 4 ? (const void*)ctx->dinv32
                                                             : (const void*)ctx->dinv);
  if (!tls::launch_trsv<T>(static_cast<const T*>(ctx->R), npad, n, dinvT, ctx->f, v.s, v.q, st)) {
    set_err(ctx, "triangular solve: n too large for one CTA's shared memory");
    return TLS_ERR_ARG;
  }
  std::vector<T> hs(npad), hq(npad);
  TLS_CK(cudaMemcpyAsync(hs.data(), v.s, sizeof(T) * npad, cudaMemcpyDeviceToHost, st));
  TLS_CK(cudaMemcpyAsync(hq.data(), v.q, sizeof(T) * npad, cudaMemcpyDeviceToHost, st));
  TLS_CK(cudaStreamSynchronize(st));
  for (int64_t j = 0; j < n; ++j) {
    if (s0) s0[j] = (double)hs[j];
    if (u) u[j] = (double)hq[j];
  }
  return TLS_OK;
}

template <typename TH, typename TU>
static tls_status condition_impl(tls_ctx* ctx, int iters, double* out) {
  cudaStream_t st = ctx->stream;
  const int64_t n = ctx->n, npad = ctx->npad;
  void* scratch = slot(ctx, kSlotCond, sizeof(double) * (size_t)(4 * npad + 2 + 4096));
  if (!scratch) return TLS_ERR_OOM;
  TH* xh = static_cast<TH*>(scratch);
  TH* yh = xh + npad;
  TU* xu = reinterpret_cast<TU*>(static_cast<double*>(scratch) + 2 * npad);
  double* lam = static_cast<double*>(scratch) + 4 * npad;
  double* part = lam + 2;
  const TH* dinvH = reinterpret_cast<const TH*>(sizeof(TH) == 4 ? (const void*)ctx->dinv32
                                                                : (const void*)ctx->dinv);
  // sigma'_1^2 = lambda_max(D H D)
  tls::launch_power_init<TH>(xh, n, npad, st);
  for (int it = 0; it < iters; ++it) {
    tls::launch_dhd<TH>(static_cast<const TH*>(ctx->H), npad, dinvH, xh, yh, st);
    tls::launch_power_finish<TH>(xh, yh, n, lam, st);
  }
  // 1 / sigma'_n^2 = lambda_max((R^T R)^{-1}) with the preconditioner products
  UVecs<TU> v = uvecs<TU>(ctx);
  tls::launch_power_init<TU>(xu, n, npad, st);
  for (int it = 0; it < iters; ++it) {
    tls::launch_vec_to_double<TU>(xu, ctx->f, n, npad, st);
    tls_status s2 = precond_apply<TU>(ctx, ctx->f);
    if (s2 != TLS_OK) return s2;
    tls::launch_power_finish<TU>(xu, v.q, n, lam + 1, st);
  }
  const int g = tls::launch_frob_dw<TU>(static_cast<const TU*>(ctx->W), n, npad, dinv_t<TU>(ctx),
                                        part, st);
  TLS_CK_LAUNCH("condition estimate");
  std::vector<double> h(2 + (size_t)g);
  TLS_CK(cudaMemcpyAsync(h.data(), lam, sizeof(double) * (2 + g), cudaMemcpyDeviceToHost, st));
  TLS_CK(cudaStreamSynchronize(st));

  double frob = 0.0;
  for (int i = 0; i < g; ++i) frob += h[2 + i];
  const double s1 = std::sqrt(std::max(h[0], 0.0));
  const double sn = (h[1] > 0.0) ? 1.0 / std::sqrt(h[1]) : 0.0;
  const double fa = std::sqrt(ctx->norm2_A), fi = std::sqrt(frob);
  const double kappa = (sn > 0.0) ? s1 / sn : INFINITY;
  const double kf = fa * fi;
  const double sig = ctx->last_sigma2 >= 0.0 ? std::sqrt(ctx->last_sigma2) : NAN;
  out[0] = s1;
  out[1] = sn;
  out[2] = kappa;
  out[3] = fa;
  out[4] = fi;
  out[5] = kf;
  out[6] = sig;
  out[7] = 1.0 / kappa;
  out[8] = (1.0 - (sig * sig) / (sn * sn)) / kf;
  return TLS_OK;
}

}  // namespace

// =========================================================================================
namespace {

// Runs fn(i) for i < count on up to `workers` host threads (each context has its own CUDA
// stream, so the kernels of different problems overlap on the GPU).
template <typename F>
void run_workers(int count, int workers, F fn) {
  workers = std::max(1, std::min(workers, count));
  std::atomic<int> next{0};
  int dev = 0;
  cudaGetDevice(&dev);
  auto body = [&]() {
    cudaSetDevice(dev);
    for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1)) fn(i);
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < workers; ++w) pool.emplace_back(body);
  body();
  for (auto& t : pool) t.join();
}

int batch_workers(int count) {
  const unsigned hc = std::thread::hardware_concurrency();
  const int cap = (int)std::min<unsigned>(16u, std::max<unsigned>(1u, hc ? hc : 4u));
  return std::min(cap, std::max(count, 1));
}

}  // namespace

namespace {

// The 16 selector features of the current factor into the context's device buffer (raw, or
// normalised with the selector's mean and scale); returns the device pointer.
template <typename TU>
float* features_impl(tls_ctx* ctx, bool normalised) {
  cudaStream_t st = ctx->stream;
  const int64_t n = ctx->n, npad = ctx->npad;
  const size_t vec = sizeof(TU) * (size_t)npad;
  const size_t sbytes = sizeof(double) * (size_t)(2 + (n + 7) / 8);
  unsigned char* buf = static_cast<unsigned char*>(slot(ctx, kSlotFeat, 2 * vec + sbytes + 64 * 4));
  if (!buf) return nullptr;
  TU* x = reinterpret_cast<TU*>(buf);
  TU* y = reinterpret_cast<TU*>(buf + vec);
  double* scratch = reinterpret_cast<double*>(buf + 2 * vec);
  float* F = reinterpret_cast<float*>(buf + 2 * vec + sbytes);
  const double log10_uf = (ctx->uf_used == TLS_FP16) ? -11.0 * std::log10(2.0)
                          : (ctx->uf_used == TLS_BF16) ? -8.0 * std::log10(2.0)
                          : (ctx->uf_used == TLS_FP32) ? -24.0 * std::log10(2.0)
                                                        : -53.0 * std::log10(2.0);
  tls::launch_features<TU>(ctx->d, static_cast<const TU*>(ctx->R), static_cast<const TU*>(ctx->W),
                           static_cast<const TU*>(ctx->WT), n, npad, ctx->m, ctx->norm2_A,
                           ctx->norm2_b, ctx->shifts, ctx->shift, (int)ctx->fail_pivot, log10_uf,
                           x, y, scratch, F, st);
  if (normalised)
    tls::launch_feature_normalise(F, ctx->dsel + TLS_MLP_PARAMS,
                                  ctx->dsel + TLS_MLP_PARAMS + TLS_SELECTOR_FEATURES, st);
  return F;
}

// TLS_AUTO: factor at FP16, let the network pick u_f (and the PCGTLS tolerance) from the
// features of that factor, refactor at the pick when it is not FP16.
tls_status factor_auto_ctx(tls_ctx* ctx) {
  tls_status s = factor_impl(ctx, TLS_FP16);
  if (s != TLS_OK || !ctx->has_sel) return s;
  float* F = (ctx->u == Prec::FP64) ? features_impl<double>(ctx, true)
                                    : features_impl<float>(ctx, true);
  if (!F) return TLS_ERR_OOM;
  float* net = F + 32;
  tls::mlp::launch_mlp_forward(ctx->dsel, 1, F, net, ctx->stream);
  TLS_CK_LAUNCH("selector network");
  float out[4];
  TLS_CK(cudaMemcpyAsync(out, net, sizeof(out), cudaMemcpyDeviceToHost, ctx->stream));
  TLS_CK(cudaStreamSynchronize(ctx->stream));
  int c = 0;
  if (out[1] > out[c]) c = 1;
  if (out[2] > out[c]) c = 2;
  ctx->sel_class = c;
  ctx->sel_cg_tol = std::pow(10.0, std::min(-1.0, std::max(-12.0, (double)out[3])));
  if (ctx->uf_used == TLS_FP16 && c != 0) s = factor_impl(ctx, c == 1 ? TLS_BF16 : TLS_FP32);
  ctx->use_sel_tol = (s == TLS_OK);
  return s;
}

}  // namespace

extern "C" {

const char* tls_options_check(const tls_options* opt) {
  if (!opt) return "no options given";
  return tls::options_error(*opt);
}

void tls_default_options(tls_options* opt) {
  if (!opt) return;
  opt->u = TLS_FP32;
  opt->mode_A = 1;
  opt->cg_fixed = 1;
  opt->cg_tol = 1e-6;
  opt->cg_max = 50;
  opt->psi_rule_ge = 0;
  opt->ls_iters = 6;
  opt->max_shifts = 3;
  opt->gram_simt = 0;
  opt->shift_first = 1;
  opt->psi_accept = 1e-15;
  opt->fallback = 1;
  opt->constr_guard = 0.0;
  opt->stall_fallback = 1;
  opt->stall_ratio = 0.9;
  opt->constraint_iters = 0;
  opt->hybrid_ratio = 0.1;
  opt->reproducible = 1;
  opt->factor = 0;
}

const char* tls_status_str(tls_status s) {
  switch (s) {
    case TLS_OK: return "TLS_OK";
    case TLS_ERR_ARG: return "TLS_ERR_ARG";
    case TLS_ERR_CUDA: return "TLS_ERR_CUDA";
    case TLS_ERR_OOM: return "TLS_ERR_OOM";
    case TLS_ERR_STATE: return "TLS_ERR_STATE";
    case TLS_ERR_FACTOR_BREAKDOWN: return "TLS_ERR_FACTOR_BREAKDOWN";
    case TLS_ERR_NOT_SPD: return "TLS_ERR_NOT_SPD";
    case TLS_ERR_NOT_UNIQUE: return "TLS_ERR_NOT_UNIQUE";
    case TLS_ERR_NO_CONVERGENCE: return "TLS_ERR_NO_CONVERGENCE";
    case TLS_ERR_TIMEOUT: return "TLS_ERR_TIMEOUT";
  }
  return "TLS_ERR_UNKNOWN";
}

const char* tls_last_error(const tls_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }


void tls_shape(const tls_ctx* ctx, int64_t* m, int64_t* n, int64_t* nnz) {
  if (!ctx) return;
  if (m) *m = ctx->m;
  if (n) *n = ctx->n;
  if (nnz) *nnz = ctx->nnz;
}

tls_status tls_create_dense(tls_ctx** out, int64_t m, int64_t n, const double* A, int64_t lda,
                            const double* b, int on_device, void* stream) {
  if (!out) return TLS_ERR_ARG;
  *out = nullptr;
  if (m < 1 || n < 1 || m < n || lda < n || !A || !b) return TLS_ERR_ARG;
  tls_ctx* ctx = new tls_ctx();
  tls_options o;
  tls_default_options(&o);
  ctx->opt = o;
  tls_status s = ctx_common_init(ctx, m, n, stream);
  if (s != TLS_OK) { destroy_ctx(ctx); return s; }
  const int64_t npad = ctx->npad;
  ctx->A64 = alloc_t<double>(ctx, m * npad);
  if (!ctx->A64) { destroy_ctx(ctx); return TLS_ERR_OOM; }
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  // zero padding columns n .. npad-1, the copy, then the NaN / Inf check on the device copy
  // (one read at copy bandwidth instead of a host pass over the caller's data); the error word
  // (zero until a solve) serves as its flag
  cudaError_t e = cudaSuccess;
  if (npad > n)
    e = cudaMemset2DAsync(ctx->A64 + n, sizeof(double) * npad, 0, sizeof(double) * (npad - n),
                          m, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(ctx->A64, sizeof(double) * npad, A, sizeof(double) * lda,
                          sizeof(double) * n, m, kind, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->b, b, sizeof(double) * m, kind, ctx->stream);
  int bad = 0;
  if (e == cudaSuccess) {
    tls::launch_nonfinite(ctx->A64, m * npad, ctx->derr, ctx->num_sms, ctx->stream);
    tls::launch_nonfinite(ctx->b, m, ctx->derr, ctx->num_sms, ctx->stream);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&bad, ctx->derr, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    tls_status st = cuda_status(ctx, e, "upload");
    destroy_ctx(ctx);
    return st;
  }
  if (bad) {
    destroy_ctx(ctx);
    return TLS_ERR_ARG;   // NaN or Inf in A or b
  }
  *out = ctx;
  return TLS_OK;
}

tls_status tls_create_csr(tls_ctx** out, int64_t m, int64_t n, int64_t nnz, const int64_t* row_ptr,
                          const int32_t* col_idx, const double* val, const double* b,
                          int on_device, void* stream) {
  if (!out) return TLS_ERR_ARG;
  *out = nullptr;
  if (on_device || m < 1 || n < 1 || m < n || nnz < 0 || !row_ptr || !b) return TLS_ERR_ARG;
  if (nnz > 0 && (!col_idx || !val)) return TLS_ERR_ARG;
  if (nnz >= (int64_t)1 << 31 || m >= (int64_t)1 << 31) return TLS_ERR_ARG;
  if (row_ptr[0] != 0 || row_ptr[m] != nnz) return TLS_ERR_ARG;
  const int64_t npad = tls::round_up(n, tls::kPad);
  if (tls::csc_build_warps(npad) < 1) return TLS_ERR_ARG;   // n too large for the CSC build
  tls_ctx* ctx = new tls_ctx();
  tls_options o;
  tls_default_options(&o);
  ctx->opt = o;
  tls_status st = ctx_common_init(ctx, m, n, stream);
  if (st != TLS_OK) { destroy_ctx(ctx); return st; }
  ctx->sparse = true;
  ctx->nnz = nnz;
  const int64_t nz = std::max<int64_t>(nnz, 1);
  const int G = ctx->num_sms;
  ctx->rp = alloc_t<int>(ctx, m + 1);
  ctx->ci = alloc_t<int>(ctx, nz);
  ctx->v64 = alloc_t<double>(ctx, nz);
  ctx->v32 = alloc_t<float>(ctx, nz);
  ctx->cp = alloc_t<int>(ctx, npad + 1);
  ctx->ri = alloc_t<int>(ctx, nz);
  ctx->cv64 = alloc_t<double>(ctx, nz);
  ctx->cv32 = alloc_t<float>(ctx, nz);
  ctx->rbuf = alloc_t<double>(ctx, m);
  // creation scratch (returned at the end): 64-bit row offsets, per-CTA column counts
  int64_t* rp64 = alloc_t<int64_t>(ctx, m + 1);
  int* work = alloc_t<int>(ctx, (int64_t)2 * G * npad + npad);
  if (!ctx->rp || !ctx->ci || !ctx->v64 || !ctx->v32 || !ctx->cp || !ctx->ri || !ctx->cv64 ||
      !ctx->cv32 || !ctx->rbuf || !rp64 || !work) {
    destroy_ctx(ctx);
    return TLS_ERR_OOM;
  }
  // upload; check the structure and the values on the device (the error word, zero until a
  // solve, is the flag) before anything indexes with the column indices; then the column
  // (CSC) index as a stable counting sort by column, also on the device
  cudaStream_t sm = ctx->stream;
  int bad = 0;
  cudaError_t e = cudaMemcpyAsync(rp64, row_ptr, sizeof(int64_t) * (m + 1), cudaMemcpyHostToDevice, sm);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(ctx->ci, col_idx, sizeof(int) * nnz, cudaMemcpyHostToDevice, sm);
  if (e == cudaSuccess && nnz > 0) e = cudaMemcpyAsync(ctx->v64, val, sizeof(double) * nnz, cudaMemcpyHostToDevice, sm);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->b, b, sizeof(double) * m, cudaMemcpyHostToDevice, sm);
  if (e == cudaSuccess) {
    tls::csr_check(rp64, ctx->ci, ctx->v64, ctx->b, m, n, nnz, ctx->rp, ctx->derr, sm);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, ctx->derr, sizeof(int), cudaMemcpyDeviceToHost, sm);
  if (e == cudaSuccess) e = cudaStreamSynchronize(sm);
  if (e == cudaSuccess && bad) {
    destroy_ctx(ctx);
    return TLS_ERR_ARG;   // malformed structure or NaN / Inf values
  }
  if (e == cudaSuccess) {
    int* cnt = work;
    int* off = work + (int64_t)G * npad;
    int* tot = work + (int64_t)2 * G * npad;
    tls::csc_build(ctx->rp, ctx->ci, ctx->v64, m, npad, nnz, G, cnt, off, tot, ctx->cp, ctx->ri,
                   ctx->cv64, sm);
    tls::sparse_to_f32(ctx->v64, ctx->v32, nnz, sm);
    tls::sparse_to_f32(ctx->cv64, ctx->cv32, nnz, sm);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(sm);
  if (e != cudaSuccess) {
    tls_status s2 = cuda_status(ctx, e, "upload");
    destroy_ctx(ctx);
    return s2;
  }
  dev_free(ctx, work);
  dev_free(ctx, rp64);
  *out = ctx;
  return TLS_OK;
}

tls_status tls_factor(tls_ctx* ctx, tls_prec u_f, const tls_options* opt) {
  if (!ctx) return TLS_ERR_ARG;
  if ((int)u_f < 0 || (int)u_f > 4) {
    set_err(ctx, "u_f must be FP16, BF16, FP32, FP64 or AUTO");
    return TLS_ERR_ARG;
  }
  tls_options o;
  tls_default_options(&o);
  if (opt) o = *opt;
  if (o.mode_A < 0 || o.mode_A > 2 || (o.mode_A == 2 && ctx->sparse)) {
    set_err(ctx, "mode_A must be 0, 1 or 2 (2: dense contexts)");
    return TLS_ERR_ARG;
  }
  if (o.u != TLS_FP32 && o.u != TLS_FP64) {
    set_err(ctx, "u must be FP32 or FP64 (a half-precision PCGTLS working precision limits the "
                 "attainable accuracy, Sec. 4.3)");
    return TLS_ERR_ARG;
  }
  if (o.factor < 0 || o.factor > 1 || (o.factor == 1 && ctx->sparse)) {
    set_err(ctx, "factor must be 0 (Cholesky of the scaled Gram matrix) or 1 (Householder QR, "
                 "dense contexts)");
    return TLS_ERR_ARG;
  }
  if (const char* why = tls::options_error(o)) {
    set_err(ctx, why);
    return TLS_ERR_ARG;
  }
  const int64_t limit = (o.u == TLS_FP64) ? 4096 : 8192;
  if (ctx->npad > limit) {
    set_err(ctx, "n too large for the dense path");
    return TLS_ERR_ARG;
  }
  ctx->opt = o;
  ctx->u = to_prec(o.u);
  ctx->use_sel_tol = false;
  ctx->sel_class = -1;
  if (u_f == TLS_AUTO) return factor_auto_ctx(ctx);
  return factor_impl(ctx, u_f);
}

tls_status tls_set_selector(tls_ctx* ctx, const float* params, const float* mean,
                            const float* scale) {
  if (!ctx || !params || !mean || !scale) return TLS_ERR_ARG;
  if (!ctx->dsel) {
    ctx->dsel = alloc_t<float>(ctx, TLS_MLP_PARAMS + 2 * TLS_SELECTOR_FEATURES);
    if (!ctx->dsel) return TLS_ERR_OOM;
  }
  cudaStream_t st = ctx->stream;
  TLS_CK(cudaMemcpyAsync(ctx->dsel, params, sizeof(float) * TLS_MLP_PARAMS, cudaMemcpyHostToDevice,
                         st));
  TLS_CK(cudaMemcpyAsync(ctx->dsel + TLS_MLP_PARAMS, mean, sizeof(float) * TLS_SELECTOR_FEATURES,
                         cudaMemcpyHostToDevice, st));
  TLS_CK(cudaMemcpyAsync(ctx->dsel + TLS_MLP_PARAMS + TLS_SELECTOR_FEATURES, scale,
                         sizeof(float) * TLS_SELECTOR_FEATURES, cudaMemcpyHostToDevice, st));
  TLS_CK(cudaStreamSynchronize(st));
  ctx->has_sel = true;
  return TLS_OK;
}

tls_status tls_features(tls_ctx* ctx, float* F_host) {
  if (!ctx || !F_host) return TLS_ERR_ARG;
  if (!ctx->factored) return TLS_ERR_STATE;
  float* F = (ctx->u == Prec::FP64) ? features_impl<double>(ctx, false)
                                    : features_impl<float>(ctx, false);
  if (!F) return TLS_ERR_OOM;
  TLS_CK_LAUNCH("features");
  TLS_CK(cudaMemcpyAsync(F_host, F, sizeof(float) * TLS_SELECTOR_FEATURES, cudaMemcpyDeviceToHost,
                         ctx->stream));
  TLS_CK(cudaStreamSynchronize(ctx->stream));
  return TLS_OK;
}

static tls_status solve_once(tls_ctx* ctx, double tol, int max_rqi, double* sigma,
                             tls_info* info) {
  if (ctx->u == Prec::FP64) return solve_impl<double>(ctx, tol, max_rqi, info, sigma);
  return solve_impl<float>(ctx, tol, max_rqi, info, sigma);
}

// Solve; when the RQI loop ends on max_rqi without converging and the factor precision is
// below FP64, refactor one precision up and solve again (the precision fallback for a factor
// that violates the stability constraints of Sec. 3.1).
constexpr int kMaxRqi = 1000;

static tls_status solve_common(tls_ctx* ctx, double tol, int max_rqi, double* sigma,
                               tls_info* info) {
  if (!ctx || !sigma || max_rqi < 0 || !(tol >= 0.0)) return TLS_ERR_ARG;
  if (max_rqi > kMaxRqi) {
    // RQI step k runs k + 1 PCGTLS steps per solve: the cap bounds the work of one call
    set_err(ctx, "max_rqi must be in [0, " + std::to_string(kMaxRqi) + "]");
    return TLS_ERR_ARG;
  }
  if (!ctx->factored) {
    set_err(ctx, "tls_solve called before a successful tls_factor");
    return TLS_ERR_STATE;
  }
  tls_info loc{};
  int trigger = ctx->escalations ? TLS_TRIGGER_CONSTRAINT : TLS_TRIGGER_NONE;
  tls_status s = solve_once(ctx, tol, max_rqi, sigma, &loc);
  int fb = 0;
  // the precision fallback (FP16/BF16 -> FP32 -> FP64): on max_rqi, and earlier on a stalled or
  // indefinite PCGTLS solve
  while (s == TLS_OK && ctx->opt.fallback &&
         (loc.stop_reason == TLS_STOP_MAX_RQI || loc.stop_reason == TLS_STOP_STALL) &&
         ctx->uf_used != TLS_FP64 && fb < 2) {
    trigger = (loc.stop_reason == TLS_STOP_MAX_RQI) ? TLS_TRIGGER_MAX_RQI : ctx->stall_trigger;
    const tls_prec next = (ctx->uf_used == TLS_FP32) ? TLS_FP64 : TLS_FP32;
    const tls_options o = ctx->opt;
    s = tls_factor(ctx, next, &o);
    if (s != TLS_OK) break;
    ++fb;
    s = solve_once(ctx, tol, max_rqi, sigma, &loc);
  }
  loc.fallbacks = fb;
  loc.fallback_trigger = trigger;
  loc.constr1 = loc.constr2 = NAN;
  if (s == TLS_OK && ctx->opt.constraint_iters > 0) {
    // the paper's constraints 1 and 2 (Eq. (5), Eq. (9)) for A, with this solve's sigma
    double c[9];
    s = ctx->H ? tls_condition(ctx, ctx->opt.constraint_iters, c) : TLS_ERR_STATE;
    if (s == TLS_ERR_STATE && !ctx->H) {
      s = TLS_OK;   // QR factor: no Gram matrix, the constraint fields stay NaN
    } else if (s == TLS_OK) {
      loc.constr1 = c[7];
      loc.constr2 = c[8];
      if (std::isnan(ctx->constr2_scaled)) s = scaled_constraint2(ctx, &ctx->constr2_scaled);
      loc.constr2_scaled = ctx->constr2_scaled;
    }
  }
  if (info) *info = loc;
  return s;
}

tls_status tls_solve(tls_ctx* ctx, double tol, int max_rqi, double* x, double* sigma,
                     tls_info* info) {
  if (!x) return TLS_ERR_ARG;
  tls_status s = solve_common(ctx, tol, max_rqi, sigma, info);
  if (s != TLS_OK) return s;
  cudaError_t e = cudaMemcpyAsync(x, ctx->x_best, sizeof(double) * ctx->n,
                                  cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  return cuda_status(ctx, e, "download x");
}

tls_status tls_solve_device(tls_ctx* ctx, double tol, int max_rqi, double* x_dev, double* sigma,
                            tls_info* info) {
  if (!x_dev) return TLS_ERR_ARG;
  tls_status s = solve_common(ctx, tol, max_rqi, sigma, info);
  if (s != TLS_OK) return s;
  cudaError_t e = cudaMemcpyAsync(x_dev, ctx->x_best, sizeof(double) * ctx->n,
                                  cudaMemcpyDeviceToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  return cuda_status(ctx, e, "copy x");
}

tls_status tls_factor_batched(int count, tls_ctx* const* ctxs, tls_prec u_f,
                              const tls_options* opt, tls_status* per_problem) {
  if (count < 0 || (count > 0 && !ctxs)) return TLS_ERR_ARG;
  std::vector<tls_status> st((size_t)std::max(count, 1), TLS_OK);
  run_workers(count, batch_workers(count), [&](int i) { st[(size_t)i] = tls_factor(ctxs[i], u_f, opt); });
  tls_status first = TLS_OK;
  for (int i = 0; i < count; ++i) {
    if (per_problem) per_problem[i] = st[(size_t)i];
    if (st[(size_t)i] != TLS_OK && first == TLS_OK) first = st[(size_t)i];
  }
  return first;
}

tls_status tls_solve_batched(int count, tls_ctx* const* ctxs, double tol, int max_rqi,
                             double* const* x, double* sigma, tls_info* infos,
                             tls_status* per_problem) {
  if (count < 0 || (count > 0 && (!ctxs || !x || !sigma))) return TLS_ERR_ARG;
  std::vector<tls_status> st((size_t)std::max(count, 1), TLS_OK);
  run_workers(count, batch_workers(count), [&](int i) {
    st[(size_t)i] = tls_solve(ctxs[i], tol, max_rqi, x[i], sigma + i, infos ? infos + i : nullptr);
  });
  tls_status first = TLS_OK;
  for (int i = 0; i < count; ++i) {
    if (per_problem) per_problem[i] = st[(size_t)i];
    if (st[(size_t)i] != TLS_OK && first == TLS_OK) first = st[(size_t)i];
  }
  return first;
}

void tls_destroy(tls_ctx* ctx) { destroy_ctx(ctx); }

// ---------------------------------------------------------------------------------------
// Inspection entry points (include/tls_debug.h)
// ---------------------------------------------------------------------------------------
tls_status tls_export_factor(tls_ctx* ctx, double* R_host, double* d_host, double* H_host) {
  if (!ctx) return TLS_ERR_ARG;
  if (!ctx->factored) return TLS_ERR_STATE;
  const int64_t n = ctx->n, npad = ctx->npad;
  std::vector<double> tmp((size_t)npad * npad);
  cudaStream_t st = ctx->stream;
  auto fetch = [&](const void* src, bool fp64) -> cudaError_t {
    if (fp64) return cudaMemcpyAsync(tmp.data(), src, 8 * npad * npad, cudaMemcpyDeviceToHost, st);
    std::vector<float> t32((size_t)npad * npad);
    cudaError_t e = cudaMemcpyAsync(t32.data(), src, 4 * npad * npad, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (size_t i = 0; i < t32.size(); ++i) tmp[i] = t32[i];
    return e;
  };
  if (R_host) {
    TLS_CK(fetch(ctx->R, ctx->u == Prec::FP64));
    TLS_CK(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) R_host[i * n + j] = tmp[i * npad + j];
  }
  if (H_host && ctx->H) {
    TLS_CK(fetch(ctx->H, ctx->H_fp64));
    TLS_CK(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) H_host[i * n + j] = tmp[i * npad + j];
  }
  if (d_host) {
    TLS_CK(cudaMemcpyAsync(d_host, ctx->d, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    TLS_CK(cudaStreamSynchronize(st));
  }
  return TLS_OK;
}

tls_status tls_set_small_path(tls_ctx* ctx, int path) {
  if (!ctx) return TLS_ERR_ARG;
  if (path < 0 || path > 3) return TLS_ERR_ARG;
  ctx->small_path = path;
  return TLS_OK;
}

tls_status tls_set_pass_variant(tls_ctx* ctx, int variant_fp64, int variant_u) {
  if (!ctx || !ctx->factored || ctx->sparse) return TLS_ERR_STATE;
  if (variant_fp64 < 0 || variant_fp64 > tls::kApassVariants || variant_u < 0 ||
      variant_u >= tls::kApassVariants)
    return TLS_ERR_ARG;
  if (variant_fp64 == tls::kApassVariants) {
    // the double-FP32 residual pass (FP32 working precision only)
    const bool was = ctx->resid_df;
    ctx->resid_df = true;
    if (!resid_df_active(ctx)) {
      ctx->resid_df = was;
      return TLS_ERR_ARG;
    }
    const tls::ApassPlan pu = (ctx->u == Prec::FP64)
                                  ? tls::plan_apass<double>(ctx->m, ctx->npad, 2, ctx->num_sms, variant_u)
                                  : tls::plan_apass<float>(ctx->m, ctx->npad, 2, ctx->num_sms, variant_u);
    if ((variant_u == 1 || variant_u == 2) && !pu.tma) return TLS_ERR_ARG;
    ctx->planU = pu;
    ctx->PU = pu.grid;
    return TLS_OK;
  }
  if (ctx->npad > 4096) return TLS_ERR_ARG;   // the FP64 passes stop at n_pad = 4096
  ctx->resid_df = false;
  const tls::ApassPlan p64 = tls::plan_apass<double>(ctx->m, ctx->npad, 1, ctx->num_sms, variant_fp64);
  const tls::ApassPlan pu = (ctx->u == Prec::FP64)
                                ? tls::plan_apass<double>(ctx->m, ctx->npad, 2, ctx->num_sms, variant_u)
                                : tls::plan_apass<float>(ctx->m, ctx->npad, 2, ctx->num_sms, variant_u);
  if (((variant_fp64 == 1 || variant_fp64 == 2) && !p64.tma) ||
      ((variant_u == 1 || variant_u == 2) && !pu.tma))
    return TLS_ERR_ARG;   // the staged kernel does not fit this n
  ctx->plan64 = p64;
  ctx->P64 = p64.grid;
  ctx->planU = pu;
  ctx->PU = pu.grid;
  return TLS_OK;
}

tls_status tls_profile_enable(tls_ctx* ctx, int on) {
  if (!ctx) return TLS_ERR_ARG;
  ctx->prof_on = on != 0;
  ctx->pused = 0;
  for (int i = 0; i < TLS_PROF_NCLASSES; ++i) {
    ctx->prof_ms[i] = 0.0;
    ctx->prof_cnt[i] = 0;
    ctx->prof_units[i] = 0;
  }
  return TLS_OK;
}

tls_status tls_profile_get(const tls_ctx* ctx, int cls, int64_t* count, double* ms) {
  if (!ctx || cls < 0 || cls >= TLS_PROF_NCLASSES) return TLS_ERR_ARG;
  if (count) *count = ctx->prof_cnt[cls];
  if (ms) *ms = ctx->prof_ms[cls];
  return TLS_OK;
}

tls_status tls_profile_units(const tls_ctx* ctx, int cls, int64_t* units) {
  if (!ctx || !units || cls < 0 || cls >= TLS_PROF_NCLASSES) return TLS_ERR_ARG;
  *units = ctx->prof_units[cls];
  return TLS_OK;
}

tls_status tls_set_factor_chain(tls_ctx* ctx, int on) {
  if (!ctx || on < 0 || on > 4) return TLS_ERR_ARG;
  ctx->chol_chain = on;
  return TLS_OK;
}

tls_status tls_set_factor_tc(tls_ctx* ctx, int on) {
  if (!ctx || on < 0 || on > 1) return TLS_ERR_ARG;
  ctx->chol_tc = on;
  return TLS_OK;
}

tls_status tls_set_pcg_l2_keep(tls_ctx* ctx, int64_t bytes) {
  if (!ctx || bytes < 0) return TLS_ERR_ARG;
  ctx->l2_keep = bytes;
  return TLS_OK;
}

tls_status tls_trace_enable(tls_ctx* ctx, int on) {
  if (!ctx) return TLS_ERR_ARG;
  if (on && !ctx->trace) {
    ctx->trace = static_cast<unsigned long long*>(
        dev_alloc(ctx, sizeof(unsigned long long) * (size_t)tls::pcg_fused_trace_words()));
    if (!ctx->trace) return TLS_ERR_OOM;
  }
  if (ctx->trace)
    TLS_CK(cudaMemsetAsync(ctx->trace, 0,
                           sizeof(unsigned long long) * (size_t)tls::pcg_fused_trace_words(),
                           ctx->stream));
  ctx->trace_on = on != 0;
  return TLS_OK;
}

tls_status tls_trace_get(tls_ctx* ctx, uint64_t* out, int cap, int* count) {
  if (!ctx || !out || cap < 0) return TLS_ERR_ARG;
  const int w = tls::pcg_fused_trace_words();
  if (count) *count = ctx->trace ? w : 0;
  if (!ctx->trace) return TLS_OK;
  TLS_CK(cudaMemcpyAsync(out, ctx->trace, sizeof(uint64_t) * (size_t)std::min(cap, w),
                         cudaMemcpyDeviceToHost, ctx->stream));
  TLS_CK(cudaStreamSynchronize(ctx->stream));
  return TLS_OK;
}

tls_status tls_set_pcg_fused(tls_ctx* ctx, int mode) {
  if (!ctx || mode < 0 || mode > 7) return TLS_ERR_ARG;
  if (mode != 0 && mode != 2 && !tls::pcg_fused_supported(ctx->npad, 2, ctx->num_sms))
    return TLS_ERR_ARG;
  ctx->pcg_fused = (mode >= 3) ? 1 : mode;
  ctx->fused_load = (mode >= 3 && mode <= 5) ? mode - 3 : 0;
  ctx->fused_pass = (mode == 5) ? 1 : (mode >= 6) ? mode - 5 : 0;
  return TLS_OK;
}

uint64_t tls_kernel_launches(void) { return tls::g_launches.load(); }

tls_status tls_condition(tls_ctx* ctx, int iters, double* out) {
  if (!ctx || !out || iters < 1 || iters > 100000) return TLS_ERR_ARG;
  if (!ctx->factored) return TLS_ERR_STATE;
  if (!ctx->H) {
    set_err(ctx, "the condition estimate uses the scaled Gram matrix, which the QR factor does "
                 "not form");
    return TLS_ERR_STATE;
  }
  if (ctx->H_fp64) {
    if (ctx->u == Prec::FP64) return condition_impl<double, double>(ctx, iters, out);
    return condition_impl<double, float>(ctx, iters, out);
  }
  if (ctx->u == Prec::FP64) return condition_impl<float, double>(ctx, iters, out);
  return condition_impl<float, float>(ctx, iters, out);
}

tls_status tls_export_working_copy(tls_ctx* ctx, float* A32_host) {
  if (!ctx || !A32_host) return TLS_ERR_ARG;
  if (!ctx->factored || !ctx->A32 || ctx->sparse) return TLS_ERR_STATE;
  TLS_CK(cudaMemcpy2DAsync(A32_host, sizeof(float) * ctx->n, ctx->A32, sizeof(float) * ctx->npad,
                           sizeof(float) * ctx->n, ctx->m, cudaMemcpyDeviceToHost, ctx->stream));
  TLS_CK(cudaStreamSynchronize(ctx->stream));
  return TLS_OK;
}

tls_status tls_residual(tls_ctx* ctx, const double* x_host, double* f_host, double* scal_host) {
  if (!ctx || !x_host) return TLS_ERR_ARG;
  cudaStream_t st = ctx->stream;
  TLS_CK(cudaMemsetAsync(ctx->x, 0, sizeof(double) * ctx->npad, st));
  TLS_CK(cudaMemcpyAsync(ctx->x, x_host, sizeof(double) * ctx->n, cudaMemcpyHostToDevice, st));
  tls::launch_xx(ctx->x, ctx->rs, ctx->n, st, ctx->gpart + 2048);
  tls_status s = residual_pass(ctx);
  if (s != TLS_OK) return s;
  TLS_CK(cudaMemcpyAsync(ctx->h_rs, ctx->rs, sizeof(RqiScalars), cudaMemcpyDeviceToHost, st));
  if (f_host)
    TLS_CK(cudaMemcpyAsync(f_host, ctx->f, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost, st));
  TLS_CK(cudaStreamSynchronize(st));
  if (scal_host) {
    scal_host[0] = ctx->h_rs->sigma2;
    scal_host[1] = ctx->h_rs->g;
    scal_host[2] = ctx->h_rs->psi;
    scal_host[3] = ctx->h_rs->rr;
    scal_host[4] = ctx->h_rs->br;
  }
  return TLS_OK;
}

tls_status tls_pcgtls(tls_ctx* ctx, int nr, double sigma2, const double* f0, const double* f1,
                      int steps, double cg_tol, double* w0, double* w1, int* iters,
                      int* not_spd) {
  if (!ctx || !f0 || !w0 || nr < 1 || nr > 2 || steps < 0 || steps > 100000 ||
      (nr == 2 && !f1) || std::isnan(cg_tol))
    return TLS_ERR_ARG;
  if (!ctx->factored) return TLS_ERR_STATE;
  if (ctx->u == Prec::FP64)
    return pcgtls_host<double>(ctx, nr, sigma2, f0, f1, steps, cg_tol, w0, w1, iters, not_spd);
  return pcgtls_host<float>(ctx, nr, sigma2, f0, f1, steps, cg_tol, w0, w1, iters, not_spd);
}

tls_status tls_precond(tls_ctx* ctx, const double* y, double* s0, double* u) {
  if (!ctx || !y) return TLS_ERR_ARG;
  if (!ctx->factored) return TLS_ERR_STATE;
  if (ctx->u == Prec::FP64) return precond_host<double>(ctx, y, s0, u);
  return precond_host<float>(ctx, y, s0, u);
}

tls_status tls_precond_trsv(tls_ctx* ctx, const double* y, double* s0, double* u) {
  if (!ctx || !y) return TLS_ERR_ARG;
  if (!ctx->factored) return TLS_ERR_STATE;
  if (ctx->R == nullptr) return TLS_ERR_STATE;
  if (ctx->u == Prec::FP64) return precond_trsv_host<double>(ctx, y, s0, u);
  return precond_trsv_host<float>(ctx, y, s0, u);
}

}  // extern "C"
