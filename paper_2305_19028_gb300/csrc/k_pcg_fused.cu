// One PCGTLS solve (Alg. 3, the A-explicit operator; paired right-hand sides) in a single
// persistent cooperative launch, FP32 working precision (the u_p of Alg. 4).
//
// Every CTA is resident (one per SM, 16 warps). A CTA owns a contiguous block of rows of the FP32
// copy of A and streams it, step after step, through a ring of shared-memory stages filled by
// 1-D bulk asynchronous copies (TMA, completion on mbarriers): as soon as every thread holds its
// part of a tile in registers, thread 0 refills that stage with the tile S positions ahead in the
// CTA's sequence of tiles (which runs on into the next step's pass). Per PCGTLS step j:
//
//   pass    t = A q_j (both right-hand sides) row by row from the ring, the CTA's partial of
//           A^T t and of ||t||^2                                  -- grid barrier 1
//   reduce  column sums of the partials (each CTA a slice of the columns): delta_j, alpha_j,
//           w += alpha q_j, y = D^{-1}(A^T t - sigma^2 q_j)        -- grid barrier 2
//   W^T     v = W^T y (rows over all warps of the grid), s_{j+1} = s_j - alpha v, ||s||^2
//                                                                  -- grid barrier 3
//           eta_{j+1}, beta_j and the stop flags (every CTA, same sums in the same order)
//   W       p_{j+1} = s_{j+1} + beta_j p_j, q_{j+1} = D^{-1} W p_{j+1}, ||q||^2
//                                                                  -- grid barrier 4
//
// with W = R_H^{-1} (R = R_H D), so that q = R^{-1} p and v = R^{-T} D^{-1}(...) are the two
// triangular solves of Alg. 3 done as row-parallel products with the explicit inverse. The rows
// of A do not depend on q: when a pass ends, the first S tiles of the next pass are already in
// flight, so HBM keeps streaming while the CTAs run the reduce / W^T / W phases and their grid
// barriers. The initialisation (s_0 = R^{-T} f, eta_0, p_0 = s_0, q_0) runs in the same launch,
// before the first pass, while the ring fills.
//
// Every wait is bounded: mbarrier waits by a global-timer deadline, grid barriers by a deadline
// and an abort word that a CTA whose wait expired raises, so that the others leave too; a CTA
// waits for its own copies in flight before it exits. Error codes land in *err.
#include "tls_internal.h"
#include "tls_ptx.cuh"

#include <algorithm>

namespace tls {
namespace {

constexpr int kFcWarps = 16;                   // warps per CTA
constexpr int kFcThreads = kFcWarps * 32;      // 512
constexpr int kFTileMaxBytes = 32768;          // largest ring stage
constexpr int kFMaxStages = 8;
constexpr int kFStepU = 16;                    // float4 loads in flight per lane (W products)
constexpr uint64_t kFBarrierNs = 2000ull * 1000 * 1000;   // grid barrier deadline: 2 s

// scalar partial sums in gpart (doubles): [0, 2G) ||t||^2, [2G, 4G) ||s||^2, [4G, 6G) ||q||^2
constexpr int kOffTT = 0, kOffSS = 2, kOffQQ = 4;   // multiples of G

struct FusedArgs {
  const float* A;        // m x npad, row-major, rows back to back (lda = npad)
  int64_t m, n, npad;
  int nr, steps, stages, tile_rows;
  const double* fin0;    // right-hand side 0 is fin0_scale * fin0, 1 is fin1 (FP64, n values)
  double fin0_scale;
  const double* fin1;
  const double* dinv64;  // 1 / d (FP64, npad)
  const float* dinv;     // 1 / d (FP32, npad)
  const float* W;        // R_H^{-1}, upper triangular, npad x npad
  const float* WT;       // W^T, lower triangular
  float* w;              // solutions, nr x npad
  float* y;              // D^{-1}(A^T t - sigma^2 q), nr x npad
  float* s;              // s_j, nr x npad
  float* pa;             // p_j, ping-pong, nr x npad each
  float* pb;
  float* q;              // q_j = D^{-1} W p_j, nr x npad
  float* part;           // G x nr x npad pass partials
  double* gpart;         // scalar partials, 6 G doubles
  PcgScalars* sc;
  double sigma2, cg_tol2;
  unsigned int* bar;     // [0] arrivals, [32] generation, [64] abort (zero between launches)
  int* err;
  unsigned long long* trace;   // optional phase timestamps of CTA 0 (kFTraceCap words)
};

// Trace layout (global-timer nanoseconds, CTA 0, thread 0): [0] start, [1] initialisation done,
// then per step j < kFTraceSteps, at 2 + kFTracePer * j: pass start, pass end, barrier 1 done,
// reduce done, barrier 2 done, W^T done, barrier 3 done, W done, barrier 4 done, and the time
// thread 0 spent waiting for tiles of that pass.
constexpr int kFTracePer = 10;
constexpr int kFTraceSteps = 64;
// then, for the first kFTraceTiles tiles of step 0: tile data ready, first barrier passed, copy
// issued, second barrier passed, tile done (5 words each)
constexpr int kFTraceTiles = 64;
constexpr int kFTraceTileBase = 2 + kFTracePer * kFTraceSteps;

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void cons_sync() { __syncthreads(); }

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sumd(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp sums of NV values (NV a power of two <= 32) by recursive halving; lane l returns the
// total of value l >> (5 - log2 NV).
template <int NV>
__device__ __forceinline__ float warp_reduce_scatter(const float (&v)[NV]) {
  const int lane = threadIdx.x & 31;
  float x[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) x[i] = v[i];
  int o = 16;
#pragma unroll
  for (int k = NV; k > 1; k >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < k / 2; ++i) {
      const float keep = up ? x[k / 2 + i] : x[i];
      const float give = up ? x[i] : x[k / 2 + i];
      x[i] = keep + __shfl_xor_sync(0xffffffffu, give, o);
    }
  }
  float r = x[0];
  for (; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  return r;
}

__device__ __forceinline__ float dot4(const float4& a, const float4& b, float acc) {
  acc = fmaf(a.x, b.x, acc);
  acc = fmaf(a.y, b.y, acc);
  acc = fmaf(a.z, b.z, acc);
  return fmaf(a.w, b.w, acc);
}

__device__ __forceinline__ float4 ldcg4(const float* p) {
  return __ldcg(reinterpret_cast<const float4*>(p));
}

// Grid-wide barrier of every CTA (a cooperative launch: all resident).
// Returns false when the barrier was abandoned (its deadline passed here, or another CTA raised
// the abort word); the caller then leaves its loop.
__device__ bool grid_barrier(unsigned int* bar, int* err, volatile int* s_fail) {
  cons_sync();
  if (threadIdx.x == 0) {
    unsigned int* cnt = bar;
    unsigned int* gen = bar + 32;
    unsigned int* abort_w = bar + 64;
    const unsigned int g = ld_acquire(gen);
    __threadfence();
    if (atomicAdd(cnt, 1u) == gridDim.x - 1) {
      atomicExch(cnt, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const uint64_t t0 = ptx::global_ns();
      unsigned int it = 0;
      while (ld_acquire(gen) == g) {
        if ((++it & 255u) == 0) {
          if (ld_acquire(abort_w) != 0u) {
            *s_fail = 1;
            break;
          }
          if (ptx::global_ns() - t0 > kFBarrierNs) {
            atomicCAS(err, 0, 21);
            atomicExch(abort_w, 1u);
            *s_fail = 1;
            break;
          }
        }
      }
    }
    __threadfence();
  }
  cons_sync();
  return *s_fail == 0;
}

// Sum of the G per-CTA partials part[c * 2 + r] (r < 2) by warp 0, in one fixed order, so that
// every CTA obtains bit-identical totals (and takes identical decisions from them).
constexpr int kFMaxGrid = 256;   // CTAs of the launch at most (one per SM)

__device__ __forceinline__ void grid_sum2(const double* part, int G, double* out2) {
  const int lane = threadIdx.x & 31;
  // every load first (one round trip to L2), then the sums in a fixed order
  double2 v[kFMaxGrid / 32];
#pragma unroll
  for (int u = 0; u < kFMaxGrid / 32; ++u) {
    const int c = lane + 32 * u;
    v[u] = (c < G) ? __ldcg(reinterpret_cast<const double2*>(part) + c) : make_double2(0.0, 0.0);
  }
  double a0 = 0.0, a1 = 0.0;
#pragma unroll
  for (int u = 0; u < kFMaxGrid / 32; ++u) {
    a0 += v[u].x;
    a1 += v[u].y;
  }
  a0 = warp_sumd(a0);
  a1 = warp_sumd(a1);
  if (lane == 0) {
    out2[0] = a0;
    out2[1] = a1;
  }
}

// CTA sum of two per-thread FP32 values, published as doubles at
// gpart[slot * 2 + r] by thread 0. red: kFcWarps * 2 doubles of shared memory.
__device__ __forceinline__ void cta_publish2(float v0, float v1, double* red, double* dst) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v0 = warp_sumf(v0);
  v1 = warp_sumf(v1);
  if (lane == 0) {
    red[warp * 2] = (double)v0;
    red[warp * 2 + 1] = (double)v1;
  }
  cons_sync();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w2 = 0; w2 < kFcWarps; ++w2) {
      t0 += red[w2 * 2];
      t1 += red[w2 * 2 + 1];
    }
    dst[0] = t0;
    dst[1] = t1;
  }
}

struct alignas(16) FusedShared {
  uint64_t full[kFMaxStages];
  float red[kFcWarps][32];
  float tot[32];
  float red2[kFcWarps][33];
  double dred[kFcWarps * 2];
  double eta[2], eta0[2], beta[2], delta[2], alpha[2], qq[2], sums[2];
  int done[2], iters[2], nspd[2], ok[2];
  int fail;
};

// v = W^T y rows (init: s = v; step: s -= alpha v for the active right-hand sides); returns the
// lane's share of ||s||^2 (lane 0 of each warp holds its rows').
template <int NR>
__device__ __forceinline__ void wt_phase(const FusedArgs& a, const float* vs, bool init,
                                         const FusedShared& sh, float (&ss)[2]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t npad = a.npad;
  const int64_t GW = (int64_t)gridDim.x * kFcWarps;
  const bool act0 = init || (!sh.done[0] && sh.ok[0]);
  const bool act1 = NR > 1 && (init || (!sh.done[1] && sh.ok[1]));
  const float al0 = init ? 0.f : (float)sh.alpha[0];
  const float al1 = (NR > 1 && !init) ? (float)sh.alpha[1] : 0.f;
  for (int64_t j = (int64_t)blockIdx.x * kFcWarps + warp; j < npad; j += GW) {
    const float* row = a.WT + j * npad;
    const int64_t lim = ((j + 4) / 4) * 4;      // entries 0..j, rounded up (zeros beyond j)
    float a0 = 0.f, a1 = 0.f;
    for (int64_t cb = (int64_t)lane * 4; cb < lim; cb += 128 * kFStepU) {
      float4 wv[kFStepU];
#pragma unroll
      for (int u = 0; u < kFStepU; ++u) {
        const int64_t c = cb + (int64_t)u * 128;
        wv[u] = (c < lim) ? __ldg(reinterpret_cast<const float4*>(row + c))
                          : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < kFStepU; ++u) {
        const int64_t c = cb + (int64_t)u * 128;
        if (c < lim) {
          a0 = dot4(wv[u], *reinterpret_cast<const float4*>(vs + c), a0);
          if (NR > 1) a1 = dot4(wv[u], *reinterpret_cast<const float4*>(vs + npad + c), a1);
        }
      }
    }
    a0 = warp_sumf(a0);
    if (NR > 1) a1 = warp_sumf(a1);
    if (lane == 0) {
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const float v = r ? a1 : a0;
        const bool act = r ? act1 : act0;
        float* sp = a.s + r * npad + j;
        float sv;
        if (init) sv = v;
        else sv = __ldcg(sp);
        if (!init && act) sv = sv - (r ? al1 : al0) * v;
        if (init || act) *sp = sv;
        ss[r] = fmaf(sv, sv, ss[r]);
      }
    }
  }
}

// q = D^{-1} W p rows from the staged p; returns the lane's share of ||q||^2.
template <int NR>
__device__ __forceinline__ void w_phase(const FusedArgs& a, const float* vs, float (&qq)[2]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t npad = a.npad;
  const int64_t GW = (int64_t)gridDim.x * kFcWarps;
  for (int64_t i = (int64_t)blockIdx.x * kFcWarps + warp; i < npad; i += GW) {
    const float* row = a.W + i * npad;
    float a0 = 0.f, a1 = 0.f;
    for (int64_t cb = (i / 4) * 4 + (int64_t)lane * 4; cb < npad; cb += 128 * kFStepU) {
      float4 wv[kFStepU];
#pragma unroll
      for (int u = 0; u < kFStepU; ++u) {
        const int64_t c = cb + (int64_t)u * 128;
        wv[u] = (c < npad) ? __ldg(reinterpret_cast<const float4*>(row + c))
                           : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < kFStepU; ++u) {
        const int64_t c = cb + (int64_t)u * 128;
        if (c < npad) {
          a0 = dot4(wv[u], *reinterpret_cast<const float4*>(vs + c), a0);
          if (NR > 1) a1 = dot4(wv[u], *reinterpret_cast<const float4*>(vs + npad + c), a1);
        }
      }
    }
    a0 = warp_sumf(a0);
    if (NR > 1) a1 = warp_sumf(a1);
    if (lane == 0) {
      const float di = __ldg(a.dinv + i);
      const float q0 = a0 * di;
      a.q[i] = q0;
      qq[0] = fmaf(q0, q0, qq[0]);
      if (NR > 1) {
        const float q1 = a1 * di;
        a.q[npad + i] = q1;
        qq[1] = fmaf(q1, q1, qq[1]);
      }
    }
  }
}

// eta_{j+1}, beta_j and the termination flags of Alg. 3 for right-hand side r (thread 0).
__device__ __forceinline__ void step_flags(FusedShared& sh, int r, double eta_new, double tol2) {
  if (sh.done[r]) return;
  if (!sh.ok[r]) {                 // delta_j <= 0: "while delta_j != 0"; < 0 is loss of SPD
    sh.done[r] = 1;
    sh.nspd[r] = (sh.delta[r] < 0.0) ? 1 : 0;
    return;
  }
  sh.beta[r] = eta_new / sh.eta[r];
  sh.eta[r] = eta_new;
  sh.iters[r] += 1;
  if (eta_new == 0.0 || (tol2 > 0.0 && eta_new <= tol2 * sh.eta0[r])) sh.done[r] = 1;
}

__device__ __forceinline__ void trace_at(const FusedArgs& a, int idx) {
  if (a.trace != nullptr && blockIdx.x == 0 && threadIdx.x == 0 &&
      idx < kFTraceTileBase + 5 * kFTraceTiles)
    a.trace[idx] = ptx::global_ns();
}

template <int NR, int VPT, int RT>
__global__ void __launch_bounds__(kFcThreads, 1) pcg_fused_kernel(const FusedArgs a) {
  extern __shared__ __align__(128) unsigned char fsm[];
  __shared__ FusedShared sh;
  constexpr int NV = NR * RT;          // row values per tile
  static_assert(NV <= 32 && (NV & (NV - 1)) == 0, "row values per tile: a power of two <= 32");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = (int)gridDim.x;
  const int64_t npad = a.npad, E = (int64_t)NR * npad;
  const int S = a.stages;
  const int64_t stage_floats = (int64_t)RT * npad;
  float* ring = reinterpret_cast<float*>(fsm);
  float* vs = ring + (int64_t)S * stage_floats;     // staged vector (NR x npad)
  // this CTA's rows and tiles
  const int64_t per = (a.m + G - 1) / G;
  const int64_t r0 = min(a.m, (int64_t)blockIdx.x * per);
  const int64_t r1 = min(a.m, r0 + per);
  const int T = (r1 > r0) ? (int)((r1 - r0 + RT - 1) / RT) : 0;

  // the CTA's tiles in sequence: tile k is local tile k % T of pass k / T
  const int64_t total = (int64_t)a.steps * T;
  const uint64_t pol = ptx::policy_evict_first();   // each row of A is read once per pass
  auto issue = [&](int64_t k) {                     // thread 0 only
    const int slot = (int)(k % S);
    const int64_t row = r0 + (int64_t)(k % T) * RT;
    const int rows = (int)min((int64_t)RT, r1 - row);
    const uint32_t bytes = (uint32_t)(rows * npad * (int64_t)sizeof(float));
    ptx::fence_proxy_async();
    ptx::mbar_expect_tx(&sh.full[slot], bytes);
    ptx::bulk_g2s_hint(ring + slot * stage_floats, a.A + row * npad, bytes, &sh.full[slot], pol);
  };
  int64_t issued = 0;                               // meaningful in thread 0
  trace_at(a, 0);
  if (tid == 0) {
    for (int k = 0; k < S; ++k) ptx::mbar_init(&sh.full[k], 1);
    ptx::fence_mbar_init();
    sh.fail = 0;
    for (; issued < S && issued < total; ++issued) issue(issued);
  }
  __syncthreads();

  volatile int* fail = &sh.fail;
  double* gp_tt = a.gpart + (int64_t)kOffTT * G;
  double* gp_ss = a.gpart + (int64_t)kOffSS * G;
  double* gp_qq = a.gpart + (int64_t)kOffQQ * G;
  const float sig2f = (float)a.sigma2;
  long long consumed = 0;
  bool alive = true;

  // ---- initialisation: y = D^{-1} f (every CTA the whole vector), s_0 = W^T y, eta_0
  for (int64_t j = tid; j < npad; j += kFcThreads) {
    const double di = a.dinv64[j];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      double f = 0.0;
      if (j < a.n) f = (r == 0) ? a.fin0_scale * a.fin0[j] : a.fin1[j];
      vs[r * npad + j] = (float)(f * di);
    }
  }
  if (tid == 0) {
    for (int r = 0; r < 2; ++r) {
      sh.eta[r] = sh.eta0[r] = sh.beta[r] = sh.alpha[r] = sh.qq[r] = 0.0;
      sh.delta[r] = 1.0;
      sh.done[r] = (r < NR) ? 0 : 1;
      sh.iters[r] = sh.nspd[r] = 0;
      sh.ok[r] = 1;
    }
  }
  cons_sync();
  {
    float ss[2] = {0.f, 0.f};
    wt_phase<NR>(a, vs, true, sh, ss);
    cta_publish2(ss[0], ss[1], sh.dred, gp_ss + 2 * blockIdx.x);
  }
  alive = grid_barrier(a.bar, a.err, fail);
  if (alive) {
    if (warp == 0) grid_sum2(gp_ss, G, sh.sums);
    cons_sync();
    if (tid == 0)
      for (int r = 0; r < NR; ++r) {
        sh.eta[r] = sh.eta0[r] = sh.sums[r];
        sh.done[r] = (sh.sums[r] == 0.0) ? 1 : 0;
      }
    // p_0 = s_0 (staged from the s every CTA wrote), q_0 = D^{-1} W p_0
    for (int64_t e = (int64_t)tid * 4; e < E; e += 4 * kFcThreads)
      *reinterpret_cast<float4*>(vs + e) = ldcg4(a.s + e);
    cons_sync();
    {
      const int64_t e_lo = (int64_t)blockIdx.x * E / G, e_hi = (int64_t)(blockIdx.x + 1) * E / G;
      for (int64_t e = e_lo + tid; e < e_hi; e += kFcThreads) a.pa[e] = vs[e];
    }
    float qq[2] = {0.f, 0.f};
    w_phase<NR>(a, vs, qq);
    cta_publish2(qq[0], qq[1], sh.dred, gp_qq + 2 * blockIdx.x);
    alive = grid_barrier(a.bar, a.err, fail);
  }
  if (alive) {
    if (warp == 0) grid_sum2(gp_qq, G, sh.sums);
    cons_sync();
    if (tid == 0) { sh.qq[0] = sh.sums[0]; sh.qq[1] = sh.sums[1]; }
    cons_sync();
  }

  // ---- the PCGTLS steps
  trace_at(a, 1);
  int passes = 0;
  for (int j = 0; alive && j < a.steps; ++j) {
    if (sh.done[0] && (NR < 2 || sh.done[1])) break;
    ++passes;
    const int tb = 2 + kFTracePer * j;
    trace_at(a, tb);
    unsigned long long tile_wait = 0;
    float* p_cur = (j & 1) ? a.pb : a.pa;
    float* p_next = (j & 1) ? a.pa : a.pb;
    // ---------------- pass over the CTA's rows: t = A q, partial A^T t, ||t||^2
    {
      float4 qv[NR][VPT], acc[NR][VPT];
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        const int64_t col = ((int64_t)v * kFcThreads + tid) * 4;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          qv[r][v] = (col < npad) ? ldcg4(a.q + r * npad + col) : make_float4(0.f, 0.f, 0.f, 0.f);
          acc[r][v] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      float tt_acc = 0.f;          // warp 0, lane < NV: squares of the row values it totals
      for (int lt = 0; lt < T; ++lt, ++consumed) {
        const int slot = (int)(consumed % S);
        const uint64_t tw0 = (a.trace != nullptr && tid == 0) ? ptx::global_ns() : 0;
        const bool got = ptx::mbar_wait(&sh.full[slot], (uint32_t)((consumed / S) & 1), a.err, 24);
        if (a.trace != nullptr && tid == 0) tile_wait += ptx::global_ns() - tw0;
        const bool tt_on = (j == 0 && lt < kFTraceTiles);
        if (tt_on) trace_at(a, kFTraceTileBase + 5 * lt);
        const float* tile = ring + slot * stage_floats;
        const int rows = (int)min((int64_t)RT, r1 - (r0 + (int64_t)lt * RT));
        float4 av[RT][VPT];
#pragma unroll
        for (int rt = 0; rt < RT; ++rt)
#pragma unroll
          for (int v = 0; v < VPT; ++v) {
            const int64_t col = ((int64_t)v * kFcThreads + tid) * 4;
            av[rt][v] = (rt < rows && col < npad)
                            ? *reinterpret_cast<const float4*>(tile + rt * npad + col)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        float dv[NV];
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
          for (int rt = 0; rt < RT; ++rt) {
            float t = 0.f;
#pragma unroll
            for (int v = 0; v < VPT; ++v) t = dot4(av[rt][v], qv[r][v], t);
            dv[r * RT + rt] = t;
          }
        {
          constexpr int kSh = (NV >= 32) ? 0 : (NV >= 16 ? 1 : (NV >= 8 ? 2 : (NV >= 4 ? 3 : (NV >= 2 ? 4 : 5))));
          const float t = warp_reduce_scatter<NV>(dv);
          if ((lane & ((1 << kSh) - 1)) == 0) sh.red[warp][lane >> kSh] = t;
        }
        if (__syncthreads_or(!got)) {   // a copy never arrived: leave (uniformly) and abort
          if (tid == 0) {
            atomicExch(a.bar + 64, 1u);
            *fail = 1;
          }
          break;
        }
        if (tt_on) trace_at(a, kFTraceTileBase + 5 * lt + 1);
        // every thread holds its part of the tile: refill the stage with tile consumed + S
        if (tid == 0 && issued < total) issue(issued++);
        if (tt_on) trace_at(a, kFTraceTileBase + 5 * lt + 2);
        if (warp == 0 && lane < NV) {
          float t = 0.f;
#pragma unroll
          for (int w2 = 0; w2 < kFcWarps; ++w2) t += sh.red[w2][lane];
          sh.tot[lane] = t;
          tt_acc = fmaf(t, t, tt_acc);             // rows beyond the block are zero
        }
        cons_sync();
        if (tt_on) trace_at(a, kFTraceTileBase + 5 * lt + 3);
#pragma unroll
        for (int rt = 0; rt < RT; ++rt) {
          if (rt >= rows) break;
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            const float c = sh.tot[r * RT + rt];
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
              acc[r][v].x = fmaf(c, av[rt][v].x, acc[r][v].x);
              acc[r][v].y = fmaf(c, av[rt][v].y, acc[r][v].y);
              acc[r][v].z = fmaf(c, av[rt][v].z, acc[r][v].z);
              acc[r][v].w = fmaf(c, av[rt][v].w, acc[r][v].w);
            }
          }
        }
        if (tt_on) trace_at(a, kFTraceTileBase + 5 * lt + 4);
      }
      // this CTA's partial of A^T t and of ||t||^2
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        const int64_t col = ((int64_t)v * kFcThreads + tid) * 4;
        if (col < npad)
#pragma unroll
          for (int r = 0; r < NR; ++r)
            *reinterpret_cast<float4*>(a.part + (int64_t)blockIdx.x * E + r * npad + col) =
                acc[r][v];
      }
      if (warp == 0) {
        const int rl = lane / RT;
        float t0 = (lane < NV && rl == 0) ? tt_acc : 0.f;
        float t1 = (lane < NV && rl == 1) ? tt_acc : 0.f;
        t0 = warp_sumf(t0);
        t1 = warp_sumf(t1);
        if (lane == 0) {
          gp_tt[2 * blockIdx.x] = (double)t0;
          gp_tt[2 * blockIdx.x + 1] = (double)t1;
        }
      }
    }
    trace_at(a, tb + 1);
    if (a.trace != nullptr && blockIdx.x == 0 && tid == 0 && j < kFTraceSteps)
      a.trace[tb + 9] = tile_wait;
    if (!(alive = grid_barrier(a.bar, a.err, fail))) break;
    trace_at(a, tb + 2);
    // ---------------- delta_j, alpha_j (every CTA), column reduction, w and y
    if (warp == 0) grid_sum2(gp_tt, G, sh.sums);
    cons_sync();
    if (tid == 0)
      for (int r = 0; r < NR; ++r) {
        sh.ok[r] = 0;
        if (!sh.done[r]) {
          const double delta = sh.sums[r] - a.sigma2 * sh.qq[r];
          sh.delta[r] = delta;
          sh.ok[r] = (delta > 0.0) ? 1 : 0;
          sh.alpha[r] = sh.ok[r] ? sh.eta[r] / delta : 0.0;
        }
      }
    cons_sync();
    {
      const int64_t e_lo = (int64_t)blockIdx.x * E / G, e_hi = (int64_t)(blockIdx.x + 1) * E / G;
      const int ps = warp;            // partial slice
      for (int64_t e0 = e_lo; e0 < e_hi; e0 += 32) {
        const int64_t e = e0 + lane;
        float t = 0.f;
        if (e < e_hi) {
          // all of this thread's partials in flight at once, then a fixed-order sum
          float pv[kFMaxGrid / kFcWarps];
#pragma unroll
          for (int u = 0; u < kFMaxGrid / kFcWarps; ++u) {
            const int p = ps + kFcWarps * u;
            pv[u] = (p < G) ? __ldcg(a.part + (int64_t)p * E + e) : 0.f;
          }
#pragma unroll
          for (int u = 0; u < kFMaxGrid / kFcWarps; ++u) t += pv[u];
        }
        sh.red2[ps][lane] = t;
        cons_sync();
        if (warp == 0 && e < e_hi) {
          float at = 0.f;
#pragma unroll
          for (int k = 0; k < kFcWarps; ++k) at += sh.red2[k][lane];
          const int r = (int)(e / npad);
          const int64_t jj = e - (int64_t)r * npad;
          if (sh.ok[r]) {
            const float qj = __ldcg(a.q + e);
            a.w[e] = fmaf((float)sh.alpha[r], qj, __ldcg(a.w + e));
            a.y[e] = (at - sig2f * qj) * __ldg(a.dinv + jj);
          }
        }
        cons_sync();
      }
    }
    trace_at(a, tb + 3);
    if (!(alive = grid_barrier(a.bar, a.err, fail))) break;
    trace_at(a, tb + 4);
    // ---------------- v = W^T y, s_{j+1} = s_j - alpha v, ||s_{j+1}||^2
    for (int64_t e = (int64_t)tid * 4; e < E; e += 4 * kFcThreads)
      *reinterpret_cast<float4*>(vs + e) = ldcg4(a.y + e);
    cons_sync();
    {
      float ss[2] = {0.f, 0.f};
      wt_phase<NR>(a, vs, false, sh, ss);
      cta_publish2(ss[0], ss[1], sh.dred, gp_ss + 2 * blockIdx.x);
    }
    trace_at(a, tb + 5);
    if (!(alive = grid_barrier(a.bar, a.err, fail))) break;
    trace_at(a, tb + 6);
    if (warp == 0) grid_sum2(gp_ss, G, sh.sums);
    cons_sync();
    if (tid == 0)
      for (int r = 0; r < NR; ++r) step_flags(sh, r, sh.sums[r], a.cg_tol2);
    cons_sync();
    if (j + 1 >= a.steps || (sh.done[0] && (NR < 2 || sh.done[1]))) break;
    // ---------------- p_{j+1} = s_{j+1} + beta_j p_j, q_{j+1} = D^{-1} W p_{j+1}, ||q||^2
    {
      const float b0 = (float)sh.beta[0], b1 = (NR > 1) ? (float)sh.beta[1] : 0.f;
      for (int64_t e = (int64_t)tid * 4; e < E; e += 4 * kFcThreads) {
        const float4 sv = ldcg4(a.s + e), pv = ldcg4(p_cur + e);
        const float bt = (e < npad) ? b0 : b1;
        *reinterpret_cast<float4*>(vs + e) = make_float4(
            fmaf(bt, pv.x, sv.x), fmaf(bt, pv.y, sv.y), fmaf(bt, pv.z, sv.z), fmaf(bt, pv.w, sv.w));
      }
      cons_sync();
      const int64_t e_lo = (int64_t)blockIdx.x * E / G, e_hi = (int64_t)(blockIdx.x + 1) * E / G;
      for (int64_t e = e_lo + tid; e < e_hi; e += kFcThreads) p_next[e] = vs[e];
      float qq[2] = {0.f, 0.f};
      w_phase<NR>(a, vs, qq);
      cta_publish2(qq[0], qq[1], sh.dred, gp_qq + 2 * blockIdx.x);
    }
    trace_at(a, tb + 7);
    if (!(alive = grid_barrier(a.bar, a.err, fail))) break;
    trace_at(a, tb + 8);
    if (warp == 0) grid_sum2(gp_qq, G, sh.sums);
    cons_sync();
    if (tid == 0) { sh.qq[0] = sh.sums[0]; sh.qq[1] = sh.sums[1]; }
    cons_sync();
  }

  // ---- results for the host (CTA 0); then wait for the copies still in flight
  if (blockIdx.x == 0 && tid == 0) {
    PcgScalars* sc = a.sc;
    for (int r = 0; r < 2; ++r) {
      sc->eta[r] = sh.eta[r];
      sc->eta0[r] = sh.eta0[r];
      sc->beta[r] = sh.beta[r];
      sc->alpha[r] = sh.alpha[r];
      sc->delta[r] = sh.delta[r];
      sc->qq[r] = sh.qq[r];
      sc->done[r] = sh.done[r];
      sc->iters[r] = sh.iters[r];
      sc->not_spd[r] = sh.nspd[r];
    }
    sc->sigma2 = a.sigma2;
    sc->cg_tol2 = a.cg_tol2;
    sc->nr = NR;
    sc->passes = passes;
  }
  if (tid == 0)
    for (int64_t kk = consumed; kk < issued; ++kk)
      ptx::mbar_wait(&sh.full[kk % S], (uint32_t)((kk / S) & 1), a.err, 23);
}

template <int NR, int VPT, int RT>
cudaError_t launch_one(const FusedArgs& a, int grid, size_t smem, cudaStream_t st) {
  auto kern = pcg_fused_kernel<NR, VPT, RT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFcThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  void* args[] = {(void*)&a};
  e = cudaLaunchCooperativeKernel((const void*)kern, grid, kFcThreads, args, smem, st);
  count_launch();
  return e;
}

}  // namespace

// Ring geometry for npad: rows per tile (a power of two, tile <= 32 KB), float4 column groups per
// consumer thread; 0 when npad is outside the kernel's range.
static bool fused_geometry(int64_t npad, int nr, int* vpt, int* rt, int* stages, size_t* smem) {
  if (npad < 64 || npad > 8192 || npad % 4 != 0) return false;
  const int v = (int)((npad + 4 * kFcThreads - 1) / (4 * kFcThreads));
  int r = 1;
  while (r < 8 && (int64_t)(2 * r) * npad * 4 <= kFTileMaxBytes) r *= 2;
  const size_t tile = (size_t)r * npad * 4;
  const size_t vec = (size_t)nr * npad * 4;
  const size_t budget = 227 * 1024 - sizeof(FusedShared) - 1024;
  if (vec + 2 * tile > budget) return false;
  int s = (int)std::min<size_t>(kFMaxStages, (budget - vec) / tile);
  *vpt = v;
  *rt = r;
  *stages = s;
  *smem = (size_t)s * tile + vec;
  return true;
}

int pcg_fused_trace_words() { return kFTraceTileBase + 5 * kFTraceTiles; }

bool pcg_fused_supported(int64_t npad, int nr) {
  int v, r, s;
  size_t sm;
  return fused_geometry(npad, nr, &v, &r, &s, &sm);
}

cudaError_t launch_pcg_fused(const float* A, int64_t m, int64_t n, int64_t npad, int nr,
                             const double* fin0, double fin0_scale, const double* fin1,
                             const double* dinv64, const float* dinv, const float* W,
                             const float* WT, float* w, float* y, float* s, float* pa, float* pb,
                             float* q, float* part, double* gpart, PcgScalars* sc, double sigma2,
                             double cg_tol, int steps, unsigned int* bar, int* err, int num_sms,
                             cudaStream_t st, unsigned long long* trace) {
  int vpt, rt, stages;
  size_t smem;
  if (!fused_geometry(npad, nr, &vpt, &rt, &stages, &smem)) return cudaErrorInvalidValue;
  FusedArgs a{};
  a.A = A; a.m = m; a.n = n; a.npad = npad; a.nr = nr; a.steps = steps; a.stages = stages;
  a.tile_rows = rt; a.fin0 = fin0; a.fin0_scale = fin0_scale; a.fin1 = fin1;
  a.dinv64 = dinv64; a.dinv = dinv; a.W = W; a.WT = WT; a.w = w; a.y = y; a.s = s; a.pa = pa;
  a.pb = pb; a.q = q; a.part = part; a.gpart = gpart; a.sc = sc; a.sigma2 = sigma2;
  a.cg_tol2 = cg_tol * cg_tol; a.bar = bar; a.err = err; a.trace = trace;
  const int grid = num_sms;
  if (grid > kFMaxGrid) return cudaErrorInvalidValue;
  // the solution starts at zero (w_0 = 0)
  cudaError_t e = cudaMemsetAsync(w, 0, sizeof(float) * (size_t)nr * npad, st);
  if (e != cudaSuccess) return e;
#define TLS_FUSED_CASE(NR_, V_, R_) \
  if (nr == NR_ && vpt == V_ && rt == R_) return launch_one<NR_, V_, R_>(a, grid, smem, st);
  TLS_FUSED_CASE(1, 1, 8) TLS_FUSED_CASE(1, 1, 4) TLS_FUSED_CASE(1, 2, 2)
  TLS_FUSED_CASE(1, 3, 1) TLS_FUSED_CASE(1, 4, 1)
  TLS_FUSED_CASE(2, 1, 8) TLS_FUSED_CASE(2, 1, 4) TLS_FUSED_CASE(2, 2, 2)
  TLS_FUSED_CASE(2, 3, 1) TLS_FUSED_CASE(2, 4, 1)
#undef TLS_FUSED_CASE
  return cudaErrorInvalidValue;
}

}  // namespace tls
