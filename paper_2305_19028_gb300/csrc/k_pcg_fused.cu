// One PCGTLS solve (Alg. 3, the A-explicit operator; one or two right-hand sides) in a single
// persistent cooperative launch, FP32 working precision (the u_p of Alg. 4), scalars included.
//
// The iteration is preconditioned CG for K w = f, K = A^T A - sigma^2 I, with the preconditioner
// applied as one product with M = (R^T R)^{-1} = D^{-1} W W^T D^{-1} (W = R_H^{-1}, R = R_H D,
// formed once per factor): Alg. 3's s_j = R^{-T} r_j and q_j = R^{-1} p_j become z_j = M r_j,
// eta_j = ||s_j||^2 = r_j^T z_j and the search direction d_j = q_j = z_j + beta_{j-1} d_{j-1},
// the same iterates in exact arithmetic with one product per step instead of two dependent ones.
// delta_j = ||A d_j||^2 - sigma^2 ||d_j||^2 is evaluated as d_j^T (A^T A d_j - sigma^2 d_j), the
// same number in exact arithmetic, from the vector every CTA already needs.
//
// Every CTA is resident (one per SM, 16 warps). A CTA owns a contiguous block of rows of the FP32
// copy of A and streams it, step after step, through a ring of shared-memory stages filled by
// 1-D bulk asynchronous copies (TMA, completion on mbarriers). Every CTA keeps the whole residual
// r in shared memory and each thread the columns of d it multiplies with. Per step j:
//
//   pass    t = A d_j row by row from the ring; the CTA's share of A^T t is added into a vector
//           in global memory with vector atomics                            -- grid barrier 1
//   update  K d = A^T t - sigma^2 d for the thread's columns; delta_j = d^T K d and alpha_j
//           (every CTA, from the whole vectors); r -= alpha K d (every CTA the whole vector),
//           w += alpha d (the CTA's slice)
//   M       z = M r for the rows each warp owns                             -- grid barrier 2
//   next    eta_{j+1} = r^T z, beta_j and the stop flags (every CTA alike); d_{j+1} = z + beta d
//
// Every CTA adds the same numbers in the same order for each scalar, so all take identical
// decisions without exchanging them. A^T t is summed either in a fixed order (the default,
// bitwise reproducible: each CTA writes its share, then after barrier 1 every CTA adds the
// shares of its slice of the entries in CTA order, forms its slice of K d and its part of
// d^T K d, and a second grid barrier follows) or with float vector atomics (one barrier less;
// the order of the adds, and so the last bits, can change from run to run). What keeps the step short on this GPU, where a dependent round trip to
// L2 costs about a microsecond and FP64 arithmetic is slow:
//  * two grid barriers per step, each one atomic add and one polled word per CTA;
//  * scalars in FP32, combined by warp shuffles (no FP64 on the critical path);
//  * each warp loads the leading part of its row of M into registers before it is needed;
//  * in the pass no CTA barrier per tile: a warp waits only for the row values of a tile it needs
//    for its axpy (the last warp to publish its share of a tile's dot products adds the shares),
//    and the last warp done with a stage refills it; when a pass ends the first stages of the
//    next pass are already in flight, so HBM keeps streaming through the step's tail. A variant
//    with one CTA barrier per tile and the tile held in registers across it is kept for the
//    cp.async loading mode and for comparison.
//
// Every wait is bounded: mbarrier waits by a global-timer deadline, grid barriers by a deadline
// and an abort word that a CTA whose wait expired raises, so that the others leave too; a CTA
// waits for its own copies in flight before it exits. Error codes land in *err.
#include "tls_internal.h"
#include "tls_ptx.cuh"

#include <algorithm>

namespace tls {
namespace {

constexpr int kW = 16;                         // warps per CTA
constexpr int kT = kW * 32;                    // 512 threads
constexpr int kFMaxStages = 8;
constexpr int kFMaxGrid = 256;                 // CTAs of the launch at most (one per SM)
constexpr int kFMaxRows = 4;                   // rows of W / W^T per warp at most
constexpr int kFMaxSlice = 256;                // entries of the column slice per CTA at most
constexpr int kPre = 8;                        // float4 per lane of a prefetched row of M
constexpr uint64_t kFBarrierNs = 2000ull * 1000 * 1000;   // grid barrier deadline: 2 s

struct FusedArgs {
  const float* A;        // m x npad, row-major, rows back to back (lda = npad)
  int64_t m, n, npad;
  int nr, steps, stages;
  const double* fin0;    // right-hand side 0 is fin0_scale * fin0, 1 is fin1 (FP64, n values)
  double fin0_scale;
  const double* fin1;
  const float* M;        // the preconditioner (R^T R)^{-1} = D^{-1} W W^T D^{-1}, npad x npad
  float* w;              // solutions, nr x npad (written at the end)
  float* z;              // M r, nr x npad
  float* atd;            // atomic form: A^T t of the passes, 2 x nr x npad (alternating between
                         // steps, accumulated by every CTA with vector atomics); fixed-order
                         // form: K d, nr x npad
  float* part;           // fixed-order form: the CTAs' shares of A^T t (G x nr x npad), then
                         // their shares of d^T K d (G x 2)
  int det;               // 1: the fixed-order form (bitwise reproducible, one more grid barrier)
  PcgScalars* sc;
  double sigma2, cg_tol2;
  unsigned int* bar;     // [0] grid-barrier counter, [64] abort word (both zero between launches)
  int* err;
  unsigned long long* trace;   // optional phase timestamps of CTA 0
  int load_mode;         // how a tile reaches shared memory (see issue_next)
  int keep_tiles;        // the first keep_tiles tiles of every CTA's block are loaded with an
                         // L2 evict-last policy (they stay resident across the steps), the rest
                         // with evict-first
};

// Trace layout (global-timer nanoseconds, CTA 0, thread 0): [0] start, [1] initialisation done,
// then per step j < kFTraceSteps, at 2 + kFTracePer * j: pass start, pass end, barrier 1 done,
// slice done, barrier 2 done, M product done, barrier 3 done, next direction done (twice), and
// the time thread 0 spent waiting for tiles of that pass.
// After them, for the grid barriers b (0: after the pass, 2: after the M product) of steps
// j < kFArrSteps (index i = 3 j + b): the time every CTA c arrived at the barrier, at
// kFTraceMain + i kFMaxGrid + c, and the time its arrival was counted, kFArrSteps * 3 * kFMaxGrid
// words further on; then, for CTA 0, the time it saw the last arrival and the time its acquire
// fence completed, at kFTraceCta0 + 2 i.
constexpr int kFTracePer = 10;
constexpr int kFTraceSteps = 64;
constexpr int kFTraceMain = 2 + kFTracePer * kFTraceSteps;
constexpr int kFArrSteps = 8;
constexpr int kFTraceCta0 = kFTraceMain + 2 * 3 * kFArrSteps * kFMaxGrid;
constexpr int kFTraceWords = kFTraceCta0 + 2 * 3 * kFArrSteps;

__device__ __forceinline__ void trace_at(const FusedArgs& a, int idx) {
  if (a.trace != nullptr && blockIdx.x == 0 && threadIdx.x == 0 && idx < kFTraceWords)
    a.trace[idx] = ptx::global_ns();
}

__device__ __forceinline__ unsigned int ld_acquire32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ float warp_sumf(float v) {
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
__device__ __forceinline__ float4 f4zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

struct alignas(16) FusedShared {
  uint64_t full[kFMaxStages];
  uint64_t totb[2];             // decoupled pass: row values of tile k ready (buffer k & 1)
  int rcnt[2];                  // ... warps that published their share of tile k
  int ecnt[kFMaxStages];        // ... warps done with the tile in a stage
  float red[2][kW][16];         // per-warp row values of a tile (double-buffered)
  float red2[kW][33];           // fixed-order form: partial sums of the slice reduction
  float tot[2][16];             // row values of a tile summed over the warps
  float cta2[kW][2];
  float w_sl[kFMaxSlice];       // this CTA's slice of w
  float d_sl[kFMaxSlice];       // ... of the search direction d (= q of Alg. 3)
  float sums[2];
  // the PCGTLS scalars in the working precision u_p (FP32): FP64 arithmetic on this GPU runs at a
  // small fraction of the FP32 rate and would sit on the critical path of every step
  float eta[2], eta0[2], beta[2], delta[2], alpha[2];
  int done[2], iters[2], nspd[2], ok[2];
  int fail;
};

__device__ __forceinline__ unsigned int ld_relaxed32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Barrier over every CTA of the launch on one counter word (bar[0]): thread 0 of each CTA fences
// the CTA's writes and adds 1 (CTA 0 adds 2^31 - (G - 1)), so the word's top bit flips once all
// G CTAs have arrived and its low bits return to their value before the barrier; thread 0 polls
// the word (one load per round) until the bit differs from the one its own add saw, then fences.
// Returns false when abandoned (deadline here, or the abort word bar[64] raised elsewhere). All
// threads must call it.
__device__ __forceinline__ bool grid_sync(const FusedArgs& a, FusedShared& sh, int arr = -1) {
  __syncthreads();                      // this CTA's global writes of the phase are done
  if (threadIdx.x == 0) {
    const bool tr = a.trace != nullptr && arr >= 0 && arr < 3 * kFArrSteps;
    if (tr) a.trace[kFTraceMain + arr * kFMaxGrid + blockIdx.x] = ptx::global_ns();
    const unsigned int nb = (blockIdx.x == 0) ? (0x80000000u - (gridDim.x - 1u)) : 1u;
    __threadfence();
    const unsigned int old = atomicAdd(a.bar, nb);
    if (tr)
      a.trace[kFTraceMain + (3 * kFArrSteps + arr) * kFMaxGrid + blockIdx.x] = ptx::global_ns();
    const uint64_t t0 = ptx::global_ns();
    unsigned int it = 0;
    while (((old ^ ld_relaxed32(a.bar)) & 0x80000000u) == 0u) {
      if ((++it & 63u) == 0) {
        if (ld_acquire32(a.bar + 64) != 0u) {
          sh.fail = 1;
          break;
        }
        if (ptx::global_ns() - t0 > kFBarrierNs) {
          atomicCAS(a.err, 0, 21);
          atomicExch(a.bar + 64, 1u);
          sh.fail = 1;
          break;
        }
      }
    }
    if (tr && blockIdx.x == 0) a.trace[kFTraceCta0 + 2 * arr] = ptx::global_ns();
    __threadfence();   // the arrivals were observed: later reads see what the CTAs wrote before
    if (tr && blockIdx.x == 0) a.trace[kFTraceCta0 + 2 * arr + 1] = ptx::global_ns();
  }
  __syncthreads();
  return sh.fail == 0;
}

// CTA sums of two per-thread FP32 values into sh.sums (warp sums, then the 16 warp sums added by
// a butterfly over the lanes of warp 0: the same order in every CTA), visible to every thread on
// return (all threads call it).
__device__ __forceinline__ void cta_sum2(float v0, float v1, FusedShared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v0 = warp_sumf(v0);
  v1 = warp_sumf(v1);
  if (lane == 0) {
    sh.cta2[warp][0] = v0;
    sh.cta2[warp][1] = v1;
  }
  __syncthreads();
  if (warp == 0) {
    float t0 = (lane < kW) ? sh.cta2[lane][0] : 0.f;
    float t1 = (lane < kW) ? sh.cta2[lane][1] : 0.f;
#pragma unroll
    for (int o = kW / 2; o > 0; o >>= 1) {
      t0 += __shfl_xor_sync(0xffffffffu, t0, o);
      t1 += __shfl_xor_sync(0xffffffffu, t1, o);
    }
    if (lane == 0) {
      sh.sums[0] = t0;
      sh.sums[1] = t1;
    }
  }
  __syncthreads();
}

// Loads the first kPre float4 of the lane's share of a row (columns c0 + lane*4 + 128 u, u < kPre)
// below lim.
__device__ __forceinline__ void prefetch_row(const float* row, int64_t c0, int64_t lim,
                                             float4 (&r)[kPre]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int u = 0; u < kPre; ++u) {
    const int64_t c = c0 + (int64_t)lane * 4 + (int64_t)u * 128;
    r[u] = (c < lim) ? __ldg(reinterpret_cast<const float4*>(row + c)) : f4zero();
  }
}

// Dot products of a row (entries [c0, lim)) with the one or two staged vectors: the first
// 128 * kPre entries from the prefetched registers pre, the rest loaded here into the same
// registers (they are free by then). Warp totals in a0, a1.
template <int NR>
__device__ __forceinline__ void row_dot(const float* row, int64_t c0, int64_t lim,
                                        float4 (&pre)[kPre], const float* vs, int64_t npad,
                                        float& a0, float& a1) {
  const int lane = threadIdx.x & 31;
  for (int64_t cb = c0; cb < lim; cb += 128 * kPre) {
    if (cb != c0) prefetch_row(row, cb, lim, pre);
#pragma unroll
    for (int u = 0; u < kPre; ++u) {
      const int64_t c = cb + (int64_t)lane * 4 + (int64_t)u * 128;
      if (c < lim) {
        a0 = dot4(pre[u], *reinterpret_cast<const float4*>(vs + c), a0);
        if (NR > 1) a1 = dot4(pre[u], *reinterpret_cast<const float4*>(vs + npad + c), a1);
      }
    }
  }
  a0 = warp_sumf(a0);
  if (NR > 1) a1 = warp_sumf(a1);
}

// z_i = M_i . r for the warp's rows i = gw, gw + GW, ... (the first row's leading chunk already in
// pre); lane 0 writes z_i
template <int NR>
__device__ __forceinline__ void m_phase(const FusedArgs& a, const float* vs, float4 (&pre)[kPre],
                                        int64_t gw, int64_t GW, int64_t npad) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < kFMaxRows; ++k) {
    const int64_t i = gw + k * GW;
    if (i >= npad) break;
    if (k > 0) prefetch_row(a.M + i * npad, 0, npad, pre);
    float v0 = 0.f, v1 = 0.f;
    row_dot<NR>(a.M + i * npad, 0, npad, pre, vs, npad, v0, v1);
    if (lane == 0) {
      a.z[i] = v0;
      if (NR > 1) a.z[npad + i] = v1;
    }
  }
}

// eta_{j+1}, beta_j and the termination flags of Alg. 3 for right-hand side r (thread 0).
__device__ __forceinline__ void step_flags(FusedShared& sh, int r, float eta_new, float tol2) {
  if (sh.done[r]) return;
  if (!sh.ok[r]) {                 // delta_j <= 0: "while delta_j != 0"; < 0 is loss of SPD
    sh.done[r] = 1;
    sh.nspd[r] = (sh.delta[r] < 0.f) ? 1 : 0;
    return;
  }
  sh.beta[r] = eta_new / sh.eta[r];
  sh.eta[r] = eta_new;
  sh.iters[r] += 1;
  if (eta_new == 0.f || (tol2 > 0.f && eta_new <= tol2 * sh.eta0[r])) sh.done[r] = 1;
}

// State of a CTA's pass over its rows (shared by the tile steps below). The ring positions are
// kept as small counters (no 64-bit division per tile): c_slot / c_phase the stage and mbarrier
// parity of the next tile to consume, i_slot / i_lt the stage and local tile index of the next
// tile to issue.
struct PassState {
  float* ring;
  int64_t stage_floats;
  int S;
  int64_t r0, r1;
  int T;
  int64_t npad, total;
  int64_t consumed, issued;     // tiles consumed / copies issued
  int c_slot, i_slot, i_lt;
  uint32_t c_phase;
  uint64_t pol_keep;            // L2 policy of the tiles kept resident
  unsigned long long tile_wait; // thread 0: ns spent waiting for tiles (trace)
  bool gotall;
  int64_t kd, ka;               // decoupled pass: tiles whose dot products / axpy this warp did
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint64_t pol) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(
                   ptx::smem_u32(dst)),
               "l"(src), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(ptx::smem_u32(bar))
               : "memory");
}

// Starts the copy of the CTA's next tile in sequence (stage ps.i_slot, local tile ps.i_lt) and
// advances the issue position. Every thread calls it. load_mode 0: one 1-D bulk copy (TMA) of the
// tile by thread 0; 1: one bulk copy per row by thread 0; 2: every thread copies 16-byte chunks
// with cp.async and arrives on the mbarrier when its chunks have landed (the mbarrier then
// counts kT arrivals).
// The copy of local tile i_lt into stage slot by the calling thread (load modes 0 and 1: one
// bulk copy (TMA) of the tile, or one per row).
template <int RT>
__device__ __forceinline__ void issue_copy(const FusedArgs& a, FusedShared& sh, const PassState& ps,
                                           int slot, int i_lt, uint64_t pol_stream) {
  const uint64_t pol = (i_lt < a.keep_tiles) ? ps.pol_keep : pol_stream;
  const int64_t row = ps.r0 + (int64_t)i_lt * RT;
  const int rows = (int)min((int64_t)RT, ps.r1 - row);
  float* dst = ps.ring + slot * ps.stage_floats;
  const float* src = a.A + row * ps.npad;
  const uint32_t bytes = (uint32_t)(rows * ps.npad * (int64_t)sizeof(float));
  ptx::mbar_expect_tx(&sh.full[slot], bytes);
  if (a.load_mode == 0) {
    ptx::bulk_g2s_hint(dst, src, bytes, &sh.full[slot], pol);
  } else {
    const uint32_t rb = (uint32_t)(ps.npad * sizeof(float));
    for (int r = 0; r < rows; ++r)
      ptx::bulk_g2s_hint(dst + r * ps.npad, src + r * ps.npad, rb, &sh.full[slot], pol);
  }
}

// Advances the issue position (stage, local tile) by one copy.
__device__ __forceinline__ void advance_issue(PassState& ps) {
  ++ps.issued;
  if (++ps.i_slot == ps.S) ps.i_slot = 0;
  if (++ps.i_lt == ps.T) ps.i_lt = 0;
}

// Starts the copy of the CTA's next tile in sequence (stage ps.i_slot, local tile ps.i_lt) and
// advances the issue position. Every thread calls it. load_mode 0 / 1: thread 0 issues bulk
// copies; 2: every thread copies 16-byte chunks with cp.async and arrives on the mbarrier when
// its chunks have landed (the mbarrier then counts kT arrivals).
template <int RT>
__device__ __forceinline__ void issue_next(const FusedArgs& a, FusedShared& sh, PassState& ps,
                                           uint64_t pol_stream) {
  const int slot = ps.i_slot, i_lt = ps.i_lt;
  advance_issue(ps);
  if (a.load_mode == 2) {
    const uint64_t pol = (i_lt < a.keep_tiles) ? ps.pol_keep : pol_stream;
    const int64_t row = ps.r0 + (int64_t)i_lt * RT;
    const int rows = (int)min((int64_t)RT, ps.r1 - row);
    float* dst = ps.ring + slot * ps.stage_floats;
    const float* src = a.A + row * ps.npad;
    const int chunks = (int)((int64_t)rows * ps.npad / 4);
    for (int c = threadIdx.x; c < chunks; c += kT) cp_async16(dst + 4 * c, src + 4 * c, pol);
    cp_async_arrive(&sh.full[slot]);
    return;
  }
  if (threadIdx.x == 0) issue_copy<RT>(a, sh, ps, slot, i_lt, pol_stream);
}

// One tile step of the pipelined pass: the dot products of local tile lt (its rows into the
// registers cur and the per-warp row values into red[lt & 1]) and the cross-warp sums of tile
// lt - 1, one CTA barrier, then the refill of tile lt's stage and the axpy of tile lt - 1 from
// the registers prev. Returns false (uniformly) when a copy never arrived.
template <int NR, int VPT, int RT>
__device__ __forceinline__ bool pass_tile(const FusedArgs& a, FusedShared& sh, PassState& ps,
                                          const float4 (&qv)[NR][VPT], float4 (&acc)[NR][VPT],
                                          float4 (&cur)[RT][VPT], float4 (&prev)[RT][VPT], int lt,
                                          uint64_t pol) {
  constexpr int NV = NR * RT;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (lt < ps.T) {
    const int slot = ps.c_slot;
    const uint64_t tw0 = (a.trace != nullptr && tid == 0) ? ptx::global_ns() : 0;
    const bool got = ptx::mbar_wait(&sh.full[slot], ps.c_phase, a.err, 24);
    if (a.trace != nullptr && tid == 0) ps.tile_wait += ptx::global_ns() - tw0;
    ps.gotall = ps.gotall && got;
    if (got) {                 // a tile that never arrived stays in the drain at the end
      ++ps.consumed;
      if (++ps.c_slot == ps.S) {
        ps.c_slot = 0;
        ps.c_phase ^= 1u;
      }
    }
    const float* tile = ps.ring + slot * ps.stage_floats;
    const int rows = (int)min((int64_t)RT, ps.r1 - (ps.r0 + (int64_t)lt * RT));
#pragma unroll
    for (int rt = 0; rt < RT; ++rt)
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        const int64_t col = ((int64_t)v * kT + tid) * 4;
        cur[rt][v] = (rt < rows && col < ps.npad)
                         ? *reinterpret_cast<const float4*>(tile + rt * ps.npad + col)
                         : f4zero();
      }
    float dv[NV];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int rt = 0; rt < RT; ++rt) {
        float t = 0.f;
#pragma unroll
        for (int v = 0; v < VPT; ++v) t = dot4(cur[rt][v], qv[r][v], t);
        dv[r * RT + rt] = t;
      }
    constexpr int kSh = (NV >= 16 ? 1 : (NV >= 8 ? 2 : (NV >= 4 ? 3 : (NV >= 2 ? 4 : 5))));
    const float t = warp_reduce_scatter<NV>(dv);
    if ((lane & ((1 << kSh) - 1)) == 0) sh.red[lt & 1][warp][lane >> kSh] = t;
  }
  if (lt >= 1 && warp < NV) {
    // warp w < NV: row value w of tile lt - 1 summed over the warps
    const int b = (lt - 1) & 1;
    float x = (lane < kW) ? sh.red[b][lane][warp] : 0.f;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh.tot[b][warp] = x;
  }
  if (__syncthreads_or(!ps.gotall)) return false;
  // every thread holds tile lt in registers: refill its stage
  if (lt < ps.T && ps.issued < ps.total) issue_next<RT>(a, sh, ps, pol);
  if (lt >= 1) {
    const int b = (lt - 1) & 1;
    const int rows = (int)min((int64_t)RT, ps.r1 - (ps.r0 + (int64_t)(lt - 1) * RT));
#pragma unroll
    for (int rt = 0; rt < RT; ++rt) {
      if (rt >= rows) break;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const float c = sh.tot[b][r * RT + rt];
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          acc[r][v].x = fmaf(c, prev[rt][v].x, acc[r][v].x);
          acc[r][v].y = fmaf(c, prev[rt][v].y, acc[r][v].y);
          acc[r][v].z = fmaf(c, prev[rt][v].z, acc[r][v].z);
          acc[r][v].w = fmaf(c, prev[rt][v].w, acc[r][v].w);
        }
      }
    }
  }
  return true;
}

__device__ __forceinline__ void mbar_arrive_cta(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(ptx::smem_u32(bar))
               : "memory");
}

// The pass with the warps decoupled (no CTA barrier): tiles stay in their stage until every warp
// has done its axpy with them. Per tile k a warp computes its dot products and publishes its
// share of the row values (red[k & 1]); the warp that publishes last adds the 16 shares in warp
// order (the same sums as the CTA-barrier form) and arrives on totb[k & 1]. A warp does the axpy of tile k - 1 once totb says its row values are ready, so a
// warp waits only for the data it needs and the others keep working; the last warp done with a
// stage refills it. Load modes 0 and 1 only. Returns false when a wait expired.
template <int NR, int VPT, int RT>
__device__ __forceinline__ bool pass_decoupled(const FusedArgs& a, FusedShared& sh, PassState& ps,
                                               const float4 (&qv)[NR][VPT],
                                               float4 (&acc)[NR][VPT], uint64_t pol) {
  constexpr int NV = NR * RT;
  constexpr int kSh = (NV >= 16 ? 1 : (NV >= 8 ? 2 : (NV >= 4 ? 3 : (NV >= 2 ? 4 : 5))));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  bool ok = true;
  int prev_slot = 0;
  for (int lt = 0; lt <= ps.T; ++lt) {
    int slot = 0;
    if (lt < ps.T) {
      slot = ps.c_slot;
      const uint64_t tw0 = (a.trace != nullptr && tid == 0) ? ptx::global_ns() : 0;
      const bool got = ptx::mbar_wait(&sh.full[slot], ps.c_phase, a.err, 24);
      if (a.trace != nullptr && tid == 0) ps.tile_wait += ptx::global_ns() - tw0;
      ok = ok && got;
      if (got) {
        ++ps.consumed;
        if (++ps.c_slot == ps.S) {
          ps.c_slot = 0;
          ps.c_phase ^= 1u;
        }
      }
      const float* tile = ps.ring + slot * ps.stage_floats;
      const int rows = (int)min((int64_t)RT, ps.r1 - (ps.r0 + (int64_t)lt * RT));
      float dv[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) dv[i] = 0.f;
#pragma unroll
      for (int rt = 0; rt < RT; ++rt)
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          const int64_t col = ((int64_t)v * kT + tid) * 4;
          const float4 x = (rt < rows && col < ps.npad)
                               ? *reinterpret_cast<const float4*>(tile + rt * ps.npad + col)
                               : f4zero();
#pragma unroll
          for (int r = 0; r < NR; ++r) dv[r * RT + rt] = dot4(x, qv[r][v], dv[r * RT + rt]);
        }
      const float t = warp_reduce_scatter<NV>(dv);
      const int b = (int)(ps.kd & 1);
      if ((lane & ((1 << kSh) - 1)) == 0) sh.red[b][warp][lane >> kSh] = t;
      __syncwarp();
      int last = 0;
      if (lane == 0) {
        __threadfence_block();
        last = (atomicAdd(&sh.rcnt[b], 1) == kW - 1) ? 1 : 0;
      }
      if (__shfl_sync(0xffffffffu, last, 0)) {
        __threadfence_block();
        if (lane < NV) {
          float x = 0.f;
#pragma unroll
          for (int w2 = 0; w2 < kW; ++w2) x += sh.red[b][w2][lane];
          sh.tot[b][lane] = x;
        }
        __syncwarp();
        if (lane == 0) {
          sh.rcnt[b] = 0;
          mbar_arrive_cta(&sh.totb[b]);
        }
      }
      ++ps.kd;
    }
    if (lt >= 1) {
      const int b = (int)(ps.ka & 1);
      ok = ptx::mbar_wait(&sh.totb[b], (uint32_t)((ps.ka >> 1) & 1), a.err, 25) && ok;
      const float* tile = ps.ring + prev_slot * ps.stage_floats;
      const int rows = (int)min((int64_t)RT, ps.r1 - (ps.r0 + (int64_t)(lt - 1) * RT));
#pragma unroll
      for (int rt = 0; rt < RT; ++rt) {
        if (rt >= rows) break;
        float c[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) c[r] = sh.tot[b][r * RT + rt];
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          const int64_t col = ((int64_t)v * kT + tid) * 4;
          if (col < ps.npad) {
            const float4 x = *reinterpret_cast<const float4*>(tile + rt * ps.npad + col);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
              acc[r][v].x = fmaf(c[r], x.x, acc[r][v].x);
              acc[r][v].y = fmaf(c[r], x.y, acc[r][v].y);
              acc[r][v].z = fmaf(c[r], x.z, acc[r][v].z);
              acc[r][v].w = fmaf(c[r], x.w, acc[r][v].w);
            }
          }
        }
      }
      // the stage of tile lt - 1 is free once every warp is past this point: the last refills it
      // (the copies are issued in tile order, so ps.i_slot is that stage)
      __syncwarp();
      if (lane == 0 && atomicAdd(&sh.ecnt[prev_slot], 1) == kW - 1) {
        sh.ecnt[prev_slot] = 0;
        if (ps.issued < ps.total) issue_copy<RT>(a, sh, ps, ps.i_slot, ps.i_lt, pol);
      }
      if (ps.issued < ps.total) advance_issue(ps);
      ++ps.ka;
    }
    prev_slot = slot;
  }
  return ok;
}

template <int NR, int VPT, int RT, bool HOLD>
__global__ void __launch_bounds__(kT, 1) pcg_fused_kernel(const FusedArgs a) {
  extern __shared__ __align__(128) unsigned char fsm[];
  __shared__ FusedShared sh;
  constexpr int NV = NR * RT;          // row values per tile
  static_assert(NV <= 16 && (NV & (NV - 1)) == 0, "row values per tile: a power of two <= 16");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = (int)gridDim.x;
  const int64_t npad = a.npad, E = (int64_t)NR * npad;
  const int S = a.stages;
  const int64_t stage_floats = (int64_t)RT * npad;
  float* ring = reinterpret_cast<float*>(fsm);
  float* vs = ring + (int64_t)S * stage_floats;     // the residual r (NR x npad), in every CTA
  // this CTA's rows of A and its tiles
  const int64_t per = (a.m + G - 1) / G;
  const int64_t r0 = min(a.m, (int64_t)blockIdx.x * per);
  const int64_t r1 = min(a.m, r0 + per);
  const int T = (r1 > r0) ? (int)((r1 - r0 + RT - 1) / RT) : 0;
  // this CTA's slice of the entries of the nr x npad vectors (w and d there are kept in shared
  // memory; the slice of A^T t is the one it clears) and each warp's rows of M
  const int64_t e_lo = (int64_t)blockIdx.x * E / G, e_hi = (int64_t)(blockIdx.x + 1) * E / G;
  const int nsl = (int)(e_hi - e_lo);
  const int64_t GW = (int64_t)G * kW, gw = (int64_t)blockIdx.x * kW + warp;

  // the CTA's tiles in sequence: tile k is local tile k % T of pass k / T
  const int64_t total = (int64_t)a.steps * T;
  const uint64_t pol = ptx::policy_evict_first();   // rows of A not kept in L2
  trace_at(a, 0);
  if (tid == 0) {
    for (int k = 0; k < S; ++k) {
      ptx::mbar_init(&sh.full[k], (HOLD && a.load_mode == 2) ? kT : 1);
      sh.ecnt[k] = 0;
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&sh.totb[b], 1);
      sh.rcnt[b] = 0;
    }
    ptx::fence_mbar_init();
    sh.fail = 0;
  }
  __syncthreads();
  uint64_t pol_keep;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol_keep));
  PassState ps{ring, stage_floats, S, r0, r1, T, npad, total, 0, 0, 0, 0, 0, 0u, pol_keep, 0ull,
               true, 0, 0};
  while (ps.issued < S && ps.issued < total) issue_next<RT>(a, sh, ps, pol);

  // ---- initialisation: r_0 = f (every CTA the whole vector), z_0 = M r_0, eta_0 = r_0^T z_0,
  // d_0 = z_0; both A^T t buffers cleared (each CTA its slice)
  float4 pre[kPre];
  if (gw < npad) prefetch_row(a.M + gw * npad, 0, npad, pre);
  for (int64_t j = tid; j < npad; j += kT) {
    double f0 = 0.0, f1 = 0.0;
    if (j < a.n) {
      f0 = a.fin0_scale * a.fin0[j];
      if (NR > 1) f1 = a.fin1[j];
    }
    vs[j] = (float)f0;
    if (NR > 1) vs[npad + j] = (float)f1;
  }
  if (tid == 0) {
    for (int r = 0; r < 2; ++r) {
      sh.eta[r] = sh.eta0[r] = sh.beta[r] = sh.alpha[r] = 0.f;
      sh.delta[r] = 1.f;
      sh.done[r] = (r < NR) ? 0 : 1;
      sh.iters[r] = sh.nspd[r] = 0;
      sh.ok[r] = 1;
    }
  }
  for (int e = tid; e < nsl; e += kT) {
    sh.w_sl[e] = 0.f;
    a.atd[e_lo + e] = 0.f;
    a.atd[E + e_lo + e] = 0.f;
  }
  __syncthreads();
  m_phase<NR>(a, vs, pre, gw, GW, npad);
  bool alive = grid_sync(a, sh);
  // d_0 = z_0: the thread's columns (registers) and the CTA's slice; eta_0 = r_0^T z_0 (every
  // CTA alike, from the whole vectors)
  float4 qv[NR][VPT];
  if (alive) {
    float e0 = 0.f, e1 = 0.f;
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int64_t col = ((int64_t)v * kT + tid) * 4;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        qv[r][v] = f4zero();
        if (col < npad) {
          qv[r][v] = ldcg4(a.z + r * npad + col);
          const float rz = dot4(qv[r][v], *reinterpret_cast<const float4*>(vs + r * npad + col), 0.f);
          if (r == 0) e0 += rz; else e1 += rz;
        }
      }
    }
    for (int e = tid; e < nsl; e += kT) sh.d_sl[e] = __ldcg(a.z + e_lo + e);
    cta_sum2(e0, e1, sh);
    if (tid == 0)
      for (int r = 0; r < NR; ++r) {
        sh.eta[r] = sh.eta0[r] = sh.sums[r];
        sh.done[r] = (sh.sums[r] == 0.f) ? 1 : 0;
      }
  }

  // ---- the PCGTLS steps
  trace_at(a, 1);
  int passes = 0;
  for (int j = 0; alive && j < a.steps; ++j) {
    __syncthreads();
    if (sh.done[0] && (NR < 2 || sh.done[1])) break;
    ++passes;
    const int tb = 2 + kFTracePer * j;
    trace_at(a, tb);
    float* atd = a.atd + (int64_t)(j & 1) * E;
    // ---------------- pass over the CTA's rows: t = A d and the CTA's share of A^T t, added
    // into atd with vector atomics
    bool ok = true;
    {
      float4 acc[NR][VPT];
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int v = 0; v < VPT; ++v) acc[r][v] = f4zero();
      ps.tile_wait = 0ull;
      if constexpr (HOLD) {
        float4 a0[RT][VPT], a1[RT][VPT];
        // one CTA barrier per tile: [dots(lt) | sums(lt - 1)] barrier [refill, axpy(lt - 1)]
        for (int lt = 0; ok && lt <= T; lt += 2) {
          ok = pass_tile<NR, VPT, RT>(a, sh, ps, qv, acc, a0, a1, lt, pol);
          if (ok && lt + 1 <= T)
            ok = pass_tile<NR, VPT, RT>(a, sh, ps, qv, acc, a1, a0, lt + 1, pol);
        }
      } else {
        ok = pass_decoupled<NR, VPT, RT>(a, sh, ps, qv, acc, pol);
      }
      ok = !__syncthreads_or(!ok);
      if (a.det) {
        // the CTA's share of A^T t as its own partial (a CTA without rows writes zeros)
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          const int64_t col = ((int64_t)v * kT + tid) * 4;
          if (col < npad)
#pragma unroll
            for (int r = 0; r < NR; ++r)
              *reinterpret_cast<float4*>(a.part + (int64_t)blockIdx.x * E + r * npad + col) =
                  acc[r][v];
        }
      } else {
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          const int64_t col = ((int64_t)v * kT + tid) * 4;
          if (col < npad && T > 0)
#pragma unroll
            for (int r = 0; r < NR; ++r)
              atomicAdd(reinterpret_cast<float4*>(atd + r * npad + col), acc[r][v]);
        }
      }
    }
    if (!ok && tid == 0) {
      atomicExch(a.bar + 64, 1u);
      sh.fail = 1;
    }
    trace_at(a, tb + 1);
    if (a.trace != nullptr && blockIdx.x == 0 && tid == 0 && j < kFTraceSteps)
      a.trace[tb + 9] = ps.tile_wait;
    if (!(alive = grid_sync(a, sh, 3 * j))) break;
    trace_at(a, tb + 2);
    if (a.det) {
      // fixed-order form: the CTA's slice of K d = (the partials summed in CTA order) - sigma^2 d
      // into atd, and the slice's share of d^T K d; then a grid barrier
      const float sig2f = (float)a.sigma2;
      float* dpart = a.part + (int64_t)G * E;
      float de0 = 0.f, de1 = 0.f;
      for (int c0 = 0; c0 < nsl; c0 += 32) {
        const int e = c0 + lane;
        float t = 0.f;
        if (e < nsl) {
          float pv[kFMaxGrid / kW];
#pragma unroll
          for (int u = 0; u < kFMaxGrid / kW; ++u) {
            const int pc = warp + kW * u;
            pv[u] = (pc < G) ? __ldcg(a.part + (int64_t)pc * E + e_lo + e) : 0.f;
          }
#pragma unroll
          for (int u = 0; u < kFMaxGrid / kW; ++u) t += pv[u];
        }
        sh.red2[warp][lane] = t;
        __syncthreads();
        if (warp == 0 && e < nsl) {
          float at = 0.f;
#pragma unroll
          for (int k = 0; k < kW; ++k) at += sh.red2[k][lane];
          const float dj = sh.d_sl[e];
          const float kdv = fmaf(-sig2f, dj, at);
          a.atd[e_lo + e] = kdv;
          if ((e_lo + e) / npad == 0) de0 = fmaf(dj, kdv, de0);
          else de1 = fmaf(dj, kdv, de1);
        }
        __syncthreads();
      }
      if (warp == 0) {
        de0 = warp_sumf(de0);
        de1 = warp_sumf(de1);
        if (lane == 0) {
          dpart[2 * blockIdx.x] = de0;
          dpart[2 * blockIdx.x + 1] = de1;
        }
      }
      if (!(alive = grid_sync(a, sh, 3 * j + 1))) break;
    }
    // ---------------- K d = A^T t - sigma^2 d (the thread's columns, registers);
    // delta_j = d^T K d (= ||A d||^2 - sigma^2 ||d||^2), alpha_j = eta_j / delta_j (every CTA
    // alike, from the whole vectors); r -= alpha K d (every CTA the whole vector), w += alpha d
    // (the CTA's slice)
    {
      const float sig2f = (float)a.sigma2;
      float4 kd[NR][VPT];
      float de0 = 0.f, de1 = 0.f;
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        const int64_t col = ((int64_t)v * kT + tid) * 4;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          kd[r][v] = f4zero();
          if (col < npad) {
            if (a.det) {
              kd[r][v] = ldcg4(a.atd + r * npad + col);
            } else {
              const float4 at = ldcg4(atd + r * npad + col);
              const float4 q = qv[r][v];
              kd[r][v] = make_float4(fmaf(-sig2f, q.x, at.x), fmaf(-sig2f, q.y, at.y),
                                     fmaf(-sig2f, q.z, at.z), fmaf(-sig2f, q.w, at.w));
              const float dk = dot4(q, kd[r][v], 0.f);
              if (r == 0) de0 += dk; else de1 += dk;
            }
          }
        }
      }
      // this warp's first row of M (needed after the update)
      if (gw < npad) prefetch_row(a.M + gw * npad, 0, npad, pre);
      if (a.det) {
        // delta from the CTAs' shares in CTA order (each lane its CTAs, then a butterfly)
        if (warp == 0) {
          const float* dpart = a.part + (int64_t)G * E;
          float s0 = 0.f, s1 = 0.f;
#pragma unroll
          for (int u = 0; u < kFMaxGrid / 32; ++u) {
            const int c = lane + 32 * u;
            if (c < G) {
              s0 += __ldcg(dpart + 2 * c);
              s1 += __ldcg(dpart + 2 * c + 1);
            }
          }
          s0 = warp_sumf(s0);
          s1 = warp_sumf(s1);
          if (lane == 0) {
            sh.sums[0] = s0;
            sh.sums[1] = s1;
          }
        }
        __syncthreads();
      } else {
        cta_sum2(de0, de1, sh);
      }
      if (tid == 0)
        for (int r = 0; r < NR; ++r) {
          sh.ok[r] = 0;
          if (!sh.done[r]) {
            const float delta = sh.sums[r];
            sh.delta[r] = delta;
            sh.ok[r] = (delta > 0.f) ? 1 : 0;
            sh.alpha[r] = sh.ok[r] ? sh.eta[r] / delta : 0.f;
          }
        }
      __syncthreads();
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        const int64_t col = ((int64_t)v * kT + tid) * 4;
        if (col < npad)
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            if (!sh.ok[r]) continue;
            const float al = sh.alpha[r];
            float4& rv = *reinterpret_cast<float4*>(vs + r * npad + col);
            rv.x = fmaf(-al, kd[r][v].x, rv.x);
            rv.y = fmaf(-al, kd[r][v].y, rv.y);
            rv.z = fmaf(-al, kd[r][v].z, rv.z);
            rv.w = fmaf(-al, kd[r][v].w, rv.w);
          }
      }
      float* atd_next = a.atd + (int64_t)((j + 1) & 1) * E;
      for (int e = tid; e < nsl; e += kT) {
        const int r = (int)((e_lo + e) / npad);
        if (sh.ok[r]) sh.w_sl[e] = fmaf(sh.alpha[r], sh.d_sl[e], sh.w_sl[e]);
        if (!a.det) atd_next[e_lo + e] = 0.f;
      }
    }
    __syncthreads();
    trace_at(a, tb + 3);
    trace_at(a, tb + 4);
    // ---------------- z = M r for the warps' rows
    m_phase<NR>(a, vs, pre, gw, GW, npad);
    trace_at(a, tb + 5);
    if (!(alive = grid_sync(a, sh, 3 * j + 2))) break;
    trace_at(a, tb + 6);
    // ---------------- eta_{j+1} = r^T z, beta_j, the stop flags (every CTA alike, from the
    // whole vectors); d_{j+1} = z + beta_j d_j: the thread's columns and the CTA's slice
    {
      float4 zv[NR][VPT];
      float e0 = 0.f, e1 = 0.f;
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        const int64_t col = ((int64_t)v * kT + tid) * 4;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          zv[r][v] = f4zero();
          if (col < npad) {
            zv[r][v] = ldcg4(a.z + r * npad + col);
            const float rz =
                dot4(zv[r][v], *reinterpret_cast<const float4*>(vs + r * npad + col), 0.f);
            if (r == 0) e0 += rz; else e1 += rz;
          }
        }
      }
      float zs[(kFMaxSlice + kT - 1) / kT];
#pragma unroll
      for (int u = 0; u < (kFMaxSlice + kT - 1) / kT; ++u) {
        const int e = tid + u * kT;
        zs[u] = (e < nsl) ? __ldcg(a.z + e_lo + e) : 0.f;
      }
      cta_sum2(e0, e1, sh);
      if (tid == 0)
        for (int r = 0; r < NR; ++r) step_flags(sh, r, sh.sums[r], (float)a.cg_tol2);
      __syncthreads();
      trace_at(a, tb + 7);
      if (j + 1 >= a.steps || (sh.done[0] && (NR < 2 || sh.done[1]))) break;
      const float b0 = sh.beta[0], b1 = (NR > 1) ? sh.beta[1] : 0.f;
#pragma unroll
      for (int v = 0; v < VPT; ++v)
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const float bt = r ? b1 : b0;
          float4& q = qv[r][v];
          const float4& z = zv[r][v];
          q = make_float4(fmaf(bt, q.x, z.x), fmaf(bt, q.y, z.y), fmaf(bt, q.z, z.z),
                          fmaf(bt, q.w, z.w));
        }
#pragma unroll
      for (int u = 0; u < (kFMaxSlice + kT - 1) / kT; ++u) {
        const int e = tid + u * kT;
        if (e < nsl) {
          const int r = (int)((e_lo + e) / npad);
          sh.d_sl[e] = fmaf(r ? b1 : b0, sh.d_sl[e], zs[u]);
        }
      }
      trace_at(a, tb + 8);
    }
  }
  __syncthreads();

  // ---- results: w (each CTA its slice), the scalars (CTA 0); then the copies in flight
  for (int e = tid; e < nsl; e += kT) a.w[e_lo + e] = sh.w_sl[e];
  if (blockIdx.x == 0 && tid == 0) {
    PcgScalars* sc = a.sc;
    for (int r = 0; r < 2; ++r) {
      sc->eta[r] = sh.eta[r];
      sc->eta0[r] = sh.eta0[r];
      sc->beta[r] = sh.beta[r];
      sc->alpha[r] = sh.alpha[r];
      sc->delta[r] = sh.delta[r];
      sc->qq[r] = 0.0;
      sc->done[r] = sh.done[r];
      sc->iters[r] = sh.iters[r];
      sc->not_spd[r] = sh.nspd[r];
    }
    sc->sigma2 = a.sigma2;
    sc->cg_tol2 = a.cg_tol2;
    sc->nr = NR;
    sc->passes = passes;
  }
  if (HOLD && a.load_mode == 2) {
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (tid == 0) {
    for (int64_t kk = ps.consumed; kk < ps.issued; ++kk)
      ptx::mbar_wait(&sh.full[kk % S], (uint32_t)((kk / S) & 1), a.err, 23);
  }
}

template <int NR, int VPT, int RT, bool HOLD>
cudaError_t launch_one(const FusedArgs& a, int grid, size_t smem, cudaStream_t st) {
  auto kern = pcg_fused_kernel<NR, VPT, RT, HOLD>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  void* args[] = {(void*)&a};
  e = cudaLaunchCooperativeKernel((const void*)kern, grid, kT, args, smem, st);
  count_launch();
  return e;
}

// Ring geometry for npad: float4 column groups per thread (vpt), rows per tile (rt, a power of
// two with nr * rt <= 16) and the number of stages; false when npad is outside the kernel's range.
// Tiles held in registers (hold): rt * vpt <= 4, so that two tiles fit in registers, with at
// least four stages; in shared memory: the largest rt with rt * vpt <= 8 that still leaves
// min_stages stages.
bool fused_geometry(int64_t npad, int nr, int num_sms, bool hold, int min_stages, int* vpt,
                    int* rt, int* stages, size_t* smem) {
  if (npad < 64 || npad > 8192 || npad % 4 != 0) return false;
  if (num_sms < 1 || num_sms > kFMaxGrid) return false;
  if ((npad + (int64_t)num_sms * kW - 1) / ((int64_t)num_sms * kW) > kFMaxRows) return false;
  if ((nr * npad + num_sms - 1) / num_sms > kFMaxSlice) return false;
  const int v = (int)((npad + 4 * kT - 1) / (4 * kT));
  const size_t vec = (size_t)nr * npad * 4;
  const size_t budget = 227 * 1024 - sizeof(FusedShared) - 1024;
  if (vec >= budget) return false;
  const size_t room = budget - vec;
  int r = 1;
  if (hold) {
    while (2 * r <= 8 && 2 * r * v <= 4 && nr * 2 * r <= 16 && (size_t)(2 * r) * npad * 4 * 4 <= room)
      r *= 2;
  } else {
    while (2 * r <= 8 && 2 * r * v <= 8 && nr * 2 * r <= 16 &&
           (size_t)(2 * r) * npad * 4 * min_stages <= room)
      r *= 2;
  }
  const size_t tile = (size_t)r * npad * 4;
  if (2 * tile > room) return false;
  const int s = (int)std::min<size_t>(kFMaxStages, room / tile);
  if (!hold && s < 3) return false;
  *vpt = v;
  *rt = r;
  *stages = s;
  *smem = (size_t)s * tile + vec;
  return true;
}

}  // namespace

int pcg_fused_trace_words() { return kFTraceWords; }

bool pcg_fused_supported(int64_t npad, int nr, int num_sms) {
  int v, r, s;
  size_t sm;
  return fused_geometry(npad, nr, num_sms, false, 3, &v, &r, &s, &sm) &&
         fused_geometry(npad, nr, num_sms, false, 5, &v, &r, &s, &sm) &&
         fused_geometry(npad, nr, num_sms, true, 4, &v, &r, &s, &sm);
}

cudaError_t launch_pcg_fused(const float* A, int64_t m, int64_t n, int64_t npad, int nr,
                             const double* fin0, double fin0_scale, const double* fin1,
                             const float* M, float* w, float* z, float* atd, float* part,
                             int det, PcgScalars* sc,
                             double sigma2, double cg_tol, int steps, unsigned int* bar, int* err,
                             int num_sms, cudaStream_t st, unsigned long long* trace,
                             int load_mode, int64_t keep_bytes, int pass_kind) {
  int vpt, rt, stages;
  size_t smem;
  // pass_kind 0: decoupled warps, tiles in shared memory, the largest tiles that leave three
  // stages (at 2048 columns: 8 rows, 64 KB, which measured fastest); 1: tiles held in registers
  // across one CTA barrier per tile; 2: as 0 with smaller tiles and at least five stages
  const bool hold = (pass_kind == 1);
  if (!fused_geometry(npad, nr, num_sms, hold, pass_kind == 2 ? 5 : 3, &vpt, &rt, &stages, &smem))
    return cudaErrorInvalidValue;
  FusedArgs a{};
  a.A = A; a.m = m; a.n = n; a.npad = npad; a.nr = nr; a.steps = steps; a.stages = stages;
  a.fin0 = fin0; a.fin0_scale = fin0_scale; a.fin1 = fin1; a.M = M; a.w = w; a.z = z;
  a.atd = atd; a.part = part; a.det = det ? 1 : 0; a.sc = sc; a.sigma2 = sigma2;
  a.cg_tol2 = cg_tol * cg_tol; a.bar = bar; a.err = err; a.trace = trace;
  a.load_mode = (load_mode >= 0 && load_mode <= (hold ? 2 : 1)) ? load_mode : 0;
  // tiles per CTA kept in L2 across the steps: keep_bytes over all CTAs (0: none)
  a.keep_tiles = (keep_bytes > 0)
                     ? (int)std::min<int64_t>(1 << 20, keep_bytes / num_sms /
                                                           ((int64_t)rt * npad * (int64_t)sizeof(float)))
                     : 0;
  cudaError_t e = cudaErrorInvalidValue;
#define TLS_FUSED_CASE(NR_, V_, R_, H_)                                             \
  else if (nr == NR_ && vpt == V_ && rt == R_ && hold == H_) e =                   \
      launch_one<NR_, V_, R_, H_>(a, num_sms, smem, st);
  if (false) {
  }
  TLS_FUSED_CASE(1, 1, 8, false) TLS_FUSED_CASE(1, 1, 4, false) TLS_FUSED_CASE(1, 2, 4, false)
  TLS_FUSED_CASE(1, 2, 2, false) TLS_FUSED_CASE(1, 3, 2, false) TLS_FUSED_CASE(1, 3, 1, false)
  TLS_FUSED_CASE(1, 4, 1, false) TLS_FUSED_CASE(1, 4, 2, false)
  TLS_FUSED_CASE(2, 1, 8, false) TLS_FUSED_CASE(2, 1, 4, false) TLS_FUSED_CASE(2, 2, 4, false)
  TLS_FUSED_CASE(2, 2, 2, false) TLS_FUSED_CASE(2, 3, 2, false) TLS_FUSED_CASE(2, 3, 1, false)
  TLS_FUSED_CASE(2, 4, 1, false) TLS_FUSED_CASE(2, 4, 2, false)
  TLS_FUSED_CASE(1, 1, 4, true) TLS_FUSED_CASE(1, 2, 2, true) TLS_FUSED_CASE(1, 3, 1, true)
  TLS_FUSED_CASE(1, 4, 1, true)
  TLS_FUSED_CASE(2, 1, 4, true) TLS_FUSED_CASE(2, 2, 2, true) TLS_FUSED_CASE(2, 3, 1, true)
  TLS_FUSED_CASE(2, 4, 1, true)
#undef TLS_FUSED_CASE
  return e;
}

}  // namespace tls
