// One PCGTLS solve (Alg. 3, the A-explicit operator; one or two right-hand sides) in a single
// persistent cooperative launch, FP32 working precision (the u_p of Alg. 4).
//
// Every CTA is resident (one per SM, 16 warps). A CTA owns a contiguous block of rows of the FP32
// copy of A and streams it, step after step, through a ring of shared-memory stages filled by
// 1-D bulk asynchronous copies (TMA, completion on mbarriers). Per PCGTLS step j:
//
//   pass    t = A q_j row by row from the ring, the CTA's partial of A^T t and of ||t||^2
//                                                                    -- grid barrier 1 (||t||^2)
//   reduce  the CTA's slice of the columns of A^T t summed over all partials: delta_j, alpha_j,
//           w += alpha q_j, y = D^{-1}(A^T t - sigma^2 q_j)          -- grid barrier 2
//   W^T     v = W^T y for the rows each warp owns, s_{j+1} = s_j - alpha v  -- barrier 3 (||s||^2)
//           eta_{j+1}, beta_j and the stop flags
//   W       p_{j+1} = s_{j+1} + beta_j p_j, q_{j+1} = D^{-1} W p_{j+1}  -- barrier 4 (||q||^2)
//
// with W = R_H^{-1} (R = R_H D): q = R^{-1} p and v = R^{-T} D^{-1}(...) are the two triangular
// solves of Alg. 3, done as row-parallel products with the explicit inverse.
//
// What keeps the step short on this GPU, where a dependent round trip to L2 costs about a
// microsecond:
//  * the grid barriers are flag barriers that carry the CTA's partial sums: CTA c publishes
//    (partial, tag) words in its own slot and every CTA reads all slots, so one round trip both
//    synchronises and delivers the data for the next scalar (no atomic counter, no second read);
//    every CTA adds the partials in the same order, so all take identical decisions;
//  * state that only one CTA or warp touches stays on chip: the CTA's slice of w, 1/d and q in
//    shared memory, each warp's entries of s and 1/d in registers;
//  * each warp loads its rows of W^T and W into registers before the barrier that precedes the
//    phase that needs them;
//  * the pass is software-pipelined with one CTA barrier per tile: the dot products of tile i
//    overlap the cross-warp sums of tile i - 1, whose axpy follows the barrier; tile data is kept
//    in registers across the barrier, so a stage is refilled as soon as every thread has read it,
//    and when a pass ends the first stages of the next pass are already in flight, so HBM keeps
//    streaming through the step's tail.
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
constexpr int kPre = 8;                        // float4 per lane of a prefetched W row
constexpr uint64_t kFBarrierNs = 2000ull * 1000 * 1000;   // grid barrier deadline: 2 s

struct FusedArgs {
  const float* A;        // m x npad, row-major, rows back to back (lda = npad)
  int64_t m, n, npad;
  int nr, steps, stages;
  const double* fin0;    // right-hand side 0 is fin0_scale * fin0, 1 is fin1 (FP64, n values)
  double fin0_scale;
  const double* fin1;
  const double* dinv64;  // 1 / d (FP64, npad)
  const float* dinv;     // 1 / d (FP32, npad)
  const float* W;        // R_H^{-1}, upper triangular, npad x npad
  const float* WT;       // W^T, lower triangular
  float* w;              // solutions, nr x npad (written at the end)
  float* y;              // D^{-1}(A^T t - sigma^2 q), nr x npad
  float* s;              // s_j, nr x npad
  float* pa;             // p_j, ping-pong, nr x npad each
  float* pb;
  float* q;              // q_j = D^{-1} W p_j, nr x npad
  float* part;           // G x nr x npad pass partials
  unsigned long long* slots;   // flag-barrier words: 2 parities x kFMaxGrid CTAs x 2 values
  unsigned int epoch;    // tag of this launch's first grid barrier (see launch_pcg_fused)
  PcgScalars* sc;
  double sigma2, cg_tol2;
  unsigned int* bar;     // [64] abort word (zero between launches)
  int* err;
  unsigned long long* trace;   // optional phase timestamps of CTA 0
  int load_mode;         // how a tile reaches shared memory (see issue_next)
  int keep_tiles;        // the first keep_tiles tiles of every CTA's block are loaded with an
                         // L2 evict-last policy (they stay resident across the steps), the rest
                         // with evict-first
};

// Trace layout (global-timer nanoseconds, CTA 0, thread 0): [0] start, [1] initialisation done,
// then per step j < kFTraceSteps, at 2 + kFTracePer * j: pass start, pass end, barrier 1 done,
// reduce done, barrier 2 done, W^T done, barrier 3 done, W done, barrier 4 done, and the time
// thread 0 spent waiting for tiles of that pass.
constexpr int kFTracePer = 10;
constexpr int kFTraceSteps = 64;
constexpr int kFTraceWords = 2 + kFTracePer * kFTraceSteps;

__device__ __forceinline__ void trace_at(const FusedArgs& a, int idx) {
  if (a.trace != nullptr && blockIdx.x == 0 && threadIdx.x == 0 && idx < kFTraceWords)
    a.trace[idx] = ptx::global_ns();
}

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
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
__device__ __forceinline__ float4 f4zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

struct alignas(16) FusedShared {
  uint64_t full[kFMaxStages];
  float red[2][kW][16];         // per-warp row values of a tile (double-buffered)
  float tot[2][16];             // row values of a tile summed over the warps
  float red2[kW][33];
  float cta2[kW][2];
  float tt_w[16];
  float w_sl[kFMaxSlice];       // this CTA's slice of w
  float q_sl[kFMaxSlice];       // ... of q_j
  float di_sl[kFMaxSlice];      // ... of 1/d
  float s_row[kW][kFMaxRows][2];  // s_j of each warp's rows of W^T (lane 0)
  float di_row[kW][kFMaxRows];    // 1/d of each warp's rows of W
  double sums[2];
  double eta[2], eta0[2], beta[2], delta[2], alpha[2], qq[2];
  int done[2], iters[2], nspd[2], ok[2];
  int fail;
};

// Flag barrier over every CTA of the launch that also all-gathers two FP32 partial sums per CTA
// (v0, v1): CTA c fences its writes and stores (v, tag) words in its slot; warp 0 of every CTA
// polls all slots with relaxed loads (all in flight at once: an acquire load would order the
// next one behind it) until every tag is this barrier's, fences (acquire side of the fence
// pairing), then adds the partials in CTA order (FP64) into sh.sums. Slots alternate between two
// parities, so a CTA can only overwrite a slot once every CTA has passed the barrier before.
// Returns false when abandoned (deadline here, or the abort word raised elsewhere). All threads
// must call it.
__device__ __forceinline__ bool flag_barrier(const FusedArgs& a, FusedShared& sh, unsigned int tag, float v0,
                             float v1) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = (int)gridDim.x;
  unsigned long long* base = a.slots + (size_t)(tag & 1u) * kFMaxGrid * 2;
  __syncthreads();                      // this CTA's global writes of the phase are done
  if (tid == 0) {
    __threadfence();
    const unsigned long long t = (unsigned long long)tag << 32;
    st_relaxed64(base + 2 * blockIdx.x, t | __float_as_uint(v0));
    st_relaxed64(base + 2 * blockIdx.x + 1, t | __float_as_uint(v1));
  }
  if (warp == 0) {
    constexpr int kU = kFMaxGrid / 32;
    const uint64_t t0 = ptx::global_ns();
    unsigned int it = 0;
    bool ok = true;
    double s0, s1;
    for (;;) {
      // one round: every slot of this lane, its tags checked and its values summed in CTA order
      bool mine = true;
      s0 = 0.0;
      s1 = 0.0;
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int c = lane + 32 * u;
        if (c < G) {
          const unsigned long long w0 = ld_relaxed64(base + 2 * c);
          const unsigned long long w1 = ld_relaxed64(base + 2 * c + 1);
          mine = mine && ((unsigned int)(w0 >> 32) == tag) && ((unsigned int)(w1 >> 32) == tag);
          s0 += (double)__uint_as_float((unsigned int)w0);
          s1 += (double)__uint_as_float((unsigned int)w1);
        }
      }
      if (__all_sync(0xffffffffu, mine)) break;
      if ((++it & 63u) == 0) {
        int stop = 0;
        if (lane == 0) {
          if (ld_acquire32(a.bar + 64) != 0u) {
            stop = 1;
          } else if (ptx::global_ns() - t0 > kFBarrierNs) {
            atomicCAS(a.err, 0, 21);
            atomicExch(a.bar + 64, 1u);
            stop = 1;
          }
        }
        if (__shfl_sync(0xffffffffu, stop, 0)) {
          ok = false;
          break;
        }
      }
    }
    __threadfence();   // the slots were observed: later reads see what their writers fenced
    s0 = warp_sumd(s0);
    s1 = warp_sumd(s1);
    if (lane == 0) {
      sh.sums[0] = s0;
      sh.sums[1] = s1;
      if (!ok) sh.fail = 1;
    }
  }
  __syncthreads();
  return sh.fail == 0;
}

// CTA sum of two per-thread FP32 values (all threads call it); thread 0 returns the totals.
__device__ __forceinline__ void cta_sum2(float& v0, float& v1, FusedShared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v0 = warp_sumf(v0);
  v1 = warp_sumf(v1);
  if (lane == 0) {
    sh.cta2[warp][0] = v0;
    sh.cta2[warp][1] = v1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float t0 = 0.f, t1 = 0.f;
#pragma unroll
    for (int w2 = 0; w2 < kW; ++w2) {
      t0 += sh.cta2[w2][0];
      t1 += sh.cta2[w2][1];
    }
    v0 = t0;
    v1 = t1;
  }
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

// Row j of W^T holds entries 0..j (rounded up to a float4); row i of W entries i..npad-1
// (from the float4 containing i).
__device__ __forceinline__ int64_t wt_lim(int64_t j) { return ((j + 4) / 4) * 4; }
__device__ __forceinline__ int64_t w_start(int64_t i) { return (i / 4) * 4; }

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
  float tt_acc;                 // lane 0 of warps < NV: squares of the row values it summed
  bool gotall;
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
template <int RT>
__device__ __forceinline__ void issue_next(const FusedArgs& a, FusedShared& sh, PassState& ps,
                                           uint64_t pol_stream) {
  const uint64_t pol = (ps.i_lt < a.keep_tiles) ? ps.pol_keep : pol_stream;
  const int slot = ps.i_slot;
  const int64_t row = ps.r0 + (int64_t)ps.i_lt * RT;
  const int rows = (int)min((int64_t)RT, ps.r1 - row);
  float* dst = ps.ring + slot * ps.stage_floats;
  const float* src = a.A + row * ps.npad;
  ++ps.issued;
  if (++ps.i_slot == ps.S) ps.i_slot = 0;
  if (++ps.i_lt == ps.T) ps.i_lt = 0;
  if (a.load_mode == 2) {
    const int chunks = (int)((int64_t)rows * ps.npad / 4);
    for (int c = threadIdx.x; c < chunks; c += kT) cp_async16(dst + 4 * c, src + 4 * c, pol);
    cp_async_arrive(&sh.full[slot]);
    return;
  }
  if (threadIdx.x != 0) return;
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
    if (lane == 0) {
      sh.tot[b][warp] = x;
      ps.tt_acc = fmaf(x, x, ps.tt_acc);     // rows beyond the block are zero
    }
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

template <int NR, int VPT, int RT>
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
  float* vs = ring + (int64_t)S * stage_floats;     // staged vector (NR x npad)
  // this CTA's rows of A and its tiles
  const int64_t per = (a.m + G - 1) / G;
  const int64_t r0 = min(a.m, (int64_t)blockIdx.x * per);
  const int64_t r1 = min(a.m, r0 + per);
  const int T = (r1 > r0) ? (int)((r1 - r0 + RT - 1) / RT) : 0;
  // this CTA's slice of the columns (entries of the nr x npad vectors) and each warp's rows of
  // W / W^T
  const int64_t e_lo = (int64_t)blockIdx.x * E / G, e_hi = (int64_t)(blockIdx.x + 1) * E / G;
  const int nsl = (int)(e_hi - e_lo);
  const int64_t GW = (int64_t)G * kW, gw = (int64_t)blockIdx.x * kW + warp;
  unsigned int tag = a.epoch;

  // the CTA's tiles in sequence: tile k is local tile k % T of pass k / T
  const int64_t total = (int64_t)a.steps * T;
  const uint64_t pol = ptx::policy_evict_first();   // each row of A is read once per pass
  trace_at(a, 0);
  if (tid == 0) {
    for (int k = 0; k < S; ++k) ptx::mbar_init(&sh.full[k], a.load_mode == 2 ? kT : 1);
    ptx::fence_mbar_init();
    sh.fail = 0;
  }
  __syncthreads();
  uint64_t pol_keep;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol_keep));
  PassState ps{ring, stage_floats, S, r0, r1, T, npad, total, 0, 0, 0, 0, 0, 0u, pol_keep, 0ull,
               0.f, true};
  while (ps.issued < S && ps.issued < total) issue_next<RT>(a, sh, ps, pol);
  for (int e = tid; e < nsl; e += kT) {
    sh.w_sl[e] = 0.f;
    sh.di_sl[e] = __ldg(a.dinv + (e_lo + e) % npad);
  }
  // each warp's rows: their 1/d and their s (lane 0 uses them; shared memory, per warp)
  float (&s_row)[kFMaxRows][2] = sh.s_row[warp];
  float (&di_row)[kFMaxRows] = sh.di_row[warp];
  if (lane < kFMaxRows) {
    const int64_t i = gw + lane * GW;
    di_row[lane] = (i < npad) ? __ldg(a.dinv + i) : 0.f;
    s_row[lane][0] = s_row[lane][1] = 0.f;
  }
  __syncwarp();
  // ---- initialisation: y = D^{-1} f (every CTA the whole vector), s_0 = W^T y, eta_0
  float4 pre[kPre];
  if (gw < npad) prefetch_row(a.WT + gw * npad, 0, wt_lim(gw), pre);
  for (int64_t j = tid; j < npad; j += kT) {
    const double di = a.dinv64[j];
    double f0 = 0.0, f1 = 0.0;
    if (j < a.n) {
      f0 = a.fin0_scale * a.fin0[j];
      if (NR > 1) f1 = a.fin1[j];
    }
    vs[j] = (float)(f0 * di);
    if (NR > 1) vs[npad + j] = (float)(f1 * di);
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
  __syncthreads();
  bool alive;
  {
    float ss0 = 0.f, ss1 = 0.f;
#pragma unroll
    for (int k = 0; k < kFMaxRows; ++k) {
      const int64_t j = gw + k * GW;
      if (j >= npad) break;
      if (k > 0) prefetch_row(a.WT + j * npad, 0, wt_lim(j), pre);
      float v0 = 0.f, v1 = 0.f;
      row_dot<NR>(a.WT + j * npad, 0, wt_lim(j), pre, vs, npad, v0, v1);
      if (lane == 0) {
        s_row[k][0] = v0;
        s_row[k][1] = v1;
        a.s[j] = v0;
        ss0 = fmaf(v0, v0, ss0);
        if (NR > 1) {
          a.s[npad + j] = v1;
          ss1 = fmaf(v1, v1, ss1);
        }
      }
    }
    if (gw < npad) prefetch_row(a.W + gw * npad, w_start(gw), npad, pre);
    cta_sum2(ss0, ss1, sh);
    alive = flag_barrier(a, sh, tag++, ss0, ss1);
  }
  if (alive) {
    if (tid == 0)
      for (int r = 0; r < NR; ++r) {
        sh.eta[r] = sh.eta0[r] = sh.sums[r];
        sh.done[r] = (sh.sums[r] == 0.0) ? 1 : 0;
      }
    // p_0 = s_0 (staged from the s every CTA wrote; this CTA publishes its slice), q_0
    for (int64_t e = (int64_t)tid * 4; e < E; e += 4 * kT)
      *reinterpret_cast<float4*>(vs + e) = ldcg4(a.s + e);
    __syncthreads();
    for (int e = tid; e < nsl; e += kT) a.pa[e_lo + e] = vs[e_lo + e];
    float qq0 = 0.f, qq1 = 0.f;
#pragma unroll
    for (int k = 0; k < kFMaxRows; ++k) {
      const int64_t i = gw + k * GW;
      if (i >= npad) break;
      if (k > 0) prefetch_row(a.W + i * npad, w_start(i), npad, pre);
      float v0 = 0.f, v1 = 0.f;
      row_dot<NR>(a.W + i * npad, w_start(i), npad, pre, vs, npad, v0, v1);
      if (lane == 0) {
        const float q0 = v0 * di_row[k];
        a.q[i] = q0;
        qq0 = fmaf(q0, q0, qq0);
        if (NR > 1) {
          const float q1 = v1 * di_row[k];
          a.q[npad + i] = q1;
          qq1 = fmaf(q1, q1, qq1);
        }
      }
    }
    cta_sum2(qq0, qq1, sh);
    alive = flag_barrier(a, sh, tag++, qq0, qq1);
  }
  if (alive && tid == 0) {
    sh.qq[0] = sh.sums[0];
    sh.qq[1] = sh.sums[1];
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
    float* p_cur = (j & 1) ? a.pb : a.pa;
    float* p_next = (j & 1) ? a.pa : a.pb;
    // q_j: the thread's columns (registers) and the CTA's slice (shared memory)
    float4 qv[NR][VPT];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int64_t col = ((int64_t)v * kT + tid) * 4;
#pragma unroll
      for (int r = 0; r < NR; ++r)
        qv[r][v] = (col < npad) ? ldcg4(a.q + r * npad + col) : f4zero();
    }
    for (int e = tid; e < nsl; e += kT) sh.q_sl[e] = __ldcg(a.q + e_lo + e);
    // ---------------- pass over the CTA's rows: t = A q, partial A^T t, ||t||^2
    unsigned long long tile_wait = 0;
    float tt_acc = 0.f;
    bool ok = true;
    {
      float4 acc[NR][VPT];
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int v = 0; v < VPT; ++v) acc[r][v] = f4zero();
      float4 a0[RT][VPT], a1[RT][VPT];
      ps.tile_wait = 0ull;
      ps.tt_acc = 0.f;
      // one CTA barrier per tile: [dots(lt) | sums(lt - 1)] barrier [refill, axpy(lt - 1)]
      for (int lt = 0; ok && lt <= T; lt += 2) {
        ok = pass_tile<NR, VPT, RT>(a, sh, ps, qv, acc, a0, a1, lt, pol);
        if (ok && lt + 1 <= T) ok = pass_tile<NR, VPT, RT>(a, sh, ps, qv, acc, a1, a0, lt + 1, pol);
      }
      tile_wait = ps.tile_wait;
      tt_acc = ps.tt_acc;
      // this CTA's partial of A^T t
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        const int64_t col = ((int64_t)v * kT + tid) * 4;
        if (col < npad)
#pragma unroll
          for (int r = 0; r < NR; ++r)
            *reinterpret_cast<float4*>(a.part + (int64_t)blockIdx.x * E + r * npad + col) =
                acc[r][v];
      }
    }
    if (!ok && tid == 0) {
      atomicExch(a.bar + 64, 1u);
      sh.fail = 1;
    }
    if (warp < NV && lane == 0) sh.tt_w[warp] = tt_acc;
    // prefetch this warp's first row of W^T (needed after barrier 2)
    if (gw < npad) prefetch_row(a.WT + gw * npad, 0, wt_lim(gw), pre);
    __syncthreads();
    float tt0 = 0.f, tt1 = 0.f;
    if (tid == 0) {
      for (int w2 = 0; w2 < NV; ++w2) {
        if (w2 / RT == 0) tt0 += sh.tt_w[w2];
        else tt1 += sh.tt_w[w2];
      }
    }
    trace_at(a, tb + 1);
    if (a.trace != nullptr && blockIdx.x == 0 && tid == 0 && j < kFTraceSteps)
      a.trace[tb + 9] = tile_wait;
    if (!(alive = flag_barrier(a, sh, tag++, tt0, tt1))) break;
    trace_at(a, tb + 2);
    // ---------------- delta_j, alpha_j (every CTA alike), column slice: w and y
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
    {
      // slice entries in chunks of 32: warp ps sums partials ps, ps + 16, ... (all loads in
      // flight at once), then warp 0 adds the 16 slices in a fixed order
      const float sig2f = (float)a.sigma2;
      for (int c0 = 0; c0 < nsl; c0 += 32) {
        const int e = c0 + lane;
        float t = 0.f;
        if (e < nsl) {
          float pv[kFMaxGrid / kW];
#pragma unroll
          for (int u = 0; u < kFMaxGrid / kW; ++u) {
            const int p = warp + kW * u;
            pv[u] = (p < G) ? __ldcg(a.part + (int64_t)p * E + e_lo + e) : 0.f;
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
          const int r = (int)((e_lo + e) / npad);
          if (sh.ok[r]) {
            const float qj = sh.q_sl[e];
            sh.w_sl[e] = fmaf((float)sh.alpha[r], qj, sh.w_sl[e]);
            a.y[e_lo + e] = (at - sig2f * qj) * sh.di_sl[e];
          }
        }
        __syncthreads();
      }
    }
    trace_at(a, tb + 3);
    if (!(alive = flag_barrier(a, sh, tag++, 0.f, 0.f))) break;
    trace_at(a, tb + 4);
    // ---------------- v = W^T y, s_{j+1} = s_j - alpha v, ||s_{j+1}||^2
    for (int64_t e = (int64_t)tid * 4; e < E; e += 4 * kT)
      *reinterpret_cast<float4*>(vs + e) = ldcg4(a.y + e);
    __syncthreads();
    {
      const bool act0 = !sh.done[0] && sh.ok[0];
      const bool act1 = NR > 1 && !sh.done[1] && sh.ok[1];
      const float al0 = (float)sh.alpha[0], al1 = (NR > 1) ? (float)sh.alpha[1] : 0.f;
      float ss0 = 0.f, ss1 = 0.f;
#pragma unroll
      for (int k = 0; k < kFMaxRows; ++k) {
        const int64_t jr = gw + k * GW;
        if (jr >= npad) break;
        if (k > 0) prefetch_row(a.WT + jr * npad, 0, wt_lim(jr), pre);
        float v0 = 0.f, v1 = 0.f;
        row_dot<NR>(a.WT + jr * npad, 0, wt_lim(jr), pre, vs, npad, v0, v1);
        if (lane == 0) {
          if (act0) s_row[k][0] -= al0 * v0;
          if (act1) s_row[k][1] -= al1 * v1;
          if (act0) a.s[jr] = s_row[k][0];
          ss0 = fmaf(s_row[k][0], s_row[k][0], ss0);
          if (NR > 1) {
            if (act1) a.s[npad + jr] = s_row[k][1];
            ss1 = fmaf(s_row[k][1], s_row[k][1], ss1);
          }
        }
      }
      // prefetch this warp's first row of W (needed after barrier 3)
      if (gw < npad) prefetch_row(a.W + gw * npad, w_start(gw), npad, pre);
      cta_sum2(ss0, ss1, sh);
      trace_at(a, tb + 5);
      if (!(alive = flag_barrier(a, sh, tag++, ss0, ss1))) break;
      trace_at(a, tb + 6);
    }
    if (tid == 0)
      for (int r = 0; r < NR; ++r) step_flags(sh, r, sh.sums[r], a.cg_tol2);
    __syncthreads();
    if (j + 1 >= a.steps || (sh.done[0] && (NR < 2 || sh.done[1]))) break;
    // ---------------- p_{j+1} = s_{j+1} + beta_j p_j, q_{j+1} = D^{-1} W p_{j+1}, ||q||^2
    {
      const float b0 = (float)sh.beta[0], b1 = (NR > 1) ? (float)sh.beta[1] : 0.f;
      for (int64_t e = (int64_t)tid * 4; e < E; e += 4 * kT) {
        const float4 sv = ldcg4(a.s + e), pv = ldcg4(p_cur + e);
        const float bt = (e < npad) ? b0 : b1;
        *reinterpret_cast<float4*>(vs + e) = make_float4(
            fmaf(bt, pv.x, sv.x), fmaf(bt, pv.y, sv.y), fmaf(bt, pv.z, sv.z), fmaf(bt, pv.w, sv.w));
      }
      __syncthreads();
      for (int e = tid; e < nsl; e += kT) p_next[e_lo + e] = vs[e_lo + e];
      float qq0 = 0.f, qq1 = 0.f;
#pragma unroll
      for (int k = 0; k < kFMaxRows; ++k) {
        const int64_t i = gw + k * GW;
        if (i >= npad) break;
        if (k > 0) prefetch_row(a.W + i * npad, w_start(i), npad, pre);
        float v0 = 0.f, v1 = 0.f;
        row_dot<NR>(a.W + i * npad, w_start(i), npad, pre, vs, npad, v0, v1);
        if (lane == 0) {
          const float q0 = v0 * di_row[k];
          a.q[i] = q0;
          qq0 = fmaf(q0, q0, qq0);
          if (NR > 1) {
            const float q1 = v1 * di_row[k];
            a.q[npad + i] = q1;
            qq1 = fmaf(q1, q1, qq1);
          }
        }
      }
      cta_sum2(qq0, qq1, sh);
      trace_at(a, tb + 7);
      if (!(alive = flag_barrier(a, sh, tag++, qq0, qq1))) break;
      trace_at(a, tb + 8);
    }
    if (tid == 0) {
      sh.qq[0] = sh.sums[0];
      sh.qq[1] = sh.sums[1];
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
  if (a.load_mode == 2) {
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (tid == 0) {
    for (int64_t kk = ps.consumed; kk < ps.issued; ++kk)
      ptx::mbar_wait(&sh.full[kk % S], (uint32_t)((kk / S) & 1), a.err, 23);
  }
}

template <int NR, int VPT, int RT>
cudaError_t launch_one(const FusedArgs& a, int grid, size_t smem, cudaStream_t st) {
  auto kern = pcg_fused_kernel<NR, VPT, RT>;
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

// Ring geometry for npad: float4 column groups per thread (vpt), rows per tile (rt: a power of
// two, rt * vpt <= 4 so that two tiles fit in registers, with at least four stages in the ring)
// and the number of stages; false when npad is outside the kernel's range.
bool fused_geometry(int64_t npad, int nr, int num_sms, int* vpt, int* rt, int* stages,
                    size_t* smem) {
  if (npad < 64 || npad > 8192 || npad % 4 != 0) return false;
  if (num_sms < 1 || num_sms > kFMaxGrid) return false;
  if ((npad + (int64_t)num_sms * kW - 1) / ((int64_t)num_sms * kW) > kFMaxRows) return false;
  if ((nr * npad + num_sms - 1) / num_sms > kFMaxSlice) return false;
  const int v = (int)((npad + 4 * kT - 1) / (4 * kT));
  const size_t vec = (size_t)nr * npad * 4;
  const size_t budget = 227 * 1024 - sizeof(FusedShared) - 1024;
  if (vec >= budget) return false;
  int r = 1;
  while (2 * r <= 8 && 2 * r * v <= 4 && nr * 2 * r <= 16 &&
         (size_t)(2 * r) * npad * 4 * 4 <= budget - vec)
    r *= 2;
  const size_t tile = (size_t)r * npad * 4;
  if (vec + 2 * tile > budget) return false;
  const int s = (int)std::min<size_t>(kFMaxStages, (budget - vec) / tile);
  *vpt = v;
  *rt = r;
  *stages = s;
  *smem = (size_t)s * tile + vec;
  return true;
}

}  // namespace

int pcg_fused_trace_words() { return kFTraceWords; }
size_t pcg_fused_slot_bytes() { return sizeof(unsigned long long) * 2 * kFMaxGrid * 2; }

bool pcg_fused_supported(int64_t npad, int nr, int num_sms) {
  int v, r, s;
  size_t sm;
  return fused_geometry(npad, nr, num_sms, &v, &r, &s, &sm);
}

cudaError_t launch_pcg_fused(const float* A, int64_t m, int64_t n, int64_t npad, int nr,
                             const double* fin0, double fin0_scale, const double* fin1,
                             const double* dinv64, const float* dinv, const float* W,
                             const float* WT, float* w, float* y, float* s, float* pa, float* pb,
                             float* q, float* part, unsigned long long* slots,
                             unsigned int* epoch, PcgScalars* sc, double sigma2, double cg_tol,
                             int steps, unsigned int* bar, int* err, int num_sms, cudaStream_t st,
                             unsigned long long* trace, int load_mode, int64_t keep_bytes) {
  int vpt, rt, stages;
  size_t smem;
  if (!fused_geometry(npad, nr, num_sms, &vpt, &rt, &stages, &smem)) return cudaErrorInvalidValue;
  FusedArgs a{};
  a.A = A; a.m = m; a.n = n; a.npad = npad; a.nr = nr; a.steps = steps; a.stages = stages;
  a.fin0 = fin0; a.fin0_scale = fin0_scale; a.fin1 = fin1;
  a.dinv64 = dinv64; a.dinv = dinv; a.W = W; a.WT = WT; a.w = w; a.y = y; a.s = s; a.pa = pa;
  a.pb = pb; a.q = q; a.part = part; a.slots = slots; a.sc = sc; a.sigma2 = sigma2;
  a.cg_tol2 = cg_tol * cg_tol; a.bar = bar; a.err = err; a.trace = trace;
  a.load_mode = (load_mode >= 0 && load_mode <= 2) ? load_mode : 0;
  // tiles per CTA kept in L2 across the steps: keep_bytes over all CTAs (0: none)
  a.keep_tiles = (keep_bytes > 0)
                     ? (int)std::min<int64_t>(1 << 20, keep_bytes / num_sms /
                                                           ((int64_t)rt * npad * (int64_t)sizeof(float)))
                     : 0;
  // tags of this launch's barriers: epoch, epoch + 1, ... (at most 2 + 4 steps of them); the
  // next launch starts past them, so a slot never holds a matching tag from an earlier barrier
  a.epoch = *epoch;
  *epoch += 8u + 4u * (unsigned int)steps;
  if (*epoch < 8u) *epoch = 8u;          // wrapped: restart past the zero-initialised slots
  cudaError_t e = cudaErrorInvalidValue;
#define TLS_FUSED_CASE(NR_, V_, R_) \
  else if (nr == NR_ && vpt == V_ && rt == R_) e = launch_one<NR_, V_, R_>(a, num_sms, smem, st);
  if (false) {
  }
  TLS_FUSED_CASE(1, 1, 4) TLS_FUSED_CASE(1, 1, 2) TLS_FUSED_CASE(1, 2, 2) TLS_FUSED_CASE(1, 2, 1)
  TLS_FUSED_CASE(1, 3, 1) TLS_FUSED_CASE(1, 4, 1)
  TLS_FUSED_CASE(2, 1, 4) TLS_FUSED_CASE(2, 1, 2) TLS_FUSED_CASE(2, 2, 2) TLS_FUSED_CASE(2, 2, 1)
  TLS_FUSED_CASE(2, 3, 1) TLS_FUSED_CASE(2, 4, 1)
#undef TLS_FUSED_CASE
  return e;
}

}  // namespace tls
