// RQI-PCGTLS solve kernels (Oktay & Carson, arXiv 2305.19028, Alg. 2, 3, 4).
//
//  * apass: one streaming pass over the row-major A for one or two right-hand sides. For every
//    row it forms the row dot product, turns it into the row coefficient c_i (t_i = A_i q for
//    PCGTLS, r_i = b_i - A_i x for the RQI residual), and accumulates c_i A_i into per-CTA
//    partials of A^T c while the row is still in registers, so A is read once per pass.
//  * pcg_reduce / resid_reduce: deterministic column reduction of those partials plus the
//    vector updates that follow them in Alg. 3 / Alg. 2.
//  * gemv_w / gemv_wt: q = R^{-1} p and v = R^{-T} y as products with the explicit inverse
//    W = R_H^{-1} (R = R_H D), fused with the p and s recurrences of Alg. 3.
//  * FP64 RQI vector kernels: the x_{k+1} update of Alg. 2 and the inverse-iteration start.
#include "tls_internal.h"
#include "tls_ptx.cuh"
#include "tls_device.cuh"

#include <algorithm>

namespace tls {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <typename T> struct VecOf;
template <> struct VecOf<float> { using type = float4; static constexpr int W = 4; };
template <> struct VecOf<double> { using type = double2; static constexpr int W = 2; };

__device__ __forceinline__ float get(const float4& v, int c) {
  return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}
__device__ __forceinline__ double get(const double2& v, int c) { return c == 0 ? v.x : v.y; }
__device__ __forceinline__ float4 zero_vec(float) { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ double2 zero_vec(double) { return make_double2(0.0, 0.0); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp sums of NV values at once (NV a power of two <= 32) by recursive halving: at each of the
// first log2(NV) butterfly stages a lane keeps half of its values and adds the partner's copy
// of them, so the stages cost NV/2, NV/4, ... adds instead of NV each; plain butterfly stages
// finish. Lane l returns the warp total of value l >> (5 - log2 NV).
template <typename T, int NV>
__device__ __forceinline__ T warp_reduce_scatter(const T (&v)[NV]) {
  static_assert(NV >= 1 && NV <= 32 && (NV & (NV - 1)) == 0, "NV: a power of two <= 32");
  const int lane = threadIdx.x & 31;
  T x[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) x[i] = v[i];
  int o = 16;
#pragma unroll
  for (int k = NV; k > 1; k >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < k / 2; ++i) {
      const T keep = up ? x[k / 2 + i] : x[i];
      const T give = up ? x[i] : x[k / 2 + i];
      x[i] = keep + __shfl_xor_sync(0xffffffffu, give, o);
    }
  }
  T r = x[0];
  for (; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  return r;
}

// Block-wide sum of up to 4 doubles per thread into smem result (all threads get it).
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* sh /* kWarps*K */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[warp * K + k] = v[k];
  __syncthreads();
  // second level as a shuffle tree (FP64 latency is long: keep dependency chains short)
  const int nw = (int)(blockDim.x >> 5);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double t = (lane < nw) ? sh[lane * K + k] : 0.0;
    v[k] = warp_sum(t);
  }
}

// Last-CTA detection after every CTA has published its partials (threadfence reduction).
__device__ __forceinline__ bool arrive_last(unsigned int* counter) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x * gridDim.y * gridDim.z - 1);
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Sum of K interleaved partial vectors part[p*K + k] (p < P) by the whole block; the result
// for k < K lands in out[k] (written by thread 0). Used by the last CTA of a grid.
template <int K>
__device__ __forceinline__ void reduce_partials(const double* part, int P, double* out) {
  __shared__ double sh[32 * K];      // one slot per warp of the largest block (1024 threads)
  double v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = 0.0;
  for (int p = threadIdx.x; p < P; p += blockDim.x)
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] += __ldcg(part + (int64_t)p * K + k);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[warp * K + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w * K + k];
      out[k] = t;
    }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------
// Fused pass over A
// ---------------------------------------------------------------------------------------
template <typename T, int NR, bool RESID, int VPT>
__global__ void __launch_bounds__(kThreads) apass_kernel(
    const T* __restrict__ A, int64_t lda, int64_t m, int64_t npad, const T* __restrict__ v,
    int64_t ldv, const double* __restrict__ b, T* __restrict__ part,
    double* __restrict__ spart, double* __restrict__ sout, unsigned int* counter,
    const int* __restrict__ done) {
  using V = typename VecOf<T>::type;
  constexpr int VW = VecOf<T>::W;
  constexpr int RT = (VPT >= 8) ? 1 : (8 / VPT);   // rows per tile
  constexpr int E = VPT * VW;                      // elements per thread per row
  __shared__ T red[2][kWarps][NR * RT];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (done != nullptr) {
    bool all = true;
#pragma unroll
    for (int r = 0; r < NR; ++r) all = all && (done[r] != 0);
    if (all) return;   // uniform over the grid: no CTA touches the counter
  }
  T vv[NR][E], acc[NR][E];
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    const int64_t col = ((int64_t)k * kThreads + tid) * VW;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      V x = zero_vec(T(0));
      if (col < npad) x = *reinterpret_cast<const V*>(v + r * ldv + col);
#pragma unroll
      for (int c = 0; c < VW; ++c) { vv[r][k * VW + c] = get(x, c); acc[r][k * VW + c] = T(0); }
    }
  }
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = min(m, r0 + per);
  // per-row scalar sums in the working type: FP64 instructions are very slow on this GPU, so
  // an FP32 kernel must not issue them per row
  T s_cc[NR], s_bc[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) { s_cc[r] = T(0); s_bc[r] = T(0); }
  int buf = 0;
  for (int64_t i0 = r0; i0 < r1; i0 += RT) {
    V a[RT][VPT];
#pragma unroll
    for (int rt = 0; rt < RT; ++rt) {
      const int64_t row = i0 + rt;
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        const int64_t col = ((int64_t)k * kThreads + tid) * VW;
        a[rt][k] = (row < r1 && col < npad)
                       ? __ldcs(reinterpret_cast<const V*>(A + row * lda + col))
                       : zero_vec(T(0));
      }
    }
    T pd[NR][RT];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int rt = 0; rt < RT; ++rt) {
        T t = T(0);
#pragma unroll
        for (int k = 0; k < VPT; ++k)
#pragma unroll
          for (int c = 0; c < VW; ++c) t = fma(get(a[rt][k], c), vv[r][k * VW + c], t);
        pd[r][rt] = warp_sum(t);
      }
    if (lane == 0)
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int rt = 0; rt < RT; ++rt) red[buf][warp][r * RT + rt] = pd[r][rt];
    __syncthreads();
#pragma unroll
    for (int rt = 0; rt < RT; ++rt) {
      const int64_t row = i0 + rt;
      const bool valid = row < r1;
      T brow = T(0);
      if (RESID && valid) brow = (T)b[row];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        T dot = T(0);
#pragma unroll
        for (int w = 0; w < kWarps; ++w) dot += red[buf][w][r * RT + rt];
        T c = T(0);
        if (valid) c = RESID ? (brow - dot) : dot;
        if (tid == 0) {
          s_cc[r] = fma(c, c, s_cc[r]);
          s_bc[r] = fma(brow, c, s_bc[r]);
        }
#pragma unroll
        for (int k = 0; k < VPT; ++k)
#pragma unroll
          for (int cc = 0; cc < VW; ++cc)
            acc[r][k * VW + cc] = fma(c, get(a[rt][k], cc), acc[r][k * VW + cc]);
      }
    }
    buf ^= 1;
  }
  // publish this CTA's partial of A^T c
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    const int64_t col = ((int64_t)k * kThreads + tid) * VW;
    if (col < npad)
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        V x;
        if constexpr (VW == 4) {
          x = make_float4(acc[r][k * 4], acc[r][k * 4 + 1], acc[r][k * 4 + 2], acc[r][k * 4 + 3]);
        } else {
          x = make_double2(acc[r][k * 2], acc[r][k * 2 + 1]);
        }
        *reinterpret_cast<V*>(part + ((int64_t)blockIdx.x * NR + r) * npad + col) = x;
      }
  }
  if (tid == 0)
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      spart[((int64_t)blockIdx.x * NR + r) * 2 + 0] = (double)s_cc[r];
      spart[((int64_t)blockIdx.x * NR + r) * 2 + 1] = (double)s_bc[r];
    }
  if (arrive_last(counter)) {
    reduce_partials<2 * NR>(spart, (int)gridDim.x, sout);
    if (tid == 0) *counter = 0u;
  }
}

// ---------------------------------------------------------------------------------------
// The same fused pass with direct vector loads, software pipelined: a tile of RW rows is
// loaded into registers while the previous tile is reduced, so every thread keeps RW * VPT
// vector loads in flight across the two barriers of a tile. Dots: one shuffle tree per (row,
// RHS) value and warp, then warp 0 sums the kWarps warp partials and broadcasts the NR * RW
// results through shared memory (one read per value per thread instead of kWarps).
// ---------------------------------------------------------------------------------------
template <typename T, int NR, bool RESID, int VPT>
__global__ void __launch_bounds__(kThreads, 1) apass_pipe_kernel(
    const T* __restrict__ A, int64_t lda, int64_t m, int64_t npad, const T* __restrict__ v,
    int64_t ldv, const double* __restrict__ b, T* __restrict__ part,
    double* __restrict__ spart, double* __restrict__ sout, unsigned int* counter,
    const int* __restrict__ done) {
  using V = typename VecOf<T>::type;
  constexpr int VW = VecOf<T>::W;
  constexpr int RW = (VPT >= 16) ? 1 : (16 / VPT);  // rows per tile
  constexpr int E = VPT * VW;
  constexpr int NV = NR * RW;                        // dot values per tile
  __shared__ T red[kWarps][NV];
  __shared__ T full[NV];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (done != nullptr) {
    bool all = true;
#pragma unroll
    for (int r = 0; r < NR; ++r) all = all && (done[r] != 0);
    if (all) return;   // uniform over the grid: no CTA touches the counter
  }
  T vv[NR][E], acc[NR][E];
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    const int64_t col = ((int64_t)k * kThreads + tid) * VW;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      V x = zero_vec(T(0));
      if (col < npad) x = *reinterpret_cast<const V*>(v + r * ldv + col);
#pragma unroll
      for (int c = 0; c < VW; ++c) { vv[r][k * VW + c] = get(x, c); acc[r][k * VW + c] = T(0); }
    }
  }
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = min(m, r0 + per);
  // lane l < NV of warp 0 always reduces value l (RHS l / RW): its sums stay in two scalars
  T s_cc = T(0), s_bc = T(0);
  auto load = [&](V (&a)[RW][VPT], int64_t i0) {
#pragma unroll
    for (int rt = 0; rt < RW; ++rt) {
      const int64_t row = i0 + rt;
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        const int64_t col = ((int64_t)k * kThreads + tid) * VW;
        a[rt][k] = (row < r1 && col < npad)
                       ? __ldcs(reinterpret_cast<const V*>(A + row * lda + col))
                       : zero_vec(T(0));
      }
    }
  };
  auto process = [&](const V (&a)[RW][VPT], int64_t i0) {
    T tv[NV];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int rt = 0; rt < RW; ++rt) {
        T t = T(0);
#pragma unroll
        for (int k = 0; k < VPT; ++k)
#pragma unroll
          for (int c = 0; c < VW; ++c) t = fma(get(a[rt][k], c), vv[r][k * VW + c], t);
        tv[r * RW + rt] = t;
      }
    {
      // one reduce-scatter for the NV row values of the tile (value index lane >> kSh)
      constexpr int kSh = (NV >= 32) ? 0 : (NV >= 16 ? 1 : (NV >= 8 ? 2 : (NV >= 4 ? 3 : (NV >= 2 ? 4 : 5))));
      const T t = warp_reduce_scatter<T, NV>(tv);
      if ((lane & ((1 << kSh) - 1)) == 0) red[warp][lane >> kSh] = t;
    }
    __syncthreads();
    if (warp == 0 && lane < NV) {
      const int rt = lane % RW;
      const int64_t row = i0 + rt;
      T dot = T(0);
#pragma unroll
      for (int w = 0; w < kWarps; ++w) dot += red[w][lane];
      T brow = T(0);
      if (RESID && row < r1) brow = (T)b[row];
      T c = T(0);
      if (row < r1) c = RESID ? (brow - dot) : dot;
      full[lane] = c;
      s_cc = fma(c, c, s_cc);
      s_bc = fma(brow, c, s_bc);
    }
    __syncthreads();
#pragma unroll
    for (int rt = 0; rt < RW; ++rt)
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const T c = full[r * RW + rt];
#pragma unroll
        for (int k = 0; k < VPT; ++k)
#pragma unroll
          for (int cc = 0; cc < VW; ++cc)
            acc[r][k * VW + cc] = fma(c, get(a[rt][k], cc), acc[r][k * VW + cc]);
      }
  };
  V a0[RW][VPT], a1[RW][VPT];
  int64_t i0 = r0;
  if (i0 < r1) load(a0, i0);
  while (i0 < r1) {
    if (i0 + RW < r1) load(a1, i0 + RW);   // next tile in flight during this tile's barriers
    process(a0, i0);
    i0 += RW;
    if (i0 >= r1) break;
    if (i0 + RW < r1) load(a0, i0 + RW);
    process(a1, i0);
    i0 += RW;
  }
  // publish this CTA's partial of A^T c
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    const int64_t col = ((int64_t)k * kThreads + tid) * VW;
    if (col < npad)
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        V x;
        if constexpr (VW == 4) {
          x = make_float4(acc[r][k * 4], acc[r][k * 4 + 1], acc[r][k * 4 + 2], acc[r][k * 4 + 3]);
        } else {
          x = make_double2(acc[r][k * 2], acc[r][k * 2 + 1]);
        }
        *reinterpret_cast<V*>(part + ((int64_t)blockIdx.x * NR + r) * npad + col) = x;
      }
  }
  // scalar sums: lanes < NV of warp 0 hold partials of the rows they reduced
  if (warp == 0) {
    const int rl = lane / RW;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const T cc = warp_sum((lane < NV && rl == r) ? s_cc : T(0));
      const T bc = warp_sum((lane < NV && rl == r) ? s_bc : T(0));
      if (lane == 0) {
        spart[((int64_t)blockIdx.x * NR + r) * 2 + 0] = (double)cc;
        spart[((int64_t)blockIdx.x * NR + r) * 2 + 1] = (double)bc;
      }
    }
  }
  if (arrive_last(counter)) {
    reduce_partials<2 * NR>(spart, (int)gridDim.x, sout);
    if (tid == 0) *counter = 0u;
  }
}

// ---------------------------------------------------------------------------------------
// The same fused pass with the rows staged through shared memory by 1-D bulk async copies
// (cp.async.bulk, completion on mbarriers). A CTA owns a contiguous block of rows, i.e. one
// contiguous span of A, and streams it in tiles of RT rows through a kApStages-deep ring, so
// up to kApStages-1 tiles are in flight while the block reduces the current one. A stage is
// refilled right after the barrier of the following tile, when every thread has finished with
// it. Requires lda == npad (rows back to back).
// ---------------------------------------------------------------------------------------
constexpr int kApStages = 4;

// Layout of the work inside a CTA (kApThreads = 256 or 512 threads), RT = 4 / VPT rows per tile
// (a stage of RT * n_pad elements, about 32 KB at the sizes that matter; VPT is the number of
// axpy-phase vectors per thread, so RT depends on the thread count too):
//  * dot phase: WPR = warps / RT warps share a row; warp w takes segment (w % WPR) of row (w / WPR),
//    so each lane keeps the q values of a fixed column segment (at most 4 vectors) in registers
//    and reduces them with one shuffle tree per row;
//  * axpy phase (after the tile's barrier): thread t owns columns (k * threads + t) * VW, k < VPT,
//    and accumulates c_i A_i over the tile's rows, c_i being the WPR segment sums of row i.
template <typename T, int NR, bool RESID, int VPT, int kApThreads>
__global__ void __launch_bounds__(kApThreads, 1) apass_tma_kernel(
    const T* __restrict__ A, int64_t m, int64_t npad, const T* __restrict__ v, int64_t ldv,
    const double* __restrict__ b, T* __restrict__ part, double* __restrict__ spart,
    double* __restrict__ sout, unsigned int* counter, const int* __restrict__ done, int* err) {
  using V = typename VecOf<T>::type;
  constexpr int VW = VecOf<T>::W;
  constexpr int kApWarps = kApThreads / 32;
  constexpr int RT = 4 / VPT;                      // rows per tile
  constexpr int WPR = kApWarps / RT;               // warps per row in the dot phase
  constexpr int VPS = 4;                           // max vectors per lane in a segment
  constexpr int E = VPT * VW;
  extern __shared__ __align__(128) unsigned char dsm[];
  T* ring = reinterpret_cast<T*>(dsm);
  __shared__ uint64_t full[kApStages];
  __shared__ __align__(16) T segsum[2][RT][NR][WPR];   // double-buffered by tile parity
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (done != nullptr) {
    bool all = true;
#pragma unroll
    for (int r = 0; r < NR; ++r) all = all && (done[r] != 0);
    if (all) return;
  }
  const int my_row = warp / WPR, my_seg = warp % WPR;
  const int64_t seg_len = npad / WPR;
  const int64_t seg0 = (int64_t)my_seg * seg_len;
  T vq[NR][VPS * VW];
#pragma unroll
  for (int u = 0; u < VPS; ++u) {
    const bool ok = ((int64_t)u * 32 + lane) * VW < seg_len;
    const int64_t c = seg0 + ((int64_t)u * 32 + lane) * VW;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      V x = zero_vec(T(0));
      if (ok) x = *reinterpret_cast<const V*>(v + r * ldv + c);
#pragma unroll
      for (int cc = 0; cc < VW; ++cc) vq[r][u * VW + cc] = get(x, cc);
    }
  }
  T acc[NR][E];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int e = 0; e < E; ++e) acc[r][e] = T(0);
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per;
  const int64_t r1 = min(m, r0 + per);
  const int ntiles = (r1 > r0) ? (int)((r1 - r0 + RT - 1) / RT) : 0;
  const int64_t stage_elems = (int64_t)RT * npad;
  const uint64_t pol = ptx::policy_evict_first();   // A is streamed once per pass
  auto issue = [&](int t) {
    const int64_t row = r0 + (int64_t)t * RT;
    const int rows = (int)min((int64_t)RT, r1 - row);
    const uint32_t bytes = (uint32_t)(rows * npad * (int64_t)sizeof(T));
    uint64_t* bar = &full[t % kApStages];
    ptx::mbar_expect_tx(bar, bytes);
    ptx::bulk_g2s_hint(ring + (t % kApStages) * stage_elems, A + row * npad, bytes, bar, pol);
  };
  if (tid == 0) {
    for (int s2 = 0; s2 < kApStages; ++s2) ptx::mbar_init(&full[s2], 1);
    ptx::fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int t = 0; t < kApStages && t < ntiles; ++t) issue(t);
  T s_cc[NR], s_bc[NR];      // per-row scalar sums in the working type (see apass_kernel)
#pragma unroll
  for (int r = 0; r < NR; ++r) { s_cc[r] = T(0); s_bc[r] = T(0); }
  for (int t = 0; t < ntiles; ++t) {
    const int64_t i0 = r0 + (int64_t)t * RT;
    ptx::mbar_wait(&full[t % kApStages], (uint32_t)((t / kApStages) & 1), err, 11);
    const T* tile = ring + (t % kApStages) * stage_elems;
    // ---- dot phase: this warp's segment of row my_row
    {
      T d0[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) d0[r] = T(0);
      if (i0 + my_row < r1) {
        const T* rowp = tile + (int64_t)my_row * npad + seg0;
        V a[VPS];
#pragma unroll
        for (int u = 0; u < VPS; ++u)
          a[u] = (((int64_t)u * 32 + lane) * VW < seg_len)
                     ? *reinterpret_cast<const V*>(rowp + ((int64_t)u * 32 + lane) * VW)
                     : zero_vec(T(0));
#pragma unroll
        for (int u = 0; u < VPS; ++u)
#pragma unroll
          for (int r = 0; r < NR; ++r)
#pragma unroll
            for (int cc = 0; cc < VW; ++cc) d0[r] = fma(get(a[u], cc), vq[r][u * VW + cc], d0[r]);
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) d0[r] = warp_sum(d0[r]);
      if (lane == 0)
#pragma unroll
        for (int r = 0; r < NR; ++r) segsum[t & 1][my_row][r][my_seg] = d0[r];
    }
    __syncthreads();
    // every thread is done with tile t-1: refill its stage with tile t-1+kApStages
    if (tid == 0 && t >= 1 && t - 1 + kApStages < ntiles) {
      ptx::fence_proxy_async();
      issue(t - 1 + kApStages);
    }
    // ---- axpy phase
    V a[RT][VPT];
#pragma unroll
    for (int rt = 0; rt < RT; ++rt)
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        const int64_t col = ((int64_t)k * kApThreads + tid) * VW;
        a[rt][k] = (col < npad && i0 + rt < r1)
                       ? *reinterpret_cast<const V*>(tile + rt * npad + col)
                       : zero_vec(T(0));
      }
#pragma unroll
    for (int rt = 0; rt < RT; ++rt) {
      const int64_t row = i0 + rt;
      if (row >= r1) break;
      T brow = T(0);
      if (RESID) brow = (T)b[row];
      T c[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        T dot = T(0);
        if constexpr (WPR % VW == 0) {
#pragma unroll
          for (int sg = 0; sg < WPR; sg += VW) {
            const V sv = *reinterpret_cast<const V*>(&segsum[t & 1][rt][r][sg]);
#pragma unroll
            for (int cc = 0; cc < VW; ++cc) dot += get(sv, cc);
          }
        } else {
#pragma unroll
          for (int sg = 0; sg < WPR; ++sg) dot += segsum[t & 1][rt][r][sg];
        }
        c[r] = RESID ? (brow - dot) : dot;
        if (tid == 0) {
          s_cc[r] = fma(c[r], c[r], s_cc[r]);
          s_bc[r] = fma(brow, c[r], s_bc[r]);
        }
      }
#pragma unroll
      for (int k = 0; k < VPT; ++k)
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
          for (int cc = 0; cc < VW; ++cc)
            acc[r][k * VW + cc] = fma(c[r], get(a[rt][k], cc), acc[r][k * VW + cc]);
    }
  }
#pragma unroll
  for (int k = 0; k < VPT; ++k) {
    const int64_t col = ((int64_t)k * kApThreads + tid) * VW;
    if (col < npad)
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        V x;
        if constexpr (VW == 4) {
          x = make_float4(acc[r][k * 4], acc[r][k * 4 + 1], acc[r][k * 4 + 2], acc[r][k * 4 + 3]);
        } else {
          x = make_double2(acc[r][k * 2], acc[r][k * 2 + 1]);
        }
        *reinterpret_cast<V*>(part + ((int64_t)blockIdx.x * NR + r) * npad + col) = x;
      }
  }
  if (tid == 0)
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      spart[((int64_t)blockIdx.x * NR + r) * 2 + 0] = (double)s_cc[r];
      spart[((int64_t)blockIdx.x * NR + r) * 2 + 1] = (double)s_bc[r];
    }
  if (arrive_last(counter)) {
    reduce_partials<2 * NR>(spart, (int)gridDim.x, sout);
    if (tid == 0) *counter = 0u;
  }
}

// ---------------------------------------------------------------------------------------
// PCGTLS: reduction of the pass partials and the w / y updates (A-explicit operator)
//   delta = ||t||^2 - sigma^2 ||q||^2, alpha = eta / delta, w += alpha q,
//   y = D^{-1} (A^T t - sigma^2 q)     (so that W^T y = R^{-T}(A^T A q - sigma^2 q))
// grid (npad/32, nr), block 256: warp w sums partial rows w, w+8, ... for 32 columns.
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) pcg_reduce_kernel(
    const T* __restrict__ part, int P, int nr, int64_t npad, const T* __restrict__ q,
    T* __restrict__ w, T* __restrict__ y, const T* __restrict__ dinv, PcgScalars* sc,
    const double* __restrict__ tt) {
  __shared__ T sh[kWarps][33];
  __shared__ T s_alpha, s_sigma2;
  __shared__ int s_ok;
  const int r = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (sc->done[r]) return;
  if (threadIdx.x == 0) {
    // delta_j and alpha_j once per CTA (FP64 instructions are slow; keep them off the threads)
    const double sigma2 = sc->sigma2;
    const double delta = tt[r * 2] - sigma2 * sc->qq[r];
    if (blockIdx.x == 0) sc->delta[r] = delta;
    s_ok = (delta > 0.0) ? 1 : 0;
    const double alpha = s_ok ? sc->eta[r] / delta : 0.0;
    if (blockIdx.x == 0 && s_ok) sc->alpha[r] = alpha;
    s_alpha = (T)alpha;
    s_sigma2 = (T)sigma2;
  }
  const int64_t j = (int64_t)blockIdx.x * 32 + lane;
  T t = T(0);
  if (j < npad) {
    T t0 = T(0), t1 = T(0), t2 = T(0), t3 = T(0);
    int p = warp;
    for (; p + 3 * kWarps < P; p += 4 * kWarps) {
      t0 += part[((int64_t)p * nr + r) * npad + j];
      t1 += part[((int64_t)(p + kWarps) * nr + r) * npad + j];
      t2 += part[((int64_t)(p + 2 * kWarps) * nr + r) * npad + j];
      t3 += part[((int64_t)(p + 3 * kWarps) * nr + r) * npad + j];
    }
    for (; p < P; p += kWarps) t0 += part[((int64_t)p * nr + r) * npad + j];
    t = (t0 + t1) + (t2 + t3);
  }
  sh[warp][lane] = t;
  __syncthreads();
  if (warp != 0) return;
  T at = T(0);
#pragma unroll
  for (int k = 0; k < kWarps; ++k) at += sh[k][lane];
  if (!s_ok) return;                              // loss of positive definiteness (Sec. 3)
  if (j < npad) {
    const T qj = q[r * npad + j];
    w[r * npad + j] = fma(s_alpha, qj, w[r * npad + j]);
    y[r * npad + j] = (at - s_sigma2 * qj) * dinv[j];
  }
}

// Alg. 3 as printed: delta = ||p||^2 - sigma^2 ||q||^2, w += alpha q, y = D^{-1} q.
template <typename T>
__global__ void pcg_update_R_kernel(const T* __restrict__ q, T* __restrict__ w, T* __restrict__ y,
                                    const T* __restrict__ dinv, PcgScalars* sc, int nr,
                                    int64_t npad) {
  __shared__ T s_alpha;
  __shared__ int s_ok;
  const int r = blockIdx.y;
  if (sc->done[r]) return;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (threadIdx.x == 0) {
    const double delta = sc->pp[r] - sc->sigma2 * sc->qq[r];
    if (blockIdx.x == 0) sc->delta[r] = delta;
    s_ok = (delta > 0.0) ? 1 : 0;
    const double alpha = s_ok ? sc->eta[r] / delta : 0.0;
    if (blockIdx.x == 0 && s_ok) sc->alpha[r] = alpha;
    s_alpha = (T)alpha;
  }
  __syncthreads();
  if (!s_ok) return;
  if (j < npad) {
    const T qj = q[r * npad + j];
    w[r * npad + j] = fma(s_alpha, qj, w[r * npad + j]);
    y[r * npad + j] = qj * dinv[j];
  }
}

// ---------------------------------------------------------------------------------------
// Pieces of the two triangular products of a PCGTLS step, shared by the separate kernels and
// the fused step kernel below. `cg` selects L2-only loads (ld.global.cg) for data that other
// CTAs of the same launch wrote (the fused kernel); the separate kernels read through L1.
// ---------------------------------------------------------------------------------------
template <typename T, bool CG>
__device__ __forceinline__ typename VecOf<T>::type ldv(const T* p) {
  using V = typename VecOf<T>::type;
  if constexpr (CG) return __ldcg(reinterpret_cast<const V*>(p));
  else return *reinterpret_cast<const V*>(p);
}

// stage y (nr x npad) into shared memory with vector loads, several in flight per thread
template <typename T, bool CG>
__device__ __forceinline__ void stage_vec(const T* __restrict__ y, T* ys, int nr, int64_t npad) {
  using V = typename VecOf<T>::type;
  constexpr int VW = VecOf<T>::W;
  const int tid = threadIdx.x;
  const int64_t nv = nr * npad / VW;
  for (int64_t e0 = tid; e0 < nv; e0 += 4 * kThreads) {
    V t[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t e = e0 + (int64_t)u * kThreads;
      t[u] = (e < nv) ? ldv<T, CG>(y + e * VW) : zero_vec(T(0));
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t e = e0 + (int64_t)u * kThreads;
      if (e < nv) reinterpret_cast<V*>(ys)[e] = t[u];
    }
  }
}

// stage p_j = s + beta_{j-1} p_{j-1} (nr x npad) into shared memory
template <typename T, bool CG>
__device__ __forceinline__ void stage_p(const T* __restrict__ s, const T* __restrict__ p_prev,
                                        T* ps, int nr, int64_t npad, T beta0, T beta1) {
  using V = typename VecOf<T>::type;
  constexpr int VW = VecOf<T>::W;
  const int tid = threadIdx.x;
  const int64_t nv = nr * npad / VW;
  for (int64_t e0 = tid; e0 < nv; e0 += 4 * kThreads) {
    V sv[4], pv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t e = e0 + (int64_t)u * kThreads;
      sv[u] = (e < nv) ? ldv<T, CG>(s + e * VW) : zero_vec(T(0));
      pv[u] = (e < nv) ? ldv<T, CG>(p_prev + e * VW) : zero_vec(T(0));
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t e = e0 + (int64_t)u * kThreads;
      if (e < nv) {
        const T bt = (e * VW < npad) ? beta0 : beta1;
        V o;
        if constexpr (VW == 4) {
          o = make_float4(sv[u].x + bt * pv[u].x, sv[u].y + bt * pv[u].y,
                          sv[u].z + bt * pv[u].z, sv[u].w + bt * pv[u].w);
        } else {
          o = make_double2(sv[u].x + bt * pv[u].x, sv[u].y + bt * pv[u].y);
        }
        reinterpret_cast<V*>(ps)[e] = o;
      }
    }
  }
}

// Rows gw, gw + GW, ... of v = W^T y (WT = W^T lower triangular, entries 0..j of row j) and the
// s recurrence of those rows; ss accumulates ||s||^2 over the rows of the calling lane 0.
template <typename T, int U>
__device__ __forceinline__ void wt_rows(const T* __restrict__ WT, int64_t npad, const T* ys,
                                        T* __restrict__ s, const T* __restrict__ p, bool act0,
                                        bool act1, T alpha0, T alpha1, T sigma2, bool init,
                                        bool modeA, int nr, int64_t gw, int64_t GW, T (&ss)[2]) {
  using V = typename VecOf<T>::type;
  constexpr int VW = VecOf<T>::W;
  const int lane = threadIdx.x & 31;
  for (int64_t j = gw; j < npad; j += GW) {
    const T* row = WT + j * npad;
    const int64_t lim = ((j + VW) / VW) * VW;    // entries 0..j, rounded up (zeros beyond j)
    T a0 = T(0), a1 = T(0);
    for (int64_t cb = (int64_t)lane * VW; cb < lim; cb += 32 * VW * U) {
      V wv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t c = cb + (int64_t)u * 32 * VW;
        wv[u] = (c < lim) ? *reinterpret_cast<const V*>(row + c) : zero_vec(T(0));
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t c = cb + (int64_t)u * 32 * VW;
        if (c < lim) {
          const V y0 = *reinterpret_cast<const V*>(ys + c);
#pragma unroll
          for (int k = 0; k < VW; ++k) a0 = fma(get(wv[u], k), get(y0, k), a0);
          if (nr > 1) {
            const V y1 = *reinterpret_cast<const V*>(ys + npad + c);
#pragma unroll
            for (int k = 0; k < VW; ++k) a1 = fma(get(wv[u], k), get(y1, k), a1);
          }
        }
      }
    }
    a0 = warp_sum(a0);
    if (nr > 1) a1 = warp_sum(a1);
    if (lane == 0) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        if (r >= nr) break;
        const T vr = r ? a1 : a0;
        const bool act = r ? act1 : act0;
        const T al = r ? alpha1 : alpha0;
        T* sp = s + r * npad + j;
        T sv = *sp;
        if (init) sv = vr;
        else if (act) {
          if (modeA) sv = sv - al * vr;
          else sv = sv - al * (p[r * npad + j] - sigma2 * vr);
        }
        if (init || act) *sp = sv;
        ss[r] = fma(sv, sv, ss[r]);
      }
    }
  }
}

// Rows gw, gw + GW, ... of q = D^{-1} W p (W upper triangular) from the staged p; acc4
// accumulates ||q||^2 (two RHS) and ||p||^2 (two RHS) over the rows of the calling lane 0.
template <typename T, int U>
__device__ __forceinline__ void w_rows(const T* __restrict__ W, int64_t npad, const T* ps,
                                       const T* __restrict__ dinv, T* __restrict__ q, int nr,
                                       int64_t gw, int64_t GW, T (&acc4)[4]) {
  using V = typename VecOf<T>::type;
  constexpr int VW = VecOf<T>::W;
  const int lane = threadIdx.x & 31;
  for (int64_t i = gw; i < npad; i += GW) {
    const T* row = W + i * npad;
    T a0 = T(0), a1 = T(0);
    for (int64_t cb = (i / VW) * VW + (int64_t)lane * VW; cb < npad; cb += 32 * VW * U) {
      V wv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t c = cb + (int64_t)u * 32 * VW;
        wv[u] = (c < npad) ? *reinterpret_cast<const V*>(row + c) : zero_vec(T(0));
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t c = cb + (int64_t)u * 32 * VW;
        if (c < npad) {
          const V p0 = *reinterpret_cast<const V*>(ps + c);
#pragma unroll
          for (int k = 0; k < VW; ++k) a0 = fma(get(wv[u], k), get(p0, k), a0);
          if (nr > 1) {
            const V p1 = *reinterpret_cast<const V*>(ps + npad + c);
#pragma unroll
            for (int k = 0; k < VW; ++k) a1 = fma(get(wv[u], k), get(p1, k), a1);
          }
        }
      }
    }
    a0 = warp_sum(a0);
    if (nr > 1) a1 = warp_sum(a1);
    if (lane == 0) {
      const T di = dinv[i];
      const T q0 = a0 * di;
      q[i] = q0;
      acc4[0] = fma(q0, q0, acc4[0]);
      acc4[2] = fma(ps[i], ps[i], acc4[2]);
      if (nr > 1) {
        const T q1 = a1 * di;
        q[npad + i] = q1;
        acc4[1] = fma(q1, q1, acc4[1]);
        acc4[3] = fma(ps[npad + i], ps[npad + i], acc4[3]);
      }
    }
  }
}

// CTA partial sums (FP64) of K per-lane values into part[slot * K + k]
template <typename T, int K>
__device__ __forceinline__ void cta_partials(T (&v)[K], double* red /* kWarps * K */,
                                             double* part, int64_t slot) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) red[warp * K + k] = (double)v[k];
  __syncthreads();
  if (tid == 0)   // one writer: its fence before the arrival publishes all K values
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double t = 0.0;
      for (int w2 = 0; w2 < kWarps; ++w2) t += red[w2 * K + k];
      part[slot * K + k] = t;
    }
}

// eta_{j+1}, beta_j and the termination flags of Alg. 3 from eta_new (one RHS r).
__device__ __forceinline__ void eta_update(double eta_new, bool init, double& eta, double& eta0,
                                           double& beta, int& done, int& iters, int& not_spd,
                                           double delta, double cg_tol2) {
  if (init) {
    eta = eta_new;
    eta0 = eta_new;
    beta = 0.0;
    done = (eta_new == 0.0) ? 1 : 0;
    iters = 0;
  } else if (!done) {
    if (!(delta > 0.0)) {
      done = 1;
      not_spd = (delta < 0.0) ? 1 : 0;
    } else {
      beta = eta_new / eta;
      eta = eta_new;
      iters += 1;
      if (eta_new == 0.0 || (cg_tol2 > 0.0 && eta_new <= cg_tol2 * eta0)) done = 1;
    }
  }
}

// ---------------------------------------------------------------------------------------
// v = W^T y (row products with WT = W^T, lower triangular), then the s recurrence:
//   init: s = v, eta_0 = ||s||^2                     (s_0 = R^{-T} f)
//   step: s -= alpha v (A-explicit) or s -= alpha (p - sigma^2 v) (as printed)
// last CTA: eta_{j+1}, beta_j = eta_{j+1}/eta_j, termination flags.
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) gemv_wt_kernel(
    const T* __restrict__ WT, int64_t npad, const T* __restrict__ y, T* __restrict__ s,
    const T* __restrict__ p, double* __restrict__ part, PcgScalars* sc, int init, int modeA,
    int nr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ys = reinterpret_cast<T*>(smem_raw);
  __shared__ double red[kWarps * 2];
  const int tid = threadIdx.x, warp = tid >> 5;
  const bool act0 = 0 < nr && (init || (!sc->done[0] && sc->delta[0] > 0.0));
  const bool act1 = 1 < nr && (init || (!sc->done[1] && sc->delta[1] > 0.0));
  const T alpha0 = init ? T(0) : (T)sc->alpha[0];
  const T alpha1 = init ? T(0) : (T)sc->alpha[1];
  const T sigma2 = (T)sc->sigma2;
  stage_vec<T, false>(y, ys, nr, npad);
  __syncthreads();
  T ss[2] = {T(0), T(0)};
  wt_rows<T, 8>(WT, npad, ys, s, p, act0, act1, alpha0, alpha1, sigma2, init != 0, modeA != 0, nr,
             (int64_t)blockIdx.x * kWarps + warp, (int64_t)gridDim.x * kWarps, ss);
  cta_partials<T, 2>(ss, red, part, blockIdx.x);
  if (arrive_last(&sc->counter[0])) {
    __shared__ double eta_sum[2];
    reduce_partials<2>(part, (int)gridDim.x, eta_sum);
    if (tid < nr) {
      const int r = tid;
      double eta = sc->eta[r], eta0 = sc->eta0[r], beta = sc->beta[r];
      int done = sc->done[r], iters = sc->iters[r], nspd = sc->not_spd[r];
      eta_update(eta_sum[r], init != 0, eta, eta0, beta, done, iters, nspd, sc->delta[r],
                 sc->cg_tol2);
      sc->eta[r] = eta;
      sc->eta0[r] = eta0;
      sc->beta[r] = beta;
      sc->done[r] = done;
      sc->iters[r] = iters;
      sc->not_spd[r] = nspd;
    }
    if (tid == 0) sc->counter[0] = 0u;
  }
}

// ---------------------------------------------------------------------------------------
// p_j = s_j + beta_{j-1} p_{j-1}; q_j = D^{-1} W p_j; partials of ||q||^2 and ||p||^2.
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) gemv_w_kernel(
    const T* __restrict__ W, int64_t npad, const T* __restrict__ s, const T* __restrict__ p_prev,
    T* __restrict__ p_out, const T* __restrict__ dinv, T* __restrict__ q,
    double* __restrict__ part, PcgScalars* sc, int nr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ps = reinterpret_cast<T*>(smem_raw);
  __shared__ double red[kWarps * 4];
  const int tid = threadIdx.x, warp = tid >> 5;
  const T beta0 = (T)sc->beta[0], beta1 = (T)(nr > 1 ? sc->beta[1] : 0.0);
  stage_p<T, false>(s, p_prev, ps, nr, npad, beta0, beta1);
  __syncthreads();
  {
    const int64_t chunk = (nr * npad + gridDim.x - 1) / gridDim.x;
    const int64_t e0 = (int64_t)blockIdx.x * chunk, e1 = min((int64_t)nr * npad, e0 + chunk);
    for (int64_t e = e0 + tid; e < e1; e += kThreads) p_out[e] = ps[e];
  }
  T acc4[4] = {T(0), T(0), T(0), T(0)};   // qq0, qq1, pp0, pp1 (working type: no FP64 per row)
  w_rows<T, 8>(W, npad, ps, dinv, q, nr, (int64_t)blockIdx.x * kWarps + warp,
            (int64_t)gridDim.x * kWarps, acc4);
  cta_partials<T, 4>(acc4, red, part, blockIdx.x);
  if (arrive_last(&sc->counter[1])) {
    __shared__ double qp[4];
    reduce_partials<4>(part, (int)gridDim.x, qp);
    if (tid < 4) {
      if (tid < 2) sc->qq[tid] = qp[tid];
      else sc->pp[tid - 2] = qp[tid];
    }
    if (tid == 0) sc->counter[1] = 0u;
  }
}

// Arrival count over the grid (thread 0 only): true in the last CTA to arrive, which also resets
// the counter. The caller has fenced its writes. (A two-level count, 8 groups then the top,
// measured no faster: the barrier's cost is the round trip through L2, not contention.)
__device__ __forceinline__ bool arrive_count(unsigned int* cnt) {
  if (atomicAdd(cnt, 1u) != gridDim.x - 1u) return false;
  atomicExch(cnt, 0u);
  return true;
}

// ---------------------------------------------------------------------------------------
// Grid-wide barrier of a cooperative launch (every CTA is resident). bar: [0] the arrival
// counter, [9] the generation word. The last CTA to arrive runs `last(...)` with all
// its threads before it releases the others (a reduction every CTA needs after the barrier
// is done once there instead of by every CTA). The wait is bounded: after 2^22 polls (each an
// L2 round trip, a few seconds in all) it records code 3 in *err and goes on; the host then
// reports the solve as timed out.
// ---------------------------------------------------------------------------------------
template <typename F>
__device__ __forceinline__ void grid_sync_last(unsigned int* bar, int* err, F&& last) {
  __shared__ int s_last;
  __shared__ unsigned int s_gen;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = bar + 9;
    s_gen = *gen;
    __threadfence();
    s_last = arrive_count(bar) ? 1 : 0;
  }
  __syncthreads();
  if (s_last) {
    last();
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(bar + 9, 1u);
    }
  } else if (threadIdx.x == 0) {
    volatile unsigned int* gen = bar + 9;
    unsigned int it = 0;
    while (*gen == s_gen) {
      if (++it > (1u << 22)) {
        atomicExch(err, 3);
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------
// The tail of PCGTLS step j and the head of step j + 1 in one cooperative launch, A-explicit
// operator (Alg. 3 / 4), every CTA resident:
//   R: column sums of the pass partials, delta_j, alpha_j, w += alpha q, y = D^{-1}(A^T t - s2 q)
//   -- grid barrier --
//   T: v = W^T y, s -= alpha v; partials of ||s||^2
//   -- grid barrier --
//   every CTA sums those partials itself (same order everywhere): eta_{j+1}, beta_j, flags;
//   CTA 0 stores them. If a step j + 1 follows:
//   S: p_{j+1} = s + beta_j p_j, q_{j+1} = D^{-1} W p_{j+1}; the last CTA stores ||q||^2, ||p||^2.
// Data written by other CTAs of this launch is read with ld.global.cg (L1 is not coherent).
// The three phases replace the pcg_reduce, gemv_wt and gemv_w launches with the same
// arithmetic; virtual block b of a phase stands for CTA b of the separate launch.
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) pcg_step_kernel(
    const T* __restrict__ part, int P, int nr, int64_t npad, T* __restrict__ q,
    T* __restrict__ w, T* __restrict__ y, const T* __restrict__ dinv, PcgScalars* sc,
    const double* __restrict__ tt, const T* __restrict__ WT, const T* __restrict__ W,
    T* __restrict__ s, const T* __restrict__ p_cur, T* __restrict__ p_next, double* gpart,
    int gemv_blocks, int next, unsigned int* bar, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* vs = reinterpret_cast<T*>(smem_raw);
  __shared__ T sh[16][17];
  __shared__ T s_alpha[2], s_sigma2;
  __shared__ int s_ok[2];
  __shared__ double red[kWarps * 4];
  __shared__ double s_eta_new[2];
  constexpr int kStepU = (sizeof(T) == 4) ? 16 : 8;   // vector loads in flight per lane
  const int tid = threadIdx.x, warp = tid >> 5;
  // nothing to do once every right-hand side has stopped (the flags are only written after the
  // second barrier, so every CTA takes the same branch)
  if (sc->done[0] && (nr < 2 || sc->done[1])) return;
  // scalars of step j as the previous launches left them (thread 0; shared with the CTA)
  __shared__ double s_eta[2], s_eta0[2], s_beta[2], s_delta[2];
  __shared__ int s_done[2], s_iters[2], s_nspd[2];
  if (tid == 0) {
    const double sigma2 = sc->sigma2;
    for (int r = 0; r < 2; ++r) {
      s_done[r] = sc->done[r];
      s_eta[r] = sc->eta[r];
      s_eta0[r] = sc->eta0[r];
      s_beta[r] = sc->beta[r];
      s_iters[r] = sc->iters[r];
      s_nspd[r] = sc->not_spd[r];
      s_delta[r] = sc->delta[r];
      s_ok[r] = 0;
      s_alpha[r] = T(0);
      if (r < nr && !s_done[r]) {
        const double delta = tt[r * 2] - sigma2 * sc->qq[r];
        s_delta[r] = delta;
        s_ok[r] = (delta > 0.0) ? 1 : 0;
        const double alpha = s_ok[r] ? s_eta[r] / delta : 0.0;
        if (blockIdx.x == 0) {
          sc->delta[r] = delta;
          if (s_ok[r]) sc->alpha[r] = alpha;
        }
        s_alpha[r] = (T)alpha;
      }
    }
    s_sigma2 = (T)sigma2;
  }
  __syncthreads();
  // ---- R: reduction of the pass partials: virtual blocks of 16 consecutive entries of the
  // nr x npad partial vectors; thread (slice ps, entry c) sums the partials p = ps (mod 16)
  // with every load in flight, then 16 threads add the 16 slices
  {
    const int c = tid & 15, ps = tid >> 4;
    const int64_t nvb = (int64_t)nr * npad / 16;
    for (int64_t vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
      const int64_t e0 = vb * 16;
      const int r = (int)(e0 / npad);
      if (s_done[r]) continue;   // uniform over the CTA
      const int64_t e = e0 + c;
      T t0 = T(0), t1 = T(0);
      int pp = ps;
      for (; pp + 16 < P; pp += 32) {
        t0 += part[(int64_t)pp * nr * npad + e];
        t1 += part[(int64_t)(pp + 16) * nr * npad + e];
      }
      if (pp < P) t0 += part[(int64_t)pp * nr * npad + e];
      sh[ps][c] = t0 + t1;
      __syncthreads();
      if (tid < 16 && s_ok[r]) {
        T at = T(0);
#pragma unroll
        for (int k = 0; k < 16; ++k) at += sh[k][tid];
        const int64_t j = e - (int64_t)r * npad;
        const T qj = q[e];
        w[e] = fma(s_alpha[r], qj, w[e]);
        y[e] = (at - s_sigma2 * qj) * dinv[j];
      }
      __syncthreads();
    }
  }
  grid_sync_last(bar, err, [] {});
  // ---- T: v = W^T y and the s recurrence (virtual grid gemv_blocks)
  const bool act0 = 0 < nr && !s_done[0] && s_delta[0] > 0.0;
  const bool act1 = 1 < nr && !s_done[1] && s_delta[1] > 0.0;
  for (int vb = blockIdx.x; vb < gemv_blocks; vb += gridDim.x) {
    stage_vec<T, true>(y, vs, nr, npad);
    __syncthreads();
    T ss[2] = {T(0), T(0)};
    wt_rows<T, kStepU>(WT, npad, vs, s, p_cur, act0, act1, s_alpha[0], s_alpha[1], s_sigma2, false,
               true, nr, (int64_t)vb * kWarps + warp, (int64_t)gemv_blocks * kWarps, ss);
    cta_partials<T, 2>(ss, red, gpart, vb);
    __syncthreads();
  }
  // ---- eta_{j+1}, beta_j and the flags, by the last CTA to reach the barrier; every CTA
  // reads beta from sc afterwards (L2 loads: the values were written after this launch began)
  grid_sync_last(bar, err, [&] {
    reduce_partials<2>(gpart, gemv_blocks, s_eta_new);
    __syncthreads();
    if (tid == 0) {
      const double cg_tol2 = sc->cg_tol2;
      for (int r = 0; r < nr; ++r) {
        double eta = s_eta[r], eta0 = s_eta0[r], beta = s_beta[r];
        int done = s_done[r], iters = s_iters[r], nspd = s_nspd[r];
        eta_update(s_eta_new[r], false, eta, eta0, beta, done, iters, nspd, s_delta[r], cg_tol2);
        sc->eta[r] = eta;
        sc->eta0[r] = eta0;
        sc->beta[r] = beta;
        sc->done[r] = done;
        sc->iters[r] = iters;
        sc->not_spd[r] = nspd;
      }
    }
  });
  if (tid == 0) {
    s_beta[0] = __ldcg(&sc->beta[0]);
    s_beta[1] = __ldcg(&sc->beta[1]);
  }
  __syncthreads();
  if (!next) return;
  // ---- S: p_{j+1}, q_{j+1} (virtual grid gemv_blocks)
  const T beta0 = (T)s_beta[0], beta1 = (T)(nr > 1 ? s_beta[1] : 0.0);
  for (int vb = blockIdx.x; vb < gemv_blocks; vb += gridDim.x) {
    stage_p<T, true>(s, p_cur, vs, nr, npad, beta0, beta1);
    __syncthreads();
    {
      const int64_t chunk = (nr * npad + gemv_blocks - 1) / gemv_blocks;
      const int64_t e0 = (int64_t)vb * chunk, e1 = min((int64_t)nr * npad, e0 + chunk);
      for (int64_t e = e0 + tid; e < e1; e += kThreads) p_next[e] = vs[e];
    }
    T acc4[4] = {T(0), T(0), T(0), T(0)};
    w_rows<T, kStepU>(W, npad, vs, dinv, q, nr, (int64_t)vb * kWarps + warp,
              (int64_t)gemv_blocks * kWarps, acc4);
    cta_partials<T, 4>(acc4, red, gpart + 2048, vb);
    __syncthreads();
  }
  // ||q||^2, ||p||^2 by the last CTA to finish (the others leave)
  __shared__ int s_lastq;
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    s_lastq = arrive_count(bar + 10) ? 1 : 0;
  }
  __syncthreads();
  if (s_lastq) {
    __threadfence();
    __shared__ double qp[4];
    reduce_partials<4>(gpart + 2048, gemv_blocks, qp);
    if (tid < 4) {
      if (tid < 2) sc->qq[tid] = qp[tid];
      else sc->pp[tid - 2] = qp[tid];
    }
  }
}

template <typename T>
__global__ void pcg_prep_kernel(const double* __restrict__ fin0, double fin0_scale,
                                const double* __restrict__ fin1, int nr, int64_t n,
                                int64_t npad, const double* __restrict__ dinv, T* y, T* w,
                                T* p0, T* p1, PcgScalars* sc, double sigma2, double cg_tol) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < npad) {
    for (int r = 0; r < nr; ++r) {
      double f = 0.0;
      if (j < n) f = (r == 0) ? fin0_scale * fin0[j] : fin1[j];
      y[r * npad + j] = (T)(f * dinv[j]);
      w[r * npad + j] = T(0);
      p0[r * npad + j] = T(0);
      p1[r * npad + j] = T(0);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int r = 0; r < 2; ++r) {
      sc->eta[r] = 0.0; sc->eta0[r] = 0.0; sc->qq[r] = 0.0; sc->pp[r] = 0.0; sc->tt[r] = 0.0;
      sc->alpha[r] = 0.0; sc->beta[r] = 0.0; sc->delta[r] = 1.0;
      sc->done[r] = (r < nr) ? 0 : 1; sc->not_spd[r] = 0; sc->iters[r] = 0;
    }
    sc->sigma2 = sigma2;
    sc->cg_tol2 = cg_tol * cg_tol;
    sc->nr = nr;
  }
}

// ---------------------------------------------------------------------------------------
// RQI residual (FP64): f = -A^T r - sigma2 x, sigma2 = rr / (1 + xx), g = -b^T r + sigma2,
// psi = sqrt((||f||^2 + g^2)/(xx + 1))   (Alg. 2 lines r_k..g_k, Eq. (2), Eq. (4))
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) resid_reduce_kernel(
    const double* __restrict__ part, int P, int64_t npad, const double* __restrict__ x,
    double* __restrict__ f, const double* __restrict__ sout, RqiScalars* rs,
    double* __restrict__ fpart) {
  __shared__ double sh[kWarps][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * 32 + lane;
  double t = 0.0;
  if (j < npad) {
    double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
    int p = warp;
    for (; p + 3 * kWarps < P; p += 4 * kWarps) {
      t0 += part[(int64_t)p * npad + j];
      t1 += part[(int64_t)(p + kWarps) * npad + j];
      t2 += part[(int64_t)(p + 2 * kWarps) * npad + j];
      t3 += part[(int64_t)(p + 3 * kWarps) * npad + j];
    }
    for (; p < P; p += kWarps) t0 += part[(int64_t)p * npad + j];
    t = (t0 + t1) + (t2 + t3);
  }
  sh[warp][lane] = t;
  __syncthreads();
  const double xx = rs->xx;
  const double sigma2 = sout[0] / (1.0 + xx);
  double ff = 0.0;
  if (warp == 0) {
    double at = 0.0;
#pragma unroll
    for (int k = 0; k < kWarps; ++k) at += sh[k][lane];
    if (j < npad) {
      const double fj = -at - sigma2 * x[j];
      f[j] = fj;
      ff = fj * fj;
    }
    ff = warp_sum(ff);
    if (lane == 0) fpart[blockIdx.x] = ff;
  }
  if (arrive_last(&rs->counter[0])) {
    __shared__ double tfs[1];
    reduce_partials<1>(fpart, (int)gridDim.x, tfs);
    if (threadIdx.x == 0) {
      const double tf = tfs[0];
      const double rr = sout[0], br = sout[1];
      const double g = -br + sigma2;
      rs->rr = rr;
      rs->br = br;
      rs->sigma2 = sigma2;
      rs->g = g;
      rs->ff = tf;
      rs->psi = sqrt((tf + g * g) / (xx + 1.0));
      rs->counter[0] = 0u;
    }
  }
}

// x_{k+1} = z_k + beta_k u_k, z_k = x_k + w_k, beta_k = (z^T f - g)/(z^T x + 1) (Alg. 2)
template <typename T>
__global__ void __launch_bounds__(1024) rqi_update_kernel(double* __restrict__ x,
                                                          const T* __restrict__ w,
                                                          const T* __restrict__ u,
                                                          const double* __restrict__ f,
                                                          RqiScalars* rs, int64_t n) {
  __shared__ double sh[32 * 2];
  double v[2] = {0.0, 0.0};
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double z = x[j] + (double)w[j];
    v[0] = fma(z, f[j], v[0]);
    v[1] = fma(z, x[j], v[1]);
  }
  block_sum<2>(v, sh);
  const double betak = (v[0] - rs->g) / (v[1] + 1.0);
  double xx[1] = {0.0};
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double z = x[j] + (double)w[j];
    const double xn = fma(betak, (double)u[j], z);
    x[j] = xn;
    xx[0] = fma(xn, xn, xx[0]);
  }
  block_sum<1>(xx, sh);
  if (threadIdx.x == 0) {
    rs->zf = v[0];
    rs->zx = v[1];
    rs->betak = betak;
    rs->xx = xx[0];
  }
}

// The same update over several CTAs (the FP64 arithmetic of one CTA on this GPU, at 2 lanes
// per clock per SM, made the single-block form take about 20 us): rqi_dots_kernel forms the
// CTAs' partials of z^T f and z^T x and the last CTA adds them in CTA order into beta_k;
// xupd_kernel<T, 2> writes x_{k+1} and ||x_{k+1}||^2.
template <typename T>
__global__ void __launch_bounds__(256) rqi_dots_kernel(const double* __restrict__ x,
                                                       const T* __restrict__ w,
                                                       const double* __restrict__ f,
                                                       RqiScalars* rs, int64_t n,
                                                       double* __restrict__ part) {
  __shared__ double sh[kWarps * 2];
  double v[2] = {0.0, 0.0};
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const double z = x[j] + (double)w[j];
    v[0] = fma(z, f[j], v[0]);
    v[1] = fma(z, x[j], v[1]);
  }
  block_sum<2>(v, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = v[0];
    part[2 * blockIdx.x + 1] = v[1];
  }
  if (arrive_last(&rs->counter[1])) {
    if (threadIdx.x == 0) {
      double zf = 0.0, zx = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b) {
        zf += __ldcg(part + 2 * b);
        zx += __ldcg(part + 2 * b + 1);
      }
      rs->zf = zf;
      rs->zx = zx;
      rs->betak = (zf - rs->g) / (zx + 1.0);
      rs->counter[1] = 0u;
    }
  }
}

// x updates with ||x||^2 over several CTAs (partials added in CTA order by the last CTA):
// MODE 0: x = w (the LS start); 1: x = x + sigma^2 u (the inverse-iteration step);
// 2: x = x + w + beta_k u (the RQI update). Any T for w and u.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) xupd_kernel(double* __restrict__ x,
                                                   const T* __restrict__ w,
                                                   const T* __restrict__ u, RqiScalars* rs,
                                                   int64_t n, double* __restrict__ part) {
  __shared__ double sh[kWarps];
  const double c = (MODE == 1) ? rs->sigma2 : (MODE == 2 ? rs->betak : 0.0);
  double xx[1] = {0.0};
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    double xn;
    if constexpr (MODE == 0) xn = (double)w[j];
    else if constexpr (MODE == 1) xn = fma(c, (double)u[j], x[j]);
    else xn = fma(c, (double)u[j], x[j] + (double)w[j]);
    x[j] = xn;
    xx[0] = fma(xn, xn, xx[0]);
  }
  block_sum<1>(xx, sh);
  if (threadIdx.x == 0) part[64 + blockIdx.x] = xx[0];
  if (arrive_last(&rs->counter[2])) {
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(part + 64 + b);
      rs->xx = t;
      rs->counter[2] = 0u;
    }
  }
}

// ||x||^2 over several CTAs (same partial scheme; x read only)
__global__ void __launch_bounds__(256) xx_multi_kernel(const double* __restrict__ x,
                                                       RqiScalars* rs, int64_t n,
                                                       double* __restrict__ part) {
  __shared__ double sh[kWarps];
  double xx[1] = {0.0};
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    xx[0] = fma(x[j], x[j], xx[0]);
  block_sum<1>(xx, sh);
  if (threadIdx.x == 0) part[64 + blockIdx.x] = xx[0];
  if (arrive_last(&rs->counter[2])) {
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(part + 64 + b);
      rs->xx = t;
      rs->counter[2] = 0u;
    }
  }
}

// x = x + sigma2 * u (Alg. 2, the inverse-iteration step before the loop)
template <typename T>
__global__ void __launch_bounds__(1024) inverse_step_kernel(double* __restrict__ x,
                                                            const T* __restrict__ u,
                                                            RqiScalars* rs, int64_t n) {
  __shared__ double sh[32];
  const double s2 = rs->sigma2;
  double xx[1] = {0.0};
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double xn = fma(s2, (double)u[j], x[j]);
    x[j] = xn;
    xx[0] = fma(xn, xn, xx[0]);
  }
  block_sum<1>(xx, sh);
  if (threadIdx.x == 0) rs->xx = xx[0];
}

template <typename T>
__global__ void __launch_bounds__(1024) copy_to_x_kernel(double* __restrict__ x,
                                                         const T* __restrict__ w, RqiScalars* rs,
                                                         int64_t n) {
  __shared__ double sh[32];
  double xx[1] = {0.0};
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double xn = (double)w[j];
    x[j] = xn;
    xx[0] = fma(xn, xn, xx[0]);
  }
  block_sum<1>(xx, sh);
  if (threadIdx.x == 0) rs->xx = xx[0];
}

__global__ void __launch_bounds__(1024) xx_kernel(const double* __restrict__ x, RqiScalars* rs,
                                                  int64_t n) {
  __shared__ double sh[32];
  double xx[1] = {0.0};
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) xx[0] = fma(x[j], x[j], xx[0]);
  block_sum<1>(xx, sh);
  if (threadIdx.x == 0) rs->xx = xx[0];
}

template <typename T>
__global__ void vec_convert_kernel(const double* __restrict__ in, T* __restrict__ out, int64_t n,
                                   int64_t npad) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < npad) out[j] = (j < n) ? (T)in[j] : T(0);
}

inline int blocks_for(int64_t count, int threads) { return (int)((count + threads - 1) / threads); }

template <typename T, int NR, bool RESID, int TH>
void apass_tma_dispatch_th(int vpt, dim3 grid, size_t smem, const T* A, int64_t m, int64_t npad,
                           const T* v, int64_t ldv, const double* b, T* part, double* spart,
                           double* sout, unsigned int* counter, const int* done, int* err,
                           cudaStream_t s) {
  switch (vpt) {
#define TLS_AT(V)                                                                               \
  case V: {                                                                                     \
    static const bool attr = [] {                                                               \
      cudaFuncSetAttribute(apass_tma_kernel<T, NR, RESID, V, TH>,                              \
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);            \
      return true;                                                                              \
    }();                                                                                        \
    (void)attr;                                                                                 \
    apass_tma_kernel<T, NR, RESID, V, TH><<<grid, TH, smem, s>>>(A, m, npad, v, ldv, b, part,   \
                                                               spart, sout, counter, done,    \
                                                               err);                          \
    count_launch();                                                                             \
    break;                                                                                      \
  }
    TLS_AT(1) TLS_AT(2) TLS_AT(4)
#undef TLS_AT
    default: break;
  }
}

template <typename T, int NR, bool RESID>
void apass_tma_dispatch(int threads, int vpt, dim3 grid, size_t smem, const T* A, int64_t m,
                        int64_t npad, const T* v, int64_t ldv, const double* b, T* part,
                        double* spart, double* sout, unsigned int* counter, const int* done,
                        int* err, cudaStream_t s) {
  if (threads == 512)
    apass_tma_dispatch_th<T, NR, RESID, 512>(vpt, grid, smem, A, m, npad, v, ldv, b, part, spart,
                                              sout, counter, done, err, s);
  else
    apass_tma_dispatch_th<T, NR, RESID, 256>(vpt, grid, smem, A, m, npad, v, ldv, b, part, spart,
                                              sout, counter, done, err, s);
}

template <typename T, int NR, bool RESID>
void apass_pipe_dispatch(int vpt, dim3 grid, const T* A, int64_t lda, int64_t m, int64_t npad,
                         const T* v, int64_t ldv, const double* b, T* part, double* spart,
                         double* sout, unsigned int* counter, const int* done, cudaStream_t s) {
  switch (vpt) {
#define TLS_AP(V) \
  case V: apass_pipe_kernel<T, NR, RESID, V><<<grid, kThreads, 0, s>>>(A, lda, m, npad, v, ldv, b, part, spart, sout, counter, done); count_launch(); break;
    TLS_AP(1) TLS_AP(2) TLS_AP(4) TLS_AP(8)
#undef TLS_AP
    default: break;
  }
}
template <typename T, int NR, bool RESID>
void apass_dispatch(int vpt, dim3 grid, const T* A, int64_t lda, int64_t m, int64_t npad,
                    const T* v, int64_t ldv, const double* b, T* part, double* spart,
                    double* sout, unsigned int* counter, const int* done, cudaStream_t s) {
  switch (vpt) {
#define TLS_AP(V) \
  case V: apass_kernel<T, NR, RESID, V><<<grid, kThreads, 0, s>>>(A, lda, m, npad, v, ldv, b, part, spart, sout, counter, done); count_launch(); break;
    TLS_AP(1) TLS_AP(2) TLS_AP(4) TLS_AP(8)
#undef TLS_AP
    default: break;
  }
}

// ---------------------------------------------------------------------------------------
// RQI residual pass in double-FP32 arithmetic (Alg. 2, the u_r quantities r = b - A x,
// A^T r, ||r||^2, b^T r). On this GPU an FP64 FMA issues at 1/64 of the FP32 rate, which makes
// the FP64 pass (2 FMA per entry of A) arithmetic-bound at about 2.6 times its HBM time. Here
// A is read as the FP32 pair A32 + Alo (A to 2^-48 relative, Alo = fl32(A - A32)), x as FP32
// pairs, and every product a x is formed as the exact FP32 product of the leading parts
// (TwoProd by FMA) plus the two cross terms, accumulated in unevaluated FP32 pairs (TwoSum);
// the dropped a_lo x_lo term and the pair rounding keep each partial sum to about 2^-47 of the
// sum of the magnitudes of its terms. r_i is formed as a pair from b_i; ||r||^2 and b^T r are
// accumulated in FP64, and the per-CTA column partials of A^T r are written in FP64 for the
// same reduction as the FP64 pass.
// ---------------------------------------------------------------------------------------
constexpr int kDfThreads = 512;
constexpr int kDfWarps = kDfThreads / 32;
constexpr int kDfMaxStages = 8;

// Two FP32 lanes per instruction (the packed f32x2 forms of sm_100 and later), each lane
// rounded to nearest exactly as the scalar instruction: two independent double-FP32
// accumulations for the issue slots of one. A lane pair is a 64-bit value, low lane first.
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2pack(float lo, float hi) {
  return ((f2_t)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
__device__ __forceinline__ float f2lo(f2_t v) { return __uint_as_float((unsigned)(v & 0xffffffffull)); }
__device__ __forceinline__ float f2hi(f2_t v) { return __uint_as_float((unsigned)(v >> 32)); }
__device__ __forceinline__ f2_t f2add(f2_t a, f2_t b) {
  f2_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2_t f2sub(f2_t a, f2_t b) {
  f2_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2_t f2mul(f2_t a, f2_t b) {
  f2_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2_t f2fma(f2_t a, f2_t b, f2_t c) {
  f2_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ f2_t f2neg(f2_t a) { return a ^ 0x8000000080000000ull; }

// df_fma on both lanes, operation for operation: the product enters negated (pn = -p, exact),
// so that e = fma(ah, xh, pn) and the TwoSum of hi and p = -pn are the scalar form's values
__device__ __forceinline__ void df_fma2(f2_t ah, f2_t al, f2_t xh, f2_t xl, f2_t& hi,
                                        f2_t& lo) {
  const f2_t pn = f2mul(f2neg(ah), xh);
  f2_t e = f2fma(ah, xh, pn);
  e = f2fma(ah, xl, e);
  e = f2fma(al, xh, e);
  const f2_t sm = f2sub(hi, pn);                                   // hi + p
  const f2_t bb = f2sub(sm, hi);
  const f2_t t = f2sub(f2sub(hi, f2sub(sm, bb)), f2add(pn, bb));   // (hi - (s - bb)) + (p - bb)
  hi = sm;
  lo = f2add(lo, f2add(t, e));
}


// Warp sums of NV FP32 pairs by recursive halving (as warp_reduce_scatter): lane l returns the
// warp total of pair l >> (5 - log2 NV).
template <int NV>
__device__ __forceinline__ void df_reduce_scatter(float (&h)[NV], float (&l)[NV], float& oh,
                                                  float& ol) {
  const int lane = threadIdx.x & 31;
  int o = 16;
#pragma unroll
  for (int k = NV; k > 1; k >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < k / 2; ++i) {
      const float kh = up ? h[k / 2 + i] : h[i], kl = up ? l[k / 2 + i] : l[i];
      const float gh = up ? h[i] : h[k / 2 + i], gl = up ? l[i] : l[k / 2 + i];
      const float rh = __shfl_xor_sync(0xffffffffu, gh, o);
      const float rl = __shfl_xor_sync(0xffffffffu, gl, o);
      h[i] = kh;
      l[i] = kl;
      df_add(h[i], l[i], rh, rl);
    }
  }
  oh = h[0];
  ol = l[0];
  for (; o > 0; o >>= 1) {
    const float rh = __shfl_xor_sync(0xffffffffu, oh, o);
    const float rl = __shfl_xor_sync(0xffffffffu, ol, o);
    df_add(oh, ol, rh, rl);
  }
}

// Grid barrier of the cooperative residual launch (bar[0] counter, bar[1] abort word): thread 0
// of each CTA fences and adds 1 (CTA 0 adds 2^31 - (G - 1)), so the top bit flips once every CTA
// has arrived; it polls until the bit differs from the one its add saw. Bounded by a 2 s
// deadline (then code 33 in *err and the abort word raised). Returns false when abandoned.
__device__ __forceinline__ bool df_grid_sync(unsigned int* bar, int* err) {
  __shared__ int fail;
  __syncthreads();
  if (threadIdx.x == 0) {
    fail = 0;
    const unsigned int nb = (blockIdx.x == 0) ? (0x80000000u - (gridDim.x - 1u)) : 1u;
    __threadfence();
    const unsigned int old = atomicAdd(bar, nb);
    const uint64_t t0 = ptx::global_ns();
    unsigned int it = 0;
    while (((old ^ *(volatile unsigned int*)bar) & 0x80000000u) == 0u) {
      if ((++it & 63u) == 0) {
        if (*(volatile unsigned int*)(bar + 1) != 0u) {
          fail = 1;
          break;
        }
        if (ptx::global_ns() - t0 > 2000ull * 1000 * 1000) {
          atomicCAS(err, 0, 33);
          atomicExch(bar + 1, 1u);
          fail = 1;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return fail == 0;
}

// One CTA per SM streams its block of rows of A32 and Alo through a ring of bulk-copy stages;
// thread t owns the float4 column groups (v * 512 + t) of every row, for the row dot products
// and for the axpy alike, so a tile is read from shared memory once and held in registers
// across its CTA barrier. Per tile (RT rows): each thread's pair partials of the RT dot
// products, a warp reduce-scatter, and the sums of tile t - 1 over the warps (warp rt adds row
// rt's 16 warp shares in warp order and forms r_i = b_i - A_i x); one CTA barrier; then the
// refill of tile t's stage and the axpy of tile t - 1.
// With rs set (a cooperative launch), the reduction of resid_reduce_kernel follows in the same
// launch: after a grid barrier every CTA adds the CTAs' partials of its slice of the columns
// (lanes over the CTAs, a butterfly), forms f_j = -(A^T r)_j - sigma^2 x_j and its part of
// ||f||^2, and the last CTA to finish forms sigma^2, g, ||f||^2 and psi into rs.
template <int RT, int VPT>
__global__ void __launch_bounds__(kDfThreads, 1) resid_df_kernel(
    const float* __restrict__ Ahi, const float* __restrict__ Alo, int64_t m, int64_t npad,
    const double* __restrict__ x, const double* __restrict__ b, double* __restrict__ part,
    double* __restrict__ spart, double* __restrict__ sout, unsigned int* counter, int stages,
    int* err, RqiScalars* rs, double* __restrict__ f, double* __restrict__ fpart,
    unsigned int* gbar) {
  constexpr int kSh = (RT >= 16 ? 1 : (RT >= 8 ? 2 : (RT >= 4 ? 3 : (RT >= 2 ? 4 : 5))));
  extern __shared__ __align__(128) unsigned char dsm[];
  float* ring = reinterpret_cast<float*>(dsm);
  __shared__ uint64_t full[kDfMaxStages];
  __shared__ float2 red[2][kDfWarps][RT];      // per-warp pair shares of a tile's rows
  __shared__ float2 rsm[2][RT];                // the tile's r_i as FP32 pairs
  __shared__ double sred[kDfWarps][2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // the thread's x values as FP32 pairs, packed by neighbouring columns (lanes: even, odd)
  f2_t xh2[VPT * 2], xl2[VPT * 2];
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    const int64_t col = ((int64_t)v * kDfThreads + tid) * 4;
    float xh[4], xl[4];
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) f64_split_f32(col < npad ? x[col + cc] : 0.0, xh[cc], xl[cc]);
    xh2[2 * v] = f2pack(xh[0], xh[1]);
    xh2[2 * v + 1] = f2pack(xh[2], xh[3]);
    xl2[2 * v] = f2pack(xl[0], xl[1]);
    xl2[2 * v + 1] = f2pack(xl[2], xl[3]);
  }
  // the thread's column partials of A^T r, packed by neighbouring columns
  f2_t ach2[VPT * 2], acl2[VPT * 2];
#pragma unroll
  for (int e = 0; e < VPT * 2; ++e) ach2[e] = acl2[e] = 0ull;
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = min(m, (int64_t)blockIdx.x * per);
  const int64_t r1 = min(m, r0 + per);
  const int ntiles = (r1 > r0) ? (int)((r1 - r0 + RT - 1) / RT) : 0;
  const int64_t half_floats = (int64_t)RT * npad;        // the A32 rows, then the Alo rows
  const int64_t stage_floats = 2 * half_floats;
  const uint64_t pol = ptx::policy_evict_first();
  auto issue = [&](int t) {
    const int64_t row = r0 + (int64_t)t * RT;
    const int rows = (int)min((int64_t)RT, r1 - row);
    const uint32_t bytes = (uint32_t)(rows * npad * (int64_t)sizeof(float));
    uint64_t* bar = &full[t % stages];
    float* dst = ring + (t % stages) * stage_floats;
    ptx::mbar_expect_tx(bar, 2 * bytes);
    ptx::bulk_g2s_hint(dst, Ahi + row * npad, bytes, bar, pol);
    ptx::bulk_g2s_hint(dst + half_floats, Alo + row * npad, bytes, bar, pol);
  };
  if (tid == 0) {
    for (int s2 = 0; s2 < stages; ++s2) ptx::mbar_init(&full[s2], 1);
    ptx::fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int t = 0; t < stages && t < ntiles; ++t) issue(t);
  double rr = 0.0, br = 0.0;      // lane 0 of warps < RT: its rows' ||r||^2 and b^T r
  ulonglong2 ph[RT][VPT], pl[RT][VPT];  // the previous tile (its axpy follows the barrier)
  double bn = 0.0;   // lane 0 of warp w < RT: b of row w of the tile whose r comes next
  for (int t = 0; t <= ntiles; ++t) {
    const double bc = bn;   // b of row `warp` of tile t - 1, loaded one tile ahead
    if (lane == 0 && warp < RT && t < ntiles) {
      const int64_t nrow = r0 + (int64_t)t * RT + warp;
      bn = (nrow < r1) ? b[nrow] : 0.0;
    }
    ulonglong2 ch[RT][VPT], cl[RT][VPT];   // four entries as two packed column pairs
    if (t < ntiles) {
      const int64_t i0 = r0 + (int64_t)t * RT;
      ptx::mbar_wait(&full[t % stages], (uint32_t)((t / stages) & 1), err, 12);
      const float* th = ring + (t % stages) * stage_floats;
      const float* tl = th + half_floats;
      const int rows = (int)min((int64_t)RT, r1 - i0);
      float dh[RT], dl[RT];
#pragma unroll
      for (int rt = 0; rt < RT; ++rt) {
        // the row's even and odd columns in the two lanes, the lanes added at the end
        f2_t h2 = 0ull, l2 = 0ull;
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          const int64_t col = ((int64_t)v * kDfThreads + tid) * 4;
          const bool ok = rt < rows && col < npad;
          ch[rt][v] = ok ? *reinterpret_cast<const ulonglong2*>(th + rt * npad + col)
                         : make_ulonglong2(0ull, 0ull);
          cl[rt][v] = ok ? *reinterpret_cast<const ulonglong2*>(tl + rt * npad + col)
                         : make_ulonglong2(0ull, 0ull);
          df_fma2(ch[rt][v].x, cl[rt][v].x, xh2[2 * v], xl2[2 * v], h2, l2);
          df_fma2(ch[rt][v].y, cl[rt][v].y, xh2[2 * v + 1], xl2[2 * v + 1], h2, l2);
        }
        dh[rt] = f2lo(h2);
        dl[rt] = f2lo(l2);
        df_add(dh[rt], dl[rt], f2hi(h2), f2hi(l2));
      }
      float oh, ol;
      df_reduce_scatter<RT>(dh, dl, oh, ol);
      if ((lane & ((1 << kSh) - 1)) == 0) red[t & 1][warp][lane >> kSh] = make_float2(oh, ol);
    }
    if (t >= 1 && warp < RT) {
      // row `warp` of tile t - 1: the 16 warp shares in warp order, then r_i = b_i - A_i x
      const int bb = (t - 1) & 1;
      const int64_t row = r0 + (int64_t)(t - 1) * RT + warp;
      float2 q = (lane < kDfWarps) ? red[bb][lane][warp] : make_float2(0.f, 0.f);
#pragma unroll
      for (int o = kDfWarps / 2; o > 0; o >>= 1) {
        const float rh = __shfl_xor_sync(0xffffffffu, q.x, o);
        const float rl = __shfl_xor_sync(0xffffffffu, q.y, o);
        df_add(q.x, q.y, rh, rl);
      }
      if (lane == 0) {
        float2 rv = make_float2(0.f, 0.f);
        if (row < r1) {
          float bh, bl;
          f64_split_f32(bc, bh, bl);
          df_add(bh, bl, -q.x, -q.y);            // r = b - A_i x as a pair,
          two_sum(bh, bl, rv.x, rv.y);           // renormalised for the products that follow
          const double r = (double)rv.x + (double)rv.y;
          rr = fma(r, r, rr);
          br = fma(bc, r, br);
        }
        rsm[bb][warp] = rv;
      }
    }
    __syncthreads();
    // every thread holds tile t in registers: refill its stage
    if (tid == 0 && t < ntiles && t + stages < ntiles) {
      ptx::fence_proxy_async();
      issue(t + stages);
    }
    if (t >= 1) {
      const int bb = (t - 1) & 1;
      const int rows = (int)min((int64_t)RT, r1 - (r0 + (int64_t)(t - 1) * RT));
#pragma unroll
      for (int rt = 0; rt < RT; ++rt) {
        if (rt >= rows) break;
        const float2 rv = rsm[bb][rt];
        const f2_t rh2 = f2pack(rv.x, rv.x), rl2 = f2pack(rv.y, rv.y);
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          df_fma2(ph[rt][v].x, pl[rt][v].x, rh2, rl2, ach2[2 * v], acl2[2 * v]);
          df_fma2(ph[rt][v].y, pl[rt][v].y, rh2, rl2, ach2[2 * v + 1], acl2[2 * v + 1]);
        }
      }
    }
    if (t < ntiles) {
#pragma unroll
      for (int rt = 0; rt < RT; ++rt)
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
          ph[rt][v] = ch[rt][v];
          pl[rt][v] = cl[rt][v];
        }
    }
  }
  // ---- the CTA's column partials of A^T r and its ||r||^2, b^T r (FP64)
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    const int64_t col = ((int64_t)v * kDfThreads + tid) * 4;
    if (col < npad) {
      double2* dst = reinterpret_cast<double2*>(part + (int64_t)blockIdx.x * npad + col);
      const f2_t h0 = ach2[2 * v], l0 = acl2[2 * v], h1 = ach2[2 * v + 1], l1 = acl2[2 * v + 1];
      dst[0] = make_double2((double)f2lo(h0) + (double)f2lo(l0), (double)f2hi(h0) + (double)f2hi(l0));
      dst[1] = make_double2((double)f2lo(h1) + (double)f2lo(l1), (double)f2hi(h1) + (double)f2hi(l1));
    }
  }
  if (lane == 0) {
    sred[warp][0] = rr;
    sred[warp][1] = br;
  }
  __syncthreads();
  if (tid == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int w = 0; w < RT && w < kDfWarps; ++w) {
      a0 += sred[w][0];
      a1 += sred[w][1];
    }
    spart[(int64_t)blockIdx.x * 2 + 0] = a0;
    spart[(int64_t)blockIdx.x * 2 + 1] = a1;
  }
  if (arrive_last(counter)) {
    reduce_partials<2>(spart, (int)gridDim.x, sout);
    if (tid == 0) *counter = 0u;
  }
  if (rs == nullptr) return;
  if (!df_grid_sync(gbar, err)) return;
  const int G = (int)gridDim.x;
  const double xx = rs->xx;
  const double sigma2 = __ldcg(sout) / (1.0 + xx);
  const int64_t per_c = (npad + G - 1) / G;
  const int64_t c0 = min(npad, (int64_t)blockIdx.x * per_c), c1 = min(npad, c0 + per_c);
  double ffl = 0.0;
  for (int64_t j = c0 + warp; j < c1; j += kDfWarps) {
    double t = 0.0;
    for (int p = lane; p < G; p += 32) t += __ldcg(part + (int64_t)p * npad + j);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    const double fj = -t - sigma2 * x[j];
    if (lane == 0) f[j] = fj;
    ffl = fma(fj, fj, ffl);
  }
  if (lane == 0) sred[warp][0] = ffl;
  __syncthreads();
  if (tid == 0) {
    double a0 = 0.0;
    for (int w = 0; w < kDfWarps; ++w) a0 += sred[w][0];
    fpart[blockIdx.x] = a0;
  }
  if (arrive_last(&rs->counter[0])) {
    __shared__ double tfs[1];
    reduce_partials<1>(fpart, G, tfs);
    if (tid == 0) {
      const double tf = tfs[0];
      const double rr = __ldcg(sout), br = __ldcg(sout + 1);
      const double g = -br + sigma2;
      rs->rr = rr;
      rs->br = br;
      rs->sigma2 = sigma2;
      rs->g = g;
      rs->ff = tf;
      rs->psi = sqrt((tf + g * g) / (xx + 1.0));
      rs->counter[0] = 0u;
    }
  }
}

}  // namespace

// =========================================================================================
template <typename T>
ApassPlan plan_apass(int64_t m, int64_t npad, int nr, int num_sms, int variant) {
  (void)nr;
  constexpr int VW = VecOf<T>::W;
  ApassPlan p;
  p.variant = variant;
  int64_t need = (npad + (int64_t)kThreads * VW - 1) / ((int64_t)kThreads * VW);
  p.vpt = 1;
  while (p.vpt < need) p.vpt *= 2;
  // variant 0: registers only (apass_kernel); 1: staged, 256 threads; 2: staged, 512 threads;
  // 3: registers, software pipelined (apass_pipe_kernel)
  p.threads = (variant == 2) ? 512 : 256;
  int64_t need2 = (npad + (int64_t)p.threads * VW - 1) / ((int64_t)p.threads * VW);
  int vpt2 = 1;
  while (vpt2 < need2) vpt2 *= 2;
  const int rt = (vpt2 <= 4) ? (4 / vpt2) : 1;
  const size_t stage = (size_t)rt * (size_t)npad * sizeof(T);
  p.smem = kApStages * stage;
  p.tma = (variant == 1 || variant == 2) && vpt2 <= 4 && p.smem <= 200 * 1024;
  if (variant == 3) {
    // pipelined register kernel: one CTA per SM, at least two tiles per CTA
    p.threads = kThreads;
    const int rw = (p.vpt >= 16) ? 1 : (16 / p.vpt);
    const int64_t by_rows = std::max<int64_t>(1, m / (2 * rw));
    p.grid = (int)std::min<int64_t>((int64_t)num_sms, by_rows);
    return p;
  }
  if (p.tma) {
    p.vpt = vpt2;
    // one CTA per SM (the ring takes most of shared memory), at least a few tiles per CTA
    const int64_t by_rows = std::max<int64_t>(1, m / (2 * rt));
    p.grid = (int)std::min<int64_t>((int64_t)num_sms, by_rows);
  } else {
    const int rt_reg = (p.vpt >= 8) ? 1 : (8 / p.vpt);   // rows per tile of apass_kernel
    const int64_t by_rows = std::max<int64_t>(1, m / (4 * rt_reg));
    p.grid = (int)std::min<int64_t>(2 * (int64_t)num_sms, by_rows);
  }
  return p;
}

template <typename T>
void launch_apass(const ApassPlan& plan, const T* A, int64_t lda, int64_t m, int64_t npad,
                  int nr, bool resid, const T* v, int64_t ldv, const double* b, T* part,
                  double* spart, double* sout, unsigned int* counter, const int* done,
                  int* err, cudaStream_t s) {
  dim3 grid(plan.grid);
  if (plan.tma && lda == npad) {
    if (nr == 1) {
      if (resid) apass_tma_dispatch<T, 1, true>(plan.threads, plan.vpt, grid, plan.smem, A, m, npad, v, ldv, b, part, spart, sout, counter, done, err, s);
      else apass_tma_dispatch<T, 1, false>(plan.threads, plan.vpt, grid, plan.smem, A, m, npad, v, ldv, b, part, spart, sout, counter, done, err, s);
    } else {
      apass_tma_dispatch<T, 2, false>(plan.threads, plan.vpt, grid, plan.smem, A, m, npad, v, ldv, b, part, spart, sout, counter, done, err, s);
    }
    return;
  }
  if (plan.variant == 3) {
    if (nr == 1) {
      if (resid) apass_pipe_dispatch<T, 1, true>(plan.vpt, grid, A, lda, m, npad, v, ldv, b, part, spart, sout, counter, done, s);
      else apass_pipe_dispatch<T, 1, false>(plan.vpt, grid, A, lda, m, npad, v, ldv, b, part, spart, sout, counter, done, s);
    } else {
      apass_pipe_dispatch<T, 2, false>(plan.vpt, grid, A, lda, m, npad, v, ldv, b, part, spart, sout, counter, done, s);
    }
    return;
  }
  if (nr == 1) {
    if (resid) apass_dispatch<T, 1, true>(plan.vpt, grid, A, lda, m, npad, v, ldv, b, part, spart, sout, counter, done, s);
    else apass_dispatch<T, 1, false>(plan.vpt, grid, A, lda, m, npad, v, ldv, b, part, spart, sout, counter, done, s);
  } else {
    apass_dispatch<T, 2, false>(plan.vpt, grid, A, lda, m, npad, v, ldv, b, part, spart, sout, counter, done, s);
  }
}

template <typename T>
void launch_pcg_prep(const double* fin0, double fin0_scale, const double* fin1, int nr,
                     int64_t n, int64_t npad, const double* dinv, T* y, T* w, T* p0, T* p1,
                     PcgScalars* sc, double sigma2, double cg_tol, cudaStream_t s) {
  pcg_prep_kernel<T><<<blocks_for(npad, 256), 256, 0, s>>>(fin0, fin0_scale, fin1, nr, n, npad,
                                                          dinv, y, w, p0, p1, sc, sigma2,
                                                          cg_tol); count_launch();
}

static int gemv_grid(int64_t npad) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(304, (npad + kWarps - 1) / kWarps));
}

template <typename K>
static void allow_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024)
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T>
void launch_gemv_wt(const T* WT, int64_t npad, const T* y, T* s, const T* p, T* unused,
                    double* part, PcgScalars* sc, bool init, bool modeA, int nr,
                    cudaStream_t st) {
  (void)unused;
  const size_t smem = sizeof(T) * nr * npad;
  allow_smem(gemv_wt_kernel<T>, smem);
  gemv_wt_kernel<T><<<gemv_grid(npad), kThreads, smem, st>>>(WT, npad, y, s, p, part, sc,
                                                             init ? 1 : 0, modeA ? 1 : 0, nr); count_launch();
}

template <typename T>
void launch_gemv_w(const T* W, int64_t npad, const T* s, const T* p_prev, T* p_out,
                   const T* dinv, T* q, double* part, PcgScalars* sc, int nr,
                   cudaStream_t st) {
  const size_t smem = sizeof(T) * nr * npad;
  allow_smem(gemv_w_kernel<T>, smem);
  gemv_w_kernel<T><<<gemv_grid(npad), kThreads, smem, st>>>(W, npad, s, p_prev, p_out, dinv, q,
                                                            part, sc, nr); count_launch();
}

template <typename T>
bool launch_pcg_step(const T* part, int P, int nr, int64_t npad, T* q, T* w, T* y,
                     const T* dinv, PcgScalars* sc, const double* tt, const T* WT, const T* W,
                     T* s, const T* p_cur, T* p_next, double* gpart, bool next,
                     unsigned int* bar, int* err, int num_sms, cudaStream_t st) {
  const size_t smem = sizeof(T) * nr * npad;
  allow_smem(pcg_step_kernel<T>, smem);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_step_kernel<T>, kThreads,
                                                    smem) != cudaSuccess || per_sm < 1)
    return false;
  int gb = gemv_grid(npad);
  const int grid = std::max(1, std::min(gb, per_sm * num_sms));
  int nx = next ? 1 : 0;
  void* args[] = {(void*)&part, (void*)&P,  (void*)&nr,    (void*)&npad,  (void*)&q,
                  (void*)&w,    (void*)&y,  (void*)&dinv,  (void*)&sc,    (void*)&tt,
                  (void*)&WT,   (void*)&W,  (void*)&s,     (void*)&p_cur, (void*)&p_next,
                  (void*)&gpart, (void*)&gb, (void*)&nx,   (void*)&bar,   (void*)&err};
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)pcg_step_kernel<T>, grid,
                                                    kThreads, args, smem, st);
  count_launch();
  return e == cudaSuccess;
}

template <typename T>
void launch_pcg_reduce(const T* part, int P, int64_t npad, const T* q, T* w, T* y,
                       const T* dinv, PcgScalars* sc, const double* tt, int nr,
                       cudaStream_t s) {
  dim3 grid((unsigned)((npad + 31) / 32), nr);
  pcg_reduce_kernel<T><<<grid, kThreads, 0, s>>>(part, P, nr, npad, q, w, y, dinv, sc, tt); count_launch();
}

template <typename T>
void launch_pcg_update_R(const T* q, T* w, T* y, const T* dinv, PcgScalars* sc, int nr,
                         int64_t npad, cudaStream_t s) {
  dim3 grid((unsigned)blocks_for(npad, 256), nr);
  pcg_update_R_kernel<T><<<grid, 256, 0, s>>>(q, w, y, dinv, sc, nr, npad); count_launch();
}

void launch_resid_reduce(const double* part, int P, int64_t npad, const double* x, double* f,
                         const double* sout, RqiScalars* rs, double* fpart, cudaStream_t s) {
  resid_reduce_kernel<<<(unsigned)((npad + 31) / 32), kThreads, 0, s>>>(part, P, npad, x, f,
                                                                         sout, rs, fpart); count_launch();
}

template <typename T>
void launch_rqi_update(double* x, const T* w, const T* u, const double* f, RqiScalars* rs,
                       int64_t n, cudaStream_t s, double* part) {
  if (part == nullptr) {
    rqi_update_kernel<T><<<1, 1024, 0, s>>>(x, w, u, f, rs, n); count_launch();
    return;
  }
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(32, (n + 255) / 256));
  rqi_dots_kernel<T><<<grid, 256, 0, s>>>(x, w, f, rs, n, part); count_launch();
  xupd_kernel<T, 2><<<grid, 256, 0, s>>>(x, w, u, rs, n, part); count_launch();
}

template <typename T>
void launch_inverse_step(double* x, const T* u, RqiScalars* rs, int64_t n, cudaStream_t s,
                         double* part) {
  if (part == nullptr) {
    inverse_step_kernel<T><<<1, 1024, 0, s>>>(x, u, rs, n); count_launch();
    return;
  }
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(32, (n + 255) / 256));
  xupd_kernel<T, 1><<<grid, 256, 0, s>>>(x, u, u, rs, n, part); count_launch();
}

template <typename T>
void launch_copy_to_x(double* x, const T* w, RqiScalars* rs, int64_t n, cudaStream_t s,
                      double* part) {
  if (part == nullptr) {
    copy_to_x_kernel<T><<<1, 1024, 0, s>>>(x, w, rs, n); count_launch();
    return;
  }
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(32, (n + 255) / 256));
  xupd_kernel<T, 0><<<grid, 256, 0, s>>>(x, w, w, rs, n, part); count_launch();
}

void launch_xx(const double* x, RqiScalars* rs, int64_t n, cudaStream_t s, double* part) {
  if (part == nullptr) {
    xx_kernel<<<1, 1024, 0, s>>>(x, rs, n); count_launch();
    return;
  }
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(32, (n + 255) / 256));
  xx_multi_kernel<<<grid, 256, 0, s>>>(x, rs, n, part); count_launch();
}

template <typename T>
void launch_vec_convert(const double* in, T* out, int64_t n, int64_t npad, cudaStream_t s) {
  vec_convert_kernel<T><<<blocks_for(npad, 256), 256, 0, s>>>(in, out, n, npad); count_launch();
}

#define TLS_INST(T)                                                                            \
  template ApassPlan plan_apass<T>(int64_t, int64_t, int, int, int);                           \
  template void launch_apass<T>(const ApassPlan&, const T*, int64_t, int64_t, int64_t, int,    \
                                bool, const T*, int64_t, const double*, T*, double*, double*,  \
                                unsigned int*, const int*, int*, cudaStream_t);                \
  template void launch_pcg_prep<T>(const double*, double, const double*, int, int64_t,         \
                                   int64_t, const double*, T*, T*, T*, T*, PcgScalars*,        \
                                   double, double, cudaStream_t);                              \
  template void launch_gemv_wt<T>(const T*, int64_t, const T*, T*, const T*, T*, double*,      \
                                  PcgScalars*, bool, bool, int, cudaStream_t);                 \
  template void launch_gemv_w<T>(const T*, int64_t, const T*, const T*, T*, const T*, T*,      \
                                 double*, PcgScalars*, int, cudaStream_t);                     \
  template void launch_pcg_reduce<T>(const T*, int, int64_t, const T*, T*, T*, const T*,       \
                                     PcgScalars*, const double*, int, cudaStream_t);           \
  template bool launch_pcg_step<T>(const T*, int, int, int64_t, T*, T*, T*, const T*,          \
                                   PcgScalars*, const double*, const T*, const T*, T*,         \
                                   const T*, T*, double*, bool, unsigned int*, int*, int,      \
                                   cudaStream_t);                                              \
  template void launch_pcg_update_R<T>(const T*, T*, T*, const T*, PcgScalars*, int,           \
                                       int64_t, cudaStream_t);                                 \
  template void launch_rqi_update<T>(double*, const T*, const T*, const double*, RqiScalars*,  \
                                     int64_t, cudaStream_t, double*);                          \
  template void launch_inverse_step<T>(double*, const T*, RqiScalars*, int64_t, cudaStream_t,  \
                                       double*);                                               \
  template void launch_copy_to_x<T>(double*, const T*, RqiScalars*, int64_t, cudaStream_t,     \
                                    double*);                                                  \
  template void launch_vec_convert<T>(const double*, T*, int64_t, int64_t, cudaStream_t);

TLS_INST(float)
TLS_INST(double)
#undef TLS_INST

// The RQI residual pass in double-FP32 arithmetic (resid_df_kernel): A as the pair A32 + Alo
// (m x npad each, row-major, rows back to back), x and b FP64; per-CTA FP64 partials of A^T r
// in part (grid x npad) and (||r||^2, b^T r) in spart, their totals in sout[0..1] by the last
// CTA. Returns the grid (the number of partials), or 0 when npad is outside the kernel's range
// (npad <= 8192, a multiple of 64) and nothing was launched.
int launch_resid_df(const float* Ahi, const float* Alo, int64_t m, int64_t npad,
                    const double* x, const double* b, double* part, double* spart, double* sout,
                    unsigned int* counter, int* err, int num_sms, cudaStream_t s,
                    RqiScalars* rs, double* f, double* fpart, unsigned int* gbar, bool* fused) {
  if (fused) *fused = false;
  if (npad <= 0 || npad > 8192 || npad % 64 != 0 || m <= 0) return 0;
  // float4 column groups per thread and rows per tile (RT * VPT <= 4: two tiles of both planes
  // in registers)
  const int vpt = (int)((npad + 4 * kDfThreads - 1) / (4 * kDfThreads));
  const int rt = (vpt == 1) ? 4 : (vpt == 2 ? 2 : 1);
  const size_t stage = (size_t)2 * rt * npad * sizeof(float);
  const int stages = (int)std::min<size_t>(kDfMaxStages, (size_t)(200 * 1024) / stage);
  if (stages < 2) return 0;
  const int grid = (int)std::min<int64_t>((int64_t)num_sms, std::max<int64_t>(1, m / (2 * rt)));
  const size_t smem = (size_t)stages * stage;
#define TLS_DF(R, V)                                                                           \
  {                                                                                            \
    static const bool attr = [] {                                                              \
      cudaFuncSetAttribute(resid_df_kernel<R, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                           200 * 1024);                                                        \
      return true;                                                                             \
    }();                                                                                       \
    (void)attr;                                                                                \
    bool done = false;                                                                         \
    if (rs != nullptr && fused != nullptr && gbar != nullptr) {                                \
      /* the reduction in the same, cooperative launch */                                     \
      RqiScalars* rs_ = rs;                                                                    \
      double* f_ = f;                                                                          \
      double* fp_ = fpart;                                                                     \
      unsigned int* gb_ = gbar;                                                                \
      int st_ = stages;                                                                        \
      void* args[] = {(void*)&Ahi, (void*)&Alo, (void*)&m, (void*)&npad, (void*)&x, (void*)&b, \
                      (void*)&part, (void*)&spart, (void*)&sout, (void*)&counter, (void*)&st_, \
                      (void*)&err, (void*)&rs_, (void*)&f_, (void*)&fp_, (void*)&gb_};          \
      done = cudaLaunchCooperativeKernel((const void*)resid_df_kernel<R, V>, grid, kDfThreads,  \
                                         args, smem, s) == cudaSuccess;                        \
      if (!done) (void)cudaGetLastError();                                                     \
      *fused = done;                                                                           \
    }                                                                                          \
    if (!done)                                                                                 \
      resid_df_kernel<R, V><<<grid, kDfThreads, smem, s>>>(Ahi, Alo, m, npad, x, b, part,      \
                                                           spart, sout, counter, stages, err,  \
                                                           nullptr, nullptr, nullptr, nullptr); \
    count_launch();                                                                            \
  }
  if (vpt == 1) TLS_DF(4, 1) else if (vpt == 2) TLS_DF(2, 2) else if (vpt == 3) TLS_DF(1, 3)
  else TLS_DF(1, 4)
#undef TLS_DF
  return grid;
}

}  // namespace tls
