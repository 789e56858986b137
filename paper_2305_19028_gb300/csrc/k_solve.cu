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
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w * K + k];
    v[k] = t;
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
  __shared__ double sh[kWarps * K];
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
  double s_cc[NR], s_bc[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) { s_cc[r] = 0.0; s_bc[r] = 0.0; }
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
      double brow = 0.0;
      if (RESID && valid) brow = b[row];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        T dot = T(0);
#pragma unroll
        for (int w = 0; w < kWarps; ++w) dot += red[buf][w][r * RT + rt];
        T c = T(0);
        if (valid) c = RESID ? (T)(brow - (double)dot) : dot;
        if (tid == 0) {
          s_cc[r] = fma((double)c, (double)c, s_cc[r]);
          s_bc[r] = fma(brow, (double)c, s_bc[r]);
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
      spart[((int64_t)blockIdx.x * NR + r) * 2 + 0] = s_cc[r];
      spart[((int64_t)blockIdx.x * NR + r) * 2 + 1] = s_bc[r];
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

template <typename T, int NR, bool RESID, int VPT>
__global__ void __launch_bounds__(kThreads, 1) apass_tma_kernel(
    const T* __restrict__ A, int64_t m, int64_t npad, const T* __restrict__ v, int64_t ldv,
    const double* __restrict__ b, T* __restrict__ part, double* __restrict__ spart,
    double* __restrict__ sout, unsigned int* counter, const int* __restrict__ done, int* err) {
  using V = typename VecOf<T>::type;
  constexpr int VW = VecOf<T>::W;
  constexpr int RT = (VPT >= 8) ? 1 : (8 / VPT);   // rows per tile
  constexpr int E = VPT * VW;
  extern __shared__ __align__(128) unsigned char dsm[];
  T* ring = reinterpret_cast<T*>(dsm);
  __shared__ uint64_t full[kApStages];
  __shared__ T red[2][kWarps][NR * RT];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (done != nullptr) {
    bool all = true;
#pragma unroll
    for (int r = 0; r < NR; ++r) all = all && (done[r] != 0);
    if (all) return;
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
  const int ntiles = (r1 > r0) ? (int)((r1 - r0 + RT - 1) / RT) : 0;
  const int64_t stage_elems = (int64_t)RT * npad;
  auto issue = [&](int t) {
    const int64_t row = r0 + (int64_t)t * RT;
    const int rows = (int)min((int64_t)RT, r1 - row);
    const uint32_t bytes = (uint32_t)(rows * npad * (int64_t)sizeof(T));
    uint64_t* bar = &full[t % kApStages];
    ptx::mbar_expect_tx(bar, bytes);
    ptx::bulk_g2s(ring + (t % kApStages) * stage_elems, A + row * npad, bytes, bar);
  };
  if (tid == 0) {
    for (int s2 = 0; s2 < kApStages; ++s2) ptx::mbar_init(&full[s2], 1);
    ptx::fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int t = 0; t < kApStages && t < ntiles; ++t) issue(t);
  double s_cc[NR], s_bc[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) { s_cc[r] = 0.0; s_bc[r] = 0.0; }
  int buf = 0;
  for (int t = 0; t < ntiles; ++t) {
    const int64_t i0 = r0 + (int64_t)t * RT;
    ptx::mbar_wait(&full[t % kApStages], (uint32_t)((t / kApStages) & 1), err, 11);
    const T* tile = ring + (t % kApStages) * stage_elems;
    T pd[NR][RT];
#pragma unroll
    for (int rt = 0; rt < RT; ++rt) {
      const bool rv = (i0 + rt) < r1;
      V a[VPT];
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        const int64_t col = ((int64_t)k * kThreads + tid) * VW;
        a[k] = (rv && col < npad) ? *reinterpret_cast<const V*>(tile + rt * npad + col)
                                  : zero_vec(T(0));
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        T tt = T(0);
#pragma unroll
        for (int k = 0; k < VPT; ++k)
#pragma unroll
          for (int c = 0; c < VW; ++c) tt = fma(get(a[k], c), vv[r][k * VW + c], tt);
        pd[r][rt] = warp_sum(tt);
      }
    }
    if (lane == 0)
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int rt = 0; rt < RT; ++rt) red[buf][warp][r * RT + rt] = pd[r][rt];
    __syncthreads();
    // every thread is done with tile t-1: refill its stage with tile t-1+kApStages
    if (tid == 0 && t >= 1 && t - 1 + kApStages < ntiles) {
      ptx::fence_proxy_async();
      issue(t - 1 + kApStages);
    }
#pragma unroll
    for (int rt = 0; rt < RT; ++rt) {
      const int64_t row = i0 + rt;
      const bool valid = row < r1;
      double brow = 0.0;
      if (RESID && valid) brow = b[row];
      V a[VPT];
#pragma unroll
      for (int k = 0; k < VPT; ++k) {
        const int64_t col = ((int64_t)k * kThreads + tid) * VW;
        a[k] = (valid && col < npad) ? *reinterpret_cast<const V*>(tile + rt * npad + col)
                                     : zero_vec(T(0));
      }
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        T dot = T(0);
#pragma unroll
        for (int w = 0; w < kWarps; ++w) dot += red[buf][w][r * RT + rt];
        T c = T(0);
        if (valid) c = RESID ? (T)(brow - (double)dot) : dot;
        if (tid == 0) {
          s_cc[r] = fma((double)c, (double)c, s_cc[r]);
          s_bc[r] = fma(brow, (double)c, s_bc[r]);
        }
#pragma unroll
        for (int k = 0; k < VPT; ++k)
#pragma unroll
          for (int cc = 0; cc < VW; ++cc)
            acc[r][k * VW + cc] = fma(c, get(a[k], cc), acc[r][k * VW + cc]);
      }
    }
    buf ^= 1;
  }
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
      spart[((int64_t)blockIdx.x * NR + r) * 2 + 0] = s_cc[r];
      spart[((int64_t)blockIdx.x * NR + r) * 2 + 1] = s_bc[r];
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
    T* __restrict__ w, T* __restrict__ y, const double* __restrict__ dinv, PcgScalars* sc,
    const double* __restrict__ tt) {
  __shared__ T sh[kWarps][33];
  const int r = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (sc->done[r]) return;
  const int64_t j = (int64_t)blockIdx.x * 32 + lane;
  T t = T(0);
  if (j < npad)
    for (int p = warp; p < P; p += kWarps) t += part[((int64_t)p * nr + r) * npad + j];
  sh[warp][lane] = t;
  __syncthreads();
  if (warp != 0) return;
  T at = T(0);
#pragma unroll
  for (int k = 0; k < kWarps; ++k) at += sh[k][lane];
  const double sigma2 = sc->sigma2;
  const double delta = tt[r * 2] - sigma2 * sc->qq[r];
  if (blockIdx.x == 0 && lane == 0) sc->delta[r] = delta;
  if (!(delta > 0.0)) return;                     // loss of positive definiteness (Sec. 3)
  const double alpha = sc->eta[r] / delta;
  if (blockIdx.x == 0 && lane == 0) sc->alpha[r] = alpha;
  if (j < npad) {
    const T qj = q[r * npad + j];
    w[r * npad + j] = fma((T)alpha, qj, w[r * npad + j]);
    y[r * npad + j] = (at - (T)sigma2 * qj) * (T)dinv[j];
  }
}

// Alg. 3 as printed: delta = ||p||^2 - sigma^2 ||q||^2, w += alpha q, y = D^{-1} q.
template <typename T>
__global__ void pcg_update_R_kernel(const T* __restrict__ q, T* __restrict__ w, T* __restrict__ y,
                                    const double* __restrict__ dinv, PcgScalars* sc, int nr,
                                    int64_t npad) {
  const int r = blockIdx.y;
  if (sc->done[r]) return;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double delta = sc->pp[r] - sc->sigma2 * sc->qq[r];
  if (blockIdx.x == 0 && threadIdx.x == 0) sc->delta[r] = delta;
  if (!(delta > 0.0)) return;
  const double alpha = sc->eta[r] / delta;
  if (blockIdx.x == 0 && threadIdx.x == 0) sc->alpha[r] = alpha;
  if (j < npad) {
    const T qj = q[r * npad + j];
    w[r * npad + j] = fma((T)alpha, qj, w[r * npad + j]);
    y[r * npad + j] = qj * (T)dinv[j];
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
  using V = typename VecOf<T>::type;
  constexpr int VW = VecOf<T>::W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ys = reinterpret_cast<T*>(smem_raw);
  __shared__ double red[kWarps * 2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  bool active[2];
  double alpha[2];
  for (int r = 0; r < 2; ++r) {
    active[r] = r < nr && (init || (!sc->done[r] && sc->delta[r] > 0.0));
    alpha[r] = init ? 0.0 : sc->alpha[r];
  }
  const double sigma2 = sc->sigma2;
  for (int64_t e = tid; e < nr * npad; e += kThreads) ys[e] = y[e];
  __syncthreads();
  double ss[2] = {0.0, 0.0};
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp, GW = (int64_t)gridDim.x * kWarps;
  for (int64_t j = gw; j < npad; j += GW) {
    const T* row = WT + j * npad;
    const int64_t lim = ((j + VW) / VW) * VW;    // entries 0..j, rounded up (zeros beyond j)
    T a0 = T(0), a1 = T(0);
    for (int64_t c = (int64_t)lane * VW; c < lim; c += 32 * VW) {
      V wv = *reinterpret_cast<const V*>(row + c);
#pragma unroll
      for (int k = 0; k < VW; ++k) {
        a0 = fma(get(wv, k), ys[c + k], a0);
        if (nr > 1) a1 = fma(get(wv, k), ys[npad + c + k], a1);
      }
    }
    a0 = warp_sum(a0);
    if (nr > 1) a1 = warp_sum(a1);
    if (lane == 0) {
      T vr[2] = {a0, a1};
      for (int r = 0; r < nr; ++r) {
        T* sp = s + r * npad + j;
        T sv = *sp;
        if (init) sv = vr[r];
        else if (active[r]) {
          if (modeA) sv = sv - (T)alpha[r] * vr[r];
          else sv = sv - (T)alpha[r] * (p[r * npad + j] - (T)sigma2 * vr[r]);
        }
        if (init || active[r]) *sp = sv;
        ss[r] += (double)sv * (double)sv;
      }
    }
  }
  // CTA partials of ||s||^2
  ss[0] = warp_sum(ss[0]);
  ss[1] = warp_sum(ss[1]);
  if (lane == 0) { red[warp * 2] = ss[0]; red[warp * 2 + 1] = ss[1]; }
  __syncthreads();
  if (tid < 2) {
    double t = 0.0;
    for (int w2 = 0; w2 < kWarps; ++w2) t += red[w2 * 2 + tid];
    part[(int64_t)blockIdx.x * 2 + tid] = t;
  }
  if (arrive_last(&sc->counter[0])) {
    __shared__ double eta_sum[2];
    reduce_partials<2>(part, (int)gridDim.x, eta_sum);
    if (tid < nr) {
      const int r = tid;
      const double eta_new = eta_sum[r];
      if (init) {
        sc->eta[r] = eta_new;
        sc->eta0[r] = eta_new;
        sc->beta[r] = 0.0;
        sc->done[r] = (eta_new == 0.0) ? 1 : 0;
        sc->iters[r] = 0;
      } else if (!sc->done[r]) {
        if (!(sc->delta[r] > 0.0)) {
          sc->done[r] = 1;
          sc->not_spd[r] = (sc->delta[r] < 0.0) ? 1 : 0;
        } else {
          sc->beta[r] = eta_new / sc->eta[r];
          sc->eta[r] = eta_new;
          sc->iters[r] += 1;
          if (eta_new == 0.0 || (sc->cg_tol2 > 0.0 && eta_new <= sc->cg_tol2 * sc->eta0[r]))
            sc->done[r] = 1;
        }
      }
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
    T* __restrict__ p_out, const double* __restrict__ dinv, T* __restrict__ q,
    double* __restrict__ part, PcgScalars* sc, int nr) {
  using V = typename VecOf<T>::type;
  constexpr int VW = VecOf<T>::W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ps = reinterpret_cast<T*>(smem_raw);
  __shared__ double red[kWarps * 4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T beta0 = (T)sc->beta[0], beta1 = (T)(nr > 1 ? sc->beta[1] : 0.0);
  for (int64_t e = tid; e < nr * npad; e += kThreads) {
    const T bt = (e < npad) ? beta0 : beta1;
    ps[e] = s[e] + bt * p_prev[e];
  }
  __syncthreads();
  {
    const int64_t chunk = (nr * npad + gridDim.x - 1) / gridDim.x;
    const int64_t e0 = (int64_t)blockIdx.x * chunk, e1 = min((int64_t)nr * npad, e0 + chunk);
    for (int64_t e = e0 + tid; e < e1; e += kThreads) p_out[e] = ps[e];
  }
  double acc4[4] = {0.0, 0.0, 0.0, 0.0};   // qq0, qq1, pp0, pp1
  const int64_t gw = (int64_t)blockIdx.x * kWarps + warp, GW = (int64_t)gridDim.x * kWarps;
  for (int64_t i = gw; i < npad; i += GW) {
    const T* row = W + i * npad;
    T a0 = T(0), a1 = T(0);
    for (int64_t c = (i / VW) * VW + (int64_t)lane * VW; c < npad; c += 32 * VW) {
      V wv = *reinterpret_cast<const V*>(row + c);
#pragma unroll
      for (int k = 0; k < VW; ++k) {
        a0 = fma(get(wv, k), ps[c + k], a0);
        if (nr > 1) a1 = fma(get(wv, k), ps[npad + c + k], a1);
      }
    }
    a0 = warp_sum(a0);
    if (nr > 1) a1 = warp_sum(a1);
    if (lane == 0) {
      const T di = (T)dinv[i];
      const T q0 = a0 * di;
      q[i] = q0;
      acc4[0] += (double)q0 * (double)q0;
      acc4[2] += (double)ps[i] * (double)ps[i];
      if (nr > 1) {
        const T q1 = a1 * di;
        q[npad + i] = q1;
        acc4[1] += (double)q1 * (double)q1;
        acc4[3] += (double)ps[npad + i] * (double)ps[npad + i];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) acc4[k] = warp_sum(acc4[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) red[warp * 4 + k] = acc4[k];
  __syncthreads();
  if (tid < 4) {
    double t = 0.0;
    for (int w2 = 0; w2 < kWarps; ++w2) t += red[w2 * 4 + tid];
    part[(int64_t)blockIdx.x * 4 + tid] = t;
  }
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
  if (j < npad)
    for (int p = warp; p < P; p += kWarps) t += part[(int64_t)p * npad + j];
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

template <typename T, int NR, bool RESID>
void apass_tma_dispatch(int vpt, dim3 grid, size_t smem, const T* A, int64_t m, int64_t npad,
                        const T* v, int64_t ldv, const double* b, T* part, double* spart,
                        double* sout, unsigned int* counter, const int* done, int* err,
                        cudaStream_t s) {
  switch (vpt) {
#define TLS_AT(V)                                                                               \
  case V: {                                                                                     \
    static bool attr = false;                                                                   \
    if (!attr) {                                                                                \
      cudaFuncSetAttribute(apass_tma_kernel<T, NR, RESID, V>,                                  \
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);            \
      attr = true;                                                                              \
    }                                                                                           \
    apass_tma_kernel<T, NR, RESID, V><<<grid, kThreads, smem, s>>>(A, m, npad, v, ldv, b, part, \
                                                                   spart, sout, counter, done,  \
                                                                   err);                        \
    count_launch();                                                                             \
    break;                                                                                      \
  }
    TLS_AT(1) TLS_AT(2) TLS_AT(4) TLS_AT(8)
#undef TLS_AT
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

}  // namespace

// =========================================================================================
template <typename T>
ApassPlan plan_apass(int64_t m, int64_t npad, int nr, int num_sms) {
  (void)nr;
  constexpr int VW = VecOf<T>::W;
  ApassPlan p;
  int64_t need = (npad + (int64_t)kThreads * VW - 1) / ((int64_t)kThreads * VW);
  p.vpt = 1;
  while (p.vpt < need) p.vpt *= 2;
  const int rt = (p.vpt >= 8) ? 1 : (8 / p.vpt);
  const size_t stage = (size_t)rt * (size_t)npad * sizeof(T);
  p.smem = kApStages * stage;
  p.tma = p.smem <= 200 * 1024;
  if (p.tma) {
    // one CTA per SM (the ring takes most of shared memory), at least a few tiles per CTA
    const int64_t by_rows = std::max<int64_t>(1, m / (2 * rt));
    p.grid = (int)std::min<int64_t>((int64_t)num_sms, by_rows);
  } else {
    const int64_t by_rows = std::max<int64_t>(1, m / (4 * rt));
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
      if (resid) apass_tma_dispatch<T, 1, true>(plan.vpt, grid, plan.smem, A, m, npad, v, ldv, b, part, spart, sout, counter, done, err, s);
      else apass_tma_dispatch<T, 1, false>(plan.vpt, grid, plan.smem, A, m, npad, v, ldv, b, part, spart, sout, counter, done, err, s);
    } else {
      apass_tma_dispatch<T, 2, false>(plan.vpt, grid, plan.smem, A, m, npad, v, ldv, b, part, spart, sout, counter, done, err, s);
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
                   const double* dinv, T* q, double* part, PcgScalars* sc, int nr,
                   cudaStream_t st) {
  const size_t smem = sizeof(T) * nr * npad;
  allow_smem(gemv_w_kernel<T>, smem);
  gemv_w_kernel<T><<<gemv_grid(npad), kThreads, smem, st>>>(W, npad, s, p_prev, p_out, dinv, q,
                                                            part, sc, nr); count_launch();
}

template <typename T>
void launch_pcg_reduce(const T* part, int P, int64_t npad, const T* q, T* w, T* y,
                       const double* dinv, PcgScalars* sc, const double* tt, int nr,
                       cudaStream_t s) {
  dim3 grid((unsigned)((npad + 31) / 32), nr);
  pcg_reduce_kernel<T><<<grid, kThreads, 0, s>>>(part, P, nr, npad, q, w, y, dinv, sc, tt); count_launch();
}

template <typename T>
void launch_pcg_update_R(const T* q, T* w, T* y, const double* dinv, PcgScalars* sc, int nr,
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
                       int64_t n, cudaStream_t s) {
  rqi_update_kernel<T><<<1, 1024, 0, s>>>(x, w, u, f, rs, n); count_launch();
}

template <typename T>
void launch_inverse_step(double* x, const T* u, RqiScalars* rs, int64_t n, cudaStream_t s) {
  inverse_step_kernel<T><<<1, 1024, 0, s>>>(x, u, rs, n); count_launch();
}

template <typename T>
void launch_copy_to_x(double* x, const T* w, RqiScalars* rs, int64_t n, cudaStream_t s) {
  copy_to_x_kernel<T><<<1, 1024, 0, s>>>(x, w, rs, n); count_launch();
}

void launch_xx(const double* x, RqiScalars* rs, int64_t n, cudaStream_t s) {
  xx_kernel<<<1, 1024, 0, s>>>(x, rs, n); count_launch();
}

template <typename T>
void launch_vec_convert(const double* in, T* out, int64_t n, int64_t npad, cudaStream_t s) {
  vec_convert_kernel<T><<<blocks_for(npad, 256), 256, 0, s>>>(in, out, n, npad); count_launch();
}

#define TLS_INST(T)                                                                            \
  template ApassPlan plan_apass<T>(int64_t, int64_t, int, int);                                \
  template void launch_apass<T>(const ApassPlan&, const T*, int64_t, int64_t, int64_t, int,    \
                                bool, const T*, int64_t, const double*, T*, double*, double*,  \
                                unsigned int*, const int*, int*, cudaStream_t);                \
  template void launch_pcg_prep<T>(const double*, double, const double*, int, int64_t,         \
                                   int64_t, const double*, T*, T*, T*, T*, PcgScalars*,        \
                                   double, double, cudaStream_t);                              \
  template void launch_gemv_wt<T>(const T*, int64_t, const T*, T*, const T*, T*, double*,      \
                                  PcgScalars*, bool, bool, int, cudaStream_t);                 \
  template void launch_gemv_w<T>(const T*, int64_t, const T*, const T*, T*, const double*, T*, \
                                 double*, PcgScalars*, int, cudaStream_t);                     \
  template void launch_pcg_reduce<T>(const T*, int, int64_t, const T*, T*, T*, const double*,  \
                                     PcgScalars*, const double*, int, cudaStream_t);           \
  template void launch_pcg_update_R<T>(const T*, T*, T*, const double*, PcgScalars*, int,      \
                                       int64_t, cudaStream_t);                                 \
  template void launch_rqi_update<T>(double*, const T*, const T*, const double*, RqiScalars*,  \
                                     int64_t, cudaStream_t);                                   \
  template void launch_inverse_step<T>(double*, const T*, RqiScalars*, int64_t, cudaStream_t); \
  template void launch_copy_to_x<T>(double*, const T*, RqiScalars*, int64_t, cudaStream_t);    \
  template void launch_vec_convert<T>(const double*, T*, int64_t, int64_t, cudaStream_t);

TLS_INST(float)
TLS_INST(double)
#undef TLS_INST

}  // namespace tls
