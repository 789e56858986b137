// Kernels of the packed batched path: many dense TLS problems of uneven sizes, every phase of
// RQI-PCGTLS (Alg. 2; PCGTLS of Alg. 3 with the precisions of Alg. 4) launched once for the
// whole batch.
//
//  * pass kernels: one CTA per row tile of any problem (one tile table for the batch). A group
//    of `lr` lanes owns a row; each lane holds `ch` chunks of 4 columns and keeps the vector
//    entries of its columns (q or x) in registers. Per row: the dot products with the vectors
//    (group shuffle), then the row's contribution to A^T t (or A^T r) into per-lane column
//    accumulators; at the end the CTA writes its partial column sums (deterministic two-stage
//    reduction, no atomics).
//  * per-problem kernels: one CTA (512 threads) per problem for the n-sized work -- summing the
//    tile partials, the Rayleigh quotient and psi (Eq. (2), Eq. (4)), the PCGTLS scalars, and
//    the products with the explicit inverse factor W = R_H^{-1} (row-per-warp GEMVs from L2).
//  * factor kernels: Gram tiles of every problem in one grid (FP32 FMA on the u_f-rounded,
//    column-scaled entries, i.e. exactly the products a tensor core forms), then one CTA per
//    problem for the blocked Cholesky (64-blocks) and for the blocked triangular inverse.
#include "../../include/tls.h"
#include "tls_batch_internal.h"
#include "tls_device.cuh"
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "chol64.cuh"

namespace tls {
namespace bat {

namespace {

constexpr int kPW = kPT / 32;   // warps of a pass CTA
constexpr int kCW = kCT / 32;   // warps of a per-problem CTA
constexpr int kLd = kNB + 4;    // shared-memory row stride of 64-wide tiles (16-byte rows)

template <typename T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of K values over the CTA; every thread receives the totals. sh: 32 * K entries.
template <typename T, int K>
__device__ __forceinline__ void bsum(T (&v)[K], T* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = wsum(v[k]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[warp * K + k] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = wsum(lane < nw ? sh[lane * K + k] : T(0));
}

__device__ __forceinline__ void load4(const float* p, float (&o)[4]) {
  const float4 t = __ldcs(reinterpret_cast<const float4*>(p));
  o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void load4(const double* p, double (&o)[4]) {
  const double2 t0 = __ldcs(reinterpret_cast<const double2*>(p));
  const double2 t1 = __ldcs(reinterpret_cast<const double2*>(p) + 1);
  o[0] = t0.x; o[1] = t0.y; o[2] = t1.x; o[3] = t1.y;
}
// 4 consecutive entries of a row that stays in cache (W, W^T)
__device__ __forceinline__ void ldrow4(const float* p, float (&o)[4]) {
  const float4 t = __ldg(reinterpret_cast<const float4*>(p));
  o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void ldrow4(const double* p, double (&o)[4]) {
  const double2 t0 = __ldg(reinterpret_cast<const double2*>(p));
  const double2 t1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
  o[0] = t0.x; o[1] = t0.y; o[2] = t1.x; o[3] = t1.y;
}

// 4 consecutive entries from shared memory (16-byte aligned)
__device__ __forceinline__ void lds4(const float* p, float (&o)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void lds4(const double* p, double (&o)[4]) {
  const double2 t0 = *reinterpret_cast<const double2*>(p);
  const double2 t1 = *reinterpret_cast<const double2*>(p + 2);
  o[0] = t0.x; o[1] = t0.y; o[2] = t1.x; o[3] = t1.y;
}

// rounding to the factor precision u_f (Table 2): FP16 / BF16 round to nearest even
__device__ __forceinline__ float round_uf(float v, int prec) {
  if (prec == (int)Prec::FP16) return __half2float(__float2half_rn(v));
  if (prec == (int)Prec::BF16) return __bfloat162float(__float2bfloat16_rn(v));
  return v;
}
__device__ __forceinline__ double round_uf(double v, int prec) {
  if (prec == (int)Prec::FP16) return (double)__half2float(__double2half(v));
  if (prec == (int)Prec::BF16) return (double)__bfloat162float(__double2bfloat16(v));
  if (prec == (int)Prec::FP32) return (double)__double2float_rn(v);
  return v;
}

template <typename T> __device__ __forceinline__ const T* dinv_of(const BArrays& a);
template <> __device__ __forceinline__ const float* dinv_of<float>(const BArrays& a) { return a.dinv32; }
template <> __device__ __forceinline__ const double* dinv_of<double>(const BArrays& a) { return a.dinv; }

// =========================================================================================
// Pass over the rows of one tile
// =========================================================================================
template <typename TA, int NR, int MODE, int LR, int CH>
__device__ __forceinline__ void pass_body(const BArrays& a, const BProb& P, const BTile& t,
                                          int tile, unsigned char* smem) {
  constexpr int G = 32 / LR;      // row groups per warp
  constexpr int NG = kPW * G;     // row groups per CTA
  constexpr int NC = 4 * LR * CH; // columns covered by a group
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gl = lane & (LR - 1);
  const int lda = (int)P.lda;
  const int npb = (int)P.npb;
  const TA* A;
  if constexpr (sizeof(TA) == 4) A = reinterpret_cast<const TA*>(a.A32);
  else A = reinterpret_cast<const TA*>(a.A64);
  const TA* Ab = A + P.offA + (int64_t)t.row0 * lda;
  const TA* vec = nullptr;
  if constexpr (MODE == kPcg) vec = static_cast<const TA*>(a.vq) + 2 * P.offV;
  if constexpr (MODE == kResid) vec = reinterpret_cast<const TA*>(a.x) + P.offV;

  TA vq[NR][CH][4];
  TA acc[NR][CH][4];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int col = 4 * (gl + LR * c);
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        acc[r][c][e] = TA(0);
        vq[r][c][e] = (MODE != kColnorm && col < lda) ? vec[r * npb + col + e] : TA(0);
      }
  }
  TA sc0 = TA(0), sc1 = TA(0);
  // rows per group in flight: ~8 vector loads per lane (FP32), ~4 (FP64: twice the bytes per
  // load and twice the registers per value; two CTAs per SM hide the FP64 pipe's latency)
  constexpr int RU = (sizeof(TA) == 8) ? (CH >= 4 ? 1 : 4 / CH) : 8 / CH;
  for (int base = warp * G; base < t.rows; base += RU * NG) {   // warp-uniform trip count
    int rr[RU];
    bool hv[RU];
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      rr[u] = base + lane / LR + u * NG;
      hv[u] = rr[u] < t.rows;
    }
    TA x[RU][CH][4];
#pragma unroll
    for (int u = 0; u < RU; ++u)
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int col = 4 * (gl + LR * c);
        if (hv[u] && col < lda) load4(Ab + (int64_t)rr[u] * lda + col, x[u][c]);
        else x[u][c][0] = x[u][c][1] = x[u][c][2] = x[u][c][3] = TA(0);
      }
    if constexpr (MODE == kColnorm) {
#pragma unroll
      for (int u = 0; u < RU; ++u)
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const int col = 4 * (gl + LR * c);
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[0][c][e] = fma(x[u][c][e], x[u][c][e], acc[0][c][e]);
          // the FP32 working copy fl32(A) (round to nearest) and its low parts A - fl32(A)
          if (hv[u] && col < lda) {
            float hi[4], lo[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) f64_split_f32((double)x[u][c][e], hi[e], lo[e]);
            const int64_t off = P.offA + (int64_t)(t.row0 + rr[u]) * lda + col;
            *reinterpret_cast<float4*>(a.A32 + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
            if (a.Alo != nullptr)
              *reinterpret_cast<float4*>(a.Alo + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
          }
        }
    } else {
      TA d[RU][NR];
#pragma unroll
      for (int u = 0; u < RU; ++u)
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          d[u][r] = TA(0);
#pragma unroll
          for (int c = 0; c < CH; ++c)
#pragma unroll
            for (int e = 0; e < 4; ++e) d[u][r] = fma(x[u][c][e], vq[r][c][e], d[u][r]);
        }
#pragma unroll
      for (int o = LR / 2; o > 0; o >>= 1)
#pragma unroll
        for (int u = 0; u < RU; ++u)
#pragma unroll
          for (int r = 0; r < NR; ++r) d[u][r] += __shfl_xor_sync(0xffffffffu, d[u][r], o);
      if constexpr (MODE == kResid) {
        // r_i = b_i - a_i^T x (FP64), Alg. 2
#pragma unroll
        for (int u = 0; u < RU; ++u) {
          const double bv = hv[u] ? a.b[P.offB + t.row0 + rr[u]] : 0.0;
          const TA rv = (TA)bv - d[u][0];
#pragma unroll
          for (int c = 0; c < CH; ++c)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[0][c][e] = fma(rv, x[u][c][e], acc[0][c][e]);
          if (gl == 0) {
            sc0 = fma(rv, rv, sc0);
            sc1 = fma((TA)bv, rv, sc1);
          }
        }
      } else {
        // t = A q; the row's share of A^T t; ||t||^2
#pragma unroll
        for (int u = 0; u < RU; ++u) {
#pragma unroll
          for (int r = 0; r < NR; ++r)
#pragma unroll
            for (int c = 0; c < CH; ++c)
#pragma unroll
              for (int e = 0; e < 4; ++e) acc[r][c][e] = fma(d[u][r], x[u][c][e], acc[r][c][e]);
          if (gl == 0) {
            sc0 = fma(d[u][0], d[u][0], sc0);
            if constexpr (NR > 1) sc1 = fma(d[u][1], d[u][1], sc1);
          }
        }
      }
    }
  }
  // the G groups of a warp cover the same columns
#pragma unroll
  for (int o = LR; o < 32; o <<= 1)
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int e = 0; e < 4; ++e)
          acc[r][c][e] += __shfl_xor_sync(0xffffffffu, acc[r][c][e], o);
  TA* red = reinterpret_cast<TA*>(smem);   // [kPW][NR][NC]
  if (lane < LR)
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int e = 0; e < 4; ++e)
          red[(warp * NR + r) * NC + 4 * (gl + LR * c) + e] = acc[r][c][e];
  __shared__ double sred[kPW][2];
  sc0 = wsum(sc0);
  sc1 = wsum(sc1);
  if (lane == 0) {
    sred[warp][0] = (double)sc0;
    sred[warp][1] = (double)sc1;
  }
  __syncthreads();
  TA* out;
  if constexpr (MODE == kPcg) out = static_cast<TA*>(a.partU);
  else out = reinterpret_cast<TA*>(a.part64);
  const int64_t slab = (P.poff + (int64_t)(tile - P.tile0) * lda) * NR;
  for (int e = threadIdx.x; e < NR * lda; e += kPT) {
    const int r = e / lda, col = e - r * lda;
    TA s = TA(0);
#pragma unroll
    for (int w = 0; w < kPW; ++w) s += red[(w * NR + r) * NC + col];
    out[slab + e] = s;
  }
  if (threadIdx.x < 2) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kPW; ++w) s += sred[w][threadIdx.x];
    a.spart[(int64_t)tile * 4 + threadIdx.x] = s;
  }
}

// The residual pass of one tile in double-FP32 arithmetic (FP32 working precision): A as the
// pair A32 + Alo, x and b split into FP32 pairs, each row's dot product summed in pairs
// (TwoProd, TwoSum) and reduced over the row's lanes, r_i = b_i - a_i^T x as a pair, the
// axpy A^T r in pairs; the outputs in FP64 as the FP64 pass writes them (part64, spart).
template <int LR, int CH>
__device__ __forceinline__ void pass_body_df(const BArrays& a, const BProb& P, const BTile& t,
                                             int tile, unsigned char* smem) {
  constexpr int G = 32 / LR;
  constexpr int NG = kPW * G;
  constexpr int NC = 4 * LR * CH;
  constexpr int RU = (CH >= 4) ? 1 : 4 / CH;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gl = lane & (LR - 1);
  const int lda = (int)P.lda;
  const float* Ah = a.A32 + P.offA + (int64_t)t.row0 * lda;
  const float* Al = a.Alo + P.offA + (int64_t)t.row0 * lda;
  const double* xv = a.x + P.offV;
  float xh[CH][4], xl[CH][4], ach[CH][4], acl[CH][4];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int col = 4 * (gl + LR * c);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      ach[c][e] = acl[c][e] = 0.f;
      f64_split_f32(col < lda ? xv[col + e] : 0.0, xh[c][e], xl[c][e]);
    }
  }
  double sc0 = 0.0, sc1 = 0.0;
  for (int base = warp * G; base < t.rows; base += RU * NG) {   // warp-uniform trip count
    int rr[RU];
    bool hv[RU];
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      rr[u] = base + lane / LR + u * NG;
      hv[u] = rr[u] < t.rows;
    }
    float ah[RU][CH][4], al[RU][CH][4];
#pragma unroll
    for (int u = 0; u < RU; ++u)
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const int col = 4 * (gl + LR * c);
        if (hv[u] && col < lda) {
          const float4 vh = *reinterpret_cast<const float4*>(Ah + (int64_t)rr[u] * lda + col);
          const float4 vl = *reinterpret_cast<const float4*>(Al + (int64_t)rr[u] * lda + col);
          ah[u][c][0] = vh.x; ah[u][c][1] = vh.y; ah[u][c][2] = vh.z; ah[u][c][3] = vh.w;
          al[u][c][0] = vl.x; al[u][c][1] = vl.y; al[u][c][2] = vl.z; al[u][c][3] = vl.w;
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) ah[u][c][e] = al[u][c][e] = 0.f;
        }
      }
    float dh[RU], dl[RU];
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      dh[u] = dl[u] = 0.f;
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int e = 0; e < 4; ++e) df_fma(ah[u][c][e], al[u][c][e], xh[c][e], xl[c][e], dh[u], dl[u]);
    }
    // the row's lanes (a butterfly: TwoSum is symmetric, so every lane ends with the same pair)
#pragma unroll
    for (int o = LR / 2; o > 0; o >>= 1)
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        const float rh = __shfl_xor_sync(0xffffffffu, dh[u], o);
        const float rl = __shfl_xor_sync(0xffffffffu, dl[u], o);
        df_add(dh[u], dl[u], rh, rl);
      }
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const double bv = hv[u] ? a.b[P.offB + t.row0 + rr[u]] : 0.0;
      float bh, bl, rh, rl;
      f64_split_f32(bv, bh, bl);
      df_add(bh, bl, -dh[u], -dl[u]);   // r = b - A_i x as a pair,
      two_sum(bh, bl, rh, rl);          // renormalised for the products that follow
      if (!hv[u]) rh = rl = 0.f;
#pragma unroll
      for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int e = 0; e < 4; ++e) df_fma(ah[u][c][e], al[u][c][e], rh, rl, ach[c][e], acl[c][e]);
      if (gl == 0 && hv[u]) {
        const double r = (double)rh + (double)rl;
        sc0 = fma(r, r, sc0);
        sc1 = fma(bv, r, sc1);
      }
    }
  }
  // the G groups of a warp cover the same columns
#pragma unroll
  for (int o = LR; o < 32; o <<= 1)
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float rh = __shfl_xor_sync(0xffffffffu, ach[c][e], o);
        const float rl = __shfl_xor_sync(0xffffffffu, acl[c][e], o);
        df_add(ach[c][e], acl[c][e], rh, rl);
      }
  double* red = reinterpret_cast<double*>(smem);   // [kPW][NC]
  if (lane < LR)
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int e = 0; e < 4; ++e)
        red[warp * NC + 4 * (gl + LR * c) + e] = (double)ach[c][e] + (double)acl[c][e];
  __shared__ double sred[kPW][2];
  sc0 = wsum(sc0);
  sc1 = wsum(sc1);
  if (lane == 0) {
    sred[warp][0] = sc0;
    sred[warp][1] = sc1;
  }
  __syncthreads();
  double* out = a.part64;
  const int64_t slab = P.poff + (int64_t)(tile - P.tile0) * lda;
  for (int e = threadIdx.x; e < lda; e += kPT) {
    double s2 = 0.0;
#pragma unroll
    for (int w = 0; w < kPW; ++w) s2 += red[w * NC + e];
    out[slab + e] = s2;
  }
  if (threadIdx.x < 2) {
    double s2 = 0.0;
#pragma unroll
    for (int w = 0; w < kPW; ++w) s2 += sred[w][threadIdx.x];
    a.spart[(int64_t)tile * 4 + threadIdx.x] = s2;
  }
}

// ntile: device count of the tile list (a persistent grid loops over it), or NULL: one tile
// per CTA (tlist NULL: tile = CTA index)
template <typename TA, int NR, int MODE>
__global__ void __launch_bounds__(kPT, (sizeof(TA) == 8 && NR == 2) ? 1 : 2) pass_kernel(BArrays a, const int* __restrict__ tlist,
                                                   const int* __restrict__ ntile) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int nt = ntile ? *ntile : (int)gridDim.x;
  for (int ti = blockIdx.x; ti < nt; ti += gridDim.x) {
    const int tile = tlist ? tlist[ti] : ti;
    const BTile t = a.tiles[tile];   // tile lists hold only active problems' tiles
    if constexpr (MODE == kPcg) {
      // both shifted solves of this problem already met their tolerance: nothing to add
      const BState& st = a.st[t.prob];
      if (st.done[0] && (NR < 2 || st.done[1])) continue;
    }
    const BProb P = a.probs[t.prob];
    if constexpr (MODE == kResidDf) {
      switch (P.cfg) {
        case 0: pass_body_df<8, 1>(a, P, t, tile, smem); break;
        case 1: pass_body_df<16, 1>(a, P, t, tile, smem); break;
        case 2: pass_body_df<32, 1>(a, P, t, tile, smem); break;
        case 3: pass_body_df<32, 2>(a, P, t, tile, smem); break;
        default: pass_body_df<32, 4>(a, P, t, tile, smem); break;
      }
    } else {
      switch (P.cfg) {
        case 0: pass_body<TA, NR, MODE, 8, 1>(a, P, t, tile, smem); break;
        case 1: pass_body<TA, NR, MODE, 16, 1>(a, P, t, tile, smem); break;
        case 2: pass_body<TA, NR, MODE, 32, 1>(a, P, t, tile, smem); break;
        case 3: pass_body<TA, NR, MODE, 32, 2>(a, P, t, tile, smem); break;
        default: pass_body<TA, NR, MODE, 32, 4>(a, P, t, tile, smem); break;
      }
    }
    __syncthreads();   // shared memory is reused by the next tile
  }
}

template <typename TA, int NR>
constexpr size_t pass_smem() { return sizeof(TA) * kPW * NR * 4 * 32 * 4; }

// =========================================================================================
// Column norms: d_j = ||a_j||_2 (zero columns and padding: d = 1), ||A||_F^2, ||b||^2
// =========================================================================================
__global__ void __launch_bounds__(kCT) colnorm_post_kernel(BArrays a, const int* list) {
  const int pi = list[blockIdx.x];
  const BProb P = a.probs[pi];
  const int lda = (int)P.lda, npb = (int)P.npb, n = (int)P.n;
  __shared__ double sh[32 * 2];
  double s2[2] = {0.0, 0.0};
  for (int c = threadIdx.x; c < npb; c += kCT) {
    double dd = 1.0;
    if (c < n) {
      const double* base = a.part64 + P.poff + c;
      double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
      int i = 0;
      for (; i + 3 < P.ntiles; i += 4) {
        t0 += base[(int64_t)i * lda];
        t1 += base[(int64_t)(i + 1) * lda];
        t2 += base[(int64_t)(i + 2) * lda];
        t3 += base[(int64_t)(i + 3) * lda];
      }
      for (; i < P.ntiles; ++i) t0 += base[(int64_t)i * lda];
      dd = sqrt((t0 + t1) + (t2 + t3));
      if (!(dd > 0.0)) dd = 1.0;
      s2[0] = fma(dd, dd, s2[0]);
    }
    a.d[P.offV + c] = dd;
    a.dinv[P.offV + c] = 1.0 / dd;
    a.dinv32[P.offV + c] = (float)(1.0 / dd);
  }
  for (int64_t i = threadIdx.x; i < P.m; i += kCT) {
    const double bv = a.b[P.offB + i];
    s2[1] = fma(bv, bv, s2[1]);
  }
  bsum<double, 2>(s2, sh);
  if (threadIdx.x == 0) {
    BState& st = a.st[pi];
    st.norm2_A = s2[0];
    st.norm2_b = s2[1];
    st.scale = s2[0] + s2[1];
  }
}

// =========================================================================================
// Gram H = A_s^T A_s, A_s = fl_uf(A D^{-1}) (upper 64 x 64 tiles of every problem)
// =========================================================================================
// fl_uf(a_ij / d_j): FP32 path fl32(fl32(a_ij) * fl32(1/d_j)) rounded to u_f (the product a
// tensor core would form from the stored operand); FP64 path a_ij * (1/d_j) in FP64
template <typename C> struct GramSrc;
template <> struct GramSrc<float> {
  static __device__ __forceinline__ const float* A(const BArrays& a) { return a.A32; }
  static __device__ __forceinline__ float dinv(const BArrays& a, int64_t k) { return a.dinv32[k]; }
};
template <> struct GramSrc<double> {
  static __device__ __forceinline__ const double* A(const BArrays& a) { return a.A64; }
  static __device__ __forceinline__ double dinv(const BArrays& a, int64_t k) { return a.dinv[k]; }
};

// One CTA (64 threads, 8 x 8 outputs each) forms the 64 x 64 tile H[I][J] over the rows
// [r0, r1) of its problem: staged 32-row chunks of the scaled, u_f-rounded columns of I and J
// (a diagonal tile stages one block for both), FMA into registers. Tiles whose rows are split
// write their partial tile to a workspace slot; the others write H directly.
template <typename C>
__global__ void __launch_bounds__(64) gram_kernel(BArrays a, const GTile* __restrict__ gt,
                                                  C* __restrict__ work) {
  const GTile g = gt[blockIdx.x];
  const BProb P = a.probs[g.prob];
  const int n = (int)P.n, npb = (int)P.npb;
  const int c0 = g.bi * kNB, c1 = g.bj * kNB;
  const bool diag = (g.bi == g.bj);
  __shared__ __align__(16) C SA[32][kLd];
  __shared__ __align__(16) C SB[32][kLd];
  const int tid = threadIdx.x, ty = tid >> 3, tx = tid & 7;
  C acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = C(0);
  // this thread stages column tid of each block; its scale factor stays in a register
  const bool okA = c0 + tid < n, okB = c1 + tid < n;
  const C* Ab = GramSrc<C>::A(a) + P.offA;
  const C dA = okA ? GramSrc<C>::dinv(a, P.offV + c0 + tid) : C(0);
  const C dB = okB ? GramSrc<C>::dinv(a, P.offV + c1 + tid) : C(0);
  const int lda = (int)P.lda, prec = P.prec;
  for (int64_t r0 = g.r0; r0 < g.r1; r0 += 32) {
    const int rows = (int)min((int64_t)32, (int64_t)g.r1 - r0);
    // the loads of 16 rows first, then their scaling and the stores to shared memory
#pragma unroll
    for (int h = 0; h < 32; h += 16) {
      C ra[16], rb[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int rr = h + u;
        const int64_t row = r0 + rr;
        ra[u] = (rr < rows && okA) ? Ab[row * lda + c0 + tid] : C(0);
        rb[u] = (!diag && rr < rows && okB) ? Ab[row * lda + c1 + tid] : C(0);
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        SA[h + u][tid] = round_uf(ra[u] * dA, prec);
        if (!diag) SB[h + u][tid] = round_uf(rb[u] * dB, prec);
      }
    }
    __syncthreads();
    const C (*B)[kLd] = diag ? SA : SB;
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {
      // vector reads from shared memory: 4 loads (FP32) for 64 FMA
      C av[8], bv[8];
      lds4(&SA[k][ty * 8], *reinterpret_cast<C(*)[4]>(av));
      lds4(&SA[k][ty * 8 + 4], *reinterpret_cast<C(*)[4]>(av + 4));
      lds4(&B[k][tx * 8], *reinterpret_cast<C(*)[4]>(bv));
      lds4(&B[k][tx * 8 + 4], *reinterpret_cast<C(*)[4]>(bv + 4));
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (g.slot >= 0) {
    C* w = work + (int64_t)g.slot * kNB * kNB;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) w[(ty * 8 + i) * kNB + tx * 8 + j] = acc[i][j];
    return;
  }
  C* H = static_cast<C*>(a.H) + P.offM;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int r = c0 + ty * 8 + i, c = c1 + tx * 8 + j;
      // identity on the padding (rows / columns >= n): padded entries never couple
      H[(int64_t)r * npb + c] = (r == c && r >= n) ? C(1) : acc[i][j];
    }
}

// Sum of the row-split partial tiles of one H tile, in slot order (deterministic).
template <typename C>
__global__ void __launch_bounds__(256) gram_reduce_kernel(BArrays a, const GTile* __restrict__ gr,
                                                          const C* __restrict__ work) {
  const GTile g = gr[blockIdx.x];     // slot = first slot, r1 - r0 = number of slots
  const BProb P = a.probs[g.prob];
  const int n = (int)P.n, npb = (int)P.npb;
  const int ns = g.r1 - g.r0;
  C* H = static_cast<C*>(a.H) + P.offM;
  for (int e = threadIdx.x; e < kNB * kNB; e += 256) {
    C v = C(0);
    for (int sidx = 0; sidx < ns; ++sidx) v += work[(int64_t)(g.slot + sidx) * kNB * kNB + e];
    const int r = g.bi * kNB + e / kNB, c = g.bj * kNB + e % kNB;
    H[(int64_t)r * npb + c] = (r == c && r >= n) ? C(1) : v;
  }
}

// =========================================================================================
// Inverse of an upper-triangular 64 x 64 block S (shared, row stride kLd) into X (shared), by
// doubling: the eight 8 x 8 diagonal blocks by substitution (chains of at most 8), then for
// SB = 8, 16, 32 every pair of SB-blocks A, B gets X_AB = -X_AA (R_AB X_BB) as two products
// through Tm (scratch, 64 x kLd). The k sums run over the whole block length (the entries of
// X_BB below and of X_AA left of the diagonal are zero), so they unroll. Call with all
// threads of the CTA.
// =========================================================================================
template <typename C, int SB>
__device__ __forceinline__ void inv_level(const C* S, C* X, C* Tm) {
  constexpr int pairs = kNB / (2 * SB), cnt = pairs * SB * SB;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int pr = e / (SB * SB), rem = e % (SB * SB), i = rem / SB, j = rem % SB;
    const int a = 2 * pr * SB;
    C v = C(0);
#pragma unroll
    for (int k = 0; k < SB; ++k)
      v = fma(S[(a + i) * kLd + a + SB + k], X[(a + SB + k) * kLd + a + SB + j], v);
    Tm[(pr * SB + i) * kLd + j] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int pr = e / (SB * SB), rem = e % (SB * SB), i = rem / SB, j = rem % SB;
    const int a = 2 * pr * SB;
    C v = C(0);
#pragma unroll
    for (int k = 0; k < SB; ++k) v = fma(X[(a + i) * kLd + a + k], Tm[(pr * SB + k) * kLd + j], v);
    X[(a + i) * kLd + a + SB + j] = -v;
  }
  __syncthreads();
}

template <typename C>
__device__ void inv_upper64(const C* S, C* X, C* Tm) {
  const int tid = threadIdx.x;
  for (int e = tid; e < kNB * kLd; e += blockDim.x) X[e] = C(0);
  __syncthreads();
  if (tid < 64) {
    const int o = (tid >> 3) * 8, j = tid & 7;
    for (int i = j; i >= 0; --i) {
      C v = (i == j) ? C(1) : C(0);
      for (int k = i + 1; k <= j; ++k) v = fma(-S[(o + i) * kLd + o + k], X[(o + k) * kLd + o + j], v);
      X[(o + i) * kLd + o + j] = v / S[(o + i) * kLd + o + i];
    }
  }
  __syncthreads();
  inv_level<C, 8>(S, X, Tm);
  inv_level<C, 16>(S, X, Tm);
  inv_level<C, 32>(S, X, Tm);
}

// =========================================================================================
// Blocked Cholesky H + s I = R_H^T R_H (upper, 64-blocks) and W = R_H^{-1}, as task lists over
// all listed problems: step s of every problem runs in the same three launches (diagonal
// blocks, panels, trailing tiles), so the work of the large problems spreads over the GPU
// instead of one CTA each. A CTask names a problem and a block step; the host builds the lists.
// =========================================================================================

// 64 x 64 global tile G (row stride ld) into shared memory D (row stride kLd), transposed
// (D[c][r] = G[r][c]) or not; 256 threads.
template <typename Tin, typename T>
__device__ __forceinline__ void stage64(const Tin* __restrict__ G, int64_t ld, T* D, bool trans) {
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const int r = e >> 6, c = e & 63;
    const T v = (T)G[(int64_t)r * ld + c];
    if (trans) D[c * kLd + r] = v;
    else D[r * kLd + c] = v;
  }
}


// acc += As^T Bs over k = 0..63 for the 4 x 4 outputs of this thread: rows 4 ty .. +3, columns
// 4 tx .. +3 (tx = tid % 16, ty = tid / 16; 256 threads); As[k][i], Bs[k][j] in shared memory.
template <typename T>
__device__ __forceinline__ void tile_atb(const T* As, const T* Bs, T (&acc)[4][4]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll 8
  for (int k = 0; k < kNB; ++k) {
    T av[4], bv[4];
    lds4(As + k * kLd + 4 * ty, av);
    lds4(Bs + k * kLd + 4 * tx, bv);
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] = fma(av[p], bv[q], acc[p][q]);
  }
}

// M = H + shift I for the listed problems; info = 0. Grid (problems, 8).
template <typename C>
__global__ void __launch_bounds__(256) chol_init_kernel(BArrays a, const int* list,
                                                        const double* shift, int* info) {
  const int pi = list[blockIdx.x];
  const BProb P = a.probs[pi];
  const int64_t npb = P.npb;
  const C* H = static_cast<const C*>(a.H) + P.offM;
  C* M = static_cast<C*>(a.R) + P.offM;
  const C sh = (C)shift[pi];
  for (int64_t e = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < npb * npb;
       e += (int64_t)blockDim.x * gridDim.y) {
    const int64_t r = e / npb, c = e % npb;
    C v = H[e];
    if (r == c && r < P.n) v += sh;
    M[e] = v;
  }
  if (blockIdx.y == 0 && threadIdx.x == 0) info[pi] = 0;
}

// Step s, diagonal block: R_ss (rows rounded to u_f as they are written) and, when a panel
// follows, W_ss = R_ss^{-1} of the rounded block, parked in the unused block (s+1, s) below the
// diagonal. A non-positive (or NaN) pivot stops the problem: info = pivot + 1.
template <typename C>
__global__ void __launch_bounds__(256) chol_diag_kernel(BArrays a, const CTask* tasks, int* info) {
  const CTask t = tasks[blockIdx.x];
  if (*(volatile int*)(info + t.prob) != 0) return;
  const BProb P = a.probs[t.prob];
  const int64_t npb = P.npb;
  const int nb = (int)(npb / kNB), kb = t.s * kNB, prec = P.prec;
  C* M = static_cast<C*>(a.R) + P.offM;
  extern __shared__ __align__(16) unsigned char smem[];
  C* S = reinterpret_cast<C*>(smem);
  C* X = S + kNB * kLd;
  C* Tm = X + kNB * kLd;
  __shared__ chol64::Scratch<C> sc;
  const int bad = chol64::factor_block<C>(M + (int64_t)kb * npb + kb, npb, S, kLd, sc,
                                          [prec](C v) { return round_uf(v, prec); });
  if (bad) {
    if (threadIdx.x == 0) info[t.prob] = kb + bad;
    return;
  }
  if (t.s + 1 < nb) {
    inv_upper64<C>(S, X, Tm);
    C* Wp = M + (int64_t)(kb + kNB) * npb + kb;
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x)
      Wp[(int64_t)(e >> 6) * npb + (e & 63)] = X[(e >> 6) * kLd + (e & 63)];
  }
}

// Step s, panel block (s, bj): R_s,bj = W_ss^T H_s,bj in place.
// Step s, trailing block (bi, bj), s < bi <= bj: H_bi,bj -= R_s,bi^T R_s,bj.
template <typename C, bool PANEL>
__global__ void __launch_bounds__(256) chol_tile_kernel(BArrays a, const CTask* tasks,
                                                        const int* info) {
  const CTask t = tasks[blockIdx.x];
  if (*(volatile const int*)(info + t.prob) != 0) return;
  const BProb P = a.probs[t.prob];
  const int64_t npb = P.npb;
  const int kb = t.s * kNB;
  C* M = static_cast<C*>(a.R) + P.offM;
  extern __shared__ __align__(16) unsigned char smem[];
  C* As = reinterpret_cast<C*>(smem);
  C* Bs = As + kNB * kLd;
  const C* Ag = PANEL ? M + (int64_t)(kb + kNB) * npb + kb : M + (int64_t)kb * npb + t.bi * kNB;
  const C* Bg = M + (int64_t)kb * npb + t.bj * kNB;
  C* Cg = PANEL ? M + (int64_t)kb * npb + t.bj * kNB
                : M + (int64_t)t.bi * kNB * npb + t.bj * kNB;
  stage64<C, C>(Ag, npb, As, false);
  stage64<C, C>(Bg, npb, Bs, false);
  __syncthreads();
  C acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = C(0);
  tile_atb<C>(As, Bs, acc);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      C* cp = Cg + (int64_t)(4 * ty + p) * npb + 4 * tx + q;
      *cp = PANEL ? acc[p][q] : *cp - acc[p][q];
    }
}

// Every entry of R_H rounded to u_f, the lower part zeroed (W_ss blocks included).
// Grid (problems, 8).
template <typename C>
__global__ void __launch_bounds__(256) chol_final_kernel(BArrays a, const int* list,
                                                         const int* info) {
  const int pi = list[blockIdx.x];
  if (info[pi] != 0) return;
  const BProb P = a.probs[pi];
  const int64_t npb = P.npb;
  const int prec = P.prec;
  C* M = static_cast<C*>(a.R) + P.offM;
  for (int64_t e = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < npb * npb;
       e += (int64_t)blockDim.x * gridDim.y) {
    const int64_t r = e / npb, c = e % npb;
    M[e] = (c < r) ? C(0) : round_uf(M[e], prec);
  }
}

// W = R_H^{-1} (u type T) by block diagonals. Level 0, task (prob, I): W_II = R_II^{-1} and the
// zero blocks left of it. Level d, task (prob, I, J = I + d): W_IJ = -W_II sum_{I<K<=J} R_IK W_KJ
// (the W_KJ are on lower levels). Each task also writes its block of W^T.
template <typename C, typename T>
__global__ void __launch_bounds__(256) trtri_tile_kernel(BArrays a, const CTask* tasks) {
  const CTask t = tasks[blockIdx.x];
  const BProb P = a.probs[t.prob];
  const int64_t npb = P.npb;
  const int I = t.bi, J = t.bj;
  const C* R = static_cast<const C*>(a.R) + P.offM;
  T* W = static_cast<T*>(a.W) + P.offM;
  T* WT = static_cast<T*>(a.WT) + P.offM;
  extern __shared__ __align__(16) unsigned char smem[];
  T* S = reinterpret_cast<T*>(smem);      // 64 x kLd
  T* X = S + kNB * kLd;                   // 64 x kLd
  T* Tm = X + kNB * kLd;                  // 64 x kLd
  const int tid = threadIdx.x;
  if (I == J) {
    for (int e = tid; e < kNB * kNB; e += blockDim.x) {
      const int r = e >> 6, c = e & 63;
      S[r * kLd + c] = (c >= r) ? (T)R[(int64_t)(I * kNB + r) * npb + I * kNB + c] : T(0);
    }
    __syncthreads();
    inv_upper64<T>(S, X, Tm);
    for (int e = tid; e < kNB * kNB; e += blockDim.x) {
      const int r = e >> 6, c = e & 63;
      const T v = X[r * kLd + c];
      W[(int64_t)(I * kNB + r) * npb + I * kNB + c] = v;
      WT[(int64_t)(I * kNB + c) * npb + I * kNB + r] = v;
    }
    // blocks (I, K < I) of W and (K < I, I) of W^T are zero
    for (int64_t e = tid; e < (int64_t)I * kNB * kNB; e += blockDim.x) {
      const int64_t r = e / (I * kNB), c = e % (I * kNB);
      W[(int64_t)(I * kNB + r) * npb + c] = T(0);
      WT[c * npb + I * kNB + r] = T(0);
    }
    return;
  }
  // Tacc = sum_K R_IK W_KJ: As[k][i] = R_IK[i][k] (transposed stage), Bs[k][j] = W_KJ[k][j]
  T acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = T(0);
  for (int K = I + 1; K <= J; ++K) {
    stage64<C, T>(R + (int64_t)(I * kNB) * npb + K * kNB, npb, S, true);
    stage64<T, T>(W + (int64_t)(K * kNB) * npb + J * kNB, npb, X, false);
    __syncthreads();
    tile_atb<T>(S, X, acc);
    __syncthreads();
  }
  const int tx = tid & 15, ty = tid >> 4;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) Tm[(4 * ty + p) * kLd + 4 * tx + q] = acc[p][q];
  // W_IJ = -W_II Tacc: As[k][i] = W_II[i][k]
  stage64<T, T>(W + (int64_t)(I * kNB) * npb + I * kNB, npb, S, true);
  __syncthreads();
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = T(0);
  tile_atb<T>(S, Tm, acc);
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t r = I * kNB + 4 * ty + p, c = J * kNB + 4 * tx + q;
      W[r * npb + c] = -acc[p][q];
      WT[c * npb + r] = -acc[p][q];
    }
}

// =========================================================================================
// Per-problem GEMVs with the inverse factor (one warp per row, rows from L2)
// =========================================================================================
// v_r[i] = sum_{j <= i} WT[i][j] y_r[j]   (WT = W^T lower triangular), r < nr.
// A warp takes two rows at a time and issues every load of both rows before its FMAs (the
// rows come from L2 / HBM; a loop of dependent load-FMA rounds would be latency bound).
template <typename T, bool LOWER>
__device__ __forceinline__ void gemv_tri(const T* __restrict__ M, int npb, const T* xs, T* vs,
                                         int nr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int U = kMaxN / 128;   // 4-column chunks per lane of a full row
  for (int i0 = warp; i0 < npb; i0 += 2 * kCW) {
    const int i1 = i0 + kCW;
    T w0[U][4], w1[U][4];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int c = lane * 4 + 128 * u;
      // lower: columns c <= i; upper: columns from the chunk holding i to the end
      const bool ok0 = LOWER ? (c <= i0) : (c + 3 >= i0 && c < npb);
      const bool ok1 = (i1 < npb) && (LOWER ? (c <= i1) : (c + 3 >= i1 && c < npb));
      if (ok0) ldrow4(M + (int64_t)i0 * npb + c, w0[u]);
      else w0[u][0] = w0[u][1] = w0[u][2] = w0[u][3] = T(0);
      if (ok1) ldrow4(M + (int64_t)i1 * npb + c, w1[u]);
      else w1[u][0] = w1[u][1] = w1[u][2] = w1[u][3] = T(0);
    }
    T a00 = T(0), a01 = T(0), a10 = T(0), a11 = T(0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int c = lane * 4 + 128 * u;
      if (c < npb) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const T x0 = xs[c + e];
          a00 = fma(w0[u][e], x0, a00);
          a10 = fma(w1[u][e], x0, a10);
          if (nr > 1) {
            const T x1 = xs[npb + c + e];
            a01 = fma(w0[u][e], x1, a01);
            a11 = fma(w1[u][e], x1, a11);
          }
        }
      }
    }
    a00 = wsum(a00);
    a10 = wsum(a10);
    if (nr > 1) {
      a01 = wsum(a01);
      a11 = wsum(a11);
    }
    if (lane == 0) {
      vs[i0] = a00;
      if (nr > 1) vs[npb + i0] = a01;
      if (i1 < npb) {
        vs[i1] = a10;
        if (nr > 1) vs[npb + i1] = a11;
      }
    }
  }
}
template <typename T>
__device__ void gemv_lower(const T* __restrict__ WT, int npb, const T* ys, T* vs, int nr) {
  gemv_tri<T, true>(WT, npb, ys, vs, nr);
}
// v_r[i] = sum_{j >= i} W[i][j] p_r[j]   (W upper triangular)
template <typename T>
__device__ void gemv_upper(const T* __restrict__ W, int npb, const T* ps, T* vs, int nr) {
  gemv_tri<T, false>(W, npb, ps, vs, nr);
}

// sum over the tiles of a problem of part[i * step] (8 loads in flight)
template <typename T>
__device__ __forceinline__ T sum_tiles(const T* __restrict__ base, int ntiles, int64_t step) {
  T t[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) t[k] = T(0);
  int i = 0;
  for (; i + 7 < ntiles; i += 8)
#pragma unroll
    for (int k = 0; k < 8; ++k) t[k] += base[(int64_t)(i + k) * step];
  for (; i < ntiles; ++i) t[0] += base[(int64_t)i * step];
  return ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
}

// Shared memory of the per-problem solve kernels: 4 vectors of 2 x kMaxN in T plus FP64 scratch
template <typename T>
constexpr size_t post_smem() { return sizeof(T) * 4 * 2 * kMaxN; }

struct PVec {   // u-type vector pairs of one problem
  template <typename T> __device__ static T* at(void* base, const BProb& P) {
    return static_cast<T*>(base) + 2 * P.offV;
  }
};

// PCGTLS start (Alg. 3): s_0 = R^{-T} rhs (y = D^{-1} rhs staged in ys by the caller),
// eta_0 = ||s_0||^2, p_0 = s_0, q_0 = R^{-1} p_0 = D^{-1} W p_0, w = 0.
template <typename T>
__device__ void pcg_start(const BArrays& a, const BProb& P, BState& st, int nr, T* ys, T* vs,
                          double* dsh) {
  const int npb = (int)P.npb;
  const T* W = static_cast<const T*>(a.W) + P.offM;
  const T* WT = static_cast<const T*>(a.WT) + P.offM;
  const T* dv = dinv_of<T>(a) + P.offV;
  T* s = PVec::at<T>(a.vs, P);
  T* p = PVec::at<T>(a.vp, P);
  T* q = PVec::at<T>(a.vq, P);
  T* w = PVec::at<T>(a.vw, P);
  __syncthreads();
  gemv_lower<T>(WT, npb, ys, vs, nr);
  __syncthreads();
  double e[2] = {0.0, 0.0};
  {
    T el[2] = {T(0), T(0)};
    for (int c = threadIdx.x; c < npb; c += kCT)
      for (int r = 0; r < 2; ++r) {
        const T sv = (r < nr) ? vs[r * npb + c] : T(0);
        s[r * npb + c] = sv;
        p[r * npb + c] = sv;
        w[r * npb + c] = T(0);
        ys[r * npb + c] = sv;
        el[r] = fma(sv, sv, el[r]);
      }
    e[0] = (double)el[0];
    e[1] = (double)el[1];
  }
  bsum<double, 2>(e, dsh);
  if (threadIdx.x == 0) {
    for (int r = 0; r < 2; ++r) {
      st.eta[r] = e[r];
      st.eta0[r] = e[r];
      st.beta[r] = 0.0;
      st.alpha[r] = 0.0;
      st.delta[r] = 1.0;
      st.done[r] = (r < nr) ? (e[r] == 0.0 ? 1 : 0) : 1;
      st.not_spd[r] = 0;
      st.iters[r] = 0;
    }
    st.nr = nr;
  }
  __syncthreads();
  gemv_upper<T>(W, npb, ys, vs, nr);
  __syncthreads();
  T qp[4] = {T(0), T(0), T(0), T(0)};
  for (int c = threadIdx.x; c < npb; c += kCT)
    for (int r = 0; r < nr; ++r) {
      const T qv = vs[r * npb + c] * dv[c];
      q[r * npb + c] = qv;
      qp[r] = fma(qv, qv, qp[r]);
      qp[2 + r] = fma(ys[r * npb + c], ys[r * npb + c], qp[2 + r]);
    }
  double qd[4] = {(double)qp[0], (double)qp[1], (double)qp[2], (double)qp[3]};
  bsum<double, 4>(qd, dsh);
  if (threadIdx.x == 0) {
    st.qq[0] = qd[0];
    st.qq[1] = qd[1];
    st.pp[0] = qd[2];
    st.pp[1] = qd[3];
  }
}

template <typename T>
__global__ void __launch_bounds__(kCT) solve_init_kernel(BArrays a, const int* list) {
  const int pi = list[blockIdx.x];
  const BProb P = a.probs[pi];
  for (int c = threadIdx.x; c < P.npb; c += kCT) {
    a.x[P.offV + c] = 0.0;
    a.xbest[P.offV + c] = 0.0;
    a.f[P.offV + c] = 0.0;
  }
  if (threadIdx.x == 0) {
    BState& st = a.st[pi];
    st.xx = 0.0;
    st.k = 0;
    st.best_k = 0;
    st.best_psi = INFINITY;
    st.prev_psi = INFINITY;
    st.best_s2 = 0.0;
    st.stop = TLS_STOP_MAX_RQI;
    st.active = 1;
    st.n_psi = 0;
    st.cg_total = 0;
    st.not_spd_any = 0;
    st.nr = 1;
  }
}

// Residual block of Alg. 2 in FP64 (r = b - A x, sigma^2 = ||r||^2 / (1 + ||x||^2),
// f = -A^T r - sigma^2 x, g = -b^T r + sigma^2, psi of Eq. (4)), then by `mode`:
//  kResidLs    start PCGTLS with sigma^2 = 0 on -f (the LS start x_0, Alg. 2 line 1)
//  kResidStart the inverse-iteration step x_1 = x_0 + sigma_0^2 (R^T R)^{-1} x_0
//  kResidRqi   the stopping rules (Sec. 3 after Eq. (4)) and, if the problem goes on, the
//              two shifted solves' start on -f and x
template <typename T>
__device__ void resid_post_body(const BArrays& a, const int pi, int mode, const SolveParams& sp) {
  BState& st = a.st[pi];
  if (!st.active) return;
  const BProb P = a.probs[pi];
  const int npb = (int)P.npb, n = (int)P.n, lda = (int)P.lda;
  extern __shared__ __align__(16) unsigned char smem[];
  T* ys = reinterpret_cast<T*>(smem);
  T* vs = ys + 2 * kMaxN;
  double* at = reinterpret_cast<double*>(vs + 2 * kMaxN);   // kMaxN doubles
  __shared__ double dsh[32 * 4];
  __shared__ int s_dec[2];
  double* x = a.x + P.offV;
  double* f = a.f + P.offV;
  const double* dinv = a.dinv + P.offV;
  // sum of the tile partials of A^T r, ||r||^2, b^T r
  double rs[2] = {0.0, 0.0};
  for (int c = threadIdx.x; c < npb; c += kCT)
    at[c] = (c < lda) ? sum_tiles<double>(a.part64 + P.poff + c, P.ntiles, lda) : 0.0;
  for (int i = threadIdx.x; i < P.ntiles; i += kCT) {
    rs[0] += a.spart[(int64_t)(P.tile0 + i) * 4 + 0];
    rs[1] += a.spart[(int64_t)(P.tile0 + i) * 4 + 1];
  }
  bsum<double, 2>(rs, dsh);
  const double xx = st.xx;
  const double sigma2 = rs[0] / (1.0 + xx);
  double ff[1] = {0.0};
  for (int c = threadIdx.x; c < npb; c += kCT) {
    const double fj = (c < n) ? (-at[c] - sigma2 * x[c]) : 0.0;
    f[c] = fj;
    ff[0] = fma(fj, fj, ff[0]);
  }
  bsum<double, 1>(ff, dsh);
  const double g = -rs[1] + sigma2;
  const double psi = sqrt((ff[0] + g * g) / (xx + 1.0));
  if (threadIdx.x == 0) {
    st.rr = rs[0];
    st.br = rs[1];
    st.sigma2 = sigma2;
    st.g = g;
    st.ff = ff[0];
    st.psi = psi;
  }
  if (mode == kResidLs) {
    for (int c = threadIdx.x; c < npb; c += kCT) {
      ys[c] = (T)(-f[c] * dinv[c]);
      ys[npb + c] = T(0);
    }
    if (threadIdx.x == 0) {
      st.cg_sigma2 = 0.0;
      st.cg_tol2 = 0.0;
    }
    pcg_start<T>(a, P, st, 1, ys, vs, dsh);
    return;
  }
  if (mode == kResidStart) {
    // u_0 = R^{-1} R^{-T} x_0 = D^{-1} W W^T D^{-1} x_0; x_1 = x_0 + sigma_0^2 u_0
    const T* W = static_cast<const T*>(a.W) + P.offM;
    const T* WT = static_cast<const T*>(a.WT) + P.offM;
    const T* dv = dinv_of<T>(a) + P.offV;
    for (int c = threadIdx.x; c < npb; c += kCT) ys[c] = (T)(x[c] * dinv[c]);
    __syncthreads();
    gemv_lower<T>(WT, npb, ys, vs, 1);
    __syncthreads();
    gemv_upper<T>(W, npb, vs, ys, 1);
    __syncthreads();
    double xs[1] = {0.0};
    for (int c = threadIdx.x; c < npb; c += kCT) {
      double xn = 0.0;
      if (c < n) xn = fma(sigma2, (double)(ys[c] * dv[c]), x[c]);
      x[c] = xn;
      xs[0] = fma(xn, xn, xs[0]);
    }
    bsum<double, 1>(xs, dsh);
    if (threadIdx.x == 0) st.xx = xs[0];
    return;
  }
  // RQI step k: stopping rules, best iterate
  if (threadIdx.x == 0) {
    const int k = st.k + 1;
    st.k = k;
    if (st.n_psi < 24) st.psi_hist[st.n_psi++] = psi;
    int stop = 0, improve = 0;
    if (!isfinite(psi) || !isfinite(sigma2)) {
      stop = TLS_STOP_PSI_UP;
    } else {
      const bool up = sp.psi_rule_ge ? (psi >= st.prev_psi) : (psi > st.prev_psi);
      if (up && st.best_psi <= sp.psi_accept * st.scale) {
        stop = TLS_STOP_PSI_UP;
      } else {
        if (psi < st.best_psi) {
          improve = 1;
          st.best_k = k;
          st.best_psi = psi;
          st.best_s2 = sigma2;
        }
        // tolerance test from the second RQI step on (psi_1 is taken at the start x_1)
        if (!up && k >= 2 && psi <= sp.tol * st.scale) stop = TLS_STOP_TOL;
        else if (k > sp.max_rqi) stop = TLS_STOP_MAX_RQI;
      }
    }
    st.prev_psi = psi;
    s_dec[0] = stop;
    s_dec[1] = improve;
  }
  __syncthreads();
  if (s_dec[1])
    for (int c = threadIdx.x; c < npb; c += kCT) a.xbest[P.offV + c] = x[c];
  if (s_dec[0]) {
    if (threadIdx.x == 0) {
      st.stop = s_dec[0];
      st.active = 0;
    }
    return;
  }
  for (int c = threadIdx.x; c < npb; c += kCT) {
    ys[c] = (T)(-f[c] * dinv[c]);
    ys[npb + c] = (T)(x[c] * dinv[c]);
  }
  if (threadIdx.x == 0) {
    st.cg_sigma2 = sigma2;
    const double ct = a.cg_tol ? a.cg_tol[pi] : sp.cg_tol;
    st.cg_tol2 = sp.cg_fixed ? 0.0 : ct * ct;
  }
  pcg_start<T>(a, P, st, 2, ys, vs, dsh);
}

template <typename T>
__global__ void __launch_bounds__(kCT) resid_post_kernel(BArrays a, const int* list,
                                                         const int* cnt, int mode,
                                                         SolveParams sp) {
  const int n = cnt ? *cnt : (int)gridDim.x;
  for (int li = blockIdx.x; li < n; li += gridDim.x) {
    resid_post_body<T>(a, list[li], mode, sp);
    __syncthreads();
  }
}

// One PCGTLS step after the pass t = A q (Alg. 3, operator with A):
// delta = ||t||^2 - sigma^2 ||q||^2, alpha = eta / delta, w += alpha q,
// s -= alpha R^{-T}(A^T t - sigma^2 q), eta' = ||s||^2, beta = eta'/eta, p = s + beta p,
// q = R^{-1} p.
template <typename T>
__device__ void pcg_post_body(const BArrays& a, const int pi) {
  BState& st = a.st[pi];
  if (!st.active) return;
  const int nr = st.nr;
  if (st.done[0] && (nr < 2 || st.done[1])) return;
  const BProb P = a.probs[pi];
  const int npb = (int)P.npb, lda = (int)P.lda;
  extern __shared__ __align__(16) unsigned char smem[];
  T* ys = reinterpret_cast<T*>(smem);
  T* vs = ys + 2 * kMaxN;
  T* at = vs + 2 * kMaxN;
  __shared__ double dsh[32 * 4];
  __shared__ T s_alpha[2];
  __shared__ int s_ok[2];
  const T* W = static_cast<const T*>(a.W) + P.offM;
  const T* WT = static_cast<const T*>(a.WT) + P.offM;
  const T* dv = dinv_of<T>(a) + P.offV;
  T* s = PVec::at<T>(a.vs, P);
  T* p = PVec::at<T>(a.vp, P);
  T* q = PVec::at<T>(a.vq, P);
  T* w = PVec::at<T>(a.vw, P);
  const T* part = static_cast<const T*>(a.partU);
  // sum of the tile partials of A^T t (per right-hand side) and ||t||^2
  for (int e = threadIdx.x; e < nr * npb; e += kCT) {
    const int r = e / npb, c = e - r * npb;
    at[e] = (c < lda) ? sum_tiles<T>(part + P.poff * nr + (int64_t)r * lda + c, P.ntiles,
                                     (int64_t)lda * nr)
                      : T(0);
  }
  double tt[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < P.ntiles; i += kCT) {
    tt[0] += a.spart[(int64_t)(P.tile0 + i) * 4 + 0];
    tt[1] += a.spart[(int64_t)(P.tile0 + i) * 4 + 1];
  }
  bsum<double, 2>(tt, dsh);
  if (threadIdx.x == 0) {
    for (int r = 0; r < 2; ++r) {
      s_ok[r] = 0;
      s_alpha[r] = T(0);
      if (r < nr && !st.done[r]) {
        const double delta = tt[r] - st.cg_sigma2 * st.qq[r];
        st.delta[r] = delta;
        if (delta > 0.0) {
          const double alpha = st.eta[r] / delta;
          st.alpha[r] = alpha;
          s_alpha[r] = (T)alpha;
          s_ok[r] = 1;
        }
      }
    }
  }
  __syncthreads();
  const T sig2 = (T)st.cg_sigma2;
  for (int e = threadIdx.x; e < nr * npb; e += kCT) {
    const int r = e / npb, c = e - r * npb;
    T yv = T(0);
    if (s_ok[r]) {
      const T qv = q[e];
      w[e] = fma(s_alpha[r], qv, w[e]);
      yv = (at[e] - sig2 * qv) * dv[c];
    }
    ys[e] = yv;
  }
  __syncthreads();
  gemv_lower<T>(WT, npb, ys, vs, nr);
  __syncthreads();
  T el[2] = {T(0), T(0)};
  for (int e = threadIdx.x; e < nr * npb; e += kCT) {
    const int r = e / npb;
    T sv = s[e];
    if (s_ok[r]) {
      sv = sv - s_alpha[r] * vs[e];
      s[e] = sv;
    }
    el[r] = fma(sv, sv, el[r]);
  }
  double eta2[2] = {(double)el[0], (double)el[1]};
  bsum<double, 2>(eta2, dsh);
  if (threadIdx.x == 0) {
    for (int r = 0; r < nr; ++r) {
      if (st.done[r]) continue;
      if (!(st.delta[r] > 0.0)) {
        st.done[r] = 1;
        st.not_spd[r] = (st.delta[r] < 0.0) ? 1 : 0;
      } else {
        const double en = eta2[r];
        st.beta[r] = en / st.eta[r];
        st.eta[r] = en;
        st.iters[r] += 1;
        if (en == 0.0 || (st.cg_tol2 > 0.0 && en <= st.cg_tol2 * st.eta0[r])) st.done[r] = 1;
      }
    }
  }
  __syncthreads();
  const T b0 = (T)st.beta[0], b1 = (T)st.beta[1];
  for (int e = threadIdx.x; e < nr * npb; e += kCT) {
    const T pv = s[e] + (e < npb ? b0 : b1) * p[e];
    p[e] = pv;
    ys[e] = pv;
  }
  __syncthreads();
  gemv_upper<T>(W, npb, ys, vs, nr);
  __syncthreads();
  T qp[4] = {T(0), T(0), T(0), T(0)};
  for (int e = threadIdx.x; e < nr * npb; e += kCT) {
    const int r = e / npb, c = e - r * npb;
    const T qv = vs[e] * dv[c];
    q[e] = qv;
    qp[r] = fma(qv, qv, qp[r]);
    qp[2 + r] = fma(ys[e], ys[e], qp[2 + r]);
  }
  double qd[4] = {(double)qp[0], (double)qp[1], (double)qp[2], (double)qp[3]};
  bsum<double, 4>(qd, dsh);
  if (threadIdx.x == 0) {
    st.qq[0] = qd[0];
    st.qq[1] = qd[1];
    st.pp[0] = qd[2];
    st.pp[1] = qd[3];
  }
}

template <typename T>
__global__ void __launch_bounds__(kCT) pcg_post_kernel(BArrays a, const int* list, const int* cnt) {
  const int n = cnt ? *cnt : (int)gridDim.x;
  for (int li = blockIdx.x; li < n; li += gridDim.x) {
    pcg_post_body<T>(a, list[li]);
    __syncthreads();
  }
}

// x_0 = w (the LS solution of the sigma^2 = 0 solve), ||x_0||^2
template <typename T>
__device__ void ls_finish_body(const BArrays& a, const int pi) {
  BState& st = a.st[pi];
  if (!st.active) return;
  const BProb P = a.probs[pi];
  const T* w = PVec::at<T>(a.vw, P);
  __shared__ double dsh[32];
  double xs[1] = {0.0};
  for (int c = threadIdx.x; c < P.npb; c += kCT) {
    const double xn = (c < P.n) ? (double)w[c] : 0.0;
    a.x[P.offV + c] = xn;
    xs[0] = fma(xn, xn, xs[0]);
  }
  bsum<double, 1>(xs, dsh);
  if (threadIdx.x == 0) st.xx = xs[0];
}

template <typename T>
__global__ void __launch_bounds__(kCT) ls_finish_kernel(BArrays a, const int* list, const int* cnt) {
  const int n = cnt ? *cnt : (int)gridDim.x;
  for (int li = blockIdx.x; li < n; li += gridDim.x) {
    ls_finish_body<T>(a, list[li]);
    __syncthreads();
  }
}

// z = x + w_f, beta_k = (z^T f - g) / (z^T x + 1), x = z + beta_k u (Alg. 2), u = w_x
template <typename T>
__device__ void rqi_update_body(const BArrays& a, const int pi) {
  BState& st = a.st[pi];
  if (!st.active) return;
  const BProb P = a.probs[pi];
  const int npb = (int)P.npb, n = (int)P.n;
  const T* w = PVec::at<T>(a.vw, P);
  double* x = a.x + P.offV;
  const double* f = a.f + P.offV;
  __shared__ double dsh[32 * 2];
  double v[2] = {0.0, 0.0};
  for (int c = threadIdx.x; c < n; c += kCT) {
    const double z = x[c] + (double)w[c];
    v[0] = fma(z, f[c], v[0]);
    v[1] = fma(z, x[c], v[1]);
  }
  bsum<double, 2>(v, dsh);
  const double betak = (v[0] - st.g) / (v[1] + 1.0);
  __syncthreads();
  double xs[1] = {0.0};
  for (int c = threadIdx.x; c < npb; c += kCT) {
    double xn = 0.0;
    if (c < n) xn = fma(betak, (double)w[npb + c], x[c] + (double)w[c]);
    x[c] = xn;
    xs[0] = fma(xn, xn, xs[0]);
  }
  bsum<double, 1>(xs, dsh);
  if (threadIdx.x == 0) {
    st.betak = betak;
    st.xx = xs[0];
    st.cg_total += st.iters[0] + st.iters[1];
    st.not_spd_any |= st.not_spd[0] | st.not_spd[1];
  }
}

template <typename T>
__global__ void __launch_bounds__(kCT) rqi_update_kernel(BArrays a, const int* list, const int* cnt) {
  const int n = cnt ? *cnt : (int)gridDim.x;
  for (int li = blockIdx.x; li < n; li += gridDim.x) {
    rqi_update_body<T>(a, list[li]);
    __syncthreads();
  }
}

// Exclusive prefix sum of one int per thread over the CTA (blockDim.x <= 1024); returns the
// thread's offset and writes the CTA total to *total.
__device__ __forceinline__ int block_excl_scan(int v, int* sh, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  __syncthreads();
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = (lane < nw) ? sh[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < nw) sh[lane] = wi - w;       // exclusive offset of each warp
    if (lane == 31) sh[32] = wi;            // total
  }
  __syncthreads();
  const int off = sh[warp] + incl - v;
  *total = sh[32];
  return off;
}

// Active set of the problems in `list`: out[0] = active problems, out[1] = their row tiles,
// out[2..3] = sum of m n over them (one 64-bit count); act_probs / act_tiles receive the
// compacted problem and tile lists the next launches run over. One CTA.
__global__ void __launch_bounds__(1024) count_active_kernel(BArrays a, const int* list, int cnt,
                                                            int* out, int* act_probs,
                                                            int* act_tiles) {
  __shared__ int sh[33];
  __shared__ unsigned long long she[32];
  int base_p = 0, base_t = 0;
  unsigned long long el = 0ull;
  for (int c0 = 0; c0 < cnt; c0 += (int)blockDim.x) {
    const int i = c0 + (int)threadIdx.x;
    int pi = -1, act = 0, nt = 0;
    if (i < cnt) {
      pi = list[i];
      act = a.st[pi].active ? 1 : 0;
      if (act) {
        nt = a.probs[pi].ntiles;
        el += (unsigned long long)(a.probs[pi].m * a.probs[pi].n);
      }
    }
    int tot_p = 0, tot_t = 0;
    const int op = block_excl_scan(act, sh, &tot_p);
    const int ot = block_excl_scan(nt, sh, &tot_t);
    if (act) {
      act_probs[base_p + op] = pi;
      const int t0 = a.probs[pi].tile0;
      for (int t = 0; t < nt; ++t) act_tiles[base_t + ot + t] = t0 + t;
    }
    base_p += tot_p;
    base_t += tot_t;
  }
  el = wsum(el);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) she[threadIdx.x >> 5] = el;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long te = 0ull;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) te += she[w];
    out[0] = base_p;
    out[1] = base_t;
    *reinterpret_cast<unsigned long long*>(out + 2) = te;
  }
}

// -----------------------------------------------------------------------------------------
// Features of the selector network (16 per problem) from the problem data and the factor just
// computed: sizes, the column-norm spread of A, ||b|| / ||A||_F, the spread of diag(R_H), the
// shifts the factorisation needed, ||W||_F and ||W||_2 (power iteration; W = R_H^{-1}, so
// ||W||_2 estimates kappa of the scaled A), and the two constraint values of Sec. 3.1 written
// with these estimates (u_f ||W||_2^2 for the Cholesky route, u_f ||W||_2 for Eq. (5)).
// Normalised in place as (f - mean) / scale when mean / scale are given.
// -----------------------------------------------------------------------------------------
__device__ __forceinline__ double lg(double v) { return log10(fmax(v, 1e-300)); }

template <typename C, typename T>
__global__ void __launch_bounds__(kCT) features_kernel(BArrays a, const int* list,
                                                       const int* nshift, const int* fpiv,
                                                       const int* prec, const double* shift,
                                                       const float* mean, const float* scale,
                                                       float* F) {
  const int pi = list[blockIdx.x];
  // log10 of the unit roundoff of the problem's factor precision (Table 2)
  const int pr = prec[pi];
  const double log10_uf = (pr == 0) ? -11.0 * 0.30102999566398120
                          : (pr == 1) ? -8.0 * 0.30102999566398120
                          : (pr == 2) ? -24.0 * 0.30102999566398120 : -53.0 * 0.30102999566398120;
  const BProb P = a.probs[pi];
  const int n = (int)P.n, npb = (int)P.npb;
  extern __shared__ __align__(16) unsigned char smem[];
  T* ys = reinterpret_cast<T*>(smem);
  T* vs = ys + 2 * kMaxN;
  __shared__ double dsh[32 * 4];
  __shared__ double mx[32 * 2];
  const double* d = a.d + P.offV;
  const C* R = static_cast<const C*>(a.R) + P.offM;
  const T* W = static_cast<const T*>(a.W) + P.offM;
  const T* WT = static_cast<const T*>(a.WT) + P.offM;
  // spreads of d and diag(R_H): max via sums of -min / max through shuffles
  double dmax = 0.0, dmin = 1e300, rmax = 0.0, rmin = 1e300, sums[2] = {0.0, 0.0};
  for (int j = threadIdx.x; j < n; j += kCT) {
    const double dj = d[j], rj = (double)R[(int64_t)j * npb + j];
    dmax = fmax(dmax, dj);
    dmin = fmin(dmin, dj);
    rmax = fmax(rmax, rj);
    rmin = fmin(rmin, rj);
    sums[0] += lg(dj);
  }
  // ||W||_F^2 over the n x n block
  for (int64_t e = threadIdx.x; e < (int64_t)n * npb; e += kCT) {
    const int c = (int)(e % npb);
    if (c < n) {
      const double w = (double)W[e];
      sums[1] = fma(w, w, sums[1]);
    }
  }
  bsum<double, 2>(sums, dsh);
  double ext[4] = {dmax, -dmin, rmax, -rmin};
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ext[k] = fmax(ext[k], __shfl_xor_sync(0xffffffffu, ext[k], o));
    __syncthreads();
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < 4; ++k) dsh[warp * 4 + k] = ext[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double v = (lane < kCW) ? dsh[lane * 4 + k] : -1e300;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
      ext[k] = v;
    }
  }
  // ||W||_2 by power iteration on W^T W (8 steps from the vector of ones)
  for (int j = threadIdx.x; j < npb; j += kCT) ys[j] = (j < n) ? T(1) : T(0);
  double wn = 0.0;
  for (int it = 0; it < 9; ++it) {
    __syncthreads();
    gemv_upper<T>(W, npb, ys, vs, 1);            // y = W v
    __syncthreads();
    double yy[1] = {0.0};
    for (int j = threadIdx.x; j < npb; j += kCT) yy[0] = fma((double)vs[j], (double)vs[j], yy[0]);
    bsum<double, 1>(yy, mx);
    double vv[1] = {0.0};
    for (int j = threadIdx.x; j < npb; j += kCT) vv[0] = fma((double)ys[j], (double)ys[j], vv[0]);
    bsum<double, 1>(vv, mx + 32);
    wn = sqrt(yy[0] / fmax(vv[0], 1e-300));      // ||W v|| / ||v||
    if (it == 8) break;
    __syncthreads();
    gemv_lower<T>(WT, npb, vs, vs + npb, 1);     // z = W^T y
    __syncthreads();
    double zz[1] = {0.0};
    for (int j = threadIdx.x; j < npb; j += kCT) zz[0] = fma((double)vs[npb + j], (double)vs[npb + j], zz[0]);
    bsum<double, 1>(zz, mx);
    const double inv = 1.0 / sqrt(fmax(zz[0], 1e-300));
    for (int j = threadIdx.x; j < npb; j += kCT) ys[j] = (T)((double)vs[npb + j] * inv);
  }
  if (threadIdx.x == 0) {
    const BState& st = a.st[pi];
    float f[16];
    const double lw2 = lg(wn), lwf = 0.5 * lg(sums[1]);
    f[0] = (float)lg((double)P.m);
    f[1] = (float)lg((double)n);
    f[2] = (float)lg((double)P.m / (double)n);
    f[3] = (float)(lg(ext[0]) - lg(-ext[1]));
    f[4] = (float)(sums[0] / n - lg(ext[0]));
    f[5] = (float)(0.5 * (lg(st.norm2_b) - lg(st.norm2_A)));
    f[6] = (float)(lg(ext[2]) - lg(-ext[3]));
    f[7] = (float)lg(-ext[3]);
    f[8] = (float)nshift[pi];
    f[9] = (float)lg(1.0 + shift[pi] / pow(10.0, log10_uf));
    f[10] = (float)lwf;
    f[11] = (float)lw2;
    f[12] = (float)(lwf - lw2);
    f[13] = (float)(log10_uf + 2.0 * lw2);
    f[14] = (float)(log10_uf + lw2);
    f[15] = (fpiv[pi] >= 0) ? (float)fpiv[pi] / (float)n : 0.f;
    for (int k = 0; k < 16; ++k) {
      float v = f[k];
      if (mean && scale) v = (v - mean[k]) / scale[k];
      F[(int64_t)pi * 16 + k] = v;
    }
  }
}

template <typename K>
void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------------
void launch_pass_colnorm(const BArrays& a, int ntiles, cudaStream_t s) {
  if (ntiles <= 0) return;
  constexpr size_t sm = pass_smem<double, 1>();
  static const bool once = [] { set_smem(pass_kernel<double, 1, kColnorm>, sm); return true; }();
  (void)once;
  pass_kernel<double, 1, kColnorm><<<ntiles, kPT, sm, s>>>(a, nullptr, nullptr);
  count_launch();
}

void launch_colnorm_post(const BArrays& a, const int* list, int cnt, cudaStream_t s) {
  if (cnt <= 0) return;
  colnorm_post_kernel<<<cnt, kCT, 0, s>>>(a, list);
  count_launch();
}

void launch_pass_resid_df(const BArrays& a, const int* tlist, const int* ntile, int grid,
                          cudaStream_t s) {
  if (grid <= 0) return;
  constexpr size_t sm = pass_smem<double, 1>();
  static const bool once = [] { set_smem(pass_kernel<float, 1, kResidDf>, sm); return true; }();
  (void)once;
  pass_kernel<float, 1, kResidDf><<<grid, kPT, sm, s>>>(a, tlist, ntile);
  count_launch();
}

void launch_pass_resid(const BArrays& a, const int* tlist, const int* ntile, int grid,
                       cudaStream_t s) {
  if (grid <= 0) return;
  constexpr size_t sm = pass_smem<double, 1>();
  static const bool once = [] { set_smem(pass_kernel<double, 1, kResid>, sm); return true; }();
  (void)once;
  pass_kernel<double, 1, kResid><<<grid, kPT, sm, s>>>(a, tlist, ntile);
  count_launch();
}

template <typename T>
void launch_pass_pcg(const BArrays& a, const int* tlist, const int* ntile, int grid, int nr,
                     cudaStream_t s) {
  if (grid <= 0) return;
  if (nr == 2) {
    constexpr size_t sm = pass_smem<T, 2>();
    static const bool once = [] { set_smem(pass_kernel<T, 2, kPcg>, sm); return true; }();
    (void)once;
    pass_kernel<T, 2, kPcg><<<grid, kPT, sm, s>>>(a, tlist, ntile);
  } else {
    constexpr size_t sm = pass_smem<T, 1>();
    static const bool once = [] { set_smem(pass_kernel<T, 1, kPcg>, sm); return true; }();
    (void)once;
    pass_kernel<T, 1, kPcg><<<grid, kPT, sm, s>>>(a, tlist, ntile);
  }
  count_launch();
}

template <typename C>
void launch_gram(const BArrays& a, const GTile* gtiles, int ngt, const GTile* groups, int ngr,
                 void* work, cudaStream_t s) {
  if (ngt > 0) {
    gram_kernel<C><<<ngt, 64, 0, s>>>(a, gtiles, static_cast<C*>(work));
    count_launch();
  }
  if (ngr > 0) {
    gram_reduce_kernel<C><<<ngr, 256, 0, s>>>(a, groups, static_cast<const C*>(work));
    count_launch();
  }
}

template <typename C>
void launch_chol(const BArrays& a, const int* list, int cnt, const double* shift, int* info,
                 const CTask* tasks, const int* off, int steps, cudaStream_t s) {
  if (cnt <= 0) return;
  constexpr size_t sm_diag = sizeof(C) * 3 * kNB * kLd;
  constexpr size_t sm_tile = sizeof(C) * 2 * kNB * kLd;
  static const bool once = [] {
    set_smem(chol_diag_kernel<C>, sm_diag);
    set_smem(chol_tile_kernel<C, true>, sm_tile);
    set_smem(chol_tile_kernel<C, false>, sm_tile);
    return true;
  }();
  (void)once;
  chol_init_kernel<C><<<dim3(cnt, 8), 256, 0, s>>>(a, list, shift, info);
  count_launch();
  // off[3 s + 0 .. 2]: starts of the diagonal, panel and trailing lists of step s; off[3 steps]
  // the end of the last list
  for (int st = 0; st < steps; ++st) {
    const int d0 = off[3 * st], p0 = off[3 * st + 1], u0 = off[3 * st + 2], e = off[3 * st + 3];
    if (p0 > d0) { chol_diag_kernel<C><<<p0 - d0, 256, sm_diag, s>>>(a, tasks + d0, info); count_launch(); }
    if (u0 > p0) { chol_tile_kernel<C, true><<<u0 - p0, 256, sm_tile, s>>>(a, tasks + p0, info); count_launch(); }
    if (e > u0) { chol_tile_kernel<C, false><<<e - u0, 256, sm_tile, s>>>(a, tasks + u0, info); count_launch(); }
  }
  chol_final_kernel<C><<<dim3(cnt, 8), 256, 0, s>>>(a, list, info);
  count_launch();
}

template <typename C, typename T>
void launch_trtri(const BArrays& a, const CTask* tasks, const int* off, int levels,
                  cudaStream_t s) {
  constexpr size_t sm = sizeof(T) * 3 * kNB * kLd;
  static const bool once = [] { set_smem(trtri_tile_kernel<C, T>, sm); return true; }();
  (void)once;
  for (int l = 0; l < levels; ++l) {
    const int n = off[l + 1] - off[l];
    if (n > 0) { trtri_tile_kernel<C, T><<<n, 256, sm, s>>>(a, tasks + off[l]); count_launch(); }
  }
}

template <typename T>
void launch_solve_init(const BArrays& a, const int* list, int cnt, cudaStream_t s) {
  if (cnt <= 0) return;
  solve_init_kernel<T><<<cnt, kCT, 0, s>>>(a, list);
  count_launch();
}

template <typename T>
void launch_resid_post(const BArrays& a, const int* list, const int* cnt, int grid, int mode,
                       const SolveParams& sp, cudaStream_t s) {
  if (grid <= 0) return;
  constexpr size_t sm = post_smem<T>() + sizeof(double) * kMaxN;
  static const bool once = [] { set_smem(resid_post_kernel<T>, sm); return true; }();
  (void)once;
  resid_post_kernel<T><<<grid, kCT, sm, s>>>(a, list, cnt, mode, sp);
  count_launch();
}

template <typename T>
void launch_pcg_post(const BArrays& a, const int* list, const int* cnt, int grid, cudaStream_t s) {
  if (grid <= 0) return;
  constexpr size_t sm = post_smem<T>();
  static const bool once = [] { set_smem(pcg_post_kernel<T>, sm); return true; }();
  (void)once;
  pcg_post_kernel<T><<<grid, kCT, sm, s>>>(a, list, cnt);
  count_launch();
}

template <typename T>
void launch_ls_finish(const BArrays& a, const int* list, const int* cnt, int grid,
                      cudaStream_t s) {
  if (grid <= 0) return;
  ls_finish_kernel<T><<<grid, kCT, 0, s>>>(a, list, cnt);
  count_launch();
}

template <typename T>
void launch_rqi_update(const BArrays& a, const int* list, const int* cnt, int grid,
                       cudaStream_t s) {
  if (grid <= 0) return;
  rqi_update_kernel<T><<<grid, kCT, 0, s>>>(a, list, cnt);
  count_launch();
}

template <typename C, typename T>
void launch_features(const BArrays& a, const int* list, int cnt, const int* nshift,
                     const int* fpiv, const int* prec, const double* shift, const float* mean,
                     const float* scale, float* F, cudaStream_t s) {
  if (cnt <= 0) return;
  constexpr size_t sm = post_smem<T>();
  static const bool once = [] { set_smem(features_kernel<C, T>, sm); return true; }();
  (void)once;
  features_kernel<C, T><<<cnt, kCT, sm, s>>>(a, list, nshift, fpiv, prec, shift, mean, scale, F);
  count_launch();
}
template void launch_features<float, float>(const BArrays&, const int*, int, const int*, const int*,
    const int*, const double*, const float*, const float*, float*, cudaStream_t);
template void launch_features<double, float>(const BArrays&, const int*, int, const int*, const int*,
    const int*, const double*, const float*, const float*, float*, cudaStream_t);
template void launch_features<float, double>(const BArrays&, const int*, int, const int*, const int*,
    const int*, const double*, const float*, const float*, float*, cudaStream_t);
template void launch_features<double, double>(const BArrays&, const int*, int, const int*, const int*,
    const int*, const double*, const float*, const float*, float*, cudaStream_t);

void launch_count_active(const BArrays& a, const int* list, int cnt, int* out, int* act_probs,
                         int* act_tiles, cudaStream_t s) {
  count_active_kernel<<<1, 1024, 0, s>>>(a, list, cnt, out, act_probs, act_tiles);
  count_launch();
}

namespace {
// grid (X, njobs): the warps of the X CTAs of job j take its rows in turn; a row is read and
// written with consecutive lanes on consecutive columns.
__global__ void __launch_bounds__(256) repack_kernel(double* __restrict__ A64,
                                                     const RepackJob* __restrict__ jobs,
                                                     int* __restrict__ bad) {
  const RepackJob J = jobs[blockIdx.y];
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int64_t ws = (int64_t)gridDim.x * 8;
  bool err = false;
  for (int64_t i = w0; i < J.m; i += ws) {
    const double* src = J.src + i * J.src_ld;
    double* dst = A64 + J.dst + i * J.lda;
    for (int64_t c = lane; c < J.n; c += 32) {
      const double v = src[c];
      err |= !isfinite(v);
      dst[c] = v;
    }
  }
  if (__syncthreads_or(err) && threadIdx.x == 0) atomicOr(bad, 1);
}
}  // namespace

void launch_repack(double* A64, const RepackJob* jobs, int njobs, int* bad, int num_sms,
                   cudaStream_t s) {
  for (int j0 = 0; j0 < njobs; j0 += 65535) {
    const int nj = std::min(65535, njobs - j0);
    const int X = std::max(1, (4 * num_sms + nj - 1) / nj);
    repack_kernel<<<dim3((unsigned)X, (unsigned)nj), 256, 0, s>>>(A64, jobs + j0, bad);
    count_launch();
  }
}

template void launch_pass_pcg<float>(const BArrays&, const int*, const int*, int, int, cudaStream_t);
template void launch_pass_pcg<double>(const BArrays&, const int*, const int*, int, int, cudaStream_t);
template void launch_gram<float>(const BArrays&, const GTile*, int, const GTile*, int, void*,
                                 cudaStream_t);
template void launch_gram<double>(const BArrays&, const GTile*, int, const GTile*, int, void*,
                                  cudaStream_t);
template void launch_chol<float>(const BArrays&, const int*, int, const double*, int*,
                                 const CTask*, const int*, int, cudaStream_t);
template void launch_chol<double>(const BArrays&, const int*, int, const double*, int*,
                                  const CTask*, const int*, int, cudaStream_t);
template void launch_trtri<float, float>(const BArrays&, const CTask*, const int*, int, cudaStream_t);
template void launch_trtri<double, float>(const BArrays&, const CTask*, const int*, int, cudaStream_t);
template void launch_trtri<double, double>(const BArrays&, const CTask*, const int*, int, cudaStream_t);
template void launch_trtri<float, double>(const BArrays&, const CTask*, const int*, int, cudaStream_t);
#define TLS_BI(T)                                                                                 \
  template void launch_solve_init<T>(const BArrays&, const int*, int, cudaStream_t);              \
  template void launch_resid_post<T>(const BArrays&, const int*, const int*, int, int,             \
                                     const SolveParams&, cudaStream_t);                           \
  template void launch_pcg_post<T>(const BArrays&, const int*, const int*, int, cudaStream_t);    \
  template void launch_ls_finish<T>(const BArrays&, const int*, const int*, int, cudaStream_t);   \
  template void launch_rqi_update<T>(const BArrays&, const int*, const int*, int, cudaStream_t);
TLS_BI(float)
TLS_BI(double)
#undef TLS_BI

}  // namespace bat
}  // namespace tls
