// Preconditioner construction (Sec. 3.1 of Oktay & Carson, arXiv 2305.19028): column scaling
// D = diag(||a_j||), the Gram matrix H = (A D^{-1})^T (A D^{-1}) of the u_f-rounded scaled
// matrix, blocked Cholesky H + sI = R_H^T R_H, rounding of R_H to u_f, and the explicit inverse
// W = R_H^{-1} that the PCGTLS iteration applies as two triangular products per step.
#include "tls_internal.h"
#include "tls_device.cuh"
#include "tls_ptx.cuh"
#include "tls_tc.cuh"
#include "chol64.cuh"

#include <algorithm>
#include <type_traits>

namespace tls {

namespace {

// Two FP32 fused multiply-adds in one instruction (the packed f32x2 form of sm_100 and later):
// c.lo = fma(a.lo, b.lo, c.lo), c.hi = fma(a.hi, b.hi, c.hi), each rounded to nearest like
// fmaf; halves the FMA issue slots of the 8 x 8-per-thread GEMM tile (measured faster there; in
// the 4 x 4-per-thread tile the packing of the broadcast operand cost more than it saved).
__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
  return ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
__device__ __forceinline__ void ffma2(unsigned long long& c, unsigned long long a,
                                      unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(c) : "l"(a), "l"(b));
}
__device__ __forceinline__ float lo2(unsigned long long v) { return __uint_as_float((unsigned)(v & 0xffffffffull)); }
__device__ __forceinline__ float hi2(unsigned long long v) { return __uint_as_float((unsigned)(v >> 32)); }

__device__ __forceinline__ float load_f(const __half* p) { return __half2float(*p); }
__device__ __forceinline__ float load_f(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float load_f(const float* p) { return *p; }
__device__ __forceinline__ double load_f(const double* p) { return *p; }

// ---------------------------------------------------------------------------------------
// Column norms (and the FP32 copy of A for the PCGTLS pass)
// grid (ceil(npad/256), P); each CTA: 256 columns x a chunk of rows.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) colnorm_kernel(const double* __restrict__ A, int64_t lda,
                                                      int64_t m, int64_t n, int64_t npad,
                                                      float* __restrict__ A32,
                                                      float* __restrict__ Alo, int64_t ldo,
                                                      double* __restrict__ part) {
  const int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const int64_t rows_per = (m + gridDim.y - 1) / gridDim.y;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per;
  const int64_t r1 = min(m, r0 + rows_per);
  if (c >= npad) return;
  constexpr int U = 8;   // rows in flight per thread
  if (A32 != nullptr) {
    // the FP32 path: the norm is accumulated in FP32 from the FP32-rounded entries
    float acc = 0.f;
    for (int64_t i0 = r0; i0 < r1; i0 += U) {
      double v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = (c < n && i0 + u < r1) ? __ldcs(A + (i0 + u) * lda + c) : 0.0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        float f, lo;
        if (Alo != nullptr) {
          f64_split_f32(v[u], f, lo);
          if (i0 + u < r1) Alo[(i0 + u) * ldo + c] = lo;
        } else {
          f = f64_to_f32_rn(v[u]);
        }
        if (i0 + u < r1) A32[(i0 + u) * ldo + c] = f;
        acc = fmaf(f, f, acc);
      }
    }
    part[(int64_t)blockIdx.y * npad + c] = (double)acc;
  } else {
    double acc = 0.0;
    for (int64_t i0 = r0; i0 < r1; i0 += U) {
      double v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = (c < n && i0 + u < r1) ? __ldcs(A + (i0 + u) * lda + c) : 0.0;
#pragma unroll
      for (int u = 0; u < U; ++u) acc = fma(v[u], v[u], acc);
    }
    part[(int64_t)blockIdx.y * npad + c] = acc;
  }
}

__global__ void colnorm_finish_kernel(const double* __restrict__ part, int P, int64_t n,
                                      int64_t npad, double* __restrict__ d,
                                      float* __restrict__ dinv32, double* __restrict__ dinv64) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= npad) return;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int p = 0;
  for (; p + 3 < P; p += 4) {
    s0 += part[(int64_t)p * npad + c];
    s1 += part[(int64_t)(p + 1) * npad + c];
    s2 += part[(int64_t)(p + 2) * npad + c];
    s3 += part[(int64_t)(p + 3) * npad + c];
  }
  for (; p < P; ++p) s0 += part[(int64_t)p * npad + c];
  double dd = sqrt((s0 + s1) + (s2 + s3));
  // padded (and all-zero) columns get d = 1 so that D stays invertible; a zero column makes
  // A^T A singular and shows up as a Cholesky breakdown.
  if (c >= n || !(dd > 0.0)) dd = 1.0;
  if (d) d[c] = dd;
  if (dinv32) dinv32[c] = (float)(1.0 / dd);
  if (dinv64) dinv64[c] = 1.0 / dd;
}

// ---------------------------------------------------------------------------------------
// AsT[j][i] = fl(A[i][j] / d_j): scaled, rounded and transposed (n x mpad), via 32x32 tiles (FP64
// input) or 64x64 tiles (the FP32 working copy)
// ---------------------------------------------------------------------------------------
template <typename Tout> __device__ __forceinline__ Tout cvt_out(double v);
template <> __device__ __forceinline__ __half cvt_out<__half>(double v) { return __double2half(v); }
template <> __device__ __forceinline__ __nv_bfloat16 cvt_out<__nv_bfloat16>(double v) {
  return __double2bfloat16(v);
}
template <> __device__ __forceinline__ float cvt_out<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ double cvt_out<double>(double v) { return v; }

template <typename Tout> __device__ __forceinline__ Tout cvt_out_f(float v);
template <> __device__ __forceinline__ __half cvt_out_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 cvt_out_f<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

// two neighbouring entries of a row of A_s^T as one packed store (the pair starts at an even
// column of an even-length row, so it is aligned to its own size)
template <typename Tout> __device__ __forceinline__ void store_pair(Tout* p, float a, float b);
template <> __device__ __forceinline__ void store_pair<__half>(__half* p, float a, float b) {
  *reinterpret_cast<__half2*>(p) = __halves2half2(__float2half_rn(a), __float2half_rn(b));
}
template <> __device__ __forceinline__ void store_pair<__nv_bfloat16>(__nv_bfloat16* p, float a,
                                                                      float b) {
  *reinterpret_cast<__nv_bfloat162*>(p) =
      __halves2bfloat162(__float2bfloat16_rn(a), __float2bfloat16_rn(b));
}
template <> __device__ __forceinline__ void store_pair<float>(float* p, float a, float b) {
  *reinterpret_cast<float2*>(p) = make_float2(a, b);
}

// FP32 input (the working copy of A): A_s = fl(fl32(A32 * dinv32)), all in FP32 arithmetic.
// 64 x 64 tiles, 256 threads: warp w reads rows 8w..8w+7 of the tile, each lane two
// neighbouring columns per row (all eight loads of a thread issued before the first is used),
// and writes rows 8w..8w+7 of the transposed tile, each lane two neighbouring entries as one
// packed word. m_pad and n_pad are multiples of 64, lda is even.
template <typename Tout>
__global__ void __launch_bounds__(256) scale_cast_T32_kernel(
    const float* __restrict__ A, int64_t lda, int64_t m, int64_t n, int64_t npad, int64_t mpad,
    const float* __restrict__ dinv, Tout* __restrict__ AsT) {
  __shared__ float tile[64][65];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * 64;   // rows of A (columns of AsT)
  const int64_t j0 = (int64_t)blockIdx.y * 64;   // columns of A (rows of AsT)
  const int64_t j = j0 + 2 * lane;
  const bool c0 = j < n, c1 = j + 1 < n;
  const float d0 = c0 ? dinv[j] : 0.f, d1 = c1 ? dinv[j + 1] : 0.f;
  float2 a[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int64_t i = i0 + warp * 8 + t;
    a[t] = (i < m && c0) ? *reinterpret_cast<const float2*>(A + i * lda + j)
                         : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int r = warp * 8 + t;
    const bool row = i0 + r < m;
    tile[r][2 * lane] = (row && c0) ? a[t].x * d0 : 0.f;
    tile[r][2 * lane + 1] = (row && c1) ? a[t].y * d1 : 0.f;
  }
  __syncthreads();
  const int64_t i = i0 + 2 * lane;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int c = warp * 8 + t;
    store_pair<Tout>(AsT + (j0 + c) * mpad + i, tile[2 * lane][c], tile[2 * lane + 1][c]);
  }
}

template <typename Tin, typename Tout>
__global__ void scale_cast_T_kernel(const Tin* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                                    int64_t npad, int64_t mpad, const double* __restrict__ dinv,
                                    Tout* __restrict__ AsT) {
  __shared__ double tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;   // rows of A (columns of AsT)
  const int64_t j0 = (int64_t)blockIdx.y * 32;   // columns of A (rows of AsT)
  for (int r = threadIdx.y; r < 32; r += 8) {
    int64_t i = i0 + r, j = j0 + threadIdx.x;
    double v = 0.0;
    if (i < m && j < n) v = (double)A[i * lda + j] * dinv[j];
    tile[r][threadIdx.x] = v;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    int64_t j = j0 + r, i = i0 + threadIdx.x;
    if (j < npad && i < mpad) AsT[j * mpad + i] = cvt_out<Tout>(tile[threadIdx.x][r]);
  }
}

// ---------------------------------------------------------------------------------------
// Generic tiled SIMT GEMM, C = alpha * op(A) op(B) + beta * C, 64 x 64 tiles, BK = 16,
// 256 threads with a 4 x 4 register tile each. Layouts:
//   AK: A(i,k) = A[i*lda + k]   else A(i,k) = A[k*lda + i]
//   BK: B(k,j) = B[j*ldb + k]   else B(k,j) = B[k*ldb + j]
// upper: only tiles with tile_row <= tile_col are computed; mirror: write C[j][i] too.
// blockIdx.z selects a batch entry through the strides.
// ---------------------------------------------------------------------------------------
template <typename Tin, typename Tc, bool AK, bool BKM>
__global__ void __launch_bounds__(256) gemm_simt_kernel(
    int M, int N, int K, const Tin* __restrict__ A, int64_t lda, int64_t sA,
    const Tin* __restrict__ B, int64_t ldb, int64_t sB, Tc* __restrict__ C, int64_t ldc,
    int64_t sC, Tc alpha, Tc beta, int upper, int mirror, const int* skip) {
  constexpr int BM = 64, BN = 64, BKT = 16;
  if (skip != nullptr && *(volatile const int*)skip != 0) return;
  __shared__ Tc As[BKT][BM + 4];
  __shared__ Tc Bs[BKT][BN + 4];
  const int tile_i = blockIdx.y, tile_j = blockIdx.x;
  if (upper && tile_i > tile_j) return;
  A += (int64_t)blockIdx.z * sA;
  B += (int64_t)blockIdx.z * sB;
  C += (int64_t)blockIdx.z * sC;
  const int i0 = tile_i * BM, j0 = tile_j * BN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  Tc acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = Tc(0);
  for (int k0 = 0; k0 < K; k0 += BKT) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      int e = tid + 256 * l;
      int r, kk;
      if (AK) { r = e / BKT; kk = e % BKT; } else { r = e % BM; kk = e / BM; }
      int gi = i0 + r, gk = k0 + kk;
      Tc v = Tc(0);
      if (gi < M && gk < K) v = (Tc)load_f(AK ? (A + (int64_t)gi * lda + gk) : (A + (int64_t)gk * lda + gi));
      As[kk][r] = v;
      int c, kb;
      if (BKM) { c = e / BKT; kb = e % BKT; } else { c = e % BN; kb = e / BN; }
      int gj = j0 + c, gk2 = k0 + kb;
      Tc w = Tc(0);
      if (gj < N && gk2 < K) w = (Tc)load_f(BKM ? (B + (int64_t)gj * ldb + gk2) : (B + (int64_t)gk2 * ldb + gj));
      Bs[kb][c] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BKT; ++kk) {
      Tc a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = As[kk][ty + 16 * q]; b[q] = Bs[kk][tx + 16 * q]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int gi = i0 + ty + 16 * p, gj = j0 + tx + 16 * q;
      if (gi < M && gj < N) {
        if (upper && gi > gj) continue;
        Tc* cp = C + (int64_t)gi * ldc + gj;
        Tc v = alpha * acc[p][q];
        if (beta != Tc(0)) v += beta * (*cp);
        *cp = v;
        if (mirror && gi != gj) C[(int64_t)gj * ldc + gi] = v;
      }
    }
}

// ---------------------------------------------------------------------------------------
// FP32 SIMT GEMM for the larger products of the factor (trailing updates, the inverse by
// doubling, the FP32 Gram): 128 x 128 tiles, BK = 8, 256 threads with an 8 x 8 register tile
// each (two 4-row and two 4-column strips, read from shared memory as float4), the next k-slab
// prefetched into registers while the current one is used (one barrier per slab).
// Same layouts and flags as gemm_simt_kernel; in addition
//   kfrom_i: 1: the k range of a tile row block starts at i0 (A upper triangular: A(i,k) = 0,
//            k < i); 2: the k range of a tile starts at j0 (B(k,j) = 0 for k < j)
//   kto_j:   the k range of a tile column block ends at j0 + 128 (B upper triangular).
// Requires M, N multiples of 4, K a multiple of 8, lda, ldb multiples of 4 and 16-byte aligned
// A, B (the dispatcher checks).
// ---------------------------------------------------------------------------------------
template <bool AK, bool BKM>
__device__ __forceinline__ void gemm_big_tile(
    int M, int N, int K, const float* __restrict__ A, int64_t lda, const float* __restrict__ B,
    int64_t ldb, float* __restrict__ C, int64_t ldc, float alpha, float beta, int upper,
    int mirror, int kfrom_i, int kto_j, int tile_i, int tile_j) {
  constexpr int BM = 128, BN = 128, BK = 8;
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];
  const int i0 = tile_i * BM, j0 = tile_j * BN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  int k_lo = (kfrom_i == 1) ? (i0 / BK) * BK : (kfrom_i == 2 ? (j0 / BK) * BK : 0);
  int k_hi = kto_j ? min(K, j0 + BN) : K;
  if (k_lo > K) k_lo = K;
  // global -> register slab loader: one float4 of A and one of B per thread
  // A: AK: row i = tid / 2, k = (tid & 1) * 4 (contiguous in k); else k = tid / 32, i = (tid & 31) * 4
  // B: BKM: col j = tid / 2, k = (tid & 1) * 4; else k = tid / 32, j = (tid & 31) * 4
  const int a_r = AK ? (tid >> 1) : ((tid & 31) * 4);
  const int a_k = AK ? ((tid & 1) * 4) : (tid >> 5);
  const int b_c = BKM ? (tid >> 1) : ((tid & 31) * 4);
  const int b_k = BKM ? ((tid & 1) * 4) : (tid >> 5);
  auto load_a = [&](int k0) -> float4 {
    const int gi = i0 + a_r, gk = k0 + a_k;
    if (AK) {
      if (gi < M && gk < K) return *reinterpret_cast<const float4*>(A + (int64_t)gi * lda + gk);
    } else {
      if (gi < M && gk < K) return *reinterpret_cast<const float4*>(A + (int64_t)gk * lda + gi);
    }
    return make_float4(0.f, 0.f, 0.f, 0.f);
  };
  auto load_b = [&](int k0) -> float4 {
    const int gj = j0 + b_c, gk = k0 + b_k;
    if (BKM) {
      if (gj < N && gk < K) return *reinterpret_cast<const float4*>(B + (int64_t)gj * ldb + gk);
    } else {
      if (gj < N && gk < K) return *reinterpret_cast<const float4*>(B + (int64_t)gk * ldb + gj);
    }
    return make_float4(0.f, 0.f, 0.f, 0.f);
  };
  auto store = [&](int buf, const float4& va, const float4& vb) {
    if (AK) {
      As[buf][a_k + 0][a_r] = va.x;
      As[buf][a_k + 1][a_r] = va.y;
      As[buf][a_k + 2][a_r] = va.z;
      As[buf][a_k + 3][a_r] = va.w;
    } else {
      *reinterpret_cast<float4*>(&As[buf][a_k][a_r]) = va;
    }
    if (BKM) {
      Bs[buf][b_k + 0][b_c] = vb.x;
      Bs[buf][b_k + 1][b_c] = vb.y;
      Bs[buf][b_k + 2][b_c] = vb.z;
      Bs[buf][b_k + 3][b_c] = vb.w;
    } else {
      *reinterpret_cast<float4*>(&Bs[buf][b_k][b_c]) = vb;
    }
  };
  unsigned long long acc2[8][4];   // packed pairs: columns 2q, 2q + 1 of the thread's row p
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc2[a][b] = 0ull;
  if (k_lo < k_hi) {
    float4 va = load_a(k_lo), vb = load_b(k_lo);
    store(0, va, vb);
    __syncthreads();
    int buf = 0;
    for (int k0 = k_lo; k0 < k_hi; k0 += BK) {
      const bool more = k0 + BK < k_hi;
      if (more) {
        va = load_a(k0 + BK);
        vb = load_b(k0 + BK);
      }
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
        const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const unsigned long long bp[4] = {pk2(b0.x, b0.y), pk2(b0.z, b0.w), pk2(b1.x, b1.y),
                                          pk2(b1.z, b1.w)};
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          const unsigned long long ap = pk2(av[p], av[p]);
#pragma unroll
          for (int q = 0; q < 4; ++q) ffma2(acc2[p][q], ap, bp[q]);
        }
      }
      if (more) {
        store(buf ^ 1, va, vb);
        __syncthreads();
        buf ^= 1;
      }
    }
  }
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    const int gi = i0 + (p < 4 ? ty * 4 + p : 64 + ty * 4 + p - 4);
    if (gi >= M) continue;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int gj = j0 + (q < 4 ? tx * 4 + q : 64 + tx * 4 + q - 4);
      if (gj >= N || (upper && gi > gj)) continue;
      float* cp = C + (int64_t)gi * ldc + gj;
      const float a = (q & 1) ? hi2(acc2[p][q >> 1]) : lo2(acc2[p][q >> 1]);
      float v = alpha * a;
      if (beta != 0.f) v += beta * (*cp);
      *cp = v;
      if (mirror && gi != gj) C[(int64_t)gj * ldc + gi] = v;
    }
  }
}

template <bool AK, bool BKM>
__global__ void __launch_bounds__(256, 2) gemm_big_kernel(
    int M, int N, int K, const float* __restrict__ A, int64_t lda, int64_t sA,
    const float* __restrict__ B, int64_t ldb, int64_t sB, float* __restrict__ C, int64_t ldc,
    int64_t sC, float alpha, float beta, int upper, int mirror, int kfrom_i, int kto_j,
    const int* skip) {
  if (skip != nullptr && *(volatile const int*)skip != 0) return;
  const int tile_i = blockIdx.y, tile_j = blockIdx.x;
  if (upper && tile_i > tile_j) return;
  gemm_big_tile<AK, BKM>(M, N, K, A + (int64_t)blockIdx.z * sA, lda, B + (int64_t)blockIdx.z * sB,
                         ldb, C + (int64_t)blockIdx.z * sC, ldc, alpha, beta, upper, mirror,
                         kfrom_i, kto_j, tile_i, tile_j);
}

// FP32 64 x 64-tile variant of the same product for grids too small for 128 x 128 tiles (or K
// too short to amortise them): BK = 16, 256 threads with a 4 x 4 register tile each, operands
// read from shared memory as float4, the next k-slab prefetched into registers (one barrier per
// slab). Same requirements as gemm_big_kernel, K a multiple of 16.
template <bool AK, bool BKM>
__device__ __forceinline__ void gemm_mid_tile(
    int M, int N, int K, const float* __restrict__ A, int64_t lda, const float* __restrict__ B,
    int64_t ldb, float* __restrict__ C, int64_t ldc, float alpha, float beta, int upper,
    int mirror, int kfrom_i, int kto_j, int tile_i, int tile_j, int kc_lo = 0,
    int kc_hi = 1 << 30) {
  constexpr int BM = 64, BN = 64, BK = 16, LD = 68;
  __shared__ __align__(16) float As[2][BK][LD];
  __shared__ __align__(16) float Bs[2][BK][LD];
  const int i0 = tile_i * BM, j0 = tile_j * BN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  int k_lo = (kfrom_i == 1) ? (i0 / BK) * BK : (kfrom_i == 2 ? (j0 / BK) * BK : 0);
  const int k_hi = min(kto_j ? min(K, j0 + BN) : K, kc_hi);   // (kc_*: one chunk of a split k)
  k_lo = max(k_lo, kc_lo);
  if (k_lo > K) k_lo = K;
  // A: AK: row i = tid / 4, k = (tid & 3) * 4; else k = tid / 16, i = (tid & 15) * 4
  const int a_r = AK ? (tid >> 2) : ((tid & 15) * 4);
  const int a_k = AK ? ((tid & 3) * 4) : (tid >> 4);
  const int b_c = BKM ? (tid >> 2) : ((tid & 15) * 4);
  const int b_k = BKM ? ((tid & 3) * 4) : (tid >> 4);
  auto load_a = [&](int k0) -> float4 {
    const int gi = i0 + a_r, gk = k0 + a_k;
    if (gi < M && gk < K)
      return *reinterpret_cast<const float4*>(AK ? (A + (int64_t)gi * lda + gk)
                                                 : (A + (int64_t)gk * lda + gi));
    return make_float4(0.f, 0.f, 0.f, 0.f);
  };
  auto load_b = [&](int k0) -> float4 {
    const int gj = j0 + b_c, gk = k0 + b_k;
    if (gj < N && gk < K)
      return *reinterpret_cast<const float4*>(BKM ? (B + (int64_t)gj * ldb + gk)
                                                  : (B + (int64_t)gk * ldb + gj));
    return make_float4(0.f, 0.f, 0.f, 0.f);
  };
  auto store = [&](int buf, const float4& va, const float4& vb) {
    if (AK) {
      As[buf][a_k + 0][a_r] = va.x;
      As[buf][a_k + 1][a_r] = va.y;
      As[buf][a_k + 2][a_r] = va.z;
      As[buf][a_k + 3][a_r] = va.w;
    } else {
      *reinterpret_cast<float4*>(&As[buf][a_k][a_r]) = va;
    }
    if (BKM) {
      Bs[buf][b_k + 0][b_c] = vb.x;
      Bs[buf][b_k + 1][b_c] = vb.y;
      Bs[buf][b_k + 2][b_c] = vb.z;
      Bs[buf][b_k + 3][b_c] = vb.w;
    } else {
      *reinterpret_cast<float4*>(&Bs[buf][b_k][b_c]) = vb;
    }
  };
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  if (k_lo < k_hi) {
    float4 va = load_a(k_lo), vb = load_b(k_lo);
    store(0, va, vb);
    __syncthreads();
    int buf = 0;
    for (int k0 = k_lo; k0 < k_hi; k0 += BK) {
      const bool more = k0 + BK < k_hi;
      if (more) {
        va = load_a(k0 + BK);
        vb = load_b(k0 + BK);
      }
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        const float4 a4 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
        const float4 b4 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
        const float av[4] = {a4.x, a4.y, a4.z, a4.w};
        const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(av[p], bv[q], acc[p][q]);
      }
      if (more) {
        store(buf ^ 1, va, vb);
        __syncthreads();
        buf ^= 1;
      }
    }
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int gi = i0 + ty * 4 + p;
    if (gi >= M) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gj = j0 + tx * 4 + q;
      if (gj >= N || (upper && gi > gj)) continue;
      float* cp = C + (int64_t)gi * ldc + gj;
      float v = alpha * acc[p][q];
      if (beta != 0.f) v += beta * (*cp);
      *cp = v;
      if (mirror && gi != gj) C[(int64_t)gj * ldc + gi] = v;
    }
  }
}

template <bool AK, bool BKM>
__global__ void __launch_bounds__(256) gemm_mid_kernel(
    int M, int N, int K, const float* __restrict__ A, int64_t lda, int64_t sA,
    const float* __restrict__ B, int64_t ldb, int64_t sB, float* __restrict__ C, int64_t ldc,
    int64_t sC, float alpha, float beta, int upper, int mirror, int kfrom_i, int kto_j,
    const int* skip) {
  if (skip != nullptr && *(volatile const int*)skip != 0) return;
  const int tile_i = blockIdx.y, tile_j = blockIdx.x;
  if (upper && tile_i > tile_j) return;
  gemm_mid_tile<AK, BKM>(M, N, K, A + (int64_t)blockIdx.z * sA, lda, B + (int64_t)blockIdx.z * sB,
                         ldb, C + (int64_t)blockIdx.z * sC, ldc, alpha, beta, upper, mirror,
                         kfrom_i, kto_j, tile_i, tile_j);
}

// Split-k form of gemm_mid_kernel (FP32, beta = 0, no upper / mirror) for products with few
// tiles and long k: chunk z of tile (I, J) of batch member b covers [k_lo + z kc, k_lo + (z+1) kc)
// of the tile's own k range (k_lo, k_hi from kfrom_i / kto_j as in gemm_mid_tile); chunk 0 goes
// to C, chunk z > 0 to part + (z - 1) pstride at C's offsets; gemm_splitk_reduce_kernel adds the
// chunks in order and applies alpha. blockIdx.z = b nzc + z.
template <bool AK, bool BKM>
__global__ void __launch_bounds__(256) gemm_mid_splitk_kernel(
    int M, int N, int K, const float* __restrict__ A, int64_t lda, int64_t sA,
    const float* __restrict__ B, int64_t ldb, int64_t sB, float* __restrict__ C, int64_t ldc,
    int64_t sC, float* __restrict__ part, int64_t pstride, int kc, int nzc, int kfrom_i,
    int kto_j) {
  const int tile_i = blockIdx.y, tile_j = blockIdx.x;
  const int b = blockIdx.z / nzc, z = blockIdx.z - b * nzc;
  const int i0 = tile_i * 64, j0 = tile_j * 64;
  const int klo = (kfrom_i == 1) ? i0 : (kfrom_i == 2 ? j0 : 0);
  const int khi = kto_j ? min(K, j0 + 64) : K;
  const int c0 = klo + z * kc;
  if (c0 >= khi && z > 0) return;
  float* out = (z == 0 ? C : part + (int64_t)(z - 1) * pstride) + (int64_t)b * sC;
  gemm_mid_tile<AK, BKM>(M, N, K, A + (int64_t)b * sA, lda, B + (int64_t)b * sB, ldb, out, ldc,
                         1.f, 0.f, 0, 0, kfrom_i, kto_j, tile_i, tile_j, c0, c0 + kc);
}

__global__ void gemm_splitk_reduce_kernel(int M, int N, int K, float* __restrict__ C, int64_t ldc,
                                          int64_t sC, const float* __restrict__ part,
                                          int64_t pstride, int kc, int kfrom_i, int kto_j,
                                          float alpha) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (e >= (int64_t)M * N) return;
  const int i = (int)(e / N), j = (int)(e - (int64_t)i * N);
  const int i0 = (i / 64) * 64, j0 = (j / 64) * 64;
  const int klo = (kfrom_i == 1) ? i0 : (kfrom_i == 2 ? j0 : 0);
  const int khi = kto_j ? min(K, j0 + 64) : K;
  const int nz = (khi > klo) ? (khi - klo + kc - 1) / kc : 1;
  const int64_t off = (int64_t)b * sC + (int64_t)i * ldc + j;
  float v = C[off];
  for (int z = 1; z < nz; ++z) v += part[(int64_t)(z - 1) * pstride + off];
  C[off] = alpha * v;
}

// C = alpha op(A) op(B) (beta = 0) through the split-k kernels when the grid of 64 x 64 tiles is
// small and k long (part: kSplitChunks - 1 buffers of pstride floats, each covering C's extent);
// returns false (nothing launched) when the product does not qualify.
constexpr int kSplitChunks = 4;
template <bool AK, bool BKM>
bool gemm_splitk(int M, int N, int K, const float* A, int64_t lda, int64_t sA, const float* B,
                 int64_t ldb, int64_t sB, float* C, int64_t ldc, int64_t sC, float alpha,
                 int batch, int kfrom_i, int kto_j, float* part, int64_t pstride,
                 cudaStream_t s) {
  if (part == nullptr || M % 64 || N % 64 || K % 16 || lda % 4 || ldb % 4) return false;
  const int64_t tiles = (int64_t)(M / 64) * (N / 64) * batch;
  const int kc = std::max(256, (K / kSplitChunks + 63) / 64 * 64);
  if (tiles >= 4 * 152 || K <= kc) return false;
  const int nzc = (K + kc - 1) / kc;   // <= kSplitChunks
  if ((int64_t)(batch - 1) * sC + (int64_t)(M - 1) * ldc + N > pstride) return false;
  dim3 g((unsigned)(N / 64), (unsigned)(M / 64), (unsigned)(batch * nzc));
  gemm_mid_splitk_kernel<AK, BKM><<<g, 256, 0, s>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC,
                                                    part, pstride, kc, nzc, kfrom_i, kto_j);
  dim3 gr((unsigned)(((int64_t)M * N + 255) / 256), (unsigned)batch);
  gemm_splitk_reduce_kernel<<<gr, 256, 0, s>>>(M, N, K, C, ldc, sC, part, pstride, kc, kfrom_i,
                                               kto_j, alpha);
  count_launch(2);
  return true;
}

template <typename Tin, typename Tc, bool AK, bool BKM>
void gemm_simt(int M, int N, int K, const Tin* A, int64_t lda, int64_t sA, const Tin* B,
               int64_t ldb, int64_t sB, Tc* C, int64_t ldc, int64_t sC, Tc alpha, Tc beta,
               int upper, int mirror, int batch, cudaStream_t s, const int* skip = nullptr,
               int kfrom_i = 0, int kto_j = 0) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if constexpr (std::is_same<Tin, float>::value && std::is_same<Tc, float>::value) {
    const bool aligned = (M % 4 == 0) && (N % 4 == 0) && (K % 8 == 0) && (lda % 4 == 0) &&
                         (ldb % 4 == 0) && (sA % 4 == 0) && (sB % 4 == 0) &&
                         (reinterpret_cast<uintptr_t>(A) % 16 == 0) &&
                         (reinterpret_cast<uintptr_t>(B) % 16 == 0);
    if (aligned) {
      // 128 x 128 tiles when they still fill the GPU twice over and K is long enough to
      // amortise them; 64 x 64 otherwise
      const int64_t t128 = (int64_t)((N + 127) / 128) * ((M + 127) / 128) * batch;
      const int64_t busy = upper ? (t128 + (int64_t)((N + 127) / 128) * batch) / 2 : t128;
      if (M >= 128 && N >= 128 && K >= 256 && busy >= 2 * 152) {
        dim3 g((N + 127) / 128, (M + 127) / 128, batch);
        gemm_big_kernel<AK, BKM><<<g, 256, 0, s>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC,
                                                   alpha, beta, upper, mirror, kfrom_i, kto_j,
                                                   skip);
        count_launch();
        return;
      }
      if (K % 16 == 0) {
        dim3 g((N + 63) / 64, (M + 63) / 64, batch);
        gemm_mid_kernel<AK, BKM><<<g, 256, 0, s>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC,
                                                   alpha, beta, upper, mirror, kfrom_i, kto_j,
                                                   skip);
        count_launch();
        return;
      }
    }
  }
  dim3 grid((N + 63) / 64, (M + 63) / 64, batch);
  gemm_simt_kernel<Tin, Tc, AK, BKM><<<grid, 256, 0, s>>>(M, N, K, A, lda, sA, B, ldb, sB, C,
                                                         ldc, sC, alpha, beta, upper, mirror,
                                                         skip); count_launch();
}

// M_ij *= dinv_i dinv_j
__global__ void scale_two_sided_kernel(float* __restrict__ M, const float* __restrict__ dinv,
                                       int64_t npad) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npad * npad) return;
  const int64_t i = e / npad, j = e - i * npad;
  M[e] *= dinv[i] * dinv[j];
}

__global__ void set_identity_pad_kernel(void* M, int fp64, int64_t n, int64_t npad) {
  int64_t j = n + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= npad) return;
  if (fp64) static_cast<double*>(M)[j * npad + j] = 1.0;
  else static_cast<float*>(M)[j * npad + j] = 1.f;
}

// ---------------------------------------------------------------------------------------
// Cholesky pieces (upper, H = R^T R), block size 64.
// ---------------------------------------------------------------------------------------
constexpr int NB = 64;
constexpr int kPmChunks = 4;    // k chunks of the split preconditioner-matrix product
constexpr int LDT = 68;   // row stride (floats) of the 64 x 64 FP32 tiles staged in shared memory

template <typename T>
__global__ void add_shift_kernel(T* M, int64_t n, int64_t npad, double shift) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) M[j * npad + j] += (T)shift;
}

// Round to the factor precision (round to nearest even), straight from the working type.
__device__ __forceinline__ float round_prec(float v, int prec) {
  if (prec == (int)Prec::FP16) return __half2float(__float2half_rn(v));
  if (prec == (int)Prec::BF16) return __bfloat162float(__float2bfloat16_rn(v));
  return v;
}
__device__ __forceinline__ double round_prec(double v, int prec) {
  if (prec == (int)Prec::FP16) return (double)__half2float(__double2half(v));
  if (prec == (int)Prec::BF16) return (double)__bfloat162float(__double2bfloat16(v));
  if (prec == (int)Prec::FP32) return (double)(float)v;
  return v;
}

// Diagonal block K = [kb, kb+64) of the blocked Cholesky H = R^T R (upper):
//  1. factor the block (chol64::factor_block: four pivots per step, the block's upper triangle
//     in registers as 4 x 4 tiles; each finished row of R_KK, rounded to the factor precision,
//     goes to global memory and to S, while the block's own update uses the unrounded rows);
//  2. invert the rounded R_KK by doubling from 8 x 8 blocks,
//     [[X11, -X11 R12 X22], [0, X22]] at block sizes 8, 16, 32, into W.
// W_KK turns the panel solve R_KJ = R_KK^{-T} H_KJ into a product, and it is also the diagonal
// block of W = R^{-1}. Nothing runs if an earlier block broke down (*info != 0).
// One doubling level of the inverse of the 64 x 64 upper-triangular block S into X: for every
// pair of SB-blocks A, B, Tm = R_AB X_BB (kept in the zero lower part of S), then
// X_AB = -X_AA Tm. The k sums run over the whole block length (the entries of X_BB below and of
// X_AA left of the diagonal are zero), so they unroll and the loads pipeline.
template <typename T, int SB>
__device__ __forceinline__ void inv_double_level(T (*S)[NB + 1], T (*X)[NB + 1], int tid) {
  constexpr int pairs = NB / (2 * SB), cnt = pairs * SB * SB;
  for (int e = tid; e < cnt; e += 256) {
    const int pr = e / (SB * SB), rem = e % (SB * SB), i = rem / SB, j = rem % SB;
    const int a = 2 * pr * SB;
    T v = T(0);
#pragma unroll
    for (int k = 0; k < SB; ++k) v = fma(S[a + i][a + SB + k], X[a + SB + k][a + SB + j], v);
    S[a + SB + i][a + j] = v;
  }
  __syncthreads();
  for (int e = tid; e < cnt; e += 256) {
    const int pr = e / (SB * SB), rem = e % (SB * SB), i = rem / SB, j = rem % SB;
    const int a = 2 * pr * SB;
    T v = T(0);
#pragma unroll
    for (int k = 0; k < SB; ++k) v = fma(X[a + i][a + k], S[a + SB + k][a + j], v);
    X[a + i][a + SB + j] = -v;
  }
  __syncthreads();
}

// FP64 level of the doubling inverse with the zero parts skipped (FP64 arithmetic runs at a
// 64th of the FP32 rate, so the full-length sums of inv_double_level would cost real time):
// k runs over the upper-triangular support of X_BB and X_AA only, and over the nb leading
// (non-padding) rows and columns of the block; the padding part of X_AB is zero.
template <int SB>
__device__ __forceinline__ void inv_double_level_f64(double (*S)[NB + 1], double (*X)[NB + 1],
                                                     int tid, int nb) {
  constexpr int pairs = NB / (2 * SB), cnt = pairs * SB * SB;
  for (int e = tid; e < cnt; e += 256) {
    const int pr = e / (SB * SB), rem = e % (SB * SB), i = rem / SB, j = rem % SB;
    const int a = 2 * pr * SB, nbB = nb - (a + SB);
    double v = 0.0;
    const int kmax = min(j + 1, nbB);
    for (int k = 0; k < kmax; ++k) v = fma(S[a + i][a + SB + k], X[a + SB + k][a + SB + j], v);
    S[a + SB + i][a + j] = v;
  }
  __syncthreads();
  for (int e = tid; e < cnt; e += 256) {
    const int pr = e / (SB * SB), rem = e % (SB * SB), i = rem / SB, j = rem % SB;
    const int a = 2 * pr * SB, nbB = nb - (a + SB);
    double v = 0.0;
    if (j < nbB)
      for (int k = i; k < SB; ++k) v = fma(X[a + i][a + k], S[a + SB + k][a + j], v);
    X[a + i][a + SB + j] = -v;
  }
  __syncthreads();
}

// nb: the leading non-padding order of the block (a multiple of 8; NB unless this is the last
// block of a problem whose n is not a multiple of 64); used by the FP64 factor only.
// Sbuf, Xbuf: NB x (NB + 1) each in shared memory. Gin, ldin (optional): the block's input, read
// before the factor's first barrier (Xbuf may hold it). Wcopy (optional, FP32): the inverse also
// goes there, row stride LDT, for the caller's next panel products. Returns the breakdown
// (non-zero: the first bad pivot + 1, after which *info is set and nothing else is written).
template <typename T>
__device__ __forceinline__ int potrf_inv_diag_core(T* M, T* W, int64_t npad, int64_t kb,
                                                   int* info, int prec, T* Sbuf, T* Xbuf,
                                                   const T* Gin, int64_t ldin, T* Wcopy,
                                                   int nb, unsigned long long* stamp = nullptr) {
  T (*S)[NB + 1] = reinterpret_cast<T (*)[NB + 1]>(Sbuf);
  T (*X)[NB + 1] = reinterpret_cast<T (*)[NB + 1]>(Xbuf);
  const int tid = threadIdx.x;
  __shared__ chol64::Scratch<T> sc;
  if constexpr (sizeof(T) != 8) nb = NB;
  const int bad = chol64::factor_block<T>(M + kb * npad + kb, npad, &S[0][0], NB + 1, sc,
                                          [prec](T v) { return round_prec(v, prec); }, nb,
                                          Gin, ldin);
  if (stamp != nullptr && tid == 0) *stamp = ptx::global_ns();
  if (bad) {
    if (tid == 0) atomicCAS(info, 0, (int)kb + bad);
    return bad;   // uniform: every thread saw the same pivots
  }
  for (int e = tid; e < NB * NB; e += 256) X[e / NB][e % NB] = T(0);
  __syncthreads();
  if constexpr (sizeof(T) == 8) {
    // reciprocals of the diagonal once, then the 8 x 8 diagonal blocks by substitution with
    // multiplications, then the levels with the zero parts skipped
    T* rd = &sc.rowk[0][0];
    if (tid < NB) rd[tid] = T(1) / S[tid][tid];
    __syncthreads();
    if (tid < 64) {
      const int o = (tid >> 3) * 8, j = tid & 7;
      for (int i = j; i >= 0; --i) {
        T v = (i == j) ? T(1) : T(0);
        for (int k = i + 1; k <= j; ++k) v = fma(-S[o + i][o + k], X[o + k][o + j], v);
        X[o + i][o + j] = v * rd[o + i];
      }
    }
    __syncthreads();
    inv_double_level_f64<8>(S, X, tid, nb);
    inv_double_level_f64<16>(S, X, tid, nb);
    inv_double_level_f64<32>(S, X, tid, nb);
    for (int e = tid; e < NB * NB; e += 256) {
      const int r = e / NB, c = e % NB;
      W[(kb + r) * npad + kb + c] = X[r][c];
    }
    return 0;
  }
  // inverse by doubling: the eight 8 x 8 diagonal blocks by substitution (thread: one column,
  // chains of at most 8), then for s = 8, 16, 32 every pair of s-blocks A, B gets
  // X_AB = -X_AA (R_AB X_BB) as two small products; Tm = R_AB X_BB lives in the (zero, unused)
  // lower part of S
  if (tid < 64) {
    const int o = (tid >> 3) * 8, j = tid & 7;
    for (int i = j; i >= 0; --i) {
      T v = (i == j) ? T(1) : T(0);
      for (int k = i + 1; k <= j; ++k) v = fma(-S[o + i][o + k], X[o + k][o + j], v);
      X[o + i][o + j] = v / S[o + i][o + i];
    }
  }
  __syncthreads();
  inv_double_level<T, 8>(S, X, tid);
  inv_double_level<T, 16>(S, X, tid);
  inv_double_level<T, 32>(S, X, tid);
  for (int e = tid; e < NB * NB; e += 256) {
    const int r = e / NB, c = e % NB;
    W[(kb + r) * npad + kb + c] = X[r][c];
    if (Wcopy) Wcopy[r * LDT + c] = X[r][c];
  }
  return 0;
}

template <typename T>
__device__ __forceinline__ void potrf_inv_diag_body(T* M, T* W, int64_t npad, int64_t kb,
                                                    int* info, int prec, unsigned char* dsm,
                                                    int nb = NB) {
  T* S = reinterpret_cast<T*>(dsm);
  (void)potrf_inv_diag_core<T>(M, W, npad, kb, info, prec, S, S + NB * (NB + 1), nullptr, 0,
                               nullptr, nb);
}

template <typename T>
__global__ void __launch_bounds__(256) potrf_inv_diag_kernel(T* M, T* W, int64_t npad, int64_t kb,
                                                             int* info, int prec, int nb) {
  if (*(volatile int*)info != 0) return;
  extern __shared__ __align__(16) unsigned char dsm[];
  potrf_inv_diag_body<T>(M, W, npad, kb, info, prec, dsm, nb);
}

// Trailing update of block step K, H_22 -= R_K2^T R_K2 (upper 64 x 64 tiles), with the factor
// of the next diagonal block fused in: the CTA of tile (0, 0), which is that block, updates it
// and then factors and inverts it as potrf_inv_diag_kernel does, while the other CTAs update
// the rest of the trailing matrix. FP32 working type.
// BIG: 128 x 128 update tiles (for large trailing matrices; tile (0, 0) still holds the next
// diagonal block at its top left).
template <bool BIG>
__global__ void __launch_bounds__(256) chol_update_next_kernel(float* M, float* W, int64_t npad,
                                                               int64_t kb, int* info, int prec) {
  if (*(volatile int*)info != 0) return;
  const int tile_i = blockIdx.y, tile_j = blockIdx.x;
  if (tile_i > tile_j) return;
  const int64_t k2 = kb + NB, n2 = npad - k2;
  float* P = M + kb * npad + k2;
  if constexpr (BIG)
    gemm_big_tile<false, false>((int)n2, (int)n2, NB, P, npad, P, npad, M + k2 * npad + k2, npad,
                                -1.f, 1.f, 1, 0, 0, 0, tile_i, tile_j);
  else
    gemm_mid_tile<false, false>((int)n2, (int)n2, NB, P, npad, P, npad, M + k2 * npad + k2, npad,
                                -1.f, 1.f, 1, 0, 0, 0, tile_i, tile_j);
  if (tile_i != 0 || tile_j != 0) return;
  __syncthreads();   // the updated block (written by this CTA) before it is factored
  extern __shared__ __align__(16) unsigned char dsm[];
  potrf_inv_diag_body<float>(M, W, npad, k2, info, prec, dsm);
}

// ---------------------------------------------------------------------------------------
// Trailing update on the tensor cores (FP16 / BF16 factors, block steps before the persistent
// chain): H22 -= R_K2^T R_K2 with the panel rows R_K2 rounded to u_f, which are the rows of
// R-hat that the factor keeps, accumulated in FP32 in TMEM.
// ---------------------------------------------------------------------------------------
// PT[j][k] = u_f(R_K2[k][j]) (j < n2, k < 64; rows n2 .. up to the next multiple of 64 zero):
// the panel transposed, K-major for the MMA, through a 64 x 32 shared-memory tile per CTA (each
// thread's eight loads in flight together).
template <typename Tq>
__global__ void __launch_bounds__(256) chol_pt_kernel(const float* __restrict__ M, int64_t npad,
                                                      int64_t kb, int n2, Tq* __restrict__ PT) {
  __shared__ float tl[NB][33];
  const int j0 = blockIdx.x * 32, tid = threadIdx.x, jj = tid & 31, k0 = tid >> 5;
  const float* P = M + kb * npad + kb + NB;
  float v[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int k = k0 + 8 * t;
    v[t] = (j0 + jj < n2) ? P[(int64_t)k * npad + j0 + jj] : 0.f;
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) tl[k0 + 8 * t][jj] = v[t];
  __syncthreads();
  // row j0 + j of PT: 64 values, 8 per thread of a 8-thread group
  const int j = tid >> 3, kq = (tid & 7) * 8;
#pragma unroll
  for (int t = 0; t < 8; ++t)
    PT[(int64_t)(j0 + j) * NB + kq + t] = cvt_out_f<Tq>(tl[kq + t][j]);
}

// CTA (I, J), I <= J, of the 128 x 128 tiles of H22 (n2 x n2 at (k2, k2), k2 = kb + 64): one
// TMA box of each 128-row strip of PT (64 wide, 128-byte swizzle), four MMAs (M = N = 128,
// K = 16) into 128 TMEM columns, and the epilogue subtracts the tile from H22 on and above the
// diagonal. The CTA of tile (0, 0), whose top left is the next diagonal block, then factors and
// inverts that block as chol_update_next_kernel does. Waits are bounded (codes 21-23 in *err).
constexpr int kTcThreads = 256;
constexpr size_t kTcSmem = 2 * sizeof(float) * NB * (NB + 1) + 1024;   // >= 32 KB of strips
__global__ void __launch_bounds__(kTcThreads, 1) chol_tc_update_kernel(
    const __grid_constant__ CUtensorMap pt, float* M, float* W, int64_t npad, int64_t kb,
    int n2, int* info, int prec, uint32_t idesc, int* err) {
  if (*(volatile int*)info != 0) return;   // an earlier block broke down (uniform)
  const int tile_i = blockIdx.y, tile_j = blockIdx.x;
  if (tile_i > tile_j) return;
  extern __shared__ __align__(1024) unsigned char dsm_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sA = smem;
  unsigned char* sB = smem + 128 * NB * 2;
  __shared__ uint64_t full_bar, acc_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const bool diag = (tile_i == tile_j);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k2 = kb + NB;
  if (threadIdx.x == 0) {
    ptx::mbar_init(&full_bar, 1);
    ptx::mbar_init(&acc_bar, 1);
    abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     ptx::smem_u32(&tmem_base)),
                 "r"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_base;
  if (warp == 0 && lane == 0) {
    ptx::mbar_expect_tx(&full_bar, diag ? 128 * NB * 2 : 2 * 128 * NB * 2);
    tc::tma_load_2d(sA, &pt, &full_bar, 0, tile_i * 128);
    if (!diag) tc::tma_load_2d(sB, &pt, &full_bar, 0, tile_j * 128);
    // the copies have landed before this CTA's shared memory is reused or released
    if (!ptx::mbar_wait(&full_bar, 0, err, 21)) abort_flag = 1;
  } else if (warp == 1 && lane == 0) {
    const bool ok = ptx::mbar_wait(&full_bar, 0, err, 22);
    if (ok) {
      tc::tc_fence_after();
      const uint32_t a0 = ptx::smem_u32(sA);
      const uint32_t b0 = diag ? a0 : ptx::smem_u32(sB);
#pragma unroll
      for (int kk = 0; kk < NB / 16; ++kk)
        tc::umma_f16(tmem, tc::sw128_desc(a0 + kk * 32), tc::sw128_desc(b0 + kk * 32), idesc,
                     kk != 0 ? 1u : 0u);
    } else {
      abort_flag = 1;
    }
    tc::umma_commit(&acc_bar);
  } else if (warp >= 2 && warp < 6) {
    const int q = warp & 3;   // TMEM lane quadrant of this warp
    const bool mine = ptx::mbar_wait(&acc_bar, 0, err, 23);
    const bool ready = __all_sync(0xffffffffu, mine) && !*(volatile int*)&abort_flag;
    tc::tc_fence_after();
    if (ready) {
      const int r = tile_i * 128 + q * 32 + lane;   // row of H22
#pragma unroll 1
      for (int c0 = 0; c0 < 128; c0 += 32) {
        uint32_t acc[32];
        tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, acc);
        const int cb = tile_j * 128 + c0;
        if (r < n2 && cb < n2 && cb + 31 >= r) {
          float* dst = M + (k2 + r) * npad + k2 + cb;
          if (cb >= r && cb + 31 < n2) {
#pragma unroll
            for (int v = 0; v < 8; ++v) {
              float4 o = reinterpret_cast<float4*>(dst)[v];
              o.x -= __uint_as_float(acc[4 * v]);
              o.y -= __uint_as_float(acc[4 * v + 1]);
              o.z -= __uint_as_float(acc[4 * v + 2]);
              o.w -= __uint_as_float(acc[4 * v + 3]);
              reinterpret_cast<float4*>(dst)[v] = o;
            }
          } else {
#pragma unroll
            for (int cc = 0; cc < 32; ++cc)
              if (cb + cc >= r && cb + cc < n2) dst[cc] -= __uint_as_float(acc[cc]);
          }
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc::tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128)
                 : "memory");
  }
  if (tile_i != 0 || tile_j != 0 || abort_flag) return;
  __syncthreads();   // the updated block (written by this CTA) before it is factored
  potrf_inv_diag_body<float>(M, W, npad, k2, info, prec, smem);
}

// acc += As^T Bs over k < 64 for the 4 x 4 outputs of this thread (rows 4 ty .. +3, columns
// 4 tx .. +3; tx = tid % 16, ty = tid / 16; 256 threads); As[k][i], Bs[k][j] in shared memory
// with row stride LDT (float4 reads).
__device__ __forceinline__ void tile_atb64(const float* As, const float* Bs, float (&acc)[4][4]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll 8
  for (int k = 0; k < NB; ++k) {
    const float4 a = *reinterpret_cast<const float4*>(As + k * LDT + 4 * ty);
    const float4 b = *reinterpret_cast<const float4*>(Bs + k * LDT + 4 * tx);
    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(av[p], bv[q], acc[p][q]);
  }
}

// Block step K with the panel folded in (FP32). CTA (I, J), I <= J, of the trailing tiles forms
// the panel blocks it needs, P_I = W_KK^T H_KI and P_J = W_KK^T H_KJ (W_KK the inverse of the
// rounded diagonal block), and updates H_IJ -= P_I^T P_J. The CTA of a diagonal tile (I, I)
// also stores P_I, transposed, in the unused lower part of M (column block K), from where
// mirror_panels_kernel copies it into row block K at the end; the CTA of tile (0, 0) then
// factors and inverts the next diagonal block. One launch per block step instead of two (the
// panel products are repeated by the CTAs of a tile row and column; the same arithmetic, in the
// same order, as the separate panel and update products).
// One trailing tile (ti, tj), ti <= tj, of block step kb (the body of chol_step_kernel; all
// threads of the CTA; dsm: 3 x NB x LDT floats).
__device__ __forceinline__ void chol_step_tile(float* M, const float* W, int64_t npad, int64_t kb,
                                               int ti, int tj, unsigned char* dsm) {
  const bool diag = (ti == tj);
  const int64_t k2 = kb + NB;
  float* Wk = reinterpret_cast<float*>(dsm);
  float* Hi = Wk + NB * LDT;
  float* Hj = Hi + NB * LDT;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const float* Wsrc = W + kb * npad + kb;
  const float* Ri = M + kb * npad + k2 + (int64_t)ti * NB;
  const float* Rj = M + kb * npad + k2 + (int64_t)tj * NB;
  // every copy in flight before the first wait (one round trip, not one per row group)
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int e = tid + 256 * i, r = e >> 4, c = (e & 15) * 4;
    ptx::cp_async16(Wk + r * LDT + c, Wsrc + (int64_t)r * npad + c);
    ptx::cp_async16(Hi + r * LDT + c, Ri + (int64_t)r * npad + c);
    if (!diag) ptx::cp_async16(Hj + r * LDT + c, Rj + (int64_t)r * npad + c);
  }
  ptx::cp_async_commit();
  ptx::cp_async_wait_all();
  __syncthreads();
  float pi[4][4], pj[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) pi[p][q] = pj[p][q] = 0.f;
  tile_atb64(Wk, Hi, pi);
  if (!diag) tile_atb64(Wk, Hj, pj);
  __syncthreads();
  // this thread's 4 x 4 entries of the tile into the W_KK area (read by no one from here on), in
  // flight during the second product (no other CTA writes the tile during the step)
  float* C = M + (k2 + (int64_t)ti * NB) * npad + k2 + (int64_t)tj * NB;
#pragma unroll
  for (int p = 0; p < 4; ++p)
    ptx::cp_async16(Wk + (4 * ty + p) * LDT + 4 * tx, C + (int64_t)(4 * ty + p) * npad + 4 * tx);
  ptx::cp_async_commit();
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    *reinterpret_cast<float4*>(Hi + (4 * ty + p) * LDT + 4 * tx) =
        make_float4(pi[p][0], pi[p][1], pi[p][2], pi[p][3]);
    if (!diag)
      *reinterpret_cast<float4*>(Hj + (4 * ty + p) * LDT + 4 * tx) =
          make_float4(pj[p][0], pj[p][1], pj[p][2], pj[p][3]);
  }
  if (diag) {
    // P_I transposed into rows k2 + 64 I .. of column block K (below the diagonal)
    float* low = M + (k2 + (int64_t)ti * NB) * npad + kb;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) low[(int64_t)(4 * tx + q) * npad + 4 * ty + p] = pi[p][q];
  }
  __syncthreads();
  float acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = 0.f;
  tile_atb64(Hi, diag ? Hi : Hj, acc);
  ptx::cp_async_wait_all();   // this thread's own copies of the tile
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const float4 cv = *reinterpret_cast<const float4*>(Wk + (4 * ty + p) * LDT + 4 * tx);
    const float4 o = make_float4(-acc[p][0] + cv.x, -acc[p][1] + cv.y, -acc[p][2] + cv.z,
                                 -acc[p][3] + cv.w);
    float* cp = C + (int64_t)(4 * ty + p) * npad + 4 * tx;
    if (!diag || 4 * ty + p <= 4 * tx) {
      *reinterpret_cast<float4*>(cp) = o;   // the whole row segment is on or above the diagonal
    } else if (4 * ty + p <= 4 * tx + 3) {
      const int a = 4 * ty + p;
      if (a <= 4 * tx + 1) cp[1] = o.y;
      if (a <= 4 * tx + 2) cp[2] = o.z;
      cp[3] = o.w;
    }
  }
}

__global__ void __launch_bounds__(256, 3) chol_step_kernel(float* M, float* W, int64_t npad,
                                                        int64_t kb, int* info, int prec) {
  if (*(volatile int*)info != 0) return;
  const int ti = blockIdx.y, tj = blockIdx.x;
  if (ti > tj) return;
  extern __shared__ __align__(16) unsigned char dsm[];
  chol_step_tile(M, W, npad, kb, ti, tj, dsm);
  if (ti != 0 || tj != 0) return;
  __syncthreads();   // the updated block (written by this CTA) before it is factored
  potrf_inv_diag_body<float>(M, W, npad, kb + NB, info, prec, dsm);
}

// CTA 0's part of block step kb in the persistent chain: tile (0, 0) of the trailing matrix
// (the next diagonal block), then that block's factor and inverse. The arithmetic and its order
// are chol_step_tile's and potrf_inv_diag_body's; what differs is where the operands live:
// W_KK stays in shared memory from the previous step's inverse (read from W on the first step
// only), and the updated block goes to the factor through shared memory rather than through M.
// Shared memory (floats): [0, NB LDT) W_KK; [NB LDT, 2 NB LDT) the panel block P, then the
// updated block, then the inverse X; from 2 NB LDT the factor's S. Returns the factor's
// breakdown code (0: none). tr, tf (optional): the times the update and the factor were done.
__device__ __forceinline__ int chol_cta0_step(float* M, float* W, int64_t npad, int64_t kb,
                                              int* info, int prec, unsigned char* dsm,
                                              bool load_w, unsigned long long* tr,
                                              unsigned long long* tf) {
  const int64_t k2 = kb + NB;
  float* Wk = reinterpret_cast<float*>(dsm);
  float* R2 = Wk + NB * LDT;
  float* R3 = R2 + NB * LDT;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const float* Hsrc = M + kb * npad + k2;
  const float* C = M + k2 * npad + k2;
  // the panel block into R2, this thread's 4 x 4 entries of the block into R3 (free until the
  // factor), W_KK on the first step
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int e = tid + 256 * i, r = e >> 4, c = (e & 15) * 4;
    if (load_w) ptx::cp_async16(Wk + r * LDT + c, W + (kb + r) * npad + kb + c);
    ptx::cp_async16(R2 + r * LDT + c, Hsrc + (int64_t)r * npad + c);
    ptx::cp_async16(R3 + (4 * ty + i) * LDT + 4 * tx, C + (int64_t)(4 * ty + i) * npad + 4 * tx);
  }
  ptx::cp_async_commit();
  ptx::cp_async_wait_all();
  __syncthreads();
  float pi[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) pi[p][q] = 0.f;
  tile_atb64(Wk, R2, pi);
  __syncthreads();
  float* low = M + k2 * npad + kb;   // P transposed below the diagonal (mirror_panels_kernel)
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    *reinterpret_cast<float4*>(R2 + (4 * ty + p) * LDT + 4 * tx) =
        make_float4(pi[p][0], pi[p][1], pi[p][2], pi[p][3]);
#pragma unroll
    for (int q = 0; q < 4; ++q) low[(int64_t)(4 * tx + q) * npad + 4 * ty + p] = pi[p][q];
  }
  __syncthreads();
  float acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = 0.f;
  tile_atb64(R2, R2, acc);
  __syncthreads();   // every read of P done before the updated block replaces it
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const float4 cv = *reinterpret_cast<const float4*>(R3 + (4 * ty + p) * LDT + 4 * tx);
    *reinterpret_cast<float4*>(R2 + (4 * ty + p) * LDT + 4 * tx) =
        make_float4(-acc[p][0] + cv.x, -acc[p][1] + cv.y, -acc[p][2] + cv.z, -acc[p][3] + cv.w);
  }
  __syncthreads();
  if (tr != nullptr && tid == 0) *tr = ptx::global_ns();
  return potrf_inv_diag_core<float>(M, W, npad, k2, info, prec, R3, R2, R2, LDT, Wk, NB, tf);
}

// Grid barrier of a cooperative launch on bar[0] (bar[1]: abort word): thread 0 of each CTA
// fences and adds 1 (CTA 0 adds 2^31 - (G - 1)), so the top bit flips once every CTA has
// arrived and the low bits return to their value; it polls until the bit differs from the one
// its own add saw. Bounded by a 2 s deadline (then code 31 in *err and the abort word raised,
// which the other CTAs see at their next poll). Returns false when abandoned. All threads call it.
__device__ __forceinline__ bool chol_grid_sync(unsigned int* bar, int* err) {
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
          atomicCAS(err, 0, 31);
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

// The block steps kb_from, kb_from + NB, ... of the FP32 factor in one persistent cooperative
// launch, instead of one chol_step_kernel launch per step: per step, CTA 0 updates tile (0, 0)
// and then factors and inverts the next diagonal block (the step's critical path;
// chol_cta0_step), the other CTAs take the remaining trailing tiles from a per-step queue (an
// atomic counter, so the load balances itself; each CTA claims its next tile while it works on
// the current one), and a grid barrier separates the steps. CTAs on CTA 0's SM (its SM id is
// published before the first step) take no tiles, so that the critical path has the SM to
// itself. Every CTA also learns its rank among the CTAs of its SM; a step with few tiles is
// left to the lower ranks, so that its tiles spread over the SMs instead of sharing some. The
// arithmetic of every tile and block is chol_step_kernel's, in the same order.
// bar: [0] barrier counter, [1] abort word, [2] CTA 0's SM id (one 128-byte line), [32 + s] the
// queue of step s (s < 160), [192 + i] the CTA count of SM i (i < 256); all zeroed before the
// launch.
// trace (optional): per step s < 64, [4 s] its start, [4 s + 1] CTA 0's update done, [4 s + 2]
// its factor and inverse done, [4 s + 3] the last worker done; [256 + 4 s] CTA 0's factor done.
__global__ void __launch_bounds__(256, 3) chol_chain_kernel(float* M, float* W, int64_t npad,
                                                         int64_t kb_from, int* info, int prec,
                                                         unsigned int* bar, int* err,
                                                         int num_sms,
                                                         unsigned long long* trace) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ int claim, sm_rank;
  const int c = (int)blockIdx.x;
  unsigned int my_sm;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(my_sm));
  if (threadIdx.x == 0) {
    if (c == 0) bar[2] = my_sm;
    sm_rank = (my_sm < 256u) ? (int)atomicAdd(bar + 192 + my_sm, 1u) : 0;
  }
  if (!chol_grid_sync(bar, err)) return;
  const bool worker = (c != 0) && (*(volatile unsigned int*)(bar + 2) != my_sm);
  const int rank = sm_rank;
  const int worker_sms = max(1, num_sms - 1);
  // CTA 0 is the only writer of *info during the launch: it reads the flag once and then keeps
  // its own breakdown code; the others read the flag after every barrier
  int bad0 = (c == 0) ? *(volatile int*)info : 0;
  int step = 0;
  for (int64_t kb = kb_from; kb + NB < npad; kb += NB, ++step) {
    if (c == 0 ? bad0 != 0 : *(volatile int*)info != 0) return;   // uniform across the grid
    if (step >= 160) {   // more steps than queues (not reached: the chain starts at <= 34 tiles)
      if (c == 0 && threadIdx.x == 0) atomicCAS(err, 0, 32);
      return;
    }
    const int nt = (int)((npad - kb - NB) / NB);
    const int ntiles = nt * (nt + 1) / 2;
    const bool tr = trace != nullptr && step < 64 && threadIdx.x == 0;
    if (c == 0) {
      if (tr) trace[4 * step] = ptx::global_ns();
      const bool trs = trace != nullptr && step < 64;
      bad0 = chol_cta0_step(M, W, npad, kb, info, prec, dsm, step == 0,
                            trs ? trace + 4 * step + 1 : nullptr,
                            trs ? trace + 256 + 4 * step : nullptr);
      if (tr) trace[4 * step + 2] = ptx::global_ns();
    } else if (worker && rank < (ntiles - 1 + worker_sms - 1) / worker_sms) {
      // tiles 1 .. ntiles - 1 in row-major order of the upper triangle, from the step's queue
      unsigned int* q = bar + 32 + step;
      int ti = 0, row_start = 0;
      if (threadIdx.x == 0) claim = 1 + (int)atomicAdd(q, 1u);
      __syncthreads();
      int t = claim;
      while (t < ntiles) {   // t is the same in every thread
        unsigned int nxt = 0u;
        if (threadIdx.x == 0) nxt = atomicAdd(q, 1u);   // in flight during this tile
        while (t >= row_start + (nt - ti)) {
          row_start += nt - ti;
          ++ti;
        }
        chol_step_tile(M, W, npad, kb, ti, ti + (t - row_start), dsm);
        // (the tile's own barriers come after every thread's read of claim)
        if (threadIdx.x == 0) claim = 1 + (int)nxt;
        __syncthreads();   // claim published; shared memory reused by the next tile
        t = claim;
      }
      if (tr) atomicMax(trace + 4 * step + 3, (unsigned long long)ptx::global_ns());
    }
    if (!chol_grid_sync(bar, err)) return;
  }
}

// Row blocks K >= kb_from kept their panels transposed below the diagonal (chol_step_kernel):
// M[r][c] = M[c][r] for r in those row blocks and c right of their diagonal block.
__global__ void mirror_panels_kernel(float* M, int64_t npad, int64_t kb_from) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npad * npad) return;
  const int64_t r = e / npad, c = e % npad;
  if (r >= kb_from && c >= (r / NB + 1) * NB) M[e] = M[c * npad + r];
}

template <typename T>
__global__ void zero_lower_kernel(T* M, int64_t npad) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npad * npad) return;
  int64_t r = e / npad, c = e % npad;
  if (c < r) M[e] = T(0);
}

// ---------------------------------------------------------------------------------------
// Triangular inverse pieces
// ---------------------------------------------------------------------------------------
// W_II = R_II^{-1} for every 64 x 64 diagonal block (one CTA per block, one column per thread).
template <typename T>
__global__ void __launch_bounds__(NB) trtri_diag_kernel(const T* R, T* W, int64_t npad) {
  __shared__ T S[NB][NB + 1];
  __shared__ T X[NB][NB + 1];
  const int64_t o = (int64_t)blockIdx.x * NB;
  const int j = threadIdx.x;
  for (int r = 0; r < NB; ++r) S[r][j] = R[(o + r) * npad + o + j];
  __syncthreads();
  // column j of the inverse: back substitution R x = e_j
  for (int i = NB - 1; i >= 0; --i) {
    T v = (i == j) ? T(1) : T(0);
    if (i <= j) {
      for (int k = i + 1; k <= j; ++k) v = fma(-S[i][k], X[k][j], v);
      X[i][j] = v / S[i][i];
    } else {
      X[i][j] = T(0);
    }
  }
  __syncthreads();
  for (int r = 0; r < NB; ++r) W[(o + r) * npad + o + j] = X[r][j];
}

template <typename T>
__global__ void transpose_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t npad) {
  __shared__ T tile[32][33];
  int64_t x0 = (int64_t)blockIdx.x * 32, y0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) tile[r][threadIdx.x] = in[(y0 + r) * npad + x0 + threadIdx.x];
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) out[(x0 + r) * npad + y0 + threadIdx.x] = tile[threadIdx.x][r];
}

template <typename T>
__global__ void round_kernel(T* R, int64_t count, int prec) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  R[e] = round_prec(R[e], prec);
}

__global__ void f2d_kernel(const float* in, double* out, int64_t count) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) out[e] = (double)in[e];
}
__global__ void d2f_kernel(const double* in, float* out, int64_t count) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) out[e] = (float)in[e];
}

inline int blocks_for(int64_t count, int threads) { return (int)((count + threads - 1) / threads); }

// Sets *flag = 1 when one of the `count` FP64 values at p (16-byte aligned) is NaN or infinite.
// Grid-stride, 16-byte loads: one read of the data at copy bandwidth.
__global__ void __launch_bounds__(256) nonfinite_kernel(const double* __restrict__ p,
                                                        int64_t count, int* __restrict__ flag) {
  const double2* p2 = reinterpret_cast<const double2*>(p);
  const int64_t n2 = count / 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
    const double2 v = p2[i];
    bad |= !(isfinite(v.x) && isfinite(v.y));
  }
  if ((count & 1) && blockIdx.x == 0 && threadIdx.x == 0) bad |= !isfinite(p[count - 1]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

}  // namespace

void launch_nonfinite(const double* p, int64_t count, int* flag, int num_sms, cudaStream_t s) {
  if (count <= 0) return;
  const int64_t want = (count / 2 + 255) / 256;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms * 8));
  nonfinite_kernel<<<grid, 256, 0, s>>>(p, count, flag); count_launch();
}

// =========================================================================================
void launch_colnorm(const double* A, int64_t lda, int64_t m, int64_t n, int64_t npad,
                    float* A32, float* Alo, int64_t ldo, double* d_out, float* dinv32,
                    double* dinv64, double* part, cudaStream_t s) {
  const int P = (int)std::min<int64_t>(64, std::max<int64_t>(1, m / 64));
  dim3 grid((unsigned)((npad + 255) / 256), P);
  colnorm_kernel<<<grid, 256, 0, s>>>(A, lda, m, n, npad, A32, A32 ? Alo : nullptr, ldo, part);
  count_launch();
  colnorm_finish_kernel<<<blocks_for(npad, 256), 256, 0, s>>>(part, P, n, npad, d_out, dinv32,
                                                              dinv64); count_launch();
}

void launch_scale_cast_T(const void* A, bool a_is_fp64, int64_t lda, int64_t m, int64_t n,
                         int64_t npad, int64_t mpad, const double* dinv, const float* dinv32,
                         void* AsT, Prec prec, cudaStream_t s) {
  dim3 grid((unsigned)(mpad / 32), (unsigned)(npad / 32));
  dim3 block(32, 8);
  if (!a_is_fp64 && dinv32 != nullptr && prec != Prec::FP64) {
    const float* Af = static_cast<const float*>(A);
    grid = dim3((unsigned)(mpad / 64), (unsigned)(npad / 64));
    block = dim3(256);
    switch (prec) {
      case Prec::FP16:
        scale_cast_T32_kernel<__half><<<grid, block, 0, s>>>(Af, lda, m, n, npad, mpad, dinv32, static_cast<__half*>(AsT));
        break;
      case Prec::BF16:
        scale_cast_T32_kernel<__nv_bfloat16><<<grid, block, 0, s>>>(Af, lda, m, n, npad, mpad, dinv32, static_cast<__nv_bfloat16*>(AsT));
        break;
      default:
        scale_cast_T32_kernel<float><<<grid, block, 0, s>>>(Af, lda, m, n, npad, mpad, dinv32, static_cast<float*>(AsT));
        break;
    }
    count_launch();
    return;
  }
#define TLS_SC(TIN, TOUT)                                                                     \
  scale_cast_T_kernel<TIN, TOUT><<<grid, block, 0, s>>>(static_cast<const TIN*>(A), lda, m, n, \
                                                        npad, mpad, dinv, static_cast<TOUT*>(AsT))
  if (a_is_fp64) {
    switch (prec) {
      case Prec::FP16: TLS_SC(double, __half); break;
      case Prec::BF16: TLS_SC(double, __nv_bfloat16); break;
      case Prec::FP32: TLS_SC(double, float); break;
      case Prec::FP64: TLS_SC(double, double); break;
    }
  } else {
    switch (prec) {
      case Prec::FP16: TLS_SC(float, __half); break;
      case Prec::BF16: TLS_SC(float, __nv_bfloat16); break;
      case Prec::FP32: TLS_SC(float, float); break;
      case Prec::FP64: TLS_SC(float, double); break;
    }
  }
#undef TLS_SC
  count_launch();
}

// Sum of `chunks` partial npad x npad FP64 Gram matrices (fixed order) into H, mirrored
__global__ void gram_sum_kernel(const double* __restrict__ part, int chunks, int64_t npad,
                                double* __restrict__ H) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npad * npad) return;
  const int64_t r = e / npad, c = e % npad;
  const int64_t src = (r <= c) ? e : c * npad + r;   // partials hold the upper triangle
  double a = 0.0;
  for (int k = 0; k < chunks; ++k) a += part[(int64_t)k * npad * npad + src];
  H[e] = a;
}

int gram_split_chunks(int64_t npad, int64_t mpad, int num_sms) {
  // an FP64 Gram of a few output tiles runs on a few SMs: split its rows into chunks of at least
  // 8 rows, up to one per SM (a chunk's tile is FP64-bound on its SM: 400 x 64 in 14 chunks of
  // 32 rows took 48 us). Each chunk writes a full npad x npad FP64 partial that the sum kernel
  // reads back; the partials are capped at 32 MB in all so that they stay in L2 (npad <= 128
  // gives at most 128 KB per chunk, so the cap only binds for unusually many SMs).
  if (npad > 128) return 1;
  const int64_t by_rows = std::max<int64_t>(1, mpad / 8);
  const int64_t by_bytes = std::max<int64_t>(1, (int64_t)(32u << 20) / (npad * npad * 8));
  return (int)std::min<int64_t>(std::max(1, num_sms), std::min(by_rows, by_bytes));
}

void launch_gram_simt(const void* AsT, Prec prec, int64_t n, int64_t npad, int64_t mpad,
                      void* H, cudaStream_t s, void* work, int chunks) {
  const int M = (int)npad, K = (int)mpad;
  if (prec == Prec::FP64 && work != nullptr) {
    if (chunks > 1) {
      // chunk z: rows [z*kc, min(K, (z+1)*kc)) of A_s^T A_s (upper tiles) into work[z]
      const int kc = (int)(((int64_t)K + chunks - 1) / chunks);
      const int full = K / kc, rest = K - full * kc;
      gemm_simt<double, double, true, true>(M, M, kc, (const double*)AsT, mpad, kc,
                                            (const double*)AsT, mpad, kc, (double*)work, npad,
                                            npad * npad, 1.0, 0.0, 1, 0, full, s);
      int used = full;
      if (rest > 0) {
        gemm_simt<double, double, true, true>(M, M, rest, (const double*)AsT + (int64_t)full * kc,
                                              mpad, 0, (const double*)AsT + (int64_t)full * kc,
                                              mpad, 0, (double*)work + (int64_t)full * npad * npad,
                                              npad, 0, 1.0, 0.0, 1, 0, 1, s);
        ++used;
      }
      gram_sum_kernel<<<blocks_for(npad * npad, 256), 256, 0, s>>>((const double*)work, used, npad,
                                                                  (double*)H);
      count_launch();
      launch_set_identity_pad(H, true, n, npad, s);
      return;
    }
  }
  switch (prec) {
    case Prec::FP16:
      gemm_simt<__half, float, true, true>(M, M, K, (const __half*)AsT, mpad, 0, (const __half*)AsT,
                                          mpad, 0, (float*)H, npad, 0, 1.f, 0.f, 1, 1, 1, s);
      break;
    case Prec::BF16:
      gemm_simt<__nv_bfloat16, float, true, true>(M, M, K, (const __nv_bfloat16*)AsT, mpad, 0,
                                                  (const __nv_bfloat16*)AsT, mpad, 0, (float*)H,
                                                  npad, 0, 1.f, 0.f, 1, 1, 1, s);
      break;
    case Prec::FP32:
      gemm_simt<float, float, true, true>(M, M, K, (const float*)AsT, mpad, 0, (const float*)AsT,
                                          mpad, 0, (float*)H, npad, 0, 1.f, 0.f, 1, 1, 1, s);
      break;
    case Prec::FP64:
      gemm_simt<double, double, true, true>(M, M, K, (const double*)AsT, mpad, 0,
                                            (const double*)AsT, mpad, 0, (double*)H, npad, 0,
                                            1.0, 0.0, 1, 1, 1, s);
      break;
  }
  launch_set_identity_pad(H, prec == Prec::FP64, n, npad, s);
}

void launch_set_identity_pad(void* M, bool fp64, int64_t n, int64_t npad, cudaStream_t s) {
  if (npad > n)
    set_identity_pad_kernel<<<blocks_for(npad - n, 128), 128, 0, s>>>(M, fp64 ? 1 : 0, n, npad); count_launch();
}

template <typename T>
void launch_cholesky(T* M, int64_t n, int64_t npad, double shift, int* info, T* Wd, Prec prec,
                     cudaStream_t s, unsigned int* gbar, int* err, int num_sms,
                     unsigned long long* trace, int chain_per_sm, void* ptbuf) {
  // (chain_per_sm 2 measured best at n = 2048: 756 us per factor against 807 us for 3 or 4
  // CTAs per SM and 838 us with one launch per block step)
  if (shift != 0.0) { add_shift_kernel<T><<<blocks_for(n, 256), 256, 0, s>>>(M, n, npad, shift); count_launch(); }
  const size_t dsmem = 2 * sizeof(T) * NB * (NB + 1);
  static const bool attr = [dsmem] {   // thread-safe one-time initialisation
    cudaFuncSetAttribute(potrf_inv_diag_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)dsmem);
    return true;
  }();
  (void)attr;
  constexpr bool fused = std::is_same<T, float>::value;
  if constexpr (fused) {
    static const bool attr2 = [dsmem] {
      cudaFuncSetAttribute(chol_update_next_kernel<false>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem);
      cudaFuncSetAttribute(chol_update_next_kernel<true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem);
      return true;
    }();
    (void)attr2;
  }
  // leading non-padding order of the diagonal block at kb (multiple of 8, at most 64)
  auto active = [n](int64_t kb) {
    return (int)std::min<int64_t>(NB, std::max<int64_t>(8, (n - kb + 7) / 8 * 8));
  };
  potrf_inv_diag_kernel<T><<<1, 256, dsmem, s>>>(M, Wd, npad, 0, info, (int)prec, active(0));
  count_launch();
  int64_t kb_from = npad;   // first block step with the panel folded into the update
  for (int64_t kb = 0; kb < npad; kb += NB) {
    const int64_t n2 = npad - kb - NB;
    if (n2 <= 0) break;
    if constexpr (fused) {
      // one launch per step while the trailing tiles fit in about four CTAs per SM (the panel
      // products are then repeated at little cost and the step is the diagonal block's chain)
      const int64_t nt = n2 / NB;
      if (nt * (nt + 1) / 2 <= 4 * 152) {
        static const bool attr3 = [] {
          cudaFuncSetAttribute(chol_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(3 * NB * LDT * sizeof(float)));
          cudaFuncSetAttribute(chol_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(3 * NB * LDT * sizeof(float)));
          return true;
        }();
        (void)attr3;
        if (kb_from == npad) kb_from = kb;
        if (gbar != nullptr && num_sms > 1) {
          // this and every later step in one persistent cooperative launch
          int per_sm = 0;
          const size_t cs = 3 * NB * LDT * sizeof(float);
          if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chol_chain_kernel, 256, cs) ==
                  cudaSuccess &&
              per_sm >= 1) {
            float* Mf = reinterpret_cast<float*>(M);
            float* Wf = reinterpret_cast<float*>(Wd);
            int pr = (int)prec;
            int64_t kbv = kb;
            int64_t npv = npad;
            int nsm = num_sms;
            void* args[] = {&Mf, &Wf, &npv, &kbv, &info, &pr, &gbar, &err, &nsm, &trace};
            const int grid = std::max(1, std::min(per_sm, chain_per_sm)) * num_sms;
            cudaMemsetAsync(gbar + 2, 0, sizeof(unsigned int) * 446, s);   // SM id, queues, ranks
            const cudaError_t e = cudaLaunchCooperativeKernel((const void*)chol_chain_kernel,
                                                              grid, 256, args, cs, s);
            count_launch();
            if (e == cudaSuccess) break;
            (void)cudaGetLastError();   // not launchable: one launch per step below
          }
        }
        chol_step_kernel<<<dim3((unsigned)nt, (unsigned)nt), 256, 3 * NB * LDT * sizeof(float),
                           s>>>(M, Wd, npad, kb, info, (int)prec);
        count_launch();
        continue;
      }
    }
    // panel R_KJ = W_KK^T H_KJ, in place over H_KJ
    gemm_simt<T, T, false, false>(NB, (int)n2, NB, Wd + kb * npad + kb, npad, 0,
                                  M + kb * npad + kb + NB, npad, 0, M + kb * npad + kb + NB, npad,
                                  0, T(1), T(0), 0, 0, 1, s, info);
    // trailing update H22 -= R_K2^T R_K2 (upper part), then the next diagonal block
    if constexpr (fused) {
      if (ptbuf != nullptr && err != nullptr && (prec == Prec::FP16 || prec == Prec::BF16) &&
          gram_tc_available()) {
        // on the tensor cores: the panel rounded to u_f and transposed, then the update
        const bool bf = (prec == Prec::BF16);
        const int ntp = (int)((n2 + NB - 1) / NB);
        const unsigned gpt = (unsigned)(ntp * NB / 32);
        if (bf)
          chol_pt_kernel<__nv_bfloat16><<<gpt, 256, 0, s>>>(
              reinterpret_cast<const float*>(M), npad, kb, (int)n2,
              static_cast<__nv_bfloat16*>(ptbuf));
        else
          chol_pt_kernel<__half><<<gpt, 256, 0, s>>>(reinterpret_cast<const float*>(M), npad, kb,
                                                     (int)n2, static_cast<__half*>(ptbuf));
        CUtensorMap map;
        if (tc::encode_kmajor_map(&map, ptbuf, bf, NB, (uint64_t)ntp * NB, NB * 2, NB, 128)) {
          static const bool attr_tc = [] {
            cudaFuncSetAttribute(chol_tc_update_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
            return true;
          }();
          (void)attr_tc;
          const unsigned nt = (unsigned)((n2 + 127) / 128);
          chol_tc_update_kernel<<<dim3(nt, nt), kTcThreads, kTcSmem, s>>>(
              map, reinterpret_cast<float*>(M), reinterpret_cast<float*>(Wd), npad, kb, (int)n2,
              info, (int)prec, tc::idesc_f16_mn(bf ? 1u : 0u, 128, 128), err);
          count_launch(2);
          continue;
        }
        count_launch();
      }
      // 128 x 128 tiles once they still give about two CTAs per SM
      if (n2 >= 2048) {
        const unsigned nt = (unsigned)((n2 + 127) / 128);
        chol_update_next_kernel<true><<<dim3(nt, nt), 256, dsmem, s>>>(M, Wd, npad, kb, info,
                                                                      (int)prec);
      } else {
        const unsigned nt = (unsigned)(n2 / NB);
        chol_update_next_kernel<false><<<dim3(nt, nt), 256, dsmem, s>>>(M, Wd, npad, kb, info,
                                                                       (int)prec);
      }
      count_launch();
    } else {
      T* P = M + kb * npad + kb + NB;
      T* C = M + (kb + NB) * npad + kb + NB;
      gemm_simt<T, T, false, false>((int)n2, (int)n2, NB, P, npad, 0, P, npad, 0, C, npad, 0,
                                    T(-1), T(1), 1, 0, 1, s, info);
      potrf_inv_diag_kernel<T><<<1, 256, dsmem, s>>>(M, Wd, npad, kb + NB, info, (int)prec,
                                                     active(kb + NB));
      count_launch();
    }
  }
  if constexpr (fused) {
    if (kb_from < npad) {
      mirror_panels_kernel<<<blocks_for(npad * npad, 256), 256, 0, s>>>(M, npad, kb_from);
      count_launch();
    }
  }
  zero_lower_kernel<T><<<blocks_for(npad * npad, 256), 256, 0, s>>>(M, npad); count_launch();
}

template <typename T>
void launch_round_to(T* R, int64_t npad, Prec prec, cudaStream_t s) {
  if (prec != Prec::FP16 && prec != Prec::BF16) return;
  round_kernel<T><<<blocks_for(npad * npad, 256), 256, 0, s>>>(R, npad * npad, (int)prec); count_launch();
}

template <typename T>
void launch_trtri(const T* R, T* W, T* WT, T* work, int64_t npad, bool have_diag,
                  cudaStream_t s, T* part) {
  if (!have_diag) {
    cudaMemsetAsync(W, 0, sizeof(T) * npad * npad, s);
    trtri_diag_kernel<T><<<(unsigned)(npad / NB), NB, 0, s>>>(R, W, npad); count_launch();
  }
  // recursive doubling: for blocks A = [o, o+sz), B = [o+sz, o+sz+sB):
  //   W_AB = -W_AA R_AB W_BB
  for (int64_t sz = NB; sz < npad; sz *= 2) {
    const int64_t full_pairs = npad / (2 * sz);
    if (full_pairs > 0) {
      // work_AB = R_AB W_BB ; W_AB = -W_AA work_AB   (batched over the full pairs)
      const int64_t st = 2 * sz * npad + 2 * sz;   // stride between pairs along the diagonal
      // (W_BB and W_AA are upper triangular: the products skip their zero k-slabs; the top
      // levels, with few tiles and long k, split k over more CTAs)
      bool split = false;
      if constexpr (std::is_same<T, float>::value)
        split = gemm_splitk<true, false>((int)sz, (int)sz, (int)sz, R + sz, npad, st,
                                         W + sz * npad + sz, npad, st, work + sz, npad, st, 1.f,
                                         (int)full_pairs, 0, 1, part, npad * npad, s);
      if (!split)
        gemm_simt<T, T, true, false>((int)sz, (int)sz, (int)sz, R + sz, npad, st,
                                     W + sz * npad + sz, npad, st, work + sz, npad, st, T(1),
                                     T(0), 0, 0, (int)full_pairs, s, nullptr, 0, 1);
      split = false;
      if constexpr (std::is_same<T, float>::value)
        split = gemm_splitk<true, false>((int)sz, (int)sz, (int)sz, W, npad, st, work + sz, npad,
                                         st, W + sz, npad, st, -1.f, (int)full_pairs, 1, 0, part,
                                         npad * npad, s);
      if (!split)
        gemm_simt<T, T, true, false>((int)sz, (int)sz, (int)sz, W, npad, st, work + sz, npad, st,
                                     W + sz, npad, st, T(-1), T(0), 0, 0, (int)full_pairs, s,
                                     nullptr, 1, 0);
    }
    const int64_t o = full_pairs * 2 * sz;
    const int64_t sB = npad - o - sz;
    if (sB > 0) {
      const T* Rab = R + o * npad + o + sz;
      const T* Wbb = W + (o + sz) * npad + o + sz;
      T* Wk = work + o * npad + o + sz;
      gemm_simt<T, T, true, false>((int)sz, (int)sB, (int)sB, Rab, npad, 0, Wbb, npad, 0, Wk, npad,
                                   0, T(1), T(0), 0, 0, 1, s, nullptr, 0, 1);
      gemm_simt<T, T, true, false>((int)sz, (int)sB, (int)sz, W + o * npad + o, npad, 0, Wk, npad,
                                   0, W + o * npad + o + sz, npad, 0, T(-1), T(0), 0, 0, 1, s,
                                   nullptr, 1, 0);
    }
  }
  dim3 grid((unsigned)(npad / 32), (unsigned)(npad / 32));
  transpose_kernel<T><<<grid, dim3(32, 8), 0, s>>>(W, WT, npad); count_launch();
}

void launch_f2d(const float* in, double* out, int64_t count, cudaStream_t s) {
  f2d_kernel<<<blocks_for(count, 256), 256, 0, s>>>(in, out, count); count_launch();
}
void launch_d2f(const double* in, float* out, int64_t count, cudaStream_t s) {
  d2f_kernel<<<blocks_for(count, 256), 256, 0, s>>>(in, out, count); count_launch();
}

template void launch_cholesky<float>(float*, int64_t, int64_t, double, int*, float*, Prec,
                                     cudaStream_t, unsigned int*, int*, int, unsigned long long*,
                                     int, void*);
template void launch_cholesky<double>(double*, int64_t, int64_t, double, int*, double*, Prec,
                                      cudaStream_t, unsigned int*, int*, int, unsigned long long*,
                                      int, void*);
template void launch_round_to<float>(float*, int64_t, Prec, cudaStream_t);
template void launch_round_to<double>(double*, int64_t, Prec, cudaStream_t);
template void launch_trtri<float>(const float*, float*, float*, float*, int64_t, bool, cudaStream_t,
                                  float*);
template void launch_trtri<double>(const double*, double*, double*, double*, int64_t, bool,
                                   cudaStream_t, double*);

// The PCGTLS preconditioner as one matrix: M = D^{-1} (W W^T) D^{-1}, W = R_H^{-1} upper
// triangular: (W W^T)_ij = sum over k >= max(i, j) of W_ik W_jk, so an upper tile (I <= J)
// starts its k range at j0; mirrored to the lower triangle, FP32.
// M = D^{-1} W W^T D^{-1} with the k sums split into chunks of kc (npad / kPmChunks rounded up
// to 64, at least 512): upper 64 x 64 tile (I, J) sums over k >= 64 J (W upper triangular), so
// the first tile columns carry sums of length n and the last of 64; chunk z of tile (I, J)
// covers k in [64 J + z kc, + kc) (chunk 0 into M, chunk z > 0 into part[z - 1]), and
// precond_reduce_kernel adds the chunks in order, scales by d_i^{-1} d_j^{-1} and mirrors. The
// same products as one launch, the k sums regrouped by chunk.
__global__ void __launch_bounds__(256) precond_splitk_kernel(const float* __restrict__ W,
                                                             int64_t npad, float* __restrict__ M,
                                                             float* __restrict__ part, int kc) {
  const int tile_i = blockIdx.y, tile_j = blockIdx.x, z = blockIdx.z;
  if (tile_i > tile_j) return;
  const int k0 = tile_j * 64 + z * kc;
  if (k0 >= npad) return;
  float* out = (z == 0) ? M : part + (int64_t)(z - 1) * npad * npad;
  const int n = (int)npad;
  gemm_mid_tile<true, true>(n, n, n, W, npad, W, npad, out, npad, 1.f, 0.f, /*upper=*/1,
                            /*mirror=*/0, /*kfrom_i=*/2, 0, tile_i, tile_j, k0, k0 + kc);
}

__global__ void precond_reduce_kernel(float* __restrict__ M, const float* __restrict__ part,
                                      const float* __restrict__ dinv, int64_t npad, int kc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npad * npad) return;
  const int64_t i = e / npad, j = e - i * npad;
  if (i > j) return;
  const int64_t j0 = (j / 64) * 64;
  const int nz = (int)((npad - j0 + kc - 1) / kc);
  float v = M[e];
  for (int z = 1; z < nz; ++z) v += part[(int64_t)(z - 1) * npad * npad + e];
  v *= dinv[i] * dinv[j];
  M[e] = v;
  if (i != j) M[j * npad + i] = v;
}

void launch_precond_matrix(const float* W, const float* dinv, int64_t npad, float* M,
                           cudaStream_t s, float* part) {
  const int n = (int)npad;
  const int kc = (int)std::max<int64_t>(512, (npad / kPmChunks + 63) / 64 * 64);
  if (part == nullptr || npad <= kc) {
    gemm_simt<float, float, true, true>(n, n, n, W, npad, 0, W, npad, 0, M, npad, 0, 1.f, 0.f,
                                        /*upper=*/1, /*mirror=*/1, 1, s, nullptr, /*kfrom_i=*/2, 0);
    scale_two_sided_kernel<<<(unsigned)((npad * npad + 255) / 256), 256, 0, s>>>(M, dinv, npad);
    count_launch();
    return;
  }
  const int nz = (int)((npad + kc - 1) / kc);   // <= kPmChunks: part holds kPmChunks - 1 matrices
  dim3 g((unsigned)(npad / 64), (unsigned)(npad / 64), (unsigned)nz);
  precond_splitk_kernel<<<g, 256, 0, s>>>(W, npad, M, part, kc);
  precond_reduce_kernel<<<(unsigned)((npad * npad + 255) / 256), 256, 0, s>>>(M, part, dinv, npad,
                                                                             kc);
  count_launch(2);
}

}  // namespace tls
