// Preconditioner construction (Sec. 3.1 of Oktay & Carson, arXiv 2305.19028): column scaling
// D = diag(||a_j||), the Gram matrix H = (A D^{-1})^T (A D^{-1}) of the u_f-rounded scaled
// matrix, blocked Cholesky H + sI = R_H^T R_H, rounding of R_H to u_f, and the explicit inverse
// W = R_H^{-1} that the PCGTLS iteration applies as two triangular products per step.
#include "tls_internal.h"
#include "tls_device.cuh"

#include <algorithm>
#include <type_traits>

namespace tls {

namespace {

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
                                                      float* __restrict__ A32, int64_t ldo,
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
        const float f = f64_to_f32_rn(v[u]);
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
// AsT[j][i] = fl(A[i][j] / d_j): scaled, rounded and transposed (n x mpad), via 32x32 tiles
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
template <> __device__ __forceinline__ float cvt_out_f<float>(float v) { return v; }
template <> __device__ __forceinline__ double cvt_out_f<double>(float v) { return (double)v; }

// FP32 input (the working copy of A): A_s = fl(fl32(A32 * dinv32)), all in FP32 arithmetic
template <typename Tout>
__global__ void scale_cast_T32_kernel(const float* __restrict__ A, int64_t lda, int64_t m,
                                      int64_t n, int64_t npad, int64_t mpad,
                                      const float* __restrict__ dinv, Tout* __restrict__ AsT) {
  __shared__ float tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int64_t j0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t i = i0 + r, j = j0 + threadIdx.x;
    float v = 0.f;
    if (i < m && j < n) v = A[i * lda + j] * dinv[j];
    tile[r][threadIdx.x] = v;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int64_t j = j0 + r, i = i0 + threadIdx.x;
    if (j < npad && i < mpad) AsT[j * mpad + i] = cvt_out_f<Tout>(tile[threadIdx.x][r]);
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

template <typename Tin, typename Tc, bool AK, bool BKM>
void gemm_simt(int M, int N, int K, const Tin* A, int64_t lda, int64_t sA, const Tin* B,
               int64_t ldb, int64_t sB, Tc* C, int64_t ldc, int64_t sC, Tc alpha, Tc beta,
               int upper, int mirror, int batch, cudaStream_t s, const int* skip = nullptr) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  dim3 grid((N + 63) / 64, (M + 63) / 64, batch);
  gemm_simt_kernel<Tin, Tc, AK, BKM><<<grid, 256, 0, s>>>(M, N, K, A, lda, sA, B, ldb, sB, C,
                                                         ldc, sC, alpha, beta, upper, mirror,
                                                         skip); count_launch();
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
//  1. factor the block (256 threads, the upper triangle held in registers, one barrier per
//     pivot; each finished row of R_KK, rounded to the factor precision, goes straight to
//     global memory, while the update of step k uses the unrounded row as
//     S[k][i] S[k][j] / S[k][k]);
//  2. invert the rounded R_KK by doubling from 8 x 8 blocks,
//     [[X11, -X11 R12 X22], [0, X22]] at block sizes 8, 16, 32, into W.
// W_KK turns the panel solve R_KJ = R_KK^{-T} H_KJ into a product, and it is also the diagonal
// block of W = R^{-1}. Nothing runs if an earlier block broke down (*info != 0).
template <typename T>
__global__ void __launch_bounds__(256) potrf_inv_diag_kernel(T* M, T* W, int64_t npad, int64_t kb,
                                                             int* info, int prec) {
  if (*(volatile int*)info != 0) return;
  extern __shared__ __align__(16) unsigned char dsm[];
  T (*S)[NB + 1] = reinterpret_cast<T (*)[NB + 1]>(dsm);
  T (*X)[NB + 1] = reinterpret_cast<T (*)[NB + 1]>(dsm + sizeof(T) * NB * (NB + 1));
  const int tid = threadIdx.x;
  // the 2080 entries of the block's upper triangle are dealt round-robin to the 256 threads
  // and stay in registers through the factorisation (entry e = tid + 256 p, row-major order)
  constexpr int NE = NB * (NB + 1) / 2;
  constexpr int PE = (NE + 255) / 256;
  T v[PE];
  int ei[PE], ej[PE];
#pragma unroll
  for (int p = 0; p < PE; ++p) {
    const int e = tid + 256 * p;
    ei[p] = NB;   // never updated or published
    ej[p] = 0;
    v[p] = T(0);
    if (e < NE) {
      int i = 0, off = 0;
      while (off + (NB - i) <= e) { off += NB - i; ++i; }
      ei[p] = i;
      ej[p] = i + (e - off);
      v[p] = M[(kb + i) * npad + kb + ej[p]];
    }
  }
  // four pivots per step: the owners publish rows k .. k+3 of the updated (unscaled) block;
  // 64 threads form the 4 x 4 factor R11 and Y = R11^{-T} S[k:k+4][:] (rows k .. k+3 of R,
  // unrounded) into shared memory; every entry below takes the rank-4 update
  // S[i][j] -= sum_t Y[t][i] Y[t][j]. Two barriers per step.
  constexpr int PB = 4;
  __shared__ T rowk[PB][NB];
  __shared__ T Yk[PB][NB];
  __shared__ int s_bad;
  if (tid == 0) s_bad = 0;
  bool broke = false;
  for (int k = 0; k < NB; k += PB) {
#pragma unroll
    for (int p = 0; p < PE; ++p)
      if (ei[p] >= k && ei[p] < k + PB) rowk[ei[p] - k][ej[p]] = v[p];
    __syncthreads();
    if (tid < NB && tid >= k) {
      // R11 = chol(S11) (S11 symmetric: its lower entries from the published upper ones)
      T r[PB][PB], rinv[PB];
      int bad = 0;
#pragma unroll
      for (int t = 0; t < PB; ++t) {
        T dsum = rowk[t][k + t];
#pragma unroll
        for (int q = 0; q < t; ++q) dsum = fma(-r[q][t], r[q][t], dsum);
        if (!(dsum > T(0))) {                // non-positive or NaN pivot: breakdown
          bad = bad ? bad : (k + t + 1);
          dsum = T(1);
        }
        T rtt, inv;
        if constexpr (sizeof(T) == 4) {
          inv = rsqrtf(dsum);                // R_KK is rounded to u_f or carries an FP32 error
          rtt = dsum * inv;
        } else {
          rtt = sqrt(dsum);
          inv = T(1) / rtt;
        }
        r[t][t] = rtt;
        rinv[t] = inv;
#pragma unroll
        for (int u = t + 1; u < PB; ++u) {
          T e = rowk[t][k + u];
#pragma unroll
          for (int q = 0; q < t; ++q) e = fma(-r[q][t], r[q][u], e);
          r[t][u] = e * inv;
        }
      }
      // column c = tid of rows k .. k+3 of R: the pivot block from R11, the rest by forward
      // substitution with R11^T
      const int c = tid;
      T y[PB];
      if (c < k + PB) {
#pragma unroll
        for (int t = 0; t < PB; ++t) y[t] = (c - k >= t) ? r[t][c - k] : T(0);
      } else {
#pragma unroll
        for (int t = 0; t < PB; ++t) {
          T e = rowk[t][c];
#pragma unroll
          for (int q = 0; q < t; ++q) e = fma(-r[q][t], y[q], e);
          y[t] = e * rinv[t];
        }
      }
#pragma unroll
      for (int t = 0; t < PB; ++t) {
        Yk[t][c] = y[t];
        if (c >= k + t) {
          // rows of R_KK rounded to the factor precision: global memory and S (for the inverse)
          const T val = round_prec(y[t], prec);
          M[(kb + k + t) * npad + kb + c] = val;
          S[k + t][c] = val;
        }
      }
      if (bad && tid == k) atomicCAS(&s_bad, 0, bad);
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PE; ++p)
      if (ei[p] >= k + PB) {
        T acc = v[p];
#pragma unroll
        for (int t = 0; t < PB; ++t) acc = fma(-Yk[t][ei[p]], Yk[t][ej[p]], acc);
        v[p] = acc;
      }
  }
  __syncthreads();
  if (s_bad) {
    if (tid == 0) atomicCAS(info, 0, (int)kb + s_bad);
    broke = true;
  }
  __syncthreads();
  if (broke) return;   // uniform: every thread saw the same pivots
  for (int e = tid; e < NB * NB; e += 256) {
    const int r = e / NB, c = e % NB;
    if (c < r) S[r][c] = T(0);
    X[r][c] = T(0);
  }
  __syncthreads();
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
  for (int sb = 8; sb < NB; sb *= 2) {
    const int pairs = NB / (2 * sb), cnt = pairs * sb * sb;
    for (int e = tid; e < cnt; e += 256) {
      const int pr = e / (sb * sb), rem = e % (sb * sb), i = rem / sb, j = rem % sb;
      const int a = 2 * pr * sb;
      T v = T(0);
      for (int k = 0; k <= j; ++k) v = fma(S[a + i][a + sb + k], X[a + sb + k][a + sb + j], v);
      S[a + sb + i][a + j] = v;
    }
    __syncthreads();
    for (int e = tid; e < cnt; e += 256) {
      const int pr = e / (sb * sb), rem = e % (sb * sb), i = rem / sb, j = rem % sb;
      const int a = 2 * pr * sb;
      T v = T(0);
      for (int k = i; k < sb; ++k) v = fma(X[a + i][a + k], S[a + sb + k][a + j], v);
      X[a + i][a + sb + j] = -v;
    }
    __syncthreads();
  }
  for (int e = tid; e < NB * NB; e += 256) {
    const int r = e / NB, c = e % NB;
    W[(kb + r) * npad + kb + c] = X[r][c];
  }
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

}  // namespace

// =========================================================================================
void launch_colnorm(const double* A, int64_t lda, int64_t m, int64_t n, int64_t npad,
                    float* A32, int64_t ldo, double* d_out, float* dinv32, double* dinv64,
                    double* part, cudaStream_t s) {
  const int P = (int)std::min<int64_t>(64, std::max<int64_t>(1, m / 64));
  dim3 grid((unsigned)((npad + 255) / 256), P);
  colnorm_kernel<<<grid, 256, 0, s>>>(A, lda, m, n, npad, A32, ldo, part); count_launch();
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

void launch_gram_simt(const void* AsT, Prec prec, int64_t n, int64_t npad, int64_t mpad,
                      void* H, cudaStream_t s) {
  const int M = (int)npad, K = (int)mpad;
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
                     cudaStream_t s) {
  if (shift != 0.0) { add_shift_kernel<T><<<blocks_for(n, 256), 256, 0, s>>>(M, n, npad, shift); count_launch(); }
  const size_t dsmem = 2 * sizeof(T) * NB * (NB + 1);
  static const bool attr = [dsmem] {   // thread-safe one-time initialisation
    cudaFuncSetAttribute(potrf_inv_diag_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)dsmem);
    return true;
  }();
  (void)attr;
  for (int64_t kb = 0; kb < npad; kb += NB) {
    potrf_inv_diag_kernel<T><<<1, 256, dsmem, s>>>(M, Wd, npad, kb, info, (int)prec);
    count_launch();
    const int64_t n2 = npad - kb - NB;
    if (n2 <= 0) break;
    // panel R_KJ = W_KK^T H_KJ, in place over H_KJ
    gemm_simt<T, T, false, false>(NB, (int)n2, NB, Wd + kb * npad + kb, npad, 0,
                                  M + kb * npad + kb + NB, npad, 0, M + kb * npad + kb + NB, npad,
                                  0, T(1), T(0), 0, 0, 1, s, info);
    // trailing update H22 -= R_K2^T R_K2 (upper part)
    T* P = M + kb * npad + kb + NB;
    T* C = M + (kb + NB) * npad + kb + NB;
    gemm_simt<T, T, false, false>((int)n2, (int)n2, NB, P, npad, 0, P, npad, 0, C, npad, 0,
                                  T(-1), T(1), 1, 0, 1, s, info);
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
                  cudaStream_t s) {
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
      gemm_simt<T, T, true, false>((int)sz, (int)sz, (int)sz, R + sz, npad, st, W + sz * npad + sz,
                                   npad, st, work + sz, npad, st, T(1), T(0), 0, 0,
                                   (int)full_pairs, s);
      gemm_simt<T, T, true, false>((int)sz, (int)sz, (int)sz, W, npad, st, work + sz, npad, st,
                                   W + sz, npad, st, T(-1), T(0), 0, 0, (int)full_pairs, s);
    }
    const int64_t o = full_pairs * 2 * sz;
    const int64_t sB = npad - o - sz;
    if (sB > 0) {
      const T* Rab = R + o * npad + o + sz;
      const T* Wbb = W + (o + sz) * npad + o + sz;
      T* Wk = work + o * npad + o + sz;
      gemm_simt<T, T, true, false>((int)sz, (int)sB, (int)sB, Rab, npad, 0, Wbb, npad, 0, Wk, npad,
                                   0, T(1), T(0), 0, 0, 1, s);
      gemm_simt<T, T, true, false>((int)sz, (int)sB, (int)sz, W + o * npad + o, npad, 0, Wk, npad,
                                   0, W + o * npad + o + sz, npad, 0, T(-1), T(0), 0, 0, 1, s);
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

template void launch_cholesky<float>(float*, int64_t, int64_t, double, int*, float*, Prec, cudaStream_t);
template void launch_cholesky<double>(double*, int64_t, int64_t, double, int*, double*, Prec, cudaStream_t);
template void launch_round_to<float>(float*, int64_t, Prec, cudaStream_t);
template void launch_round_to<double>(double*, int64_t, Prec, cudaStream_t);
template void launch_trtri<float>(const float*, float*, float*, float*, int64_t, bool, cudaStream_t);
template void launch_trtri<double>(const double*, double*, double*, double*, int64_t, bool, cudaStream_t);

}  // namespace tls
