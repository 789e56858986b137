// Cholesky of one 64 x 64 diagonal block of a blocked factorisation H = R^T R (upper), shared by
// the single-problem factor and the packed batch.
//
// The block's upper triangle is held in registers as the 136 4 x 4 tiles (I, J), I <= J, of its
// 16 x 16 tile grid, one tile per thread. kPB = 8 pivots per step: the threads of tile rows
// k/4 and k/4 + 1 publish rows k .. k+7 of the updated (unscaled) block; 64 threads form the
// 8 x 8 factor R11 of the pivot block and the rows k .. k+7 of R, Y = R11^{-T} S[k:k+8][:]
// (unrounded); every tile below takes the rank-8 update S[i][j] -= sum_t Y[t][i] Y[t][j] from
// registers. Two barriers per step, eight steps per block. Each finished row of R goes out
// rounded to the factor precision (global memory and the shared copy S used for the inverse),
// while the block's own update uses the unrounded rows. (Loops over the pivot block run to kPB
// with a guard rather than to t, so that they unroll and R11 stays in registers.)
#pragma once
#include <cstdint>

namespace tls {
namespace chol64 {

constexpr int kB = 64;   // block order
constexpr int kPB = 8;   // pivots per step (a multiple of 4)
constexpr int kTT = kB / 4;

template <typename T>
struct Scratch {
  T rowk[kPB][kB];
  T Yk[kPB][kB];
  T r11[kPB][kPB];   // FP64: the pivot block's factor, formed once per step
  T rinv[kPB];
  int bad;
};

// Factor the block at G (global, row stride ld; only its upper triangle is read). On return,
// when no pivot broke down: the upper triangle of G holds R_KK rounded by `rnd`, and S (shared,
// row stride lds) holds the same rows with zeros below the diagonal. Returns the first
// non-positive (or NaN) pivot + 1, or 0; the value is the same in every thread. Call with all
// threads of a CTA of at least 136 threads (blockDim.x <= 1024).
// nb (a multiple of kPB, at most kB): the block's rows and columns from nb on are the identity
// padding of an order-n problem (identity on the diagonal, zero elsewhere), so only the leading
// nb x nb part is factored; G keeps the padding as it is and S receives it.
// Gin, ldin (optional): read the block from there instead of from G (e.g. a copy in shared memory
// that the caller has just updated); the rows of R still go to G. Gin is read before the first
// barrier, so it may share storage with S.
// FP64 (sizeof(T) == 8; FP64 arithmetic runs at a 64th of the FP32 rate): R11 is formed once per
// step by one warp and shared, rather than by every column thread.
template <typename T, typename Round>
__device__ int factor_block(T* G, int64_t ld, T* S, int lds, Scratch<T>& sc, Round rnd,
                           int nb = kB, const T* Gin = nullptr, int64_t ldin = 0) {
  const int tid = threadIdx.x;
  int tI = kTT, tJ = 0;
  if (tid < kTT * (kTT + 1) / 2) {
    int off = 0, I = 0;
    while (off + (kTT - I) <= tid) { off += kTT - I; ++I; }
    tI = I;
    tJ = I + (tid - off);
  }
  // (entries below the diagonal inside the diagonal tiles ride along and are never published)
  T v[4][4];
  const T* src = Gin ? Gin : G;
  const int64_t lsrc = Gin ? ldin : ld;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c)
      v[a][c] = (tI < kTT) ? src[(int64_t)(4 * tI + a) * lsrc + 4 * tJ + c] : T(0);
  if (tid == 0) sc.bad = 0;
  if (nb < kB)
    for (int e = tid; e < kB * kB; e += blockDim.x) {
      const int rr = e / kB, cc = e % kB;
      if (rr >= nb || cc >= nb) S[rr * lds + cc] = (rr == cc) ? T(1) : T(0);
    }
  for (int k = 0; k < nb; k += kPB) {
    if (tI >= k / 4 && tI < (k + kPB) / 4)
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) sc.rowk[4 * tI - k + a][4 * tJ + c] = v[a][c];
    __syncthreads();
    if constexpr (sizeof(T) == 8) {
      if (tid < 32) {
        T r[kPB][kPB], rinv[kPB];
        int bad = 0;
#pragma unroll
        for (int t = 0; t < kPB; ++t) {
          T dsum = sc.rowk[t][k + t];
#pragma unroll
          for (int q = 0; q < kPB; ++q)
            if (q < t) dsum = fma(-r[q][t], r[q][t], dsum);
          if (!(dsum > T(0))) {
            bad = bad ? bad : (k + t + 1);
            dsum = T(1);
          }
          const T rtt = sqrt(dsum);
          const T inv = T(1) / rtt;
          r[t][t] = rtt;
          rinv[t] = inv;
#pragma unroll
          for (int u = 0; u < kPB; ++u) {
            if (u > t) {
              T e = sc.rowk[t][k + u];
#pragma unroll
              for (int q = 0; q < kPB; ++q)
                if (q < t) e = fma(-r[q][t], r[q][u], e);
              r[t][u] = e * inv;
            }
          }
        }
        if (tid == 0) {
#pragma unroll
          for (int t = 0; t < kPB; ++t) {
            sc.rinv[t] = rinv[t];
#pragma unroll
            for (int u = 0; u < kPB; ++u) sc.r11[t][u] = (u >= t) ? r[t][u] : T(0);
          }
          if (bad) atomicCAS(&sc.bad, 0, bad);
        }
      }
      __syncthreads();
      if (tid < nb && tid >= k) {
        const int c = tid;
        T y[kPB];
#pragma unroll
        for (int t = 0; t < kPB; ++t) {
          T e = sc.rowk[t][c];
#pragma unroll
          for (int q = 0; q < kPB; ++q)
            if (q < t) e = fma(-sc.r11[q][t], y[q], e);
          y[t] = (c - k < t) ? T(0) : e * sc.rinv[t];
        }
#pragma unroll
        for (int t = 0; t < kPB; ++t) {
          sc.Yk[t][c] = y[t];
          if (c >= k + t) {
            const T val = rnd(y[t]);
            G[(int64_t)(k + t) * ld + c] = val;
            S[(k + t) * lds + c] = val;
          }
        }
      } else if (tid < kB && tid >= nb) {
#pragma unroll
        for (int t = 0; t < kPB; ++t) sc.Yk[t][tid] = T(0);   // padding columns
      }
    } else if (tid < kB && tid >= k) {
      // R11 = chol(S11) from the published upper entries
      T r[kPB][kPB], rinv[kPB];
      int bad = 0;
#pragma unroll
      for (int t = 0; t < kPB; ++t) {
        T dsum = sc.rowk[t][k + t];
#pragma unroll
        for (int q = 0; q < kPB; ++q)
          if (q < t) dsum = fma(-r[q][t], r[q][t], dsum);
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
        for (int u = 0; u < kPB; ++u) {
          if (u > t) {
            T e = sc.rowk[t][k + u];
#pragma unroll
            for (int q = 0; q < kPB; ++q)
              if (q < t) e = fma(-r[q][t], r[q][u], e);
            r[t][u] = e * inv;
          }
        }
      }
      // column c = tid of rows k .. k+kPB-1 of R by forward substitution with R11^T (inside the
      // pivot block it reproduces R11's entries operation for operation; zeros below them)
      const int c = tid;
      T y[kPB];
#pragma unroll
      for (int t = 0; t < kPB; ++t) {
        T e = sc.rowk[t][c];
#pragma unroll
        for (int q = 0; q < kPB; ++q)
          if (q < t) e = fma(-r[q][t], y[q], e);
        y[t] = (c - k < t) ? T(0) : e * rinv[t];
      }
#pragma unroll
      for (int t = 0; t < kPB; ++t) {
        sc.Yk[t][c] = y[t];
        if (c >= k + t) {
          const T val = rnd(y[t]);
          G[(int64_t)(k + t) * ld + c] = val;
          S[(k + t) * lds + c] = val;
        }
      }
      if (bad && tid == k) atomicCAS(&sc.bad, 0, bad);
    }
    __syncthreads();
    if (tI < kTT && tI >= (k + kPB) / 4 && tJ < nb / 4) {
      T yi[kPB][4], yj[kPB][4];
#pragma unroll
      for (int t = 0; t < kPB; ++t)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          yi[t][c] = sc.Yk[t][4 * tI + c];
          yj[t][c] = sc.Yk[t][4 * tJ + c];
        }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          T acc = v[a][c];
#pragma unroll
          for (int t = 0; t < kPB; ++t) acc = fma(-yi[t][a], yj[t][c], acc);
          v[a][c] = acc;
        }
    }
  }
  __syncthreads();
  const int bad = sc.bad;
  for (int e = tid; e < kB * kB; e += blockDim.x) {
    const int rr = e / kB, cc = e % kB;
    if (cc < rr) S[rr * lds + cc] = T(0);
  }
  __syncthreads();
  return bad;
}

}  // namespace chol64
}  // namespace tls
