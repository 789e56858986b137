// Triangular solves with the factor itself (Alg. 3: s_0 = R^{-T} f and q = R^{-1} p; Alg. 2:
// u_0 = R^{-1} R^{-T} x_0), for R = R_H D: s = R_H^{-T} (D^{-1} y) and u = D^{-1} R_H^{-1} s, by
// blocked substitution on R_H instead of the products with its explicit inverse W = R_H^{-1}
// that the solve uses. One CTA of 1024 threads holds the right-hand side in shared memory; per
// 64-row block one warp solves the diagonal block by substitution (a chain of 64 pivots, the
// block staged in shared memory) and all warps update the rest of the right-hand side from R_H's
// rows. Forward: R_H^T s = y' with y' -= R_KL^T s_K after block K (coalesced along the rows of
// R_H); backward: R_H u' = s with the row sums R_KL u'_L (L > K) taken before block K.
#include "tls_internal.h"

namespace tls {

namespace {

constexpr int kTrThreads = 1024;
constexpr int kTrB = 64;

template <typename T>
__device__ __forceinline__ T tr_warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(kTrThreads, 1) trsv_kernel(const T* __restrict__ R, int64_t npad,
                                                            int64_t n, const T* __restrict__ dinv,
                                                            const double* __restrict__ y,
                                                            T* __restrict__ s_out,
                                                            T* __restrict__ u_out) {
  extern __shared__ __align__(16) unsigned char tr_sm[];
  T* v = reinterpret_cast<T*>(tr_sm);   // npad: the right-hand side, then the solution
  T* blk = v + npad;                    // 64 x 65: the diagonal block
  T* tsum = blk + kTrB * (kTrB + 1);    // 64: the row sums of the backward solve
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kTrThreads / 32;
  const int nb = (int)(npad / kTrB);
  for (int64_t i = tid; i < npad; i += kTrThreads) v[i] = (i < n) ? (T)y[i] * dinv[i] : T(0);
  __syncthreads();
  // ---- forward: R_H^T s = y'
  for (int K = 0; K < nb; ++K) {
    const int64_t k0 = (int64_t)K * kTrB;
    for (int e = tid; e < kTrB * kTrB; e += kTrThreads) {
      const int r = e / kTrB, c = e % kTrB;
      blk[r * (kTrB + 1) + c] = R[(k0 + r) * npad + k0 + c];
    }
    __syncthreads();
    if (warp == 0) {
      // lane l holds entries l and l + 32 of the block's right-hand side
      T t0 = v[k0 + lane], t1 = v[k0 + 32 + lane];
      for (int k = 0; k < kTrB; ++k) {
        const T tk = (k < 32) ? __shfl_sync(0xffffffffu, t0, k) : __shfl_sync(0xffffffffu, t1, k - 32);
        const T sk = tk / blk[k * (kTrB + 1) + k];
        if (lane == k) t0 = sk;
        if (lane + 32 == k) t1 = sk;
        if (lane > k) t0 = fma(-blk[k * (kTrB + 1) + lane], sk, t0);
        if (lane + 32 > k) t1 = fma(-blk[k * (kTrB + 1) + lane + 32], sk, t1);
      }
      v[k0 + lane] = t0;
      v[k0 + 32 + lane] = t1;
    }
    __syncthreads();
    for (int64_t l = k0 + kTrB + tid; l < npad; l += kTrThreads) {
      T acc = v[l];
      for (int k = 0; k < kTrB; ++k) acc = fma(-R[(k0 + k) * npad + l], v[k0 + k], acc);
      v[l] = acc;
    }
    __syncthreads();
  }
  for (int64_t i = tid; i < npad; i += kTrThreads) s_out[i] = v[i];
  __syncthreads();
  // ---- backward: R_H u' = s
  for (int K = nb - 1; K >= 0; --K) {
    const int64_t k0 = (int64_t)K * kTrB;
    for (int kr = warp; kr < kTrB; kr += NW) {
      T acc = T(0);
      for (int64_t l = k0 + kTrB + lane; l < npad; l += 32) acc = fma(R[(k0 + kr) * npad + l], v[l], acc);
      acc = tr_warp_sum(acc);
      if (lane == 0) tsum[kr] = acc;
    }
    for (int e = tid; e < kTrB * kTrB; e += kTrThreads) {
      const int r = e / kTrB, c = e % kTrB;
      blk[r * (kTrB + 1) + c] = R[(k0 + r) * npad + k0 + c];
    }
    __syncthreads();
    if (warp == 0) {
      T t0 = v[k0 + lane] - tsum[lane], t1 = v[k0 + 32 + lane] - tsum[lane + 32];
      for (int k = kTrB - 1; k >= 0; --k) {
        const T tk = (k < 32) ? __shfl_sync(0xffffffffu, t0, k) : __shfl_sync(0xffffffffu, t1, k - 32);
        const T uk = tk / blk[k * (kTrB + 1) + k];
        if (lane == k) t0 = uk;
        if (lane + 32 == k) t1 = uk;
        if (lane < k) t0 = fma(-blk[lane * (kTrB + 1) + k], uk, t0);
        if (lane + 32 < k) t1 = fma(-blk[(lane + 32) * (kTrB + 1) + k], uk, t1);
      }
      v[k0 + lane] = t0;
      v[k0 + 32 + lane] = t1;
    }
    __syncthreads();
  }
  for (int64_t i = tid; i < npad; i += kTrThreads) u_out[i] = v[i] * dinv[i];
}

}  // namespace

template <typename T>
bool launch_trsv(const T* R, int64_t npad, int64_t n, const T* dinv, const double* y, T* s_out,
                 T* u_out, cudaStream_t s) {
  const size_t smem = sizeof(T) * ((size_t)npad + kTrB * (kTrB + 1) + kTrB);
  if (npad % kTrB != 0 || smem > 227 * 1024) return false;
  static const bool attr = [] {
    cudaFuncSetAttribute(trsv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    return true;
  }();
  (void)attr;
  trsv_kernel<T><<<1, kTrThreads, smem, s>>>(R, npad, n, dinv, y, s_out, u_out);
  count_launch();
  return cudaGetLastError() == cudaSuccess;
}

template bool launch_trsv<float>(const float*, int64_t, int64_t, const float*, const double*,
                                 float*, float*, cudaStream_t);
template bool launch_trsv<double>(const double*, int64_t, int64_t, const double*, const double*,
                                  double*, double*, cudaStream_t);

}  // namespace tls
