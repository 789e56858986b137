// Condition estimates for the constraints on the factor precision (Sec. 3.1 of Oktay & Carson,
// arXiv 2305.19028): constraint 1, u_q <~ kappa(A)^{-1} (Eq. (5)), and constraint 2,
// u_q <~ kappa_F(A)^{-1} (1 - sigma_{n+1}^2 / sigma'_n^2) (Eq. (9)).
//  * sigma'_1^2 = lambda_max(A^T A) by power iteration on D H D (H the scaled Gram matrix);
//  * sigma'_n^2 = 1 / lambda_max((R^T R)^{-1}) by power iteration with the preconditioner
//    products (R from the computed factor, so this is the factor's own estimate);
//  * ||A^+||_F ~ ||R^{-1}||_F = ||D^{-1} W||_F from the explicit inverse W = R_H^{-1}.
// All in the working type T; only the final scalars are formed in FP64.
#include "tls_internal.h"

namespace tls {

namespace {

template <typename T>
__device__ __forceinline__ T cwsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// y_i = d_i sum_j H_ij d_j x_j (one warp per row; H full n_pad x n_pad)
template <typename T>
__global__ void __launch_bounds__(256) dhd_kernel(const T* __restrict__ H, int64_t npad,
                                                  const T* __restrict__ dinv,
                                                  const T* __restrict__ x, T* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= npad) return;
  const T* row = H + i * npad;
  T a = T(0);
  for (int64_t j = lane; j < npad; j += 32) a = fma(row[j], x[j] / dinv[j], a);
  a = cwsum(a);
  if (lane == 0) y[i] = a / dinv[i];
}

// One CTA: lam = x^T y, then x = y / ||y|| (x, y of length n, working type)
template <typename T>
__global__ void __launch_bounds__(1024) power_finish_kernel(T* __restrict__ x,
                                                            const T* __restrict__ y, int64_t n,
                                                            double* __restrict__ lam_out) {
  __shared__ T sh[2][32];
  T xy = T(0), yy = T(0);
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    xy = fma(x[j], y[j], xy);
    yy = fma(y[j], y[j], yy);
  }
  xy = cwsum(xy);
  yy = cwsum(yy);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { sh[0][warp] = xy; sh[1][warp] = yy; }
  __syncthreads();
  if (warp == 0) {
    T a = (lane < (int)(blockDim.x >> 5)) ? sh[0][lane] : T(0);
    T b = (lane < (int)(blockDim.x >> 5)) ? sh[1][lane] : T(0);
    a = cwsum(a);
    b = cwsum(b);
    if (lane == 0) { sh[0][0] = a; sh[1][0] = b; }
  }
  __syncthreads();
  const T nrm = sqrt(sh[1][0]);
  if (threadIdx.x == 0) *lam_out = (double)sh[0][0];
  const T inv = (nrm > T(0)) ? T(1) / nrm : T(0);
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) x[j] = y[j] * inv;
}

// x = ones / sqrt(n) on the first n entries, zero padding
template <typename T>
__global__ void power_init_kernel(T* x, int64_t n, int64_t npad) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < npad) x[j] = (j < n) ? T(1) / sqrt((T)n) : T(0);
}

// sum of (dinv_i W_ij)^2 over the first n rows / columns (one warp per row), per-CTA partials
template <typename T>
__global__ void __launch_bounds__(256) frob_dw_kernel(const T* __restrict__ W, int64_t n,
                                                      int64_t npad, const T* __restrict__ dinv,
                                                      double* __restrict__ part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * 8 + warp;
  T a = T(0);
  if (i < n) {
    const T* row = W + i * npad;
    for (int64_t j = i + lane; j < n; j += 32) a = fma(row[j], row[j], a);
    a = cwsum(a) * dinv[i] * dinv[i];
  }
  __shared__ T sh[8];
  if (lane == 0) sh[warp] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    T t = T(0);
    for (int w = 0; w < 8; ++w) t += sh[w];
    part[blockIdx.x] = (double)t;
  }
}

// x (T) from a double vector (first n) and back
template <typename T>
__global__ void vec_to_double_kernel(const T* __restrict__ x, double* __restrict__ y, int64_t n,
                                     int64_t npad) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < npad) y[j] = (j < n) ? (double)x[j] : 0.0;
}

inline int nb(int64_t c, int t) { return (int)((c + t - 1) / t); }

}  // namespace

template <typename T>
void launch_dhd(const T* H, int64_t npad, const T* dinv, const T* x, T* y, cudaStream_t s) {
  dhd_kernel<T><<<nb(npad * 32, 256), 256, 0, s>>>(H, npad, dinv, x, y);
  count_launch();
}
template <typename T>
void launch_power_finish(T* x, const T* y, int64_t n, double* lam, cudaStream_t s) {
  power_finish_kernel<T><<<1, 1024, 0, s>>>(x, y, n, lam);
  count_launch();
}
template <typename T>
void launch_power_init(T* x, int64_t n, int64_t npad, cudaStream_t s) {
  power_init_kernel<T><<<nb(npad, 256), 256, 0, s>>>(x, n, npad);
  count_launch();
}
template <typename T>
int launch_frob_dw(const T* W, int64_t n, int64_t npad, const T* dinv, double* part,
                   cudaStream_t s) {
  const int g = nb(n, 8);
  frob_dw_kernel<T><<<g, 256, 0, s>>>(W, n, npad, dinv, part);
  count_launch();
  return g;
}
template <typename T>
void launch_vec_to_double(const T* x, double* y, int64_t n, int64_t npad, cudaStream_t s) {
  vec_to_double_kernel<T><<<nb(npad, 256), 256, 0, s>>>(x, y, n, npad);
  count_launch();
}

#define TLS_CI(T)                                                                              \
  template void launch_dhd<T>(const T*, int64_t, const T*, const T*, T*, cudaStream_t);        \
  template void launch_power_finish<T>(T*, const T*, int64_t, double*, cudaStream_t);          \
  template void launch_power_init<T>(T*, int64_t, int64_t, cudaStream_t);                      \
  template int launch_frob_dw<T>(const T*, int64_t, int64_t, const T*, double*, cudaStream_t); \
  template void launch_vec_to_double<T>(const T*, double*, int64_t, int64_t, cudaStream_t);
TLS_CI(float)
TLS_CI(double)
#undef TLS_CI

}  // namespace tls
