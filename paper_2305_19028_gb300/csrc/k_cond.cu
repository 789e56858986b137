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
    a = cwsum(a);
    if (dinv != nullptr) a = a * dinv[i] * dinv[i];
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

// ---------------------------------------------------------------------------------------
// Selector features of one problem from its factor (the same 16 values as the packed batch's
// features kernel): spreads of d and diag(R_H), ||W||_F and ||W||_2 of W = R_H^{-1} (power
// iteration on W^T W, 9 products with W from the vector of ones), problem sizes, norms, shifts.
// ---------------------------------------------------------------------------------------
// y = M x with M upper (rows i: columns j >= i) or lower (j <= i) triangular; one warp per row
template <typename T, bool UPPER>
__global__ void __launch_bounds__(256) feat_gemv_kernel(const T* __restrict__ M, int64_t npad,
                                                        const T* __restrict__ x,
                                                        T* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= npad) return;
  const T* row = M + i * npad;
  T a = T(0);
  if (UPPER) {
    for (int64_t j = i + lane; j < npad; j += 32) a = fma(row[j], x[j], a);
  } else {
    for (int64_t j = lane; j <= i; j += 32) a = fma(row[j], x[j], a);
  }
  a = cwsum(a);
  if (lane == 0) y[i] = a;
}

// One CTA. mode 0: x = ones on the first n entries (zero padding). mode 1: out = sqrt(|y|^2 /
// |x|^2) (the estimate after a product y = W x). mode 2: x = z / |z|. Sums in FP64. z may be x
// itself (mode 2 normalises x in place, each thread reading and writing only its own entries),
// so x and z carry no __restrict__.
template <typename T>
__global__ void __launch_bounds__(1024) feat_power_kernel(T* x, const T* __restrict__ y,
                                                          const T* z, int64_t n,
                                                          int64_t npad, int mode,
                                                          double* __restrict__ out) {
  __shared__ double sh[2][32];
  if (mode == 0) {
    for (int64_t j = threadIdx.x; j < npad; j += blockDim.x) x[j] = (j < n) ? T(1) : T(0);
    return;
  }
  double a = 0.0, b = 0.0;
  for (int64_t j = threadIdx.x; j < npad; j += blockDim.x) {
    if (mode == 1) {
      a = fma((double)y[j], (double)y[j], a);
      b = fma((double)x[j], (double)x[j], b);
    } else {
      a = fma((double)z[j], (double)z[j], a);
    }
  }
  a = cwsum(a);
  b = cwsum(b);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { sh[0][warp] = a; sh[1][warp] = b; }
  __syncthreads();
  if (warp == 0) {
    double u = (lane < (int)(blockDim.x >> 5)) ? sh[0][lane] : 0.0;
    double v = (lane < (int)(blockDim.x >> 5)) ? sh[1][lane] : 0.0;
    u = cwsum(u);
    v = cwsum(v);
    if (lane == 0) { sh[0][0] = u; sh[1][0] = v; }
  }
  __syncthreads();
  if (mode == 1) {
    if (threadIdx.x == 0) *out = sqrt(sh[0][0] / fmax(sh[1][0], 1e-300));
    return;
  }
  const double inv = 1.0 / sqrt(fmax(sh[0][0], 1e-300));
  for (int64_t j = threadIdx.x; j < npad; j += blockDim.x) x[j] = (T)((double)z[j] * inv);
}

__device__ __forceinline__ double lg10(double v) { return log10(v); }

// One CTA: extremes of d and diag(R_H), sum of log10 d, then the 16 features from those,
// the ||W||_F^2 partials and ||W||_2 (wn), written to F.
template <typename T>
__global__ void __launch_bounds__(1024) feat_finish_kernel(
    const double* __restrict__ d, const T* __restrict__ R, int64_t n, int64_t npad, int64_t m,
    const double* __restrict__ part, int nparts, const double* __restrict__ wn, double norm2_A,
    double norm2_b, int nshift, double shift, int fail_pivot, double log10_uf,
    float* __restrict__ F) {
  double dmax = 0.0, dmin = 1e300, rmax = 0.0, rmin = 1e300, sld = 0.0, fro = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double dj = d[j], rj = (double)R[j * npad + j];
    dmax = fmax(dmax, dj);
    dmin = fmin(dmin, dj);
    rmax = fmax(rmax, rj);
    rmin = fmin(rmin, rj);
    sld += lg10(dj);
  }
  for (int p = threadIdx.x; p < nparts; p += blockDim.x) fro += part[p];
  double v[6] = {dmax, -dmin, rmax, -rmin, sld, fro};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = fmax(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
    v[4] += __shfl_xor_sync(0xffffffffu, v[4], o);
    v[5] += __shfl_xor_sync(0xffffffffu, v[5], o);
  }
  __shared__ double red[6][32];
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 6; ++k) red[k][warp] = v[k];
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < nw; ++w) {
#pragma unroll
    for (int k = 0; k < 4; ++k) red[k][0] = fmax(red[k][0], red[k][w]);
    red[4][0] += red[4][w];
    red[5][0] += red[5][w];
  }
  dmax = red[0][0];
  dmin = -red[1][0];
  rmax = red[2][0];
  rmin = -red[3][0];
  sld = red[4][0];
  fro = red[5][0];
  const double lw2 = lg10(*wn), lwf = 0.5 * lg10(fro);
  float f[16];
  f[0] = (float)lg10((double)m);
  f[1] = (float)lg10((double)n);
  f[2] = (float)lg10((double)m / (double)n);
  f[3] = (float)(lg10(dmax) - lg10(dmin));
  f[4] = (float)(sld / (double)n - lg10(dmax));
  f[5] = (float)(0.5 * (lg10(norm2_b) - lg10(norm2_A)));
  f[6] = (float)(lg10(rmax) - lg10(rmin));
  f[7] = (float)lg10(rmin);
  f[8] = (float)nshift;
  f[9] = (float)lg10(1.0 + shift / pow(10.0, log10_uf));
  f[10] = (float)lwf;
  f[11] = (float)lw2;
  f[12] = (float)(lwf - lw2);
  f[13] = (float)(log10_uf + 2.0 * lw2);
  f[14] = (float)(log10_uf + lw2);
  f[15] = (fail_pivot >= 0) ? (float)fail_pivot / (float)n : 0.f;
  for (int k = 0; k < 16; ++k) F[k] = f[k];
}

// F = (F - mean) / scale (16 values)
__global__ void feat_normalise_kernel(float* F, const float* mean, const float* scale) {
  const int k = threadIdx.x;
  if (k < 16) F[k] = (F[k] - mean[k]) / scale[k];
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

template <typename T>
void launch_features(const double* d, const T* R, const T* W, const T* WT, int64_t n, int64_t npad,
                     int64_t m, double norm2_A, double norm2_b, int nshift, double shift,
                     int fail_pivot, double log10_uf, T* x, T* y, double* scratch, float* F,
                     cudaStream_t s) {
  // scratch: [0] ||W||_2, [1 ..] the ||W||_F^2 partials
  const int g = nb(n, 8);
  frob_dw_kernel<T><<<g, 256, 0, s>>>(W, n, npad, nullptr, scratch + 1);
  feat_power_kernel<T><<<1, 1024, 0, s>>>(x, nullptr, nullptr, n, npad, 0, nullptr);
  count_launch(2);
  for (int it = 0; it < 9; ++it) {
    feat_gemv_kernel<T, true><<<nb(npad * 32, 256), 256, 0, s>>>(W, npad, x, y);
    feat_power_kernel<T><<<1, 1024, 0, s>>>(x, y, nullptr, n, npad, 1, scratch);
    count_launch(2);
    if (it == 8) break;
    feat_gemv_kernel<T, false><<<nb(npad * 32, 256), 256, 0, s>>>(WT, npad, y, x);
    feat_power_kernel<T><<<1, 1024, 0, s>>>(x, nullptr, x, n, npad, 2, nullptr);
    count_launch(2);
  }
  feat_finish_kernel<T><<<1, 1024, 0, s>>>(d, R, n, npad, m, scratch + 1, g, scratch, norm2_A,
                                           norm2_b, nshift, shift, fail_pivot, log10_uf, F);
  count_launch();
}

void launch_feature_normalise(float* F, const float* mean, const float* scale, cudaStream_t s) {
  feat_normalise_kernel<<<1, 32, 0, s>>>(F, mean, scale);
  count_launch();
}

#define TLS_CI(T)                                                                              \
  template void launch_dhd<T>(const T*, int64_t, const T*, const T*, T*, cudaStream_t);        \
  template void launch_power_finish<T>(T*, const T*, int64_t, double*, cudaStream_t);          \
  template void launch_power_init<T>(T*, int64_t, int64_t, cudaStream_t);                      \
  template int launch_frob_dw<T>(const T*, int64_t, int64_t, const T*, double*, cudaStream_t); \
  template void launch_vec_to_double<T>(const T*, double*, int64_t, int64_t, cudaStream_t);   \
  template void launch_features<T>(const double*, const T*, const T*, const T*, int64_t,       \
                                   int64_t, int64_t, double, double, int, double, int, double, \
                                   T*, T*, double*, float*, cudaStream_t);
TLS_CI(float)
TLS_CI(double)
#undef TLS_CI

}  // namespace tls
