// Sparse (CSR) A: the kernels of RQI-PCGTLS (Oktay & Carson, arXiv 2305.19028, Alg. 2-4) that
// touch A, for A held twice on the device -- by rows (CSR) and by columns (CSC, a transposed
// index built at creation) -- so that both A v and A^T v are gathers in a fixed order:
//  * column norms D = diag(||a_j||) and the u_f-rounded scaled values A D^{-1} (Sec. 3.1);
//  * the Gram matrix H = A_s^T A_s (one CTA per column i accumulates row i of H);
//  * the FP64 RQI residual: r = b - A x (rows), f = -A^T r - sigma^2 x (columns), g, psi;
//  * the PCGTLS operator: t = A q (rows, two right-hand sides), then A^T t with the Alg. 3
//    updates w += alpha q, y = D^{-1}(A^T t - sigma^2 q) (columns).
#include "tls_internal.h"
#include "tls_device.cuh"

#include <algorithm>

namespace tls {

namespace {

constexpr int kT = 256;
constexpr int kW = kT / 32;

template <typename T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ bool last_block(unsigned int* counter) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x * gridDim.y - 1);
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// sum of K interleaved partials part[p*K + k], p < P, by the whole block; thread 0 writes out[k]
template <int K>
__device__ __forceinline__ void sum_partials(const double* part, int P, double* out) {
  __shared__ double sh[kW * K];
  double v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = 0.0;
  for (int p = threadIdx.x; p < P; p += blockDim.x)
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] += __ldcg(part + (int64_t)p * K + k);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = wsum(v[k]);
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
// Factor-side kernels
// ---------------------------------------------------------------------------------------
__global__ void vals_to_f32_kernel(const double* __restrict__ v64, float* __restrict__ v32,
                                   int64_t nnz) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nnz) v32[k] = f64_to_f32_rn(v64[k]);
}

// d_j = ||a_j|| from the CSC values (one warp per column, fixed order); fp32: FP32 accumulation
// over the FP32 working copy, else FP64 over the FP64 values.
__global__ void csc_colnorm_kernel(const int* __restrict__ cp, const double* __restrict__ cv64,
                                   const float* __restrict__ cv32, int64_t n, int64_t npad,
                                   double* __restrict__ d, double* __restrict__ dinv,
                                   float* __restrict__ dinv32) {
  const int lane = threadIdx.x & 31;
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= npad) return;
  double dd = 1.0;
  if (j < n) {
    const int k0 = cp[j], k1 = cp[j + 1];
    if (cv32 != nullptr) {
      float s = 0.f;
      for (int k = k0 + lane; k < k1; k += 32) s = fmaf(cv32[k], cv32[k], s);
      s = wsum(s);
      dd = sqrt((double)s);
    } else {
      double s = 0.0;
      for (int k = k0 + lane; k < k1; k += 32) s = fma(cv64[k], cv64[k], s);
      s = wsum(s);
      dd = sqrt(s);
    }
    if (!(dd > 0.0)) dd = 1.0;
  }
  if (lane == 0) {
    d[j] = dd;
    dinv[j] = 1.0 / dd;
    dinv32[j] = (float)(1.0 / dd);
  }
}

template <typename T> __device__ __forceinline__ T round_to(T v, int prec);
template <> __device__ __forceinline__ float round_to<float>(float v, int prec) {
  if (prec == (int)Prec::FP16) return __half2float(__float2half_rn(v));
  if (prec == (int)Prec::BF16) return __bfloat162float(__float2bfloat16_rn(v));
  return v;
}

// scaled, rounded values in CSR order: as[k] = fl_uf(a_k / d_col(k))
template <typename T>
__global__ void csr_scale_kernel(const int* __restrict__ ci, const float* __restrict__ v32,
                                 const double* __restrict__ v64, const float* __restrict__ dinv32,
                                 const double* __restrict__ dinv, int64_t nnz, int prec,
                                 T* __restrict__ as) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  const int c = ci[k];
  if constexpr (sizeof(T) == 4) as[k] = round_to<float>(v32[k] * dinv32[c], prec);
  else as[k] = v64[k] * dinv[c];
}

// the same in CSC order (one warp per column)
template <typename T>
__global__ void csc_scale_kernel(const int* __restrict__ cp, const float* __restrict__ cv32,
                                 const double* __restrict__ cv64, const float* __restrict__ dinv32,
                                 const double* __restrict__ dinv, int64_t n, int prec,
                                 T* __restrict__ cas) {
  const int lane = threadIdx.x & 31;
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= n) return;
  for (int k = cp[j] + lane; k < cp[j + 1]; k += 32) {
    if constexpr (sizeof(T) == 4) cas[k] = round_to<float>(cv32[k] * dinv32[j], prec);
    else cas[k] = cv64[k] * dinv[j];
  }
}

// Row i of H = A_s^T A_s (entries j >= i), one CTA per column i: for every entry (r, a_ri) of
// column i and every entry (r, a_rj) of row r with j >= i, add a_ri a_rj into a shared row
// accumulator (shared-memory atomics: the summation order of an entry of H is not fixed, so H
// is reproducible to FP32 rounding, not bitwise). The row and its mirror are then stored.
template <typename T>
__global__ void __launch_bounds__(kT) sparse_gram_kernel(const int* __restrict__ rp,
                                                         const int* __restrict__ ci,
                                                         const T* __restrict__ as,
                                                         const int* __restrict__ cp,
                                                         const int* __restrict__ ri,
                                                         const T* __restrict__ cas, int64_t n,
                                                         int64_t npad, T* __restrict__ H) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* hrow = reinterpret_cast<T*>(smraw);
  const int64_t i = blockIdx.x;
  for (int64_t c = threadIdx.x; c < npad; c += kT) hrow[c] = T(0);
  __syncthreads();
  if (i < n) {
    for (int k = cp[i] + threadIdx.x; k < cp[i + 1]; k += kT) {
      const int r = ri[k];
      const T a = cas[k];
      const int e1 = rp[r + 1];
      for (int e = rp[r]; e < e1; ++e) {
        const int c = ci[e];
        if (c >= i) atomicAdd(&hrow[c], a * as[e]);
      }
    }
  }
  __syncthreads();
  for (int64_t c = i + threadIdx.x; c < npad; c += kT) {
    T v = hrow[c];
    if (i >= n && c == i) v = T(1);      // identity on the padded diagonal
    H[i * npad + c] = v;
    H[c * npad + i] = v;
  }
}

// ---------------------------------------------------------------------------------------
// FP64 RQI residual: r = b - A x by rows (thread per row), r^T r and b^T r per CTA
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kT) csr_resid_kernel(const int* __restrict__ rp,
                                                       const int* __restrict__ ci,
                                                       const double* __restrict__ v64,
                                                       const double* __restrict__ b,
                                                       const double* __restrict__ x, int64_t m,
                                                       double* __restrict__ r,
                                                       double* __restrict__ spart,
                                                       double* __restrict__ sout,
                                                       unsigned int* counter) {
  const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  double rr = 0.0, br = 0.0;
  if (i < m) {
    double s = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) s = fma(v64[e], x[ci[e]], s);
    const double ri = b[i] - s;
    r[i] = ri;
    rr = ri * ri;
    br = b[i] * ri;
  }
  __shared__ double sh[kW][2];
  rr = wsum(rr);
  br = wsum(br);
  if ((threadIdx.x & 31) == 0) { sh[threadIdx.x >> 5][0] = rr; sh[threadIdx.x >> 5][1] = br; }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0.0;
    for (int w = 0; w < kW; ++w) t += sh[w][threadIdx.x];
    spart[(int64_t)blockIdx.x * 2 + threadIdx.x] = t;
  }
  if (last_block(counter)) {
    sum_partials<2>(spart, (int)gridDim.x, sout);
    if (threadIdx.x == 0) *counter = 0u;
  }
}

// f_j = -(A^T r)_j - sigma^2 x_j (one warp per column), ||f||^2, then g and psi (last CTA)
__global__ void __launch_bounds__(kT) csc_resid_kernel(const int* __restrict__ cp,
                                                       const int* __restrict__ ri,
                                                       const double* __restrict__ cv64,
                                                       const double* __restrict__ r,
                                                       const double* __restrict__ x, int64_t n,
                                                       int64_t npad, double* __restrict__ f,
                                                       const double* __restrict__ sout,
                                                       RqiScalars* rs, double* __restrict__ fpart) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * kW + warp;
  const double xx = rs->xx;
  const double sigma2 = sout[0] / (1.0 + xx);
  double ff = 0.0;
  if (j < npad) {
    double s = 0.0;
    if (j < n)
      for (int k = cp[j] + lane; k < cp[j + 1]; k += 32) s = fma(cv64[k], r[ri[k]], s);
    s = wsum(s);
    if (lane == 0) {
      const double fj = (j < n) ? (-s - sigma2 * x[j]) : 0.0;
      f[j] = fj;
      ff = fj * fj;
    }
  }
  __shared__ double sh[kW];
  if (lane == 0) sh[warp] = ff;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kW; ++w) t += sh[w];
    fpart[blockIdx.x] = t;
  }
  if (last_block(&rs->counter[0])) {
    __shared__ double tfs[1];
    sum_partials<1>(fpart, (int)gridDim.x, tfs);
    if (threadIdx.x == 0) {
      const double rr = sout[0], br = sout[1];
      const double g = -br + sigma2;
      rs->rr = rr;
      rs->br = br;
      rs->sigma2 = sigma2;
      rs->g = g;
      rs->ff = tfs[0];
      rs->psi = sqrt((tfs[0] + g * g) / (xx + 1.0));
      rs->counter[0] = 0u;
    }
  }
}

// ---------------------------------------------------------------------------------------
// PCGTLS operator, u type T: t = A q (rows, 2 RHS) and ||t||^2, then A^T t with the updates
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kT) csr_tq_kernel(const int* __restrict__ rp,
                                                    const int* __restrict__ ci,
                                                    const T* __restrict__ val,
                                                    const T* __restrict__ q, int64_t m,
                                                    int64_t npad, int nr, T* __restrict__ t,
                                                    double* __restrict__ spart,
                                                    double* __restrict__ sout,
                                                    unsigned int* counter,
                                                    const int* __restrict__ done) {
  if (done[0] && (nr < 2 || done[1])) return;
  const int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x;
  T t0 = T(0), t1 = T(0);
  if (i < m) {
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      const int c = ci[e];
      const T a = val[e];
      t0 = fma(a, q[c], t0);
      if (nr > 1) t1 = fma(a, q[npad + c], t1);
    }
    t[i] = t0;
    if (nr > 1) t[m + i] = t1;
  }
  T s0 = wsum(t0 * t0), s1 = wsum(t1 * t1);
  __shared__ T sh[kW][2];
  if ((threadIdx.x & 31) == 0) { sh[threadIdx.x >> 5][0] = s0; sh[threadIdx.x >> 5][1] = s1; }
  __syncthreads();
  if (threadIdx.x < 2) {
    T a = T(0);
    for (int w = 0; w < kW; ++w) a += sh[w][threadIdx.x];
    spart[(int64_t)blockIdx.x * 4 + threadIdx.x * 2] = (double)a;   // layout [r][2] as sout
    spart[(int64_t)blockIdx.x * 4 + threadIdx.x * 2 + 1] = 0.0;
  }
  if (last_block(counter)) {
    sum_partials<4>(spart, (int)gridDim.x, sout);
    if (threadIdx.x == 0) *counter = 0u;
  }
}

template <typename T>
__global__ void __launch_bounds__(kT) csc_pcg_kernel(const int* __restrict__ cp,
                                                     const int* __restrict__ ri,
                                                     const T* __restrict__ cval,
                                                     const T* __restrict__ t, int64_t m,
                                                     int64_t n, int64_t npad, int nr,
                                                     const T* __restrict__ q, T* __restrict__ w,
                                                     T* __restrict__ y,
                                                     const T* __restrict__ dinv, PcgScalars* sc,
                                                     const double* __restrict__ tt) {
  __shared__ T s_alpha[2], s_sigma2;
  __shared__ int s_ok[2];
  if (threadIdx.x < 2) {
    const int r = threadIdx.x;
    // delta_j and alpha_j once per CTA, in FP64 on one thread
    int ok = 0;
    double alpha = 0.0;
    if (r < nr && !sc->done[r]) {
      const double delta = tt[r * 2] - sc->sigma2 * sc->qq[r];
      if (blockIdx.x == 0) sc->delta[r] = delta;
      ok = delta > 0.0;
      if (ok) {
        alpha = sc->eta[r] / delta;
        if (blockIdx.x == 0) sc->alpha[r] = alpha;
      }
    }
    s_ok[r] = ok;
    s_alpha[r] = (T)alpha;
    if (r == 0) s_sigma2 = (T)sc->sigma2;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * kW + warp;
  if (j >= npad) return;
  T a0 = T(0), a1 = T(0);
  if (j < n) {
    for (int k = cp[j] + lane; k < cp[j + 1]; k += 32) {
      const int rr = ri[k];
      const T v = cval[k];
      a0 = fma(v, t[rr], a0);
      if (nr > 1) a1 = fma(v, t[m + rr], a1);
    }
  }
  a0 = wsum(a0);
  if (nr > 1) a1 = wsum(a1);
  if (lane < nr) {
    const int r = lane;
    if (s_ok[r]) {
      const T at = (r == 0) ? a0 : a1;
      const T qj = q[r * npad + j];
      w[r * npad + j] = fma(s_alpha[r], qj, w[r * npad + j]);
      y[r * npad + j] = (at - s_sigma2 * qj) * dinv[j];
    }
  }
}

inline int nblk(int64_t count, int threads) { return (int)((count + threads - 1) / threads); }

// ---------------------------------------------------------------------------------------
// The column (CSC) index, built on the device from the uploaded CSR arrays: a stable counting
// sort of the entries by column (entries of a column in increasing row order). The row ranges
// are split over G CTAs of W warps, warp g of all G W taking rows [m g / (G W), m (g+1) / (G W)).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void warp_rows(int64_t m, int W, int64_t* r0, int64_t* r1) {
  const int64_t g = (int64_t)blockIdx.x * W + (threadIdx.x >> 5);
  const int64_t GW = (int64_t)gridDim.x * W;
  *r0 = m * g / GW;
  *r1 = m * (g + 1) / GW;
}

// Structure and value check, one warp per row: row offsets non-decreasing from 0 to nnz,
// column indices in [0, n) and strictly increasing within the row, values and b finite. Writes
// the 32-bit row offsets. *bad = 1 on any violation (nothing below runs on a bad structure).
__global__ void __launch_bounds__(kT) csr_check_kernel(const int64_t* __restrict__ rp64,
                                                       const int* __restrict__ ci,
                                                       const double* __restrict__ v64,
                                                       const double* __restrict__ b, int64_t m,
                                                       int64_t n, int64_t nnz,
                                                       int* __restrict__ rp32,
                                                       int* __restrict__ bad) {
  const int64_t r = (int64_t)blockIdx.x * kW + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= m) return;
  const int64_t lo = rp64[r], hi = rp64[r + 1];
  bool err = lo < 0 || hi < lo || hi > nnz;
  if (!err) {
    for (int64_t e = lo + lane; e < hi; e += 32) {
      const int c = ci[e];
      err |= c < 0 || c >= n || !isfinite(v64[e]) || (e > lo && ci[e - 1] >= c);
    }
  }
  if (lane == 0) {
    err |= !isfinite(b[r]);
    rp32[r] = (int)lo;
    if (r == m - 1) rp32[m] = (int)nnz;
  }
  if (__any_sync(0xffffffffu, err) && lane == 0) atomicOr(bad, 1);
}

// Column counts of each CTA's rows: cnt[blockIdx.x * npad + c]. Dynamic shared memory: W
// counters of npad ints (one set per warp, summed at the end).
__global__ void __launch_bounds__(kT) csc_count_kernel(const int* __restrict__ rp32,
                                                       const int* __restrict__ ci, int64_t m,
                                                       int64_t npad, int W,
                                                       int* __restrict__ cnt) {
  extern __shared__ int sc_cnt[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t k = threadIdx.x; k < (int64_t)W * npad; k += blockDim.x) sc_cnt[k] = 0;
  __syncthreads();
  if (warp < W) {
    int64_t r0, r1;
    warp_rows(m, W, &r0, &r1);
    int* mine = sc_cnt + (int64_t)warp * npad;
    for (int64_t e = rp32[r0] + lane; e < rp32[r1]; e += 32) atomicAdd(&mine[ci[e]], 1);
  }
  __syncthreads();
  for (int64_t c = threadIdx.x; c < npad; c += blockDim.x) {
    int t = 0;
    for (int w = 0; w < W; ++w) t += sc_cnt[(int64_t)w * npad + c];
    cnt[(int64_t)blockIdx.x * npad + c] = t;
  }
}

// Per column: off[g * npad + c] = entries of column c in CTAs before g; tot[c] = all of them.
__global__ void csc_colscan_kernel(const int* __restrict__ cnt, int G, int64_t npad,
                                   int* __restrict__ off, int* __restrict__ tot) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= npad) return;
  int run = 0;
#pragma unroll 8
  for (int g = 0; g < G; ++g) {
    const int t = cnt[(int64_t)g * npad + c];
    off[(int64_t)g * npad + c] = run;
    run += t;
  }
  tot[c] = run;
}

// cp[0..npad] = exclusive prefix sums of tot (one CTA of 1024 threads).
__global__ void __launch_bounds__(1024) csc_ptr_kernel(const int* __restrict__ tot, int64_t npad,
                                                       int* __restrict__ cp) {
  __shared__ int wsums[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t per = (npad + 1023) / 1024;
  const int64_t c0 = tid * per, c1 = min(npad, c0 + per);
  int seg = 0;
  for (int64_t c = c0; c < c1; ++c) seg += tot[c];
  // exclusive scan of the segment sums over the block
  int incl = seg;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = wsums[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += v;
    }
    wsums[lane] = w;
  }
  __syncthreads();
  int run = incl - seg + (warp > 0 ? wsums[warp - 1] : 0);
  for (int64_t c = c0; c < c1; ++c) {
    cp[c] = run;
    run += tot[c];
  }
  if (tid == 1023) cp[npad] = run;
}

// Scatter: each warp walks its rows in order and places row r's entries at the next free slot
// of their columns, starting from cp[c] + off[cta][c] + the counts of the CTA's earlier warps.
// (Columns are distinct within a row, so the lanes of one row never share a counter; the warp
// synchronises between rows so that a later row sees the earlier rows' increments.)
__global__ void __launch_bounds__(kT) csc_scatter_kernel(const int* __restrict__ rp32,
                                                         const int* __restrict__ ci,
                                                         const double* __restrict__ v64,
                                                         int64_t m, int64_t npad, int64_t nnz,
                                                         int W, const int* __restrict__ cp,
                                                         const int* __restrict__ off,
                                                         int* __restrict__ ri,
                                                         double* __restrict__ cv) {
  extern __shared__ int sc_cnt[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t k = threadIdx.x; k < (int64_t)W * npad; k += blockDim.x) sc_cnt[k] = 0;
  __syncthreads();
  int64_t r0 = 0, r1 = 0;
  if (warp < W) {
    warp_rows(m, W, &r0, &r1);
    int* mine = sc_cnt + (int64_t)warp * npad;
    for (int64_t e = rp32[r0] + lane; e < rp32[r1]; e += 32) atomicAdd(&mine[ci[e]], 1);
  }
  __syncthreads();
  for (int64_t c = threadIdx.x; c < npad; c += blockDim.x) {
    int run = cp[c] + off[(int64_t)blockIdx.x * npad + c];
    for (int w = 0; w < W; ++w) {
      const int t = sc_cnt[(int64_t)w * npad + c];
      sc_cnt[(int64_t)w * npad + c] = run;
      run += t;
    }
  }
  __syncthreads();
  if (warp >= W) return;
  int* next = sc_cnt + (int64_t)warp * npad;
  for (int64_t r = r0; r < r1; ++r) {
    const int lo = rp32[r], hi = rp32[r + 1];
    for (int e = lo + lane; e < hi; e += 32) {
      const int c = ci[e];
      const int pos = next[c];
      next[c] = pos + 1;
      if (pos < nnz) {
        ri[pos] = (int)r;
        cv[pos] = v64[e];
      }
    }
    __syncwarp();
  }
}

}  // namespace

int csc_build_warps(int64_t npad) {
  const int64_t w = (int64_t)(200 * 1024) / (npad * (int64_t)sizeof(int));
  return (int)std::min<int64_t>(kW, w);
}

void csr_check(const int64_t* rp64, const int* ci, const double* v64, const double* b, int64_t m,
               int64_t n, int64_t nnz, int* rp32, int* bad, cudaStream_t s) {
  csr_check_kernel<<<nblk(m, kW), kT, 0, s>>>(rp64, ci, v64, b, m, n, nnz, rp32, bad);
  count_launch();
}

void csc_build(const int* rp32, const int* ci, const double* v64, int64_t m, int64_t npad,
               int64_t nnz, int G, int* cnt, int* off, int* tot, int* cp, int* ri, double* cv,
               cudaStream_t s) {
  const int W = csc_build_warps(npad);
  const size_t smem = sizeof(int) * (size_t)W * (size_t)npad;
  static const bool attr = [] {
    cudaFuncSetAttribute(csc_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(csc_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    return true;
  }();
  (void)attr;
  csc_count_kernel<<<G, kT, smem, s>>>(rp32, ci, m, npad, W, cnt);
  csc_colscan_kernel<<<nblk(npad, 256), 256, 0, s>>>(cnt, G, npad, off, tot);
  csc_ptr_kernel<<<1, 1024, 0, s>>>(tot, npad, cp);
  csc_scatter_kernel<<<G, kT, smem, s>>>(rp32, ci, v64, m, npad, nnz, W, cp, off, ri, cv);
  count_launch(4);
}

// =========================================================================================
void sparse_to_f32(const double* v64, float* v32, int64_t nnz, cudaStream_t s) {
  if (nnz > 0) { vals_to_f32_kernel<<<nblk(nnz, 256), 256, 0, s>>>(v64, v32, nnz); count_launch(); }
}

void sparse_colnorm(const int* cp, const double* cv64, const float* cv32, int64_t n, int64_t npad,
                    double* d, double* dinv, float* dinv32, cudaStream_t s) {
  csc_colnorm_kernel<<<nblk(npad * 32, 256), 256, 0, s>>>(cp, cv64, cv32, n, npad, d, dinv, dinv32);
  count_launch();
}

template <typename T>
void sparse_gram(const int* rp, const int* ci, const float* v32, const double* v64,
                 const int* cp, const int* ri, const float* cv32, const double* cv64,
                 const float* dinv32, const double* dinv, int64_t n, int64_t npad, int64_t nnz,
                 Prec prec, T* as, T* cas, T* H, cudaStream_t s) {
  if (nnz > 0) {
    csr_scale_kernel<T><<<nblk(nnz, 256), 256, 0, s>>>(ci, v32, v64, dinv32, dinv, nnz, (int)prec, as);
    count_launch();
    csc_scale_kernel<T><<<nblk(n * 32, 256), 256, 0, s>>>(cp, cv32, cv64, dinv32, dinv, n, (int)prec, cas);
    count_launch();
  }
  const size_t smem = sizeof(T) * (size_t)npad;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(sparse_gram_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  sparse_gram_kernel<T><<<(unsigned)npad, kT, smem, s>>>(rp, ci, as, cp, ri, cas, n, npad, H);
  count_launch();
}

void sparse_resid(const int* rp, const int* ci, const double* v64, const int* cp, const int* ri,
                  const double* cv64, const double* b, const double* x, int64_t m, int64_t n,
                  int64_t npad, double* r, double* f, double* spart, double* sout,
                  unsigned int* counter, RqiScalars* rs, double* fpart, cudaStream_t s) {
  csr_resid_kernel<<<nblk(m, kT), kT, 0, s>>>(rp, ci, v64, b, x, m, r, spart, sout, counter);
  count_launch();
  csc_resid_kernel<<<nblk(npad, kW), kT, 0, s>>>(cp, ri, cv64, r, x, n, npad, f, sout, rs, fpart);
  count_launch();
}

template <typename T>
void sparse_pcg_pass(const int* rp, const int* ci, const T* val, const int* cp, const int* ri,
                     const T* cval, int64_t m, int64_t n, int64_t npad, int nr, const T* q, T* t,
                     T* w, T* y, const T* dinv, PcgScalars* sc, double* spart, double* sout,
                     unsigned int* counter, const int* done, cudaStream_t s) {
  csr_tq_kernel<T><<<nblk(m, kT), kT, 0, s>>>(rp, ci, val, q, m, npad, nr, t, spart, sout, counter, done);
  count_launch();
  csc_pcg_kernel<T><<<nblk(npad, kW), kT, 0, s>>>(cp, ri, cval, t, m, n, npad, nr, q, w, y, dinv, sc, sout);
  count_launch();
}

int sparse_grid_rows(int64_t m) { return nblk(m, kT); }

template void sparse_gram<float>(const int*, const int*, const float*, const double*, const int*,
                                 const int*, const float*, const double*, const float*,
                                 const double*, int64_t, int64_t, int64_t, Prec, float*, float*,
                                 float*, cudaStream_t);
template void sparse_gram<double>(const int*, const int*, const float*, const double*, const int*,
                                  const int*, const float*, const double*, const float*,
                                  const double*, int64_t, int64_t, int64_t, Prec, double*, double*,
                                  double*, cudaStream_t);
template void sparse_pcg_pass<float>(const int*, const int*, const float*, const int*, const int*,
                                     const float*, int64_t, int64_t, int64_t, int, const float*,
                                     float*, float*, float*, const float*, PcgScalars*, double*,
                                     double*, unsigned int*, const int*, cudaStream_t);
template void sparse_pcg_pass<double>(const int*, const int*, const double*, const int*,
                                      const int*, const double*, int64_t, int64_t, int64_t, int,
                                      const double*, double*, double*, double*, const double*,
                                      PcgScalars*, double*, double*, unsigned int*, const int*,
                                      cudaStream_t);

}  // namespace tls
