// The FP64 RQI residual block without any device allocation (tls_residual_noalloc).
//
// Some callers may not allocate device memory themselves: an application whose framework
// allocator has already reserved the GPU's memory and must account for every byte, a
// latency-critical loop in which cudaMalloc / cudaFree (which can synchronise the device) are
// not acceptable, or a plug-in that is handed its buffers and may create nothing. For them this
// entry point keeps all of its scratch in one file-scope device array of fixed size, which
// every GPU that loads the library holds until the process exits.
//
// Host code never uses the array's name as a device address: the device address is looked up
// once per device with cudaGetSymbolAddress (with that device current) and cached.
#include "../../include/tls.h"
#include "tls_internal.h"

#include <algorithm>
#include <mutex>

namespace tls {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaCtas = 64;                      // CTAs of the pass over A (partials)
constexpr int64_t kNaMaxN = TLS_NOALLOC_MAX_N;   // largest n accepted
constexpr int kNaCols = (int)(kNaMaxN / kNaThreads);   // columns per thread at the limit
constexpr int kNaRows = 4;                       // rows reduced per block barrier

// Scratch layout (doubles): partials kNaCtas x kNaMaxN, pass scalars kNaCtas x 2, ||x||^2,
// reduction partials kNaMaxN / 32, then two unsigned counters.
constexpr size_t kOffPart = 0;
constexpr size_t kOffSpart = kOffPart + (size_t)kNaCtas * kNaMaxN;
constexpr size_t kOffXX = kOffSpart + (size_t)kNaCtas * 2;
constexpr size_t kOffFpart = kOffXX + 1;
constexpr size_t kOffCounters = kOffFpart + (size_t)(kNaMaxN / 32);
constexpr size_t kScratchDoubles = kOffCounters + 2;   // counters fit in the last two doubles
static_assert(kScratchDoubles * 8 <= TLS_NOALLOC_SCRATCH_BYTES, "scratch size");

__device__ __align__(256) unsigned char g_noalloc_scratch[TLS_NOALLOC_SCRATCH_BYTES];

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// r_i = b_i - A_i x for the CTA's rows; partial sums of r_i A_i, r^T r, b^T r; ||x||^2.
__global__ void __launch_bounds__(kNaThreads) na_pass_kernel(const double* __restrict__ A,
                                                             int64_t lda, int64_t m, int64_t n,
                                                             const double* __restrict__ b,
                                                             const double* __restrict__ x,
                                                             double* __restrict__ scratch) {
  __shared__ double red[kNaThreads / 32][kNaRows];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double xv[kNaCols], acc[kNaCols];
  double xx = 0.0;
#pragma unroll
  for (int k = 0; k < kNaCols; ++k) {
    const int64_t c = (int64_t)k * kNaThreads + tid;
    xv[k] = (c < n) ? x[c] : 0.0;
    acc[k] = 0.0;
    xx = fma(xv[k], xv[k], xx);
  }
  const int64_t per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(m, r0 + per);
  double rr = 0.0, br = 0.0;
  for (int64_t i0 = r0; i0 < r1; i0 += kNaRows) {
    double dot[kNaRows];
#pragma unroll
    for (int q = 0; q < kNaRows; ++q) {
      double t = 0.0;
      const int64_t i = i0 + q;
      if (i < r1) {
#pragma unroll
        for (int k = 0; k < kNaCols; ++k) {
          const int64_t c = (int64_t)k * kNaThreads + tid;
          if (c < n) t = fma(A[i * lda + c], xv[k], t);
        }
      }
      dot[q] = na_warp_sum(t);
    }
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < kNaRows; ++q) red[warp][q] = dot[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kNaRows; ++q) {
      const int64_t i = i0 + q;
      if (i >= r1) break;
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < kNaThreads / 32; ++w) s += red[w][q];
      const double ri = b[i] - s;
      if (tid == 0) {
        rr = fma(ri, ri, rr);
        br = fma(b[i], ri, br);
      }
#pragma unroll
      for (int k = 0; k < kNaCols; ++k) {
        const int64_t c = (int64_t)k * kNaThreads + tid;
        if (c < n) acc[k] = fma(ri, A[i * lda + c], acc[k]);
      }
    }
    __syncthreads();
  }
  double* part = scratch + kOffPart + (size_t)blockIdx.x * kNaMaxN;
#pragma unroll
  for (int k = 0; k < kNaCols; ++k) {
    const int64_t c = (int64_t)k * kNaThreads + tid;
    if (c < n) part[c] = acc[k];
  }
  if (tid == 0) {
    scratch[kOffSpart + 2 * blockIdx.x] = rr;
    scratch[kOffSpart + 2 * blockIdx.x + 1] = br;
  }
  if (blockIdx.x == 0) {
    // ||x||^2 (every CTA holds all of x; CTA 0 publishes it)
    xx = na_warp_sum(xx);
    __shared__ double xs[kNaThreads / 32];
    if (lane == 0) xs[warp] = xx;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kNaThreads / 32; ++w) t += xs[w];
      scratch[kOffXX] = t;
    }
  }
}

// f_j = -(A^T r)_j - sigma^2 x_j; the last CTA forms sigma^2, g, psi into scal[0..4].
__global__ void __launch_bounds__(kNaThreads) na_reduce_kernel(int P, int64_t n,
                                                               const double* __restrict__ x,
                                                               double* __restrict__ f,
                                                               double* __restrict__ scal,
                                                               double* __restrict__ scratch) {
  __shared__ double sh[kNaThreads / 32][33];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * 32 + lane;
  double rr = 0.0, br = 0.0;
  for (int p = 0; p < P; ++p) {
    rr += scratch[kOffSpart + 2 * p];
    br += scratch[kOffSpart + 2 * p + 1];
  }
  const double xx = scratch[kOffXX];
  const double sigma2 = rr / (1.0 + xx);
  double t = 0.0;
  if (j < n)
    for (int p = warp; p < P; p += kNaThreads / 32) t += scratch[kOffPart + (size_t)p * kNaMaxN + j];
  sh[warp][lane] = t;
  __syncthreads();
  if (warp == 0) {
    double at = 0.0;
#pragma unroll
    for (int w = 0; w < kNaThreads / 32; ++w) at += sh[w][lane];
    double ff = 0.0;
    if (j < n) {
      const double fj = -at - sigma2 * x[j];
      f[j] = fj;
      ff = fj * fj;
    }
    ff = na_warp_sum(ff);
    if (lane == 0) scratch[kOffFpart + blockIdx.x] = ff;
  }
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kOffCounters);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double ff = 0.0;
    for (unsigned int bl = 0; bl < gridDim.x; ++bl) ff += __ldcg(scratch + kOffFpart + bl);
    const double g = -br + sigma2;
    scal[0] = sigma2;
    scal[1] = g;
    scal[2] = sqrt((ff + g * g) / (xx + 1.0));
    scal[3] = rr;
    scal[4] = br;
    *counter = 0u;
  }
}

std::mutex g_na_mutex;
void* g_na_ptr[64] = {};   // device address of the scratch array, per device ordinal

}  // namespace
}  // namespace tls

extern "C" tls_status tls_residual_noalloc(int64_t m, int64_t n, const double* A, int64_t lda,
                                           const double* b, const double* x, double* f,
                                           double* scal, void* stream) {
  using namespace tls;
  if (m < 1 || n < 1 || n > kNaMaxN || lda < n || !A || !b || !x || !f || !scal)
    return TLS_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TLS_ERR_CUDA;
  void* base = nullptr;
  {
    // set-up on the first call for this device (the device is current here)
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        (void)cudaGetLastError();
        return TLS_ERR_CUDA;
      }
      g_na_ptr[dev] = p;
    }
    base = g_na_ptr[dev];
  }
  double* scratch = static_cast<double*>(base);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the last-block counter must start at zero (the array keeps the previous call's contents)
  if (cudaMemsetAsync(scratch + kOffCounters, 0, 2 * sizeof(double), s) != cudaSuccess)
    return TLS_ERR_CUDA;
  const int P = (int)std::min<int64_t>(kNaCtas, std::max<int64_t>(1, (m + kNaRows - 1) / kNaRows));
  na_pass_kernel<<<P, kNaThreads, 0, s>>>(A, lda, m, n, b, x, scratch);
  count_launch();
  na_reduce_kernel<<<(unsigned)((n + 31) / 32), kNaThreads, 0, s>>>(P, n, x, f, scal, scratch);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? TLS_OK : TLS_ERR_CUDA;
}
