// The selector network: a multilayer perceptron 16 -> 64 -> 64 -> 4 (ReLU hidden layers) that
// maps cheap per-problem features to three logits for the factor precision u_f
// (FP16 / BF16 / FP32) and a regression output, log10 of the inner PCGTLS tolerance.
//
// Parameters are kept in FP32 (the master copy the optimiser updates); every product uses the
// weights rounded to FP16 (the stored precision of the network) with FP32 accumulation.
// Flat parameter layout (5508 floats):
//   W1[64][16], b1[64], W2[64][64], b2[64], W3[4][64], b3[4].
//
// Training step (all on the device, deterministic):
//   mlp_grad_kernel    one warp per sample: forward, loss, backward; per-sample gradients to a
//                      scratch [batch][5508] (no atomics)
//   mlp_reduce_kernel  column sums over the batch in a fixed order -> mean gradient, mean loss
//   mlp_adam_kernel    Adam update of the master parameters
// Loss per sample: cross-entropy of softmax(logits) against the class label, plus
// lambda * mask * (out[3] - y_tol)^2.
#include "../../include/tls.h"
#include "tls_internal.h"
#include <cuda_fp16.h>

namespace tls {
namespace mlp {

constexpr int kIn = 16, kH = 64, kOut = 4, kCls = 3;
constexpr int oW1 = 0, oB1 = oW1 + kH * kIn, oW2 = oB1 + kH, oB2 = oW2 + kH * kH,
              oW3 = oB2 + kH, oB3 = oW3 + kOut * kH, kParams = oB3 + kOut;
static_assert(kParams == 5508, "parameter count");

namespace {

__device__ __forceinline__ float h16(float w) { return __half2float(__float2half_rn(w)); }

template <typename T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Forward pass of one sample by one warp. Lane j owns hidden units j and j + 32.
// h1, h2 (post-activation) are returned per lane; out[4] in every lane.
__device__ __forceinline__ void forward_warp(const float* __restrict__ P, const float* x,
                                             float h1[2], float h2[2], float out[kOut],
                                             float* sh1 /* smem 64 */) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int j = lane + 32 * u;
    float a = h16(P[oB1 + j]);
#pragma unroll
    for (int i = 0; i < kIn; ++i) a = fmaf(h16(P[oW1 + j * kIn + i]), x[i], a);
    h1[u] = fmaxf(a, 0.f);
    sh1[j] = h1[u];
  }
  __syncwarp();
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int j = lane + 32 * u;
    float a = h16(P[oB2 + j]);
    for (int i = 0; i < kH; ++i) a = fmaf(h16(P[oW2 + j * kH + i]), sh1[i], a);
    h2[u] = fmaxf(a, 0.f);
  }
#pragma unroll
  for (int o = 0; o < kOut; ++o) {
    float a = h16(P[oW3 + o * kH + lane]) * h2[0];
    a = fmaf(h16(P[oW3 + o * kH + lane + 32]), h2[1], a);
    out[o] = wsum(a) + h16(P[oB3 + o]);
  }
}

__global__ void __launch_bounds__(256) mlp_grad_kernel(
    const float* __restrict__ P, int nsamp, const float* __restrict__ X,
    const int* __restrict__ idx, const int* __restrict__ ycls, const float* __restrict__ ytol,
    const float* __restrict__ ymask, float lambda, float* __restrict__ G,
    float* __restrict__ loss) {
  __shared__ float sh1[8][kH];
  __shared__ float sdh2[8][kH];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * 8 + warp;
  if (s >= nsamp) return;   // warp-uniform
  const int row = idx ? idx[s] : s;
  float x[kIn];
#pragma unroll
  for (int i = 0; i < kIn; ++i) x[i] = X[(int64_t)row * kIn + i];
  float h1[2], h2[2], out[kOut];
  forward_warp(P, x, h1, h2, out, sh1[warp]);
  // loss and its gradient with respect to the outputs
  const int y = ycls[row];
  float mx = fmaxf(out[0], fmaxf(out[1], out[2]));
  float e0 = expf(out[0] - mx), e1 = expf(out[1] - mx), e2 = expf(out[2] - mx);
  const float z = e0 + e1 + e2;
  const float p[3] = {e0 / z, e1 / z, e2 / z};
  const float m = ymask[row];
  const float dt = out[3] - ytol[row];
  float dout[kOut];
#pragma unroll
  for (int c = 0; c < kCls; ++c) dout[c] = p[c] - (c == y ? 1.f : 0.f);
  dout[3] = 2.f * lambda * m * dt;
  float* g = G + (int64_t)s * kParams;
  if (lane == 0) loss[s] = (mx + logf(z) - out[y]) + lambda * m * dt * dt;
  // layer 3
#pragma unroll
  for (int o = 0; o < kOut; ++o) {
    g[oW3 + o * kH + lane] = dout[o] * h2[0];
    g[oW3 + o * kH + lane + 32] = dout[o] * h2[1];
  }
  if (lane < kOut) g[oB3 + lane] = dout[lane];
  // back to h2 (through ReLU)
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int j = lane + 32 * u;
    float d = 0.f;
#pragma unroll
    for (int o = 0; o < kOut; ++o) d = fmaf(h16(P[oW3 + o * kH + j]), dout[o], d);
    d = (h2[u] > 0.f) ? d : 0.f;
    sdh2[warp][j] = d;
    g[oB2 + j] = d;
    for (int i = 0; i < kH; ++i) g[oW2 + j * kH + i] = d * sh1[warp][i];
  }
  __syncwarp();
  // back to h1: dh1[i] = sum_j W2[j][i] dh2[j]
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int i = lane + 32 * u;
    float d = 0.f;
    for (int j = 0; j < kH; ++j) d = fmaf(h16(P[oW2 + j * kH + i]), sdh2[warp][j], d);
    d = (h1[u] > 0.f) ? d : 0.f;
    g[oB1 + i] = d;
#pragma unroll
    for (int k = 0; k < kIn; ++k) g[oW1 + i * kIn + k] = d * x[k];
  }
}

// mean over the batch of the per-sample gradients and losses (fixed summation order)
__global__ void mlp_reduce_kernel(const float* __restrict__ G, const float* __restrict__ loss,
                                  int nsamp, float* __restrict__ grad, float* __restrict__ lmean) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const float inv = 1.f / (float)nsamp;
  if (k < kParams) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    int s = 0;
    for (; s + 3 < nsamp; s += 4) {
      a0 += G[(int64_t)s * kParams + k];
      a1 += G[(int64_t)(s + 1) * kParams + k];
      a2 += G[(int64_t)(s + 2) * kParams + k];
      a3 += G[(int64_t)(s + 3) * kParams + k];
    }
    for (; s < nsamp; ++s) a0 += G[(int64_t)s * kParams + k];
    grad[k] = ((a0 + a1) + (a2 + a3)) * inv;
  }
  if (k == kParams && lmean) {
    float a = 0.f;
    for (int s = 0; s < nsamp; ++s) a += loss[s];
    *lmean = a * inv;
  }
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
__global__ void mlp_adam_kernel(float* __restrict__ P, const float* __restrict__ g,
                                float* __restrict__ m, float* __restrict__ v, int t, float lr,
                                float b1, float b2, float eps) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kParams) return;
  const float gk = g[k];
  const float mk = b1 * m[k] + (1.f - b1) * gk;
  const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  const float mh = mk / (1.f - powf(b1, (float)t));
  const float vh = vk / (1.f - powf(b2, (float)t));
  P[k] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void __launch_bounds__(256) mlp_forward_kernel(const float* __restrict__ P, int nsamp,
                                                          const float* __restrict__ X,
                                                          float* __restrict__ out) {
  __shared__ float sh1[8][kH];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * 8 + warp;
  if (s >= nsamp) return;
  float x[kIn];
#pragma unroll
  for (int i = 0; i < kIn; ++i) x[i] = X[(int64_t)s * kIn + i];
  float h1[2], h2[2], o[kOut];
  forward_warp(P, x, h1, h2, o, sh1[warp]);
  if (lane < kOut) out[(int64_t)s * kOut + lane] = o[lane];
}

}  // namespace

void launch_mlp_forward(const float* P, int nsamp, const float* X, float* out, cudaStream_t s) {
  if (nsamp <= 0) return;
  mlp_forward_kernel<<<(nsamp + 7) / 8, 256, 0, s>>>(P, nsamp, X, out);
  count_launch();
}

}  // namespace mlp
}  // namespace tls

extern "C" {

tls_status tls_mlp_grad(const float* params, int nsamp, const float* X, const int* idx,
                        const int* ycls, const float* ytol, const float* ymask, float lambda,
                        float* scratch, float* grad, float* loss_mean, void* stream) {
  using namespace tls::mlp;
  if (!params || nsamp < 1 || !X || !ycls || !ytol || !ymask || !scratch || !grad)
    return TLS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* G = scratch;
  float* loss = scratch + (size_t)nsamp * kParams;
  mlp_grad_kernel<<<(nsamp + 7) / 8, 256, 0, s>>>(params, nsamp, X, idx, ycls, ytol, ymask,
                                                  lambda, G, loss);
  mlp_reduce_kernel<<<(kParams + 1 + 255) / 256, 256, 0, s>>>(G, loss, nsamp, grad, loss_mean);
  tls::count_launch(2);
  return cudaGetLastError() == cudaSuccess ? TLS_OK : TLS_ERR_CUDA;
}

tls_status tls_mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr,
                        float beta1, float beta2, float eps, void* stream) {
  using namespace tls::mlp;
  if (!params || !grad || !m || !v || step < 1) return TLS_ERR_ARG;
  mlp_adam_kernel<<<(kParams + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      params, grad, m, v, step, lr, beta1, beta2, eps);
  tls::count_launch();
  return cudaGetLastError() == cudaSuccess ? TLS_OK : TLS_ERR_CUDA;
}

tls_status tls_mlp_forward(const float* params, int nsamp, const float* X, float* out,
                           void* stream) {
  if (!params || nsamp < 0 || (nsamp > 0 && (!X || !out))) return TLS_ERR_ARG;
  tls::mlp::launch_mlp_forward(params, nsamp, X, out, static_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? TLS_OK : TLS_ERR_CUDA;
}

}  // extern "C"
