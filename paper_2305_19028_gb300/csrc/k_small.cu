// RQI-PCGTLS for a small dense problem in one CTA (all in FP64, u = u_r = FP64): the LS start,
// the inverse-iteration step and the RQI loop of Alg. 2 with the paired PCGTLS solves of Alg. 3
// (A-explicit operator, k+1 steps in RQI step k), the same steps and stop rules as the
// multi-kernel path of the dense solve, with A, b and W = R_H^{-1} held in shared memory.
// For problems whose whole state fits in one SM the multi-kernel path is bound by launch and
// host round-trip latency (about 60 launches per solve); here one launch does the solve.
#include "../../include/tls.h"
#include "tls_internal.h"

namespace tls {

namespace {

constexpr int kST = 512;              // threads
constexpr int kSW = kST / 32;

__device__ __forceinline__ double swsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums of K values over the CTA; every thread receives the totals. sh: kSW * K doubles.
template <int K>
__device__ __forceinline__ void csum(double (&v)[K], double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = swsum(v[k]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[warp * K + k] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = swsum(lane < kSW ? sh[lane * K + k] : 0.0);
}

struct Small {
  const double* A;   // m x n (row stride n), shared
  const double* b;   // m
  const double* W;   // n x n upper triangular (row stride n)
  const double* dv;  // 1 / d
  int m, n;
  double* red;       // kSW * 4
  double* part;      // G x 2 x n partial column sums
  int G;             // row groups of the A^T products
};

// t_r = A q_r (r < nr), one thread per row; q: nr x n, t: nr x m
__device__ void mat_A(const Small& S, const double* q, double* t, int nr) {
  for (int i = threadIdx.x; i < S.m; i += kST) {
    const double* a = S.A + (int64_t)i * S.n;
    double t0 = 0.0, t1 = 0.0;
    for (int j = 0; j < S.n; ++j) {
      t0 = fma(a[j], q[j], t0);
      if (nr > 1) t1 = fma(a[j], q[S.n + j], t1);
    }
    t[i] = t0;
    if (nr > 1) t[S.m + i] = t1;
  }
}

// v_r = A^T t_r: thread (group g, column j) sums the rows i = g (mod G), then n threads add the
// G partials
__device__ void mat_At(const Small& S, const double* t, double* v, int nr) {
  const int g = threadIdx.x / S.n, j = threadIdx.x % S.n;
  if (g < S.G) {
    double a0 = 0.0, a1 = 0.0;
    for (int i = g; i < S.m; i += S.G) {
      const double aij = S.A[(int64_t)i * S.n + j];
      a0 = fma(aij, t[i], a0);
      if (nr > 1) a1 = fma(aij, t[S.m + i], a1);
    }
    S.part[(g * 2 + 0) * S.n + j] = a0;
    S.part[(g * 2 + 1) * S.n + j] = a1;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nr * S.n; e += kST) {
    const int r = e / S.n, jj = e % S.n;
    double a = 0.0;
    for (int gg = 0; gg < S.G; ++gg) a += S.part[(gg * 2 + r) * S.n + jj];
    v[r * S.n + jj] = a;
  }
}

// q_r = D^{-1} W p_r (W upper: row i from column i on)
__device__ void mat_W(const Small& S, const double* p, double* q, int nr) {
  for (int e = threadIdx.x; e < nr * S.n; e += kST) {
    const int r = e / S.n, i = e % S.n;
    const double* w = S.W + (int64_t)i * S.n;
    double a = 0.0;
    for (int j = i; j < S.n; ++j) a = fma(w[j], p[r * S.n + j], a);
    q[e] = a * S.dv[i];
  }
}

// v_r = W^T y_r (column j: rows 0..j)
__device__ void mat_Wt(const Small& S, const double* y, double* v, int nr) {
  for (int e = threadIdx.x; e < nr * S.n; e += kST) {
    const int r = e / S.n, j = e % S.n;
    double a = 0.0;
    for (int i = 0; i <= j; ++i) a = fma(S.W[(int64_t)i * S.n + j], y[r * S.n + i], a);
    v[e] = a;
  }
}

struct Pcg {
  double eta[2], eta0[2], beta[2];
  int done[2], iters[2], not_spd[2];
};

// Paired PCGTLS (Alg. 3, A-explicit operator) for RHS fin0 * s0 (r = 0) and fin1 (r = 1):
// iterates in w (nr x n). Scratch vectors: y, s, p, q, v (nr x n each), t (nr x m).
__device__ void pcg(const Small& S, int nr, const double* fin0, double s0, const double* fin1,
                    double sigma2, int steps, double* w, double* y, double* s, double* p,
                    double* q, double* v, double* t, Pcg& st) {
  const int n = S.n;
  for (int e = threadIdx.x; e < nr * n; e += kST) {
    const int r = e / n, j = e % n;
    const double f = (r == 0) ? s0 * fin0[j] : fin1[j];
    y[e] = f * S.dv[j];
    w[e] = 0.0;
    p[e] = 0.0;
  }
  __syncthreads();
  mat_Wt(S, y, s, nr);   // s_0 = R^{-T} f
  __syncthreads();
  {
    double a[2] = {0.0, 0.0};
    for (int e = threadIdx.x; e < nr * n; e += kST) a[e / n] = fma(s[e], s[e], a[e / n]);
    csum<2>(a, S.red);
    for (int r = 0; r < 2; ++r) {
      st.eta[r] = a[r];
      st.eta0[r] = a[r];
      st.beta[r] = 0.0;
      st.done[r] = (r < nr) ? (a[r] == 0.0 ? 1 : 0) : 1;
      st.iters[r] = 0;
      st.not_spd[r] = 0;
    }
  }
  for (int it = 0; it < steps; ++it) {
    if (st.done[0] && st.done[1]) break;   // the remaining steps change nothing
    // p = s + beta p; q = D^{-1} W p
    for (int e = threadIdx.x; e < nr * n; e += kST) p[e] = s[e] + st.beta[e / n] * p[e];
    __syncthreads();
    mat_W(S, p, q, nr);
    __syncthreads();
    mat_A(S, q, t, nr);
    __syncthreads();
    double a[4] = {0.0, 0.0, 0.0, 0.0};   // qq0, qq1, tt0, tt1
    for (int e = threadIdx.x; e < nr * n; e += kST) a[e / n] = fma(q[e], q[e], a[e / n]);
    for (int e = threadIdx.x; e < nr * S.m; e += kST) {
      const int r = e / S.m;
      a[2 + r] = fma(t[e], t[e], a[2 + r]);
    }
    csum<4>(a, S.red);
    mat_At(S, t, v, nr);
    __syncthreads();
    double delta[2], alpha[2];
    bool ok[2];
    for (int r = 0; r < 2; ++r) {
      delta[r] = a[2 + r] - sigma2 * a[r];
      ok[r] = r < nr && !st.done[r] && delta[r] > 0.0;
      alpha[r] = ok[r] ? st.eta[r] / delta[r] : 0.0;
    }
    for (int e = threadIdx.x; e < nr * n; e += kST) {
      const int r = e / n, j = e % n;
      if (!ok[r]) continue;
      w[e] = fma(alpha[r], q[e], w[e]);
      y[e] = (v[e] - sigma2 * q[e]) * S.dv[j];
    }
    __syncthreads();
    mat_Wt(S, y, v, nr);
    __syncthreads();
    double ss[2] = {0.0, 0.0};
    for (int e = threadIdx.x; e < nr * n; e += kST) {
      const int r = e / n;
      if (ok[r]) s[e] = s[e] - alpha[r] * v[e];
      ss[r] = fma(s[e], s[e], ss[r]);
    }
    csum<2>(ss, S.red);
    for (int r = 0; r < nr; ++r) {
      if (st.done[r]) continue;
      if (!(delta[r] > 0.0)) {
        st.done[r] = 1;
        st.not_spd[r] = (delta[r] < 0.0) ? 1 : 0;
      } else {
        st.beta[r] = ss[r] / st.eta[r];
        st.eta[r] = ss[r];
        st.iters[r] += 1;
        if (ss[r] == 0.0) st.done[r] = 1;
      }
    }
  }
  __syncthreads();
}

struct Rq {
  double rr, br, xx, sigma2, g, ff, psi;
};

// r = b - A x, sigma^2 = ||r||^2 / (1 + ||x||^2), f = -A^T r - sigma^2 x, g = -b^T r + sigma^2,
// psi (Alg. 2, Eq. (2), Eq. (4)); x, f: n; r: m scratch, v: n scratch
__device__ Rq resid(const Small& S, const double* x, double xx, double* r, double* v, double* f) {
  double a[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < S.m; i += kST) {
    const double* ai = S.A + (int64_t)i * S.n;
    double d = 0.0;
    for (int j = 0; j < S.n; ++j) d = fma(ai[j], x[j], d);
    const double ri = S.b[i] - d;
    r[i] = ri;
    a[0] = fma(ri, ri, a[0]);
    a[1] = fma(S.b[i], ri, a[1]);
  }
  csum<2>(a, S.red);
  mat_At(S, r, v, 1);
  __syncthreads();
  Rq q;
  q.rr = a[0];
  q.br = a[1];
  q.xx = xx;
  q.sigma2 = a[0] / (1.0 + xx);
  double ff[1] = {0.0};
  for (int j = threadIdx.x; j < S.n; j += kST) {
    const double fj = -v[j] - q.sigma2 * x[j];
    f[j] = fj;
    ff[0] = fma(fj, fj, ff[0]);
  }
  csum<1>(ff, S.red);
  q.ff = ff[0];
  q.g = -q.br + q.sigma2;
  q.psi = sqrt((q.ff + q.g * q.g) / (xx + 1.0));
  return q;
}

__device__ double norm2(const Small& S, const double* x) {
  double a[1] = {0.0};
  for (int j = threadIdx.x; j < S.n; j += kST) a[0] = fma(x[j], x[j], a[0]);
  csum<1>(a, S.red);
  return a[0];
}

__global__ void __launch_bounds__(kST, 1) small_solve_kernel(
    const double* __restrict__ A, int64_t lda, int m, int n, const double* __restrict__ b,
    const double* __restrict__ dinv, const double* __restrict__ W, int64_t ldw, double scale,
    SmallParams prm, double* __restrict__ x_out, SmallResult* res) {
  extern __shared__ __align__(16) double sm[];
  Small S;
  S.m = m;
  S.n = n;
  S.G = kST / n;
  double* pA = sm;
  double* pb = pA + (size_t)m * n;
  double* pW = pb + m;
  double* pdv = pW + (size_t)n * n;
  double* x = pdv + n;
  double* xb = x + n;
  double* f = xb + n;
  double* w = f + n;        // 2n each from here
  double* y = w + 2 * n;
  double* s = y + 2 * n;
  double* p = s + 2 * n;
  double* q = p + 2 * n;
  double* v = q + 2 * n;
  double* t = v + 2 * n;    // 2m
  double* part = t + 2 * m; // G x 2 x n
  double* red = part + (size_t)S.G * 2 * n;
  S.A = pA;
  S.b = pb;
  S.W = pW;
  S.dv = pdv;
  S.red = red;
  S.part = part;
  for (int e = threadIdx.x; e < m * n; e += kST) pA[e] = A[(int64_t)(e / n) * lda + e % n];
  for (int i = threadIdx.x; i < m; i += kST) pb[i] = b[i];
  for (int e = threadIdx.x; e < n * n; e += kST) pW[e] = W[(int64_t)(e / n) * ldw + e % n];
  for (int j = threadIdx.x; j < n; j += kST) {
    pdv[j] = dinv[j];
    x[j] = 0.0;
  }
  __syncthreads();
  Pcg st;
  // Alg. 2 line 1, LS start: residual at x = 0 (f = -A^T b), PCG with sigma^2 = 0
  Rq rq = resid(S, x, 0.0, t, v, f);
  pcg(S, 1, f, -1.0, nullptr, 0.0, prm.ls_iters, w, y, s, p, q, v, t, st);
  for (int j = threadIdx.x; j < n; j += kST) x[j] = w[j];
  __syncthreads();
  double xx = norm2(S, x);
  // lines 2-5: r_0, sigma_0^2, u_0 = (R^T R)^{-1} x_0 (one init step and one W product),
  // x_1 = x_0 + sigma_0^2 u_0
  rq = resid(S, x, xx, t, v, f);
  for (int j = threadIdx.x; j < n; j += kST) y[j] = x[j] * pdv[j];
  __syncthreads();
  mat_Wt(S, y, s, 1);
  __syncthreads();
  mat_W(S, s, q, 1);
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += kST) x[j] = fma(rq.sigma2, q[j], x[j]);
  __syncthreads();
  xx = norm2(S, x);
  // the RQI loop with the stop rules of the dense path
  double prev_psi = INFINITY, best_psi = INFINITY, best_s2 = 0.0;
  int k = 0, best_k = 0, stop = TLS_STOP_MAX_RQI, cg_total = 0, not_spd = 0, n_psi = 0;
  for (;;) {
    ++k;
    rq = resid(S, x, xx, t, v, f);
    if (k > 1) {
      cg_total += st.iters[0] + st.iters[1];
      not_spd |= st.not_spd[0] | st.not_spd[1];
    }
    const double psi = rq.psi, s2 = rq.sigma2;
    if (threadIdx.x == 0 && n_psi < 24) res->psi_hist[n_psi] = psi;
    ++n_psi;
    if (!isfinite(psi) || !isfinite(s2)) {
      stop = TLS_STOP_PSI_UP;
      break;
    }
    const bool up = prm.psi_rule_ge ? (psi >= prev_psi) : (psi > prev_psi);
    if (up && best_psi <= prm.psi_accept * scale) {
      stop = TLS_STOP_PSI_UP;
      break;
    }
    if (psi < best_psi) {
      best_k = k;
      best_psi = psi;
      best_s2 = s2;
      for (int j = threadIdx.x; j < n; j += kST) xb[j] = x[j];
    }
    if (!up && k >= 2 && psi <= prm.tol * scale) {
      stop = TLS_STOP_TOL;
      break;
    }
    if (k > prm.max_rqi) {
      stop = TLS_STOP_MAX_RQI;
      break;
    }
    prev_psi = psi;
    // Alg. 4: two shifted solves with k+1 PCGTLS steps, then the x update
    pcg(S, 2, f, -1.0, x, s2, k + 1, w, y, s, p, q, v, t, st);
    double a[2] = {0.0, 0.0};   // z^T f, z^T x with z = x + w_0
    for (int j = threadIdx.x; j < n; j += kST) {
      const double z = x[j] + w[j];
      a[0] = fma(z, f[j], a[0]);
      a[1] = fma(z, x[j], a[1]);
    }
    csum<2>(a, S.red);
    const double betak = (a[0] - rq.g) / (a[1] + 1.0);
    for (int j = threadIdx.x; j < n; j += kST) x[j] = fma(betak, w[n + j], x[j] + w[j]);
    __syncthreads();
    xx = norm2(S, x);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += kST) x_out[j] = xb[j];
  if (threadIdx.x == 0) {
    res->sigma2 = best_s2;
    res->psi_final = best_psi;
    res->stop = stop;
    res->rqi_steps = k;
    res->best_k = best_k;
    res->cg_iters = cg_total;
    res->not_spd = not_spd;
    res->n_psi = n_psi < 24 ? n_psi : 24;
  }
}

}  // namespace

size_t small_solve_smem(int m, int n) {
  if (n < 1 || n > 64) return 0;
  const int G = kST / n;
  return sizeof(double) * ((size_t)m * n + m + (size_t)n * n + 4 * (size_t)n + 12 * (size_t)n +
                           2 * (size_t)m + (size_t)G * 2 * n + kSW * 4);
}

bool launch_small_solve(const double* A, int64_t lda, int m, int n, const double* b,
                        const double* dinv, const double* W, int64_t ldw, double scale,
                        const SmallParams& prm, double* x_out, SmallResult* res, cudaStream_t s) {
  const size_t smem = small_solve_smem(m, n);
  if (smem == 0 || smem > kSmallSmemMax) return false;
  static const bool once = [] {
    cudaFuncSetAttribute(small_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kSmallSmemMax);
    return true;
  }();
  (void)once;
  small_solve_kernel<<<1, kST, smem, s>>>(A, lda, m, n, b, dinv, W, ldw, scale, prm, x_out, res);
  count_launch();
  return true;
}

}  // namespace tls
