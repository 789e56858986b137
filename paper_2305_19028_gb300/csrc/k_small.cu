// RQI-PCGTLS for a small dense problem in one CTA (all in FP64, u = u_r = FP64): the LS start,
// the inverse-iteration step and the RQI loop of Alg. 2 with the paired PCGTLS solves of Alg. 3
// (A-explicit operator, k+1 steps in RQI step k), the same steps and stop rules as the
// multi-kernel path of the dense solve, with A, b and W = R_H^{-1} held in shared memory.
// For problems whose whole state fits in one SM the multi-kernel path is bound by launch and
// host round-trip latency (about 60 launches per solve); here one launch does the solve.
#include "../../include/tls.h"
#include "tls_internal.h"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace tls {

namespace {

constexpr int kST = 512;              // threads
constexpr int kSW = kST / 32;

__device__ __forceinline__ double swsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sums of K values over the CTA of NT threads; every thread receives the totals. Only threads
// [0, active) may hold nonzero values: the warps beyond skip their shuffles, and one warp adds
// the per-warp sums (FP64 adds run at a 64th of the FP32 rate on this GPU, so a reduction
// repeated by every warp costs as much as the products it sums). sh: (NT / 32 + 1) * K doubles.
template <int K, int NT = kST>
__device__ __forceinline__ void csum(double (&v)[K], double* sh, int active = NT) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = min(NT / 32, (active + 31) / 32);
  if (warp < nw) {
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = swsum(v[k]);
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < K; ++k) sh[warp * K + k] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const double t = swsum(lane < nw ? sh[lane * K + k] : 0.0);
      if (lane == 0) sh[(NT / 32) * K + k] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = sh[(NT / 32) * K + k];
}

struct Small {
  const double* A;   // m x n (row stride n), shared
  const double* b;   // m
  const double* W;   // n x n upper triangular (row stride n)
  const double* dv;  // 1 / d
  int m, n;
  double* red;       // (threads / 32 + 1) * 4
  double* part;      // G x 2 x n partial column sums
  int G;             // row groups of the A^T products
};

// t_r = A q_r (r < nr), one thread per row; q: nr x n, t: nr x m
template <int NT = kST>
__device__ void mat_A(const Small& S, const double* q, double* t, int nr) {
  for (int i = threadIdx.x; i < S.m; i += NT) {
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
template <int NT = kST>
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
  for (int e = threadIdx.x; e < nr * S.n; e += NT) {
    const int r = e / S.n, jj = e % S.n;
    double a = 0.0;
    for (int gg = 0; gg < S.G; ++gg) a += S.part[(gg * 2 + r) * S.n + jj];
    v[r * S.n + jj] = a;
  }
}

// q_r = D^{-1} W p_r (W upper: row i from column i on)
template <int NT = kST>
__device__ void mat_W(const Small& S, const double* p, double* q, int nr) {
  for (int e = threadIdx.x; e < nr * S.n; e += NT) {
    const int r = e / S.n, i = e % S.n;
    const double* w = S.W + (int64_t)i * S.n;
    double a = 0.0;
    for (int j = i; j < S.n; ++j) a = fma(w[j], p[r * S.n + j], a);
    q[e] = a * S.dv[i];
  }
}

// v_r = W^T y_r (column j: rows 0..j)
template <int NT = kST>
__device__ void mat_Wt(const Small& S, const double* y, double* v, int nr) {
  for (int e = threadIdx.x; e < nr * S.n; e += NT) {
    const int r = e / S.n, j = e % S.n;
    double a = 0.0;
    for (int i = 0; i <= j; ++i) a = fma(S.W[(int64_t)i * S.n + j], y[r * S.n + i], a);
    v[e] = a;
  }
}

// State of the paired PCGTLS solves: one copy per CTA in shared memory; thread 0 computes the
// FP64 scalars (divisions and square roots) once and the others read them after a barrier.
struct Pcg {
  double eta[2], eta0[2], beta[2], alpha[2], delta[2];
  int done[2], iters[2], not_spd[2], ok[2];
};

// The rows of A may be spread over the CTAs of a cluster: every sum over rows (the m-vector dot
// products and A^T t) is then a per-CTA partial that the Comm policy completes, in the same
// order in every CTA; the n-sized work runs redundantly (and identically) in every CTA.
struct OneCta {
  template <int K>
  __device__ void sum(double (&)[K], double*, int) {}
};

// Paired PCGTLS (Alg. 3, A-explicit operator) for RHS fin0 * s0 (r = 0) and fin1 (r = 1):
// iterates in w (nr x n). Scratch vectors: y, s, p, q, v (nr x n each), t (nr x m). st: shared.
template <int NT, class Comm>
__device__ void pcg(const Small& S, Comm& comm, int nr, const double* fin0, double s0,
                    const double* fin1, double sigma2, int steps, double* w, double* y,
                    double* s, double* p, double* q, double* v, double* t, Pcg& st) {
  const int n = S.n, nn = nr * n;
  for (int e = threadIdx.x; e < nn; e += NT) {
    const int r = e / n, j = e % n;
    const double f = (r == 0) ? s0 * fin0[j] : fin1[j];
    y[e] = f * S.dv[j];
    w[e] = 0.0;
    p[e] = 0.0;
  }
  __syncthreads();
  mat_Wt<NT>(S, y, s, nr);   // s_0 = R^{-T} f
  __syncthreads();
  {
    double a[2] = {0.0, 0.0};
    for (int e = threadIdx.x; e < nn; e += NT) a[e / n] = fma(s[e], s[e], a[e / n]);
    csum<2, NT>(a, S.red, nn);
    if (threadIdx.x == 0)
      for (int r = 0; r < 2; ++r) {
        st.eta[r] = a[r];
        st.eta0[r] = a[r];
        st.beta[r] = 0.0;
        st.done[r] = (r < nr) ? (a[r] == 0.0 ? 1 : 0) : 1;
        st.iters[r] = 0;
        st.not_spd[r] = 0;
      }
    __syncthreads();
  }
  for (int it = 0; it < steps; ++it) {
    if (st.done[0] && st.done[1]) break;   // the remaining steps change nothing
    // p = s + beta p; q = D^{-1} W p
    for (int e = threadIdx.x; e < nn; e += NT) p[e] = s[e] + st.beta[e / n] * p[e];
    __syncthreads();
    mat_W<NT>(S, p, q, nr);
    __syncthreads();
    mat_A<NT>(S, q, t, nr);
    __syncthreads();
    double a[4] = {0.0, 0.0, 0.0, 0.0};   // qq0, qq1, tt0, tt1
    for (int e = threadIdx.x; e < nn; e += NT) a[e / n] = fma(q[e], q[e], a[e / n]);
    for (int e = threadIdx.x; e < nr * S.m; e += NT) {
      const int r = e / S.m;
      a[2 + r] = fma(t[e], t[e], a[2 + r]);
    }
    csum<4, NT>(a, S.red, max(nn, nr * S.m));
    mat_At<NT>(S, t, v, nr);
    __syncthreads();
    {
      double mt[2] = {a[2], a[3]};   // ||t_r||^2 and A^T t over all rows
      comm.sum(mt, v, nr);
      a[2] = mt[0];
      a[3] = mt[1];
    }
    if (threadIdx.x == 0)
      for (int r = 0; r < 2; ++r) {
        st.delta[r] = a[2 + r] - sigma2 * a[r];
        st.ok[r] = (r < nr && !st.done[r] && st.delta[r] > 0.0) ? 1 : 0;
        st.alpha[r] = st.ok[r] ? st.eta[r] / st.delta[r] : 0.0;
      }
    __syncthreads();
    for (int e = threadIdx.x; e < nn; e += NT) {
      const int r = e / n, j = e % n;
      if (!st.ok[r]) continue;
      w[e] = fma(st.alpha[r], q[e], w[e]);
      y[e] = (v[e] - sigma2 * q[e]) * S.dv[j];
    }
    __syncthreads();
    mat_Wt<NT>(S, y, v, nr);
    __syncthreads();
    double ss[2] = {0.0, 0.0};
    for (int e = threadIdx.x; e < nn; e += NT) {
      const int r = e / n;
      if (st.ok[r]) s[e] = s[e] - st.alpha[r] * v[e];
      ss[r] = fma(s[e], s[e], ss[r]);
    }
    csum<2, NT>(ss, S.red, nn);
    if (threadIdx.x == 0)
      for (int r = 0; r < nr; ++r) {
        if (st.done[r]) continue;
        if (!(st.delta[r] > 0.0)) {
          st.done[r] = 1;
          st.not_spd[r] = (st.delta[r] < 0.0) ? 1 : 0;
        } else {
          st.beta[r] = ss[r] / st.eta[r];
          st.eta[r] = ss[r];
          st.iters[r] += 1;
          if (ss[r] == 0.0) st.done[r] = 1;
        }
      }
    __syncthreads();
  }
  __syncthreads();
}

struct Rq {
  double rr, br, xx, sigma2, g, ff, psi;
};

// r = b - A x, sigma^2 = ||r||^2 / (1 + ||x||^2), f = -A^T r - sigma^2 x, g = -b^T r + sigma^2,
// psi (Alg. 2, Eq. (2), Eq. (4)); x, f: n; r: m scratch, v: n scratch; q: shared
template <int NT, class Comm>
__device__ void resid(const Small& S, Comm& comm, const double* x, double xx, double* r,
                      double* v, double* f, Rq& q) {
  double a[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < S.m; i += NT) {
    const double* ai = S.A + (int64_t)i * S.n;
    double d = 0.0;
    for (int j = 0; j < S.n; ++j) d = fma(ai[j], x[j], d);
    const double ri = S.b[i] - d;
    r[i] = ri;
    a[0] = fma(ri, ri, a[0]);
    a[1] = fma(S.b[i], ri, a[1]);
  }
  csum<2, NT>(a, S.red, S.m);
  mat_At<NT>(S, r, v, 1);
  __syncthreads();
  comm.sum(a, v, 1);
  if (threadIdx.x == 0) {
    q.rr = a[0];
    q.br = a[1];
    q.xx = xx;
    q.sigma2 = a[0] / (1.0 + xx);
    q.g = -q.br + q.sigma2;
  }
  __syncthreads();
  const double sigma2 = q.sigma2;
  double ff[1] = {0.0};
  for (int j = threadIdx.x; j < S.n; j += NT) {
    const double fj = -v[j] - sigma2 * x[j];
    f[j] = fj;
    ff[0] = fma(fj, fj, ff[0]);
  }
  csum<1, NT>(ff, S.red, S.n);
  if (threadIdx.x == 0) {
    q.ff = ff[0];
    q.psi = sqrt((q.ff + q.g * q.g) / (xx + 1.0));
  }
  __syncthreads();
}

template <int NT>
__device__ double norm2(const Small& S, const double* x) {
  double a[1] = {0.0};
  for (int j = threadIdx.x; j < S.n; j += NT) a[0] = fma(x[j], x[j], a[0]);
  csum<1, NT>(a, S.red, S.n);
  return a[0];
}

// The solve proper (LS start, inverse-iteration step, RQI loop), after S and the vectors are
// set up; `out` selects the CTA that writes x_out and res.
template <int NT, class Comm>
__device__ void rqi_solve(Small& S, Comm& comm, double scale, const SmallParams& prm,
                          double* x, double* xb, double* f, double* w, double* y, double* s,
                          double* p, double* q, double* v, double* t, bool out,
                          double* __restrict__ x_out, SmallResult* res) {
  const int n = S.n;
  const double* pdv = S.dv;
  __shared__ Pcg st;
  __shared__ Rq rq;
  __shared__ double betak_sh;
  // Alg. 2 line 1, LS start: residual at x = 0 (f = -A^T b), PCG with sigma^2 = 0
  resid<NT>(S, comm, x, 0.0, t, v, f, rq);
  pcg<NT>(S, comm, 1, f, -1.0, nullptr, 0.0, prm.ls_iters, w, y, s, p, q, v, t, st);
  for (int j = threadIdx.x; j < n; j += NT) x[j] = w[j];
  __syncthreads();
  double xx = norm2<NT>(S, x);
  // lines 2-5: r_0, sigma_0^2, u_0 = (R^T R)^{-1} x_0 (one init step and one W product),
  // x_1 = x_0 + sigma_0^2 u_0
  resid<NT>(S, comm, x, xx, t, v, f, rq);
  for (int j = threadIdx.x; j < n; j += NT) y[j] = x[j] * pdv[j];
  __syncthreads();
  mat_Wt<NT>(S, y, s, 1);
  __syncthreads();
  mat_W<NT>(S, s, q, 1);
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += NT) x[j] = fma(rq.sigma2, q[j], x[j]);
  __syncthreads();
  xx = norm2<NT>(S, x);
  // the RQI loop with the stop rules of the dense path
  double prev_psi = INFINITY, best_psi = INFINITY, best_s2 = 0.0;
  int k = 0, best_k = 0, stop = TLS_STOP_MAX_RQI, cg_total = 0, not_spd = 0, n_psi = 0;
  for (;;) {
    ++k;
    resid<NT>(S, comm, x, xx, t, v, f, rq);
    if (k > 1) {
      cg_total += st.iters[0] + st.iters[1];
      not_spd |= st.not_spd[0] | st.not_spd[1];
    }
    const double psi = rq.psi, s2 = rq.sigma2;
    if (out && threadIdx.x == 0 && n_psi < 24) res->psi_hist[n_psi] = psi;
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
      for (int j = threadIdx.x; j < n; j += NT) xb[j] = x[j];
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
    pcg<NT>(S, comm, 2, f, -1.0, x, s2, k + 1, w, y, s, p, q, v, t, st);
    double a[2] = {0.0, 0.0};   // z^T f, z^T x with z = x + w_0
    for (int j = threadIdx.x; j < n; j += NT) {
      const double z = x[j] + w[j];
      a[0] = fma(z, f[j], a[0]);
      a[1] = fma(z, x[j], a[1]);
    }
    csum<2, NT>(a, S.red, n);
    if (threadIdx.x == 0) betak_sh = (a[0] - rq.g) / (a[1] + 1.0);
    __syncthreads();
    const double betak = betak_sh;
    for (int j = threadIdx.x; j < n; j += NT) x[j] = fma(betak, w[n + j], x[j] + w[j]);
    __syncthreads();
    xx = norm2<NT>(S, x);
  }
  __syncthreads();
  if (!out) return;
  for (int j = threadIdx.x; j < n; j += NT) x_out[j] = xb[j];
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
  double* red = part + (size_t)S.G * 2 * n;   // (kSW + 1) * 4
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
  OneCta one;
  rqi_solve<kST>(S, one, scale, prm, x, xb, f, w, y, s, p, q, v, t, true, x_out, res);
}
// ---------------------------------------------------------------------------------------
// The same solve on a thread-block cluster of R CTAs (one per SM): CTA c holds the rows
// [m c / R, m (c+1) / R) of A and b in its shared memory, W and every n-vector in full. The
// passes over A run on R SMs' FP64 units instead of one; each PCGTLS step and each residual
// exchanges one partial vector (and up to two scalars) per CTA through distributed shared
// memory, with one cluster barrier.
// ---------------------------------------------------------------------------------------
constexpr int kCT = 256;
constexpr int kMaxCluster = 16;

// Completes the row sums over the CTAs of the cluster: every CTA publishes its partial (K
// scalars, identical in all its threads, and nv x n values in vec) in its own exchange buffer;
// after one cluster barrier every CTA adds the buffers of ranks 0, 1, ... in that order, so all
// CTAs hold bit-identical totals and take identical decisions afterwards. Two exchange buffers
// alternate: a buffer is written again only after the barrier of the next call, which every
// peer reaches after its reads of it.
struct ClusterComm {
  double* xch[2];   // own exchange buffers, 4 + 2n doubles each
  double* tot;      // 4 doubles
  int phase;
  int n;
  template <int K>
  __device__ void sum(double (&a)[K], double* vec, int nv) {
    cg::cluster_group cl = cg::this_cluster();
    double* buf = xch[phase];
    phase ^= 1;
    if (threadIdx.x == 0)
#pragma unroll
      for (int k = 0; k < K; ++k) buf[k] = a[k];
    for (int e = threadIdx.x; e < nv * n; e += kCT) buf[4 + e] = vec[e];
    cl.sync();
    const int R = (int)cl.num_blocks();
    // all remote loads first (one round trip), then the adds in rank order
    for (int e = threadIdx.x; e < nv * n; e += kCT) {
      double val[kMaxCluster];
#pragma unroll
      for (int r = 0; r < kMaxCluster; ++r)
        val[r] = (r < R) ? cl.map_shared_rank(buf, r)[4 + e] : 0.0;
      double t = 0.0;
#pragma unroll
      for (int r = 0; r < kMaxCluster; ++r)
        if (r < R) t += val[r];
      vec[e] = t;
    }
    if (threadIdx.x < K) {
      double val[kMaxCluster];
#pragma unroll
      for (int r = 0; r < kMaxCluster; ++r)
        val[r] = (r < R) ? cl.map_shared_rank(buf, r)[threadIdx.x] : 0.0;
      double t = 0.0;
#pragma unroll
      for (int r = 0; r < kMaxCluster; ++r)
        if (r < R) t += val[r];
      tot[threadIdx.x] = t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] = tot[k];
  }
};

__host__ __device__ inline int cluster_rows(int m, int R) { return (m + R - 1) / R; }

__global__ void __launch_bounds__(kCT, 1) cluster_solve_kernel(
    const double* __restrict__ A, int64_t lda, int m, int n, const double* __restrict__ b,
    const double* __restrict__ dinv, const double* __restrict__ W, int64_t ldw, double scale,
    SmallParams prm, double* __restrict__ x_out, SmallResult* res) {
  extern __shared__ __align__(16) double sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int R = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int r0 = (int)((int64_t)m * rank / R), r1 = (int)((int64_t)m * (rank + 1) / R);
  const int mc = r1 - r0, mmax = cluster_rows(m, R);
  Small S;
  S.m = mc;
  S.n = n;
  S.G = kCT / n;
  double* pA = sm;
  double* pb = pA + (size_t)mmax * n;
  double* pW = pb + mmax;
  double* pdv = pW + (size_t)n * n;
  double* x = pdv + n;
  double* xb = x + n;
  double* f = xb + n;
  double* w = f + n;          // 2n each from here
  double* y = w + 2 * n;
  double* s = y + 2 * n;
  double* p = s + 2 * n;
  double* q = p + 2 * n;
  double* v = q + 2 * n;
  double* t = v + 2 * n;      // 2 mmax
  double* part = t + 2 * mmax;
  double* red = part + (size_t)S.G * 2 * n;
  double* xch0 = red + (kCT / 32 + 1) * 4;
  double* xch1 = xch0 + 4 + 2 * n;
  double* tot = xch1 + 4 + 2 * n;
  S.A = pA;
  S.b = pb;
  S.W = pW;
  S.dv = pdv;
  S.red = red;
  S.part = part;
  for (int e = threadIdx.x; e < mc * n; e += kCT)
    pA[e] = A[(int64_t)(r0 + e / n) * lda + e % n];
  for (int i = threadIdx.x; i < mc; i += kCT) pb[i] = b[r0 + i];
  for (int e = threadIdx.x; e < n * n; e += kCT) pW[e] = W[(int64_t)(e / n) * ldw + e % n];
  for (int j = threadIdx.x; j < n; j += kCT) {
    pdv[j] = dinv[j];
    x[j] = 0.0;
  }
  __syncthreads();
  ClusterComm comm{{xch0, xch1}, tot, 0, n};
  rqi_solve<kCT>(S, comm, scale, prm, x, xb, f, w, y, s, p, q, v, t, rank == 0, x_out, res);
  cl.sync();   // no CTA leaves while a peer may still read its exchange buffers
}

size_t cluster_solve_smem(int m, int n, int R) {
  if (n < 1 || n > 64 || R < 1) return 0;
  const int G = kCT / n, mm = cluster_rows(m, R);
  return sizeof(double) * ((size_t)mm * n + mm + (size_t)n * n + 4 * (size_t)n + 12 * (size_t)n +
                           2 * (size_t)mm + (size_t)G * 2 * n + (kCT / 32 + 1) * 4 +
                           2 * (4 + 2 * (size_t)n) + 4);
}

}  // namespace

bool cluster_solve_fits(int m, int n) {
  for (int R : {16, 8, 4, 2}) {
    const size_t smem = cluster_solve_smem(m, n, R);
    if (m / R >= 16 && smem > 0 && smem <= kSmallSmemMax) return true;
  }
  return false;
}

int launch_cluster_solve(const double* A, int64_t lda, int m, int n, const double* b,
                         const double* dinv, const double* W, int64_t ldw, double scale,
                         const SmallParams& prm, double* x_out, SmallResult* res,
                         cudaStream_t s) {
  static const bool once = [] {
    cudaFuncSetAttribute(cluster_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kSmallSmemMax);
    cudaFuncSetAttribute(cluster_solve_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    (void)cudaGetLastError();
    return true;
  }();
  (void)once;
  // the largest cluster that leaves each CTA at least 16 rows
  for (int R : {16, 8, 4, 2}) {
    if (m / R < 16) continue;
    const size_t smem = cluster_solve_smem(m, n, R);
    if (smem == 0 || smem > kSmallSmemMax) continue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)R, 1, 1);
    cfg.blockDim = dim3(kCT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)R;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, cluster_solve_kernel, &cfg) != cudaSuccess ||
        clusters < 1) {
      (void)cudaGetLastError();
      continue;
    }
    if (cudaLaunchKernelEx(&cfg, cluster_solve_kernel, A, lda, m, n, b, dinv, W, ldw, scale,
                           prm, x_out, res) == cudaSuccess) {
      count_launch();
      return R;
    }
    (void)cudaGetLastError();
  }
  return 0;
}

size_t small_solve_smem(int m, int n) {
  if (n < 1 || n > 64) return 0;
  const int G = kST / n;
  return sizeof(double) * ((size_t)m * n + m + (size_t)n * n + 4 * (size_t)n + 12 * (size_t)n +
                           2 * (size_t)m + (size_t)G * 2 * n + (kSW + 1) * 4);
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
