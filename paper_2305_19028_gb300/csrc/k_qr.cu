// Householder QR preconditioner (Alg. 4 of Oktay & Carson, arXiv 2305.19028, the step
// "Compute A = Q[R 0]^T in precision u_q"; Sec. 3 prefers it to the Cholesky factor of A^T A,
// whose precision constraint is about kappa^-2 instead of kappa^-1). Only R is formed: the
// preconditioner needs R-hat, not Q.
//
// Blocked by column panels of width bw in the compact WY form Q_p = I - V_p T_p V_p^T:
//  1. qr_panel_kernel: the reflectors of the panel's bw columns on one thread-block cluster
//     whose CTAs hold the panel's rows in shared memory. Each column takes two sums over all
//     rows (its norm below the pivot, then v^T a_c for the panel's later columns); every CTA
//     publishes its partial in its own exchange buffer and, after one cluster barrier, adds the
//     buffers of ranks 0, 1, ... in that order, so all CTAs take identical decisions. Then
//     T_p from V_p^T V_p by the recurrence T[0:j, j] = -tau_j T[0:j, 0:j] (V[:, 0:j]^T v_j).
//  2. qr_vta_kernel: X = V_p^T A_trail over row chunks (partials, no atomics);
//     qr_apply_kernel: X summed in chunk order, Y = T_p^T X, A_trail -= V_p Y.
// Reflector of x = [x0; x'] (s = ||x'||^2): s = 0 gives tau = 0 (the identity) and beta = x0;
// otherwise beta = -sign(x0) sqrt(x0^2 + s), tau = (beta - x0) / beta, v = [1; x' / (x0 - beta)],
// so that (I - tau v v^T) x = beta e_1 and beta is the diagonal entry of R.
// Arithmetic in T (FP32 for u_q in {FP16, BF16, FP32}, FP64 for u_q = FP64); the caller rounds
// A D^{-1} to u_q before and R to u_q after, as the Cholesky route does.
#include "tls_internal.h"

#include <cooperative_groups.h>

#include <algorithm>

namespace cg = cooperative_groups;

namespace tls {

namespace {

constexpr int kQT = 256;          // threads per CTA
constexpr int kQMaxCl = 16;       // CTAs per cluster (non-portable size)
constexpr int kQMaxBw = 32;       // panel width limit (one warp forms T)
constexpr int kQChunk = 32;       // rows per staged tile of the trailing-update kernels
constexpr size_t kQSmemMax = 227 * 1024;

inline int qr_blocks(int64_t count, int threads) { return (int)((count + threads - 1) / threads); }

template <typename T>
__device__ __forceinline__ T warp_sum_q(T v) {
  // butterfly: every lane ends with the same value (the same tree of commutative adds)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Entry e of the exchange buffer buf summed over the cluster's R CTAs in rank order (all remote
// loads issued before the first add: one round trip).
template <typename T>
__device__ __forceinline__ T rank_order_sum(cg::cluster_group& cl, T* buf, int e, int R) {
  T val[kQMaxCl];
#pragma unroll
  for (int r = 0; r < kQMaxCl; ++r) val[r] = (r < R) ? cl.map_shared_rank(buf, r)[e] : T(0);
  T t = T(0);
#pragma unroll
  for (int r = 0; r < kQMaxCl; ++r)
    if (r < R) t += val[r];
  return t;
}

// The end of a panel (both panel kernels, all threads of every CTA). With have_g false, first
// V^T V from the panel rows in shared memory P (entry (a, b), a < b, sums V[r][a] V[r][b] over
// rows r >= k + b, with V[k + b][b] = 1 and V[r][a] = P[r][a] below row k + a), summed over
// the cluster in rank order, into the strict upper part of G. Then T by doubling: T_jj = tau_j,
// and for every pair of neighbouring s-blocks A, B (s = 1, 2, 4, 8, 16),
// T_AB = -T_AA (V_A^T V_B) T_BB, the compact WY form of Q_A Q_B. Rank 0 writes T and the taus;
// every CTA writes its rows of the panel back to A.
template <typename T>
__device__ __forceinline__ void qr_panel_finish(cg::cluster_group& cl, const T* P, int ldp, int nr,
                                                int bw, T* xch, const T* taus, T* G, T* Tl,
                                                T* A, int64_t lda, int64_t k, int64_t r0,
                                                T* tau_out, T* Tm, int* info, int bad,
                                                bool have_g) {
  const int R = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthr = blockDim.x, nw = nthr / 32;
  const int npairs = bw * (bw - 1) / 2;
  if (!have_g) {
    for (int q = warp; q < npairs; q += nw) {
      int a = 0, rem = q;
      while (rem >= bw - 1 - a) {
        rem -= bw - 1 - a;
        ++a;
      }
      const int b = a + 1 + rem;
      const int lb = (rank == 0) ? b : -1;
      T acc = T(0);
      for (int i = max(lb, 0) + lane; i < nr; i += 32) {
        const T vb = (i == lb) ? T(1) : P[i * ldp + b];
        acc = fma(P[i * ldp + a], vb, acc);
      }
      acc = warp_sum_q(acc);
      if (lane == 0) xch[q] = acc;
    }
    cl.sync();
    for (int q = tid; q < npairs; q += nthr) {
      int a = 0, rem = q;
      while (rem >= bw - 1 - a) {
        rem -= bw - 1 - a;
        ++a;
      }
      const int b = a + 1 + rem;
      G[a * bw + b] = rank_order_sum(cl, xch, q, R);
    }
  }
  for (int e = tid; e < bw * bw; e += nthr) {
    const int i = e / bw, j = e - i * bw;
    Tl[e] = (i == j) ? taus[i] : T(0);
  }
  __syncthreads();
  for (int sb = 1; sb < bw; sb *= 2) {
    // Tm_AB = G_AB T_BB into the (zero, unused) lower part of Tl: entry (a, b) of the pair at o
    // goes to Tl[o + sb + b][o + a]; then T_AB = -T_AA Tm_AB
    const int pairs = (bw + 2 * sb - 1) / (2 * sb);
    for (int e = tid; e < pairs * sb * sb; e += nthr) {
      const int pr = e / (sb * sb), rem = e - pr * sb * sb, a = rem / sb, b = rem - a * sb;
      const int o = 2 * pr * sb, ia = o + a, jb = o + sb + b;
      if (jb < bw) {
        T v = T(0);
        for (int l = o + sb; l <= jb; ++l) v = fma(G[ia * bw + l], Tl[l * bw + jb], v);
        Tl[jb * bw + ia] = v;
      }
    }
    __syncthreads();
    for (int e = tid; e < pairs * sb * sb; e += nthr) {
      const int pr = e / (sb * sb), rem = e - pr * sb * sb, a = rem / sb, b = rem - a * sb;
      const int o = 2 * pr * sb, ia = o + a, jb = o + sb + b;
      if (jb < bw) {
        T v = T(0);
        for (int l = ia; l < o + sb; ++l) v = fma(Tl[ia * bw + l], Tl[jb * bw + l], v);
        Tl[ia * bw + jb] = -v;
      }
    }
    __syncthreads();
  }
  if (rank == 0) {
    for (int e = tid; e < bw * bw; e += nthr) {
      const int i = e / bw, j = e - i * bw;
      Tm[e] = (j >= i) ? Tl[e] : T(0);
    }
    for (int e = tid; e < bw; e += nthr) tau_out[k + e] = taus[e];
    if (tid == 0 && bad) atomicCAS(info, 0, (int)(k + bad));
  }
  for (int e = tid; e < nr * bw; e += nthr) {
    const int i = e / bw, c = e - i * bw;
    A[(r0 + i) * lda + k + c] = P[i * ldp + c];
  }
  cl.sync();   // no CTA leaves while a peer may still read its exchange buffers
}

// extra shared memory of the panel kernel beside the rows: the per-column exchange slots (two
// sets of kQMaxCl slots of bw + 2), the V^T V exchange buffer, column sums, taus, reduction
// scratch, V^T V and T
__host__ __device__ inline size_t qr_panel_extra(int bw) {
  const size_t xw = (size_t)bw * (bw + 1) / 2 + 2;
  return 2 * (size_t)kQMaxCl * (bw + 2) + xw + 2 * (size_t)bw + 40 + 2 * (size_t)bw * bw;
}

template <typename T>
__global__ void __launch_bounds__(kQT, 1) qr_panel_kernel(T* __restrict__ A, int64_t lda,
                                                          int64_t m, int64_t k, int bw, int rpc,
                                                          T* __restrict__ tau_out,
                                                          T* __restrict__ Tm,
                                                          int* __restrict__ info) {
  cg::cluster_group cl = cg::this_cluster();
  const int R = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nw = kQT / 32;
  const int ldp = bw + 1;   // odd row stride: a column read by consecutive rows is conflict-free
  const int xw = bw * (bw + 1) / 2 + 2;
  const int sw = bw + 2;    // one slot of the per-column exchange
  extern __shared__ __align__(16) unsigned char qsm[];
  T* P = reinterpret_cast<T*>(qsm);    // this CTA's rows of the panel, rpc x ldp
  T* slots = P + (size_t)rpc * ldp;    // [2][kQMaxCl][sw]: slot r of set s holds rank r's partials
  T* xch = slots + 2 * kQMaxCl * sw;   // the V^T V exchange buffer, xw
  T* wtot = xch + xw;                  // tau * (v^T a_c) per column c
  T* taus = wtot + bw;
  T* red = taus + bw;                  // 40: per-warp partials, broadcast scalars
  T* G = red + 40;                     // V^T V (strict upper part), bw x bw
  T* Tl = G + bw * bw;                 // T, bw x bw
  const int64_t r0 = k + (int64_t)rank * rpc;
  const int nr = (int)max((int64_t)0, min(m, r0 + rpc) - r0);
  for (int e0 = tid; e0 < nr * bw; e0 += 8 * kQT) {
    T v[8];   // eight loads in flight per thread
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = e0 + t * kQT, i = e / bw, c = e - i * bw;
      v[t] = (e < nr * bw) ? A[(r0 + i) * lda + k + c] : T(0);
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = e0 + t * kQT, i = e / bw, c = e - i * bw;
      if (e < nr * bw) P[i * ldp + c] = v[t];
    }
  }
  cl.sync();   // every CTA of the cluster running before the first write into a peer's slots
  // the pivot row k + j lies in rank 0's rows (the host keeps rpc >= bw)
  int ph = 0, bad = 0;
  for (int j = 0; j < bw; ++j) {
    const int lj = (rank == 0) ? j : -1;   // local index of the pivot row, -1 if not here
    const int lo = lj + 1;                 // first local row below the pivot (0 off rank 0)
    // (1) sum of squares of column j below the pivot
    T ss = T(0);
    for (int i = lo + tid; i < nr; i += kQT) {
      const T a = P[i * ldp + j];
      ss = fma(a, a, ss);
    }
    ss = warp_sum_q(ss);
    if (lane == 0) red[warp] = ss;
    __syncthreads();
    // every CTA pushes its partial into its own slot of every peer before the barrier, and
    // after it reads the R slots locally (no remote load on the critical path)
    T* set = slots + ph * kQMaxCl * sw;
    ph ^= 1;
    if (tid < R) {
      T t = T(0);
      for (int w = 0; w < nw; ++w) t += red[w];
      T* dst = cl.map_shared_rank(set + rank * sw, tid);
      dst[0] = t;
      dst[1] = (lj >= 0) ? P[lj * ldp + j] : T(0);
    }
    cl.sync();
    T s_tot = T(0);
    for (int r = 0; r < R; ++r) s_tot += set[r * sw];
    const T x0 = set[1];   // rank 0 holds the pivot row
    T tau, beta, scal;
    if (s_tot == T(0)) {
      tau = T(0);
      beta = x0;
      scal = T(1);
    } else {
      const T nrm = sqrt(fma(x0, x0, s_tot));
      beta = (x0 >= T(0)) ? -nrm : nrm;
      tau = (beta - x0) / beta;
      scal = T(1) / (x0 - beta);
    }
    if (!bad && (!(beta == beta) || beta == T(0) || isinf(beta))) bad = j + 1;
    if (tid == 0) taus[j] = tau;
    for (int i = lo + tid; i < nr; i += kQT) P[i * ldp + j] *= scal;
    if (lj >= 0 && tid == 0) P[lj * ldp + j] = beta;
    __syncthreads();
    if (j + 1 < bw) {
      // (2) w_c = v^T a_c over the rows from the pivot down (v = 1 at the pivot), c > j
      T* set2 = slots + ph * kQMaxCl * sw;
      ph ^= 1;
      const int i0 = max(lj, 0);
      for (int c = j + 1 + warp; c < bw; c += nw) {
        T acc = T(0);
        for (int i = i0 + lane; i < nr; i += 32) {
          const T v = (i == lj) ? T(1) : P[i * ldp + j];
          acc = fma(v, P[i * ldp + c], acc);
        }
        acc = warp_sum_q(acc);
        if (lane < R) cl.map_shared_rank(set2 + rank * sw, lane)[c] = acc;
      }
      cl.sync();
      if (tid > j && tid < bw) {
        T t = T(0);
        for (int r = 0; r < R; ++r) t += set2[r * sw + tid];
        wtot[tid] = tau * t;
      }
      __syncthreads();
      // (3) a_c -= (tau w_c) v over the same rows
      for (int i = i0 + tid; i < nr; i += kQT) {
        const T v = (i == lj) ? T(1) : P[i * ldp + j];
        for (int c = j + 1; c < bw; ++c) P[i * ldp + c] = fma(-wtot[c], v, P[i * ldp + c]);
      }
      __syncthreads();
    }
  }
  qr_panel_finish<T>(cl, P, ldp, nr, bw, xch, taus, G, Tl, A, lda, k, r0, tau_out, Tm, info,
                     bad, false);
}

// Sums over the 32 lanes of a warp of 32 values per lane at once: lane l ends with the total of
// value l (recursive halving, 31 shuffles instead of 32 x 5).
__device__ __forceinline__ float warp_transpose_sum32(float (&v)[32], int lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const float send = up ? v[i] : v[i + s];
      const float keep = up ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return v[0];
}

constexpr int kQRT = 512;   // threads per CTA of the register panel kernel

// extra shared memory of the register panel kernel beside the rows (floats)
__host__ __device__ inline size_t qr_panel_reg_extra() {
  const int bw = kQMaxBw;
  const size_t xw = (size_t)bw * (bw + 1) / 2 + 2;
  return 2 * (size_t)kQMaxCl * (bw + 2) + xw + (size_t)(kQRT / 32) * (bw + 1) + 2 * (size_t)bw +
         40 + 2 * (size_t)bw * bw;
}

// The panel kernel with the rows in registers (FP32, 32-column panels): thread t of a CTA holds
// local rows t + kQRT q (q < RPT) of the panel, all bw columns, so the column steps read and
// update registers rather than shared memory. Per column: the norm below the pivot (warp sums,
// then every CTA's partial pushed into its slot of every peer before one cluster barrier), the
// reflector, then v^T a_c for the later columns (each lane's 32 partial products reduced over
// the warp in one transposed pass, then over the warps, then over the cluster in rank order
// the same way; the same exchange carries column j of V^T V), and the rank-1 update in
// registers. T and the write-back go through shared memory (qr_panel_finish).
template <int RPT>
__global__ void __launch_bounds__(kQRT, 1) qr_panel_reg_kernel(float* __restrict__ A, int64_t lda,
                                                              int64_t m, int64_t k, int bw,
                                                              int rpc, float* __restrict__ tau_out,
                                                              float* __restrict__ Tm,
                                                              int* __restrict__ info) {
  constexpr int BW = kQMaxBw, NW = kQRT / 32, SW = BW + 2;
  cg::cluster_group cl = cg::this_cluster();
  const int R = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ldp = BW + 1;
  extern __shared__ __align__(16) unsigned char qsm[];
  float* P = reinterpret_cast<float*>(qsm);       // rpc x ldp, for the finish
  float* slots = P + (size_t)rpc * ldp;           // [2][kQMaxCl][SW]
  float* xch = slots + 2 * kQMaxCl * SW;          // V^T V exchange, BW (BW + 1) / 2 + 2
  float* wsum = xch + BW * (BW + 1) / 2 + 2;      // [NW][BW + 1] per-warp column sums
  float* wtot = wsum + NW * (BW + 1);             // tau * (v^T a_c)
  float* taus = wtot + BW;
  float* red = taus + BW;                         // 40
  float* G = red + 40;
  float* Tl = G + BW * BW;
  const int64_t r0 = k + (int64_t)rank * rpc;
  const int nr = (int)max((int64_t)0, min(m, r0 + rpc) - r0);
  // the rows through shared memory (coalesced loads, eight in flight per thread), then into
  // registers
  for (int e0 = tid; e0 < nr * BW; e0 += 8 * kQRT) {
    float v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = e0 + t * kQRT, i = e / BW, c = e - i * BW;
      v[t] = (e < nr * BW && c < bw) ? A[(r0 + i) * lda + k + c] : 0.f;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = e0 + t * kQRT, i = e / BW, c = e - i * BW;
      if (e < nr * BW) P[i * ldp + c] = v[t];
    }
  }
  __syncthreads();
  float a[RPT][BW];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int lr = tid + kQRT * q;
#pragma unroll
    for (int c = 0; c < BW; ++c) a[q][c] = (lr < nr) ? P[lr * ldp + c] : 0.f;
  }
  if (tid < BW) wtot[tid] = 0.f;
  cl.sync();   // every CTA of the cluster running before the first write into a peer's slots
  int ph = 0, bad = 0;
#pragma unroll
  for (int j = 0; j < BW; ++j) {
    if (j < bw) {
      const int lj = (rank == 0) ? j : -1;   // the pivot row is thread j's first row on rank 0
      // (1) sum of squares of column j below the pivot
      float ss = 0.f;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int lr = tid + kQRT * q;
        if (lr < nr && lr > lj) ss = fmaf(a[q][j], a[q][j], ss);
      }
      ss = warp_sum_q(ss);
      if (lane == 0) red[warp] = ss;
      if (lj >= 0 && tid == j) red[34] = a[0][j];
      __syncthreads();
      float* set = slots + ph * kQMaxCl * SW;
      ph ^= 1;
      if (tid < R) {
        float t = 0.f;
        for (int w = 0; w < NW; ++w) t += red[w];
        float* dst = cl.map_shared_rank(set + rank * SW, tid);
        dst[0] = t;
        dst[1] = (rank == 0) ? red[34] : 0.f;
      }
      cl.sync();
      float s_tot = 0.f;
      for (int r = 0; r < R; ++r) s_tot += set[r * SW];
      const float x0 = set[1];
      float tau, beta, scal;
      if (s_tot == 0.f) {
        tau = 0.f;
        beta = x0;
        scal = 1.f;
      } else {
        const float nrm = sqrtf(fmaf(x0, x0, s_tot));
        beta = (x0 >= 0.f) ? -nrm : nrm;
        tau = (beta - x0) / beta;
        scal = 1.f / (x0 - beta);
      }
      if (!bad && (!(beta == beta) || beta == 0.f || isinf(beta))) bad = j + 1;
      if (tid == 0) taus[j] = tau;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int lr = tid + kQRT * q;
        if (lr < nr && lr > lj) a[q][j] *= scal;
        if (lr == lj) a[q][j] = beta;
      }
      {
        // (2) sums v^T a_c over the rows from the pivot down (v = 1 at the pivot, the scaled
        // column below, 0 above): for c > j the w_c of the update; for c < j the entry
        // G[c][j] = v_c^T v_j of V^T V (every row here lies below pivot c, where column c holds
        // v_c), so V^T V costs no extra exchange
        float d[BW];
#pragma unroll
        for (int c = 0; c < BW; ++c) d[c] = 0.f;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          const int lr = tid + kQRT * q;
          const float v = (lr >= nr || lr < lj) ? 0.f : (lr == lj ? 1.f : a[q][j]);
#pragma unroll
          for (int c = 0; c < BW; ++c)
            if (c != j) d[c] = fmaf(v, a[q][c], d[c]);
        }
        const float wv = warp_transpose_sum32(d, lane);   // column `lane`, this warp's rows
        wsum[warp * (BW + 1) + lane] = wv;
        __syncthreads();
        float* set2 = slots + ph * kQMaxCl * SW;
        ph ^= 1;
        if (tid < bw && tid != j) {
          float t = 0.f;
          for (int w = 0; w < NW; ++w) t += wsum[w * (BW + 1) + tid];
          for (int r = 0; r < R; ++r) cl.map_shared_rank(set2 + rank * SW, r)[tid] = t;
        }
        cl.sync();
        if (tid < bw && tid != j) {
          float t = 0.f;
          for (int r = 0; r < R; ++r) t += set2[r * SW + tid];
          if (tid > j) wtot[tid] = tau * t;
          else G[tid * bw + j] = t;
        }
        __syncthreads();
        if (j + 1 < bw) {
          // (3) a_c -= (tau w_c) v
#pragma unroll
          for (int q = 0; q < RPT; ++q) {
            const int lr = tid + kQRT * q;
            const float v = (lr >= nr || lr < lj) ? 0.f : (lr == lj ? 1.f : a[q][j]);
#pragma unroll
            for (int c = j + 1; c < BW; ++c) a[q][c] = fmaf(-wtot[c], v, a[q][c]);
          }
        }
      }
    }
  }
  // the panel to shared memory for V^T V and the write-back
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int lr = tid + kQRT * q;
    if (lr < nr)
#pragma unroll
      for (int c = 0; c < BW; ++c) P[lr * ldp + c] = a[q][c];
  }
  __syncthreads();
  qr_panel_finish<float>(cl, P, ldp, nr, bw, xch, taus, G, Tl, A, lda, k, r0, tau_out, Tm, info,
                         bad, true);
}

// V[r][i] of panel (k, bw): 1 at r = k + i, the stored entry below, 0 above
template <typename T>
__device__ __forceinline__ T qr_v(const T* A, int64_t lda, int64_t k, int64_t r, int i) {
  const int64_t d = r - (k + i);
  return d == 0 ? T(1) : (d > 0 ? A[r * lda + k + i] : T(0));
}

constexpr int kQCB = 128;   // columns of the trailing matrix per block of the update kernels

// four consecutive shared elements in 16-byte reads (p 16-byte aligned)
__device__ __forceinline__ void ld4(const float* p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&o)[4]) {
  const double2 u = *reinterpret_cast<const double2*>(p);
  const double2 v = *reinterpret_cast<const double2*>(p + 2);
  o[0] = u.x; o[1] = u.y; o[2] = v.x; o[3] = v.y;
}

// Partial X_p = V[rows of chunk p]^T A_trail[rows, columns of block cb] (bw x kQCB), into
// part[(p bw + i) nt + c]. Thread tile: X rows 4 (tid / 32) .. + 3, columns 4 (tid % 32) .. + 3
// (the V row part is the same in a warp, the A part consecutive).
template <typename T>
__global__ void __launch_bounds__(kQT, 3) qr_vta_kernel(const T* __restrict__ A, int64_t lda,
                                                       int64_t m, int64_t k, int bw, int64_t nt,
                                                       int64_t rc, T* __restrict__ part) {
  constexpr int NV = kQChunk * kQMaxBw / kQT, NA = kQChunk * kQCB / kQT;
  __shared__ __align__(16) T Vs[kQChunk][kQMaxBw + 4];
  __shared__ __align__(16) T As[kQChunk][kQCB + 4];
  const int tid = threadIdx.x, cg4 = 4 * (tid & 31), ig4 = 4 * (tid >> 5);
  const int64_t c0 = (int64_t)blockIdx.x * kQCB, p = blockIdx.y;
  const int64_t rbeg = k + p * rc, rend = min(m, rbeg + rc);
  const int64_t col0 = k + bw + c0;
  // the next chunk's share of V and A in registers: every load of a chunk in flight at once,
  // and during the previous chunk's products
  T pv[NV], pa[NA];
  auto fetch = [&](int64_t r) {
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const int e = tid + t * kQT, rr = e / kQMaxBw, i = e % kQMaxBw;
      const int64_t g = r + rr;
      pv[t] = (g < rend && i < bw) ? qr_v(A, lda, k, g, i) : T(0);
    }
#pragma unroll
    for (int t = 0; t < NA; ++t) {
      const int e = tid + t * kQT, rr = e / kQCB, cc = e % kQCB;
      const int64_t g = r + rr;
      pa[t] = (g < rend && c0 + cc < nt) ? A[g * lda + col0 + cc] : T(0);
    }
  };
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  if (rbeg < rend) fetch(rbeg);
  for (int64_t r = rbeg; r < rend; r += kQChunk) {
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const int e = tid + t * kQT;
      Vs[e / kQMaxBw][e % kQMaxBw] = pv[t];
    }
#pragma unroll
    for (int t = 0; t < NA; ++t) {
      const int e = tid + t * kQT;
      As[e / kQCB][e % kQCB] = pa[t];
    }
    __syncthreads();
    if (r + kQChunk < rend) fetch(r + kQChunk);
#pragma unroll 4
    for (int rr = 0; rr < kQChunk; ++rr) {
      T v[4], a[4];
      ld4(&Vs[rr][ig4], v);
      ld4(&As[rr][cg4], a);
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fma(v[x], a[y], acc[x][y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int i = ig4 + x;
    if (i < bw)
#pragma unroll
      for (int y = 0; y < 4; ++y)
        if (c0 + cg4 + y < nt) part[(p * bw + i) * nt + c0 + cg4 + y] = acc[x][y];
  }
}

// Y[:, c] = T^T X[:, c] with X = the sum of the P partials in chunk order; a CTA takes 8
// columns: thread (i, c) sums X[i][c], then forms Y[i][c] = sum_{l <= i} T[l][i] X[l][c].
template <typename T>
__global__ void __launch_bounds__(kQT) qr_reduce_kernel(const T* __restrict__ part, int P,
                                                       int bw, int64_t nt,
                                                       const T* __restrict__ Tm,
                                                       T* __restrict__ Y) {
  __shared__ T Xs[kQMaxBw][9];
  __shared__ T Ts[kQMaxBw][kQMaxBw + 1];
  const int tid = threadIdx.x, i = tid >> 3, cc = tid & 7;
  const int64_t c = (int64_t)blockIdx.x * 8 + cc;
  for (int e = tid; e < bw * bw; e += kQT) Ts[e / bw][e % bw] = Tm[e];
  T sum = T(0);
  if (i < bw && c < nt) {
    const T* src = part + (int64_t)i * nt + c;
    const int64_t stride = (int64_t)bw * nt;
    int q0 = 0;
    for (; q0 + 16 <= P; q0 += 16) {
      T v[16];   // sixteen loads in flight, then the adds in chunk order
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = src[(q0 + q) * stride];
#pragma unroll
      for (int q = 0; q < 16; ++q) sum += v[q];
    }
    for (; q0 < P; ++q0) sum += src[q0 * stride];
  }
  Xs[i][cc] = sum;
  __syncthreads();
  if (i < bw && c < nt) {
    T y = T(0);
    for (int l = 0; l <= i; ++l) y = fma(Ts[l][i], Xs[l][cc], y);
    Y[(int64_t)i * nt + c] = y;
  }
}

// A_trail[rows of chunk p, columns of block cb] -= V Y (Y from qr_reduce_kernel).
// Thread tile: rows 4 (tid / 32) .. + 3 of each 32-row chunk, columns 4 (tid % 32) .. + 3; V
// staged transposed (Vt[i][row]) so that both operands are 16-byte shared reads.
template <typename T>
__global__ void __launch_bounds__(kQT, 3) qr_apply_kernel(T* __restrict__ A, int64_t lda,
                                                         int64_t m, int64_t k, int bw, int64_t nt,
                                                         int64_t rc, const T* __restrict__ Y) {
  constexpr int NV = kQChunk * kQMaxBw / kQT;
  __shared__ __align__(16) T Ys[kQMaxBw][kQCB + 4];
  __shared__ __align__(16) T Vt[kQMaxBw][kQChunk + 4];
  const int tid = threadIdx.x, cg4 = 4 * (tid & 31), rg4 = 4 * (tid >> 5);
  const int64_t c0 = (int64_t)blockIdx.x * kQCB, p = blockIdx.y;
  const int64_t rbeg = k + p * rc, rend = min(m, rbeg + rc);
  const int64_t col0 = k + bw + c0;
  {
    constexpr int NY = kQMaxBw * kQCB / kQT;
    T yv[NY];   // every load of Y's block in flight at once
#pragma unroll
    for (int t = 0; t < NY; ++t) {
      const int e = tid + t * kQT, i = e / kQCB, cc = e % kQCB;
      yv[t] = (i < bw && c0 + cc < nt) ? Y[(int64_t)i * nt + c0 + cc] : T(0);
    }
#pragma unroll
    for (int t = 0; t < NY; ++t) {
      const int e = tid + t * kQT;
      Ys[e / kQCB][e % kQCB] = yv[t];
    }
  }
  // this thread's 4 x 4 entries of A and its share of the V rows for the next chunk, in flight
  // during the current chunk's products
  T pa[4][4], pv[NV];
  auto fetch = [&](int64_t r) {
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int64_t g = r + rg4 + x;
#pragma unroll
      for (int y = 0; y < 4; ++y)
        pa[x][y] = (g < rend && c0 + cg4 + y < nt) ? A[g * lda + col0 + cg4 + y] : T(0);
    }
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const int e = tid + t * kQT, rr = e / kQMaxBw, i = e % kQMaxBw;
      const int64_t g = r + rr;
      pv[t] = (g < rend && i < bw) ? qr_v(A, lda, k, g, i) : T(0);
    }
  };
  if (rbeg < rend) fetch(rbeg);
  for (int64_t r = rbeg; r < rend; r += kQChunk) {
    T a[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) a[x][y] = pa[x][y];
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      const int e = tid + t * kQT;
      Vt[e % kQMaxBw][e / kQMaxBw] = pv[t];
    }
    __syncthreads();
    if (r + kQChunk < rend) fetch(r + kQChunk);
    T acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = T(0);
#pragma unroll 4
    for (int i = 0; i < kQMaxBw; ++i) {
      T v[4], yv[4];
      ld4(&Vt[i][rg4], v);
      ld4(&Ys[i][cg4], yv);
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fma(v[x], yv[y], acc[x][y]);
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int64_t g = r + rg4 + x;
      if (g < rend)
#pragma unroll
        for (int y = 0; y < 4; ++y)
          if (c0 + cg4 + y < nt) A[g * lda + col0 + cg4 + y] = a[x][y] - acc[x][y];
    }
    __syncthreads();
  }
}

// R (upper triangle of the factored matrix's first n rows) into the npad x npad factor M with
// the signs made positive on the diagonal (row i times sign(R_ii), Q absorbs the signs), zero
// below the diagonal and the identity on the padding.
template <typename T, typename Tout>
__global__ void qr_extract_kernel(const T* __restrict__ Aq, int64_t lda, int64_t n, int64_t npad,
                                  Tout* __restrict__ M) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npad * npad) return;
  const int64_t i = e / npad, j = e - i * npad;
  T v;
  if (i < n && j < n) {
    if (j < i) {
      v = T(0);
    } else {
      const T d = Aq[i * lda + i];
      v = (d < T(0)) ? -Aq[i * lda + j] : Aq[i * lda + j];
    }
  } else {
    v = (i == j) ? T(1) : T(0);
  }
  M[e] = (Tout)v;
}

// Aq[i][j] = round_to_prec(A[i][j] d_j^{-1}) for j < n (the column-scaled matrix in u_q),
// from the FP64 master (from64) or the FP32 working copy; columns n .. npad-1 are not read.
template <typename T>
__device__ __forceinline__ T round_q(double v, int prec) {
  if (prec == (int)Prec::FP16) return (T)__half2float(__double2half(v));
  if (prec == (int)Prec::BF16) return (T)__bfloat162float(__double2bfloat16(v));
  if (prec == (int)Prec::FP32) return (T)(float)v;
  return (T)v;
}
template <typename T>
__device__ __forceinline__ T round_qf(float v, int prec) {
  if (prec == (int)Prec::FP16) return (T)__half2float(__float2half_rn(v));
  if (prec == (int)Prec::BF16) return (T)__bfloat162float(__float2bfloat16_rn(v));
  return (T)v;
}
template <typename T>
__global__ void qr_scale_kernel(const void* __restrict__ Asrc, bool from64, int64_t lda_src,
                                int64_t m, int64_t n, const double* __restrict__ dinv,
                                const float* __restrict__ dinv32, int prec, T* __restrict__ Aq,
                                int64_t ldq) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * n) return;
  const int64_t i = e / n, j = e - i * n;
  T v;
  if (from64)
    v = round_q<T>(static_cast<const double*>(Asrc)[i * lda_src + j] * dinv[j], prec);
  else
    v = round_qf<T>(static_cast<const float*>(Asrc)[i * lda_src + j] * dinv32[j], prec);
  Aq[i * ldq + j] = v;
}

}  // namespace

template <typename T>
int qr_panel_width(int64_t m) {
  for (int bw : {32, 16, 8}) {
    if (sizeof(T) == 8 && bw == 32) continue;
    const int64_t rpc = (m + kQMaxCl - 1) / kQMaxCl;
    const size_t smem = sizeof(T) * ((size_t)rpc * (bw + 1) + qr_panel_extra(bw));
    if (smem <= kQSmemMax) return bw;
  }
  return 0;
}

constexpr int kQMaxChunks = 64;   // row chunks of the trailing update (partials per column)

// chunks per column block of the trailing update: about four CTAs per SM over the whole grid,
// at most kQMaxChunks (the partial sums per column), at least 32 rows each
inline int64_t qr_chunks(int64_t mk, int64_t ncb, int num_sms) {
  int64_t P = std::max<int64_t>(1, (4 * (int64_t)std::max(num_sms, 1) + ncb - 1) / ncb);
  P = std::min<int64_t>(P, kQMaxChunks);
  return std::min<int64_t>(P, std::max<int64_t>(1, (mk + kQChunk - 1) / kQChunk));
}

// work layout (elements of T): T_p (kQMaxBw^2) | Y (kQMaxBw n) | partials (kQMaxChunks kQMaxBw n)
template <typename T>
size_t qr_work_elems(int64_t m, int64_t n, int num_sms) {
  (void)m;
  (void)num_sms;
  const size_t nn = (size_t)std::max<int64_t>(n, 1);
  return (size_t)kQMaxBw * kQMaxBw + (size_t)kQMaxBw * nn + (size_t)kQMaxChunks * kQMaxBw * nn;
}

template <typename T>
int launch_qr_scale(const void* Asrc, bool from64, int64_t lda_src, int64_t m, int64_t n,
                    const double* dinv, const float* dinv32, Prec prec, T* Aq, int64_t ldq,
                    cudaStream_t s) {
  const int64_t cnt = m * n;
  qr_scale_kernel<T><<<qr_blocks(cnt, 256), 256, 0, s>>>(Asrc, from64, lda_src, m, n, dinv,
                                                          dinv32, (int)prec, Aq, ldq);
  count_launch();
  return 0;
}

template <typename T>
int launch_qr_r(T* A, int64_t lda, int64_t m, int64_t n, T* tau, T* work, int* info,
                int num_sms, cudaStream_t s) {
  if (m < n || n < 1) return -1;
  const int bw_max = qr_panel_width<T>(m);
  if (bw_max == 0) return -2;
  static const bool attr = [] {
    cudaFuncSetAttribute(qr_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kQSmemMax);
    cudaFuncSetAttribute(qr_panel_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if constexpr (sizeof(T) == 4) {
      for (const void* f : {(const void*)qr_panel_reg_kernel<1>, (const void*)qr_panel_reg_kernel<2>}) {
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kQSmemMax);
        cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      }
    }
    (void)cudaGetLastError();
    return true;
  }();
  (void)attr;
  T* Tm = work;
  T* Y = Tm + kQMaxBw * kQMaxBw;
  T* part = Y + (size_t)kQMaxBw * n;

  for (int64_t k = 0; k < n; k += bw_max) {
    const int bw = (int)std::min<int64_t>(bw_max, n - k);
    const int64_t mk = m - k;
    // cluster size: at least 64 rows per CTA (so the pivot rows stay on rank 0)
    int R = (int)std::max<int64_t>(1, std::min<int64_t>(kQMaxCl, mk / 64));
    if (R > 8) R = 16;
    else if (R > 4) R = 8;
    else if (R > 2) R = 4;
    const int rpc = (int)((mk + R - 1) / R);
    const size_t smem = sizeof(T) * ((size_t)rpc * (bw + 1) + qr_panel_extra(bw));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)R, 1, 1);
    cfg.blockDim = dim3(kQT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)R;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t le;
    if constexpr (sizeof(T) == 4) {
      if (bw_max == kQMaxBw && rpc <= 2 * kQRT) {
        // rows in registers: 512 threads, one or two rows each
        cfg.blockDim = dim3(kQRT, 1, 1);
        cfg.dynamicSmemBytes = sizeof(float) * ((size_t)rpc * (kQMaxBw + 1) + qr_panel_reg_extra());
        if (rpc <= kQRT)
          le = cudaLaunchKernelEx(&cfg, qr_panel_reg_kernel<1>, A, lda, m, k, bw, rpc, tau, Tm,
                                  info);
        else
          le = cudaLaunchKernelEx(&cfg, qr_panel_reg_kernel<2>, A, lda, m, k, bw, rpc, tau, Tm,
                                  info);
      } else {
        le = cudaLaunchKernelEx(&cfg, qr_panel_kernel<T>, A, lda, m, k, bw, rpc, tau, Tm, info);
      }
    } else {
      le = cudaLaunchKernelEx(&cfg, qr_panel_kernel<T>, A, lda, m, k, bw, rpc, tau, Tm, info);
    }
    if (le != cudaSuccess) {
      (void)cudaGetLastError();   // a refused launch: clear it so later checks see only their own
      return -3;
    }
    count_launch();
    const int64_t nt = n - k - bw;
    if (nt <= 0) break;
    const int64_t ncb = (nt + kQCB - 1) / kQCB;
    int64_t P = qr_chunks(mk, ncb, num_sms);
    int64_t rc = (mk + P - 1) / P;
    rc = (rc + kQChunk - 1) / kQChunk * kQChunk;
    P = (mk + rc - 1) / rc;   // <= kQMaxChunks: the partials fit the work buffer
    const dim3 grid((unsigned)ncb, (unsigned)P);
    qr_vta_kernel<T><<<grid, kQT, 0, s>>>(A, lda, m, k, bw, nt, rc, part);
    qr_reduce_kernel<T><<<(unsigned)((nt + 7) / 8), kQT, 0, s>>>(part, (int)P, bw, nt, Tm, Y);
    qr_apply_kernel<T><<<grid, kQT, 0, s>>>(A, lda, m, k, bw, nt, rc, Y);
    count_launch(3);
  }
  return 0;
}

template <typename T, typename Tout>
void launch_qr_extract(const T* Aq, int64_t lda, int64_t n, int64_t npad, Tout* M,
                       cudaStream_t s) {
  qr_extract_kernel<T, Tout><<<qr_blocks(npad * npad, 256), 256, 0, s>>>(Aq, lda, n, npad, M);
  count_launch();
}

template int qr_panel_width<float>(int64_t);
template int qr_panel_width<double>(int64_t);
template size_t qr_work_elems<float>(int64_t, int64_t, int);
template size_t qr_work_elems<double>(int64_t, int64_t, int);
template int launch_qr_scale<float>(const void*, bool, int64_t, int64_t, int64_t, const double*,
                                    const float*, Prec, float*, int64_t, cudaStream_t);
template int launch_qr_scale<double>(const void*, bool, int64_t, int64_t, int64_t, const double*,
                                     const float*, Prec, double*, int64_t, cudaStream_t);
template int launch_qr_r<float>(float*, int64_t, int64_t, int64_t, float*, float*, int*, int,
                                cudaStream_t);
template int launch_qr_r<double>(double*, int64_t, int64_t, int64_t, double*, double*, int*, int,
                                 cudaStream_t);
template void launch_qr_extract<float, float>(const float*, int64_t, int64_t, int64_t, float*,
                                              cudaStream_t);
template void launch_qr_extract<double, double>(const double*, int64_t, int64_t, int64_t,
                                                double*, cudaStream_t);

}  // namespace tls
