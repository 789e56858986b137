// Gram matrix H = A_s^T A_s of the u_f-rounded, column-scaled A on the 5th-generation tensor
// cores (Sec. 3.1 of Oktay & Carson, arXiv 2305.19028: the preconditioner is built from
// fl(A^T A) of the scaled matrix in the low precision u_q; here FP16/BF16 inputs with FP32
// accumulation).
//
// A_s^T is stored n x mpad (K-major: the contraction index m is contiguous). With a partial-sum
// buffer (npad a multiple of 256) gram_tc_wide_kernel below computes 128 x 256 tiles over two
// halves of K; otherwise one CTA computes one 128 x 128 tile (I, J), I <= J, of the upper
// triangle over the whole K and also writes its mirror:
//   warp 0   one thread issues TMA loads (128B-swizzled boxes of 128 rows x 64 K) into a
//            6-stage shared-memory ring, completion tracked by mbarriers;
//   warp 1   allocates 128 TMEM columns and one thread issues tcgen05.mma (M = N = 128,
//            K = 16, FP32 accumulator in TMEM), releasing ring stages with tcgen05.commit;
//   warps 2-5 read the accumulator with tcgen05.ld (32 lanes x 32 columns per load) and
//            store the tile and its transpose to H.
// Every mbarrier wait is bounded by a global-timer deadline: on expiry the kernel records an
// error code, stops issuing work, frees its TMEM and returns (the host then falls back).
#include "tls_internal.h"
#include "tls_ptx.cuh"
#include "tls_tc.cuh"

#include <cuda.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

namespace tls {

namespace {

constexpr int TBM = 128, TBN = 128, TBK = 64;     // tile, K block (64 x 2 B = one 128B atom)
constexpr int STAGES = 6;
constexpr int STAGE_BYTES = TBM * TBK * 2;        // 16 KB per operand per stage
constexpr int THREADS = 192;

// the mbarrier helpers (bounded waits) and the tcgen05 / TMA building blocks shared with the
// other tensor-core kernels
using ptx::mbar_expect_tx;
using ptx::mbar_init;
using ptx::mbar_wait;
using ptx::smem_u32;
using tc::sw128_desc;
using tc::tc_fence_after;
using tc::tc_fence_before;
using tc::tma_load_2d;
using tc::tmem_ld32;
using tc::umma_commit;
using tc::umma_f16;

// Instruction descriptor for kind::f16: D = FP32, A/B = FP16 (fmt 0) or BF16 (fmt 1), both
// K-major, M = 128, N = 128.
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t ab_fmt) {
  return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((uint32_t)(TBN >> 3) << 17) |
         ((uint32_t)(TBM >> 4) << 24);
}

__global__ void __launch_bounds__(THREADS, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap tmap, int nt, int kblocks, int npad,
                   float* __restrict__ H, uint32_t idesc, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the swizzled stages
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sA = smem;                                  // STAGES x 16 KB
  unsigned char* sB = smem + STAGES * STAGE_BYTES;           // STAGES x 16 KB
  __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], acc_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;

  // tile (I, J), I <= J, from the linear block index over the upper triangle
  int t = blockIdx.x, I = 0;
  while (t >= nt - I) { t -= nt - I; ++I; }
  const int J = I + t;
  const bool diag = (I == J);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&acc_bar, 1);
    abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    const uint32_t bytes = diag ? STAGE_BYTES : 2 * STAGE_BYTES;
    int issued = 0;
    for (int kb = 0; kb < kblocks; ++kb) {
      const int s = kb % STAGES, it = kb / STAGES;
      if (kb >= STAGES && !mbar_wait(&empty_bar[s], (it - 1) & 1, err, 1)) {
        abort_flag = 1;
        break;
      }
      if (*(volatile int*)&abort_flag) break;
      mbar_expect_tx(&full_bar[s], bytes);
      tma_load_2d(sA + s * STAGE_BYTES, &tmap, &full_bar[s], kb * TBK, I * TBM);
      if (!diag) tma_load_2d(sB + s * STAGE_BYTES, &tmap, &full_bar[s], kb * TBK, J * TBN);
      issued = kb + 1;
    }
    // make sure no issued copy is still landing in shared memory when the CTA retires
    const int first = issued > STAGES ? issued - STAGES : 0;
    for (int kb = first; kb < issued; ++kb)
      mbar_wait(&full_bar[kb % STAGES], (kb / STAGES) & 1, err, 2);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    bool ok = true;
    for (int kb = 0; kb < kblocks && ok; ++kb) {
      const int s = kb % STAGES, it = kb / STAGES;
      if (!mbar_wait(&full_bar[s], it & 1, err, 3) || *(volatile int*)&abort_flag) {
        abort_flag = 1;
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA + s * STAGE_BYTES);
      const uint32_t b0 = diag ? a0 : smem_u32(sB + s * STAGE_BYTES);
#pragma unroll
      for (int kk = 0; kk < TBK / 16; ++kk) {
        umma_f16(tmem, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc,
                 (kb | kk) != 0 ? 1u : 0u);
      }
      umma_commit(&empty_bar[s]);
    }
    umma_commit(&acc_bar);
  } else if (warp >= 2) {
    // ---------------- epilogue: TMEM -> H (tile and mirror) ----------------
    const int q = warp & 3;                         // TMEM lane quadrant of this warp
    const bool mine = mbar_wait(&acc_bar, 0, err, 4) && !*(volatile int*)&abort_flag;
    const bool ready = __all_sync(0xffffffffu, mine);   // warp-uniform for tcgen05.ld
    tc_fence_after();
    if (ready) {
      const int row = I * TBM + q * 32 + lane;
#pragma unroll 1
      for (int c0 = 0; c0 < TBN; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, r);
        const int col0 = J * TBN + c0;
        if (row < npad && col0 < npad) {
          float4* dst = reinterpret_cast<float4*>(H + (int64_t)row * npad + col0);
#pragma unroll
          for (int v = 0; v < 8; ++v)
            dst[v] = make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]),
                                 __uint_as_float(r[4 * v + 2]), __uint_as_float(r[4 * v + 3]));
          if (!diag) {
#pragma unroll
            for (int cc = 0; cc < 32; ++cc) H[(int64_t)(col0 + cc) * npad + row] = __uint_as_float(r[cc]);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128)
                 : "memory");
  }
}

// The same product with 128 x 256 output tiles and the K range split in two: tile (I, J) covers
// rows 128 I .. + 127 and columns 256 J .. + 255 (the tiles with I <= 2 J + 1, which cover the
// upper triangle), so each 64-wide K block brings 48 KB (A strip, then the B strip as two
// 128-row boxes laid end to end) for twice the MMA work of a 128 x 128 tile, and the 72 tiles of
// n = 2048 times two halves of K give 144 CTAs. Split s writes the entries on or above the
// diagonal of its partial sum, s = 0 into H and s = 1 into part; gram_split_sum_kernel adds
// them in that order and mirrors. Four stages of 48 KB, 256 TMEM columns.
constexpr int WBN = 256, WSTAGES = 4;
constexpr int WSTAGE_BYTES = (TBM + WBN) * TBK * 2;   // 48 KB: A (16 KB) then B (32 KB)

__host__ __device__ constexpr uint32_t idesc_f16_wide(uint32_t ab_fmt) {
  return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((uint32_t)(WBN >> 3) << 17) |
         ((uint32_t)(TBM >> 4) << 24);
}

__global__ void __launch_bounds__(THREADS, 1)
    gram_tc_wide_kernel(const __grid_constant__ CUtensorMap tmap, int nt128, int nt256,
                        int kblocks, int kb_split, int npad, float* __restrict__ H,
                        float* __restrict__ part, uint32_t idesc, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t full_bar[WSTAGES], empty_bar[WSTAGES], acc_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;

  // tile (I, J) from the linear block index: column strips J in order, rows I <= 2 J + 1
  int t = blockIdx.x, J = 0;
  while (J < nt256 - 1 && t >= min(2 * J + 2, nt128)) { t -= min(2 * J + 2, nt128); ++J; }
  const int I = t;
  const int split = blockIdx.y;
  const int kb0 = split * kb_split, kb1 = min(kblocks, kb0 + kb_split);
  const int nkb = max(0, kb1 - kb0);
  float* out = (split == 0) ? H : part;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < WSTAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&acc_bar, 1);
    abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(WBN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int issued = 0;
    for (int q = 0; q < nkb; ++q) {
      const int s = q % WSTAGES, it = q / WSTAGES;
      if (q >= WSTAGES && !mbar_wait(&empty_bar[s], (it - 1) & 1, err, 5)) {
        abort_flag = 1;
        break;
      }
      if (*(volatile int*)&abort_flag) break;
      unsigned char* st = smem + s * WSTAGE_BYTES;
      mbar_expect_tx(&full_bar[s], WSTAGE_BYTES);
      const int kx = (kb0 + q) * TBK;
      tma_load_2d(st, &tmap, &full_bar[s], kx, I * TBM);
      tma_load_2d(st + STAGE_BYTES, &tmap, &full_bar[s], kx, J * WBN);
      tma_load_2d(st + 2 * STAGE_BYTES, &tmap, &full_bar[s], kx, J * WBN + TBM);
      issued = q + 1;
    }
    const int first = issued > WSTAGES ? issued - WSTAGES : 0;
    for (int q = first; q < issued; ++q)
      mbar_wait(&full_bar[q % WSTAGES], (q / WSTAGES) & 1, err, 6);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    bool ok = true;
    for (int q = 0; q < nkb && ok; ++q) {
      const int s = q % WSTAGES, it = q / WSTAGES;
      if (!mbar_wait(&full_bar[s], it & 1, err, 7) || *(volatile int*)&abort_flag) {
        abort_flag = 1;
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t a0 = smem_u32(smem + s * WSTAGE_BYTES);
      const uint32_t b0 = a0 + STAGE_BYTES;
#pragma unroll
      for (int kk = 0; kk < TBK / 16; ++kk)
        umma_f16(tmem, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc,
                 (q | kk) != 0 ? 1u : 0u);
      umma_commit(&empty_bar[s]);
    }
    umma_commit(&acc_bar);
  } else if (warp >= 2) {
    // ---------------- epilogue: TMEM -> the entries on or above the diagonal ----------------
    const int q4 = warp & 3;
    const bool mine = mbar_wait(&acc_bar, 0, err, 8) && !*(volatile int*)&abort_flag;
    const bool ready = __all_sync(0xffffffffu, mine);
    tc_fence_after();
    if (ready) {
      const int row = I * TBM + q4 * 32 + lane;
#pragma unroll 1
      for (int c0 = 0; c0 < WBN; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)c0, r);
        const int col0 = J * WBN + c0;
        if (nkb == 0)
#pragma unroll
          for (int cc = 0; cc < 32; ++cc) r[cc] = 0u;
        if (row < npad && col0 < npad && col0 + 31 >= row) {
          float* dst = out + (int64_t)row * npad + col0;
          if (col0 >= row) {
#pragma unroll
            for (int v = 0; v < 8; ++v)
              reinterpret_cast<float4*>(dst)[v] =
                  make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]),
                              __uint_as_float(r[4 * v + 2]), __uint_as_float(r[4 * v + 3]));
          } else {
#pragma unroll
            for (int cc = 0; cc < 32; ++cc)
              if (col0 + cc >= row) dst[cc] = __uint_as_float(r[cc]);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(WBN)
                 : "memory");
  }
}

// H[r][c] = H[r][c] + part[r][c] for r <= c (the two K halves, in that order), mirrored: one
// CTA per 32 x 32 tile (I, J), I <= J, the sums staged in shared memory so that the transposed
// tile (J, I) is written row by row as well.
__global__ void __launch_bounds__(256) gram_split_sum_kernel(float* __restrict__ H,
                                                             const float* __restrict__ part,
                                                             int64_t npad) {
  __shared__ float tl[32][33];
  const int nt = (int)(npad / 32);
  int t = blockIdx.x, I = 0;
  while (t >= nt - I) { t -= nt - I; ++I; }
  const int J = I + t;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int r = ty; r < 32; r += 8) {
    const int64_t gr = (int64_t)I * 32 + r, gc = (int64_t)J * 32 + tx;
    float v = 0.f;
    if (gr <= gc) {
      const int64_t e = gr * npad + gc;
      v = H[e] + part[e];
      H[e] = v;
    }
    tl[r][tx] = v;
  }
  __syncthreads();
#pragma unroll
  for (int r = ty; r < 32; r += 8) {
    // entry (32 J + r, 32 I + tx) of the lower triangle mirrors (32 I + tx, 32 J + r)
    if (I != J || r > tx) H[((int64_t)J * 32 + r) * npad + (int64_t)I * 32 + tx] = tl[tx][r];
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encoder() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      (void)cudaGetLastError();
  });
  return fn;
}

}  // namespace

namespace tc {
bool encode_kmajor_map(CUtensorMap* map, const void* base, bool bf16, uint64_t k_extent,
                       uint64_t rows, uint64_t row_bytes, uint32_t box_k, uint32_t box_rows) {
  EncodeTiledFn enc = get_encoder();
  if (enc == nullptr || (reinterpret_cast<uintptr_t>(base) & 15) != 0 || row_bytes % 16 != 0)
    return false;
  const cuuint64_t gdim[2] = {(cuuint64_t)k_extent, (cuuint64_t)rows};
  const cuuint64_t gstride[1] = {(cuuint64_t)row_bytes};
  const cuuint32_t box[2] = {box_k, box_rows};
  const cuuint32_t estride[2] = {1, 1};
  return enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
             const_cast<void*>(base), gdim, gstride, box, estride,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}
}  // namespace tc

bool gram_tc_available() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && get_encoder() != nullptr;
}

int gram_tc_error(int* err, cudaStream_t s) {
  int h = 0;
  cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  if (h) cudaMemsetAsync(err, 0, sizeof(int), s);
  return h;
}

bool launch_gram_tc(const void* AsT, Prec prec, int64_t n, int64_t npad, int64_t mpad, float* H,
                    int* err, cudaStream_t s, float* part) {
  if (prec != Prec::FP16 && prec != Prec::BF16) return false;
  if (!gram_tc_available()) return false;
  if ((reinterpret_cast<uintptr_t>(AsT) & 15) != 0 || (mpad % TBK) != 0 || err == nullptr)
    return false;
  CUtensorMap map;
  const cuuint64_t gdim[2] = {(cuuint64_t)mpad, (cuuint64_t)npad};
  const cuuint64_t gstride[1] = {(cuuint64_t)mpad * 2};
  const cuuint32_t box[2] = {(cuuint32_t)TBK, (cuuint32_t)TBM};
  const cuuint32_t estride[2] = {1, 1};
  CUresult r = get_encoder()(&map,
                             prec == Prec::FP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                             2, const_cast<void*>(AsT), gdim, gstride, box, estride,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return false;
  const int nt = (int)((npad + TBM - 1) / TBM);
  const int tiles = nt * (nt + 1) / 2;
  const size_t smem = 2 * STAGES * STAGE_BYTES + 1024;
  static const bool attr = [smem] {   // thread-safe one-time initialisation
    cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return true;
  }();
  (void)attr;
  const int kblocks = (int)(mpad / TBK);
  if (part != nullptr && npad >= WBN && npad % WBN == 0 && kblocks >= 2) {
    // 128 x 256 tiles, K in two halves
    const size_t wsmem = WSTAGES * (size_t)WSTAGE_BYTES + 1024;
    static const bool wattr = [wsmem] {
      cudaFuncSetAttribute(gram_tc_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)wsmem);
      return true;
    }();
    (void)wattr;
    const int nt256 = (int)(npad / WBN);
    int wtiles = 0;
    for (int J = 0; J < nt256; ++J) wtiles += std::min(2 * J + 2, nt);
    const int kb_split = (kblocks + 1) / 2;
    gram_tc_wide_kernel<<<dim3((unsigned)wtiles, 2), THREADS, wsmem, s>>>(
        map, nt, nt256, kblocks, kb_split, (int)npad, H, part,
        idesc_f16_wide(prec == Prec::FP16 ? 0u : 1u), err);
    const int64_t t32 = npad / 32;
    gram_split_sum_kernel<<<(unsigned)(t32 * (t32 + 1) / 2), 256, 0, s>>>(H, part, npad);
    count_launch(2);
  } else {
    const uint32_t idesc = idesc_f16(prec == Prec::FP16 ? 0u : 1u);
    gram_tc_kernel<<<tiles, THREADS, smem, s>>>(map, nt, kblocks, (int)npad, H, idesc, err);
    count_launch();
  }
  launch_set_identity_pad(H, false, n, npad, s);
  return cudaGetLastError() == cudaSuccess;
}

}  // namespace tls
