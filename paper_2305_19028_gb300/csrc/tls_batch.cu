// C ABI of the packed batched path (include/tls.h, tls_batch_*): many dense TLS problems of
// uneven sizes solved together by RQI-PCGTLS (Alg. 2 / Alg. 4), each phase one launch for the
// whole batch (kernels in k_batch.cu). The host only sequences the phases, runs the shift ladder
// of the factorisation and the precision fallback, and reads one counter per RQI step.
#include "../../include/tls.h"
#include "../../include/tls_debug.h"
#include "tls_batch_internal.h"
#include "tls_options.h"

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

using tls::Prec;
using namespace tls::bat;

struct tls_batch {
  int count = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  std::vector<std::pair<void*, size_t>> bufs;
  std::vector<BProb> hp;
  std::vector<BTile> ht;

  std::vector<double> hshift;
  std::vector<int> hinfo, shifts, fail_pivot, fallbacks, broke;
  std::vector<tls_prec> uf_used;
  BArrays a{};
  BProb* dprobs = nullptr;
  BTile* dtiles = nullptr;
  BState* dst = nullptr;
  GTile* dgram = nullptr;           // Gram CTA list and split-tile reduction list
  size_t cap_gram = 0;
  void* gwork = nullptr;            // Gram partial tiles of row-split tiles
  size_t cap_gwork = 0;
  CTask* dtask = nullptr;           // Cholesky / inverse task lists
  size_t cap_task = 0;
  int* dlist = nullptr;             // problem list of the current launch sequence
  int* dact_probs = nullptr;        // its active problems (compacted)
  int* dact_tiles = nullptr;        // their row tiles (compacted)
  double* dshift = nullptr;
  int* dinfo = nullptr;
  int* dcount = nullptr;
  int* hcount = nullptr;            // pinned
  int ntiles = 0;
  int cap_tiles = 0;                // capacity of the tile arrays and partial buffers
  int64_t cap_poff = 0;
  int64_t tile_bytes[kNumCfg] = {};  // row-tile size (FP32 bytes) per pass lane layout
  int tuned_u = 0;                  // sizeof the u type the tile sizes were tuned for
  bool use_graph = true;            // replay the solve as one CUDA graph
  struct Graph {
    std::vector<double> key;
    cudaGraphExec_t exec;
    unsigned long long kernels;     // kernel nodes (for the launch count)
  };
  std::vector<Graph> graphs;        // a few captured solves (full list, fallback subsets)
  // selector network
  float* dsel = nullptr;            // parameters (TLS_MLP_PARAMS) + mean (16) + scale (16)
  bool has_sel = false;
  float* dF = nullptr;              // features (count x 16)
  float* dnet = nullptr;            // network outputs (count x 4)
  int* dfint = nullptr;             // shifts and failed pivot per problem (2 x count)
  double* dcgtol = nullptr;         // per-problem PCGTLS tolerance
  std::vector<double> hcgtol;
  bool use_cgtol = false;
  std::vector<int> sel_class;       // the network's choice per problem (-1: none)
  Prec u = Prec::FP32;
  bool factored = false;
  tls_options opt{};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double t_factor_ms = 0.0;
  // per-class kernel timing (tls_batch_profile_enable): event pairs around every launch
  bool prof = false;
  std::vector<cudaEvent_t> evpool;
  size_t evused = 0;
  std::vector<std::pair<int, size_t>> marks;
  int64_t prof_cnt[TLS_PROF_NCLASSES] = {};
  double prof_ms[TLS_PROF_NCLASSES] = {};
  int64_t prof_elems[TLS_PROF_NCLASSES] = {};   // entries of A read by the pass launches
};

namespace {

void set_err(tls_batch* bt, const std::string& s) { bt->err = s; }

void* balloc(tls_batch* bt, size_t bytes) {
  void* p = tls::hook_alloc(bytes, bt->stream);
  if (p) bt->bufs.push_back({p, bytes});
  return p;
}

// Return a device buffer of the batch once the work queued on its stream is done.
void bfree(tls_batch* bt, void* p) {
  cudaStreamSynchronize(bt->stream);
  for (size_t i = 0; i < bt->bufs.size(); ++i)
    if (bt->bufs[i].first == p) {
      tls::hook_free(p, bt->bufs[i].second, bt->stream);
      bt->bufs.erase(bt->bufs.begin() + (long)i);
      return;
    }
}

// Grow a device buffer owned by the batch to at least `bytes` (contents are not kept).
bool ensure_cap(tls_batch* bt, void** p, size_t* cap, size_t bytes) {
  if (*p && *cap >= bytes) return true;
  if (*p) {
    cudaStreamSynchronize(bt->stream);
    for (size_t i = 0; i < bt->bufs.size(); ++i)
      if (bt->bufs[i].first == *p) {
        tls::hook_free(*p, bt->bufs[i].second, bt->stream);
        bt->bufs.erase(bt->bufs.begin() + (long)i);
        break;
      }
    *p = nullptr;
    *cap = 0;
  }
  *p = balloc(bt, bytes);
  if (!*p) return false;
  *cap = bytes;
  return true;
}

tls_status cuda_st(tls_batch* bt, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return TLS_OK;
  set_err(bt, std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? TLS_ERR_OOM : TLS_ERR_CUDA;
}

#define BT_CK(call)                                           \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_st(bt, e_, #call);     \
  } while (0)
#define BT_CK_LAUNCH(what)                                    \
  do {                                                        \
    cudaError_t e_ = cudaGetLastError();                      \
    if (e_ != cudaSuccess) return cuda_st(bt, e_, what);      \
  } while (0)

int64_t rup(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// Row tiles of roughly `target` bytes of FP32 data (at least one row)
int64_t rows_per_tile(int64_t lda, int64_t target) {
  return std::max<int64_t>(1, target / (lda * 4));
}

constexpr int64_t kTileMin = 64 * 1024;   // smallest tile the partial buffers are sized for
constexpr int64_t kTileCand[] = {64 * 1024, 128 * 1024, 256 * 1024, 512 * 1024, 1024 * 1024};

// (Re)build the row-tile table from tile_bytes: tiles of every problem, their partial-sum
// offsets (poff) and counts. Host side only.
void build_tiles(tls_batch* bt) {
  bt->ht.clear();
  int64_t poff = 0;
  for (size_t i = 0; i < bt->hp.size(); ++i) {
    BProb& P = bt->hp[i];
    const int64_t rpt = std::min<int64_t>(rows_per_tile(P.lda, bt->tile_bytes[P.cfg]), P.m);
    P.tile0 = (int)bt->ht.size();
    P.poff = poff;
    for (int64_t r = 0; r < P.m; r += rpt) {
      BTile t{};
      t.prob = (int)i;
      t.row0 = (int)r;
      t.rows = (int)std::min<int64_t>(rpt, P.m - r);
      bt->ht.push_back(t);
    }
    P.ntiles = (int)bt->ht.size() - P.tile0;
    poff += (int64_t)P.ntiles * P.lda;
  }
  bt->ntiles = (int)bt->ht.size();
}

double unit_roundoff(Prec p) {
  switch (p) {
    case Prec::FP16: return std::ldexp(1.0, -11);
    case Prec::BF16: return std::ldexp(1.0, -8);
    case Prec::FP32: return std::ldexp(1.0, -24);
    default: return std::ldexp(1.0, -53);
  }
}

cudaEvent_t pool_event(tls_batch* bt) {
  if (bt->evused == bt->evpool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    bt->evpool.push_back(e);
  }
  return bt->evpool[bt->evused++];
}

// Brackets the launches of one scope with an event pair when profiling is on.
struct BProfScope {
  tls_batch* bt;
  int cls;
  size_t i0 = 0;
  bool on = false;
  BProfScope(tls_batch* b, int c) : bt(b), cls(c) {
    if (!bt->prof) return;
    cudaEvent_t e = pool_event(bt);
    if (!e) return;
    i0 = bt->evused - 1;
    on = cudaEventRecord(e, bt->stream) == cudaSuccess;
  }
  ~BProfScope() {
    if (!on) return;
    cudaEvent_t e = pool_event(bt);
    if (!e || cudaEventRecord(e, bt->stream) != cudaSuccess) return;
    bt->marks.push_back({cls, i0});
  }
};

void prof_collect(tls_batch* bt) {
  if (!bt->prof || bt->marks.empty()) {
    bt->evused = 0;
    bt->marks.clear();
    return;
  }
  cudaStreamSynchronize(bt->stream);
  for (auto& mk : bt->marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, bt->evpool[mk.second], bt->evpool[mk.second + 1]) ==
        cudaSuccess) {
      bt->prof_cnt[mk.first] += 1;
      bt->prof_ms[mk.first] += ms;
    }
  }
  bt->marks.clear();
  bt->evused = 0;
}

void destroy(tls_batch* bt) {
  if (!bt) return;
  if (bt->stream) cudaStreamSynchronize(bt->stream);
  for (cudaEvent_t e : bt->evpool) cudaEventDestroy(e);
  for (auto& g : bt->graphs) cudaGraphExecDestroy(g.exec);
  for (auto& b : bt->bufs) tls::hook_free(b.first, b.second, bt->stream);
  tls::host_free(bt->hcount);
  if (bt->ev0) cudaEventDestroy(bt->ev0);
  if (bt->ev1) cudaEventDestroy(bt->ev1);
  if (bt->own_stream && bt->stream) cudaStreamDestroy(bt->stream);
  delete bt;
}

tls_status upload_list(tls_batch* bt, const std::vector<int>& L) {
  BT_CK(cudaMemcpyAsync(bt->dlist, L.data(), sizeof(int) * L.size(), cudaMemcpyHostToDevice,
                        bt->stream));
  return TLS_OK;
}

tls_status upload_tasks(tls_batch* bt, const std::vector<CTask>& tk) {
  if (!ensure_cap(bt, reinterpret_cast<void**>(&bt->dtask), &bt->cap_task,
                  sizeof(CTask) * std::max<size_t>(tk.size(), 1))) {
    set_err(bt, "device allocation failed (factor task lists)");
    return TLS_ERR_OOM;
  }
  if (!tk.empty())
    BT_CK(cudaMemcpyAsync(bt->dtask, tk.data(), sizeof(CTask) * tk.size(), cudaMemcpyHostToDevice,
                          bt->stream));
  return TLS_OK;
}

// Task lists of the blocked Cholesky of the problems in L: for every block step s the diagonal
// blocks, then the panel blocks, then the trailing blocks. off: 3 entries per step + the end.
int chol_tasks(const tls_batch* bt, const std::vector<int>& L, std::vector<CTask>& tk,
               std::vector<int>& off) {
  int steps = 0;
  for (int i : L) steps = std::max(steps, (int)(bt->hp[(size_t)i].npb / kNB));
  tk.clear();
  off.clear();
  for (int st = 0; st < steps; ++st) {
    off.push_back((int)tk.size());
    for (int i : L)
      if (st < (int)(bt->hp[(size_t)i].npb / kNB)) tk.push_back(CTask{i, st, st, st});
    off.push_back((int)tk.size());
    for (int i : L) {
      const int nb = (int)(bt->hp[(size_t)i].npb / kNB);
      for (int bj = st + 1; bj < nb; ++bj) tk.push_back(CTask{i, st, st, bj});
    }
    off.push_back((int)tk.size());
    for (int i : L) {
      const int nb = (int)(bt->hp[(size_t)i].npb / kNB);
      for (int bi = st + 1; bi < nb; ++bi)
        for (int bj = bi; bj < nb; ++bj) tk.push_back(CTask{i, st, bi, bj});
    }
  }
  off.push_back((int)tk.size());
  return steps;
}

// Task lists of W = R^{-1} by block diagonals: level d holds the blocks (I, I + d).
int trtri_tasks(const tls_batch* bt, const std::vector<int>& L, std::vector<CTask>& tk,
                std::vector<int>& off) {
  int levels = 0;
  for (int i : L) levels = std::max(levels, (int)(bt->hp[(size_t)i].npb / kNB));
  tk.clear();
  off.clear();
  for (int d = 0; d < levels; ++d) {
    off.push_back((int)tk.size());
    for (int i : L) {
      const int nb = (int)(bt->hp[(size_t)i].npb / kNB);
      for (int I = 0; I + d < nb; ++I) tk.push_back(CTask{i, d, I, I + d});
    }
  }
  off.push_back((int)tk.size());
  return levels;
}

// Gram + shift ladder + triangular inverse for the problems in L at factor precision p;
// problems whose every shift breaks down move on to the next precision.
template <typename T>
tls_status factor_list(tls_batch* bt, std::vector<int> L, Prec p) {
  cudaStream_t st = bt->stream;
  while (!L.empty()) {
    for (int i : L) bt->hp[(size_t)i].prec = (int)p;
    BT_CK(cudaMemcpyAsync(bt->dprobs, bt->hp.data(), sizeof(BProb) * bt->hp.size(),
                          cudaMemcpyHostToDevice, st));
    // Gram CTAs of the listed problems: every upper 64 x 64 tile, its rows split into chunks
    // of kc rows (FP64 rows cost far more on this GPU, so they are split finer), longest
    // chunks first; split tiles are summed in slot order afterwards.
    const bool c64 = (p == Prec::FP64);
    const int64_t kc = c64 ? 512 : 2048;
    std::vector<GTile> gl, gred;
    int slots = 0;
    for (int i : L) {
      const BProb& P = bt->hp[(size_t)i];
      const int nbk = (int)(P.npb / kNB);
      const int ns = (int)((P.m + kc - 1) / kc);
      for (int bi = 0; bi < nbk; ++bi)
        for (int bj = bi; bj < nbk; ++bj) {
          if (ns == 1) {
            gl.push_back(GTile{i, bi, bj, 0, (int)P.m, -1, 0, 0});
            continue;
          }
          gred.push_back(GTile{i, bi, bj, 0, ns, slots, 0, 0});
          for (int k = 0; k < ns; ++k)
            gl.push_back(GTile{i, bi, bj, (int)(k * kc), (int)std::min<int64_t>(P.m, (k + 1) * kc),
                               slots + k, 0, 0});
          slots += ns;
        }
    }
    std::stable_sort(gl.begin(), gl.end(), [](const GTile& x, const GTile& y) {
      return (x.r1 - x.r0) > (y.r1 - y.r0);
    });
    const size_t ngl = gl.size(), ngr = gred.size();
    gl.insert(gl.end(), gred.begin(), gred.end());
    if (!ensure_cap(bt, reinterpret_cast<void**>(&bt->dgram), &bt->cap_gram,
                    sizeof(GTile) * std::max<size_t>(gl.size(), 1)) ||
        !ensure_cap(bt, &bt->gwork, &bt->cap_gwork,
                    (c64 ? 8 : 4) * (size_t)kNB * kNB * std::max(slots, 1))) {
      set_err(bt, "device allocation failed (Gram workspace)");
      return TLS_ERR_OOM;
    }
    BT_CK(cudaMemcpyAsync(bt->dgram, gl.data(), sizeof(GTile) * gl.size(), cudaMemcpyHostToDevice,
                          st));
    {
      BProfScope pr(bt, TLS_PROF_GRAM);
      if (c64)
        launch_gram<double>(bt->a, bt->dgram, (int)ngl, bt->dgram + ngl, (int)ngr, bt->gwork, st);
      else
        launch_gram<float>(bt->a, bt->dgram, (int)ngl, bt->dgram + ngl, (int)ngr, bt->gwork, st);
    }
    BT_CK_LAUNCH("batched Gram");
    // shift ladder (the diagonal perturbation of low-precision Cholesky)
    const bool low = (p == Prec::FP16 || p == Prec::BF16);
    const int first = (low && bt->opt.shift_first) ? 1 : 0;
    const int max_shift = std::max(0, bt->opt.max_shifts);
    const double u = unit_roundoff(p);
    std::vector<int> pending = L, ok;
    for (int sh = first; sh <= max_shift + first && !pending.empty(); ++sh) {
      const double shift = (sh == 0) ? 0.0 : 2.0 * u * std::pow(4.0, sh - 1);
      for (int i : pending) bt->hshift[(size_t)i] = shift;
      BT_CK(cudaMemcpyAsync(bt->dshift, bt->hshift.data(), sizeof(double) * bt->count,
                            cudaMemcpyHostToDevice, st));
      tls_status s = upload_list(bt, pending);
      if (s != TLS_OK) return s;
      std::vector<CTask> tk;
      std::vector<int> off;
      const int steps = chol_tasks(bt, pending, tk, off);
      s = upload_tasks(bt, tk);
      if (s != TLS_OK) return s;
      {
        BProfScope pr(bt, TLS_PROF_CHOL);
        if (c64)
          launch_chol<double>(bt->a, bt->dlist, (int)pending.size(), bt->dshift, bt->dinfo,
                              bt->dtask, off.data(), steps, st);
        else
          launch_chol<float>(bt->a, bt->dlist, (int)pending.size(), bt->dshift, bt->dinfo,
                             bt->dtask, off.data(), steps, st);
      }
      BT_CK_LAUNCH("batched Cholesky");
      BT_CK(cudaMemcpyAsync(bt->hinfo.data(), bt->dinfo, sizeof(int) * bt->count,
                            cudaMemcpyDeviceToHost, st));
      BT_CK(cudaStreamSynchronize(st));
      std::vector<int> failed;
      for (int i : pending) {
        const int inf = bt->hinfo[(size_t)i];
        if (inf == 0) {
          ok.push_back(i);
        } else {
          failed.push_back(i);
          bt->shifts[(size_t)i] += 1;
          bt->fail_pivot[(size_t)i] = inf - 1;
        }
      }
      pending.swap(failed);
    }
    if (!ok.empty()) {
      std::vector<CTask> tk;
      std::vector<int> off;
      const int levels = trtri_tasks(bt, ok, tk, off);
      tls_status s = upload_tasks(bt, tk);
      if (s != TLS_OK) return s;
      BProfScope pr(bt, TLS_PROF_TRTRI);
      if (c64) launch_trtri<double, T>(bt->a, bt->dtask, off.data(), levels, st);
      else launch_trtri<float, T>(bt->a, bt->dtask, off.data(), levels, st);
      BT_CK_LAUNCH("batched triangular inverse");
      for (int i : ok) bt->uf_used[(size_t)i] = (tls_prec)(int)p;
    }
    if (pending.empty()) break;
    if (p == Prec::FP64) {
      for (int i : pending) bt->broke[(size_t)i] = 1;
      break;
    }
    p = (p == Prec::FP32) ? Prec::FP64 : Prec::FP32;
    L = pending;
  }
  return TLS_OK;
}

// Lock-step RQI-PCGTLS over the problems in L (Alg. 2 with the PCGTLS of Alg. 3 / 4).
//
// The launch sequence of a whole solve needs no host knowledge of which problems are still
// active: after every stop test the count_active kernel compacts the active problems and their
// row tiles into device lists, and the pass / per-problem kernels run persistent grids over
// those lists. The sequence is issued for k = 1 .. max_rqi + 1 (a stopped problem drops out of
// the lists; once none is left the remaining kernels find empty lists and return at once), so
// it is captured once as a CUDA graph and replayed: one graph launch and one synchronisation
// per solve. With profiling on, the same sequence runs eagerly with one synchronisation per RQI
// step (event pairs per launch class and per-step work accounting).
struct SolveGrid {
  int pass, post;
};

template <typename T>
void issue_solve(tls_batch* bt, int cnt, const SolveParams& sp, const SolveGrid& g, bool eager,
                 tls_status* err) {
  cudaStream_t st = bt->stream;
  const BArrays& a = bt->a;
  const int* dl = bt->dact_probs;
  const int* tl = bt->dact_tiles;
  const int* n_prob = bt->dcount;       // device counts written by count_active
  const int* n_tile = bt->dcount + 1;
  int64_t elems = 0;
  auto refresh = [&]() -> bool {        // returns false when no problem is left (eager only)
    {
      BProfScope pr(bt, TLS_PROF_VEC);
      launch_count_active(a, bt->dlist, cnt, bt->dcount, bt->dact_probs, bt->dact_tiles, st);
    }
    if (!eager) return true;
    if (cudaMemcpyAsync(bt->hcount, bt->dcount, 4 * sizeof(int), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      *err = TLS_ERR_CUDA;
      return false;
    }
    unsigned long long el = 0ull;
    std::memcpy(&el, bt->hcount + 2, sizeof(el));
    elems = (int64_t)el;
    return bt->hcount[0] > 0;
  };
  auto resid = [&](int mode) {
    {
      BProfScope pr(bt, TLS_PROF_RESID_PASS);
      // FP32 working precision: the residual in double-FP32 arithmetic on A32 + Alo
      if (std::is_same<T, float>::value && a.Alo != nullptr)
        launch_pass_resid_df(a, tl, n_tile, g.pass, st);
      else
        launch_pass_resid(a, tl, n_tile, g.pass, st);
      if (bt->prof) bt->prof_elems[TLS_PROF_RESID_PASS] += elems;
    }
    BProfScope pr(bt, TLS_PROF_RESID_REDUCE);
    launch_resid_post<T>(a, dl, n_prob, g.post, mode, sp, st);
  };
  auto pcg_step = [&](int nr) {
    {
      BProfScope pr(bt, nr == 2 ? TLS_PROF_PCG_PASS2 : TLS_PROF_PCG_PASS1);
      launch_pass_pcg<T>(a, tl, n_tile, g.pass, nr, st);
      if (bt->prof) bt->prof_elems[nr == 2 ? TLS_PROF_PCG_PASS2 : TLS_PROF_PCG_PASS1] += elems;
    }
    BProfScope pr(bt, TLS_PROF_PCG_REDUCE);
    launch_pcg_post<T>(a, dl, n_prob, g.post, st);
  };
  {
    BProfScope pr(bt, TLS_PROF_VEC);
    launch_solve_init<T>(a, bt->dlist, cnt, st);
  }
  if (!refresh()) return;
  // line 1: LS start, x = 0 residual (f = -A^T b), PCGTLS with sigma^2 = 0
  resid(kResidLs);
  for (int j = 0; j < std::max(1, bt->opt.ls_iters); ++j) pcg_step(1);
  {
    BProfScope pr(bt, TLS_PROF_VEC);
    launch_ls_finish<T>(a, dl, n_prob, g.post, st);
  }
  // lines 2-5: sigma_0^2 and the inverse-iteration step
  resid(kResidStart);
  for (int k = 1; k <= sp.max_rqi + 1; ++k) {
    resid(kResidRqi);
    if (!refresh()) return;
    const int steps = sp.cg_fixed ? (k + 1) : std::max(1, sp.cg_max);
    for (int j = 0; j < steps; ++j) pcg_step(2);
    BProfScope pr(bt, TLS_PROF_VEC);
    launch_rqi_update<T>(a, dl, n_prob, g.post, st);
  }
}

template <typename T>
tls_status solve_list(tls_batch* bt, const std::vector<int>& L, const SolveParams& sp) {
  cudaStream_t st = bt->stream;
  const int cnt = (int)L.size();
  if (cnt == 0) return TLS_OK;
  tls_status s = upload_list(bt, L);
  if (s != TLS_OK) return s;
  int tiles = 0;
  for (int i : L) tiles += bt->hp[(size_t)i].ntiles;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  SolveGrid g{std::max(1, std::min(tiles, 4 * sms)), std::max(1, std::min(cnt, 4 * sms))};
  tls_status err = TLS_OK;
  if (bt->prof || !bt->use_graph) {
    issue_solve<T>(bt, cnt, sp, g, true, &err);
    if (err != TLS_OK) return err;
    BT_CK_LAUNCH("batched solve");
    return TLS_OK;
  }
  // graph: captured once per (problem list, solve parameters, grids), replayed afterwards
  std::vector<double> key = {(double)sizeof(T), (double)cnt, (double)tiles, (double)g.pass,
                             (double)g.post, sp.tol, sp.psi_accept, (double)sp.max_rqi,
                             (double)sp.psi_rule_ge, (double)sp.cg_fixed, (double)sp.cg_max,
                             sp.cg_tol, (double)bt->opt.ls_iters, bt->a.cg_tol ? 1.0 : 0.0};
  for (int i : L) key.push_back((double)i);
  tls_batch::Graph* gr = nullptr;
  for (auto& c : bt->graphs)
    if (c.key == key) gr = &c;
  if (!gr) {
    if (bt->graphs.size() >= 4) {
      cudaGraphExecDestroy(bt->graphs.front().exec);
      bt->graphs.erase(bt->graphs.begin());
    }
    cudaGraph_t graph = nullptr;
    const unsigned long long l0 = tls::g_launches.load();
    BT_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    issue_solve<T>(bt, cnt, sp, g, false, &err);
    const cudaError_t ce = cudaStreamEndCapture(st, &graph);
    // capturing launches nothing: the nodes are counted when the graph is launched
    const unsigned long long nodes = tls::g_launches.load() - l0;
    tls::g_launches.fetch_sub(nodes);
    if (err != TLS_OK) return err;
    BT_CK(ce);
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    BT_CK(ie);
    bt->graphs.push_back({key, exec, nodes});
    gr = &bt->graphs.back();
  }
  BT_CK(cudaGraphLaunch(gr->exec, st));
  tls::count_launch((int)gr->kernels);
  return TLS_OK;
}

// Autotuner of the row-tile size per pass lane layout (size bucket): for each layout present,
// every candidate size is timed on this batch's own problems of that bucket (the paired FP32
// PCGTLS pass and the FP64 residual pass, weighted as in a solve: ~5 PCGTLS passes per
// residual pass); the fastest is kept and cached per device, u type and bucket.
std::map<std::tuple<int, int, int>, int64_t> g_tile_tune;
std::mutex g_tile_mu;

tls_status upload_tiles(tls_batch* bt) {
  BT_CK(cudaMemcpyAsync(bt->dprobs, bt->hp.data(), sizeof(BProb) * bt->hp.size(),
                        cudaMemcpyHostToDevice, bt->stream));
  BT_CK(cudaMemcpyAsync(bt->dtiles, bt->ht.data(), sizeof(BTile) * bt->ht.size(),
                        cudaMemcpyHostToDevice, bt->stream));
  return TLS_OK;
}

template <typename T>
tls_status tune_tiles(tls_batch* bt) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaStream_t st = bt->stream;
  bool present[kNumCfg] = {};
  for (const BProb& P : bt->hp) present[P.cfg] = true;
  for (int c = 0; c < kNumCfg; ++c) {
    if (!present[c]) continue;
    const auto key = std::make_tuple(dev, c, (int)sizeof(T));
    {
      std::lock_guard<std::mutex> lk(g_tile_mu);
      auto it = g_tile_tune.find(key);
      if (it != g_tile_tune.end()) {
        bt->tile_bytes[c] = it->second;
        continue;
      }
    }
    double best = 1e30;
    int64_t best_b = bt->tile_bytes[c];
    for (int64_t cand : kTileCand) {
      bt->tile_bytes[c] = cand;
      build_tiles(bt);
      std::vector<int> tl;
      for (const BProb& P : bt->hp)
        if (P.cfg == c)
          for (int t = 0; t < P.ntiles; ++t) tl.push_back(P.tile0 + t);
      tls_status s = upload_tiles(bt);
      if (s != TLS_OK) return s;
      BT_CK(cudaMemcpyAsync(bt->dact_tiles, tl.data(), sizeof(int) * tl.size(),
                            cudaMemcpyHostToDevice, st));
      const int nt = (int)tl.size();
      auto resid_pass = [&]() {
        if (std::is_same<T, float>::value && bt->a.Alo != nullptr)
          launch_pass_resid_df(bt->a, bt->dact_tiles, nullptr, nt, st);
        else
          launch_pass_resid(bt->a, bt->dact_tiles, nullptr, nt, st);
      };
      launch_pass_pcg<T>(bt->a, bt->dact_tiles, nullptr, nt, 2, st);   // warm-up
      resid_pass();
      BT_CK(cudaEventRecord(bt->ev0, st));
      for (int r = 0; r < 3; ++r) launch_pass_pcg<T>(bt->a, bt->dact_tiles, nullptr, nt, 2, st);
      BT_CK(cudaEventRecord(bt->ev1, st));
      BT_CK(cudaEventSynchronize(bt->ev1));
      float ms_p = 0.f, ms_r = 0.f;
      cudaEventElapsedTime(&ms_p, bt->ev0, bt->ev1);
      BT_CK(cudaEventRecord(bt->ev0, st));
      resid_pass();
      BT_CK(cudaEventRecord(bt->ev1, st));
      BT_CK(cudaEventSynchronize(bt->ev1));
      cudaEventElapsedTime(&ms_r, bt->ev0, bt->ev1);
      BT_CK_LAUNCH("tile autotuner");
      const double cost = ms_p / 3.0 + 0.2 * ms_r;
      if (cost < best) {
        best = cost;
        best_b = cand;
      }
    }
    bt->tile_bytes[c] = best_b;
    std::lock_guard<std::mutex> lk(g_tile_mu);
    g_tile_tune[key] = best_b;
  }
  build_tiles(bt);
  return upload_tiles(bt);
}

// Features of every problem from its current factor (normalised by the selector's mean /
// scale when `norm`) into bt->dF.
template <typename T>
tls_status compute_features(tls_batch* bt, bool norm) {
  cudaStream_t st = bt->stream;
  std::vector<int> fi((size_t)3 * bt->count);
  std::vector<int> l32, l64;
  for (int i = 0; i < bt->count; ++i) {
    fi[(size_t)i] = bt->shifts[(size_t)i];
    fi[(size_t)bt->count + i] = bt->fail_pivot[(size_t)i];
    fi[(size_t)2 * bt->count + i] = (int)bt->uf_used[(size_t)i];
    if (bt->broke[(size_t)i]) continue;
    (bt->uf_used[(size_t)i] == TLS_FP64 ? l64 : l32).push_back(i);
  }
  BT_CK(cudaMemcpyAsync(bt->dfint, fi.data(), sizeof(int) * fi.size(), cudaMemcpyHostToDevice, st));
  const float* mean = norm ? bt->dsel + TLS_MLP_PARAMS : nullptr;
  const float* scale = norm ? bt->dsel + TLS_MLP_PARAMS + 16 : nullptr;
  for (int pass = 0; pass < 2; ++pass) {
    const std::vector<int>& L = pass ? l64 : l32;
    if (L.empty()) continue;
    tls_status s = upload_list(bt, L);
    if (s != TLS_OK) return s;
    const int* fi_d = bt->dfint;
    if (pass)
      launch_features<double, T>(bt->a, bt->dlist, (int)L.size(), fi_d, fi_d + bt->count,
                                 fi_d + 2 * bt->count, bt->dshift, mean, scale, bt->dF, st);
    else
      launch_features<float, T>(bt->a, bt->dlist, (int)L.size(), fi_d, fi_d + bt->count,
                                fi_d + 2 * bt->count, bt->dshift, mean, scale, bt->dF, st);
    BT_CK_LAUNCH("selector features");
  }
  return TLS_OK;
}

// TLS_AUTO: FP16 factor, features, network, then each problem refactored at its chosen u_f.
template <typename T>
tls_status factor_auto(tls_batch* bt) {
  std::vector<int> all((size_t)bt->count);
  for (int i = 0; i < bt->count; ++i) all[(size_t)i] = i;
  tls_status s = factor_list<T>(bt, all, Prec::FP16);
  if (s != TLS_OK || !bt->has_sel) return s;
  s = compute_features<T>(bt, true);
  if (s != TLS_OK) return s;
  tls::mlp::launch_mlp_forward(bt->dsel, bt->count, bt->dF, bt->dnet, bt->stream);
  BT_CK_LAUNCH("selector network");
  std::vector<float> out((size_t)4 * bt->count);
  BT_CK(cudaMemcpyAsync(out.data(), bt->dnet, sizeof(float) * out.size(), cudaMemcpyDeviceToHost,
                        bt->stream));
  BT_CK(cudaStreamSynchronize(bt->stream));
  std::vector<int> to_bf16, to_fp32;
  for (int i = 0; i < bt->count; ++i) {
    const float* o = out.data() + (size_t)4 * i;
    int c = 0;
    if (o[1] > o[c]) c = 1;
    if (o[2] > o[c]) c = 2;
    bt->sel_class[(size_t)i] = c;
    bt->hcgtol[(size_t)i] = std::pow(10.0, std::min(-1.0, std::max(-12.0, (double)o[3])));
    if (bt->broke[(size_t)i] || bt->uf_used[(size_t)i] != TLS_FP16) continue;
    if (c == 1) to_bf16.push_back(i);
    if (c == 2) to_fp32.push_back(i);
  }
  if (!to_bf16.empty()) {
    s = factor_list<T>(bt, to_bf16, Prec::BF16);
    if (s != TLS_OK) return s;
  }
  if (!to_fp32.empty()) {
    s = factor_list<T>(bt, to_fp32, Prec::FP32);
    if (s != TLS_OK) return s;
  }
  BT_CK(cudaMemcpyAsync(bt->dcgtol, bt->hcgtol.data(), sizeof(double) * bt->count,
                        cudaMemcpyHostToDevice, bt->stream));
  bt->use_cgtol = true;
  return TLS_OK;
}

template <typename T>
tls_status batch_solve_impl(tls_batch* bt, double tol, int max_rqi, std::vector<BState>& hst) {
  const tls_options& o = bt->opt;
  SolveParams sp{};
  sp.tol = tol;
  sp.psi_accept = o.psi_accept;
  sp.max_rqi = max_rqi;
  sp.psi_rule_ge = o.psi_rule_ge;
  sp.cg_fixed = o.cg_fixed;
  sp.cg_max = o.cg_max;
  sp.cg_tol = o.cg_tol;
  bt->a.cg_tol = bt->use_cgtol ? bt->dcgtol : nullptr;
  std::vector<int> L;
  for (int i = 0; i < bt->count; ++i)
    if (!bt->broke[(size_t)i]) L.push_back(i);
  for (int round = 0; round < 3 && !L.empty(); ++round) {
    tls_status s = solve_list<T>(bt, L, sp);
    if (s != TLS_OK) return s;
    BT_CK(cudaMemcpyAsync(hst.data(), bt->dst, sizeof(BState) * hst.size(),
                          cudaMemcpyDeviceToHost, bt->stream));
    BT_CK(cudaStreamSynchronize(bt->stream));
    if (!o.fallback || round == 2) break;
    // precision fallback: a problem that ended on max_rqi gets a factor one precision up
    std::vector<int> to32, to64;
    for (int i : L) {
      if (hst[(size_t)i].stop != TLS_STOP_MAX_RQI) continue;
      const tls_prec uf = bt->uf_used[(size_t)i];
      if (uf == TLS_FP64) continue;
      (uf == TLS_FP32 ? to64 : to32).push_back(i);
      bt->fallbacks[(size_t)i] += 1;
    }
    if (!to32.empty()) {
      tls_status s2 = factor_list<T>(bt, to32, Prec::FP32);
      if (s2 != TLS_OK) return s2;
    }
    if (!to64.empty()) {
      tls_status s2 = factor_list<T>(bt, to64, Prec::FP64);
      if (s2 != TLS_OK) return s2;
    }
    L.clear();
    for (int i : to32) if (!bt->broke[(size_t)i]) L.push_back(i);
    for (int i : to64) if (!bt->broke[(size_t)i]) L.push_back(i);
  }
  return TLS_OK;
}

}  // namespace

extern "C" {

tls_status tls_batch_create_dense(tls_batch** out, int count, const int64_t* m, const int64_t* n,
                                  const double* const* A, const int64_t* lda,
                                  const double* const* b, int on_device, void* stream) {
  if (!out) return TLS_ERR_ARG;
  *out = nullptr;
  if (count < 1 || !m || !n || !A || !lda || !b) return TLS_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    if (m[i] < n[i] || n[i] < 1 || n[i] > TLS_BATCH_MAX_N || lda[i] < n[i] || !A[i] || !b[i] ||
        m[i] > (int64_t)INT32_MAX)
      return TLS_ERR_ARG;
  }
  tls_batch* bt = new tls_batch();
  bt->count = count;
  if (stream) {
    bt->stream = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete bt;
      return TLS_ERR_CUDA;
    }
    bt->own_stream = true;
  }
  // layout
  int64_t offA = 0, offB = 0, offV = 0, offM = 0;
  bt->hp.resize((size_t)count);
  for (int i = 0; i < count; ++i) {
    BProb& P = bt->hp[(size_t)i];
    P.m = m[i];
    P.n = n[i];
    P.lda = rup(n[i], 4);
    P.npb = rup(n[i], kNB);
    P.offA = offA;
    P.offB = offB;
    P.offV = offV;
    P.offM = offM;
    P.cfg = cfg_for(P.lda);
    P.prec = (int)Prec::FP16;
    offA += rup(P.m * P.lda, 64);
    offB += rup(P.m, 32);
    offV += P.npb;
    offM += P.npb * P.npb;
  }
  // the smallest tiles give the most tiles and partials: size the buffers for them
  for (int c = 0; c < kNumCfg; ++c) bt->tile_bytes[c] = kTileMin;
  build_tiles(bt);
  const int64_t poff = bt->hp.back().poff + (int64_t)bt->hp.back().ntiles * bt->hp.back().lda;
  bt->cap_tiles = bt->ntiles;
  bt->cap_poff = poff;
  const size_t vbytes = sizeof(double) * (size_t)offV;
  BArrays& a = bt->a;
  bt->dprobs = static_cast<BProb*>(balloc(bt, sizeof(BProb) * count));
  bt->dtiles = static_cast<BTile*>(balloc(bt, sizeof(BTile) * bt->ht.size()));
  bt->dst = static_cast<BState*>(balloc(bt, sizeof(BState) * count));
  bt->dlist = static_cast<int*>(balloc(bt, sizeof(int) * count));
  bt->dact_probs = static_cast<int*>(balloc(bt, sizeof(int) * count));
  bt->dact_tiles = static_cast<int*>(balloc(bt, sizeof(int) * bt->ht.size()));
  bt->dshift = static_cast<double*>(balloc(bt, sizeof(double) * count));
  bt->dinfo = static_cast<int*>(balloc(bt, sizeof(int) * count));
  bt->dcount = static_cast<int*>(balloc(bt, 4 * sizeof(int)));
  bt->dsel = static_cast<float*>(balloc(bt, sizeof(float) * (TLS_MLP_PARAMS + 32)));
  bt->dF = static_cast<float*>(balloc(bt, sizeof(float) * 16 * count));
  bt->dnet = static_cast<float*>(balloc(bt, sizeof(float) * 4 * count));
  bt->dfint = static_cast<int*>(balloc(bt, sizeof(int) * 3 * count));
  bt->dcgtol = static_cast<double*>(balloc(bt, sizeof(double) * count));
  double* A64 = static_cast<double*>(balloc(bt, sizeof(double) * (size_t)offA));
  a.A32 = static_cast<float*>(balloc(bt, sizeof(float) * (size_t)offA));
  a.Alo = static_cast<float*>(balloc(bt, sizeof(float) * (size_t)offA));
  double* bb = static_cast<double*>(balloc(bt, sizeof(double) * (size_t)offB));
  a.d = static_cast<double*>(balloc(bt, vbytes));
  a.dinv = static_cast<double*>(balloc(bt, vbytes));
  a.dinv32 = static_cast<float*>(balloc(bt, sizeof(float) * (size_t)offV));
  a.x = static_cast<double*>(balloc(bt, vbytes));
  a.xbest = static_cast<double*>(balloc(bt, vbytes));
  a.f = static_cast<double*>(balloc(bt, vbytes));
  a.vw = balloc(bt, 2 * vbytes);
  a.vs = balloc(bt, 2 * vbytes);
  a.vp = balloc(bt, 2 * vbytes);
  a.vq = balloc(bt, 2 * vbytes);
  a.H = balloc(bt, sizeof(double) * (size_t)offM);
  a.R = balloc(bt, sizeof(double) * (size_t)offM);
  a.W = balloc(bt, sizeof(double) * (size_t)offM);
  a.WT = balloc(bt, sizeof(double) * (size_t)offM);
  a.partU = balloc(bt, sizeof(double) * 2 * (size_t)std::max<int64_t>(poff, 1));
  a.part64 = static_cast<double*>(balloc(bt, sizeof(double) * (size_t)std::max<int64_t>(poff, 1)));
  a.spart = static_cast<double*>(balloc(bt, sizeof(double) * 4 * bt->ht.size()));
  if (!bt->dprobs || !bt->dtiles || !bt->dst || !bt->dlist || !bt->dshift ||
      !bt->dact_probs || !bt->dact_tiles || !bt->dsel || !bt->dF || !bt->dnet || !bt->dfint ||
      !bt->dcgtol ||
      !bt->dinfo || !bt->dcount || !A64 || !a.A32 || !a.Alo || !bb || !a.d || !a.dinv ||
      !a.dinv32 ||
      !a.x || !a.xbest || !a.f || !a.vw || !a.vs || !a.vp || !a.vq || !a.H || !a.R || !a.W ||
      !a.WT || !a.partU || !a.part64 || !a.spart) {
    destroy(bt);
    return TLS_ERR_OOM;
  }
  a.A64 = A64;
  a.b = bb;
  a.probs = bt->dprobs;
  a.tiles = bt->dtiles;
  a.st = bt->dst;
  cudaStream_t st = bt->stream;
  bt->hcount = static_cast<int*>(tls::host_alloc(4 * sizeof(int)));
  cudaError_t e = bt->hcount ? cudaSuccess : cudaErrorMemoryAllocation;
  if (e == cudaSuccess) e = cudaEventCreate(&bt->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&bt->ev1);
  if (e == cudaSuccess) e = cudaMemsetAsync(A64, 0, sizeof(double) * (size_t)offA, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(bb, 0, sizeof(double) * (size_t)offB, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(bt->dcount, 0, 4 * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(bt->dst, 0, sizeof(BState) * count, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.H, 0, sizeof(double) * (size_t)offM, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.vw, 0, 2 * vbytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.vs, 0, 2 * vbytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.vp, 0, 2 * vbytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.vq, 0, 2 * vbytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.x, 0, vbytes, st);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int i = 0; i < count && e == cudaSuccess; ++i)
    e = cudaMemcpyAsync(bb + bt->hp[(size_t)i].offB, b[i], sizeof(double) * m[i], kind, st);
  // A into the padded layout: rows of a few hundred bytes make row-by-row (2D) copies slow, so
  // each problem's block is copied whole (host data through a staging buffer, in chunks) and one
  // kernel per chunk places the rows and checks them for NaN / Inf
  {
    std::vector<RepackJob> jobs;
    RepackJob* djobs = nullptr;
    double* stage = nullptr;
    int64_t cap = 0;   // staging capacity (doubles)
    if (!on_device) {
      int64_t most = 0, total = 0;
      for (int i = 0; i < count; ++i) {
        const int64_t span = (m[i] - 1) * lda[i] + n[i];
        most = std::max(most, span);
        total += span;
      }
      cap = std::max(most, std::min<int64_t>(total, (int64_t)64 << 20));   // <= 512 MB
      stage = static_cast<double*>(balloc(bt, sizeof(double) * (size_t)cap));
    }
    djobs = static_cast<RepackJob*>(balloc(bt, sizeof(RepackJob) * (size_t)count));
    if (!djobs || (!on_device && !stage)) e = cudaErrorMemoryAllocation;
    int64_t used = 0;
    auto flush = [&]() {
      if (jobs.empty() || e != cudaSuccess) return;
      e = cudaMemcpyAsync(djobs, jobs.data(), sizeof(RepackJob) * jobs.size(),
                          cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) {
        launch_repack(A64, djobs, (int)jobs.size(), bt->dcount, sms, st);
        e = cudaGetLastError();
      }
      // the next chunk's copies into the staging buffer and its job list queue behind this
      // kernel on the same stream (and the pageable job upload has read `jobs` on return)
      jobs.clear();
      used = 0;
    };
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
      const BProb& P = bt->hp[(size_t)i];
      const int64_t span = (m[i] - 1) * lda[i] + n[i];
      const double* src = A[i];
      if (!on_device) {
        if (used + span > cap) flush();
        if (e != cudaSuccess) break;
        e = cudaMemcpyAsync(stage + used, A[i], sizeof(double) * (size_t)span,
                            cudaMemcpyHostToDevice, st);
        src = stage + used;
        used += span;
      }
      jobs.push_back({src, lda[i], P.offA, P.m, P.n, P.lda});
    }
    flush();
    if (stage) bfree(bt, stage);
    if (djobs) bfree(bt, djobs);
  }
  if (e == cudaSuccess) {
    tls::launch_nonfinite(bb, offB, bt->dcount, sms, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bt->hcount, bt->dcount, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && bt->hcount[0] != 0) {
    destroy(bt);
    return TLS_ERR_ARG;   // NaN or Inf in some A_i or b_i
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bt->dprobs, bt->hp.data(), sizeof(BProb) * count, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bt->dtiles, bt->ht.data(), sizeof(BTile) * bt->ht.size(),
                        cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    destroy(bt);
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? TLS_ERR_OOM : TLS_ERR_CUDA;
  }
  bt->hshift.assign((size_t)count, 0.0);
  bt->hinfo.assign((size_t)count, 0);
  bt->shifts.assign((size_t)count, 0);
  bt->fail_pivot.assign((size_t)count, -1);
  bt->fallbacks.assign((size_t)count, 0);
  bt->broke.assign((size_t)count, 0);
  bt->uf_used.assign((size_t)count, TLS_FP16);
  bt->hcgtol.assign((size_t)count, 0.0);
  bt->sel_class.assign((size_t)count, -1);
  // column norms d_j, ||A||_F^2, ||b||^2 and the FP32 working copy, for the whole batch
  std::vector<int> all((size_t)count);
  for (int i = 0; i < count; ++i) all[(size_t)i] = i;
  if (upload_list(bt, all) != TLS_OK) {
    destroy(bt);
    return TLS_ERR_CUDA;
  }
  launch_pass_colnorm(a, bt->ntiles, st);
  launch_colnorm_post(a, bt->dlist, count, st);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    destroy(bt);
    return TLS_ERR_CUDA;
  }
  *out = bt;
  return TLS_OK;
}

tls_status tls_batch_factor(tls_batch* bt, tls_prec u_f, const tls_options* opt) {
  if (!bt || (int)u_f < 0 || (int)u_f > (int)TLS_AUTO) return TLS_ERR_ARG;
  tls_options o;
  if (opt) o = *opt;
  else tls_default_options(&o);
  if (o.u != TLS_FP32 && o.u != TLS_FP64) return TLS_ERR_ARG;
  if (!o.mode_A) {
    set_err(bt, "the packed batch implements the A-explicit PCGTLS operator (mode_A = 1)");
    return TLS_ERR_ARG;
  }
  if (const char* why = tls::options_error(o)) {
    set_err(bt, why);
    return TLS_ERR_ARG;
  }
  bt->opt = o;
  bt->u = (o.u == TLS_FP64) ? Prec::FP64 : Prec::FP32;
  bt->factored = false;
  std::fill(bt->shifts.begin(), bt->shifts.end(), 0);
  std::fill(bt->fail_pivot.begin(), bt->fail_pivot.end(), -1);
  std::fill(bt->fallbacks.begin(), bt->fallbacks.end(), 0);
  std::fill(bt->broke.begin(), bt->broke.end(), 0);
  std::fill(bt->sel_class.begin(), bt->sel_class.end(), -1);
  bt->use_cgtol = false;
  std::vector<int> all((size_t)bt->count);
  for (int i = 0; i < bt->count; ++i) all[(size_t)i] = i;
  const int usz = (bt->u == Prec::FP64) ? 8 : 4;
  if (bt->tuned_u != usz) {
    tls_status s0 = (usz == 8) ? tune_tiles<double>(bt) : tune_tiles<float>(bt);
    if (s0 != TLS_OK) return s0;
    bt->tuned_u = usz;
  }
  BT_CK(cudaEventRecord(bt->ev0, bt->stream));
  tls_status s;
  if (u_f == TLS_AUTO)
    s = (bt->u == Prec::FP64) ? factor_auto<double>(bt) : factor_auto<float>(bt);
  else
    s = (bt->u == Prec::FP64) ? factor_list<double>(bt, all, (Prec)(int)u_f)
                              : factor_list<float>(bt, all, (Prec)(int)u_f);
  if (s != TLS_OK) return s;
  BT_CK(cudaEventRecord(bt->ev1, bt->stream));
  BT_CK(cudaEventSynchronize(bt->ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, bt->ev0, bt->ev1);
  bt->t_factor_ms = ms;
  prof_collect(bt);
  bt->factored = true;
  for (int i = 0; i < bt->count; ++i)
    if (bt->broke[(size_t)i]) {
      set_err(bt, "Cholesky breakdown at every shift and precision for problem " +
                      std::to_string(i));
      return TLS_ERR_FACTOR_BREAKDOWN;
    }
  return TLS_OK;
}

tls_status tls_batch_solve(tls_batch* bt, double tol, int max_rqi, double* const* x,
                           double* sigma, tls_info* infos, tls_status* per_problem) {
  if (!bt || !x || !sigma || max_rqi < 0 || !(tol >= 0.0)) return TLS_ERR_ARG;
  if (max_rqi > 100) {
    // the captured graph holds every RQI step up to max_rqi + 1 with its k + 1 PCGTLS steps
    set_err(bt, "max_rqi must be in [0, 100] for the packed batch");
    return TLS_ERR_ARG;
  }
  if (!bt->factored) {
    set_err(bt, "tls_batch_solve called before tls_batch_factor");
    return TLS_ERR_STATE;
  }
  std::vector<BState> hst((size_t)bt->count);
  BT_CK(cudaEventRecord(bt->ev0, bt->stream));
  tls_status s = (bt->u == Prec::FP64) ? batch_solve_impl<double>(bt, tol, max_rqi, hst)
                                       : batch_solve_impl<float>(bt, tol, max_rqi, hst);
  if (s != TLS_OK) return s;
  BT_CK(cudaEventRecord(bt->ev1, bt->stream));
  int64_t nv = 0;
  for (const BProb& P : bt->hp) nv += P.npb;
  std::vector<double> xb((size_t)nv);
  BT_CK(cudaMemcpyAsync(xb.data(), bt->a.xbest, sizeof(double) * (size_t)nv,
                        cudaMemcpyDeviceToHost, bt->stream));
  BT_CK(cudaStreamSynchronize(bt->stream));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, bt->ev0, bt->ev1);
  prof_collect(bt);
  tls_status first = TLS_OK;
  for (int i = 0; i < bt->count; ++i) {
    const BProb& P = bt->hp[(size_t)i];
    const BState& S = hst[(size_t)i];
    const tls_status si = bt->broke[(size_t)i] ? TLS_ERR_FACTOR_BREAKDOWN : TLS_OK;
    if (per_problem) per_problem[i] = si;
    if (si != TLS_OK && first == TLS_OK) first = si;
    if (x[i]) std::memcpy(x[i], xb.data() + P.offV, sizeof(double) * (size_t)P.n);
    sigma[i] = std::sqrt(std::max(S.best_s2, 0.0));
    if (infos) {
      tls_info& in = infos[i];
      std::memset(&in, 0, sizeof(in));
      in.stop_reason = S.stop;
      in.rqi_steps = S.k;
      in.best_k = S.best_k;
      in.cg_iters = S.cg_total;
      in.shifts = bt->shifts[(size_t)i];
      in.not_spd = S.not_spd_any;
      in.u_f_used = bt->uf_used[(size_t)i];
      in.psi_final = S.best_psi;
      in.sigma2 = S.best_s2;
      in.shift = bt->hshift[(size_t)i];
      in.t_factor_ms = bt->t_factor_ms;
      in.t_solve_ms = ms;
      in.fail_pivot = bt->fail_pivot[(size_t)i];
      in.pass_variant[0] = in.pass_variant[1] = P.cfg;
      in.n_psi = std::min(S.n_psi, 24);
      for (int k = 0; k < in.n_psi; ++k) in.psi_hist[k] = S.psi_hist[k];
      in.fallbacks = bt->fallbacks[(size_t)i];
      in.fallback_trigger = in.fallbacks ? TLS_TRIGGER_MAX_RQI : TLS_TRIGGER_NONE;
      in.constr1 = in.constr2 = in.constr2_scaled = NAN;
      in.mode_switch_k = -1;
    }
  }
  return first;
}

void tls_batch_destroy(tls_batch* bt) { destroy(bt); }

tls_status tls_batch_set_selector(tls_batch* bt, const float* params, const float* mean,
                                  const float* scale) {
  if (!bt) return TLS_ERR_ARG;
  if (!params || !mean || !scale) {
    bt->has_sel = false;
    return TLS_OK;
  }
  for (int k = 0; k < 16; ++k)
    if (!(scale[k] != 0.f) || !std::isfinite(scale[k]) || !std::isfinite(mean[k])) return TLS_ERR_ARG;
  std::vector<float> h((size_t)TLS_MLP_PARAMS + 32);
  std::memcpy(h.data(), params, sizeof(float) * TLS_MLP_PARAMS);
  std::memcpy(h.data() + TLS_MLP_PARAMS, mean, sizeof(float) * 16);
  std::memcpy(h.data() + TLS_MLP_PARAMS + 16, scale, sizeof(float) * 16);
  BT_CK(cudaMemcpyAsync(bt->dsel, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice,
                        bt->stream));
  BT_CK(cudaStreamSynchronize(bt->stream));
  bt->has_sel = true;
  return TLS_OK;
}

tls_status tls_batch_features(tls_batch* bt, float* F_host) {
  if (!bt || !F_host) return TLS_ERR_ARG;
  if (!bt->factored) return TLS_ERR_STATE;
  tls_status s = (bt->u == Prec::FP64) ? compute_features<double>(bt, false)
                                       : compute_features<float>(bt, false);
  if (s != TLS_OK) return s;
  BT_CK(cudaMemcpyAsync(F_host, bt->dF, sizeof(float) * 16 * bt->count, cudaMemcpyDeviceToHost,
                        bt->stream));
  BT_CK(cudaStreamSynchronize(bt->stream));
  return TLS_OK;
}

tls_status tls_batch_profile_enable(tls_batch* bt, int on) {
  if (!bt) return TLS_ERR_ARG;
  bt->prof = on != 0;
  for (int k = 0; k < TLS_PROF_NCLASSES; ++k) {
    bt->prof_cnt[k] = 0;
    bt->prof_ms[k] = 0.0;
    bt->prof_elems[k] = 0;
  }
  bt->marks.clear();
  bt->evused = 0;
  return TLS_OK;
}

tls_status tls_batch_profile_get(const tls_batch* bt, int cls, int64_t* count, double* ms) {
  if (!bt || cls < 0 || cls >= TLS_PROF_NCLASSES) return TLS_ERR_ARG;
  if (count) *count = bt->prof_cnt[cls];
  if (ms) *ms = bt->prof_ms[cls];
  return TLS_OK;
}

tls_status tls_batch_profile_elems(const tls_batch* bt, int cls, int64_t* elems) {
  if (!bt || cls < 0 || cls >= TLS_PROF_NCLASSES || !elems) return TLS_ERR_ARG;
  *elems = bt->prof_elems[cls];
  return TLS_OK;
}

tls_status tls_batch_export_factor(tls_batch* bt, int i, double* R_host, double* d_host,
                                   double* H_host) {
  if (!bt || i < 0 || i >= bt->count) return TLS_ERR_ARG;
  if (!bt->factored || bt->broke[(size_t)i]) return TLS_ERR_STATE;
  const BProb& P = bt->hp[(size_t)i];
  const int64_t n = P.n, npb = P.npb;
  const bool c64 = bt->uf_used[(size_t)i] == TLS_FP64;
  const size_t es = c64 ? 8 : 4;
  std::vector<unsigned char> buf(es * (size_t)(npb * npb));
  auto fetch = [&](const void* base, double* out, bool mirror) -> tls_status {
    const unsigned char* src = static_cast<const unsigned char*>(base) + es * (size_t)P.offM;
    BT_CK(cudaMemcpyAsync(buf.data(), src, buf.size(), cudaMemcpyDeviceToHost, bt->stream));
    BT_CK(cudaStreamSynchronize(bt->stream));
    for (int64_t r = 0; r < n; ++r)
      for (int64_t c = 0; c < n; ++c) {
        const int64_t rr = (mirror && c < r) ? c : r, cc = (mirror && c < r) ? r : c;
        const size_t e = (size_t)(rr * npb + cc);
        out[r * n + c] = c64 ? reinterpret_cast<const double*>(buf.data())[e]
                             : (double)reinterpret_cast<const float*>(buf.data())[e];
      }
    return TLS_OK;
  };
  if (R_host) {
    tls_status s = fetch(bt->a.R, R_host, false);
    if (s != TLS_OK) return s;
  }
  if (H_host) {
    tls_status s = fetch(bt->a.H, H_host, true);
    if (s != TLS_OK) return s;
  }
  if (d_host) {
    BT_CK(cudaMemcpyAsync(d_host, bt->a.d + P.offV, sizeof(double) * (size_t)n,
                          cudaMemcpyDeviceToHost, bt->stream));
    BT_CK(cudaStreamSynchronize(bt->stream));
  }
  return TLS_OK;
}

const char* tls_batch_last_error(const tls_batch* bt) { return bt ? bt->err.c_str() : ""; }

}  // extern "C"
