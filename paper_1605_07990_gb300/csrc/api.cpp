// C ABI of libssa (include/ssa.h) and the host side of the Stop-and-Stare
// drivers: device workspaces, sampling batches, and the FP64 stopping rules of
// SSA (Algorithm 1) and D-SSA (Algorithm 4) evaluated from integer counts.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <chrono>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ssa.h"
#include "kernels.h"

using namespace ssa;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
namespace {
thread_local char g_err[512] = "";

ssa_status fail(ssa_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

#define CU(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) {                                                                      \
      return fail(e_ == cudaErrorMemoryAllocation ? SSA_E_NOMEM : SSA_E_CUDA, "%s failed: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                             \
    }                                                                                             \
  } while (0)

#define TRY(call)                   \
  do {                              \
    ssa_status s_ = (call);         \
    if (s_ != SSA_OK) return s_;    \
  } while (0)

template <typename T>
ssa_status dev_alloc(T** p, size_t count, cudaStream_t st) {
  *p = nullptr;
  if (count == 0) count = 1;
  CU(cudaMallocAsync(reinterpret_cast<void**>(p), sizeof(T) * count, st));
  return SSA_OK;
}

template <typename T>
void dev_free(T*& p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
  p = nullptr;
}

// Grow a device array to `want` elements keeping the first `keep`.
template <typename T>
ssa_status dev_grow(T** p, int64_t* cap, int64_t want, int64_t keep, cudaStream_t st) {
  if (want <= *cap) return SSA_OK;
  T* q = nullptr;
  TRY(dev_alloc(&q, (size_t)want, st));
  if (*p && keep > 0) CU(cudaMemcpyAsync(q, *p, sizeof(T) * (size_t)keep, cudaMemcpyDeviceToDevice, st));
  if (*p) cudaFreeAsync(*p, st);
  *p = q;
  *cap = want;
  return SSA_OK;
}

}  // namespace

namespace {
std::atomic<long long> g_wait_polls{GREEDY_DEFAULT_WAIT_POLLS};
}  // namespace

long long ssa::greedy_wait_polls() { return g_wait_polls.load(std::memory_order_relaxed); }

// Lets other translation units of the library report an error message.
void ssa::set_last_error(const char* msg) {
  std::strncpy(g_err, msg, sizeof(g_err) - 1);
  g_err[sizeof(g_err) - 1] = 0;
}

namespace {
double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
}  // namespace

// ---------------------------------------------------------------------------
// graph
// ---------------------------------------------------------------------------
struct ssa_graph {
  int device = 0;
  int64_t n = 0, m = 0;
  int weighting = 0;
  int64_t* off = nullptr;
  uint2* edge = nullptr;
  uint64_t* wc_pow = nullptr;  // weighted cascade: gap powers per in-degree (build_wc_pow)
  int wc_pow_k = 0;
  int64_t bytes = 0;
  // IC sampler hand-over sizes chosen by the autotuner (-1: not tuned yet)
  mutable std::mutex tune_mu;
  mutable int tuned_mid_cap = -1;
  mutable int tuned_heavy = 0x7FFFFFFF;
  mutable int tuned_small_qcap = 0;  // queue of the small CTAs (0: min(n, 2^20))
  mutable int tuned_warp_global = 0;  // weighted-cascade IC: the global-bitmap warp tier takes every sample
  mutable int tuned_lane_tier = 1;    // weighted-cascade IC: the lane tier runs first
  GraphView view() const {
    GraphView v;
    v.n = n;
    v.m = m;
    v.off = off;
    v.edge = edge;
    v.wc_pow = wc_pow;
    v.wc_pow_k = wc_pow_k;
    return v;
  }
};

// ---------------------------------------------------------------------------
// per-stream execution context: kernel counting and optional event timing
// ---------------------------------------------------------------------------
namespace {
// NVTX range for a profiler's timeline (a no-op unless a tool is attached);
// ends when the scope does, error returns included
struct NvtxRange {
  nvtxRangeId_t id;
  explicit NvtxRange(const char* name) : id(nvtxRangeStartA(name)) {}
  ~NvtxRange() { nvtxRangeEnd(id); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

const char* const kClassName[SSA_K_COUNT] = {"ssa sample (warp tiers)", "ssa sample (CTA tier)", "ssa index",
                                              "ssa greedy", "ssa stare"};

struct Exec {
  cudaStream_t st = nullptr;
  int num_sms = 152;
  int64_t launches = 0;
  bool timing = false;
  struct Ev {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Ev> evs;
  std::vector<cudaEvent_t> spare;

  cudaEvent_t take() {
    if (!spare.empty()) {
      cudaEvent_t e = spare.back();
      spare.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  // begin/end a region of one kernel class: an NVTX range always, CUDA
  // events when timing.  Regions are used LIFO; one left open by an error
  // return stays on the list until collect().
  struct Mark {
    int ev;
    nvtxRangeId_t nv;
  };
  std::vector<Mark> marks;
  int begin(int cls) {
    Mark m{-1, nvtxRangeStartA(kClassName[cls])};
    if (timing) {
      Ev e{cls, take(), take()};
      cudaEventRecord(e.a, st);
      evs.push_back(e);
      m.ev = (int)evs.size() - 1;
    }
    marks.push_back(m);
    return (int)marks.size() - 1;
  }
  void end(int h) {
    if (h < 0 || (size_t)h >= marks.size()) return;
    const Mark m = marks[(size_t)h];
    if (m.ev >= 0) cudaEventRecord(evs[(size_t)m.ev].b, st);
    nvtxRangeEnd(m.nv);
    if ((size_t)h + 1 == marks.size()) marks.pop_back();
  }
  void collect(ssa_kstat* ks) {
    for (auto& e : evs) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess && ks) {
        ks[e.cls].launches += 1;
        ks[e.cls].ms += ms;
      }
      spare.push_back(e.a);
      spare.push_back(e.b);
    }
    evs.clear();
    marks.clear();
  }
  ~Exec() {
    for (auto& e : evs) {
      cudaEventDestroy(e.a);
      cudaEventDestroy(e.b);
    }
    for (auto e : spare) cudaEventDestroy(e);
  }
};

// The RR pool: flat (node, sample) entries in batch order plus per-sample
// extents; `bounds` records (sets, entries) after every batch so that the
// sets [0, N) of a batch boundary N are exactly the entries [0, E(N)).
struct DevPool {
  int64_t cap_entries = 0, cap_sets = 0;
  int32_t* nodes = nullptr;
  int32_t* samp = nullptr;
  int64_t* set_start = nullptr;
  int32_t* set_len = nullptr;
  int64_t count = 0, entries = 0;
  std::vector<std::pair<int64_t, int64_t>> bounds{{0, 0}};
  int64_t byte_cap = 0;

  int64_t bytes_for(int64_t ents, int64_t sets) const { return ents * 12 + sets * 14; }
  // entries range covering samples [a, b)
  void entry_range(int64_t a, int64_t b, int64_t* e0, int64_t* e1) const {
    *e0 = 0;
    *e1 = entries;
    for (auto& p : bounds) {
      if (p.first <= a) *e0 = p.second;
      if (p.first >= b) {
        *e1 = p.second;
        break;
      }
    }
  }
  void release(cudaStream_t st) {
    dev_free(nodes, st);
    dev_free(samp, st);
    dev_free(set_start, st);
    dev_free(set_len, st);
    cap_entries = cap_sets = 0;
  }
};

// Sampling state: counters, CTA-tier hand-off list and scratch, seed bits.
struct Sampler {
  GraphView g;
  int model = 0;
  LaunchCfg cfg;
  Counters* d_ctr = nullptr;
  Counters* h_ctr = nullptr;  // pinned
  int64_t* big_list = nullptr;
  int64_t big_cap = 0;
  int64_t* mid_list = nullptr;
  int64_t mid_list_cap = 0;
  uint32_t* mid_hash = nullptr;
  int32_t* mid_queue = nullptr;
  uint32_t* mid_slots = nullptr;
  int64_t* fail_list = nullptr;  // samples whose pool reservation did not fit
  int64_t* redo_list = nullptr;  // the previous attempt's fail list, re-run
  int64_t fail_cap = 0, redo_cap = 0;
  uint32_t* slot_bitmap = nullptr;
  int32_t* slot_queue = nullptr;
  int32_t* small_queue = nullptr;
  uint32_t* small_bitmap = nullptr;
  int64_t* big2_list = nullptr;
  int64_t big2_cap = 0;
  uint8_t* hit = nullptr;
  int64_t hit_cap = 0;
  uint32_t* seed_bits = nullptr;
  uint64_t* bprefix = nullptr;
  uint64_t wsum = 0;
  int lt_cumulative = 0;
  int wc_implicit = 0;
  int warp_global = 0;  // weighted-cascade IC: the global-bitmap warp tier takes every sample
  int lane_tier = 0;    // weighted-cascade IC: the lane tier runs first
  int64_t* lane_list = nullptr;
  int64_t lane_cap = 0;
  uint32_t* wg_bitmap = nullptr;
  int32_t* wg_queue = nullptr;
  int mid_cap = 16384;  // IC: largest set the global warp tier keeps (0 = none)
  int heavy_groups = 0x7FFFFFFF;  // IC: warp tiers hand samples with longer in-lists to the CTA tier
  int64_t edge_visits = 0, node_visits = 0, samples = 0, hit_samples = 0;
  int64_t cta_edge_visits = 0, cta_node_visits = 0, cta_samples = 0;
  int64_t cta_store_nodes = 0, cta_store_sets = 0;  // the CTA tier's sets written to the pool
  int64_t draws = 0;  // Philox draws of IC edge groups / LT picks
  int64_t cta_draws = 0;

  void tally(int64_t count) {
    draws += (int64_t)h_ctr->draws;
    cta_draws += (int64_t)h_ctr->cta_draws;
    edge_visits += (int64_t)h_ctr->edge_visits;
    node_visits += (int64_t)h_ctr->node_visits;
    cta_edge_visits += (int64_t)h_ctr->cta_edge_visits;
    cta_node_visits += (int64_t)h_ctr->cta_node_visits;
    cta_samples += (int64_t)h_ctr->big_count;
    samples += count;
  }

  ssa_status init(const ssa_graph* G, int mdl, const uint32_t* benefit, Exec& X) {
    TRY(init_scratch(G, mdl, X));
    return begin_solve(G, benefit, X);
  }
  // Per-solve state on kept scratch: tuning, WRIS prefix sums, statistics.
  ssa_status begin_solve(const ssa_graph* G, const uint32_t* benefit, Exec& X) {
    {
      std::lock_guard<std::mutex> lock(G->tune_mu);
      if (G->tuned_mid_cap >= 0) {
        mid_cap = G->tuned_mid_cap;
        heavy_groups = G->tuned_heavy;
      }
      warp_global = (G->tuned_warp_global && cfg.wg_blocks > 0) ? 1 : 0;
      lane_tier = (G->tuned_lane_tier && cfg.lane_blocks > 0) ? 1 : 0;
    }
    X.num_sms = cfg.num_sms;
    edge_visits = node_visits = samples = hit_samples = 0;
    cta_edge_visits = cta_node_visits = cta_samples = cta_store_nodes = cta_store_sets = 0;
    draws = cta_draws = 0;
    dev_free(bprefix, X.st);
    wsum = 0;
    if (benefit) {
      std::vector<uint64_t> pre((size_t)g.n + 1, 0);
      for (int64_t v = 0; v < g.n; ++v) pre[(size_t)v + 1] = pre[(size_t)v] + benefit[v];
      wsum = pre[(size_t)g.n];
      if (wsum == 0) return fail(SSA_E_ARG, "benefit weights sum to zero");
      TRY(dev_alloc(&bprefix, (size_t)g.n + 1, X.st));
      CU(cudaMemcpyAsync(bprefix, pre.data(), sizeof(uint64_t) * pre.size(), cudaMemcpyHostToDevice, X.st));
      CU(cudaStreamSynchronize(X.st));
    }
    return SSA_OK;
  }
  // Scratch of the sampler tiers for one graph and model.  The kernels clear
  // every visited bit and hash slot they set, so the scratch stays ready for
  // the next batch and the next solve.
  ssa_status init_scratch(const ssa_graph* G, int mdl, Exec& X) {
    g = G->view();
    model = mdl;
    lt_cumulative = (mdl == 1 && G->weighting == SSA_W_EXPLICIT) ? 1 : 0;
    wc_implicit = G->weighting == SSA_W_WC ? 1 : 0;
    cfg = sampler_config(g, mdl, wc_implicit != 0);
    {
      std::lock_guard<std::mutex> lock(G->tune_mu);
      if (G->tuned_small_qcap > 0 && !cfg.cta_smem_bitmap)
        cfg.small_qcap = (int)std::min<int64_t>(g.n, G->tuned_small_qcap);
    }
    X.num_sms = cfg.num_sms;
    TRY(dev_alloc(&d_ctr, 1, X.st));
    CU(cudaMallocHost(reinterpret_cast<void**>(&h_ctr), sizeof(Counters)));
    const int64_t words = (g.n + 31) / 32;
    TRY(dev_alloc(&slot_queue, (size_t)g.n * (size_t)cfg.cta_blocks, X.st));
    // the weighted-cascade CTA tier reads -1 as "queue slot not written yet"
    // and restores -1 after each sample
    if (wc_implicit && mdl == 0)
      CU(cudaMemsetAsync(slot_queue, 0xFF, sizeof(int32_t) * (size_t)g.n * (size_t)cfg.cta_blocks, X.st));
    if (!cfg.cta_smem_bitmap) {
      TRY(dev_alloc(&slot_bitmap, (size_t)words * (size_t)cfg.cta_blocks, X.st));
      CU(cudaMemsetAsync(slot_bitmap, 0, sizeof(uint32_t) * (size_t)words * (size_t)cfg.cta_blocks, X.st));
      TRY(dev_alloc(&small_queue, (size_t)cfg.small_qcap * (size_t)cfg.small_blocks, X.st));
      if (wc_implicit && mdl == 0)
        CU(cudaMemsetAsync(small_queue, 0xFF, sizeof(int32_t) * (size_t)cfg.small_qcap * (size_t)cfg.small_blocks,
                           X.st));
      TRY(dev_alloc(&small_bitmap, (size_t)words * (size_t)cfg.small_blocks, X.st));
      CU(cudaMemsetAsync(small_bitmap, 0, sizeof(uint32_t) * (size_t)words * (size_t)cfg.small_blocks, X.st));
    }
    TRY(dev_alloc(&seed_bits, (size_t)words, X.st));
    if (model == 0) {
      const size_t warps = mid_tier_words(cfg);
      TRY(dev_alloc(&mid_hash, warps * mid_hash_per_warp(), X.st));
      CU(cudaMemsetAsync(mid_hash, 0, sizeof(uint32_t) * warps * mid_hash_per_warp(), X.st));
      TRY(dev_alloc(&mid_queue, warps * mid_queue_per_warp(), X.st));
      TRY(dev_alloc(&mid_slots, warps * mid_queue_per_warp(), X.st));
    }
    if (cfg.wg_blocks > 0) {
      // the global-bitmap warp tier: an n-bit bitmap and a queue per warp
      const size_t wgw = wg_tier_warps(cfg);
      TRY(dev_alloc(&wg_bitmap, (size_t)words * wgw, X.st));
      CU(cudaMemsetAsync(wg_bitmap, 0, sizeof(uint32_t) * (size_t)words * wgw, X.st));
      TRY(dev_alloc(&wg_queue, wg_queue_per_warp() * wgw, X.st));
    }
    return SSA_OK;
  }
  void release(cudaStream_t st) {
    dev_free(d_ctr, st);
    if (h_ctr) cudaFreeHost(h_ctr);
    h_ctr = nullptr;
    dev_free(big_list, st);
    dev_free(lane_list, st);
    dev_free(mid_list, st);
    dev_free(mid_hash, st);
    dev_free(mid_queue, st);
    dev_free(mid_slots, st);
    dev_free(wg_bitmap, st);
    dev_free(wg_queue, st);
    dev_free(fail_list, st);
    dev_free(redo_list, st);
    dev_free(slot_bitmap, st);
    dev_free(slot_queue, st);
    dev_free(small_queue, st);
    dev_free(small_bitmap, st);
    dev_free(big2_list, st);
    dev_free(hit, st);
    dev_free(seed_bits, st);
    dev_free(bprefix, st);
  }

  SampleJob job(uint64_t seed, uint32_t stream, int64_t j0, int64_t count) const {
    SampleJob J;
    J.g = g;
    J.model = model;
    J.lt_cumulative = lt_cumulative;
    J.wc_implicit = wc_implicit;
    J.warp_global = warp_global;
    J.lane_tier = (model == 0 && wc_implicit && lane_tier) ? 1 : 0;
    J.lane_list = lane_list;
    J.wg_bitmap = wg_bitmap;
    J.wg_queue = wg_queue;
    J.seed = seed;
    J.stream = stream;
    J.j0 = j0;
    J.count = count;
    J.bprefix = bprefix;
    J.big_list = big_list;
    J.mid_cap = model == 0 ? mid_cap : 0;
    J.warp_heavy_groups = heavy_groups;
    J.mid_list = mid_list;
    J.mid_hash = mid_hash;
    J.mid_queue = mid_queue;
    J.mid_slots = mid_slots;
    J.slot_bitmap = slot_bitmap;
    J.slot_queue = slot_queue;
    J.small_qcap = cfg.small_qcap;
    J.small_queue = small_queue;
    J.small_bitmap = small_bitmap;
    J.big2_list = big2_list;
    J.bitmap_words = (g.n + 31) / 32;
    J.ctr = d_ctr;
    J.fail_list = fail_list;
    // Philox4x32-10 key schedule: round r uses key + r * (0x9E3779B9, 0xBB67AE85)
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
      J.rk[2 * r] = k0;
      J.rk[2 * r + 1] = k1;
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    return J;
  }

  ssa_status run(SampleJob& J, Exec& X, unsigned long long cursor0) {
    std::memset(h_ctr, 0, sizeof(Counters));
    h_ctr->cursor = cursor0;
    h_ctr->ok_end = ~0ull;  // least start of a reservation that did not fit
    CU(cudaMemcpyAsync(d_ctr, h_ctr, sizeof(Counters), cudaMemcpyHostToDevice, X.st));
    int h = X.begin(SSA_K_SAMPLE_WARP);
    CU(launch_sample_warp(J, cfg, X.st));
    X.end(h);
    h = X.begin(SSA_K_SAMPLE_CTA);
    CU(launch_sample_cta(J, cfg, X.st));
    X.end(h);
    X.launches += model == 0 ? 3 : 2;
    CU(cudaMemcpyAsync(h_ctr, d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, X.st));
    CU(cudaStreamSynchronize(X.st));
    if (h_ctr->error) return fail(SSA_E_INTERNAL, "sampler reported an internal error (wait %u gave up)", h_ctr->error);
    return SSA_OK;
  }

  // Append samples [pool.count, pool.count + count) of (seed, stream) to the pool.
  // The pool is sized from the mean set size seen so far (a pilot batch of up
  // to 8192 samples measures it when the pool is empty); samples whose
  // reservation still does not fit are listed by the kernels and re-run after
  // the pool grows, so no finished set is sampled twice.  The ones that miss
  // are the last to finish, the largest sets, so an estimate that runs short
  // re-runs the most expensive samples: set sizes are heavy-tailed (under
  // weighted cascade the mean of 512 samples is often a quarter off), hence
  // the large pilot and a wider margin while the mean rests on few samples.
  ssa_status append(DevPool& P, uint64_t seed, uint32_t stream, int64_t count, Exec& X, bool pilot_first = true) {
    if (count <= 0) return SSA_OK;
    if (pilot_first && P.count == 0 && count > 1024) {
      // one pilot batch: each batch ends with its slowest sample, so a chain of them costs a tail each
      const int64_t pilot = std::min<int64_t>(8192, count / 4);
      TRY(append(P, seed, stream, pilot, X, false));
      count -= pilot;
    }
    const int64_t j0 = P.count;
    if (j0 + count > (int64_t)0x7FFFFFFF) return fail(SSA_E_POOL_FULL, "more than 2^31 RR sets");
    TRY(dev_grow(&big_list, &big_cap, count, 0, X.st));
    TRY(dev_grow(&lane_list, &lane_cap, count, 0, X.st));
    TRY(dev_grow(&big2_list, &big2_cap, count, 0, X.st));
    TRY(dev_grow(&mid_list, &mid_list_cap, count, 0, X.st));
    TRY(dev_grow(&fail_list, &fail_cap, count, 0, X.st));
    TRY(dev_grow(&redo_list, &redo_cap, count, 0, X.st));
    if (j0 + count > P.cap_sets) {
      int64_t want = std::max<int64_t>(j0 + count, P.cap_sets * 2);
      int64_t c1 = P.cap_sets, c2 = P.cap_sets;
      TRY(dev_grow(&P.set_start, &c1, want, j0, X.st));
      TRY(dev_grow(&P.set_len, &c2, want, j0, X.st));
      P.cap_sets = want;
    }
    const double mean = P.count > 0 ? (double)P.entries / (double)P.count : 16.0;
    const double margin = P.count >= 65536 ? 1.15 : 1.5;
    int64_t want = P.entries + (int64_t)(mean * (double)count * margin) + 65536;
    TRY(grow_entries(P, want, X));
    int64_t todo = count;
    const int64_t* list = nullptr;
    unsigned long long cursor0 = (unsigned long long)P.entries;
    unsigned long long ev = 0, nv = 0, cev = 0, cnv = 0, csets = 0;
    for (int attempt = 0; todo > 0; ++attempt) {
      if (attempt >= 64) return fail(SSA_E_INTERNAL, "pool growth did not converge");
      SampleJob J = job(seed, stream, j0, todo);
      J.work_list = list;
      J.mode = MODE_STORE;
      J.pool_nodes = P.nodes;
      J.pool_samp = P.samp;
      J.pool_cap = P.cap_entries;
      J.set_start = P.set_start;
      J.set_len = P.set_len;
      TRY(run(J, X, cursor0));
      ev += h_ctr->edge_visits;
      nv += h_ctr->node_visits;
      draws += (int64_t)h_ctr->draws;
      cta_draws += (int64_t)h_ctr->cta_draws;
      cev += h_ctr->cta_edge_visits;
      cnv += h_ctr->cta_node_visits;
      csets += h_ctr->big_count;
      if (!h_ctr->pool_overflow) {
        cursor0 = h_ctr->cursor;
        break;
      }
      // [ok_end, cursor) were reserved by samples that did not fit: re-run them
      const int64_t ok_end = (int64_t)std::max<unsigned long long>(h_ctr->ok_end, cursor0);
      const int64_t need = (int64_t)h_ctr->cursor - ok_end;
      const int64_t failed = (int64_t)h_ctr->fail_count;
      P.entries = ok_end;
      TRY(grow_entries(P, ok_end + need + need / 4 + 65536, X));
      std::swap(fail_list, redo_list);
      std::swap(fail_cap, redo_cap);
      list = redo_list;
      todo = failed;
      cursor0 = (unsigned long long)ok_end;
    }
    edge_visits += (int64_t)ev;
    node_visits += (int64_t)nv;
    cta_edge_visits += (int64_t)cev;
    cta_node_visits += (int64_t)cnv;
    cta_store_nodes += (int64_t)cnv;
    cta_samples += (int64_t)csets;
    cta_store_sets += (int64_t)csets;
    samples += count;
    P.entries = (int64_t)cursor0;
    P.count = j0 + count;
    P.bounds.emplace_back(P.count, P.entries);
    return SSA_OK;
  }

  ssa_status grow_entries(DevPool& P, int64_t want, Exec& X) {
    if (want <= P.cap_entries) return SSA_OK;
    want = std::max<int64_t>(want, P.cap_entries + P.cap_entries / 2);
    if (P.byte_cap > 0 && P.bytes_for(want, P.cap_sets) > P.byte_cap) {
      const int64_t most = (P.byte_cap - P.cap_sets * 14) / 12;
      if (most <= P.cap_entries)
        return fail(SSA_E_POOL_FULL, "RR pool needs more than its %lld-byte cap", (long long)P.byte_cap);
      want = most;
    }
    int64_t a = P.cap_entries, b = P.cap_entries;
    TRY(dev_grow(&P.nodes, &a, want, P.entries, X.st));
    TRY(dev_grow(&P.samp, &b, want, P.entries, X.st));
    P.cap_entries = want;
    return SSA_OK;
  }

  // Hit-test batch (Estimate-Inf): hit[i] = R_{j0+i} meets the seed bits.
  ssa_status hits(uint64_t seed, uint32_t stream, int64_t j0, int64_t count, Exec& X) {
    TRY(hits_prepare(count, X));
    TRY(hits_issue(seed, stream, j0, count, X));
    CU(cudaStreamSynchronize(X.st));
    return hits_finish(count);
  }
  // The same batch in three parts, so that the middle one, which only queues
  // device work (no allocation, no host wait), can be captured into a CUDA
  // graph: buffers, then the kernels with the counters reset on the device
  // and read back into pinned memory, then the checks and statistics.
  ssa_status hits_prepare(int64_t count, Exec& X) {
    TRY(dev_grow(&big_list, &big_cap, count, 0, X.st));
    TRY(dev_grow(&lane_list, &lane_cap, count, 0, X.st));
    TRY(dev_grow(&big2_list, &big2_cap, count, 0, X.st));
    TRY(dev_grow(&mid_list, &mid_list_cap, count, 0, X.st));
    TRY(dev_grow(&hit, &hit_cap, count, 0, X.st));
    return SSA_OK;
  }
  ssa_status hits_issue(uint64_t seed, uint32_t stream, int64_t j0, int64_t count, Exec& X) {
    SampleJob J = job(seed, stream, j0, count);
    J.mode = MODE_HIT;
    J.seed_bits = seed_bits;
    J.hit = hit;
    CU(cudaMemsetAsync(d_ctr, 0, sizeof(Counters), X.st));
    int h = X.begin(SSA_K_SAMPLE_WARP);
    CU(launch_sample_warp(J, cfg, X.st));
    X.end(h);
    h = X.begin(SSA_K_SAMPLE_CTA);
    CU(launch_sample_cta(J, cfg, X.st));
    X.end(h);
    X.launches += model == 0 ? 3 : 2;
    CU(cudaMemcpyAsync(h_ctr, d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, X.st));
    return SSA_OK;
  }
  ssa_status hits_finish(int64_t count) {
    if (h_ctr->error) return fail(SSA_E_INTERNAL, "sampler reported an internal error (wait %u gave up)", h_ctr->error);
    tally(count);
    hit_samples += count;
    return SSA_OK;
  }
};

// One cooperative greedy grid on the device at a time: a solver holds this
// from the launch of its greedy kernel until its stream has finished it, so
// solvers on other host threads (serving slots) never run two grids whose
// blocks must all be resident at once.
std::mutex& coop_mutex() {
  static std::mutex mu;
  return mu;
}

// Node -> set index and greedy buffers.  The pool only ever appends whole
// batches, so the index is kept per batch: each batch is counted, scanned and
// scattered once, its counts are added to a running total, and Max-Coverage
// walks v*'s list in every batch.  A cut N inside a batch gets a temporary
// filtered index for the partial batch.
struct Cover {
  struct Batch {
    int64_t j0, j1;          // sample ids [j0, j1)
    int64_t* off = nullptr;  // n+1
    int32_t* samp = nullptr; // entries of the batch
    int64_t e0 = 0, e1 = 0;  // its pool entries
    bool ready = false;      // kernels queued
  };
  int64_t n = 0;
  int64_t n_pad = 0;
  std::vector<Batch> batches;
  Batch partial_batch;       // temporary, for a cut inside a batch
  int32_t* cnt_total = nullptr;  // counts of the cached batches
  int32_t* cnt_tmp = nullptr;    // one batch's counts
  int32_t* cnt = nullptr;        // working gains of the current Max-Coverage
  unsigned long long* cur = nullptr;
  void* scan_tmp = nullptr;
  uint8_t* covered = nullptr;
  int64_t covered_cap = 0;
  uint8_t* in_seed = nullptr;
  unsigned long long* argmax = nullptr;  // greedy argmax slots (3, one 128-byte line apart)
  unsigned int* sync = nullptr;
  unsigned long long* chunk_q = nullptr;
  int64_t chunk_cap = 0;
  unsigned int* hist = nullptr;   // greedy gain histograms (2 x 4096) and cache counts (2), one buffer
  int32_t* cache = nullptr;       // greedy candidate caches (2 x 8192)
  int32_t* d_seeds = nullptr;
  int32_t* d_gains = nullptr;
  int k_cap = 0;
  unsigned long long* d_count = nullptr;
  long long* d_first = nullptr;
  void* fr_tmp = nullptr;
  int64_t fr_cap = 0;
  uint8_t* hitc = nullptr;  // per-sample flags for Cov over a range
  int64_t hitc_cap = 0;
  // pinned host copies of the greedy's results and of the stare count, so the
  // copies back can sit inside a captured CUDA graph
  int32_t* h_seeds = nullptr;
  int32_t* h_gains = nullptr;
  int h_cap = 0;
  unsigned int* h_sync = nullptr;        // 128 words
  unsigned long long* h_count = nullptr;
  int64_t total_e = 0;                   // entries of the sets the next greedy covers (greedy_prepare)
  bool shared_gpu = false;               // the solve shares the GPU with others (greedy launch shape)

  ssa_status init(int64_t nn, Exec& X) {
    n = nn;
    n_pad = (n + 3) & ~int64_t(3);
    TRY(dev_alloc(&cnt_total, (size_t)n_pad, X.st));
    TRY(dev_alloc(&cnt_tmp, (size_t)n_pad, X.st));
    TRY(dev_alloc(&cnt, (size_t)n_pad, X.st));
    CU(cudaMemsetAsync(cnt_total, 0, sizeof(int32_t) * (size_t)n_pad, X.st));
    TRY(dev_alloc(&cur, (size_t)n + 1, X.st));
    TRY(dev_alloc(&in_seed, (size_t)n_pad, X.st));
    CU(cudaMallocAsync(&scan_tmp, scan_tmp_bytes(n), X.st));
    TRY(dev_alloc(&argmax, 64 + 2 * 1024, X.st));
    TRY(dev_alloc(&sync, 128, X.st));
    TRY(dev_alloc(&hist, 2 * 4096 + 2, X.st));
    TRY(dev_alloc(&cache, 2 * 8192, X.st));
    TRY(dev_alloc(&d_count, 1, X.st));
    TRY(dev_alloc(&d_first, 2, X.st));
    CU(cudaMallocHost(reinterpret_cast<void**>(&h_sync), sizeof(unsigned int) * 128));
    CU(cudaMallocHost(reinterpret_cast<void**>(&h_count), sizeof(unsigned long long)));
    return SSA_OK;
  }
  // a new solve on kept workspaces: drop the previous solve's index
  ssa_status reset(Exec& X) {
    drop_index(X.st);
    CU(cudaMemsetAsync(cnt_total, 0, sizeof(int32_t) * (size_t)n_pad, X.st));
    return SSA_OK;
  }
  void drop_index(cudaStream_t st) {
    for (auto& b : batches) free_batch(b, st);
    batches.clear();
    free_batch(partial_batch, st);
  }
  void free_batch(Batch& b, cudaStream_t st) {
    dev_free(b.off, st);
    dev_free(b.samp, st);
  }
  void release(cudaStream_t st) {
    for (auto& b : batches) free_batch(b, st);
    batches.clear();
    free_batch(partial_batch, st);
    dev_free(cnt_total, st);
    dev_free(cnt_tmp, st);
    dev_free(cnt, st);
    dev_free(cur, st);
    if (scan_tmp) cudaFreeAsync(scan_tmp, st);
    scan_tmp = nullptr;
    dev_free(covered, st);
    dev_free(in_seed, st);
    dev_free(argmax, st);
    dev_free(sync, st);
    dev_free(chunk_q, st);
    dev_free(hist, st);
    dev_free(cache, st);
    dev_free(d_seeds, st);
    dev_free(d_gains, st);
    dev_free(d_count, st);
    dev_free(d_first, st);
    if (fr_tmp) cudaFreeAsync(fr_tmp, st);
    fr_tmp = nullptr;
    dev_free(hitc, st);
    cudaStreamSynchronize(st);  // the pinned buffers may still be a copy's destination
    if (h_seeds) cudaFreeHost(h_seeds);
    if (h_gains) cudaFreeHost(h_gains);
    if (h_sync) cudaFreeHost(h_sync);
    if (h_count) cudaFreeHost(h_count);
    h_seeds = h_gains = nullptr;
    h_sync = nullptr;
    h_count = nullptr;
    h_cap = 0;
  }

  ssa_status index_alloc(Batch& B, Exec& X) {
    TRY(dev_alloc(&B.off, (size_t)n + 1, X.st));
    TRY(dev_alloc(&B.samp, (size_t)std::max<int64_t>(B.e1 - B.e0, 1), X.st));
    return SSA_OK;
  }
  // index of the samples [B.j0, B.j1) whose entries lie in [B.e0, B.e1); counts land in cnt_tmp
  ssa_status index_kernels(const DevPool& P, const Batch& B, bool filter, Exec& X) {
    CU(cudaMemsetAsync(cnt_tmp, 0, sizeof(int32_t) * (size_t)n_pad, X.st));
    CU(launch_count_nodes(P.nodes, filter ? P.samp : nullptr, B.e0, B.e1, B.j0, B.j1, cnt_tmp, X.st, X.num_sms));
    int l = 0;
    CU(launch_exclusive_scan(cnt_tmp, n, B.off, scan_tmp, X.st, &l));
    // positions inside the batch's own sample array: offsets start at 0
    CU(cudaMemcpyAsync(cur, B.off, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyDeviceToDevice, X.st));
    CU(launch_scatter_index(P.nodes, P.samp, B.e0, B.e1, B.j0, B.j1, cur, B.samp, X.st, X.num_sms));
    X.launches += 2 + l;
    return SSA_OK;
  }

  // Buffers for the index of every whole pool batch below N not indexed yet.
  // *whole: N lies on a batch boundary, so index_issue needs no temporary
  // partial batch (and allocates nothing).
  ssa_status index_prepare(const DevPool& P, int64_t N, bool* whole, Exec& X) {
    free_batch(partial_batch, X.st);
    if (!batches.empty() && batches.back().j1 > N) {
      // a smaller cut than before (direct callers): start the cache over
      for (auto& b : batches) free_batch(b, X.st);
      batches.clear();
      CU(cudaMemsetAsync(cnt_total, 0, sizeof(int32_t) * (size_t)n_pad, X.st));
    }
    for (size_t i = 1; i < P.bounds.size(); ++i) {
      const int64_t j0 = P.bounds[i - 1].first, j1 = P.bounds[i].first;
      if (j1 > N) break;
      if (!batches.empty() && batches.back().j1 >= j1) continue;
      if (batches.size() >= (size_t)GREEDY_MAX_LISTS - 1)
        return fail(SSA_E_INTERNAL, "more than %d index batches", GREEDY_MAX_LISTS - 1);
      Batch B;
      B.j0 = j0;
      B.j1 = j1;
      B.e0 = P.bounds[i - 1].second;
      B.e1 = P.bounds[i].second;
      TRY(index_alloc(B, X));
      batches.push_back(B);
    }
    *whole = (batches.empty() ? 0 : batches.back().j1) >= N;
    return SSA_OK;
  }

  // Queue the index kernels of the batches index_prepare added (each batch is
  // counted, scanned and scattered once) and, for a cut inside a batch, of a
  // temporary partial one.  Leaves the counts of [0, N) in `cnt`.
  ssa_status index_issue(const DevPool& P, int64_t N, Exec& X) {
    int h = X.begin(SSA_K_INDEX);
    for (auto& B : batches) {
      if (B.ready) continue;
      TRY(index_kernels(P, B, false, X));
      CU(launch_add_counts(cnt_total, cnt_tmp, n, X.st, X.num_sms));
      X.launches += 1;
      B.ready = true;
    }
    CU(cudaMemcpyAsync(cnt, cnt_total, sizeof(int32_t) * (size_t)n_pad, cudaMemcpyDeviceToDevice, X.st));
    const int64_t covered_to = batches.empty() ? 0 : batches.back().j1;
    if (covered_to < N) {
      partial_batch.j0 = covered_to;
      partial_batch.j1 = N;
      P.entry_range(covered_to, N, &partial_batch.e0, &partial_batch.e1);
      TRY(index_alloc(partial_batch, X));
      TRY(index_kernels(P, partial_batch, true, X));
      CU(launch_add_counts(cnt, cnt_tmp, n, X.st, X.num_sms));
      X.launches += 1;
    }
    X.end(h);
    return SSA_OK;
  }

  // Make the index cover the sets [0, N).
  ssa_status build_index(const DevPool& P, int64_t N, Exec& X) {
    bool whole = false;
    TRY(index_prepare(P, N, &whole, X));
    return index_issue(P, N, X);
  }

  // Max-Coverage (Algorithm 2) over sets [0, N) in three parts, so that the
  // middle one (device work only) can sit inside a captured CUDA graph:
  // buffers, then the kernel and the copies of its results into pinned
  // memory, then the checks once the stream has finished.
  ssa_status greedy_prepare(const DevPool& P, int64_t N, int k, Exec& X) {
    // packed argmax keys (gain + 1) << 31 | (2^31 - 1 - v) stay below 2^62
    if (N >= INT32_MAX) return fail(SSA_E_ARG, "greedy over %lld sets: at most 2^31 - 2", (long long)N);
    if (k > k_cap) {
      dev_free(d_seeds, X.st);
      dev_free(d_gains, X.st);
      TRY(dev_alloc(&d_seeds, (size_t)k, X.st));
      TRY(dev_alloc(&d_gains, (size_t)k, X.st));
      k_cap = k;
    }
    if (k > h_cap) {
      CU(cudaStreamSynchronize(X.st));  // the old buffers may still be a copy's destination
      if (h_seeds) cudaFreeHost(h_seeds);
      if (h_gains) cudaFreeHost(h_gains);
      h_seeds = h_gains = nullptr;
      h_cap = 0;
      CU(cudaMallocHost(reinterpret_cast<void**>(&h_seeds), sizeof(int32_t) * (size_t)k));
      CU(cudaMallocHost(reinterpret_cast<void**>(&h_gains), sizeof(int32_t) * (size_t)k));
      h_cap = k;
    }
    TRY(dev_grow(&covered, &covered_cap, std::max<int64_t>(N, 1), 0, X.st));
    // entries of sets [0, N), an upper bound when N cuts a batch; queued
    // decrement chunks of one pick: a set longer than 2048 entries queues
    // ceil(len / 2048) < len / 1024 chunks
    int64_t e0 = 0, e1 = 0;
    P.entry_range(0, N, &e0, &e1);
    total_e = e1 - e0;
    TRY(dev_grow(&chunk_q, &chunk_cap, e1 / 1024 + 1, 0, X.st));
    return SSA_OK;
  }
  ssa_status greedy_issue(const DevPool& P, int64_t N, int k, Exec& X) {
    int h = X.begin(SSA_K_GREEDY);
    CU(cudaMemsetAsync(covered, 0, (size_t)std::max<int64_t>(N, 1), X.st));
    CU(cudaMemsetAsync(sync, 0, sizeof(unsigned int) * 128, X.st));
    CU(cudaMemsetAsync(hist, 0, sizeof(unsigned int) * (2 * 4096 + 2), X.st));
    CU(cudaMemsetAsync(argmax, 0, sizeof(unsigned long long) * (64 + 2 * 1024), X.st));
    // padding nodes can never be picked
    if (n_pad > n) CU(cudaMemsetAsync(cnt + n, 0xC0, sizeof(int32_t) * (size_t)(n_pad - n), X.st));
    GreedyJob J{};
    J.cnt = cnt;
    J.n_pad = n_pad;
    J.nlists = 0;
    for (auto& b : batches) J.lists[J.nlists++] = InvList{b.off, b.samp};
    if (partial_batch.off) J.lists[J.nlists++] = InvList{partial_batch.off, partial_batch.samp};
    J.pool_nodes = P.nodes;
    J.set_start = P.set_start;
    J.set_len = P.set_len;
    J.covered = covered;
    J.seeds = d_seeds;
    J.gains = d_gains;
    J.k = k;
    J.argmax = argmax;
    J.n_sets = N;
    J.total_entries = (unsigned long long)total_e;
    J.sync = sync;
    J.chunk_q = chunk_q;
    J.chunk_cap = chunk_cap;
    J.hist = hist;
    J.cache = cache;
    J.cache_n = hist + 2 * 4096;
    J.wait_polls = greedy_wait_polls();
    int blocks = 0;
    CU(launch_greedy(J, X.st, X.num_sms, &blocks, shared_gpu));
    X.end(h);
    X.launches += 1;
    CU(cudaMemcpyAsync(h_seeds, d_seeds, sizeof(int32_t) * (size_t)k, cudaMemcpyDeviceToHost, X.st));
    CU(cudaMemcpyAsync(h_gains, d_gains, sizeof(int32_t) * (size_t)k, cudaMemcpyDeviceToHost, X.st));
    CU(cudaMemcpyAsync(h_sync, sync, sizeof(unsigned int) * 128, cudaMemcpyDeviceToHost, X.st));
    return SSA_OK;
  }
  ssa_status greedy_finish(int k, int32_t* seeds, int64_t* gains, int64_t* cov) {
    if (h_sync[64] == 2u) return fail(SSA_E_INTERNAL, "greedy decrement queue overflow");
    if (h_sync[64]) return fail(SSA_E_TIMEOUT, "greedy grid barrier timed out");
    int64_t c = 0;
    for (int i = 0; i < k; ++i) {
      seeds[i] = h_seeds[i];
      gains[i] = h_gains[i];
      c += h_gains[i];
    }
    *cov = c;
    return SSA_OK;
  }
  // Max-Coverage (Algorithm 2) over sets [0, N): seeds/gains to host.
  ssa_status greedy(const DevPool& P, int64_t N, int k, int32_t* seeds, int64_t* gains, int64_t* cov, Exec& X) {
    TRY(greedy_prepare(P, N, k, X));
    TRY(build_index(P, N, X));
    {
      std::lock_guard<std::mutex> coop_lock(coop_mutex());
      TRY(greedy_issue(P, N, k, X));
      CU(cudaStreamSynchronize(X.st));
    }
    return greedy_finish(k, seeds, gains, cov);
  }

  // Cov (Eq. 1) of the seeds currently flagged in in_seed over sets [a, b).
  ssa_status coverage_range(const DevPool& P, int64_t a, int64_t b, int64_t* cov, Exec& X) {
    const int64_t cnt_sets = b - a;
    if (cnt_sets <= 0) {
      *cov = 0;
      return SSA_OK;
    }
    int64_t e0, e1;
    P.entry_range(a, b, &e0, &e1);
    TRY(dev_grow(&hitc, &hitc_cap, cnt_sets, 0, X.st));
    int h = X.begin(SSA_K_STARE);
    CU(cudaMemsetAsync(hitc, 0, (size_t)cnt_sets, X.st));
    CU(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), X.st));
    CU(launch_mark_hits(P.nodes, P.samp, e0, e1, in_seed, a, b, hitc, X.st, X.num_sms));
    CU(launch_count_flags(hitc, cnt_sets, d_count, X.st, X.num_sms));
    X.end(h);
    X.launches += 2;
    unsigned long long c = 0;
    CU(cudaMemcpyAsync(&c, d_count, sizeof(c), cudaMemcpyDeviceToHost, X.st));
    CU(cudaStreamSynchronize(X.st));
    *cov = (int64_t)c;
    return SSA_OK;
  }
};

// Cov of the seeds over the fresh sets [j0, j0+count) of `stream`, sampled in
// hit-test mode (each sample stops at its first seed).
// (split like the greedy: the issue part only queues device work)
ssa_status stare_issue(Sampler& S, Cover& C, uint64_t seed, uint32_t stream, int64_t j0, int64_t count,
                       const int32_t* d_seeds, int k, Exec& X) {
  const int64_t words = (S.g.n + 31) / 32;
  CU(cudaMemsetAsync(S.seed_bits, 0, sizeof(uint32_t) * (size_t)words, X.st));
  CU(launch_set_bits(d_seeds, k, S.seed_bits, nullptr, X.st));
  X.launches += 1;
  TRY(S.hits_issue(seed, stream, j0, count, X));
  int h = X.begin(SSA_K_STARE);
  CU(cudaMemsetAsync(C.d_count, 0, sizeof(unsigned long long), X.st));
  CU(launch_count_flags(S.hit, count, C.d_count, X.st, X.num_sms));
  X.end(h);
  X.launches += 1;
  CU(cudaMemcpyAsync(C.h_count, C.d_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, X.st));
  return SSA_OK;
}
ssa_status stare_finish(Sampler& S, Cover& C, int64_t count, int64_t* cov) {
  TRY(S.hits_finish(count));
  *cov = (int64_t)*C.h_count;
  return SSA_OK;
}
ssa_status stare_hits(Sampler& S, Cover& C, uint64_t seed, uint32_t stream, int64_t j0, int64_t count,
                      const int32_t* d_seeds, int k, int64_t* cov, Exec& X) {
  TRY(S.hits_prepare(count, X));
  TRY(stare_issue(S, C, seed, stream, j0, count, d_seeds, k, X));
  CU(cudaStreamSynchronize(X.st));
  return stare_finish(S, C, count, cov);
}

// Estimate-Inf (Algorithm 3) on the device: hit-test batches of fresh sets
// of `stream`, then the first T whose prefix of successes reaches `need`.
ssa_status estimate_inf_dev(Sampler& S, Cover& C, uint64_t seed, uint32_t stream, const int32_t* d_seeds, int k,
                            int64_t need, int64_t t_max, int64_t first_batch, int64_t* T_out, int64_t* hits_out,
                            Exec& X) {
  const int64_t words = (S.g.n + 31) / 32;
  CU(cudaMemsetAsync(S.seed_bits, 0, sizeof(uint32_t) * (size_t)words, X.st));
  CU(launch_set_bits(d_seeds, k, S.seed_bits, nullptr, X.st));
  X.launches += 1;
  int64_t j = 0, before = 0, B = std::max<int64_t>(first_batch, 4096);
  *T_out = 0;
  while (j < t_max) {
    const int64_t cnt = std::min<int64_t>(B, t_max - j);
    TRY(S.hits(seed, stream, j, cnt, X));
    if ((int64_t)first_reach_tmp_bytes(cnt) > C.fr_cap) {
      if (C.fr_tmp) cudaFreeAsync(C.fr_tmp, X.st);
      C.fr_cap = (int64_t)first_reach_tmp_bytes(cnt);
      CU(cudaMallocAsync(&C.fr_tmp, (size_t)C.fr_cap, X.st));
    }
    int h = X.begin(SSA_K_STARE);
    int l = 0;
    CU(launch_first_reach(S.hit, cnt, (long long)(need - before), C.d_first, C.fr_tmp, X.st, &l));
    X.end(h);
    X.launches += l;
    long long out[2];
    CU(cudaMemcpyAsync(out, C.d_first, sizeof(out), cudaMemcpyDeviceToHost, X.st));
    CU(cudaStreamSynchronize(X.st));
    if (out[0] > 0) {
      *T_out = j + out[0];
      *hits_out = need;
      return SSA_OK;
    }
    before += out[1];
    j += cnt;
    B *= 2;
  }
  *hits_out = before;
  return SSA_OK;
}

// IC sampler autotuner: time a pilot batch of RR sets under each candidate
// hand-over size between the shared-memory warp tier, the global-memory warp
// tier and the CTA tier, and keep the fastest for this graph.  The candidates
// give identical sets (keyed randomness); only the time differs.
ssa_status autotune_ic(const ssa_graph* G, int64_t pilot, Exec& X, int* chosen, double* ms_out) {
  // (mid_cap, heavy in-list hand-over in 4-edge groups; 0x7FFFFFFF = never; global-bitmap
  // warp tier for every sample).  Weighted cascade walks in-lists by gaps, so no list is
  // heavy: its candidates are the hash tiers and, where the graph has it, the bitmap tier.
  const int cands_thr[4][3] = {{0, 0x7FFFFFFF, 0}, {mid_tier_max_cap(), 0x7FFFFFFF, 0}, {0, 4096, 0},
                               {mid_tier_max_cap(), 4096, 0}};
  // Where the global-bitmap tier exists it takes every sample: it beat the hash and CTA tiers
  // on 2M-set batches of the 2^23- and 2^25-node R-MAT graphs by 1.4-1.6x, while a pilot small
  // enough to time cheaply is ranked by its few largest sets, not by throughput.
  const int cands_wc[3][3] = {{0, 0x7FFFFFFF, 0}, {mid_tier_max_cap(), 0x7FFFFFFF, 0}, {0, 0x7FFFFFFF, 1}};
  const bool wc = G->weighting == SSA_W_WC;
  const int(*cands)[3] = wc ? cands_wc : cands_thr;
  if (wc && sampler_config(G->view(), 0, true).wg_blocks > 0) {
    std::lock_guard<std::mutex> lock(G->tune_mu);
    G->tuned_mid_cap = cands_wc[2][0];
    G->tuned_heavy = cands_wc[2][1];
    G->tuned_warp_global = cands_wc[2][2];
    if (chosen) *chosen = cands_wc[2][0];
    if (ms_out) *ms_out = 0.0;
    return SSA_OK;
  }
  double best_ms = 1e300;
  int best = cands[1][0], best_heavy = cands[1][1], best_global = 0;
  // One sampler and one pool serve every candidate: the tier settings are
  // plain fields, and the pool keeps the capacity that an untimed first pass
  // grew, so each timed pass samples the same pilot sets without re-runs.
  Sampler S;
  DevPool P;
  cudaEvent_t a = nullptr, b = nullptr;
  ssa_status st = S.init(G, 0, nullptr, X);
  if (st == SSA_OK && (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess))
    st = fail(SSA_E_CUDA, "autotune: cudaEventCreate failed");
  const int ncand = wc ? 2 : 4;
  for (int c = -1; c < ncand && st == SSA_OK; ++c) {
    const auto& cand = cands[c < 0 ? 0 : c];
    S.mid_cap = cand[0];
    S.heavy_groups = cand[1];
    S.warp_global = cand[2];
    P.count = 0;
    P.entries = 0;
    P.bounds.assign(1, {0, 0});
    if (c >= 0) cudaEventRecord(a, X.st);
    st = S.append(P, 0x5EEDull, 0, pilot, X);
    if (st != SSA_OK || c < 0) continue;
    cudaEventRecord(b, X.st);
    float ms = 0.f;
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
      st = fail(SSA_E_CUDA, "autotune: event timing failed");
      break;
    }
    if (ms < best_ms) {
      best_ms = ms;
      best = cand[0];
      best_heavy = cand[1];
      best_global = cand[2];
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  P.release(X.st);
  S.release(X.st);
  cudaStreamSynchronize(X.st);
  if (st != SSA_OK) return st;
  {
    std::lock_guard<std::mutex> lock(G->tune_mu);
    G->tuned_mid_cap = best;
    G->tuned_heavy = best_heavy;
    G->tuned_warp_global = best_global;
  }
  if (chosen) *chosen = best;
  if (ms_out) *ms_out = best_ms;
  return SSA_OK;
}

// ---------------------------------------------------------------------------
// FP64 parameters (Table 1; Algorithm 1 lines 1-3; Algorithm 4 lines 1-3;
// Eq. "set_ep").  Upsilon is taken from ln(1/delta) so that the tiny
// delta/(6 C(n,k)) inside N_max is never formed.
// ---------------------------------------------------------------------------
const double kOneMinusInvE = 1.0 - 1.0 / 2.718281828459045;

double upsilon_ln(double eps, double ln_inv_delta) {
  return (2.0 + 2.0 * eps / 3.0) * ln_inv_delta / (eps * eps);
}

struct Params {
  double n_max, lambda, lambda1, lambda2, eps1, eps2, eps3;
  int32_t i_max;
};

Params make_params(int64_t n, int k, double eps, double delta, bool dssa) {
  Params P{};
  const double lnC = std::lgamma((double)n + 1.0) - std::lgamma((double)k + 1.0) -
                     std::lgamma((double)(n - k) + 1.0);
  P.n_max = 8.0 * kOneMinusInvE / (2.0 + 2.0 * eps / 3.0) * upsilon_ln(eps, std::log(6.0 / delta) + lnC) *
            (double)n / (double)k;
  P.i_max = (int32_t)std::ceil(std::log2(2.0 * P.n_max / upsilon_ln(eps, std::log(3.0 / delta))));
  if (P.i_max < 1) P.i_max = 1;
  const double lnd = std::log(3.0 * (double)P.i_max / delta);
  P.lambda = upsilon_ln(eps, lnd);
  P.eps2 = eps / (2.0 * kOneMinusInvE);
  P.eps3 = P.eps2;
  P.eps1 = (1.0 + eps / (2.0 * (kOneMinusInvE - eps))) / (1.0 + P.eps2) - 1.0;
  if (dssa) {
    P.lambda1 = 1.0 + (1.0 + eps) * P.lambda;
    P.lambda2 = 0.0;
  } else {
    P.lambda1 = (1.0 + P.eps1) * (1.0 + P.eps2) * upsilon_ln(P.eps3, lnd);
    P.lambda2 = 1.0 + (1.0 + P.eps2) * upsilon_ln(P.eps2, lnd);
  }
  return P;
}
}  // namespace

// ---------------------------------------------------------------------------
// solver
// ---------------------------------------------------------------------------
struct ssa_solver {
  const ssa_graph* g = nullptr;
  int device = 0;
  bool own_stream = false;
  Exec X;
  int64_t byte_cap = 0;
  // workspaces kept across solves: sampler scratch per model, index and greedy buffers
  Sampler S[2];
  bool s_ready[2] = {false, false};
  Cover C;
  bool c_ready = false;
  // CUDA graphs of a round's device work (index, greedy, stare), one
  // executable per (algorithm, round), patched in place by later solves
  bool use_graphs = false;
  bool shared_gpu = false;  // concurrent solves share the GPU (serving): cluster-shaped greedy
  std::vector<cudaGraphExec_t> gexec;
  int64_t graph_launches = 0;

  void release() {
    for (auto e : gexec)
      if (e) cudaGraphExecDestroy(e);
    gexec.clear();
    for (int m = 0; m < 2; ++m)
      if (s_ready[m]) S[m].release(X.st);
    if (c_ready) C.release(X.st);
    s_ready[0] = s_ready[1] = c_ready = false;
    cudaStreamSynchronize(X.st);
  }
};

namespace {
ssa_status check_params(const ssa_graph* g, const ssa_params* p) {
  if (!g || !p) return fail(SSA_E_ARG, "null graph or params");
  if (p->k < 1 || p->k > g->n) return fail(SSA_E_ARG, "k=%d outside [1, n=%lld]", p->k, (long long)g->n);
  if (!(p->eps > 0.0 && p->eps < kOneMinusInvE)) return fail(SSA_E_ARG, "eps must lie in (0, 1-1/e)");
  if (!(p->delta > 0.0 && p->delta < 1.0)) return fail(SSA_E_ARG, "delta must lie in (0, 1)");
  if (p->model != SSA_IC && p->model != SSA_LT) return fail(SSA_E_ARG, "unknown model");
  if (p->algo != SSA_ALGO_SSA && p->algo != SSA_ALGO_DSSA) return fail(SSA_E_ARG, "unknown algorithm");
  if (p->model == SSA_LT && g->weighting == SSA_W_TRIVALENCY)
    return fail(SSA_E_ARG, "LT needs in-weights that sum to at most 1: SSA_W_WC or SSA_W_EXPLICIT");
  return SSA_OK;
}

// Run `issue` (device work only: kernels, memsets, copies into pinned
// memory) as a CUDA graph on the solver's stream: captured, patched into the
// executable cached under `slot` when the topology matches the last one
// (cudaGraphExecUpdate), else instantiated; then launched and waited for.
template <class F>
ssa_status run_graph(ssa_solver* sv, size_t slot, F&& issue) {
  Exec& X = sv->X;
  cudaGraph_t graph = nullptr;
  CU(cudaStreamBeginCapture(X.st, cudaStreamCaptureModeThreadLocal));
  const ssa_status st = issue();
  const cudaError_t ec = cudaStreamEndCapture(X.st, &graph);
  if (st != SSA_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ec != cudaSuccess || !graph) return fail(SSA_E_CUDA, "round capture failed: %s", cudaGetErrorString(ec));
  if (slot >= sv->gexec.size()) sv->gexec.resize(slot + 1, nullptr);
  cudaGraphExec_t& ex = sv->gexec[slot];
  if (ex) {
    cudaGraphExecUpdateResultInfo info{};
    if (cudaGraphExecUpdate(ex, graph, &info) != cudaSuccess) {
      (void)cudaGetLastError();
      cudaGraphExecDestroy(ex);
      ex = nullptr;
    }
  }
  cudaError_t e = cudaSuccess;
  if (!ex) e = cudaGraphInstantiate(&ex, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    ex = nullptr;
    return fail(SSA_E_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
  }
  std::lock_guard<std::mutex> lock(coop_mutex());  // the graph holds a cooperative greedy launch
  CU(cudaGraphLaunch(ex, X.st));
  CU(cudaStreamSynchronize(X.st));
  sv->graph_launches += 1;
  return SSA_OK;
}

ssa_status solve_impl(ssa_solver* sv, const ssa_params* p, ssa_result* out) {
  const double t0 = now_s();
  NvtxRange nv_solve(p && p->algo == SSA_ALGO_DSSA ? "ssa solve (D-SSA)" : "ssa solve (SSA)");
  const ssa_graph* g = sv->g;
  TRY(check_params(g, p));
  if (!out || !out->seeds) return fail(SSA_E_ARG, "result seeds buffer missing");
  Exec& X = sv->X;
  X.launches = 0;
  X.timing = out->want_kstats != 0;
  for (int i = 0; i < SSA_K_COUNT; ++i) out->kstats[i] = ssa_kstat{0, 0.0};
  const bool dssa = p->algo == SSA_ALGO_DSSA;
  const int k = p->k;
  const int64_t n = g->n;
  Params P = make_params(n, k, p->eps, p->delta, dssa);
  if (p->model == SSA_IC) {
    bool tuned;
    {
      std::lock_guard<std::mutex> lock(g->tune_mu);
      tuned = g->tuned_mid_cap >= 0;
    }
    // weighted-cascade sets are mostly one node with a long tail: a pilot of
    // 4096 holds too few large sets to rank the tiers
    if (!tuned) TRY(autotune_ic(g, g->weighting == SSA_W_WC ? 65536 : 4096, X, nullptr, nullptr));
    X.launches = 0;
  }
  Sampler& S = sv->S[p->model];
  Cover& C = sv->C;
  DevPool pool;
  pool.byte_cap = p->pool_bytes_cap > 0 ? p->pool_bytes_cap : sv->byte_cap;
  ssa_status st = SSA_OK;
  std::vector<int32_t> seeds((size_t)k);
  std::vector<int64_t> gains((size_t)k);
  int32_t t = 0;
  int64_t extra_rr = 0;
  int64_t used = 0;  // SSA: sets of the last round (the pool may hold more, sampled ahead)
  double influence = 0.0;
  const bool graphs = sv->use_graphs && !X.timing;
  // Max-Coverage over the whole batches [0, N), and for D-SSA the stare count
  // over the hit-tested check half [N, 2N): as one CUDA graph when enabled
  auto greedy_round = [&](int64_t N, int64_t* cov, int64_t* c) -> ssa_status {
    bool whole = false;
    TRY(C.greedy_prepare(pool, N, k, X));
    TRY(C.index_prepare(pool, N, &whole, X));
    if (c) TRY(S.hits_prepare(N, X));
    if (graphs && whole) {
      TRY(run_graph(sv, (size_t)(dssa ? 64 : 0) + (size_t)t, [&]() -> ssa_status {
        TRY(C.index_issue(pool, N, X));
        TRY(C.greedy_issue(pool, N, k, X));
        return c ? stare_issue(S, C, p->seed, 0, N, N, C.d_seeds, k, X) : SSA_OK;
      }));
    } else {
      TRY(C.index_issue(pool, N, X));
      {
        std::lock_guard<std::mutex> lock(coop_mutex());
        TRY(C.greedy_issue(pool, N, k, X));
        CU(cudaStreamSynchronize(X.st));
      }
      if (c) {
        TRY(stare_issue(S, C, p->seed, 0, N, N, C.d_seeds, k, X));
        CU(cudaStreamSynchronize(X.st));
      }
    }
    TRY(C.greedy_finish(k, seeds.data(), gains.data(), cov));
    return c ? stare_finish(S, C, N, c) : SSA_OK;
  };
  do {
    if (!sv->s_ready[p->model]) {
      sv->s_ready[p->model] = true;  // release() frees whatever init_scratch allocated
      if ((st = S.init_scratch(g, p->model, X)) != SSA_OK) {
        S.release(X.st);
        sv->s_ready[p->model] = false;
        break;
      }
    }
    if ((st = S.begin_solve(g, p->benefit, X)) != SSA_OK) break;
    if (!sv->c_ready) {
      sv->c_ready = true;
      if ((st = C.init(n, X)) != SSA_OK) {
        C.release(X.st);
        sv->c_ready = false;
        break;
      }
    } else if ((st = C.reset(X)) != SSA_OK) {
      break;
    }
    C.shared_gpu = sv->shared_gpu;
    const double scale = p->benefit ? (double)S.wsum : (double)n;
    const int64_t base = (int64_t)std::ceil(P.lambda);
    for (;;) {
      t += 1;
      char rname[32];
      std::snprintf(rname, sizeof(rname), "ssa round %d", (int)t);
      NvtxRange nv_round(rname);
      const int64_t N = base << (t - 1);
      ssa_round rec{};
      rec.t = t;
      rec.n_sets = N;
      rec.check_cov = -1;
      rec.check_T = 0;
      rec.stat = -1.0;
      rec.eps1 = rec.eps2 = rec.eps3 = -1.0;
      int stop = 0;
      if (!dssa) {
        rec.eps1 = P.eps1;
        rec.eps2 = P.eps2;
        rec.eps3 = P.eps3;
        if (pool.count < N) {
          // Each batch ends with its slowest sample (one warp walking the batch's
          // largest set), a fixed cost that dominates small batches.  So the pool
          // grows by at least `ahead` sets: the first rounds then read prefixes
          // of one batch.  Sets are keyed by sample id, so round t still sees
          // exactly R_t = samples [0, N); the extra samples serve the next rounds.
          const int64_t ahead = std::min<int64_t>(n / 64, 131072);
          if ((st = S.append(pool, p->seed, 0, std::max<int64_t>(N - pool.count, ahead), X)) != SSA_OK) break;
        }
        used = N;
        int64_t cov = 0;
        if ((st = greedy_round(N, &cov, nullptr)) != SSA_OK) break;
        rec.cov = cov;
        influence = (double)cov * scale / (double)N;
        if ((double)cov >= P.lambda1) {  // condition C1
          const double d2 = P.eps3 * P.eps3 / (P.eps2 * P.eps2);
          const int64_t t_max = (int64_t)std::ceil(2.0 * (double)N * (1.0 + P.eps2) / (1.0 - P.eps2) * d2);
          const int64_t need = (int64_t)std::ceil(P.lambda2);
          // first batch sized from the greedy's own hit rate cov/N
          const int64_t guess = (int64_t)((double)need * (double)N / (double)cov * 1.15) + 1024;
          int64_t T = 0, hits = 0;
          if ((st = estimate_inf_dev(S, C, p->seed, (uint32_t)t, C.d_seeds, k, need, t_max, guess, &T, &hits, X)) !=
              SSA_OK)
            break;
          extra_rr += T ? T : t_max;
          rec.check_cov = hits;
          rec.check_T = T;
          if (T > 0) {
            const double ic = scale * P.lambda2 / (double)T;
            rec.stat = ic;
            if ((double)cov * scale / (double)N <= (1.0 + P.eps1) * ic) stop = 1;  // condition C2
          }
        }
      } else {
        // R_t = samples [0, N) are in the pool; the check half R^c_t = [N, 2N)
        // only needs "does S meet R_j" now, so it is sampled in hit-test mode
        // (early exit) and stored afterwards only if the loop goes on, when
        // it becomes the second half of R_{t+1} (same keys, same sets).
        if (t == 1 && (st = S.append(pool, p->seed, 0, N, X)) != SSA_OK) break;
        int64_t cov = 0, c = 0;
        if ((st = greedy_round(N, &cov, &c)) != SSA_OK) break;
        rec.cov = cov;
        rec.check_cov = c;
        influence = (double)cov * scale / (double)N;
        if ((double)c >= P.lambda1) {  // condition D1
          const double ic = (double)c * scale / (double)N;
          const double ih = (double)cov * scale / (double)N;
          const double pw = (double)(int64_t(1) << (t - 1));
          const double e1 = ih / ic - 1.0;
          const double e2 = p->eps * std::sqrt(scale * (1.0 + p->eps) / (pw * ic));
          const double e3 = p->eps * std::sqrt(scale * (1.0 + p->eps) * (kOneMinusInvE - p->eps) /
                                               ((1.0 + p->eps / 3.0) * pw * ic));
          const double et = (e1 + e2 + e1 * e2) * (kOneMinusInvE - p->eps) + kOneMinusInvE * e3;
          rec.stat = et;
          rec.eps1 = e1;
          rec.eps2 = e2;
          rec.eps3 = e3;
          if (et <= p->eps) stop = 1;  // condition D2
        }
      }
      if (!stop && ((double)N >= P.n_max || t >= P.i_max)) stop = 2;  // sample cap
      rec.stop = stop ? 1 : 0;
      if (out->trace && t <= out->trace_cap) out->trace[t - 1] = rec;
      if (dssa) {
        if (stop) {
          extra_rr += N;  // R^c_t was drawn (hit-tested) but not stored
        } else if ((st = S.append(pool, p->seed, 0, N, X)) != SSA_OK) {
          break;
        }
      }
      if (stop) break;
    }
  } while (false);
  cudaStreamSynchronize(X.st);
  if (st == SSA_OK) {
    std::memcpy(out->seeds, seeds.data(), sizeof(int32_t) * (size_t)k);
    out->influence = influence;
    out->rounds = t;
    out->n_rr = (dssa ? pool.count : used) + extra_rr;
    out->pool_entries = pool.entries;
    out->edge_visits = S.edge_visits;
    out->node_visits = S.node_visits;
    out->cta_sets = S.cta_samples;
    out->cta_edge_visits = S.cta_edge_visits;
    out->cta_node_visits = S.cta_node_visits;
    out->cta_stored_entries = S.cta_store_nodes;
    out->cta_stored_sets = S.cta_store_sets;
    out->draws = S.draws;
    out->cta_draws = S.cta_draws;
    out->mid_cap = p->model == SSA_IC ? S.mid_cap : 0;
    out->heavy_groups = p->model == SSA_IC ? S.heavy_groups : 0;
    out->kernel_launches = X.launches;
    X.collect(out->kstats);
  } else {
    X.collect(nullptr);
  }
  // the RR pool and this solve's index go back to the device's memory pool;
  // the fixed-size scratch stays with the solver
  pool.release(X.st);
  if (sv->c_ready) C.drop_index(X.st);
  if (sv->s_ready[p->model]) dev_free(S.bprefix, X.st);
  cudaStreamSynchronize(X.st);
  out->seconds = now_s() - t0;
  return st;
}
}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* ssa_status_str(ssa_status s) {
  switch (s) {
    case SSA_OK: return "ok";
    case SSA_E_ARG: return "bad argument";
    case SSA_E_NOMEM: return "out of memory";
    case SSA_E_POOL_FULL: return "RR pool full";
    case SSA_E_CUDA: return "CUDA error";
    case SSA_E_TIMEOUT: return "device wait timed out";
    case SSA_E_CANCELLED: return "cancelled";
    case SSA_E_INTERNAL: return "internal error";
    case SSA_E_NOT_READY: return "not ready";
  }
  return "unknown status";
}

ssa_status ssa_last_error(char* buf, size_t len) {
  if (buf && len) {
    std::strncpy(buf, g_err, len - 1);
    buf[len - 1] = 0;
  }
  return SSA_OK;
}

const char* ssa_version(void) { return "ssa-gb300 0.2 sm_103a"; }

ssa_status ssa_device_code_version(int32_t* binary, int32_t* ptx) {
  if (!binary || !ptx) return fail(SSA_E_ARG, "null output");
  int b = 0, p = 0;
  CU(device_code_version(&b, &p));
  *binary = b;
  *ptx = p;
  return SSA_OK;
}

ssa_status ssa_load_graph(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, const uint32_t* thr,
                          ssa_weighting weighting, uint64_t weight_seed, ssa_graph** out) {
  if (!out) return fail(SSA_E_ARG, "null output handle");
  *out = nullptr;
  if (n < 1 || n > 0x7FFFFFFF || m < 0 || m > 0x7FFFFFFF) return fail(SSA_E_ARG, "n or m out of range");
  if (m > 0 && (!src || !dst)) return fail(SSA_E_ARG, "null edge arrays");
  if (weighting != SSA_W_WC && weighting != SSA_W_TRIVALENCY && weighting != SSA_W_EXPLICIT)
    return fail(SSA_E_ARG, "unknown weighting");
  if (weighting == SSA_W_EXPLICIT && m > 0 && !thr) return fail(SSA_E_ARG, "explicit weighting needs thr");
  ssa_graph* g = new ssa_graph();
  cudaGetDevice(&g->device);
  g->n = n;
  g->m = m;
  g->weighting = weighting;
  cudaStream_t st;
  CU(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  int32_t *d_src = nullptr, *d_dst = nullptr;
  uint32_t* d_thr = nullptr;
  unsigned int* d_err = nullptr;
  ssa_status rc = SSA_OK;
  do {
    const int64_t m_pad = ((m + 3) / 4) * 4 + 4;
    if ((rc = dev_alloc(&g->off, (size_t)n + 1, st)) != SSA_OK) break;
    if ((rc = dev_alloc(&g->edge, (size_t)m_pad, st)) != SSA_OK) break;
    if (cudaMemsetAsync(g->edge, 0, sizeof(uint2) * (size_t)m_pad, st) != cudaSuccess) {
      rc = fail(SSA_E_CUDA, "memset failed");
      break;
    }
    g->bytes = (int64_t)(sizeof(int64_t) * (size_t)(n + 1) + sizeof(uint2) * (size_t)m_pad);
    if ((rc = dev_alloc(&d_err, 1, st)) != SSA_OK) break;
    cudaMemsetAsync(d_err, 0, sizeof(unsigned int), st);
    if (m > 0) {
      if ((rc = dev_alloc(&d_src, (size_t)m, st)) != SSA_OK) break;
      if ((rc = dev_alloc(&d_dst, (size_t)m, st)) != SSA_OK) break;
      cudaMemcpyAsync(d_src, src, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(d_dst, dst, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, st);
      if (weighting == SSA_W_EXPLICIT) {
        if ((rc = dev_alloc(&d_thr, (size_t)m, st)) != SSA_OK) break;
        cudaMemcpyAsync(d_thr, thr, sizeof(uint32_t) * (size_t)m, cudaMemcpyHostToDevice, st);
      }
    }
    int launches = 0;
    cudaError_t e = build_graph(n, m, d_src, d_dst, d_thr, weighting, weight_seed, g->off, g->edge, d_err, st,
                                &launches);
    if (e != cudaSuccess) {
      rc = fail(e == cudaErrorMemoryAllocation ? SSA_E_NOMEM : SSA_E_CUDA, "graph build: %s", cudaGetErrorString(e));
      break;
    }
    unsigned int herr = 0;
    cudaMemcpyAsync(&herr, d_err, sizeof(herr), cudaMemcpyDeviceToHost, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      rc = fail(SSA_E_CUDA, "graph build: %s", cudaGetErrorString(e));
      break;
    }
    if (herr) {
      rc = fail(SSA_E_ARG, "edge endpoint outside [0, n)");
      break;
    }
    if (weighting == SSA_W_WC) {
      e = build_wc_pow(g->off, n, &g->wc_pow, &g->wc_pow_k, st);
      if (e != cudaSuccess) {
        rc = fail(e == cudaErrorMemoryAllocation ? SSA_E_NOMEM : SSA_E_CUDA, "power table: %s", cudaGetErrorString(e));
        break;
      }
      if (g->wc_pow_k > 0) g->bytes += (int64_t)(sizeof(uint64_t) * (((size_t)g->wc_pow_k - 1) << g->wc_pow_k) + 8);
    }
  } while (false);
  if (d_src) cudaFreeAsync(d_src, st);
  if (d_dst) cudaFreeAsync(d_dst, st);
  if (d_thr) cudaFreeAsync(d_thr, st);
  if (d_err) cudaFreeAsync(d_err, st);
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  if (rc != SSA_OK) {
    if (g->off) cudaFree(g->off);
    if (g->edge) cudaFree(g->edge);
    if (g->wc_pow) cudaFree(g->wc_pow);
    delete g;
    return rc;
  }
  *out = g;
  return SSA_OK;
}

namespace {
// a probability as a 32-bit threshold: floor(p 2^32), clamped to [0, 2^32 - 1]
uint32_t prob_threshold(double p) {
  if (!(p > 0.0)) return 0u;
  const double x = p * 4294967296.0;
  return x >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)x;
}
}  // namespace

ssa_status ssa_gen_rmat(int32_t scale, int64_t m_draw, double a, double b, double c, uint64_t seed,
                        ssa_weighting weighting, uint64_t weight_seed, ssa_graph** out) {
  if (!out) return fail(SSA_E_ARG, "null output handle");
  *out = nullptr;
  if (scale < 1 || scale > 30) return fail(SSA_E_ARG, "scale must lie in [1, 30]");
  if (m_draw < 0 || m_draw > 0x7FFFFFFF) return fail(SSA_E_ARG, "m_draw must lie in [0, 2^31 - 1]");
  if (!(a >= 0.0 && b >= 0.0 && c >= 0.0 && a + b + c <= 1.0))
    return fail(SSA_E_ARG, "quadrant probabilities must be >= 0 with a + b + c <= 1");
  if (weighting != SSA_W_WC && weighting != SSA_W_TRIVALENCY)
    return fail(SSA_E_ARG, "ssa_gen_rmat weights: SSA_W_WC or SSA_W_TRIVALENCY");
  cudaStream_t st;
  CU(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  ssa_graph* g = new ssa_graph();
  cudaGetDevice(&g->device);
  g->n = int64_t(1) << scale;
  g->weighting = weighting;
  int launches = 0;
  int64_t m = 0;
  cudaError_t e = rmat_graph(scale, m_draw, prob_threshold(a), prob_threshold(a + b), prob_threshold(a + b + c), seed,
                             (int)weighting, weight_seed, &m, &g->off, &g->edge, st, &launches);
  if (e == cudaSuccess && weighting == SSA_W_WC) e = build_wc_pow(g->off, g->n, &g->wc_pow, &g->wc_pow_k, st);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    if (g->off) cudaFree(g->off);
    if (g->edge) cudaFree(g->edge);
    if (g->wc_pow) cudaFree(g->wc_pow);
    delete g;
    return fail(e == cudaErrorMemoryAllocation ? SSA_E_NOMEM : SSA_E_CUDA, "R-MAT generation: %s",
                cudaGetErrorString(e));
  }
  g->m = m;
  g->bytes = (int64_t)(sizeof(int64_t) * (size_t)(g->n + 1) + sizeof(uint2) * (size_t)(((m + 3) / 4) * 4 + 4));
  if (g->wc_pow_k > 0) g->bytes += (int64_t)(sizeof(uint64_t) * (((size_t)g->wc_pow_k - 1) << g->wc_pow_k) + 8);
  *out = g;
  return SSA_OK;
}

ssa_status ssa_free_graph(ssa_graph* g) {
  if (!g) return SSA_OK;
  cudaDeviceSynchronize();
  if (g->off) cudaFree(g->off);
  if (g->edge) cudaFree(g->edge);
  if (g->wc_pow) cudaFree(g->wc_pow);
  delete g;
  return SSA_OK;
}

ssa_status ssa_graph_info(const ssa_graph* g, int64_t* n, int64_t* m, int64_t* bytes) {
  if (!g) return fail(SSA_E_ARG, "null graph");
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (bytes) *bytes = g->bytes;
  return SSA_OK;
}

ssa_status ssa_graph_export(const ssa_graph* g, int64_t* off, int32_t* src, uint32_t* thr) {
  if (!g) return fail(SSA_E_ARG, "null graph");
  if (off) CU(cudaMemcpy(off, g->off, sizeof(int64_t) * (size_t)(g->n + 1), cudaMemcpyDeviceToHost));
  if ((src || thr) && g->m > 0) {
    std::vector<uint2> e((size_t)g->m);
    CU(cudaMemcpy(e.data(), g->edge, sizeof(uint2) * (size_t)g->m, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < g->m; ++i) {
      if (src) src[i] = (int32_t)e[(size_t)i].x;
      if (thr) thr[i] = e[(size_t)i].y;
    }
  }
  return SSA_OK;
}

ssa_solver* new_solver_keep_pool_memory() {
  // Solves allocate and free multi-GB workspaces stream-ordered; keep freed
  // memory in the device's default pool instead of unmapping it at each sync.
  int dev = 0;
  cudaGetDevice(&dev);
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  return new ssa_solver();
}

ssa_status ssa_autotune(const ssa_graph* g, ssa_model model, int64_t pilot_samples, int32_t* mid_cap,
                        double* pilot_ms) {
  if (!g) return fail(SSA_E_ARG, "null graph");
  if (model != SSA_IC) {
    if (mid_cap) *mid_cap = 0;
    return SSA_OK;  // the LT walk has one tier pair and nothing to tune
  }
  if (pilot_samples < 1) pilot_samples = 8192;
  Exec X;
  CU(cudaStreamCreateWithFlags(&X.st, cudaStreamNonBlocking));
  int chosen = 0;
  double ms = 0;
  ssa_status st = autotune_ic(g, pilot_samples, X, &chosen, &ms);
  cudaStreamSynchronize(X.st);
  cudaStreamDestroy(X.st);
  X.st = nullptr;
  if (st != SSA_OK) return st;
  if (mid_cap) *mid_cap = chosen;
  if (pilot_ms) *pilot_ms = ms;
  return SSA_OK;
}

ssa_status ssa_set_warp_tier(const ssa_graph* g, int32_t global_bitmap) {
  if (!g) return fail(SSA_E_ARG, "null graph");
  std::lock_guard<std::mutex> lock(g->tune_mu);
  g->tuned_warp_global = global_bitmap != 0 ? 1 : 0;
  return SSA_OK;
}

ssa_status ssa_set_lane_tier(const ssa_graph* g, int32_t on) {
  if (!g) return fail(SSA_E_ARG, "null graph");
  std::lock_guard<std::mutex> lock(g->tune_mu);
  g->tuned_lane_tier = on != 0 ? 1 : 0;
  return SSA_OK;
}

ssa_status ssa_set_queue_tuning(const ssa_graph* g, int32_t small_queue) {
  if (!g || small_queue < 0) return fail(SSA_E_ARG, "need a graph and small_queue >= 0");
  std::lock_guard<std::mutex> lock(g->tune_mu);
  g->tuned_small_qcap = small_queue;
  return SSA_OK;
}

ssa_status ssa_set_greedy_mode(int32_t mode) {
  if (mode < 0 || mode > 2) return fail(SSA_E_ARG, "greedy mode must be 0, 1 or 2");
  set_greedy_mode(mode);
  return SSA_OK;
}

ssa_status ssa_set_wait_polls(int64_t polls) {
  if (polls < 0) return fail(SSA_E_ARG, "polls must be >= 0");
  g_wait_polls.store(polls == 0 ? GREEDY_DEFAULT_WAIT_POLLS : (long long)polls, std::memory_order_relaxed);
  return SSA_OK;
}

ssa_status ssa_set_tuning(const ssa_graph* g, int32_t mid_cap, int32_t heavy_groups) {
  if (!g || mid_cap < 0 || mid_cap > mid_tier_max_cap()) return fail(SSA_E_ARG, "mid_cap outside [0, 16384]");
  if (heavy_groups < 1) return fail(SSA_E_ARG, "heavy_groups must be >= 1");
  std::lock_guard<std::mutex> lock(g->tune_mu);
  g->tuned_mid_cap = mid_cap;
  g->tuned_heavy = heavy_groups;
  return SSA_OK;
}

ssa_status ssa_solver_create(const ssa_graph* g, void* stream, int64_t pool_bytes_cap, ssa_solver** out) {
  if (!g || !out) return fail(SSA_E_ARG, "null graph or output");
  ssa_solver* s = new_solver_keep_pool_memory();
  s->g = g;
  cudaGetDevice(&s->device);
  if (stream) {
    s->X.st = static_cast<cudaStream_t>(stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&s->X.st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete s;
      return fail(SSA_E_CUDA, "stream create: %s", cudaGetErrorString(e));
    }
    s->own_stream = true;
  }
  if (pool_bytes_cap <= 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    pool_bytes_cap = (int64_t)((double)fr * 0.6);
  }
  s->byte_cap = pool_bytes_cap;
  *out = s;
  return SSA_OK;
}

ssa_status ssa_solver_solve(ssa_solver* s, const ssa_params* p, ssa_result* out) {
  if (!s) return fail(SSA_E_ARG, "null solver");
  return solve_impl(s, p, out);
}

ssa_status ssa_solver_set_graphs(ssa_solver* s, int32_t on) {
  if (!s) return fail(SSA_E_ARG, "null solver");
  s->use_graphs = on != 0;
  return SSA_OK;
}

ssa_status ssa_solver_set_shared(ssa_solver* s, int32_t on) {
  if (!s) return fail(SSA_E_ARG, "null solver");
  s->shared_gpu = on != 0;
  return SSA_OK;
}

ssa_status ssa_solver_free(ssa_solver* s) {
  if (!s) return SSA_OK;
  cudaStreamSynchronize(s->X.st);
  s->release();
  if (s->own_stream) cudaStreamDestroy(s->X.st);
  s->X.st = nullptr;
  delete s;
  return SSA_OK;
}

ssa_status ssa_solve(const ssa_graph* g, const ssa_params* p, ssa_result* out) {
  ssa_solver* s = nullptr;
  TRY(ssa_solver_create(g, nullptr, p ? p->pool_bytes_cap : 0, &s));
  ssa_status st = ssa_solver_solve(s, p, out);
  ssa_solver_free(s);
  return st;
}

// ---- pools (hot-path steps one by one) ----
struct ssa_pool {
  const ssa_graph* g = nullptr;
  int device = 0;
  uint64_t seed = 0;
  uint32_t stream = 0;
  Exec X;
  Sampler S;
  DevPool P;
  Cover C;
};

ssa_status ssa_pool_create(const ssa_graph* g, ssa_model model, uint64_t seed, uint32_t stream,
                           const uint32_t* benefit, ssa_pool** out) {
  if (!g || !out) return fail(SSA_E_ARG, "null graph or output");
  if (model != SSA_IC && model != SSA_LT) return fail(SSA_E_ARG, "unknown model");
  if (model == SSA_LT && g->weighting == SSA_W_TRIVALENCY)
    return fail(SSA_E_ARG, "LT needs SSA_W_WC or SSA_W_EXPLICIT in-weights");
  if (stream > 255) return fail(SSA_E_ARG, "stream must be < 256");
  ssa_pool* p = new ssa_pool();
  p->g = g;
  p->seed = seed;
  p->stream = stream;
  cudaGetDevice(&p->device);
  if (cudaStreamCreateWithFlags(&p->X.st, cudaStreamNonBlocking) != cudaSuccess) {
    delete p;
    return fail(SSA_E_CUDA, "stream create failed");
  }
  ssa_status st = p->S.init(g, model, benefit, p->X);
  if (st == SSA_OK) st = p->C.init(g->n, p->X);
  if (st != SSA_OK) {
    ssa_pool_free(p);
    return st;
  }
  *out = p;
  return SSA_OK;
}

ssa_status ssa_pool_free(ssa_pool* p) {
  if (!p) return SSA_OK;
  p->P.release(p->X.st);
  p->S.release(p->X.st);
  p->C.release(p->X.st);
  cudaStreamSynchronize(p->X.st);
  cudaStreamDestroy(p->X.st);
  delete p;
  return SSA_OK;
}

ssa_status ssa_pool_grow(ssa_pool* p, int64_t count) {
  if (!p) return fail(SSA_E_ARG, "null pool");
  if (count <= p->P.count) return SSA_OK;
  return p->S.append(p->P, p->seed, p->stream, count - p->P.count, p->X);
}

ssa_status ssa_pool_info(const ssa_pool* p, int64_t* count, int64_t* entries, int64_t* edge_visits) {
  if (!p) return fail(SSA_E_ARG, "null pool");
  if (count) *count = p->P.count;
  if (entries) *entries = p->P.entries;
  if (edge_visits) *edge_visits = p->S.edge_visits;
  return SSA_OK;
}

ssa_status ssa_pool_export(const ssa_pool* pc, int64_t first, int64_t count, int64_t* off, int32_t* nodes,
                           int64_t cap) {
  ssa_pool* p = const_cast<ssa_pool*>(pc);
  if (!p || !off) return fail(SSA_E_ARG, "null pool or offsets");
  if (first < 0 || count < 0 || first + count > p->P.count) return fail(SSA_E_ARG, "set range outside the pool");
  std::vector<int32_t> len((size_t)count);
  if (count > 0)
    CU(cudaMemcpy(len.data(), p->P.set_len + first, sizeof(int32_t) * (size_t)count, cudaMemcpyDeviceToHost));
  off[0] = 0;
  for (int64_t i = 0; i < count; ++i) off[i + 1] = off[i] + len[(size_t)i];
  if (off[count] > cap || (!nodes && off[count] > 0)) return fail(SSA_E_ARG, "nodes buffer too small");
  if (off[count] == 0) return SSA_OK;
  int64_t* d_off = nullptr;
  int32_t* d_out = nullptr;
  TRY(dev_alloc(&d_off, (size_t)count + 1, p->X.st));
  TRY(dev_alloc(&d_out, (size_t)off[count], p->X.st));
  CU(cudaMemcpyAsync(d_off, off, sizeof(int64_t) * (size_t)(count + 1), cudaMemcpyHostToDevice, p->X.st));
  CU(launch_gather_sets(p->P.nodes, p->P.set_start, p->P.set_len, d_off, first, count, d_out, p->X.st));
  CU(cudaMemcpyAsync(nodes, d_out, sizeof(int32_t) * (size_t)off[count], cudaMemcpyDeviceToHost, p->X.st));
  CU(cudaStreamSynchronize(p->X.st));
  dev_free(d_off, p->X.st);
  dev_free(d_out, p->X.st);
  CU(cudaStreamSynchronize(p->X.st));
  return SSA_OK;
}

ssa_status ssa_pool_counts(ssa_pool* p, int64_t N, int32_t* cnt) {
  if (!p || !cnt) return fail(SSA_E_ARG, "null pool or output");
  if (N < 0 || N > p->P.count) return fail(SSA_E_ARG, "N outside the pool");
  TRY(p->C.build_index(p->P, N, p->X));
  CU(cudaMemcpyAsync(cnt, p->C.cnt, sizeof(int32_t) * (size_t)p->g->n, cudaMemcpyDeviceToHost, p->X.st));
  CU(cudaStreamSynchronize(p->X.st));
  return SSA_OK;
}

ssa_status ssa_max_coverage(ssa_pool* p, int64_t N, int32_t k, int32_t* seeds, int64_t* gains, int64_t* cov) {
  if (!p || !seeds || !gains || !cov) return fail(SSA_E_ARG, "null argument");
  if (N < 0 || N > p->P.count) return fail(SSA_E_ARG, "N outside the pool");
  if (k < 1 || k > p->g->n) return fail(SSA_E_ARG, "k outside [1, n]");
  return p->C.greedy(p->P, N, k, seeds, gains, cov, p->X);
}

ssa_status ssa_coverage(ssa_pool* p, int64_t first, int64_t count, const int32_t* seeds, int32_t k, int64_t* cov) {
  if (!p || !cov || (k > 0 && !seeds)) return fail(SSA_E_ARG, "null argument");
  if (first < 0 || count < 0 || first + count > p->P.count) return fail(SSA_E_ARG, "set range outside the pool");
  for (int i = 0; i < k; ++i)
    if (seeds[i] < 0 || seeds[i] >= p->g->n) return fail(SSA_E_ARG, "seed id outside [0, n)");
  int32_t* d = nullptr;
  TRY(dev_alloc(&d, (size_t)std::max(k, 1), p->X.st));
  if (k > 0) CU(cudaMemcpyAsync(d, seeds, sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, p->X.st));
  CU(cudaMemsetAsync(p->C.in_seed, 0, (size_t)p->C.n_pad, p->X.st));
  if (k > 0) CU(launch_set_bits(d, k, nullptr, p->C.in_seed, p->X.st));
  ssa_status st = p->C.coverage_range(p->P, first, first + count, cov, p->X);
  dev_free(d, p->X.st);
  cudaStreamSynchronize(p->X.st);
  return st;
}

ssa_status ssa_estimate_inf(const ssa_graph* g, ssa_model model, uint64_t seed, uint32_t stream,
                            const uint32_t* benefit, const int32_t* seeds, int32_t k, double lambda2, int64_t t_max,
                            int64_t* T, int64_t* hits) {
  if (!g || !T || !hits || (k > 0 && !seeds)) return fail(SSA_E_ARG, "null argument");
  if (stream > 255) return fail(SSA_E_ARG, "stream must be < 256");
  if (!(lambda2 >= 1.0) || t_max < 0) return fail(SSA_E_ARG, "need lambda2 >= 1 and t_max >= 0");
  for (int i = 0; i < k; ++i)
    if (seeds[i] < 0 || seeds[i] >= g->n) return fail(SSA_E_ARG, "seed id outside [0, n)");
  ssa_pool* p = nullptr;
  TRY(ssa_pool_create(g, model, seed, stream, benefit, &p));
  ssa_status st = SSA_OK;
  int32_t* d = nullptr;
  do {
    if ((st = dev_alloc(&d, (size_t)std::max(k, 1), p->X.st)) != SSA_OK) break;
    if (k > 0 && cudaMemcpyAsync(d, seeds, sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, p->X.st) !=
                     cudaSuccess) {
      st = fail(SSA_E_CUDA, "copy seeds");
      break;
    }
    const int64_t need = (int64_t)std::ceil(lambda2);
    st = estimate_inf_dev(p->S, p->C, seed, stream, d, k, need, t_max, std::min<int64_t>(t_max, 1 << 16), T, hits,
                          p->X);
  } while (false);
  dev_free(d, p->X.st);
  ssa_pool_free(p);
  return st;
}

}  // extern "C"
