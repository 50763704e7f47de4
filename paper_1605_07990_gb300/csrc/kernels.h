// Internal interface between the host driver (api.cpp) and the sm_103a
// kernels (*.cu).  Plain structs of device pointers; no torch types.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ssa {

// Sets the calling thread's message returned by ssa_last_error().
void set_last_error(const char* msg);

// Device-resident in-edge CSR (Sec. 2).  Edge records interleave the tail
// node and the uint32 live threshold so one 8-byte load serves an edge and a
// 4-edge group (the unit of one Philox draw) is one aligned 32-byte sector.
struct GraphView {
  int64_t n = 0, m = 0;
  const int64_t* off = nullptr;  // n+1
  const uint2* edge = nullptr;   // m rounded up to a multiple of 4 (+4): {src, thr}
  // weighted cascade: the gap form's powers q^(2^i) of every in-degree d < 2^wc_pow_k
  // (rows of bit-length entries, in order of d; null / 0 for other weightings)
  const uint64_t* wc_pow = nullptr;
  int wc_pow_k = 0;
};

// In-degrees of up to 2^WC_POW_K - 1 take their gap powers from the graph's
// table ((WC_POW_K - 1) 2^WC_POW_K + 1 entries, 160 MB); larger ones build them.
constexpr int WC_POW_K = 20;

// The weighted-cascade power table of a CSR (rows for every in-degree below
// min(2^WC_POW_K, 2 * max in-degree)); *tab stays null when no in-list has 2 edges.
cudaError_t build_wc_pow(const int64_t* d_off, int64_t n, uint64_t** tab, int* k, cudaStream_t st);

// Device counters of one sampling batch.
// Bounded waits of the weighted-cascade CTA tier that gave up (Counters::error).
constexpr unsigned SAMPLER_ERR_SLOT = 1;  // a claimed queue slot was never written
constexpr unsigned SAMPLER_ERR_IDLE = 2;  // a warp found no work for far longer than any sample

struct Counters {
  unsigned long long work;         // warp tier: next sample index
  unsigned long long mid_count;    // samples handed from the shared-memory warp tier to the global one
  unsigned long long mid_work;     // global warp tier: next list index
  unsigned long long big_count;    // samples handed to the CTA tier
  unsigned long long big_work;     // CTA tier: next list index
  unsigned long long big2_count;   // samples that outgrew the small CTAs' queue
  unsigned long long big2_work;
  unsigned long long cursor;       // pool entries reserved (absolute)
  unsigned long long edge_visits;  // in-edges examined
  unsigned long long node_visits;  // nodes added to RR sets
  unsigned long long cta_edge_visits;  // the CTA tier's share of the two above
  unsigned long long cta_node_visits;
  unsigned long long cta_draws;    // the CTA tier's share of draws
  unsigned long long draws;        // Philox draws (IC: one per 4-edge group that needed coins)
  unsigned long long ok_end;        // start of the first pool reservation that did not fit (the
                                    // host sets ~0 before a storing launch): the ones that fit end there
  unsigned long long fail_count;    // samples whose reservation did not fit (listed in fail_list)
  unsigned long long lane_work;    // lane tier: next sample index
  unsigned long long lane_count;   // samples the lane tier handed to the warp tiers
  unsigned int pool_overflow;      // a reservation passed pool_cap
  unsigned int error;              // internal error: 0 none, else SAMPLER_ERR_* of the first wait that gave up
};

enum : int { MODE_STORE = 0, MODE_HIT = 1 };

struct SampleJob {
  GraphView g;
  int model = 0;                 // 0 IC, 1 LT
  int lt_cumulative = 0;         // LT with explicit in-weights: pick by running threshold sums
  int wc_implicit = 0;           // IC with weighted-cascade weights: thresholds from in-degrees,
                                 // records read for live edges only
  int warp_global = 0;           // weighted-cascade IC: every sample through the global-bitmap warp tier
  int lane_tier = 0;             // weighted-cascade IC: the lane tier runs first; the warp tiers take
                                 // only the samples it lists in lane_list (capacity `count`)
  int64_t* lane_list = nullptr;
  uint32_t* wg_bitmap = nullptr; // that tier: per warp bitmap_words words, zero between samples
  int32_t* wg_queue = nullptr;   // that tier: per warp wg_queue_per_warp() entries
  uint64_t seed = 0;
  uint32_t stream = 0;
  int64_t j0 = 0, count = 0;     // samples [j0, j0+count), or work_list[0, count)
  const int64_t* work_list = nullptr;  // explicit sample ids (re-run of pool overflows) or null
  int64_t* fail_list = nullptr;        // samples whose pool reservation did not fit
  uint32_t rk[20] = {};                // Philox round keys: rk[2r], rk[2r+1] = key + r * Weyl
  const uint64_t* bprefix = nullptr;  // WRIS prefix sums (n+1) or null
  int mode = MODE_STORE;
  // MODE_STORE: flat pool entries + per-sample extents
  int32_t* pool_nodes = nullptr;
  int32_t* pool_samp = nullptr;
  int64_t pool_cap = 0;
  int64_t* set_start = nullptr;  // indexed by absolute sample id
  int32_t* set_len = nullptr;
  // MODE_HIT: seed membership bits, per-sample flag (index j - j0)
  const uint32_t* seed_bits = nullptr;
  uint8_t* hit = nullptr;
  // global-memory warp tier: hand-off list and per-warp hash / queue / slot scratch
  int warp_heavy_groups = 0x7FFFFFFF;  // warp tiers hand samples meeting an in-list of more 4-edge
                                       // groups than this to the CTA tier (tuned)
  int mid_cap = 0;               // sets above 512 nodes: 0 = straight to the CTA tier, else the
                                 // global warp tier keeps sets up to mid_cap nodes (<= 16384)
  int64_t* mid_list = nullptr;   // capacity `count`
  uint32_t* mid_hash = nullptr;  // per warp: mid_hash_per_warp() words, zero between samples
  int32_t* mid_queue = nullptr;  // per warp: mid_queue_per_warp()
  uint32_t* mid_slots = nullptr; // per warp: mid_queue_per_warp()
  // CTA tier hand-off and scratch
  int64_t* big_list = nullptr;   // capacity `count`
  uint32_t* slot_bitmap = nullptr;  // per CTA slot: bitmap_words (unused when the bitmap is in smem)
  int32_t* slot_queue = nullptr;    // per CTA slot: n entries
  // small CTAs (global bitmap only): per slot a queue of small_qcap entries and a bitmap
  int small_qcap = 0;
  int32_t* small_queue = nullptr;
  uint32_t* small_bitmap = nullptr;
  int64_t* big2_list = nullptr;     // capacity `count`
  int64_t bitmap_words = 0;
  Counters* ctr = nullptr;
};

struct LaunchCfg {
  int num_sms = 152;
  int warp_blocks = 0;   // grid of the warp tier
  int cta_blocks = 0;    // grid of the CTA tier (= number of scratch slots)
  int mid_blocks = 0;    // grid of the global-memory warp tier
  int cta_threads = 1024;
  int small_blocks = 0;  // small CTAs (256 threads) when the bitmap lives in global memory
  int small_qcap = 0;
  int wg_blocks = 0;     // global-bitmap warp tier (0: not available for this graph)
  int lane_blocks = 0;   // lane tier (weighted-cascade IC)
  bool cta_smem_bitmap = false;
  int64_t smem_bitmap_bytes = 0;
};

// ---- graph build -------------------------------------------------------
// Sorts edges by (dst, src, input position), builds off/edge records and
// thresholds.  d_src/d_dst/d_thr_in are device arrays of length m.
cudaError_t build_graph(int64_t n, int64_t m, const int32_t* d_src, const int32_t* d_dst,
                        const uint32_t* d_thr_in, int weighting, uint64_t weight_seed,
                        int64_t* d_off, uint2* d_edge, unsigned int* d_err, cudaStream_t st,
                        int* launches);

// Directed R-MAT graph on 2^scale nodes from m_draw SplitMix64-keyed draws
// (quadrant thresholds ta < tab < tabc of a 32-bit draw), self-loops and
// duplicates removed, built straight into the in-edge CSR (allocated here,
// stream-ordered; the caller owns *d_off and *d_edge).  *m_out: unique edges.
cudaError_t rmat_graph(int scale, int64_t m_draw, uint32_t ta, uint32_t tab, uint32_t tabc, uint64_t seed,
                       int weighting, uint64_t weight_seed, int64_t* m_out, int64_t** d_off, uint2** d_edge,
                       cudaStream_t st, int* launches);

// ---- sampling -----------------------------------------------------------
LaunchCfg sampler_config(const GraphView& g, int model, bool wc_implicit);
size_t sampler_scratch_bytes(const GraphView& g, const LaunchCfg& c);
size_t mid_tier_words(const LaunchCfg& c);  // number of warps of the global-memory tier
size_t wg_tier_warps(const LaunchCfg& c);   // warps of the global-bitmap tier
size_t wg_queue_per_warp();
int mid_tier_max_cap();
size_t mid_hash_per_warp();
size_t mid_queue_per_warp();
cudaError_t launch_sample_warp(const SampleJob& J, const LaunchCfg& c, cudaStream_t st);
cudaError_t launch_sample_cta(const SampleJob& J, const LaunchCfg& c, cudaStream_t st);

// ---- index, greedy, stare -----------------------------------------------
cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t st);
// entries [e0, e1); with samp non-null only samples in [jlo, jhi) count
cudaError_t launch_count_nodes(const int32_t* nodes, const int32_t* samp, int64_t e0, int64_t e1, int64_t jlo,
                               int64_t jhi, int32_t* cnt, cudaStream_t st, int num_sms);
// exclusive scan of int32 counts into int64 offsets (n+1 outputs); tmp >= scan_tmp_bytes(n)
size_t scan_tmp_bytes(int64_t n);
cudaError_t launch_exclusive_scan(const int32_t* in, int64_t n, int64_t* out, void* tmp, cudaStream_t st,
                                  int* launches);
cudaError_t launch_scatter_index(const int32_t* nodes, const int32_t* samp, int64_t e0, int64_t e1, int64_t jlo,
                                 int64_t jhi, unsigned long long* cur, int32_t* inv_samp, cudaStream_t st,
                                 int num_sms);

constexpr int GREEDY_MAX_LISTS = 48;
struct InvList {
  const int64_t* off;           // n+1 offsets of one index batch
  const int32_t* samp;          // its sample ids
};
struct GreedyJob {
  int32_t* cnt;                 // n_pad working gains; negative = picked or padding
  int64_t n_pad;                // multiple of 4
  InvList lists[GREEDY_MAX_LISTS];
  int nlists;
  const int32_t* pool_nodes;
  const int64_t* set_start;
  const int32_t* set_len;
  uint8_t* covered;             // per sample id, zeroed
  int32_t* seeds;               // k (device)
  int32_t* gains;               // k (device)
  int k;
  unsigned long long* argmax;   // 64 + 2 x 1024 words, zeroed: 3 argmax slots 16 words apart,
                                // then per-block covered-entry [64 + b] and queued-entry
                                // [64 + 1024 + b] tallies
  int64_t n_sets;               // N: sets [0, N) take part
  unsigned long long total_entries;  // entries of those sets
  unsigned int* sync;           // 128 words, zeroed: count [0], release word (64-bit) [32],
                                // timeout flag [64], chunk-queue lengths [96], [112]
  unsigned long long* chunk_q;  // (set, first member) of queued decrement chunks
  int64_t chunk_cap;
  unsigned int* hist;           // 2 x 4096 gain-histogram bins, zeroed
  int32_t* cache;               // 2 x 8192 candidate nodes
  unsigned int* cache_n;        // 2 counts, zeroed
  long long wait_polls;         // polls after which a grid-barrier wait gives up
};
constexpr long long GREEDY_DEFAULT_WAIT_POLLS = 1ll << 22;  // about a second with the poll back-off
// Process-wide poll limit of the greedy kernel's grid-barrier waits (ssa_set_wait_polls).
long long greedy_wait_polls();
// All k picks in one launch: a cooperative grid (bounded grid barriers), or,
// for a solve that shares the GPU with others and a pool of up to
// GREEDY_CLUSTER_ENTRIES entries, one thread-block cluster.
constexpr unsigned long long GREEDY_CLUSTER_ENTRIES = 1ull << 26;
cudaError_t launch_greedy(const GreedyJob& J, cudaStream_t st, int num_sms, int* blocks_used, bool shared_gpu);
// 0: by the rule above (default); 1: always the cooperative grid; 2: always a cluster (when the device has one)
void set_greedy_mode(int mode);
cudaError_t launch_add_counts(int32_t* total, const int32_t* add, int64_t n, cudaStream_t st, int num_sms);
// SASS and PTX versions (major*10 + minor) of the device code the CUDA runtime loaded for this library
cudaError_t device_code_version(int* binary, int* ptx);

cudaError_t launch_mark_hits(const int32_t* nodes, const int32_t* samp, int64_t e0, int64_t e1,
                             const uint8_t* in_seed, int64_t j0, int64_t j1, uint8_t* hit, cudaStream_t st,
                             int num_sms);
cudaError_t launch_count_flags(const uint8_t* flags, int64_t count, unsigned long long* out,
                               cudaStream_t st, int num_sms);
// First T (1-based) in flags[0, count) where base + prefix hits reaches `need`;
// out[0] = T or 0, out[1] = hits in [0, count).
cudaError_t launch_first_reach(const uint8_t* flags, int64_t count, long long need_minus_base,
                               long long* out, void* tmp, cudaStream_t st, int* launches);
size_t first_reach_tmp_bytes(int64_t count);

cudaError_t launch_set_bits(const int32_t* ids, int k, uint32_t* bits, uint8_t* bytes, cudaStream_t st);
cudaError_t launch_gather_sets(const int32_t* pool_nodes, const int64_t* set_start, const int32_t* set_len,
                               const int64_t* out_off, int64_t first, int64_t count, int32_t* out,
                               cudaStream_t st);

}  // namespace ssa
