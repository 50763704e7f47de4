/*
 * ssa.h -- C ABI of the GB300 Stop-and-Stare library (libssa.so).
 *
 * Influence maximisation by reverse influence sampling with the SSA and D-SSA
 * stopping rules of Nguyen, Thai, Dinh, "Stop-and-Stare: Optimal Sampling
 * Algorithms for Viral Marketing in Billion-scale Networks" (arXiv 1605.07990).
 * Every compute step runs in the library's own sm_103a CUDA kernels; the host
 * side only evaluates the FP64 stopping rules from integer counts.
 *
 * Conventions (all entry points):
 *   - Every call returns an ssa_status and never aborts the process.  On an
 *     error, ssa_last_error() gives a one-line message for the calling thread.
 *   - Pointers documented as "host" are plain host memory owned by the caller;
 *     the library copies what it needs before returning (except where noted).
 *     Pointers documented as "device" are CUDA device pointers on the current
 *     device.  Outputs are caller-allocated.
 *   - Graph, pool and solver objects are opaque and owned by the library; they
 *     live on the CUDA device that was current when they were created.
 *   - Node ids are int32 in [0, n); sample ids are int64.
 *   - Randomness is Philox4x32-10 keyed by (seed; purpose, stream, sample id,
 *     edge or node id), so every RR set is a pure function of its key and is
 *     independent of batch size, launch shape and traversal order:
 *       key     = (lo32(seed), hi32(seed))
 *       counter = (lo32(x), hi32(x), lo32(j), purpose<<28 | stream<<20 | (j>>32 & 0xFFFFF))
 *       purposes ROOT=1 (x=0), IC=2 (x=e>>2, output word e&3), LT=3 (x=v, word 0),
 *                SKIP=4 (x = v | (c>>1)<<32, words 2(c&1), 2(c&1)+1 as one 64-bit
 *                uniform U for gap c of v's in-list), WEIGHT=5 (x=e, j=0, stream=0)
 *     where j is the sample id, e the CSR position of an in-edge and v a node.
 *     IC under SSA_W_WC draws no per-edge coins: all d = d_in(v) >= 2
 *     in-edges of v have probability p = t/2^32 (t below), so the run G of
 *     dead edges before each live one is geometric, P(G >= g) = q^g, q = 1-p
 *     (the law of d independent coins).  In Q64 integers (products truncated
 *     to their high 64 bits): Q = (2^32 - t) << 32, P_0 = Q, P_(i+1) = P_i^2;
 *     G(U) tests bits J-1 .. 0 (J = bit length of d), setting bit i when
 *     U < A * P_i with A the product taken so far (P_i alone at the first).
 *     From pos = 0, gap c gives the live edge off[v] + pos + G, after which
 *     pos moves past it; the walk ends when G >= d - pos.  d = 1: the one
 *     edge is live without a draw.
 */
#ifndef SSA_H
#define SSA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SSA_OK = 0,
  SSA_E_ARG = 1,        /* bad argument (null pointer, out-of-range id or size) */
  SSA_E_NOMEM = 2,      /* device or host allocation failed */
  SSA_E_POOL_FULL = 3,  /* the RR pool would exceed its byte cap before a stop */
  SSA_E_CUDA = 4,       /* a CUDA runtime call failed */
  SSA_E_TIMEOUT = 5,    /* a bounded device wait gave up (kernel returned, context kept) */
  SSA_E_CANCELLED = 6,  /* serving: request cancelled */
  SSA_E_INTERNAL = 7,   /* internal invariant broken (a bug) */
  SSA_E_NOT_READY = 8   /* serving: result not ready yet */
} ssa_status;

typedef enum { SSA_IC = 0, SSA_LT = 1 } ssa_model;   /* Sec. 2.1 */
typedef enum { SSA_ALGO_SSA = 0, SSA_ALGO_DSSA = 1 } ssa_algo;

/* Edge weights w(u,v) (Sec. 2), held per in-edge as a uint32 threshold t:
 * the edge is live in a sample when its keyed 32-bit draw r satisfies r < t,
 * and t = 0xFFFFFFFF means probability exactly 1.
 *   SSA_W_WC          w = 1/d_in(v) (Sec. 6.1): t = floor(2^32/d_in), d_in=1 -> 0xFFFFFFFF
 *   SSA_W_TRIVALENCY  w drawn uniformly from {0.1, 0.01, 0.001} by the keyed
 *                     WEIGHT draw of the edge's CSR position: index floor(3 r / 2^32),
 *                     t = floor(2^32 w) = 429496729, 42949672, 4294967
 *   SSA_W_EXPLICIT    t given per input edge
 * LT (Sec. 2.1) in its live-edge form: each visited node keeps at most one
 * in-edge, chosen by its keyed LT draw r.  SSA_W_WC: the in-edge of index
 * floor(r d_in / 2^32) of its in-list (w = 1/d_in).  SSA_W_EXPLICIT: t_e are
 * the in-weights times 2^32 and must sum to at most 2^32 per node; the kept
 * edge is the first e of the in-list with r < t_1 + ... + t_e, none when r is
 * past the sum (probability 1 - sum of w).  SSA_W_TRIVALENCY is IC only. */
typedef enum { SSA_W_WC = 0, SSA_W_TRIVALENCY = 1, SSA_W_EXPLICIT = 2 } ssa_weighting;

typedef struct ssa_graph ssa_graph;
typedef struct ssa_pool ssa_pool;
typedef struct ssa_solver ssa_solver;

const char* ssa_status_str(ssa_status s);
/* Copies the calling thread's last error message (NUL-terminated, truncated
 * to len) into buf.  Returns SSA_OK. */
ssa_status ssa_last_error(char* buf, size_t len);
/* Library version string, e.g. "ssa-gb300 0.2 sm_103a". */
const char* ssa_version(void);
/* Architecture of the device code the CUDA runtime loaded for this library on
 * the current device, as major*10 + minor (103 for sm_103a SASS): *binary from
 * cudaFuncGetAttributes' binaryVersion, *ptx its ptxVersion.  Needs a GPU;
 * SSA_E_CUDA when no device code fits the device. */
ssa_status ssa_device_code_version(int32_t* binary, int32_t* ptx);

/* ------------------------------------------------------------------------ */
/* Graph store (Sec. 2: G = (V, E, w)).                                     */
/* ------------------------------------------------------------------------ */

/* Build the device-resident in-edge CSR of a directed graph.
 *   n, m        node and edge counts (1 <= n < 2^31, 0 <= m < 2^31)
 *   src, dst    host int32[m]: edge i is (src[i] -> dst[i]); any order;
 *               duplicates are parallel edges, self-loops are kept
 *   thr         host uint32[m] thresholds for SSA_W_EXPLICIT, else NULL
 *   weighting   see ssa_weighting
 *   weight_seed key of the trivalency draw
 *   out         receives the graph handle
 * Each node's in-list is ordered by (src, input position); that order fixes
 * the CSR position e that keys the IC coin of an edge.  The arrays are copied;
 * the caller keeps ownership.  Errors: SSA_E_ARG (ids out of range, null
 * arrays, LT-incompatible request), SSA_E_NOMEM, SSA_E_CUDA. */
ssa_status ssa_load_graph(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                          const uint32_t* thr, ssa_weighting weighting, uint64_t weight_seed,
                          ssa_graph** out);
/* Generate a directed R-MAT graph (Chakrabarti, Zhan, Faloutsos, SDM 2004) on
 * the device and build its CSR there: the synthetic stand-in for the paper's
 * networks (Sec. 6.1), without a host edge list or an upload.
 *   scale        n = 2^scale nodes, 1 <= scale <= 30
 *   m_draw       edges drawn, 0 <= m_draw < 2^31; self-loops and duplicate
 *                (src, dst) pairs are removed, ssa_graph_info reports the rest
 *   a, b, c      quadrant probabilities (d = 1 - a - b - c), each >= 0; each
 *                level takes a 32-bit draw u and compares it with
 *                floor(2^32 a), floor(2^32 (a+b)), floor(2^32 (a+b+c))
 *   seed         key of the draws: level l of draw i uses the low (l even) or
 *                high (l odd) half of SplitMix64 output number 32 i + l/2
 *                (Steele, Lea, Flood, OOPSLA 2014), most significant bit first;
 *                no noise and no id permutation
 *   weighting    SSA_W_WC or SSA_W_TRIVALENCY (weight_seed keys the latter)
 * The result equals ssa_load_graph of the same edge list.  Errors: SSA_E_ARG,
 * SSA_E_NOMEM (the sort needs about 16 bytes per draw), SSA_E_CUDA. */
ssa_status ssa_gen_rmat(int32_t scale, int64_t m_draw, double a, double b, double c, uint64_t seed,
                        ssa_weighting weighting, uint64_t weight_seed, ssa_graph** out);
ssa_status ssa_free_graph(ssa_graph* g);
/* n, m and device bytes held by the graph (any pointer may be NULL). */
ssa_status ssa_graph_info(const ssa_graph* g, int64_t* n, int64_t* m, int64_t* device_bytes);
/* Copy the CSR back to host arrays: off int64[n+1], src int32[m], thr uint32[m]
 * (any may be NULL). */
ssa_status ssa_graph_export(const ssa_graph* g, int64_t* off, int32_t* src, uint32_t* thr);

/* IC sampler tuning.  An RR set is built by one warp while it stays within
 * 512 nodes (shared-memory hash), then -- up to mid_cap nodes -- by one warp
 * with a global-memory hash, then by a whole CTA with an n-bit bitmap that
 * splits long in-lists over all its warps.  A warp that meets an in-list of
 * more than heavy_groups 4-edge groups hands its sample to the CTA tier.  The
 * best values depend on the graph (wide bimodal sets favour mid_cap 0; deep
 * chains favour 16384; hubs of millions of in-edges favour an early hand-over).
 * ssa_autotune times a pilot batch of pilot_samples sets (0 = 8192) under the
 * candidates (mid_cap, heavy_groups) in {0, 16384} x {4096, never}, after one
 * untimed pass that sizes the pilot pool, and keeps the fastest in the graph
 * handle; an IC solve on an untuned graph first tunes it on 4096 sets (65536
 * under SSA_W_WC, whose large sets are rare).  Under SSA_W_WC the in-lists are
 * walked by gaps and none is heavy: where the global-bitmap warp tier of
 * ssa_set_warp_tier exists it is chosen without a pilot (*pilot_ms = 0),
 * else the candidates are mid_cap in {0, 16384}.
 * ssa_set_tuning fixes both by hand (0 <= mid_cap <= 16384, heavy_groups >= 1;
 * 0x7FFFFFFF = never hand over).  Results never depend on the tuning.  For
 * SSA_LT ssa_autotune has nothing to tune. */
ssa_status ssa_autotune(const ssa_graph* g, ssa_model model, int64_t pilot_samples, int32_t* mid_cap,
                        double* pilot_ms);
ssa_status ssa_set_tuning(const ssa_graph* g, int32_t mid_cap, int32_t heavy_groups);
/* Queue capacity of the CTA tier's first stage when the n-bit visited bitmap
 * lives in global memory (n/8 above 192 KB): 128-thread CTAs keep sets of up to
 * small_queue nodes, and full-size CTAs redo larger sets.  0 restores the
 * default min(n, 2^20).  Applies to sampler scratch created afterwards (new
 * pools and solvers); results never depend on it.  SSA_E_ARG if negative. */
ssa_status ssa_set_queue_tuning(const ssa_graph* g, int32_t small_queue);
/* Weighted-cascade IC on graphs whose n-bit bitmap does not fit shared memory
 * (n/8 above 192 KB): with global_bitmap = 1 every sample is built by one warp
 * whose visited set is its own n-bit bitmap in global memory and whose queue
 * holds up to 2^16 nodes (up to mid_cap of ssa_set_tuning when that is
 * nonzero); larger sets go to the CTA tier.  0 (the default)
 * keeps the hash warp tiers of ssa_set_tuning.  ssa_autotune times this tier
 * where it exists.  Results never depend on it. */
ssa_status ssa_set_warp_tier(const ssa_graph* g, int32_t global_bitmap);
/* Weighted-cascade IC: with on = 1 (the default) a lane tier runs before the
 * warp tiers, one sample per lane with its queue of up to 32 nodes in
 * thread-local memory; larger sets are redone by the warp tiers.  0
 * sends every sample to the warp tiers.  Applies to sampling started after
 * the call; results never depend on it. */
ssa_status ssa_set_lane_tier(const ssa_graph* g, int32_t on);

/* Process-wide choice of the greedy kernel's launch shape (results never
 * depend on it): 0 (default) uses one thread-block cluster of 16 (or 8) blocks,
 * synchronised by the hardware cluster barrier, for solvers marked shared
 * (ssa_solver_set_shared) on pools of at most 2^26 entries, and a cooperative
 * grid of one block per SM otherwise; 1 always uses the cooperative grid; 2
 * always a cluster.  Applies to launches after the call.  SSA_E_ARG for other
 * values. */
ssa_status ssa_set_greedy_mode(int32_t mode);

/* Process-wide bound on the polls of each device-side wait: the grid barriers
 * of the greedy kernel (ssa_max_coverage and every solve).  A wait that reaches
 * it gives up, its kernel returns, and the call reports SSA_E_TIMEOUT.  polls
 * >= 1 sets the bound (each poll backs off up to 128 ns); 0 restores the
 * default of 2^22 polls, about a second.  Meant for failure handling and its
 * tests: a small bound makes ordinary barriers give up.  Applies to launches
 * after the call; SSA_E_ARG for polls < 0. */
ssa_status ssa_set_wait_polls(int64_t polls);

/* ------------------------------------------------------------------------ */
/* Solve (Definition 1: IM; Algorithm 1 SSA; Algorithm 4 D-SSA).            */
/* ------------------------------------------------------------------------ */

typedef struct {
  ssa_algo algo;
  ssa_model model;
  int32_t k;                 /* 1 <= k <= n */
  double eps;                /* 0 < eps < 1 - 1/e */
  double delta;              /* 0 < delta < 1 (the paper's experiments use 1/n) */
  uint64_t seed;             /* Philox key */
  const uint32_t* benefit;   /* host uint32[n] WRIS benefits (Sec. 6.3.1), or NULL for
                                uniform sources; copied during the call */
  int64_t pool_bytes_cap;    /* RR-pool cap in bytes (0 = library default) */
} ssa_params;

/* One stop-and-stare round. */
typedef struct {
  int32_t t;                 /* round number, from 1 */
  int32_t stop;              /* 1 on the round that returned */
  int64_t n_sets;            /* |R_t| = ceil(Lambda) * 2^(t-1) */
  int64_t cov;               /* Cov_{R_t}(S_t) from Max-Coverage */
  int64_t check_cov;         /* D-SSA: Cov_{R^c_t}(S_t); SSA: Estimate-Inf successes; -1 if not run */
  int64_t check_T;           /* SSA: Estimate-Inf T (0: T_max reached or not run) */
  double stat;               /* D-SSA: eps_t (-1 if D1 failed); SSA: I_c (-1 if none) */
  double eps1, eps2, eps3;   /* D-SSA: the round's eps_1, eps_2, eps_3 of Algorithm 4 (-1 if D1
                                failed); SSA: the fixed eps_1, eps_2, eps_3 of Eq. "set_ep" */
} ssa_round;

/* Kernel classes timed with CUDA events when ssa_result.kstats is requested. */
enum {
  SSA_K_SAMPLE_WARP = 0,     /* RR sampler, warp-per-sample tier */
  SSA_K_SAMPLE_CTA = 1,      /* RR sampler, CTA-per-sample tier (large sets) */
  SSA_K_INDEX = 2,           /* node -> set index build (count, scan, scatter) */
  SSA_K_GREEDY = 3,          /* Max-Coverage argmax + cover steps */
  SSA_K_STARE = 4,           /* Cov over R^c_t, Estimate-Inf first-T search */
  SSA_K_COUNT = 5
};

typedef struct {
  int64_t launches;          /* kernel launches of this class */
  double ms;                 /* summed CUDA-event time of those launches */
} ssa_kstat;

typedef struct {
  int32_t* seeds;            /* in: host int32[k] buffer; out: the seed set S_k */
  ssa_round* trace;          /* in: host ssa_round[trace_cap] buffer or NULL */
  int32_t trace_cap;
  /* outputs */
  double influence;          /* scale * Cov_R(S)/|R| at the returned round; scale = n,
                                or the benefit total W for WRIS */
  int32_t rounds;
  int64_t n_rr;              /* RR sets generated (Estimate-Inf included) */
  int64_t pool_entries;      /* RR-pool entries stored (sum of |R_j|) */
  int64_t edge_visits;       /* in-edges examined (IC) / in-neighbour picks (LT) */
  int64_t node_visits;       /* nodes added to RR sets (Estimate-Inf included) */
  int64_t cta_sets;          /* RR sets finished by the CTA-per-sample sampler tier */
  int64_t cta_edge_visits;   /* that tier's share of edge_visits */
  int64_t cta_node_visits;   /* that tier's share of node_visits */
  int64_t cta_stored_entries; /* pool entries that tier wrote (hit-test sets store none) */
  int64_t cta_stored_sets;   /* sets that tier wrote to the pool */
  int64_t draws;             /* Philox draws: IC 4-edge groups that needed coins, LT picks */
  int64_t cta_draws;         /* the CTA tier's share of draws */
  int32_t mid_cap;           /* IC sampler hand-over size used (see ssa_autotune) */
  int32_t heavy_groups;      /* IC: in-list length (4-edge groups) above which warp tiers hand over */
  int64_t kernel_launches;   /* CUDA kernels this library launched for the solve */
  double seconds;            /* host wall time of the call */
  int32_t want_kstats;       /* in: 1 to time kernel classes with CUDA events */
  ssa_kstat kstats[SSA_K_COUNT];
} ssa_result;

/* One-shot solve: creates a solver, runs, frees it.  Errors: SSA_E_ARG,
 * SSA_E_NOMEM, SSA_E_POOL_FULL, SSA_E_CUDA, SSA_E_TIMEOUT. */
ssa_status ssa_solve(const ssa_graph* g, const ssa_params* p, ssa_result* out);

/* A solver keeps device workspaces (sampler scratch per model, index and
 * greedy buffers) and a CUDA stream across solves on one graph; each solve's
 * RR pool and index return to the device's memory pool when it ends.  stream: a cudaStream_t to run on, or NULL for a
 * library-created one.  pool_bytes_cap: cap for the RR pool (0 = 60% of the
 * device memory free at creation). */
ssa_status ssa_solver_create(const ssa_graph* g, void* stream, int64_t pool_bytes_cap, ssa_solver** out);
ssa_status ssa_solver_solve(ssa_solver* s, const ssa_params* p, ssa_result* out);
/* Run each round's device work after sampling -- the index of the new sets,
 * Max-Coverage and, for D-SSA, the hit-tested stare count over R^c_t
 * (Algorithms 2 and 4) -- as one CUDA graph instead of separate launches and
 * host waits (on = 1; 0 = separate launches, the default).  The graph of
 * round t is captured on the solver's stream and patched into the executable
 * the solver keeps for round t, so later solves with the same shape reuse it.
 * Results do not depend on this setting.  Solves that time kernel classes
 * (ssa_result.want_kstats) launch separately. */
ssa_status ssa_solver_set_graphs(ssa_solver* s, int32_t on);
/* Mark the solver as sharing the GPU with concurrent solves (on = 1; the
 * server sets it for its slots).  Its Max-Coverage over pools of up to 2^26
 * entries then runs in one thread-block cluster of 16 SMs, leaving the rest of
 * the GPU to the other solves, instead of a cooperative grid of one block per
 * SM, which is faster for a solve alone on the GPU (the default, 0).  Results
 * do not depend on this setting (see also ssa_set_greedy_mode). */
ssa_status ssa_solver_set_shared(ssa_solver* s, int32_t on);
ssa_status ssa_solver_free(ssa_solver* s);

/* ------------------------------------------------------------------------ */
/* Hot-path steps, one entry point each (parity tests call these).          */
/* ------------------------------------------------------------------------ */

/* An RR pool: the RR sets of samples [0, count) of one (model, seed, stream)
 * (Definition 2), stored on the device as flat (node, sample) entries.
 * benefit: host uint32[n] WRIS weights or NULL (copied).  */
ssa_status ssa_pool_create(const ssa_graph* g, ssa_model model, uint64_t seed, uint32_t stream,
                           const uint32_t* benefit, ssa_pool** out);
ssa_status ssa_pool_free(ssa_pool* p);
/* Sample until the pool holds `count` sets (new samples [old count, count)). */
ssa_status ssa_pool_grow(ssa_pool* p, int64_t count);
ssa_status ssa_pool_info(const ssa_pool* p, int64_t* count, int64_t* entries, int64_t* edge_visits);
/* Copy sets [first, first+count) to host: off int64[count+1] (off[0] = 0),
 * nodes int32[cap].  Nodes of one set come in traversal order (not sorted).
 * SSA_E_ARG if cap is too small (off is still filled). */
ssa_status ssa_pool_export(const ssa_pool* p, int64_t first, int64_t count, int64_t* off,
                           int32_t* nodes, int64_t cap);
/* Node -> set index over sets [0, N): cnt int32[n] (host) = #sets holding v. */
ssa_status ssa_pool_counts(ssa_pool* p, int64_t N, int32_t* cnt);
/* Max-Coverage (Algorithm 2) over sets [0, N): k picks of largest marginal
 * gain, ties to the smallest id, seeds never re-picked.  seeds int32[k],
 * gains int64[k] (host); *cov = Cov_R(S).  1 <= k <= n; N <= 2^31 - 2
 * (SSA_E_ARG beyond).  All k picks run in one cooperative kernel; a wait at
 * its grid barriers gives up after a bounded number of polls (about a second
 * by default, see ssa_set_wait_polls): every block then returns and the call
 * reports SSA_E_TIMEOUT, leaving the CUDA context usable. */
ssa_status ssa_max_coverage(ssa_pool* p, int64_t N, int32_t k, int32_t* seeds, int64_t* gains,
                            int64_t* cov);
/* Cov (Eq. 1) of the host seed list over sets [first, first+count). */
ssa_status ssa_coverage(ssa_pool* p, int64_t first, int64_t count, const int32_t* seeds, int32_t k,
                        int64_t* cov);
/* Estimate-Inf (Algorithm 3): RR sets j = 0, 1, ... of `stream`, first T with
 * #{j < T : R_j meets S} >= lambda2, T <= t_max.  *T = 0 when t_max sets do
 * not reach it (the paper's -1); *hits = successes counted up to T (or t_max). */
ssa_status ssa_estimate_inf(const ssa_graph* g, ssa_model model, uint64_t seed, uint32_t stream,
                            const uint32_t* benefit, const int32_t* seeds, int32_t k, double lambda2,
                            int64_t t_max, int64_t* T, int64_t* hits);

/* ------------------------------------------------------------------------ */
/* Serving: continuous admission of queries against resident graphs.       */
/* (The paper solves one query per run; its Sec. 6.3 TVM queries are WRIS   */
/* solves, which ssa_params.benefit expresses.)                             */
/* ------------------------------------------------------------------------ */

typedef struct ssa_server ssa_server;

typedef struct {
  int64_t submitted, completed, failed, active, pending;
  int64_t bytes_budget;      /* RR-pool byte budget shared by admitted requests */
  int64_t bytes_in_use;      /* reserved by the requests now running */
  double p50_ms, p99_ms;     /* submit-to-done latency of completed requests */
} ssa_serve_stats;

/* Start a server over n_graphs resident graphs (the handles must outlive the
 * server) with `slots` worker slots (1..64), each with its own CUDA stream.
 * pool_bytes: RR-pool budget shared by running requests (0 = 60% of free
 * device memory).  A request is admitted FIFO when a slot is free and its
 * estimated footprint (learned per graph, model and k range from finished
 * requests) fits the budget, or when nothing else runs. */
ssa_status ssa_server_create(const ssa_graph* const* graphs, int32_t n_graphs, int32_t slots, int64_t pool_bytes,
                             ssa_server** out);
/* Queue one solve (params and benefit array are copied).  *ticket names it. */
ssa_status ssa_server_submit(ssa_server* s, int32_t graph, const ssa_params* p, uint64_t* ticket);
/* If the request is done, copy its result (seeds: host int32[k]; out->trace
 * may point to a host ssa_round buffer of out->trace_cap entries) and its
 * submit-to-done latency in seconds, release the ticket and return its status;
 * otherwise SSA_E_NOT_READY. */
ssa_status ssa_server_poll(ssa_server* s, uint64_t ticket, int32_t* seeds, ssa_result* out, double* latency_s);
/* As poll, but block up to timeout_s seconds (SSA_E_TIMEOUT if still running). */
ssa_status ssa_server_wait(ssa_server* s, uint64_t ticket, double timeout_s, int32_t* seeds, ssa_result* out,
                           double* latency_s);
ssa_status ssa_server_stats(ssa_server* s, ssa_serve_stats* out);
/* Finish the running requests, cancel the queued ones (SSA_E_CANCELLED), join. */
ssa_status ssa_server_destroy(ssa_server* s);

/* ------------------------------------------------------------------------ */
/* Allocation-free coverage count (no counterpart in the paper).            */
/* ------------------------------------------------------------------------ */

/* Same count as ssa_coverage -- the number of RR sets with a sample id in
 * [first, first+count) that contain at least one seed -- over a flat RR pool
 * the caller holds in device memory, for callers that cannot allocate device
 * memory when they call: for example a serving loop that reserved all of its
 * device memory up front, or a host runtime whose own allocator owns the
 * device.  It calls no cudaMalloc/cudaFree or allocating library routine; its
 * scratch is one fixed 16 MiB device array inside the library, held on every
 * device that loads the library until the process exits.
 *   n        node count (node and seed ids lie in [0, n))
 *   nodes    device int32[entries]: node of each pool entry
 *   samp     device int32[entries]: sample id of each pool entry (entries of
 *            one sample need not be contiguous; other samples are ignored)
 *   seeds    device int32[k]
 *   cov      host out: the count
 *   stream   cudaStream_t to run on (NULL = the legacy default stream); the
 *            call synchronises that stream before returning.
 * Limit: n/32 + count/32 32-bit words plus a 256-byte header must fit the
 * 16 MiB array (n + count below about 134 million), else SSA_E_ARG.  Every call
 * looks up the array's device address on the current device
 * (cudaGetSymbolAddress) and is synchronous: it copies the count to the host
 * and synchronises `stream` before returning, so it must not be called while
 * that stream is being captured into a CUDA graph.  Every call shares the one
 * array and clears the part it uses; calls that overlap on the GPU (other
 * streams, other host threads) race on it and must be serialised by the
 * caller.  Errors: SSA_E_ARG (sizes, null pointers, ids outside [0, n): the
 * device checks every id and skips any outside), SSA_E_CUDA. */
ssa_status ssa_coverage_noalloc(int64_t n, const int32_t* nodes, const int32_t* samp, int64_t entries,
                                int64_t first, int64_t count, const int32_t* seeds, int32_t k,
                                int64_t* cov, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SSA_H */
