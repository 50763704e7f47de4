/*
 * ORACLE -- test infrastructure, not the product.
 *
 * A plain, slow, single-threaded CPU statement of the Stop-and-Stare hot path
 * (Nguyen, Thai, Dinh, "Stop-and-Stare: Optimal Sampling Algorithms for Viral
 * Marketing in Billion-scale Networks", arXiv 1605.07990).  Only the tests,
 * the package smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code with the CUDA path: the two sides agree only on the
 * documented keying contract and on the formulas of the paper.
 *
 * Parts and the passages they follow:
 *   - Philox4x32-10 counter-based generator: Salmon, Moraes, Dror, Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11 (Sec. 3.3).
 *   - graph G=(V,E,w) with w(u,v) in [0,1] (Sec. 2), weighted-cascade weights
 *     w(u,v)=1/d_in(v) (Sec. 6.1 "Parameter Settings"), held as uint32
 *     thresholds: an edge is live when a uniform 32-bit draw is below its
 *     threshold; 0xFFFFFFFF means probability exactly 1.
 *   - RR set (Definition 2): random source v, random sample graph g, the nodes
 *     that reach v in g.  IC (Sec. 2.1): each edge is live independently with
 *     probability w; under weighted-cascade weights the live in-edges of a
 *     node are drawn as geometric gaps (the same law; see "gap form" below).
 *     LT (Sec. 2.1) in its live-edge form: each node keeps at most one
 *     in-edge, (u,v) with probability w(u,v).
 *   - WRIS (Sec. 6.3.1): the source is drawn proportionally to node benefit.
 *   - Cov_R(S) (Eq. 1); Max-Coverage (Algorithm 2); Estimate-Inf
 *     (Algorithm 3); SSA (Algorithm 1, default parameters Eq. "set_ep");
 *     D-SSA (Algorithm 4); Upsilon (Table 1).
 *
 * Parity pins: see the header of each function.  The stopping rules are
 * pinned round by round (tests/test_oracle_stop_rules.py): closed forms on an
 * out-star whose every RR set holds the centre, the scale-free forms of
 * Algorithm 4's eps_1, eps_2, eps_3, eps_t against Eq. "epsilon", and SSA's C2
 * as a ratio of trace counts in cases where the choice of eps decides the
 * round.  The exact round count on a random graph has no printed run in the
 * paper to pin against ("parity unpinned" for it); the final guarantee
 * (1-1/e-eps)*OPT is checked statistically on tiny graphs.
 *
 * Floating point: every FP64 decision is evaluated in the written order with
 * libm's log, sqrt, lgamma, ceil; build with -ffp-contract=off.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11): 10 rounds of the 4x32 Philox S-box; the key is    */
/* bumped by the Weyl constants between rounds.                              */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
    uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Keying contract (shared with the CUDA side as a written rule, not code):
 *   key     = (lo32(seed), hi32(seed))
 *   counter = (lo32(x), hi32(x), lo32(j), purpose<<28 | stream<<20 | (j>>32 & 0xFFFFF))
 * purposes: ROOT=1 (x=0), IC=2 (x=e>>2, word e&3), LT=3 (x=v, word 0),
 *           SKIP=4 (x = v | (c>>1)<<32, words 2(c&1), 2(c&1)+1 as one 64-bit
 *           uniform for gap c of node v's in-list), WEIGHT=5 (x=e, j=0, stream=0). */
enum { P_ROOT = 1, P_IC = 2, P_LT = 3, P_SKIP = 4, P_WEIGHT = 5 };

static void keyed(uint64_t seed, uint32_t purpose, uint32_t stream, uint64_t j, uint64_t x,
                  uint32_t out[4]) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {(uint32_t)x, (uint32_t)(x >> 32), (uint32_t)j,
                     (purpose << 28) | ((stream & 0xFFu) << 20) | (uint32_t)((j >> 32) & 0xFFFFFu)};
  orc_philox4x32_10(ctr, key, out);
}

/* uniform integer in [0, range) from a 32-bit draw: high word of r*range */
static uint32_t mulhi32(uint32_t r, uint32_t range) {
  return (uint32_t)(((uint64_t)r * (uint64_t)range) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Graph: in-edge CSR, edges of each node ordered by (src, input position).  */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t n, m;
  int64_t* off;  /* n+1 */
  int32_t* src;  /* m: tail u of in-edge (u,v) */
  uint32_t* thr; /* m: live iff draw < thr, or thr == 0xFFFFFFFF */
  int weighting; /* W_WC, W_TRIVALENCY or W_EXPLICIT */
} orc_graph;

enum { W_WC = 0, W_TRIVALENCY = 1, W_EXPLICIT = 2 };

/* thresholds of p in {0.1, 0.01, 0.001}: floor(2^32 * p) */
static const uint32_t TRIVALENCY_THR[3] = {429496729u, 42949672u, 4294967u};

void orc_graph_free(orc_graph* g) {
  if (!g) return;
  free(g->off); free(g->src); free(g->thr); free(g);
}

/* Returns NULL on a bad argument.  The CSR order (dst, src, input position)
 * is built by two stable counting sorts: first by src, then by dst. */
orc_graph* orc_graph_build(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                           int weighting, const uint32_t* thr_in, uint64_t weight_seed) {
  if (n <= 0 || m < 0 || n > 0x7FFFFFFF) return NULL;
  for (int64_t i = 0; i < m; ++i)
    if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) return NULL;
  if (weighting == W_EXPLICIT && m > 0 && !thr_in) return NULL;
  orc_graph* g = (orc_graph*)calloc(1, sizeof(orc_graph));
  g->n = n; g->m = m; g->weighting = weighting;
  g->off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  g->src = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
  g->thr = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m ? m : 1));
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t* by_src = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m ? m : 1));
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m ? m : 1));
  /* stable counting sort of input positions by src */
  for (int64_t i = 0; i < m; ++i) cnt[src[i] + 1]++;
  for (int64_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
  for (int64_t i = 0; i < m; ++i) by_src[cnt[src[i]]++] = i;
  /* stable counting sort of that sequence by dst */
  for (int64_t i = 0; i < m; ++i) g->off[dst[i] + 1]++;
  for (int64_t v = 0; v < n; ++v) g->off[v + 1] += g->off[v];
  memcpy(cnt, g->off, sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t q = 0; q < m; ++q) {
    int64_t i = by_src[q];
    order[cnt[dst[i]]++] = i;
  }
  for (int64_t e = 0; e < m; ++e) g->src[e] = src[order[e]];
  for (int64_t v = 0; v < n; ++v) {
    int64_t d = g->off[v + 1] - g->off[v];
    for (int64_t e = g->off[v]; e < g->off[v + 1]; ++e) {
      uint32_t t;
      if (weighting == W_WC) {
        /* w = 1/d_in(v) as floor(2^32/d); d = 1 is probability 1 */
        t = (d == 1) ? 0xFFFFFFFFu : (uint32_t)((UINT64_C(1) << 32) / (uint64_t)d);
      } else if (weighting == W_TRIVALENCY) {
        uint32_t r[4];
        keyed(weight_seed, P_WEIGHT, 0, 0, (uint64_t)e, r);
        t = TRIVALENCY_THR[mulhi32(r[0], 3u)];
      } else {
        t = thr_in[order[e]];
      }
      g->thr[e] = t;
    }
  }
  free(cnt); free(by_src); free(order);
  return g;
}

const int64_t* orc_graph_off(const orc_graph* g) { return g->off; }
const int32_t* orc_graph_src(const orc_graph* g) { return g->src; }
const uint32_t* orc_graph_thr(const orc_graph* g) { return g->thr; }
int64_t orc_graph_n(const orc_graph* g) { return g->n; }
int64_t orc_graph_m(const orc_graph* g) { return g->m; }

/* ------------------------------------------------------------------------ */
/* Weighted cascade in gap form.  Under IC every in-edge of v is live on its  */
/* own coin; with weighted-cascade weights all d = d_in(v) >= 2 of them have   */
/* the same probability p = t/2^32, t = floor(2^32/d), so the live edges of    */
/* v's in-list can be found by drawing the run G of dead edges before each     */
/* live one: P(G >= g) = q^g with q = 1 - p (a geometric law).  That is the    */
/* same law as d independent coins, at a cost in the number of live edges      */
/* rather than in d.  (d = 1: the one edge has probability 1, no draw.)        */
/*                                                                           */
/* Arithmetic, integers only so that every platform gets the same gaps:       */
/*   numbers in [0,1) are Q64 (x -> floor(x 2^64)), products truncate:         */
/*   mulq(a,b) = floor(a b / 2^64);  q = (2^32 - t) << 32 exactly;             */
/*   P_0 = q, P_(i+1) = mulq(P_i, P_i)  (q^(2^i));  J = bit length of d;        */
/*   G(U) = the g in [0, 2^J) found by testing bits J-1 .. 0 in turn: bit i   */
/*   is set when U < mulq(A, P_i), A the product taken so far (P_i itself     */
/*   at the first set bit), which then becomes A.                              */
/* G(U) is the largest g with U < q^g, up to the truncation (relative error   */
/* below 2^-50 at every threshold; pinned against exact powers in the tests). */
/* The walk: pos = 0, gap c = 0, 1, ...: G = G(U_c); stop when G >= d - pos;  */
/* else edge off[v] + pos + G is live and pos moves past it.                   */
/* ------------------------------------------------------------------------ */
static uint64_t mulq(uint64_t a, uint64_t b) {
  return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
}

uint32_t orc_wc_gap(int64_t d, uint64_t U) {
  if (d < 2 || d > 0x7FFFFFFF) return 0;
  uint32_t t = (uint32_t)((UINT64_C(1) << 32) / (uint64_t)d);
  uint64_t q = ((UINT64_C(1) << 32) - t) << 32;
  int J = 0;
  while ((INT64_C(1) << J) <= d) ++J;  /* 2^J > d */
  uint64_t P[32];
  P[0] = q;
  for (int i = 1; i < J; ++i) P[i] = mulq(P[i - 1], P[i - 1]);
  uint64_t A = 0;
  int first = 1;
  uint32_t g = 0;
  for (int i = J - 1; i >= 0; --i) {
    uint64_t cand = first ? P[i] : mulq(A, P[i]);
    if (U < cand) { A = cand; first = 0; g |= UINT32_C(1) << i; }
  }
  return g;
}

/* the 64-bit uniform of gap c of node v in sample j */
static uint64_t skip_uniform(uint64_t seed, uint32_t stream, uint64_t j, int32_t v, uint64_t c) {
  uint32_t r[4];
  keyed(seed, P_SKIP, stream, j, (uint64_t)(uint32_t)v | ((c >> 1) << 32), r);
  unsigned w = 2u * (unsigned)(c & 1u);
  return (uint64_t)r[w] | ((uint64_t)r[w + 1] << 32);
}

/* ------------------------------------------------------------------------ */
/* RR sets (Definition 2).                                                   */
/* ------------------------------------------------------------------------ */
enum { MODEL_IC = 0, MODEL_LT = 1 };

typedef struct {
  const orc_graph* g;
  int model;
  uint64_t seed;
  const uint64_t* benefit_prefix; /* NULL: uniform source; else n+1 prefix sums */
  uint8_t* visited;               /* n bytes, all zero between calls */
  int32_t* queue;                 /* n */
  int64_t edge_visits;            /* in-edges examined (statistics) */
} orc_sampler;

static orc_sampler* sampler_new(const orc_graph* g, int model, uint64_t seed, const uint64_t* bprefix) {
  orc_sampler* s = (orc_sampler*)calloc(1, sizeof(orc_sampler));
  s->g = g; s->model = model; s->seed = seed; s->benefit_prefix = bprefix;
  s->visited = (uint8_t*)calloc((size_t)g->n, 1);
  s->queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)g->n);
  return s;
}
static void sampler_free(orc_sampler* s) {
  if (!s) return;
  free(s->visited); free(s->queue); free(s);
}

/* Source of sample j of `stream`: uniform over V, or (WRIS) the node whose
 * benefit interval [prefix[v], prefix[v+1]) holds a uniform 64-bit target. */
static int32_t rr_source(const orc_sampler* s, uint32_t stream, uint64_t j) {
  uint32_t r[4];
  keyed(s->seed, P_ROOT, stream, j, 0, r);
  int64_t n = s->g->n;
  if (!s->benefit_prefix) return (int32_t)mulhi32(r[0], (uint32_t)n);
  uint64_t W = s->benefit_prefix[n];
  uint64_t r64 = (uint64_t)r[0] | ((uint64_t)r[1] << 32);
  uint64_t target = (uint64_t)(((unsigned __int128)r64 * W) >> 64);
  /* smallest v with prefix[v+1] > target */
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (s->benefit_prefix[mid + 1] > target) hi = mid; else lo = mid + 1;
  }
  return (int32_t)lo;
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* Writes RR set j of `stream` (ascending node ids) to out; returns its size. */
static int64_t rr_set(orc_sampler* s, uint32_t stream, uint64_t j, int32_t* out) {
  const orc_graph* g = s->g;
  int32_t root = rr_source(s, stream, j);
  int64_t size = 0;
  s->queue[size++] = root;
  s->visited[root] = 1;
  if (s->model == MODEL_IC && g->weighting == W_WC) {
    /* reverse BFS; the live in-edges of each node by the gap walk above */
    for (int64_t head = 0; head < size; ++head) {
      int32_t v = s->queue[head];
      int64_t lo = g->off[v], d = g->off[v + 1] - lo;
      s->edge_visits += d;
      int64_t pos = 0;
      for (uint64_t c = 0; pos < d; ++c) {
        int64_t e;
        if (d == 1) {
          e = lo;
          pos = 1;
        } else {
          uint32_t G = orc_wc_gap(d, skip_uniform(s->seed, stream, j, v, c));
          if ((int64_t)G >= d - pos) break;
          e = lo + pos + G;
          pos += (int64_t)G + 1;
        }
        if (!s->visited[g->src[e]]) {
          s->visited[g->src[e]] = 1;
          s->queue[size++] = g->src[e];
        }
      }
    }
  } else if (s->model == MODEL_IC) {
    /* reverse BFS over live in-edges: edge e is live in sample j iff its
     * keyed draw is below thr[e] */
    for (int64_t head = 0; head < size; ++head) {
      int32_t v = s->queue[head];
      for (int64_t e = g->off[v]; e < g->off[v + 1]; ++e) {
        uint32_t r[4];
        keyed(s->seed, P_IC, stream, j, (uint64_t)e >> 2, r);
        uint32_t coin = r[e & 3];
        int live = (g->thr[e] == 0xFFFFFFFFu) || (coin < g->thr[e]);
        s->edge_visits++;
        if (live && !s->visited[g->src[e]]) {
          s->visited[g->src[e]] = 1;
          s->queue[size++] = g->src[e];
        }
      }
    }
  } else {
    /* LT live-edge world: node v keeps at most one in-edge.  Weighted cascade
     * (w = 1/d_in): the edge of index floor(r*d_in/2^32), each with probability
     * 1/d_in.  General weights (explicit thresholds t_e = w * 2^32, sum <= 2^32):
     * the first in-edge e with r < t_1 + ... + t_e, none when r is past the
     * sum (probability 1 - sum of w).  The RR set follows kept edges backwards
     * from the source until a node with no kept edge or an already-seen node. */
    int32_t v = root;
    for (;;) {
      int64_t d = g->off[v + 1] - g->off[v];
      if (d == 0) break;
      uint32_t r[4];
      keyed(s->seed, P_LT, stream, j, (uint64_t)v, r);
      int64_t pick = -1;
      if (g->weighting == W_EXPLICIT) {
        uint64_t cum = 0;
        for (int64_t e = g->off[v]; e < g->off[v + 1]; ++e) {
          cum += g->thr[e];
          if ((uint64_t)r[0] < cum) { pick = e; break; }
        }
      } else {
        pick = g->off[v] + mulhi32(r[0], (uint32_t)d);
      }
      if (pick < 0) break;
      int32_t u = g->src[pick];
      s->edge_visits++;
      if (s->visited[u]) break;
      s->visited[u] = 1;
      s->queue[size++] = u;
      v = u;
    }
  }
  for (int64_t i = 0; i < size; ++i) s->visited[s->queue[i]] = 0;
  memcpy(out, s->queue, sizeof(int32_t) * (size_t)size);
  qsort(out, (size_t)size, sizeof(int32_t), cmp_i32);
  return size;
}

/* ------------------------------------------------------------------------ */
/* RR pool: sets of one stream in sample order.                              */
/* ------------------------------------------------------------------------ */
typedef struct {
  orc_sampler* smp;
  uint32_t stream;
  int64_t count;     /* sets held: samples [0, count) */
  int64_t cap_sets;
  int64_t* off;      /* count+1 */
  int64_t entries;
  int64_t cap_entries;
  int32_t* nodes;
} orc_pool;

orc_pool* orc_pool_new(const orc_graph* g, int model, uint64_t seed, uint32_t stream,
                       const uint64_t* benefit_prefix) {
  orc_pool* p = (orc_pool*)calloc(1, sizeof(orc_pool));
  p->smp = sampler_new(g, model, seed, benefit_prefix);
  p->stream = stream;
  p->cap_sets = 1024;
  p->off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(p->cap_sets + 1));
  p->off[0] = 0;
  p->cap_entries = 1 << 16;
  p->nodes = (int32_t*)malloc(sizeof(int32_t) * (size_t)p->cap_entries);
  return p;
}

void orc_pool_free(orc_pool* p) {
  if (!p) return;
  sampler_free(p->smp); free(p->off); free(p->nodes); free(p);
}

/* Generate samples until the pool holds `count` sets. */
void orc_pool_grow(orc_pool* p, int64_t count) {
  int64_t n = p->smp->g->n;
  while (p->count < count) {
    if (p->count + 1 > p->cap_sets) {
      p->cap_sets *= 2;
      p->off = (int64_t*)realloc(p->off, sizeof(int64_t) * (size_t)(p->cap_sets + 1));
    }
    if (p->entries + n > p->cap_entries) {
      while (p->entries + n > p->cap_entries) p->cap_entries *= 2;
      p->nodes = (int32_t*)realloc(p->nodes, sizeof(int32_t) * (size_t)p->cap_entries);
    }
    int64_t sz = rr_set(p->smp, p->stream, (uint64_t)p->count, p->nodes + p->entries);
    p->entries += sz;
    p->count++;
    p->off[p->count] = p->entries;
  }
}

int64_t orc_pool_count(const orc_pool* p) { return p->count; }
int64_t orc_pool_entries(const orc_pool* p) { return p->entries; }
const int64_t* orc_pool_off(const orc_pool* p) { return p->off; }
const int32_t* orc_pool_nodes(const orc_pool* p) { return p->nodes; }
int64_t orc_pool_edge_visits(const orc_pool* p) { return p->smp->edge_visits; }

/* Single RR set (for sampled parity at sizes where a full pool is too big). */
int64_t orc_rr_set(const orc_graph* g, int model, uint64_t seed, uint32_t stream, uint64_t j,
                   const uint64_t* benefit_prefix, int32_t* out) {
  orc_sampler* s = sampler_new(g, model, seed, benefit_prefix);
  int64_t sz = rr_set(s, stream, j, out);
  sampler_free(s);
  return sz;
}

/* ------------------------------------------------------------------------ */
/* The sampling phase over several host threads (the all-cores CPU           */
/* baseline): samples [j0, j0+count) are split into contiguous ranges, one    */
/* per thread, and each thread runs its own single-threaded sampler (the      */
/* code above) over its range.  Sets are counted, not stored.  The RR sets    */
/* are the same as one thread's: each is a function of its key alone.         */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_graph* g;
  int model;
  uint64_t seed;
  uint32_t stream;
  const uint64_t* bprefix;
  uint64_t j0, j1;
  int64_t entries, edge_visits;
} orc_range_job;

static void* sample_range(void* arg) {
  orc_range_job* a = (orc_range_job*)arg;
  orc_sampler* s = sampler_new(a->g, a->model, a->seed, a->bprefix);
  int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * (size_t)a->g->n);
  for (uint64_t j = a->j0; j < a->j1; ++j) a->entries += rr_set(s, a->stream, j, buf);
  a->edge_visits = s->edge_visits;
  free(buf);
  sampler_free(s);
  return NULL;
}

/* Returns the number of threads used (1..threads), or -1 on a bad argument. */
int orc_sample_threads(const orc_graph* g, int model, uint64_t seed, uint32_t stream,
                       const uint64_t* benefit_prefix, uint64_t j0, int64_t count, int threads,
                       int64_t* entries, int64_t* edge_visits) {
  if (count < 0 || threads < 1) return -1;
  if (threads > count && count > 0) threads = (int)count;
  orc_range_job* jobs = (orc_range_job*)calloc((size_t)threads, sizeof(orc_range_job));
  pthread_t* tid = (pthread_t*)calloc((size_t)threads, sizeof(pthread_t));
  int started = 0;
  for (int t = 0; t < threads; ++t) {
    jobs[t].g = g; jobs[t].model = model; jobs[t].seed = seed; jobs[t].stream = stream;
    jobs[t].bprefix = benefit_prefix;
    jobs[t].j0 = j0 + (uint64_t)(count * t / threads);
    jobs[t].j1 = j0 + (uint64_t)(count * (t + 1) / threads);
    if (pthread_create(&tid[t], NULL, sample_range, &jobs[t]) != 0) break;
    ++started;
  }
  /* a range whose thread could not start runs here */
  for (int t = started; t < threads; ++t) sample_range(&jobs[t]);
  int64_t e = 0, v = 0;
  for (int t = 0; t < threads; ++t) {
    if (t < started) pthread_join(tid[t], NULL);
    e += jobs[t].entries; v += jobs[t].edge_visits;
  }
  if (entries) *entries = e;
  if (edge_visits) *edge_visits = v;
  free(jobs); free(tid);
  return started > 0 ? started : 1;
}

/* ------------------------------------------------------------------------ */
/* Cov_R(S) (Eq. 1) over sets [a, b) of a pool.                              */
/* ------------------------------------------------------------------------ */
int64_t orc_coverage(const orc_pool* p, int64_t a, int64_t b, const int32_t* S, int k) {
  int64_t n = p->smp->g->n;
  uint8_t* in_s = (uint8_t*)calloc((size_t)n, 1);
  for (int i = 0; i < k; ++i) in_s[S[i]] = 1;
  int64_t cov = 0;
  for (int64_t j = a; j < b; ++j) {
    int hit = 0;
    for (int64_t q = p->off[j]; q < p->off[j + 1]; ++q) hit |= in_s[p->nodes[q]];
    cov += hit; /* min(|S n R_j|, 1) */
  }
  free(in_s);
  return cov;
}

/* ------------------------------------------------------------------------ */
/* Max-Coverage (Algorithm 2) over sets [0, N): k times, add the node of     */
/* largest marginal gain Cov(S+v) - Cov(S) = number of not-yet-covered sets  */
/* holding v; ties go to the smallest node id; nodes already in S are never  */
/* re-picked (gain-0 picks allowed, so k distinct seeds when n >= k).        */
/* gains[i] is the gain of the i-th pick; returns Cov_R(S) = sum of gains.   */
/* ------------------------------------------------------------------------ */
int64_t orc_max_coverage_sets(int64_t n, int64_t N, const int64_t* off, const int32_t* nodes, int k,
                              int32_t* seeds, int64_t* gains) {
  int64_t P = off[N];
  int64_t* cnt = (int64_t*)calloc((size_t)n, sizeof(int64_t));
  int64_t* inv_off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t* inv = (int64_t*)malloc(sizeof(int64_t) * (size_t)(P ? P : 1));
  uint8_t* covered = (uint8_t*)calloc((size_t)(N ? N : 1), 1);
  uint8_t* in_s = (uint8_t*)calloc((size_t)n, 1);
  /* cnt[v] = #sets holding v; inverted lists node -> sets */
  for (int64_t q = 0; q < P; ++q) cnt[nodes[q]]++;
  for (int64_t v = 0; v < n; ++v) inv_off[v + 1] = inv_off[v] + cnt[v];
  int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
  memcpy(cur, inv_off, sizeof(int64_t) * (size_t)n);
  for (int64_t j = 0; j < N; ++j)
    for (int64_t q = off[j]; q < off[j + 1]; ++q) inv[cur[nodes[q]]++] = j;
  free(cur);
  int64_t cov = 0;
  for (int i = 0; i < k; ++i) {
    int64_t best = -1;
    for (int64_t v = 0; v < n; ++v)
      if (!in_s[v] && (best < 0 || cnt[v] > cnt[best])) best = v;
    if (best < 0) { seeds[i] = -1; gains[i] = 0; continue; }
    seeds[i] = (int32_t)best;
    gains[i] = cnt[best];
    cov += cnt[best];
    in_s[best] = 1;
    for (int64_t q = inv_off[best]; q < inv_off[best + 1]; ++q) {
      int64_t j = inv[q];
      if (covered[j]) continue;
      covered[j] = 1;
      for (int64_t r = off[j]; r < off[j + 1]; ++r) cnt[nodes[r]]--;
    }
  }
  free(cnt); free(inv_off); free(inv); free(covered); free(in_s);
  return cov;
}

int64_t orc_max_coverage(const orc_pool* p, int64_t N, int k, int32_t* seeds, int64_t* gains) {
  return orc_max_coverage_sets(p->smp->g->n, N, p->off, p->nodes, k, seeds, gains);
}

/* Node-occurrence counts over sets [0, N) (parity of the index build). */
void orc_counts(const orc_pool* p, int64_t N, int64_t* cnt) {
  int64_t n = p->smp->g->n;
  memset(cnt, 0, sizeof(int64_t) * (size_t)n);
  for (int64_t q = 0; q < p->off[N]; ++q) cnt[p->nodes[q]]++;
}

/* ------------------------------------------------------------------------ */
/* Estimate-Inf (Algorithm 3): fresh RR sets j = 0, 1, ... of `stream`;      */
/* returns the first T with #{j < T : R_j hit by S} >= Lambda2, or 0 when    */
/* T_max sets do not reach it (the paper's "-1").  *hits = successes seen.   */
/* ------------------------------------------------------------------------ */
int64_t orc_estimate_inf(const orc_graph* g, int model, uint64_t seed, uint32_t stream,
                         const uint64_t* benefit_prefix, const int32_t* S, int k,
                         double lambda2, int64_t t_max, int64_t* hits_out, int64_t* edge_visits) {
  orc_sampler* s = sampler_new(g, model, seed, benefit_prefix);
  uint8_t* in_s = (uint8_t*)calloc((size_t)g->n, 1);
  int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * (size_t)g->n);
  for (int i = 0; i < k; ++i) in_s[S[i]] = 1;
  int64_t cov = 0, found = 0;
  for (int64_t T = 1; T <= t_max; ++T) {
    int64_t sz = rr_set(s, stream, (uint64_t)(T - 1), buf);
    int hit = 0;
    for (int64_t q = 0; q < sz; ++q) hit |= in_s[buf[q]];
    cov += hit;
    if ((double)cov >= lambda2) { found = T; break; }
  }
  if (hits_out) *hits_out = cov;
  if (edge_visits) *edge_visits += s->edge_visits;
  free(in_s); free(buf); sampler_free(s);
  return found;
}

/* ------------------------------------------------------------------------ */
/* Parameters (Table 1, Algorithm 1 lines 1-3, Algorithm 4 lines 1-3).       */
/* Upsilon(eps, delta) = (2 + 2 eps/3) ln(1/delta) / eps^2 is evaluated from */
/* L = ln(1/delta) so that the tiny delta/(6 C(n,k)) of N_max never forms.   */
/* ------------------------------------------------------------------------ */
static const double ONE_MINUS_INV_E = 1.0 - 1.0 / 2.718281828459045;

double orc_upsilon(double eps, double ln_inv_delta) {
  return (2.0 + 2.0 * eps / 3.0) * ln_inv_delta / (eps * eps);
}

typedef struct {
  double n_max;    /* N_max */
  int32_t i_max;   /* i_max (SSA) = t_max (D-SSA) */
  double lambda;   /* Lambda = Upsilon(eps, delta/(3 i_max)) */
  double lambda1;  /* SSA: (1+e1)(1+e2) Upsilon(e3, delta/(3 i_max)); D-SSA: 1 + (1+eps) Lambda */
  double lambda2;  /* SSA Estimate-Inf: 1 + (1+e2) Upsilon(e2, delta/(3 i_max)) */
  double eps1, eps2, eps3; /* SSA defaults, Eq. set_ep */
} orc_params;

void orc_params_compute(int64_t n, int k, double eps, double delta, int dssa, orc_params* P) {
  double lnC = lgamma((double)n + 1.0) - lgamma((double)k + 1.0) - lgamma((double)(n - k) + 1.0);
  P->n_max = 8.0 * ONE_MINUS_INV_E / (2.0 + 2.0 * eps / 3.0) *
             orc_upsilon(eps, log(6.0 / delta) + lnC) * (double)n / (double)k;
  P->i_max = (int32_t)ceil(log2(2.0 * P->n_max / orc_upsilon(eps, log(3.0 / delta))));
  if (P->i_max < 1) P->i_max = 1;
  double lnd = log(3.0 * (double)P->i_max / delta);
  P->lambda = orc_upsilon(eps, lnd);
  /* Eq. set_ep: eps2 = eps3 = eps / (2 (1-1/e)); eps1 = (1 + eps/(2 (1-1/e-eps))) / (1+eps2) - 1 */
  P->eps2 = eps / (2.0 * ONE_MINUS_INV_E);
  P->eps3 = P->eps2;
  P->eps1 = (1.0 + eps / (2.0 * (ONE_MINUS_INV_E - eps))) / (1.0 + P->eps2) - 1.0;
  if (dssa) {
    P->lambda1 = 1.0 + (1.0 + eps) * P->lambda;
    P->lambda2 = 0.0;
  } else {
    P->lambda1 = (1.0 + P->eps1) * (1.0 + P->eps2) * orc_upsilon(P->eps3, lnd);
    P->lambda2 = 1.0 + (1.0 + P->eps2) * orc_upsilon(P->eps2, lnd);
  }
}

/* ------------------------------------------------------------------------ */
/* SSA (Algorithm 1) and D-SSA (Algorithm 4).                                */
/* Round t works on |R_t| = ceil(Lambda) * 2^(t-1) sets of stream 0.         */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t t;
  int32_t stop;          /* 1 if this round returned */
  int64_t n_sets;        /* |R_t| */
  int64_t cov;           /* Cov_{R_t}(S_t) from Max-Coverage */
  int64_t check_cov;     /* D-SSA: Cov_{R^c_t}(S_t); SSA: Estimate-Inf successes (-1: not run) */
  int64_t check_T;       /* SSA: Estimate-Inf T (0: T_max reached / not run) */
  double stat;           /* D-SSA: eps_t (or -1 when D1 failed); SSA: I_c (or -1) */
  double eps1, eps2, eps3; /* D-SSA: the round's eps_1, eps_2, eps_3 (Algorithm 4; -1 when D1
                              failed); SSA: the fixed eps_1, eps_2, eps_3 of Eq. set_ep */
} orc_round;

typedef struct {
  double influence;      /* scale * Cov_{R}(S) / |R| at the returned round */
  int32_t rounds;
  int64_t n_rr;          /* RR sets generated, Estimate-Inf included */
  int64_t pool_entries;  /* pool entries generated (sum of |R_j|) */
  int64_t edge_visits;   /* in-edges examined (IC) / in-neighbour picks (LT) */
} orc_result;

static uint64_t* benefit_prefix_new(int64_t n, const uint32_t* benefit) {
  if (!benefit) return NULL;
  uint64_t* pre = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n + 1));
  pre[0] = 0;
  for (int64_t v = 0; v < n; ++v) pre[v + 1] = pre[v] + benefit[v];
  return pre;
}

/* algo 0 = SSA, 1 = D-SSA.  trace: up to max_rounds records.  Returns the
 * number of rounds run, or -1 on a bad argument. */
int32_t orc_solve(const orc_graph* g, int algo, int model, int k, double eps, double delta,
                  uint64_t seed, const uint32_t* benefit, int32_t* seeds_out, orc_result* res,
                  orc_round* trace, int32_t max_rounds) {
  int64_t n = g->n;
  if (k < 1 || k > n || !(eps > 0.0 && eps < 1.0) || !(delta > 0.0 && delta < 1.0)) return -1;
  if (!(eps < ONE_MINUS_INV_E)) return -1; /* 1-1/e-eps appears in Eq. set_ep and eps_3 */
  orc_params P;
  orc_params_compute(n, k, eps, delta, algo == 1, &P);
  uint64_t* bpre = benefit_prefix_new(n, benefit);
  if (bpre && bpre[n] == 0) { free(bpre); return -1; }
  double scale = bpre ? (double)bpre[n] : (double)n;
  int64_t base = (int64_t)ceil(P.lambda);
  orc_pool* pool = orc_pool_new(g, model, seed, 0, bpre);
  int32_t* S = (int32_t*)malloc(sizeof(int32_t) * (size_t)k);
  int64_t* gains = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
  int64_t extra_rr = 0, extra_entries = 0, extra_visits = 0;
  double influence = 0.0;
  int32_t t = 0;
  for (;;) {
    t += 1;
    int64_t N = base << (t - 1);
    orc_round rec;
    memset(&rec, 0, sizeof(rec));
    rec.t = t; rec.n_sets = N; rec.check_cov = -1; rec.check_T = 0; rec.stat = -1.0;
    rec.eps1 = rec.eps2 = rec.eps3 = -1.0;
    int stop = 0;
    if (algo == 0) {
      rec.eps1 = P.eps1; rec.eps2 = P.eps2; rec.eps3 = P.eps3;
      orc_pool_grow(pool, N);
      int64_t cov = orc_max_coverage(pool, N, k, S, gains);
      rec.cov = cov;
      influence = (double)cov * scale / (double)N;
      if ((double)cov >= P.lambda1) { /* condition C1 */
        double d2 = P.eps3 * P.eps3 / (P.eps2 * P.eps2);
        int64_t t_max = (int64_t)ceil(2.0 * (double)N * (1.0 + P.eps2) / (1.0 - P.eps2) * d2);
        int64_t hits = 0;
        int64_t T = orc_estimate_inf(g, model, seed, (uint32_t)t, bpre, S, k, P.lambda2, t_max,
                                     &hits, &extra_visits);
        extra_rr += T ? T : t_max;
        rec.check_cov = hits; rec.check_T = T;
        if (T > 0) {
          double ic = scale * P.lambda2 / (double)T;
          rec.stat = ic;
          if ((double)cov * scale / (double)N <= (1.0 + P.eps1) * ic) stop = 1; /* condition C2 */
        }
      }
    } else {
      orc_pool_grow(pool, 2 * N);
      int64_t cov = orc_max_coverage(pool, N, k, S, gains);
      int64_t c = orc_coverage(pool, N, 2 * N, S, k);
      rec.cov = cov; rec.check_cov = c;
      influence = (double)cov * scale / (double)N;
      if ((double)c >= P.lambda1) { /* condition D1 */
        double ic = (double)c * scale / (double)N;
        double ih = (double)cov * scale / (double)N;
        double pw = (double)(INT64_C(1) << (t - 1));
        double e1 = ih / ic - 1.0;
        double e2 = eps * sqrt(scale * (1.0 + eps) / (pw * ic));
        double e3 = eps * sqrt(scale * (1.0 + eps) * (ONE_MINUS_INV_E - eps) / ((1.0 + eps / 3.0) * pw * ic));
        double et = (e1 + e2 + e1 * e2) * (ONE_MINUS_INV_E - eps) + ONE_MINUS_INV_E * e3;
        rec.stat = et;
        rec.eps1 = e1; rec.eps2 = e2; rec.eps3 = e3;
        if (et <= eps) stop = 1; /* condition D2 */
      }
    }
    if (!stop && ((double)N >= P.n_max || t >= P.i_max)) stop = 2; /* sample cap */
    rec.stop = stop ? 1 : 0;
    if (trace && t <= max_rounds) trace[t - 1] = rec;
    if (stop) break;
  }
  memcpy(seeds_out, S, sizeof(int32_t) * (size_t)k);
  res->influence = influence;
  res->rounds = t;
  res->n_rr = orc_pool_count(pool) + extra_rr;
  res->pool_entries = orc_pool_entries(pool) + extra_entries;
  res->edge_visits = orc_pool_edge_visits(pool) + extra_visits;
  orc_pool_free(pool);
  free(S); free(gains); free(bpre);
  return t;
}
