/*
 * Seeded synthetic inputs: directed R-MAT edge lists and Zipf benefit
 * weights.  This module holds none of the influence-maximisation method's
 * arithmetic (no CSR, no thresholds, no sampling); it only produces the
 * graphs and per-node weights that both the oracle and the CUDA path consume.
 *
 * Randomness: SplitMix64's output function (Steele, Lea, Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014) applied to a
 * counter, so every draw is a pure function of (seed, counter) and the output
 * does not depend on the thread count.
 *
 * R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): each edge descends `scale`
 * levels of the adjacency matrix; at every level one uniform 32-bit draw picks
 * the quadrant a (src bit 0, dst bit 0), b (0,1), c (1,0) or d (1,1), most
 * significant bit first.  No noise, no id permutation.  Self-loops and
 * duplicate (src,dst) pairs are removed; the survivors come out sorted by
 * (dst, src).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t splitmix64_at(uint64_t seed, uint64_t ctr) {
  uint64_t z = seed + (ctr + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

typedef struct {
  int scale;
  int64_t lo, hi;
  uint32_t ta, tab, tabc;
  uint64_t seed;
  uint64_t* keys;
  int64_t kept;
} gen_job;

static void* gen_worker(void* arg) {
  gen_job* J = (gen_job*)arg;
  int64_t w = J->lo;
  for (int64_t i = J->lo; i < J->hi; ++i) {
    uint64_t s = 0, d = 0;
    uint64_t r = 0;
    for (int l = 0; l < J->scale; ++l) {
      if ((l & 1) == 0) r = splitmix64_at(J->seed, (uint64_t)i * 32u + (uint64_t)(l >> 1));
      uint32_t u = (l & 1) ? (uint32_t)(r >> 32) : (uint32_t)r;
      uint64_t sb, db;
      if (u < J->ta) { sb = 0; db = 0; }
      else if (u < J->tab) { sb = 0; db = 1; }
      else if (u < J->tabc) { sb = 1; db = 0; }
      else { sb = 1; db = 1; }
      s = (s << 1) | sb;
      d = (d << 1) | db;
    }
    if (s == d) continue; /* self-loop */
    J->keys[w++] = (d << J->scale) | s;
  }
  J->kept = w - J->lo;
  return NULL;
}

/* ---- parallel LSD radix sort of uint64 keys (stable, 11-bit digits) ---- */
#define RBITS 11
#define RSIZE (1 << RBITS)

typedef struct {
  const uint64_t* in;
  uint64_t* out;
  int64_t lo, hi;
  int shift;
  int64_t* hist; /* RSIZE counts, then offsets */
  int phase;
} sort_job;

static void* sort_worker(void* arg) {
  sort_job* J = (sort_job*)arg;
  if (J->phase == 0) {
    memset(J->hist, 0, sizeof(int64_t) * RSIZE);
    for (int64_t i = J->lo; i < J->hi; ++i) J->hist[(J->in[i] >> J->shift) & (RSIZE - 1)]++;
  } else {
    for (int64_t i = J->lo; i < J->hi; ++i) {
      uint64_t k = J->in[i];
      J->out[J->hist[(k >> J->shift) & (RSIZE - 1)]++] = k;
    }
  }
  return NULL;
}

static int radix_sort_u64(uint64_t* keys, uint64_t* tmp, int64_t n, int bits, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
  sort_job* jobs = (sort_job*)malloc(sizeof(sort_job) * nthreads);
  int64_t* hist = (int64_t*)malloc(sizeof(int64_t) * RSIZE * nthreads);
  if (!th || !jobs || !hist) { free(th); free(jobs); free(hist); return -1; }
  uint64_t* src = keys;
  uint64_t* dst = tmp;
  int passes = (bits + RBITS - 1) / RBITS;
  for (int p = 0; p < passes; ++p) {
    for (int t = 0; t < nthreads; ++t) {
      jobs[t].in = src; jobs[t].out = dst;
      jobs[t].lo = n * t / nthreads; jobs[t].hi = n * (t + 1) / nthreads;
      jobs[t].shift = p * RBITS; jobs[t].hist = hist + (int64_t)t * RSIZE; jobs[t].phase = 0;
      pthread_create(&th[t], NULL, sort_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    int64_t base = 0;
    for (int dgt = 0; dgt < RSIZE; ++dgt)
      for (int t = 0; t < nthreads; ++t) {
        int64_t c = hist[(int64_t)t * RSIZE + dgt];
        hist[(int64_t)t * RSIZE + dgt] = base;
        base += c;
      }
    for (int t = 0; t < nthreads; ++t) {
      jobs[t].phase = 1;
      pthread_create(&th[t], NULL, sort_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    uint64_t* x = src; src = dst; dst = x;
  }
  if (src != keys) memcpy(keys, src, sizeof(uint64_t) * (size_t)n);
  free(th); free(jobs); free(hist);
  return 0;
}

static uint32_t prob_to_u32(double p) {
  if (p <= 0.0) return 0;
  double x = p * 4294967296.0;
  if (x >= 4294967295.0) return 0xFFFFFFFFu;
  return (uint32_t)x;
}

/*
 * Draw m_draw R-MAT edges on 2^scale nodes; drop self-loops and duplicates.
 * src/dst must hold m_draw entries; the first returned-count entries are the
 * unique edges sorted by (dst, src).  Returns the unique count, or -1 on a bad
 * argument / allocation failure.
 */
int64_t rmat_generate(int scale, int64_t m_draw, double a, double b, double c,
                      uint64_t seed, int nthreads, int32_t* src, int32_t* dst) {
  if (scale < 1 || scale > 30 || m_draw < 0 || !src || !dst) return -1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(m_draw > 0 ? m_draw : 1));
  uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(m_draw > 0 ? m_draw : 1));
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
  gen_job* jobs = (gen_job*)malloc(sizeof(gen_job) * nthreads);
  if (!keys || !tmp || !th || !jobs) { free(keys); free(tmp); free(th); free(jobs); return -1; }
  uint32_t ta = prob_to_u32(a), tab = prob_to_u32(a + b), tabc = prob_to_u32(a + b + c);
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].scale = scale; jobs[t].lo = m_draw * t / nthreads; jobs[t].hi = m_draw * (t + 1) / nthreads;
    jobs[t].ta = ta; jobs[t].tab = tab; jobs[t].tabc = tabc; jobs[t].seed = seed; jobs[t].keys = keys;
    pthread_create(&th[t], NULL, gen_worker, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  /* compact the per-thread kept ranges (ranges are in order) */
  int64_t w = 0;
  for (int t = 0; t < nthreads; ++t) {
    if (w != jobs[t].lo) memmove(keys + w, keys + jobs[t].lo, sizeof(uint64_t) * (size_t)jobs[t].kept);
    w += jobs[t].kept;
  }
  int rc = radix_sort_u64(keys, tmp, w, 2 * scale, nthreads);
  free(th); free(jobs); free(tmp);
  if (rc != 0) { free(keys); return -1; }
  uint64_t mask = (1ULL << scale) - 1;
  int64_t m = 0;
  for (int64_t i = 0; i < w; ++i) {
    if (i > 0 && keys[i] == keys[i - 1]) continue;
    src[m] = (int32_t)(keys[i] & mask);
    dst[m] = (int32_t)(keys[i] >> scale);
    ++m;
  }
  free(keys);
  return m;
}

/*
 * Zipf benefit weights for targeted queries: w_v = max(1, floor(2^20 / rank_v^s))
 * where rank_v (1-based) is v's position in a keyed Fisher-Yates permutation.
 * The pow() here only shapes an input; both sides receive the finished table.
 */
int zipf_weights(int64_t n, double s, uint64_t seed, uint32_t* w) {
  if (n < 0 || !w) return -1;
  int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!perm) return -1;
  for (int64_t i = 0; i < n; ++i) perm[i] = i;
  for (int64_t i = n - 1; i > 0; --i) {
    uint64_t r = splitmix64_at(seed, (uint64_t)i);
    int64_t j = (int64_t)(((unsigned __int128)r * (uint64_t)(i + 1)) >> 64);
    int64_t x = perm[i]; perm[i] = perm[j]; perm[j] = x;
  }
  for (int64_t pos = 0; pos < n; ++pos) {
    double v = 1048576.0 / pow((double)(pos + 1), s);
    uint32_t q = v < 1.0 ? 1u : (uint32_t)v;
    w[perm[pos]] = q;
  }
  free(perm);
  return 0;
}

/* Uniform doubles in [0,1) from the same counter hash (arrival processes). */
void uniform_doubles(uint64_t seed, int64_t count, double* out) {
  for (int64_t i = 0; i < count; ++i)
    out[i] = (double)(splitmix64_at(seed, (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0);
}
