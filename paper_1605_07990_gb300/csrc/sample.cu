// RR-set samplers (Definition 2) for IC and LT (Sec. 2.1) on sm_103a.
//
// Tiers share one work list of sample ids:
//   * warp tiers: one warp per sample, visited set as an open-addressing hash
//     (shared memory, or global memory for mid-size sets) or, for weighted
//     cascade, a per-warp n-bit bitmap in global memory; the BFS queue beside
//     it.  Sets that outgrow the queue are handed on (their partial work is
//     dropped).
//   * CTA tier: one CTA per large sample, visited set as an n-bit bitmap
//     (shared memory when it fits, else a per-CTA global slot).
// IC with per-edge thresholds: frontier expansion is edge-balanced inside a
// warp: 32 frontier nodes' in-edge ranges are cut into 4-edge groups (the
// unit of one Philox draw, one aligned 32-byte sector of {src,thr} records)
// dealt to lanes by a warp prefix sum; the CTA tier skips the draw of a group
// whose edges all come from already-visited nodes and shares long in-lists
// between its warps.
// IC with weighted-cascade weights: every in-edge of a node has the same
// probability, so each lane walks one frontier node's in-list by geometric
// gaps between live edges (the gap form below); the work per node is a few
// 64-bit products and one Philox draw per two gaps, whatever its in-degree.
#include <algorithm>

#include "device.cuh"

namespace ssa {

namespace {

constexpr int WT_WARPS = 8;      // warps per warp-tier block
constexpr int WT_HASH = 1024;    // hash slots per warp (power of two)
constexpr int WT_QCAP = 512;     // largest IC set kept in the warp tier
constexpr int LT_QCAP = 1024;    // largest LT walk kept in the warp tier
constexpr int STAGE = 128;       // live candidates of one slab (32 lanes x 4 edges)
constexpr int CTA_HEAVY_GROUPS = 512;    // the CTA tier splits longer in-lists over all its warps
constexpr int CTA_HEAVY_CAP = 256;       // heavy in-lists per level shared this way
constexpr int SMALL_CTA_THREADS = 128;   // CTAs of the first stage when the visited bitmap is in global memory

constexpr uint32_t PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;

// Philox4x32-10 of the counter (x, 0, jlo, cw) with the per-launch round keys
// rk; s0/s1/s2 carry the sample-constant parts of the first round:
// s0 = hi(M1*jlo) ^ rk[0], s1 = lo(M1*jlo), s2 = cw ^ rk[1].
struct SampleConst {
  uint32_t s0, s1, s2;
};

__device__ __forceinline__ SampleConst sample_const(const uint32_t* rk, uint32_t jlo, uint32_t cw) {
  SampleConst c;
  c.s0 = __umulhi(PHILOX_M1, jlo) ^ rk[0];
  c.s1 = PHILOX_M1 * jlo;
  c.s2 = cw ^ rk[1];
  return c;
}

__device__ __forceinline__ uint4 philox_x(uint32_t x, const SampleConst& sc, const uint32_t* rk) {
  // round 1 with c.y = 0 and the sample constants folded in
  uint4 c = make_uint4(sc.s0, sc.s1, __umulhi(PHILOX_M0, x) ^ sc.s2, PHILOX_M0 * x);
#pragma unroll
  for (int r = 1; r < 10; ++r) {
    const uint32_t lo0 = PHILOX_M0 * c.x, hi0 = __umulhi(PHILOX_M0, c.x);
    const uint32_t lo1 = PHILOX_M1 * c.z, hi1 = __umulhi(PHILOX_M1, c.z);
    c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
  }
  return c;
}

// Philox4x32-10 of the counter (x, y, jlo, cw): philox_x with a second
// counter word y, which enters the first round beside the sample constants.
__device__ __forceinline__ uint4 philox_xy(uint32_t x, uint32_t y, const SampleConst& sc, const uint32_t* rk) {
  uint4 c = make_uint4(sc.s0 ^ y, sc.s1, __umulhi(PHILOX_M0, x) ^ sc.s2, PHILOX_M0 * x);
#pragma unroll
  for (int r = 1; r < 10; ++r) {
    const uint32_t lo0 = PHILOX_M0 * c.x, hi0 = __umulhi(PHILOX_M0, c.x);
    const uint32_t lo1 = PHILOX_M1 * c.z, hi1 = __umulhi(PHILOX_M1, c.z);
    c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
  }
  return c;
}

__device__ __forceinline__ int64_t sample_at(const SampleJob& J, unsigned long long idx) {
  return J.work_list ? J.work_list[idx] : J.j0 + (int64_t)idx;
}

__device__ __forceinline__ int32_t pick_root(const SampleJob& J, int64_t j) {
  const uint4 r = keyed_draw(J.seed, PURPOSE_ROOT, J.stream, j, 0);
  const int64_t n = J.g.n;
  if (!J.bprefix) return (int32_t)__umulhi(r.x, (uint32_t)n);
  // WRIS (Sec. 6.3.1): the node whose benefit interval holds a 64-bit target
  const uint64_t W = J.bprefix[n];
  const uint64_t r64 = (uint64_t)r.x | ((uint64_t)r.y << 32);
  const uint64_t target = __umul64hi(r64, W);
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (J.bprefix[mid + 1] > target) hi = mid; else lo = mid + 1;
  }
  return (int32_t)lo;
}

// Warp-per-sample tiers: 0 = hash and queue in shared memory (sets up to
// 512 nodes), 1 = per-warp hash and queue in global memory (up to 16384
// nodes).  Larger sets go on to the CTA tier.
template <int TIER>
struct Tier;
template <>
struct Tier<0> {
  static constexpr int HBITS = 10, QCAP = WT_QCAP;
};
template <>
struct Tier<1> {
  static constexpr int HBITS = 15, QCAP = 16384;
};
constexpr int MID_HASH = 1 << Tier<1>::HBITS;
constexpr int MID_QSLOTS = Tier<1>::QCAP + 32;  // queue/slot entries per warp (room for one round past the cap)

template <int HBITS>
__device__ __forceinline__ uint32_t hash_slot(uint32_t u) {
  return (u * 0x9E3779B1u) >> (32 - HBITS);
}

// Insert u into a warp's hash set of 2^HBITS slots; true when u was not
// there, with its slot in *slot.
template <int HBITS>
__device__ __forceinline__ bool hash_insert(uint32_t* H, uint32_t u, uint32_t* slot) {
  const uint32_t key = u + 1u;
  uint32_t h = hash_slot<HBITS>(u);
  for (int probe = 0; probe < (1 << HBITS); ++probe) {
    const uint32_t prev = atomicCAS(H + h, 0u, key);
    if (prev == 0u) {
      *slot = h;
      return true;
    }
    if (prev == key) return false;
    h = (h + 1u) & ((1u << HBITS) - 1u);
  }
  return false;  // not reached: the table is never more than half full
}

template <class Visit>
__device__ __forceinline__ bool deliver(uint32_t cand, uint32_t u0, uint32_t u1, uint32_t u2, uint32_t u3, int lane,
                                        uint32_t* stage, Visit&& visit);

// One slab: each lane holds one 4-edge group `grp` of an in-list [olo, ohi)
// (when `valid`).  Edges whose tail may be new draw their coins; the live
// ones are compacted through `stage` (STAGE entries, private to the warp) and
// handed to visit(u) in rounds of 32 (NO_NODE for idle lanes).  known(u) may
// report tails already in the set so their edges need no draw.  Returns the
// warp-uniform "stop" of visit.
template <class Known, class Visit>
__device__ __forceinline__ bool process_slab(const GraphView& g, bool valid, uint32_t grp, uint32_t olo, uint32_t ohi,
                                             const uint32_t* rk, const SampleConst& sc, int lane, uint32_t* stage,
                                             unsigned long long& draws, Known&& known, Visit&& visit) {
  uint32_t cand = 0, u0 = 0, u1 = 0, u2 = 0, u3 = 0;
  if (valid) {
    const uint32_t e = grp * 4u;
    // edges e..e+3 that belong to the in-list
    const uint32_t a = olo > e ? olo - e : 0u;
    const uint32_t b = ohi - e;
    uint32_t need = (b >= 4u ? 0xFu : ((1u << b) - 1u)) & ((0xFu << a) & 0xFu);
    const uint4* p = reinterpret_cast<const uint4*>(g.edge) + (size_t)grp * 2;
    const uint4 A = __ldg(p), B = __ldg(p + 1);
    u0 = A.x; u1 = A.z; u2 = B.x; u3 = B.z;
    if ((need & 1u) && known(u0)) need &= ~1u;
    if ((need & 2u) && known(u1)) need &= ~2u;
    if ((need & 4u) && known(u2)) need &= ~4u;
    if ((need & 8u) && known(u3)) need &= ~8u;
    if (need) {
      ++draws;
      const uint4 r = philox_x(grp, sc, rk);
      if ((need & 1u) && edge_live(r.x, A.y)) cand |= 1u;
      if ((need & 2u) && edge_live(r.y, A.w)) cand |= 2u;
      if ((need & 4u) && edge_live(r.z, B.y)) cand |= 4u;
      if ((need & 8u) && edge_live(r.w, B.w)) cand |= 8u;
    }
  }
  return deliver(cand, u0, u1, u2, u3, lane, stage, visit);
}

// Hand the live candidates of one slab (lane-held masks over 4 tails) to
// visit(u) in rounds of 32 (NO_NODE for idle lanes), compacted through
// `stage` when some lane holds more than one.  Returns visit's "stop".
template <class Visit>
__device__ __forceinline__ bool deliver(uint32_t cand, uint32_t u0, uint32_t u1, uint32_t u2, uint32_t u3, int lane,
                                        uint32_t* stage, Visit&& visit) {
  const unsigned lt_mask = (1u << lane) - 1u;
  const unsigned any = __ballot_sync(FULL_MASK, cand != 0u);
  if (!any) return false;
  if (!__any_sync(FULL_MASK, (cand & (cand - 1u)) != 0u)) {
    // at most one candidate per lane (the common case): no staging
    const uint32_t u = !cand ? NO_NODE : (cand & 1u) ? u0 : (cand & 2u) ? u1 : (cand & 4u) ? u2 : u3;
    return visit(u, lt_mask);
  }
  const int c = __popc(cand);
  const int cin = warp_inclusive_scan(c, lane);
  const int ctot = __shfl_sync(FULL_MASK, cin, 31);
  int pos = cin - c;
  if (cand & 1u) stage[pos++] = u0;
  if (cand & 2u) stage[pos++] = u1;
  if (cand & 4u) stage[pos++] = u2;
  if (cand & 8u) stage[pos++] = u3;
  __syncwarp();
  bool stop = false;
  for (int s0 = 0; s0 < ctot && !stop; s0 += 32) {
    const uint32_t u = (s0 + lane < ctot) ? stage[s0 + lane] : NO_NODE;
    stop = visit(u, lt_mask);
  }
  __syncwarp();
  return stop;
}

// Edge-balanced expansion of up to 32 frontier nodes (lane i holds node v or
// -1): their in-edge ranges are cut into 4-edge groups dealt to lanes by a
// warp prefix sum.  A node with more than heavy_groups groups is first offered
// to take_heavy(v, lo, hi, ng) (per lane); when it takes the node, the node is
// skipped here.  Returns 0, 1 when visit asked to stop, or 2 when
// take_heavy(...) == HEAVY_ABORT for some lane (the caller hands the sample on).
constexpr int HEAVY_SKIP = 1, HEAVY_ABORT = 2;

template <class Known, class Visit, class Heavy>
__device__ __forceinline__ int expand_ic(const GraphView& g, int32_t v, const uint32_t* rk, const SampleConst& sc,
                                         int lane, uint32_t* stage, unsigned long long& ev, unsigned long long& draws,
                                         int heavy_groups, Known&& known, Visit&& visit, Heavy&& take_heavy) {
  uint32_t lo = 0, hi = 0;  // edge positions fit 32 bits (m < 2^31)
  if (v >= 0) {
    lo = (uint32_t)__ldg(g.off + v);
    hi = (uint32_t)__ldg(g.off + v + 1);
  }
  int ng = (hi > lo) ? (int)(((hi + 3) >> 2) - (lo >> 2)) : 0;
  int heavy = 0;
  if (ng > heavy_groups) heavy = take_heavy(v, lo, hi, ng);
  if (__any_sync(FULL_MASK, heavy == HEAVY_ABORT)) return 2;
  if (heavy == HEAVY_SKIP) ng = 0;  // counted and expanded by the taker
  else ev += hi - lo;
  const int incl = warp_inclusive_scan(ng, lane);
  const int excl = incl - ng;
  const int total = __shfl_sync(FULL_MASK, incl, 31);
  for (int base = 0; base < total; base += 32) {
    const int q = base + lane;
    int owner = 0;
#pragma unroll
    for (int s = 16; s; s >>= 1) {
      const int t = __shfl_sync(FULL_MASK, incl, owner + s - 1);
      if (t <= q) owner += s;
    }
    owner = owner > 31 ? 31 : owner;
    const uint32_t olo = __shfl_sync(FULL_MASK, lo, owner);
    const uint32_t ohi = __shfl_sync(FULL_MASK, hi, owner);
    const int oex = __shfl_sync(FULL_MASK, excl, owner);
    const uint32_t grp = (olo >> 2) + (uint32_t)(q - oex);
    if (process_slab(g, q < total, grp, olo, ohi, rk, sc, lane, stage, draws, known, visit)) return 1;
  }
  return 0;
}

// Weighted-cascade threshold of a node with d in-edges: floor(2^32 / d), and
// 0xFFFFFFFF (probability 1) for d = 1.
__device__ __forceinline__ uint32_t wc_threshold(uint32_t d) {
  return d <= 1u ? 0xFFFFFFFFu : (uint32_t)(0x100000000ull / d);
}

// Gap form of weighted cascade.  All d >= 2 in-edges of a node are live with
// p = t / 2^32 (t = wc_threshold(d)), so the run G of dead edges before the
// next live one has P(G >= g) = q^g, q = 1 - p.  In Q64 integers (x in [0,1)
// as floor(x 2^64), products truncated): Q = (2^32 - t) << 32, P_0 = Q,
// P_(i+1) = hi64(P_i * P_i); G(U) sets bits J-1 .. 0 in turn (J the bit
// length of d, so 2^J - 1 >= d), bit i when U < hi64(A * P_i), A the product
// of the powers already taken (P_i alone for the first), which then becomes
// A.  G(U) is the largest g with U < q^g up to the truncation.  The powers of
// a node are built once, into the lane's own table P (J <= 31 entries).
__device__ __forceinline__ void wc_powers(uint64_t Q, int J, uint64_t* P) {
  uint64_t p = Q;
  for (int i = 0; i < J; ++i) {
    P[i] = p;
    p = __umul64hi(p, p);
  }
}

// The powers of in-degree d >= 2: the graph's table row when d < 2^wc_pow_k
// (rows for d in [2^k, 2^(k+1)) hold k+1 entries and follow all shorter rows,
// so row d starts at (k-1) 2^k + 1 + (d - 2^k)(k+1)), else built into `own`.
__device__ __forceinline__ const uint64_t* wc_power_row(const GraphView& g, uint32_t d, int J, uint64_t* own) {
  if (d < (1u << g.wc_pow_k)) {
    const int k = J - 1;
    return g.wc_pow + ((uint64_t)(k - 1) << k) + 1ull + (uint64_t)(d - (1u << k)) * (uint64_t)J;
  }
  wc_powers((0x100000000ull - wc_threshold(d)) << 32, J, own);
  return own;
}

__device__ __forceinline__ uint32_t wc_gap(const uint64_t* P, int J, uint64_t U) {
  uint64_t A = 0;
  bool first = true;
  uint32_t gap = 0;
  for (int i = J - 1; i >= 0; --i) {
    const uint64_t cand = first ? P[i] : __umul64hi(A, P[i]);
    if (U < cand) {
      A = cand;
      first = false;
      gap |= 1u << i;
    }
  }
  return gap;
}

// The gap walk of one weighted-cascade node as a state machine, for the CTA
// tier, whose lanes keep a node across rounds: d = 1 is one live edge
// (probability 1, no draw); otherwise gap c takes the 64-bit uniform of
// words 2(c&1), 2(c&1)+1 of the SKIP draw with counter words (v, c >> 1), the
// next live edge is lo + pos + G, and the walk ends when G reaches past the
// list.  (The lane tier and the warp BFS inline the same steps.)
struct GapWalk {
  uint32_t lo = 0, d = 0;   // the node's in-list
  uint32_t pos = 0, c = 0;  // position in it; gaps drawn
  int J = 0;                // bit length of d
  const uint64_t* P = nullptr;
  uint64_t spare = 0;
};

// Start the walk of node v; false when it has no in-edges.
__device__ __forceinline__ bool walk_begin(GapWalk& w, const GraphView& g, int32_t v, uint64_t* own) {
  w.lo = (uint32_t)__ldg(g.off + v);
  w.d = (uint32_t)__ldg(g.off + v + 1) - w.lo;
  w.pos = 0;
  w.c = 0;
  w.J = 32 - __clz((int)w.d);
  w.P = w.d >= 2u ? wc_power_row(g, w.d, w.J, own) : nullptr;
  return w.d > 0u;
}

// One step: the tail of the next live edge, or NO_NODE when the node has no
// more; *more says whether the node may still give live edges.
__device__ __forceinline__ uint32_t walk_step(GapWalk& w, const GraphView& g, int32_t v, const uint32_t* rk,
                                              const SampleConst& skc, unsigned long long& draws, bool* more) {
  uint32_t e;
  if (w.d == 1u) {
    e = w.lo;
    w.pos = 1;
  } else {
    uint64_t U;
    if (!(w.c & 1u)) {
      const uint4 r = philox_xy((uint32_t)v, w.c >> 1, skc, rk);
      ++draws;
      U = (uint64_t)r.x | ((uint64_t)r.y << 32);
      w.spare = (uint64_t)r.z | ((uint64_t)r.w << 32);
    } else {
      U = w.spare;
    }
    const uint32_t G = wc_gap(w.P, w.J, U);
    if (G >= w.d - w.pos) {
      *more = false;
      return NO_NODE;
    }
    e = w.lo + w.pos + G;
    w.pos += G + 1u;
    ++w.c;
  }
  *more = w.pos < w.d;
  return __ldg(&g.edge[e].x);
}

// Weighted-cascade BFS of one sample by one warp over its private queue
// Q[0, tail) (head = 0 at the start): every lane holds at most one node and
// takes one gap step per round; a lane whose node is done takes the next
// queued node at the start of the next round, so the lanes stay busy while
// the queue holds work (a node's walk is the gap walk of walk_step, the same
// keyed draws).  visit(u, lt_mask) appends new nodes to Q and advances tail
// (which this function reads through the reference); it returns "stop".
template <class Visit>
__device__ __forceinline__ void wc_bfs_warp(const GraphView& g, const int32_t* Q, const int& tail,
                                            const uint32_t* rk, const SampleConst& skc, int lane,
                                            unsigned long long& ev, unsigned long long& draws, Visit&& visit) {
  const unsigned lt_mask = (1u << lane) - 1u;
  int head = 0;
  int32_t v = -1;
  uint32_t lo = 0, d = 0, pos = 0, c = 0;
  int Jb = 0;
  uint64_t spare = 0;
  uint64_t own[31];  // q^(2^i), i < Jb, of the lane's node when the graph's table has no row for it
  const uint64_t* P = nullptr;
  for (;;) {
    __syncwarp();  // queue entries written by other lanes in the last round
    const bool need = v < 0;
    const unsigned nm = __ballot_sync(FULL_MASK, need);
    const int take = min(__popc(nm), tail - head);
    if (need) {
      const int r = __popc(nm & lt_mask);
      if (r < take) {
        v = Q[head + r];
        lo = (uint32_t)__ldg(g.off + v);
        d = (uint32_t)__ldg(g.off + v + 1) - lo;
        ev += d;
        pos = 0;
        c = 0;
        Jb = 32 - __clz((int)d);
        if (d >= 2u) P = wc_power_row(g, d, Jb, own);
      }
    }
    head += take;
    if (!__any_sync(FULL_MASK, v >= 0)) break;  // queue drained, no lane holds a node
    uint32_t u = NO_NODE;
    if (v >= 0) {
      if (d == 0u) {
        v = -1;
      } else if (d == 1u) {
        u = __ldg(&g.edge[lo].x);
        v = -1;
      } else {
        uint64_t U;
        if (!(c & 1u)) {
          const uint4 r = philox_xy((uint32_t)v, c >> 1, skc, rk);
          ++draws;
          U = (uint64_t)r.x | ((uint64_t)r.y << 32);
          spare = (uint64_t)r.z | ((uint64_t)r.w << 32);
        } else {
          U = spare;
        }
        const uint32_t G = wc_gap(P, Jb, U);
        if (G >= d - pos) {
          v = -1;
        } else {
          u = __ldg(&g.edge[lo + pos + G].x);
          pos += G + 1u;
          ++c;
          if (pos >= d) v = -1;
        }
      }
    }
    if (visit(u, lt_mask)) return;
  }
}

__device__ __forceinline__ void flush_stats(Counters* ctr, unsigned long long ev, unsigned long long nv,
                                            unsigned long long dr, int lane, bool cta_tier) {
  ev = warp_sum(ev);
  nv = warp_sum(nv);
  dr = warp_sum(dr);
  if (lane == 0) {
    if (dr) atomicAdd(&ctr->draws, dr);
    if (ev) atomicAdd(&ctr->edge_visits, ev);
    if (nv) atomicAdd(&ctr->node_visits, nv);
    if (cta_tier && ev) atomicAdd(&ctr->cta_edge_visits, ev);
    if (cta_tier && nv) atomicAdd(&ctr->cta_node_visits, nv);
    if (cta_tier && dr) atomicAdd(&ctr->cta_draws, dr);
  }
}

// Reserve `size` pool entries (one thread).  Reservations are handed out in
// increasing position order, so the ones that fit form a prefix; it ends where
// the first one that did not fit starts (ok_end, the least such position), and
// the rest [ok_end, cursor) are re-run by the host from fail_list.
__device__ __forceinline__ bool reserve(const SampleJob& J, int64_t j, int size, unsigned long long* pos) {
  *pos = atomicAdd(&J.ctr->cursor, (unsigned long long)size);
  if (*pos + (unsigned long long)size <= (unsigned long long)J.pool_cap) return true;
  atomicMin(&J.ctr->ok_end, *pos);
  atomicExch(&J.ctr->pool_overflow, 1u);
  const unsigned long long f = atomicAdd(&J.ctr->fail_count, 1ull);
  J.fail_list[f] = j;
  return false;
}

template <typename QT>
__device__ __forceinline__ void warp_store_set(const SampleJob& J, int64_t j, const QT* Q, int size, int lane) {
  unsigned long long pos = 0;
  int ok = 0;
  if (lane == 0) ok = reserve(J, j, size, &pos);
  ok = __shfl_sync(FULL_MASK, ok, 0);
  pos = __shfl_sync(FULL_MASK, pos, 0);
  if (!ok) return;
  for (int i = lane; i < size; i += 32) {
    J.pool_nodes[pos + i] = Q[i];
    J.pool_samp[pos + i] = (int32_t)j;
  }
  if (lane == 0) {
    J.set_start[j] = (int64_t)pos;
    J.set_len[j] = size;
  }
}

template <int MODE, int TIER, bool WC>
__global__ void __launch_bounds__(WT_WARPS * 32, 4) k_sample_warp_ic(SampleJob J) {
  constexpr int HBITS = Tier<TIER>::HBITS, QCAP = Tier<TIER>::QCAP;
  __shared__ __align__(16) uint32_t s_hash[TIER == 0 ? WT_WARPS : 1][TIER == 0 ? WT_HASH : 4];
  __shared__ int32_t s_q[TIER == 0 ? WT_WARPS : 1][TIER == 0 ? WT_QCAP : 4];
  __shared__ uint32_t s_stage[WT_WARPS][WC ? 1 : STAGE];  // the gap walk needs no staging
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const size_t gwarp = (size_t)blockIdx.x * WT_WARPS + wid;
  uint32_t* H = TIER == 0 ? s_hash[wid] : J.mid_hash + gwarp * MID_HASH;
  int32_t* Q = TIER == 0 ? s_q[wid] : J.mid_queue + gwarp * MID_QSLOTS;
  uint32_t* slots = TIER == 0 ? nullptr : J.mid_slots + gwarp * MID_QSLOTS;
  if (TIER == 0) {
    uint4* H4 = reinterpret_cast<uint4*>(H);
    for (int i = lane; i < WT_HASH / 4; i += 32) H4[i] = make_uint4(0, 0, 0, 0);
  }
  __syncwarp();
  // tier 0 takes the batch's samples (or those the lane tier listed), tier 1 the ones tier 0 handed over
  const unsigned long long count =
      TIER == 0 ? (J.lane_tier ? *((volatile unsigned long long*)&J.ctr->lane_count) : (unsigned long long)J.count)
                : *((volatile unsigned long long*)&J.ctr->mid_count);
  unsigned long long* work = TIER == 0 ? &J.ctr->work : &J.ctr->mid_work;
  unsigned long long ev = 0, nv = 0, dr = 0;
  for (;;) {
    unsigned long long idx = 0;
    if (lane == 0) idx = atomicAdd(work, 1ull);
    idx = __shfl_sync(FULL_MASK, idx, 0);
    if (idx >= count) break;
    const int64_t j = TIER == 0 ? (J.lane_tier ? J.lane_list[idx] : sample_at(J, idx)) : J.mid_list[idx];
    const SampleConst sc = sample_const(J.rk, (uint32_t)j, ctr_word3(WC ? PURPOSE_SKIP : PURPOSE_IC, J.stream, j));
    const int32_t root = pick_root(J, j);
    if (lane == 0) {
      const uint32_t h0 = hash_slot<HBITS>((uint32_t)root);
      H[h0] = (uint32_t)root + 1u;
      Q[0] = root;
      if (TIER == 1) slots[0] = h0;
    }
    int tail = 1, head = 0;
    bool overflow = false;
    bool hit = (MODE == MODE_HIT) && test_bit(J.seed_bits, (uint32_t)root);
    // tier 1's hand-over size is tuned at run time (at most its queue capacity)
    const int cap = TIER == 0 ? QCAP : min(QCAP, J.mid_cap);
    __syncwarp();
    auto known = [](uint32_t) { return false; };
    auto visit = [&](uint32_t u, unsigned lt_mask) -> bool {
      uint32_t slot = 0;
      const bool is_new = (u != NO_NODE) && hash_insert<HBITS>(H, u, &slot);
      const unsigned m = __ballot_sync(FULL_MASK, is_new);
      bool h = false;
      if (is_new) {
        const int pos = tail + __popc(m & lt_mask);
        if (TIER == 0) {
          if (pos < QCAP) Q[pos] = (int32_t)u;
        } else {
          Q[pos] = (int32_t)u;  // pos <= cap + 31 < QCAP + 32: room for one round past the cap
          slots[pos] = slot;
        }
        if (MODE == MODE_HIT) h = test_bit(J.seed_bits, u);
      }
      tail += __popc(m);
      if (MODE == MODE_HIT) hit = __any_sync(FULL_MASK, h) || hit;
      if (tail > cap) overflow = true;
      return overflow || hit;
    };
    // a node with a very long in-list needs many warps: hand the sample to the CTA tier
    // (weighted cascade: no in-list is long, its gap walk costs the same at any degree)
    auto to_cta = [](int32_t, uint32_t, uint32_t, int) { return HEAVY_ABORT; };
    bool handoff = false;
    if constexpr (WC) {
      if (!hit) wc_bfs_warp(J.g, Q, tail, J.rk, sc, lane, ev, dr, visit);
    } else {
      while (head < tail && !overflow && !hit) {
        const int cnt = min(32, tail - head);
        __syncwarp();
        const int32_t v = (lane < cnt) ? Q[head + lane] : -1;
        __syncwarp();
        if (expand_ic(J.g, v, J.rk, sc, lane, s_stage[wid], ev, dr, J.warp_heavy_groups, known, visit, to_cta) ==
            2) {
          handoff = true;
          break;
        }
        head += cnt;
      }
    }
    __syncwarp();
    if (handoff) {
      if (lane == 0) {
        const unsigned long long b = atomicAdd(&J.ctr->big_count, 1ull);
        J.big_list[b] = j;
      }
    } else if (overflow) {
      if (lane == 0) {
        if (TIER == 0 && J.mid_cap > 0) {
          const unsigned long long b = atomicAdd(&J.ctr->mid_count, 1ull);
          J.mid_list[b] = j;
        } else {
          const unsigned long long b = atomicAdd(&J.ctr->big_count, 1ull);
          J.big_list[b] = j;
        }
      }
    } else {
      if (MODE == MODE_STORE) warp_store_set(J, j, Q, tail, lane);
      else if (lane == 0) J.hit[j - J.j0] = hit ? 1 : 0;
      if (lane == 0) nv += (unsigned long long)tail;
    }
    __syncwarp();
    if (TIER == 0) {
      uint4* H4 = reinterpret_cast<uint4*>(H);
      for (int i = lane; i < WT_HASH / 4; i += 32) H4[i] = make_uint4(0, 0, 0, 0);
    } else {
      // clear only the slots this sample used (tail <= QCAP + 32 entries recorded)
      for (int i = lane; i < tail; i += 32) H[slots[i]] = 0u;
    }
    __syncwarp();
  }
  flush_stats(J.ctr, ev, nv, dr, lane, false);
}

// Weighted-cascade IC, one warp per sample of up to GQ_CAP nodes (or mid_cap,
// when set), with the visited set as a per-warp n-bit bitmap in global memory
// and the BFS queue in global memory: one tier for every set size up to the
// queue, where the hash tiers stop at 512 and 16384 nodes.  Larger sets go to
// the CTA tier.
constexpr int GQ_CAP = 1 << 16;
constexpr int GQ_SLOTS = GQ_CAP + 32;  // room for one round past the cap

template <int MODE>
__global__ void __launch_bounds__(WT_WARPS * 32, 4) k_sample_warp_wcg(SampleJob J) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const size_t gwarp = (size_t)blockIdx.x * WT_WARPS + wid;
  uint32_t* bits = J.wg_bitmap + gwarp * (size_t)J.bitmap_words;
  int32_t* Q = J.wg_queue + gwarp * (size_t)GQ_SLOTS;
  // the batch's samples, or those the lane tier listed
  const unsigned long long count =
      J.lane_tier ? *((volatile unsigned long long*)&J.ctr->lane_count) : (unsigned long long)J.count;
  // sets above mid_cap nodes (when set) go on to the CTA tier, whose warps share a sample
  const int cap = J.mid_cap > 0 ? min(J.mid_cap, GQ_CAP) : GQ_CAP;
  unsigned long long ev = 0, nv = 0, dr = 0;
  for (;;) {
    unsigned long long idx = 0;
    if (lane == 0) idx = atomicAdd(&J.ctr->work, 1ull);
    idx = __shfl_sync(FULL_MASK, idx, 0);
    if (idx >= count) break;
    const int64_t j = J.lane_tier ? J.lane_list[idx] : sample_at(J, idx);
    const SampleConst sc = sample_const(J.rk, (uint32_t)j, ctr_word3(PURPOSE_SKIP, J.stream, j));
    const int32_t root = pick_root(J, j);
    if (lane == 0) {
      atomicOr(bits + (root >> 5), 1u << (root & 31));
      Q[0] = root;
    }
    int tail = 1;
    bool overflow = false;
    bool hit = (MODE == MODE_HIT) && test_bit(J.seed_bits, (uint32_t)root);
    __syncwarp();
    auto visit = [&](uint32_t u, unsigned lt_mask) -> bool {
      bool is_new = false;
      if (u != NO_NODE) {
        const uint32_t mask = 1u << (u & 31);
        is_new = !(atomicOr(bits + (u >> 5), mask) & mask);
      }
      const unsigned m = __ballot_sync(FULL_MASK, is_new);
      bool h = false;
      if (is_new) {
        Q[tail + __popc(m & lt_mask)] = (int32_t)u;  // tail <= cap <= GQ_CAP before this round: fits GQ_SLOTS
        if (MODE == MODE_HIT) h = test_bit(J.seed_bits, u);
      }
      tail += __popc(m);
      if (MODE == MODE_HIT) hit = __any_sync(FULL_MASK, h) || hit;
      if (tail > cap) overflow = true;
      return overflow || hit;
    };
    if (!hit) wc_bfs_warp(J.g, Q, tail, J.rk, sc, lane, ev, dr, visit);
    __syncwarp();
    if (overflow) {
      if (lane == 0) {
        const unsigned long long b = atomicAdd(&J.ctr->big_count, 1ull);
        J.big_list[b] = j;
      }
    } else {
      if (MODE == MODE_STORE) warp_store_set(J, j, Q, tail, lane);
      else if (lane == 0) J.hit[j - J.j0] = hit ? 1 : 0;
      if (lane == 0) nv += (unsigned long long)tail;
    }
    __syncwarp();
    // clear the words of this sample's nodes (every set bit has its queue entry)
    for (int i = lane; i < tail; i += 32) bits[Q[i] >> 5] = 0u;
    __syncwarp();
  }
  flush_stats(J.ctr, ev, nv, dr, lane, false);
}

// Lane tier (weighted-cascade IC): one lane per sample.  Each lane runs the
// whole BFS of its own sample with the gap walk, its queue (up to LANE_Q
// nodes) in thread-local memory and membership tested by scanning that
// queue.  A sample that outgrows the queue is listed in lane_list for the
// warp tiers (its partial work is dropped).  Weighted-cascade sets are mostly
// a handful of nodes (on the 2^25-node R-MAT graph the median is one node and
// nine in ten have at most 18), so 32 independent samples per warp keep far
// more memory requests in flight than one sample per warp.  Lanes claim
// sample indices and store their sets independently of each other.
constexpr int LANE_Q = 32;

template <int MODE>
__global__ void __launch_bounds__(256) k_sample_lane_wc(SampleJob J) {
  const int lane = threadIdx.x & 31;
  int32_t q[LANE_Q];
  uint64_t own[31];  // powers of a node whose in-degree has no row in the graph's table
  unsigned long long ev = 0, nv = 0, dr = 0;
  for (;;) {
    // one sample per lane; the lanes that arrive together share one atomic
    const unsigned act = __activemask();
    const int leader = __ffs(act) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(&J.ctr->lane_work, (unsigned long long)__popc(act));
    base = __shfl_sync(act, base, leader);
    const unsigned long long idx = base + (unsigned long long)__popc(act & ((1u << lane) - 1u));
    if (idx >= (unsigned long long)J.count) break;
    const int64_t j = sample_at(J, idx);
    const SampleConst sc = sample_const(J.rk, (uint32_t)j, ctr_word3(PURPOSE_SKIP, J.stream, j));
    const int32_t root = pick_root(J, j);
    q[0] = root;
    int tail = 1;
    bool hit = (MODE == MODE_HIT) && test_bit(J.seed_bits, (uint32_t)root);
    bool overflow = false;
    for (int h = 0; h < tail && !hit && !overflow; ++h) {
      const int32_t v = q[h];
      const uint32_t lo = (uint32_t)__ldg(J.g.off + v);
      const uint32_t d = (uint32_t)__ldg(J.g.off + v + 1) - lo;
      ev += d;
      if (d == 0u) continue;
      const int Jb = 32 - __clz((int)d);
      const uint64_t* P = d >= 2u ? wc_power_row(J.g, d, Jb, own) : nullptr;
      uint32_t pos = 0, c = 0;
      uint64_t spare = 0;
      while (pos < d) {
        uint32_t e;
        if (d == 1u) {
          e = lo;
          pos = 1;
        } else {
          uint64_t U;
          if (!(c & 1u)) {
            const uint4 r = philox_xy((uint32_t)v, c >> 1, sc, J.rk);
            ++dr;
            U = (uint64_t)r.x | ((uint64_t)r.y << 32);
            spare = (uint64_t)r.z | ((uint64_t)r.w << 32);
          } else {
            U = spare;
          }
          const uint32_t G = wc_gap(P, Jb, U);
          if (G >= d - pos) break;
          e = lo + pos + G;
          pos += G + 1u;
          ++c;
        }
        const int32_t u = (int32_t)__ldg(&J.g.edge[e].x);
        bool seen = false;
        for (int i = 0; i < tail; ++i) seen |= q[i] == u;
        if (seen) continue;
        if (tail == LANE_Q) {
          overflow = true;
          break;
        }
        q[tail++] = u;
        if (MODE == MODE_HIT && test_bit(J.seed_bits, (uint32_t)u)) {
          hit = true;
          break;
        }
      }
    }
    if (overflow) {
      const unsigned long long b = atomicAdd(&J.ctr->lane_count, 1ull);
      J.lane_list[b] = j;
      continue;
    }
    if (MODE == MODE_STORE) {
      unsigned long long at = 0;
      if (reserve(J, j, tail, &at)) {
        for (int i = 0; i < tail; ++i) {
          J.pool_nodes[at + i] = q[i];
          J.pool_samp[at + i] = (int32_t)j;
        }
        J.set_start[j] = (int64_t)at;
        J.set_len[j] = tail;
      }
    } else {
      J.hit[j - J.j0] = hit ? 1 : 0;
    }
    nv += (unsigned long long)tail;
  }
  __syncwarp();
  flush_stats(J.ctr, ev, nv, dr, lane, false);
}

// LT live-edge walk (one keyed in-neighbour per node), warp per sample: every
// lane follows the same walk; membership of the next node is checked by the
// 32 lanes over the walk list in shared memory.
template <int MODE>
__global__ void __launch_bounds__(WT_WARPS * 32) k_sample_warp_lt(SampleJob J) {
  __shared__ int32_t s_q[WT_WARPS][LT_QCAP];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t* Q = s_q[wid];
  unsigned long long ev = 0, nv = 0, dr = 0;
  for (;;) {
    unsigned long long idx = 0;
    if (lane == 0) idx = atomicAdd(&J.ctr->work, 1ull);
    idx = __shfl_sync(FULL_MASK, idx, 0);
    if (idx >= (unsigned long long)J.count) break;
    const int64_t j = sample_at(J, idx);
    const SampleConst sc = sample_const(J.rk, (uint32_t)j, ctr_word3(PURPOSE_LT, J.stream, j));
    const int32_t root = pick_root(J, j);
    if (lane == 0) Q[0] = root;
    int tail = 1;
    bool overflow = false;
    bool hit = (MODE == MODE_HIT) && test_bit(J.seed_bits, (uint32_t)root);
    int32_t cur = root;
    __syncwarp();
    while (!hit) {
      const int64_t lo = __ldg(J.g.off + cur), hi = __ldg(J.g.off + cur + 1);
      const int64_t d = hi - lo;
      if (d == 0) break;
      const uint4 r = philox_x((uint32_t)cur, sc, J.rk);
      int64_t pick;
      if (!J.lt_cumulative) {
        pick = lo + __umulhi(r.x, (uint32_t)d);  // w = 1/d_in: one of the d in-edges
      } else {
        // general in-weights: first in-edge whose running threshold sum passes r, or none
        pick = -1;
        unsigned long long carry = 0;
        for (int64_t b = lo; b < hi; b += 32) {
          const int64_t e = b + lane;
          unsigned long long incl = e < hi ? (unsigned long long)__ldg(&J.g.edge[e].y) : 0ull;
#pragma unroll
          for (int dd = 1; dd < 32; dd <<= 1) {
            const unsigned long long t = __shfl_up_sync(FULL_MASK, incl, dd);
            if (lane >= dd) incl += t;
          }
          const unsigned hitm = __ballot_sync(FULL_MASK, e < hi && (unsigned long long)r.x < carry + incl);
          if (hitm) {
            pick = b + __ffs(hitm) - 1;
            break;
          }
          carry += __shfl_sync(FULL_MASK, incl, 31);
        }
        if (pick < 0) break;  // no in-edge kept: the walk ends here
      }
      const int32_t u = (int32_t)__ldg(&J.g.edge[pick].x);
      if (lane == 0) {
        ev += 1;
        dr += 1;
      }
      bool found = false;
      for (int i = lane; i < tail; i += 32) found |= (Q[i] == u);
      if (__any_sync(FULL_MASK, found)) break;
      if (tail >= LT_QCAP) {
        overflow = true;
        break;
      }
      if (lane == 0) Q[tail] = u;
      ++tail;
      __syncwarp();
      if (MODE == MODE_HIT) hit = test_bit(J.seed_bits, (uint32_t)u);
      cur = u;
    }
    __syncwarp();
    if (overflow) {
      if (lane == 0) {
        const unsigned long long b = atomicAdd(&J.ctr->big_count, 1ull);
        J.big_list[b] = j;
      }
    } else {
      if (MODE == MODE_STORE) warp_store_set(J, j, Q, tail, lane);
      else if (lane == 0) J.hit[j - J.j0] = hit ? 1 : 0;
      if (lane == 0) nv += (unsigned long long)tail;
    }
    __syncwarp();
  }
  flush_stats(J.ctr, ev, nv, dr, lane, false);
}

// CTA tier: one CTA per large sample.
// KIND 0: the only CTA stage (bitmap in shared memory, queue of n entries).
// KIND 1: small CTAs (bitmap in global memory, queue of small_qcap entries);
//         a set that outgrows the queue goes on to KIND 2.
// KIND 2: full-size CTAs (global bitmap, queue of n entries) for those sets.
template <int MODE, bool SMEM_BITMAP, int KIND, bool WC>
__global__ void __launch_bounds__(KIND == 1 ? SMALL_CTA_THREADS : 1024, KIND == 1 ? 1024 / SMALL_CTA_THREADS : 1)
    k_sample_cta(SampleJob J) {
  constexpr int WARPS = KIND == 1 ? SMALL_CTA_THREADS / 32 : 32;
  extern __shared__ __align__(16) uint32_t s_bits[];
  __shared__ long long s_item;
  __shared__ int s_tail, s_next, s_hit, s_ok;
  __shared__ unsigned long long s_pos;
  __shared__ uint32_t s_stage[WARPS][WC ? 1 : STAGE];
  // heavy in-lists of the current level, expanded by all warps together
  __shared__ uint32_t s_hlo[WC ? 1 : CTA_HEAVY_CAP], s_hhi[WC ? 1 : CTA_HEAVY_CAP];
  __shared__ int s_hpref[WC ? 1 : CTA_HEAVY_CAP];
  __shared__ int s_nheavy, s_htotal, s_hnext;
  // weighted cascade: queue head, and nodes queued or being expanded
  __shared__ int s_head, s_pending;
  const int tid = threadIdx.x, lane = tid & 31, nthr = blockDim.x;
  const int64_t n = J.g.n;
  const int64_t qcap = KIND == 1 ? (int64_t)J.small_qcap : n;
  uint32_t* bits = SMEM_BITMAP ? s_bits
                   : (KIND == 1 ? J.small_bitmap : J.slot_bitmap) + (size_t)blockIdx.x * (size_t)J.bitmap_words;
  int32_t* Q = (KIND == 1 ? J.small_queue : J.slot_queue) + (size_t)blockIdx.x * (size_t)qcap;
  uint32_t* stage = s_stage[tid >> 5];
  if (SMEM_BITMAP)
    for (int64_t i = tid; i < J.bitmap_words; i += nthr) bits[i] = 0u;
  unsigned long long* work = KIND == 2 ? &J.ctr->big2_work : &J.ctr->big_work;
  const int64_t* list = KIND == 2 ? J.big2_list : J.big_list;
  const long long big_count =
      (long long)*((volatile unsigned long long*)(KIND == 2 ? &J.ctr->big2_count : &J.ctr->big_count));
  unsigned long long ev = 0, nv = 0, dr = 0;
  __syncthreads();
  for (;;) {
    if (tid == 0) s_item = (long long)atomicAdd(work, 1ull);
    __syncthreads();
    const long long item = s_item;
    if (item >= big_count) break;
    const int64_t j = list[item];
    const int32_t root = pick_root(J, j);
    if (tid == 0) {
      bits[root >> 5] |= 1u << (root & 31);
      Q[0] = root;
      s_tail = 1;
      s_hit = (MODE == MODE_HIT) && test_bit(J.seed_bits, (uint32_t)root);
    }
    __syncthreads();
    if (J.model == 0) {
      const SampleConst sc = sample_const(J.rk, (uint32_t)j, ctr_word3(WC ? PURPOSE_SKIP : PURPOSE_IC, J.stream, j));
      // a stale 0 only costs a draw; bits are never cleared during a sample.  With the
      // bitmap in global memory the check would cost an L2 round trip per group, more
      // than the draw it can save, so only the shared-memory bitmap is consulted.
      auto known = [&](uint32_t u) -> bool {
        if (!SMEM_BITMAP) return false;
        return (bits[u >> 5] >> (u & 31)) & 1u;
      };
      auto visit = [&](uint32_t u, unsigned lt_mask) -> bool {
        bool is_new = false;
        if (u != NO_NODE) {
          const uint32_t mask = 1u << (u & 31);
          is_new = !(atomicOr(bits + (u >> 5), mask) & mask);
        }
        const unsigned m = __ballot_sync(FULL_MASK, is_new);
        int base = 0;
        if (m) {
          if (lane == 0) {
            if (WC) atomicAdd(&s_pending, __popc(m));  // before the producer's own chunk is retired
            base = atomicAdd(&s_tail, __popc(m));
          }
          base = __shfl_sync(FULL_MASK, base, 0);
          if (is_new) {
            const int pos = base + __popc(m & lt_mask);
            if (KIND != 1 || pos < qcap) Q[pos] = (int32_t)u;
            if (MODE == MODE_HIT && test_bit(J.seed_bits, u)) s_hit = 1;
          }
        }
        if (KIND == 1 && base + __popc(m) > qcap) return true;  // outgrew the small queue
        if (MODE == MODE_HIT) return __any_sync(FULL_MASK, *(volatile int*)&s_hit != 0);
        return false;
      };
      if constexpr (WC) {
        // Weighted cascade without level barriers: any visiting order reaches
        // the same set (the gaps are keyed per node), so the warps pull queued
        // nodes as they appear.  s_pending counts the nodes queued or being walked: a
        // lane's new nodes are added before its node is retired, so s_pending
        // reaches 0 only when nothing is queued and no lane holds a node, and
        // the sample ends there.  A queue slot reads -1 until its node is
        // written, so a claimed slot whose writer has reserved but not yet
        // stored it is waited for.
        auto stopped = [&]() -> bool {
          return (MODE == MODE_HIT && *(volatile int*)&s_hit) || (KIND == 1 && *(volatile int*)&s_tail > qcap);
        };
        if (tid == 0) {
          s_head = 0;
          s_pending = 1;  // the root
        }
        __syncthreads();
        const int qlim = (int)(qcap < 0x7FFFFFFF ? qcap : 0x7FFFFFFF);  // queue slots that can be written
        long long idle = 0;
        // Every lane holds at most one node and takes one walk step per round;
        // lanes without a node claim the next queued ones at the start of a
        // round (one claim per warp, taken by lane 0 and broadcast, so the warp
        // stays converged for the shuffles and ballots below).  A node is
        // retired from s_pending when its walk is done, after the nodes it
        // queued were added.
        const unsigned lt_mask = (1u << lane) - 1u;
        int32_t v = -1;
        GapWalk w;
        uint64_t own[31];  // powers of a weighted-cascade in-degree beyond the graph's table
        for (;;) {
          if (__any_sync(FULL_MASK, stopped())) break;
          const bool need = v < 0;
          const unsigned nm = __ballot_sync(FULL_MASK, need);
          int h = 0, cnt = 0;
          if (lane == 0 && nm) {
            const int want = __popc(nm);
            for (;;) {
              h = *(volatile int*)&s_head;
              const int avail = min(*(volatile int*)&s_tail, qlim) - h;
              cnt = avail < want ? avail : want;
              if (cnt <= 0 || atomicCAS(&s_head, h, h + cnt) == h) break;
            }
          }
          h = __shfl_sync(FULL_MASK, h, 0);
          cnt = __shfl_sync(FULL_MASK, cnt, 0);
          bool empty = false;  // took a node that has no in-edges (or whose slot never arrived)
          if (need) {
            const int r = __popc(nm & lt_mask);
            if (r < cnt) {
              int32_t x;
              // the slot's writer has reserved it; wait (briefly) for its store
              for (long long t = 0; (x = *(volatile int32_t*)&Q[h + r]) < 0; ++t) {
                if (t > (1ll << 22)) {
                  atomicCAS(&J.ctr->error, 0u, SAMPLER_ERR_SLOT);
                  x = -1;
                  break;
                }
              }
              if (x >= 0 && walk_begin(w, J.g, x, own)) v = x;
              else empty = true;
              if (x >= 0) ev += w.d;
            }
          }
          uint32_t u = NO_NODE;
          bool fin = false;
          if (v >= 0) {
            bool more = true;
            u = walk_step(w, J.g, v, J.rk, sc, dr, &more);
            if (!more) {
              v = -1;
              fin = true;
            }
          }
          if (visit(u, lt_mask)) break;
          const int nret = __popc(__ballot_sync(FULL_MASK, fin || empty));
          if (lane == 0 && nret) {
            __threadfence_block();  // the nodes they queued before they are retired
            atomicSub(&s_pending, nret);
          }
          if (cnt > 0 || nret > 0 || __any_sync(FULL_MASK, v >= 0)) {
            idle = 0;
            continue;
          }
          // nothing held and nothing to claim: the sample is done once nothing is pending
          if (__any_sync(FULL_MASK, *(volatile int*)&s_pending == 0)) break;
          if (++idle > (1ll << 24)) {  // far longer than any sample: give up and report
            if (lane == 0) atomicCAS(&J.ctr->error, 0u, SAMPLER_ERR_IDLE);
            break;
          }
          __nanosleep(64);
        }
        __syncthreads();
      } else {
      const int wid = tid >> 5;
      auto take_heavy = [&](int32_t, uint32_t lo, uint32_t hi, int) -> int {
        const int slot = atomicAdd(&s_nheavy, 1);
        if (slot >= CTA_HEAVY_CAP) return 0;  // list full: this warp expands it itself
        s_hlo[slot] = lo;
        s_hhi[slot] = hi;
        ev += hi - lo;
        return HEAVY_SKIP;
      };
      if (tid == 0) s_nheavy = 0;
      int lvl_begin = 0, lvl_end = 1;
      for (;;) {
        // every thread is past the previous barrier and nobody writes s_hit
        // until the next one, so this exit test is uniform across the CTA
        if (lvl_begin >= lvl_end || s_hit || (KIND == 1 && s_tail > qcap)) break;
        if (tid == 0) s_next = lvl_begin;
        __syncthreads();
        for (;;) {
          int b = 0;
          if (lane == 0) b = atomicAdd(&s_next, 32);
          b = __shfl_sync(FULL_MASK, b, 0);
          if (b >= lvl_end) break;
          const int cnt = min(32, lvl_end - b);
          const int32_t v = (lane < cnt) ? Q[b + lane] : -1;
          if (expand_ic(J.g, v, J.rk, sc, lane, stage, ev, dr, CTA_HEAVY_GROUPS, known, visit, take_heavy))
            break;
        }
        __syncthreads();
        const int nh = min(s_nheavy, CTA_HEAVY_CAP);
        if (nh > 0 && !s_hit && !(KIND == 1 && s_tail > qcap)) {
          // groups of the heavy in-lists, dealt to all warps 32 at a time
          if (wid == 0) {
            int carry = 0;
            for (int base = 0; base < nh; base += 32) {
              const int i = base + lane;
              const int ng = i < nh ? (int)(((s_hhi[i] + 3) >> 2) - (s_hlo[i] >> 2)) : 0;
              const int incl = warp_inclusive_scan(ng, lane);
              if (i < nh) s_hpref[i] = carry + incl - ng;
              carry += __shfl_sync(FULL_MASK, incl, 31);
            }
            if (lane == 0) {
              s_htotal = carry;
              s_hnext = 0;
            }
          }
          __syncthreads();
          const int htotal = s_htotal;
          for (;;) {
            int c = 0;
            if (lane == 0) c = atomicAdd(&s_hnext, 32);
            c = __shfl_sync(FULL_MASK, c, 0);
            if (c >= htotal) break;
            const int q = c + lane;
            int it = 0;  // last heavy list whose first group is <= q
            for (int step = CTA_HEAVY_CAP / 2; step; step >>= 1)
              if (it + step < nh && s_hpref[it + step] <= q) it += step;
            const uint32_t olo = s_hlo[it], ohi = s_hhi[it];
            const uint32_t grp = (olo >> 2) + (uint32_t)(q - s_hpref[it]);
            if (process_slab(J.g, q < htotal, grp, olo, ohi, J.rk, sc, lane, stage, dr, known, visit))
              break;
          }
        }
        __syncthreads();
        if (tid == 0) s_nheavy = 0;
        lvl_begin = lvl_end;
        lvl_end = s_tail;
        __syncthreads();
      }
      }
    } else if (tid == 0) {
      const SampleConst sc = sample_const(J.rk, (uint32_t)j, ctr_word3(PURPOSE_LT, J.stream, j));
      int32_t cur = root;
      int tail = 1;
      bool hit = s_hit != 0;
      while (!hit) {
        const int64_t lo = J.g.off[cur], hi = J.g.off[cur + 1];
        if (hi == lo) break;
        const uint4 r = philox_x((uint32_t)cur, sc, J.rk);
        int64_t pick = -1;
        if (!J.lt_cumulative) {
          pick = lo + __umulhi(r.x, (uint32_t)(hi - lo));
        } else {
          unsigned long long cum = 0;
          for (int64_t e = lo; e < hi; ++e) {
            cum += J.g.edge[e].y;
            if ((unsigned long long)r.x < cum) {
              pick = e;
              break;
            }
          }
          if (pick < 0) break;
        }
        const int32_t u = (int32_t)J.g.edge[pick].x;
        ev += 1;
        dr += 1;
        const uint32_t mask = 1u << (u & 31);
        if (bits[u >> 5] & mask) break;
        if (KIND == 1 && tail >= qcap) {
          tail = (int)qcap + 1;  // outgrew the small queue
          break;
        }
        bits[u >> 5] |= mask;
        Q[tail++] = u;
        if (MODE == MODE_HIT) hit = test_bit(J.seed_bits, (uint32_t)u);
        cur = u;
      }
      s_tail = tail;
      s_hit = hit;
    }
    __syncthreads();
    const int tail = s_tail;
    if (KIND == 1 && tail > qcap) {
      // the set outgrew this stage's queue: full-size CTAs redo it; clear the whole bitmap
      if (tid == 0) {
        const unsigned long long b = atomicAdd(&J.ctr->big2_count, 1ull);
        J.big2_list[b] = j;
      }
      for (int64_t i = tid; i < J.bitmap_words; i += nthr) bits[i] = 0u;
      if (WC && J.model == 0)
        for (int64_t i = tid; i < qcap; i += nthr) Q[i] = -1;  // the queue's "not written yet" marks
      __syncthreads();
      continue;
    }
    if (MODE == MODE_STORE) {
      if (tid == 0) {
        unsigned long long pos = 0;
        s_ok = reserve(J, j, tail, &pos);
        s_pos = pos;
      }
      __syncthreads();
      if (s_ok) {
        const unsigned long long pos = s_pos;
        for (int i = tid; i < tail; i += nthr) {
          J.pool_nodes[pos + i] = Q[i];
          J.pool_samp[pos + i] = (int32_t)j;
        }
        if (tid == 0) {
          J.set_start[j] = (int64_t)pos;
          J.set_len[j] = tail;
        }
      }
    } else if (tid == 0) {
      J.hit[j - J.j0] = s_hit ? 1 : 0;
    }
    if (tid == 0) nv += (unsigned long long)tail;
    // reset the visited bits of this sample only (and, for the weighted-cascade
    // IC path, the queue's "not written yet" marks)
    const bool marks = WC && J.model == 0;
    if ((int64_t)tail * 8 < J.bitmap_words) {
      for (int i = tid; i < tail; i += nthr) {
        bits[Q[i] >> 5] = 0u;
        if (marks) Q[i] = -1;
      }
    } else {
      for (int64_t i = tid; i < J.bitmap_words; i += nthr) bits[i] = 0u;
      if (marks)
        for (int i = tid; i < tail; i += nthr) Q[i] = -1;
    }
    __syncthreads();
  }
  flush_stats(J.ctr, ev, nv, dr, lane, true);
}

}  // namespace

constexpr int64_t SMEM_BITMAP_MAX_BYTES = 192 * 1024;

LaunchCfg sampler_config(const GraphView& g, int model, bool wc) {
  LaunchCfg c;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = 0;
  if (model == 0 && wc)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sample_warp_ic<MODE_STORE, 0, true>, WT_WARPS * 32, 0);
  else if (model == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sample_warp_ic<MODE_STORE, 0, false>, WT_WARPS * 32,
                                                  0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sample_warp_lt<MODE_STORE>, WT_WARPS * 32, 0);
  if (per_sm < 1) per_sm = 1;
  c.warp_blocks = c.num_sms * per_sm;
  const int64_t words = (g.n + 31) / 32;
  c.smem_bitmap_bytes = words * 4;
  c.cta_smem_bitmap = c.smem_bitmap_bytes <= SMEM_BITMAP_MAX_BYTES;
  c.cta_threads = 1024;
  c.cta_blocks = c.num_sms;
  if (!c.cta_smem_bitmap) {
    // global bitmap: many small CTAs first, a few full-size ones for the largest sets
    int small_per_sm = 0;
    if (model == 0 && wc)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&small_per_sm, k_sample_cta<MODE_STORE, false, 1, true>,
                                                    SMALL_CTA_THREADS, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&small_per_sm, k_sample_cta<MODE_STORE, false, 1, false>,
                                                    SMALL_CTA_THREADS, 0);
    if (small_per_sm < 1) small_per_sm = 1;
    c.small_blocks = c.num_sms * small_per_sm;
    c.small_qcap = (int)std::min<int64_t>(g.n, 1 << 20);
    c.cta_blocks = std::max(8, c.num_sms / 4);
  }
  c.mid_blocks = c.num_sms * 2;  // 16 warps per SM, each with its own global hash and queue
  // global-bitmap warp tier (weighted-cascade IC, bitmap in global memory): 32
  // warps per SM, each with an n-bit bitmap and a GQ_SLOTS queue, or 16 where
  // the bitmaps would pass 24 GB
  if (model == 0 && wc) {
    int lane_per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&lane_per_sm, k_sample_lane_wc<MODE_STORE>, 256, 0);
    c.lane_blocks = c.num_sms * (lane_per_sm < 1 ? 1 : lane_per_sm);
  }
  if (model == 0 && wc && !c.cta_smem_bitmap) {
    const double per_block = (double)words * 4.0 * WT_WARPS;
    c.wg_blocks = c.num_sms * ((double)c.num_sms * 4 * per_block <= 24e9 ? 4 : 2);
  }
  return c;
}

size_t mid_tier_words(const LaunchCfg& c) { return (size_t)c.mid_blocks * WT_WARPS; }
size_t wg_tier_warps(const LaunchCfg& c) { return (size_t)c.wg_blocks * WT_WARPS; }
size_t wg_queue_per_warp() { return GQ_SLOTS; }
int mid_tier_max_cap() { return Tier<1>::QCAP; }
size_t mid_hash_per_warp() { return MID_HASH; }
size_t mid_queue_per_warp() { return MID_QSLOTS; }

size_t sampler_scratch_bytes(const GraphView& g, const LaunchCfg& c) {
  const size_t words = (size_t)((g.n + 31) / 32);
  size_t per_slot = (size_t)g.n * 4 + (c.cta_smem_bitmap ? 0 : words * 4);
  return per_slot * (size_t)c.cta_blocks + ((size_t)c.small_qcap * 4 + words * 4) * (size_t)c.small_blocks;
}

template <int MODE, bool WC>
static void launch_warp_ic(const SampleJob& J, const LaunchCfg& c, cudaStream_t st) {
  const dim3 block(WT_WARPS * 32);
  k_sample_warp_ic<MODE, 0, WC><<<c.warp_blocks, block, 0, st>>>(J);
  if (J.mid_cap > 0) k_sample_warp_ic<MODE, 1, WC><<<c.mid_blocks, block, 0, st>>>(J);
}

cudaError_t launch_sample_warp(const SampleJob& J, const LaunchCfg& c, cudaStream_t st) {
  const dim3 grid(c.warp_blocks), block(WT_WARPS * 32);
  if (J.model == 0 && J.wc_implicit && J.lane_tier) {
    if (J.mode == MODE_STORE) k_sample_lane_wc<MODE_STORE><<<c.lane_blocks, 256, 0, st>>>(J);
    else k_sample_lane_wc<MODE_HIT><<<c.lane_blocks, 256, 0, st>>>(J);
  }
  if (J.model == 0 && J.wc_implicit && J.warp_global && c.wg_blocks > 0) {
    if (J.mode == MODE_STORE) k_sample_warp_wcg<MODE_STORE><<<c.wg_blocks, block, 0, st>>>(J);
    else k_sample_warp_wcg<MODE_HIT><<<c.wg_blocks, block, 0, st>>>(J);
  } else if (J.model == 0) {
    if (J.mode == MODE_STORE) {
      if (J.wc_implicit) launch_warp_ic<MODE_STORE, true>(J, c, st);
      else launch_warp_ic<MODE_STORE, false>(J, c, st);
    } else {
      if (J.wc_implicit) launch_warp_ic<MODE_HIT, true>(J, c, st);
      else launch_warp_ic<MODE_HIT, false>(J, c, st);
    }
  } else {
    if (J.mode == MODE_STORE) k_sample_warp_lt<MODE_STORE><<<grid, block, 0, st>>>(J);
    else k_sample_warp_lt<MODE_HIT><<<grid, block, 0, st>>>(J);
  }
  return cudaGetLastError();
}

template <int MODE, bool SB, bool WC>
static cudaError_t launch_cta_t(const SampleJob& J, const LaunchCfg& c, cudaStream_t st) {
  if (SB) {
    const size_t smem = (size_t)c.smem_bitmap_bytes;
    cudaError_t e = cudaFuncSetAttribute(k_sample_cta<MODE, true, 0, WC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sample_cta<MODE, true, 0, WC><<<c.cta_blocks, c.cta_threads, smem, st>>>(J);
  } else {
    k_sample_cta<MODE, false, 1, WC><<<c.small_blocks, SMALL_CTA_THREADS, 0, st>>>(J);
    k_sample_cta<MODE, false, 2, WC><<<c.cta_blocks, c.cta_threads, 0, st>>>(J);
  }
  return cudaGetLastError();
}

template <int MODE, bool SB>
static cudaError_t launch_cta_w(const SampleJob& J, const LaunchCfg& c, cudaStream_t st) {
  // the LT walk reads no thresholds: one instantiation serves it
  return (J.model == 0 && J.wc_implicit) ? launch_cta_t<MODE, SB, true>(J, c, st)
                                         : launch_cta_t<MODE, SB, false>(J, c, st);
}

cudaError_t launch_sample_cta(const SampleJob& J, const LaunchCfg& c, cudaStream_t st) {
  if (J.mode == MODE_STORE)
    return c.cta_smem_bitmap ? launch_cta_w<MODE_STORE, true>(J, c, st) : launch_cta_w<MODE_STORE, false>(J, c, st);
  return c.cta_smem_bitmap ? launch_cta_w<MODE_HIT, true>(J, c, st) : launch_cta_w<MODE_HIT, false>(J, c, st);
}

}  // namespace ssa
