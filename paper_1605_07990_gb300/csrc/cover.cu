// RR pool index, greedy Max-Coverage (Algorithm 2), coverage checks (Eq. 1)
// and the Estimate-Inf first-T search (Algorithm 3) on sm_103a.
//
// Index: cnt[v] = number of sets holding v by a counting pass over the flat
// (node, sample) entries, exclusive scan into inv_off, scatter of sample ids
// into inv_samp (order inside a list is irrelevant: each step only needs the
// set of samples holding the picked node).
// Greedy: one persistent cooperative kernel for all k picks; a pick is the
// maximum packed key (gain+1)<<32 | ~v (largest gain, then smallest id; picked
// nodes keyed to 0), then warps decrement the gains of the members of each
// newly covered set.
#include <atomic>
#include <mutex>

#include <cooperative_groups.h>

#include "device.cuh"

namespace ssa {

namespace {

constexpr int TPB = 256;

// samp == nullptr: every entry in [e0, e1) counts; else only samples in [jlo, jhi)
// Index build.  Hubs appear in a large share of the sets, so the lanes of a
// warp that hold the same node are grouped (labeled_partition) and one of
// them issues the group's atomic: one atomic per distinct node per warp
// instead of one per entry on the hub's counter.
__global__ void k_count_nodes(const int32_t* __restrict__ nodes, const int32_t* __restrict__ samp, int64_t e0,
                              int64_t e1, int64_t jlo, int64_t jhi, int32_t* cnt) {
  namespace cg = cooperative_groups;
  for (int64_t q = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < e1; q += (int64_t)gridDim.x * blockDim.x) {
    if (samp) {
      const int64_t s = samp[q];
      if (s < jlo || s >= jhi) continue;
    }
    const int32_t v = nodes[q];
    const cg::coalesced_group same = cg::labeled_partition(cg::coalesced_threads(), v);
    if (same.thread_rank() == 0) atomicAdd(cnt + v, (int)same.size());
  }
}

__global__ void k_scatter_index(const int32_t* __restrict__ nodes, const int32_t* __restrict__ samp, int64_t e0,
                                int64_t e1, int64_t jlo, int64_t jhi, unsigned long long* cur, int32_t* inv_samp) {
  namespace cg = cooperative_groups;
  for (int64_t q = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < e1;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = samp[q];
    if (s < jlo || s >= jhi) continue;
    const int32_t v = nodes[q];
    const cg::coalesced_group same = cg::labeled_partition(cg::coalesced_threads(), v);
    unsigned long long pos = 0;
    if (same.thread_rank() == 0) pos = atomicAdd(cur + v, (unsigned long long)same.size());
    pos = same.shfl(pos, 0) + same.thread_rank();
    inv_samp[pos] = s;
  }
}

// ---- block-wide helpers ----
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T x, T* s_warp, T* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T incl = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T t = __shfl_up_sync(FULL_MASK, incl, d);
    if (lane >= d) incl += t;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    T w = lane < nw ? s_warp[lane] : (T)0;
    T wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const T t = __shfl_up_sync(FULL_MASK, wi, d);
      if (lane >= d) wi += t;
    }
    if (lane < nw) s_warp[lane] = wi - w;
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  const T r = s_warp[wid] + incl - x;
  __syncthreads();
  return r;
}

constexpr int SCAN_TILE = 4096;  // 1024 threads x 4

__global__ void __launch_bounds__(1024) k_tile_sums(const int32_t* in, int64_t n, long long* part) {
  __shared__ long long s_w[32];
  __shared__ long long s_tot;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  long long sum = 0;
  for (int i = threadIdx.x; i < SCAN_TILE; i += blockDim.x)
    if (base + i < n) sum += in[base + i];
  block_exclusive_scan<long long>(sum, s_w, &s_tot);
  if (threadIdx.x == 0) part[blockIdx.x] = s_tot;
}

__global__ void __launch_bounds__(1024) k_scan_parts(long long* part, int64_t tiles) {
  __shared__ long long s_w[32];
  __shared__ long long s_tot;
  long long carry = 0;
  for (int64_t b = 0; b < tiles; b += blockDim.x) {
    const int64_t i = b + threadIdx.x;
    const long long x = i < tiles ? part[i] : 0;
    const long long ex = block_exclusive_scan<long long>(x, s_w, &s_tot);
    if (i < tiles) part[i] = carry + ex;
    carry += s_tot;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024) k_tile_scan(const int32_t* in, int64_t n, const long long* part,
                                                    int64_t* out) {
  __shared__ long long s_w[32];
  __shared__ long long s_tot;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * 4;
  long long v[4], loc = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    v[t] = (base + t < n) ? in[base + t] : 0;
    loc += v[t];
  }
  long long ex = block_exclusive_scan<long long>(loc, s_w, &s_tot) + part[blockIdx.x];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (base + t < n) out[base + t] = ex;
    ex += v[t];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = part[blockIdx.x] + s_tot;
}

// ---- greedy ----

// maximum (or sum) over the block of x, in every thread
template <bool SUM>
__device__ __forceinline__ unsigned long long block_reduce(unsigned long long x, unsigned long long* s) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int d = 16; d; d >>= 1) {
    const unsigned long long t = __shfl_xor_sync(FULL_MASK, x, d);
    x = SUM ? x + t : (t > x ? t : x);
  }
  if (lane == 0) s[wid] = x;
  __syncthreads();
  if (wid == 0) {
    x = lane < nw ? s[lane] : 0ull;
#pragma unroll
    for (int d = 16; d; d >>= 1) {
      const unsigned long long t = __shfl_xor_sync(FULL_MASK, x, d);
      x = SUM ? x + t : (t > x ? t : x);
    }
    if (lane == 0) s[0] = x;
  }
  __syncthreads();
  x = s[0];
  __syncthreads();
  return x;
}
__device__ __forceinline__ unsigned long long block_max(unsigned long long x, unsigned long long* s) {
  return block_reduce<false>(x, s);
}

// sync layout: arrival count, release word and timeout flag on separate
// 128-byte lines so that polling does not contend with the arrivals.
constexpr int SYNC_COUNT = 0, SYNC_GEN = 32, SYNC_ERR = 64, SYNC_CHUNKS = 96;
constexpr int DEC_CHUNK = 2048;    // covered sets longer than this are decremented in chunks by all warps
constexpr int CACHE_MAX = 8192;    // greedy candidate cache entries
constexpr int ARGMAX_STRIDE = 16;  // argmax slots one 128-byte line apart
constexpr int HBINS = 4096;        // gain histogram: gain g >= floor counts in bin min(g - floor, HBINS - 1)
constexpr unsigned long long PENDING = 1ull << 62;  // barrier payload flag: decrement chunks are queued
constexpr unsigned long long RECOUNT = 1ull << 61;  // with PENDING: recount the gains instead of draining
// per-block entry tallies (64-bit slots after the argmax slots): entries of
// all sets the block covered so far, and entries it queued in the last pick
// that queued any
constexpr int ACC_DONE = 64, ACC_QUEUED = 64 + 1024;

// Grid barrier for a cooperative launch.  The last block to arrive runs f()
// (all its threads; f sees every block's writes from before the barrier) and
// publishes the result (< 2^63) in the release word beside a sense bit (bit 0,
// flipped by each release), so every waiter learns it from the poll that
// releases it; all threads get it in `info`.  A wait gives up after `limit`
// polls (about a second by default), sets sync[SYNC_ERR] and returns false;
// that block then leaves the kernel, and the others give up at their next
// barrier, which it never reaches.  Every block passes every barrier in the
// same order, so each keeps the current sense in its shared `phase` (0 at
// launch, when the release word is zero) instead of reading it back.
template <class F>
__device__ __forceinline__ bool grid_barrier(unsigned int* sync, unsigned int* phase, long long limit, F&& f,
                                             unsigned long long& info) {
  __shared__ unsigned long long s_info;
  __shared__ unsigned int s_last, s_ok, s_sense;
  volatile unsigned long long* gw = reinterpret_cast<volatile unsigned long long*>(sync + SYNC_GEN);
  __syncthreads();
  if (threadIdx.x == 0) {
    s_sense = *phase;
    *phase = s_sense ^ 1u;
    s_ok = 1;
    __threadfence();
    const bool last = atomicAdd(sync + SYNC_COUNT, 1u) + 1u == gridDim.x;
    if (last) {
      atomicExch(sync + SYNC_COUNT, 0u);
      __threadfence();
    }
    s_last = last;
  }
  __syncthreads();
  if (s_last) {
    const unsigned long long r = f();
    if (threadIdx.x == 0) {
      atomicExch((unsigned long long*)gw, (r << 1) | (unsigned long long)(s_sense ^ 1u));
      s_info = r;
    }
  } else if (threadIdx.x == 0) {
    unsigned long long w;
    unsigned int ns = 8;
    for (long long spins = 0; (unsigned int)((w = *gw) & 1ull) == s_sense; ++spins) {
      if (spins > limit) {  // by default seconds: a barrier never takes that long
        atomicExch(sync + SYNC_ERR, 1u);
        s_ok = 0;
        break;
      }
      __nanosleep(ns);
      if (ns < 128) ns <<= 1;
    }
    s_info = w >> 1;
    __threadfence();
  }
  __syncthreads();
  info = s_info;
  return s_ok != 0u;
}

// The greedy's barrier.  GRID: grid_barrier across a cooperative launch.
// CLUSTER: the whole greedy runs in one thread-block cluster, so the barrier is
// the hardware cluster barrier; block 0 then computes f() and the others read
// its result from block 0's shared memory (distributed shared memory) after a
// second cluster barrier.  A cluster barrier always completes (the cluster's
// blocks are scheduled together), so it has no bound to reach.
template <bool CLUSTER, class F>
__device__ __forceinline__ bool greedy_barrier(const GreedyJob& J, unsigned int* phase, F&& f,
                                               unsigned long long& info) {
  if constexpr (!CLUSTER) {
    return grid_barrier(J.sync, phase, J.wait_polls, f, info);
  } else {
    namespace cg = cooperative_groups;
    __shared__ unsigned long long s_res;
    cg::cluster_group cluster = cg::this_cluster();
    __threadfence();  // this block's global writes and atomics before the others look
    cluster.sync();
    if (cluster.block_rank() == 0) {
      const unsigned long long r = f();
      if (threadIdx.x == 0) s_res = r;
    }
    cluster.sync();
    info = *cluster.map_shared_rank(&s_res, 0);
    return true;
  }
}

// Packed argmax key: larger gain first, then smaller id; picked nodes (negative
// gain) key to 0.  With gains below 2^31 - 1 and ids below 2^31, keys stay
// below 2^62, under the barrier payload's PENDING flag.
__device__ __forceinline__ unsigned long long gain_key(int32_t c, uint32_t v) {
  return c < 0 ? 0ull : (((unsigned long long)(uint32_t)(c + 1)) << 31) | (unsigned long long)(0x7FFFFFFFu - v);
}
__device__ __forceinline__ int32_t key_node(unsigned long long key) {
  return (int32_t)(0x7FFFFFFFu - (uint32_t)(key & 0x7FFFFFFFull));
}
__device__ __forceinline__ int32_t key_gain(unsigned long long key) { return (int32_t)(key >> 31) - 1; }

// gains of the `len` members at mem lose one each (a warp, lanes striped)
__device__ __forceinline__ void decrement_members(int32_t* cnt, const int32_t* mem, int32_t len, int lane) {
  int t = lane;
  for (; t + 96 < len; t += 128) {  // four independent loads in flight per lane
    const int32_t a = __ldg(mem + t), b = __ldg(mem + t + 32), c = __ldg(mem + t + 64), d = __ldg(mem + t + 96);
    atomicSub(cnt + a, 1);
    atomicSub(cnt + b, 1);
    atomicSub(cnt + c, 1);
    atomicSub(cnt + d, 1);
  }
  for (; t < len; t += 32) atomicSub(cnt + __ldg(mem + t), 1);
}

// Grid-wide maximum of the threads' keys, in every thread: each block folds
// its own into one of three slots by atomicMax, and the barrier publishes the
// slot.  Argmax number a uses slot a % 3; block 0 clears slot (a + 2) % 3 after
// the barrier, which no block writes before the next barrier has completed.
template <bool CLUSTER>
__device__ __forceinline__ bool grid_argmax(const GreedyJob& J, unsigned long long& best, unsigned long long* s_red,
                                            int& n_argmax, unsigned int* phase) {
  best = block_max(best, s_red);
  const int slot = n_argmax % 3;
  n_argmax += 1;
  unsigned long long* at = J.argmax + slot * ARGMAX_STRIDE;
  if (threadIdx.x == 0 && best != 0ull) atomicMax(at, best);
  if (!greedy_barrier<CLUSTER>(J, phase, [&] { return __ldcg(at); }, best)) return false;
  if (blockIdx.x == 0 && threadIdx.x == 0) J.argmax[((slot + 2) % 3) * ARGMAX_STRIDE] = 0ull;
  return true;
}

// Persistent greedy: all k picks of Algorithm 2 in one cooperative launch.
//
// Argmax.  A pick needs the node of largest gain, then smallest id.  Gains only
// fall, so after a scan of all n nodes that finds the threshold g* with at
// most CACHE_MAX nodes of gain >= g*, those nodes form a candidate cache: while
// the best cached gain is still >= g*, it beats every node outside (all
// <= g* - 1, ties included).  Every block holds the whole cache in shared
// memory, and the last block to reach the barrier that ends a pick computes
// the next pick's argmax over it, published with the release: a cached pick
// costs one grid barrier.  When the best cached gain falls below g*, the pick
// scans all n nodes (a second barrier publishes the maximum of the blocks'
// keys) and builds a new cache from a gain histogram taken in the same pass.
//
// Cover.  Warps walk v*'s inverted lists of all index batches and, for each
// newly covered set, decrement the gains of its members.  Sets longer than
// DEC_CHUNK go whole, as chunks, to a queue that every warp drains after the
// barrier that closes the pick.  When the queued entries outnumber the
// entries of the sets still uncovered (one pick can cover a bulk of huge sets
// that share one core of nodes), the last block at that barrier calls for a
// recount instead: gains are rebuilt from the uncovered sets, which costs
// fewer atomics than the decrements would.  Barrier waits are bounded
// (sync[SYNC_ERR] on timeout).
template <bool CLUSTER>
__global__ void __launch_bounds__(1024, 1) k_greedy(GreedyJob J) {
  __shared__ unsigned long long s_red[32];
  __shared__ int64_t s_lo[GREEDY_MAX_LISTS], s_hi[GREEDY_MAX_LISTS];
  // the gain histogram (HBINS) and the staged cache (CACHE_MAX ids) share
  // space: a histogram is only taken after the cache has been dropped
  __shared__ unsigned int s_buf[CACHE_MAX > HBINS ? CACHE_MAX : HBINS];
  __shared__ long long s_scan[32], s_scan_tot;
  __shared__ unsigned long long s_cov_e, s_queued_e;  // entries of the sets this block covered / queued
  __shared__ unsigned int s_phase;                     // sense of the next grid barrier
  unsigned long long my_done = 0, my_queued = 0;      // thread 0: this block's slot values
  unsigned int* s_hist = s_buf;
  int32_t* s_cache = reinterpret_cast<int32_t*>(s_buf);
  const int lane = threadIdx.x & 31;
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t warp = gtid >> 5, nwarps = gthreads >> 5;
  const int64_t n4 = J.n_pad >> 2;
  const int4* c4 = reinterpret_cast<const int4*>(J.cnt);
  int n_argmax = 0;
  if (threadIdx.x == 0) s_phase = 0u;  // the host zeroed the release word (sense 0)
  // Rebuild policy (every block tracks the same values): the first pick only
  // scans; a rebuild needs at least REBUILD_MIN picks left; a cache that served
  // fewer than REBUILD_MIN picks, or a rebuild that found no threshold,
  // postpones the next rebuild by a doubling back-off.
  constexpr int REBUILD_MIN = 8;
  int rebuilds = 0, next_try = 1, backoff = REBUILD_MIN, built_at = 0, gstar = 0, g_prev = 0;
  bool cached = false, stage = false, fused_ok = false;
  int nc = 0;                          // staged cache entries
  unsigned long long fused_key = 0;    // this pick's argmax, from the previous pick's last barrier
  // block-wide argmax over the staged cache, for the last block at a barrier
  auto cache_argmax = [&]() -> unsigned long long {
    unsigned long long b = 0;
    for (int t = threadIdx.x; t < nc; t += blockDim.x) {
      const int32_t v = s_cache[t];
      const unsigned long long key = gain_key(__ldcg(J.cnt + v), (uint32_t)v);
      b = key > b ? key : b;
    }
    return block_max(b, s_red);
  };
  for (int i = 0; i < J.k; ++i) {
    unsigned long long best = 0;
    bool have = false;
    if (cached) {
      bool valid = false;
      if (stage) {
        // first pick on a new cache: every block stages all of it, and the
        // blocks scan interleaved slices of it for this pick's argmax
        const int cb = (rebuilds - 1) & 1;
        const unsigned int m = __ldcg(J.cache_n + cb);
        nc = m <= (unsigned int)CACHE_MAX ? (int)m : 0;
        const int32_t* cache = J.cache + (size_t)cb * CACHE_MAX;
        for (int t = threadIdx.x; t < nc; t += blockDim.x) s_cache[t] = __ldcg(cache + t);
        __syncthreads();
        stage = false;
        if (m <= (unsigned int)CACHE_MAX) {
          for (int t = blockIdx.x + (int)threadIdx.x * (int)gridDim.x; t < nc; t += (int)(blockDim.x * gridDim.x)) {
            const int32_t v = s_cache[t];
            const unsigned long long key = gain_key(__ldcg(J.cnt + v), (uint32_t)v);
            best = key > best ? key : best;
          }
          if (!grid_argmax<CLUSTER>(J, best, s_red, n_argmax, &s_phase)) return;
          valid = true;
        }
      } else if (fused_ok) {
        best = fused_key;
        valid = true;
      }
      // every block holds the same maximum, so all take the same branch
      have = valid && best != 0 && key_gain(best) >= gstar;
      if (!have) {
        cached = false;
        if (i - built_at < REBUILD_MIN) {
          next_try = i + backoff;
          backoff = min(2 * backoff, 512);
        } else {
          backoff = REBUILD_MIN;
        }
      }
    }
    if (!have) {
      const bool rebuild = i >= next_try && J.k - i >= REBUILD_MIN;
      // the histogram counts gains >= floor only (bin c - floor, the top bin
      // "at least"): the cache threshold sits near the top, and low gains,
      // the bulk of the nodes, would only contend on a few bins
      const int floor_g = max(1, g_prev >> 2);
      const int hb = rebuilds & 1;
      if (rebuild) {
        for (int t = threadIdx.x; t < HBINS; t += blockDim.x) s_hist[t] = 0u;
        __syncthreads();
      }
      best = 0;
      for (int64_t q = gtid; q < n4; q += gthreads) {
        const int4 c = __ldcg(c4 + q);
        const uint32_t v = (uint32_t)(q * 4);
        unsigned long long key;
        key = gain_key(c.x, v);     best = key > best ? key : best;
        key = gain_key(c.y, v + 1); best = key > best ? key : best;
        key = gain_key(c.z, v + 2); best = key > best ? key : best;
        key = gain_key(c.w, v + 3); best = key > best ? key : best;
        if (rebuild) {
          if (c.x >= floor_g) atomicAdd(s_hist + min(c.x - floor_g, HBINS - 1), 1u);
          if (c.y >= floor_g) atomicAdd(s_hist + min(c.y - floor_g, HBINS - 1), 1u);
          if (c.z >= floor_g) atomicAdd(s_hist + min(c.z - floor_g, HBINS - 1), 1u);
          if (c.w >= floor_g) atomicAdd(s_hist + min(c.w - floor_g, HBINS - 1), 1u);
        }
      }
      if (rebuild) {
        unsigned int* h = J.hist + (size_t)hb * HBINS;
        __syncthreads();
        for (int t = threadIdx.x; t < HBINS; t += blockDim.x)
          if (s_hist[t]) atomicAdd(h + t, s_hist[t]);
      }
      if (!grid_argmax<CLUSTER>(J, best, s_red, n_argmax, &s_phase)) return;
      if (rebuild) {
        // g* = floor + the smallest bin b with at most CACHE_MAX nodes in
        // bins >= b: a descending block scan of the merged histogram (thread t
        // holds bins HBINS-1-PER*t down to HBINS-PER*(t+1)); none when the
        // top bin alone holds too many nodes
        constexpr int PER = HBINS / 1024;
        const unsigned int* h = J.hist + (size_t)hb * HBINS;
        const int top = HBINS - 1 - (int)threadIdx.x * PER;
        unsigned int hv[PER];
        long long mine = 0;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          hv[u] = __ldcg(h + top - u);
          mine += hv[u];
        }
        long long above = block_exclusive_scan<long long>(mine, s_scan, &s_scan_tot);
        unsigned long long key = 0;  // HBINS - b of the smallest qualifying bin
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          above += hv[u];
          if (above <= (long long)CACHE_MAX) key = (unsigned long long)(HBINS - (top - u));
        }
        key = block_max(key, s_red);
        int g = key ? floor_g + (HBINS - (int)key) : 0;
        // a threshold above the best gain would leave the best node outside
        if (g > key_gain(best)) g = 0;
        if (g > 0) {
          // Some blocks may already be covering for this pick, so a gain read
          // here may have fallen since the scan: below g* it stays below for
          // good; at or above g* it was counted in the histogram, which bounds
          // the cache at CACHE_MAX entries.
          const int32_t vstar = key_node(best);
          unsigned int* nout = J.cache_n + hb;
          int32_t* out = J.cache + (size_t)hb * CACHE_MAX;
          // warp-uniform trip count, so the ballots below see all 32 lanes
          for (int64_t q0 = gtid - lane; q0 < n4; q0 += gthreads) {
            const int64_t q = q0 + lane;
            int4 c = make_int4(-1, -1, -1, -1);
            if (q < n4) c = __ldcg(c4 + q);
            const int32_t v = (int32_t)(q * 4);
            const int32_t cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const bool take = cv[u] >= g && v + u != vstar;
              const unsigned int m = __ballot_sync(FULL_MASK, take);
              if (m == 0u) continue;
              const int leader = __ffs(m) - 1;
              unsigned int at = 0;
              if (lane == leader) at = atomicAdd(nout, (unsigned int)__popc(m));
              at = __shfl_sync(FULL_MASK, at, leader) + (unsigned int)__popc(m & ((1u << lane) - 1u));
              if (take && at < (unsigned int)CACHE_MAX) out[at] = v + u;
            }
          }
          gstar = g;
          cached = true;
          built_at = i;
          stage = true;
        } else {
          next_try = i + backoff;  // the top is too flat: full scans for a while
          backoff = min(2 * backoff, 512);
        }
        // this parity's histogram and cache stay read-only until the next
        // rebuild, which uses the other parity: clear that one now (nobody
        // reads it any more: its last staging ended before the barrier above)
        if (blockIdx.x == 0) {
          for (int t = threadIdx.x; t < HBINS; t += blockDim.x) J.hist[(size_t)(hb ^ 1) * HBINS + t] = 0u;
          if (threadIdx.x == 0) J.cache_n[hb ^ 1] = 0u;
        }
        rebuilds += 1;
      }
    }
    const int32_t vstar = key_node(best);
    g_prev = key_gain(best);
    if (threadIdx.x < J.nlists) {
      s_lo[threadIdx.x] = J.lists[threadIdx.x].off[vstar];
      s_hi[threadIdx.x] = J.lists[threadIdx.x].off[vstar + 1];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      J.seeds[i] = vstar;
      J.gains[i] = key_gain(best);
    }
    if (threadIdx.x == 0) {
      s_cov_e = 0ull;
      s_queued_e = 0ull;
    }
    __syncthreads();
    unsigned int* chunks = J.sync + SYNC_CHUNKS + (i & 1) * 16;
    for (int b = 0; b < J.nlists; ++b) {
      const int32_t* samp = J.lists[b].samp;
      for (int64_t q = s_lo[b] + warp; q < s_hi[b]; q += nwarps) {
        const int32_t j = samp[q];
        // the set's extent loads alongside its covered flag (one round trip, not two)
        const uint8_t was = __ldcg(J.covered + j);
        const int32_t len = J.set_len[j];
        const int64_t start = J.set_start[j];
        if (was) continue;
        __syncwarp();
        if (lane == 0) J.covered[j] = 1;
        if (lane == 0) atomicAdd(&s_cov_e, (unsigned long long)len);
        if (len > DEC_CHUNK) {
          // the whole set goes to the queue, for a drain or a recount after the barrier
          const int nq = (len + DEC_CHUNK - 1) / DEC_CHUNK;
          unsigned int at = 0;
          if (lane == 0) {
            at = atomicAdd(chunks, (unsigned int)nq);
            atomicAdd(&s_queued_e, (unsigned long long)len);
          }
          at = __shfl_sync(FULL_MASK, at, 0);
          if ((int64_t)at + nq > J.chunk_cap) {  // cannot happen with the host's sizing
            if (lane == 0) atomicExch(J.sync + SYNC_ERR, 2u);
            continue;
          }
          for (int c = lane; c < nq; c += 32)
            J.chunk_q[at + c] = ((unsigned long long)(uint32_t)j << 32) | (uint32_t)(c * DEC_CHUNK);
          continue;
        }
        decrement_members(J.cnt, J.pool_nodes + start, len, lane);
      }
    }
    // v* leaves the candidates for good (its remaining decrements keep it negative)
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(J.cnt + vstar, INT32_MIN / 2);
    // The barrier that ends the pick also yields the next pick's argmax when
    // the next pick uses a staged cache; queued chunks come first, and then
    // the drain's barrier yields it instead.
    const bool fuse = cached && !stage;
    unsigned long long pay = 0;
    __syncthreads();
    // plain stores to the block's own slots, only when they change
    if (threadIdx.x == 0) {
      if (s_cov_e) {
        my_done += s_cov_e;
        J.argmax[ACC_DONE + blockIdx.x] = my_done;
      }
      if (s_queued_e != my_queued) {
        my_queued = s_queued_e;
        J.argmax[ACC_QUEUED + blockIdx.x] = my_queued;
      }
    }
    if (!greedy_barrier<CLUSTER>(J, &s_phase, [&]() -> unsigned long long {
          const unsigned int m = __ldcg(chunks);
          if (m > 0u) {
            // entries still in uncovered sets after this pick, against the queued ones
            unsigned long long done = 0, q = 0;
            if (threadIdx.x < gridDim.x) {
              done = __ldcg(J.argmax + ACC_DONE + threadIdx.x);
              q = __ldcg(J.argmax + ACC_QUEUED + threadIdx.x);
            }
            done = block_reduce<true>(done, s_red);
            q = block_reduce<true>(q, s_red);
            // a recount costs an increment per entry left, a pass over the sets'
            // flags and the gains, and two more barriers: it must win clearly
            const unsigned long long left = done < J.total_entries ? J.total_entries - done : 0ull;
            const unsigned long long fixed = (unsigned long long)(J.n_sets + J.n_pad) / 8 + (1ull << 20);
            return PENDING | (q > 2 * left + fixed ? RECOUNT : 0ull) | m;
          }
          return fuse ? cache_argmax() : 0ull;
        }, pay)) return;
    // the other parity's queue was drained in the previous pick: reset it for the next one
    if (blockIdx.x == 0 && threadIdx.x == 0) J.sync[SYNC_CHUNKS + ((i + 1) & 1) * 16] = 0u;
    if ((pay & PENDING) && (pay & RECOUNT)) {
      // gains from scratch: zero every unpicked node (picked and padding
      // nodes stay negative), then one increment per member of each set still
      // uncovered; no uncovered set holds a picked node
      for (int64_t q = gtid; q < n4; q += gthreads) {
        int4 c = __ldcg(c4 + q);
        c.x = c.x < 0 ? c.x : 0;
        c.y = c.y < 0 ? c.y : 0;
        c.z = c.z < 0 ? c.z : 0;
        c.w = c.w < 0 ? c.w : 0;
        reinterpret_cast<int4*>(J.cnt)[q] = c;
      }
      unsigned long long unused = 0;
      if (!greedy_barrier<CLUSTER>(J, &s_phase, [] { return 0ull; }, unused)) return;
      for (int64_t j = warp; j < J.n_sets; j += nwarps) {
        if (__ldcg(J.covered + j)) continue;
        const int32_t* mem = J.pool_nodes + J.set_start[j];
        const int32_t len = J.set_len[j];
        for (int t = lane; t < len; t += 32) atomicAdd(J.cnt + __ldg(mem + t), 1);
      }
      if (!greedy_barrier<CLUSTER>(J, &s_phase, [&]() -> unsigned long long { return fuse ? cache_argmax() : 0ull; }, pay)) return;
    } else if (pay & PENDING) {
      const int64_t nchunks = (int64_t)(pay & (RECOUNT - 1ull));
      for (int64_t c = warp; c < nchunks; c += nwarps) {
        const unsigned long long e = J.chunk_q[c];
        const int32_t j = (int32_t)(e >> 32), from = (int32_t)(uint32_t)e;
        const int32_t len = J.set_len[j];
        const int32_t cnt = min(DEC_CHUNK, len - from);
        decrement_members(J.cnt, J.pool_nodes + J.set_start[j] + from, cnt, lane);
      }
      if (!greedy_barrier<CLUSTER>(J, &s_phase, [&]() -> unsigned long long { return fuse ? cache_argmax() : 0ull; }, pay)) return;
    }
    fused_key = pay;
    fused_ok = fuse;
  }
  if constexpr (CLUSTER) {
    // no block may leave while another can still read its shared memory: the
    // payload of the last barrier lives in block 0's
    cooperative_groups::this_cluster().sync();
  }
}

__global__ void k_add_counts(int32_t* __restrict__ total, const int32_t* __restrict__ add, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    total[i] += add[i];
}

// ---- stare ----
__global__ void k_mark_hits(const int32_t* __restrict__ nodes, const int32_t* __restrict__ samp, int64_t e0,
                            int64_t e1, const uint8_t* __restrict__ in_seed, int64_t j0, int64_t j1, uint8_t* hit) {
  for (int64_t q = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < e1;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = samp[q];
    if (s >= j0 && s < j1 && in_seed[nodes[q]]) hit[s - j0] = 1;
  }
}

__global__ void __launch_bounds__(TPB) k_count_flags(const uint8_t* __restrict__ f, int64_t count,
                                                     unsigned long long* out) {
  __shared__ long long s_w[32];
  __shared__ long long s_tot;
  long long c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    c += f[i];
  block_exclusive_scan<long long>(c, s_w, &s_tot);
  if (threadIdx.x == 0 && s_tot) atomicAdd(out, (unsigned long long)s_tot);
}

constexpr int FR_CHUNK = 4096;

__global__ void __launch_bounds__(1024) k_chunk_counts(const uint8_t* f, int64_t count, long long* part) {
  __shared__ long long s_w[32];
  __shared__ long long s_tot;
  const int64_t base = (int64_t)blockIdx.x * FR_CHUNK;
  long long c = 0;
  for (int i = threadIdx.x; i < FR_CHUNK; i += blockDim.x)
    if (base + i < count) c += f[base + i];
  block_exclusive_scan<long long>(c, s_w, &s_tot);
  if (threadIdx.x == 0) part[blockIdx.x] = s_tot;
}

// Single block: smallest T with prefix(T) >= need (need >= 1).
__global__ void __launch_bounds__(1024) k_find_first(const uint8_t* f, int64_t count, const long long* part,
                                                     int64_t chunks, long long need, long long* out) {
  __shared__ long long s_w[32];
  __shared__ long long s_tot;
  __shared__ long long s_chunk, s_before;
  if (threadIdx.x == 0) {
    s_chunk = -1;
    s_before = 0;
  }
  __syncthreads();
  long long carry = 0;
  for (int64_t b = 0; b < chunks; b += blockDim.x) {
    const int64_t i = b + threadIdx.x;
    const long long x = i < chunks ? part[i] : 0;
    const long long ex = block_exclusive_scan<long long>(x, s_w, &s_tot);
    const long long before = carry + ex;
    if (i < chunks && before < need && before + x >= need) {
      s_chunk = i;
      s_before = before;
    }
    carry += s_tot;
    __syncthreads();
    if (s_chunk >= 0) break;
  }
  const long long total_all = carry;
  const int64_t c = s_chunk;
  long long T = 0;
  if (c >= 0) {
    const int64_t base = c * FR_CHUNK + (int64_t)threadIdx.x * 4;
    long long v[4], loc = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      v[t] = (base + t < count) ? f[base + t] : 0;
      loc += v[t];
    }
    long long ex = s_before + block_exclusive_scan<long long>(loc, s_w, &s_tot);
    __shared__ long long s_T;
    if (threadIdx.x == 0) s_T = 0;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (v[t] && ex < need && ex + 1 >= need) s_T = base + t + 1;
      ex += v[t];
    }
    __syncthreads();
    T = s_T;
  }
  if (threadIdx.x == 0) {
    out[0] = T;
    out[1] = (c >= 0) ? -1 : total_all;  // total only meaningful when not reached
  }
}

__global__ void k_set_bits(const int32_t* ids, int k, uint32_t* bits, uint8_t* bytes) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
    const int32_t v = ids[i];
    if (bits) atomicOr(bits + (v >> 5), 1u << (v & 31));
    if (bytes) bytes[v] = 1;
  }
}

__global__ void k_gather_sets(const int32_t* pool_nodes, const int64_t* set_start, const int32_t* set_len,
                              const int64_t* out_off, int64_t first, int64_t count, int32_t* out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < count; i += nwarps) {
    const int64_t st = set_start[first + i];
    const int32_t len = set_len[first + i];
    const int64_t o = out_off[i];
    for (int t = lane; t < len; t += 32) out[o + t] = pool_nodes[st + t];
  }
}

int grid_stride_blocks(int64_t work, int num_sms, int per_sm = 8) {
  int64_t b = (work + TPB - 1) / TPB;
  if (b > (int64_t)num_sms * per_sm) b = (int64_t)num_sms * per_sm;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t st) { return cudaMemsetAsync(p, 0, bytes, st); }

cudaError_t launch_count_nodes(const int32_t* nodes, const int32_t* samp, int64_t e0, int64_t e1, int64_t jlo,
                               int64_t jhi, int32_t* cnt, cudaStream_t st, int num_sms) {
  if (e1 <= e0) return cudaSuccess;
  k_count_nodes<<<grid_stride_blocks(e1 - e0, num_sms), TPB, 0, st>>>(nodes, samp, e0, e1, jlo, jhi, cnt);
  return cudaGetLastError();
}

size_t scan_tmp_bytes(int64_t n) { return sizeof(long long) * (size_t)((n + SCAN_TILE - 1) / SCAN_TILE + 1); }

cudaError_t launch_exclusive_scan(const int32_t* in, int64_t n, int64_t* out, void* tmp, cudaStream_t st,
                                  int* launches) {
  const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  long long* part = static_cast<long long*>(tmp);
  k_tile_sums<<<(unsigned)tiles, 1024, 0, st>>>(in, n, part);
  k_scan_parts<<<1, 1024, 0, st>>>(part, tiles);
  k_tile_scan<<<(unsigned)tiles, 1024, 0, st>>>(in, n, part, out);
  *launches += 3;
  return cudaGetLastError();
}

cudaError_t launch_scatter_index(const int32_t* nodes, const int32_t* samp, int64_t e0, int64_t e1, int64_t jlo,
                                 int64_t jhi, unsigned long long* cur, int32_t* inv_samp, cudaStream_t st,
                                 int num_sms) {
  if (e1 <= e0) return cudaSuccess;
  k_scatter_index<<<grid_stride_blocks(e1 - e0, num_sms), TPB, 0, st>>>(nodes, samp, e0, e1, jlo, jhi, cur,
                                                                        inv_samp);
  return cudaGetLastError();
}

namespace {
// Largest cluster of 1024-thread greedy blocks the device can schedule (16 or
// 8), 0 if none; computed once per process.
int greedy_cluster_size() {
  static int size = -1;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (size >= 0) return size;
  size = 0;
  if (cudaFuncSetAttribute(k_greedy<true>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    (void)cudaGetLastError();
  for (int c : {16, 8}) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(1024);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k_greedy<true>, &cfg) == cudaSuccess && clusters >= 1) {
      size = c;
      break;
    }
    (void)cudaGetLastError();
  }
  return size;
}
std::atomic<int> g_greedy_mode{0};
}  // namespace

void set_greedy_mode(int mode) { g_greedy_mode.store(mode); }

cudaError_t launch_greedy(const GreedyJob& J, cudaStream_t st, int num_sms, int* blocks_used, bool shared_gpu) {
  // A solve that shares the GPU with others (serving) runs all picks of a pool
  // of up to GREEDY_CLUSTER_ENTRIES entries in one thread-block cluster: 16 SMs,
  // hardware cluster barriers, and the rest of the GPU free for the other
  // solves.  Otherwise (and for larger pools, whose first picks decrement
  // millions of gains) one 1024-thread block per SM in a cooperative launch,
  // the faster shape for a solve that has the GPU to itself.
  const int mode = g_greedy_mode.load();
  const int csize = mode == 1 ? 0 : greedy_cluster_size();
  if (csize > 0 && (mode == 2 || (shared_gpu && J.total_entries <= GREEDY_CLUSTER_ENTRIES))) {
    *blocks_used = csize;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(csize);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_greedy<true>, J);
  }
  // one 1024-thread block per SM: the fewest barrier arrivals with a full machine
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_greedy<false>, 1024, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int blocks = num_sms;
  // cache slices fit in shared memory; one tally slot and one reducing thread per block
  if ((long long)blocks * HBINS < CACHE_MAX || blocks > 1024) return cudaErrorInvalidConfiguration;
  *blocks_used = blocks;
  // a cooperative launch (all blocks resident at once), also valid inside a stream capture
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(1024);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_greedy<false>, J);
}

cudaError_t device_code_version(int* binary, int* ptx) {
  cudaFuncAttributes a{};
  const cudaError_t e = cudaFuncGetAttributes(&a, k_greedy<false>);
  if (e != cudaSuccess) return e;
  *binary = a.binaryVersion;
  *ptx = a.ptxVersion;
  return cudaSuccess;
}

cudaError_t launch_add_counts(int32_t* total, const int32_t* add, int64_t n, cudaStream_t st, int num_sms) {
  k_add_counts<<<grid_stride_blocks(n, num_sms, 4), TPB, 0, st>>>(total, add, n);
  return cudaGetLastError();
}

cudaError_t launch_mark_hits(const int32_t* nodes, const int32_t* samp, int64_t e0, int64_t e1,
                             const uint8_t* in_seed, int64_t j0, int64_t j1, uint8_t* hit, cudaStream_t st,
                             int num_sms) {
  if (e1 <= e0) return cudaSuccess;
  k_mark_hits<<<grid_stride_blocks(e1 - e0, num_sms), TPB, 0, st>>>(nodes, samp, e0, e1, in_seed, j0, j1, hit);
  return cudaGetLastError();
}

cudaError_t launch_count_flags(const uint8_t* flags, int64_t count, unsigned long long* out, cudaStream_t st,
                               int num_sms) {
  if (count <= 0) return cudaSuccess;
  k_count_flags<<<grid_stride_blocks(count, num_sms, 4), TPB, 0, st>>>(flags, count, out);
  return cudaGetLastError();
}

size_t first_reach_tmp_bytes(int64_t count) {
  return sizeof(long long) * (size_t)((count + FR_CHUNK - 1) / FR_CHUNK + 1);
}

cudaError_t launch_first_reach(const uint8_t* flags, int64_t count, long long need, long long* out, void* tmp,
                               cudaStream_t st, int* launches) {
  const int64_t chunks = (count + FR_CHUNK - 1) / FR_CHUNK;
  long long* part = static_cast<long long*>(tmp);
  k_chunk_counts<<<(unsigned)chunks, 1024, 0, st>>>(flags, count, part);
  k_find_first<<<1, 1024, 0, st>>>(flags, count, part, chunks, need, out);
  *launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_set_bits(const int32_t* ids, int k, uint32_t* bits, uint8_t* bytes, cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  k_set_bits<<<(k + TPB - 1) / TPB, TPB, 0, st>>>(ids, k, bits, bytes);
  return cudaGetLastError();
}

cudaError_t launch_gather_sets(const int32_t* pool_nodes, const int64_t* set_start, const int32_t* set_len,
                               const int64_t* out_off, int64_t first, int64_t count, int32_t* out, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int blocks = (int)((count * 32 + TPB - 1) / TPB);
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_gather_sets<<<blocks, TPB, 0, st>>>(pool_nodes, set_start, set_len, out_off, first, count, out);
  return cudaGetLastError();
}

}  // namespace ssa
