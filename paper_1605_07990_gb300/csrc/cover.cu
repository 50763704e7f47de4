// RR pool index, greedy Max-Coverage (Algorithm 2), coverage checks (Eq. 1)
// and the Estimate-Inf first-T search (Algorithm 3) on sm_103a.
//
// Index: cnt[v] = number of sets holding v by a counting pass over the flat
// (node, sample) entries, exclusive scan into inv_off, scatter of sample ids
// into inv_samp (order inside a list is irrelevant: each step only needs the
// set of samples holding the picked node).
// Greedy step: atomic-free argmax over packed keys (gain+1)<<32 | ~v (largest
// gain, then smallest id; seeds keyed to 0) as per-block partials, then one
// kernel that reduces the partials, records the pick and, warp per newly
// covered set, decrements the gains of the set's members.
#include "device.cuh"

namespace ssa {

namespace {

constexpr int TPB = 256;

// samp == nullptr: every entry in [e0, e1) counts; else only samples in [jlo, jhi)
__global__ void k_count_nodes(const int32_t* __restrict__ nodes, const int32_t* __restrict__ samp, int64_t e0,
                              int64_t e1, int64_t jlo, int64_t jhi, int32_t* cnt) {
  for (int64_t q = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < e1; q += (int64_t)gridDim.x * blockDim.x) {
    if (samp) {
      const int64_t s = samp[q];
      if (s < jlo || s >= jhi) continue;
    }
    atomicAdd(cnt + nodes[q], 1);
  }
}

__global__ void k_scatter_index(const int32_t* __restrict__ nodes, const int32_t* __restrict__ samp, int64_t e0,
                                int64_t e1, int64_t jlo, int64_t jhi, unsigned long long* cur, int32_t* inv_samp) {
  for (int64_t q = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < e1;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = samp[q];
    if (s < jlo || s >= jhi) continue;
    const unsigned long long pos = atomicAdd(cur + nodes[q], 1ull);
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
__device__ __forceinline__ unsigned long long gain_key(int32_t c, uint8_t taken, uint32_t v) {
  return taken ? 0ull : (((unsigned long long)(uint32_t)(c + 1)) << 32) | (unsigned long long)(0xFFFFFFFFu - v);
}

__device__ __forceinline__ unsigned long long block_max(unsigned long long x, unsigned long long* s) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int d = 16; d; d >>= 1) {
    const unsigned long long t = __shfl_xor_sync(FULL_MASK, x, d);
    x = t > x ? t : x;
  }
  if (lane == 0) s[wid] = x;
  __syncthreads();
  if (wid == 0) {
    x = lane < nw ? s[lane] : 0ull;
#pragma unroll
    for (int d = 16; d; d >>= 1) {
      const unsigned long long t = __shfl_xor_sync(FULL_MASK, x, d);
      x = t > x ? t : x;
    }
    if (lane == 0) s[0] = x;
  }
  __syncthreads();
  x = s[0];
  __syncthreads();
  return x;
}

__global__ void __launch_bounds__(TPB) k_argmax(const int32_t* __restrict__ cnt, const uint8_t* __restrict__ in_seed,
                                                int64_t n, unsigned long long* partial) {
  __shared__ unsigned long long s[32];
  unsigned long long best = 0;
  const int64_t n4 = n >> 2;
  const int4* c4 = reinterpret_cast<const int4*>(cnt);
  const uchar4* s4 = reinterpret_cast<const uchar4*>(in_seed);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    const int4 c = __ldg(c4 + i);
    const uchar4 t = __ldg(s4 + i);
    const uint32_t v = (uint32_t)(i * 4);
    unsigned long long k;
    k = gain_key(c.x, t.x, v);     best = k > best ? k : best;
    k = gain_key(c.y, t.y, v + 1); best = k > best ? k : best;
    k = gain_key(c.z, t.z, v + 2); best = k > best ? k : best;
    k = gain_key(c.w, t.w, v + 3); best = k > best ? k : best;
  }
  for (int64_t v = n4 * 4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = gain_key(cnt[v], in_seed[v], (uint32_t)v);
    best = k > best ? k : best;
  }
  best = block_max(best, s);
  if (threadIdx.x == 0) partial[blockIdx.x] = best;
}

__global__ void __launch_bounds__(TPB) k_cover(GreedyBufs b, int step) {
  __shared__ unsigned long long s[32];
  unsigned long long best = 0;
  for (int i = threadIdx.x; i < b.argmax_blocks; i += blockDim.x) {
    const unsigned long long k = b.partial[i];
    best = k > best ? k : best;
  }
  best = block_max(best, s);
  const int32_t vstar = (int32_t)(0xFFFFFFFFu - (uint32_t)best);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    b.seeds[step] = vstar;
    b.gains[step] = (int32_t)((uint32_t)(best >> 32) - 1u);
    b.in_seed[vstar] = 1;
  }
  const int64_t q0 = b.inv_off[vstar], q1 = b.inv_off[vstar + 1];
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t q = q0 + warp; q < q1; q += nwarps) {
    const int32_t j = b.inv_samp[q];
    if (b.covered[j]) continue;
    __syncwarp();
    if (lane == 0) b.covered[j] = 1;
    const int64_t st = b.set_start[j];
    const int32_t len = b.set_len[j];
    for (int i = lane; i < len; i += 32) atomicSub(b.cnt + b.pool_nodes[st + i], 1);
  }
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

cudaError_t launch_greedy_step(const GreedyBufs& b, int step, cudaStream_t st, int num_sms) {
  k_argmax<<<b.argmax_blocks, TPB, 0, st>>>(b.cnt, b.in_seed, b.n, b.partial);
  k_cover<<<num_sms * 4, TPB, 0, st>>>(b, step);
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
