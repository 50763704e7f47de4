// Graph store (Sec. 2): in-edge CSR with uint32 live thresholds, built on
// the device.  Edges are ordered by (dst, src, input position) with a stable
// device radix sort (CUB, header source from the CUDA toolkit); offsets come
// from segment boundaries of the sorted keys, thresholds from the weighting
// rule: weighted cascade w = 1/d_in(v) (Sec. 6.1), trivalency, or explicit.
#include <algorithm>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_select.cuh>

#include "device.cuh"

namespace ssa {

namespace {

__global__ void k_make_keys(const int32_t* src, const int32_t* dst, int64_t n, int64_t m, int bits,
                            unsigned long long* keys, int32_t* vals, unsigned int* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = src[i], d = dst[i];
    if (s < 0 || s >= n || d < 0 || d >= n) {
      atomicExch(err, 1u);
      keys[i] = 0;
    } else {
      keys[i] = ((unsigned long long)d << bits) | (unsigned long long)s;
    }
    vals[i] = (int32_t)i;
  }
}

// off[v] = first sorted position whose dst >= v.
__global__ void k_offsets(const unsigned long long* keys, int64_t n, int64_t m, int bits, int64_t* off) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e <= m; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t prev = (e == 0) ? -1 : (int64_t)(keys[e - 1] >> bits);
    const int64_t cur = (e == m) ? n : (int64_t)(keys[e] >> bits);
    for (int64_t v = prev + 1; v <= cur; ++v) off[v] = e;
  }
}

__global__ void k_fill_edges(const unsigned long long* keys, const int32_t* vals, const int64_t* off, int64_t m,
                             int bits, int weighting, uint64_t weight_seed, const uint32_t* thr_in, uint2* edge) {
  const unsigned long long mask = (1ull << bits) - 1ull;
  const uint32_t TRI[3] = {429496729u, 42949672u, 4294967u};  // floor(2^32 p), p = 0.1, 0.01, 0.001
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = keys[e];
    const uint32_t s = (uint32_t)(k & mask);
    uint32_t t;
    if (weighting == 0) {
      const int64_t v = (int64_t)(k >> bits);
      const uint64_t d = (uint64_t)(off[v + 1] - off[v]);
      t = (d == 1) ? 0xFFFFFFFFu : (uint32_t)((1ull << 32) / d);
    } else if (weighting == 1) {
      const uint4 r = keyed_draw(weight_seed, PURPOSE_WEIGHT, 0, 0, (uint64_t)e);
      t = TRI[__umulhi(r.x, 3u)];
    } else {
      t = thr_in[vals[e]];
    }
    edge[e] = make_uint2(s, t);
  }
}

// SplitMix64's output function (Steele, Lea, Flood, OOPSLA 2014) applied to
// a counter: draw number ctr of the stream keyed by seed.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t ctr) {
  uint64_t z = seed + (ctr + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): draw i descends `scale`
// levels; level l uses the 32-bit half l&1 of SplitMix64 draw 32 i + l/2 and
// picks quadrant a (src bit 0, dst bit 0), b (0,1), c (1,0) or d (1,1), most
// significant bit first.  Key (dst << scale) | src; a self-loop keys to
// `drop`, which sorts after every edge.
__global__ void k_rmat_keys(int scale, int64_t m_draw, uint32_t ta, uint32_t tab, uint32_t tabc, uint64_t seed,
                            unsigned long long drop, unsigned long long* keys) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m_draw;
       i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long s = 0, d = 0;
    uint64_t r = 0;
    for (int l = 0; l < scale; ++l) {
      if ((l & 1) == 0) r = splitmix64_at(seed, (uint64_t)i * 32u + (uint64_t)(l >> 1));
      const uint32_t u = (l & 1) ? (uint32_t)(r >> 32) : (uint32_t)r;
      const unsigned long long sb = u < tab ? 0ull : 1ull;
      const unsigned long long db = (u < ta || (u >= tab && u < tabc)) ? 0ull : 1ull;
      s = (s << 1) | sb;
      d = (d << 1) | db;
    }
    keys[i] = s == d ? drop : ((d << scale) | s);
  }
}

int grid_for(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (int)b;
}

}  // namespace

cudaError_t rmat_graph(int scale, int64_t m_draw, uint32_t ta, uint32_t tab, uint32_t tabc, uint64_t seed,
                       int weighting, uint64_t weight_seed, int64_t* m_out, int64_t** d_off, uint2** d_edge,
                       cudaStream_t st, int* launches) {
  const int64_t n = int64_t(1) << scale;
  const unsigned long long drop = 1ull << (2 * scale);  // after every (dst, src) key
  const int end_bit = 2 * scale + 1;
  unsigned long long *k_in = nullptr, *k_out = nullptr;
  long long* d_count = nullptr;
  void* tmp = nullptr;
  size_t tmp_sort = 0, tmp_uniq = 0;
  *d_off = nullptr;
  *d_edge = nullptr;
  cudaError_t e = cudaSuccess;
  do {
    const size_t cnt = (size_t)(m_draw > 0 ? m_draw : 1);
    if ((e = cudaMallocAsync(&k_in, sizeof(unsigned long long) * cnt, st)) != cudaSuccess) break;
    if ((e = cudaMallocAsync(&k_out, sizeof(unsigned long long) * cnt, st)) != cudaSuccess) break;
    if ((e = cudaMallocAsync(&d_count, sizeof(long long), st)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(d_count, 0, sizeof(long long), st)) != cudaSuccess) break;
    int64_t m = 0;
    if (m_draw > 0) {
      k_rmat_keys<<<grid_for(m_draw, 256), 256, 0, st>>>(scale, m_draw, ta, tab, tabc, seed, drop, k_in);
      ++*launches;
      if ((e = cudaGetLastError()) != cudaSuccess) break;
      if ((e = cub::DeviceRadixSort::SortKeys(nullptr, tmp_sort, k_in, k_out, m_draw, 0, end_bit, st)) !=
          cudaSuccess)
        break;
      if ((e = cub::DeviceSelect::Unique(nullptr, tmp_uniq, k_out, k_in, d_count, m_draw, st)) != cudaSuccess)
        break;
      if ((e = cudaMallocAsync(&tmp, std::max(tmp_sort, tmp_uniq), st)) != cudaSuccess) break;
      if ((e = cub::DeviceRadixSort::SortKeys(tmp, tmp_sort, k_in, k_out, m_draw, 0, end_bit, st)) != cudaSuccess)
        break;
      // unique keys in ascending order back into k_in; the one `drop` key, if any, is last
      if ((e = cub::DeviceSelect::Unique(tmp, tmp_uniq, k_out, k_in, d_count, m_draw, st)) != cudaSuccess) break;
      *launches += 2 * ((end_bit + 7) / 8) + 3;
      long long uniq = 0;
      unsigned long long last = 0;
      if ((e = cudaMemcpyAsync(&uniq, d_count, sizeof(uniq), cudaMemcpyDeviceToHost, st)) != cudaSuccess) break;
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
      if (uniq > 0) {
        if ((e = cudaMemcpyAsync(&last, k_in + uniq - 1, sizeof(last), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
          break;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
      }
      m = (uniq > 0 && last == drop) ? uniq - 1 : uniq;
    }
    const int64_t m_pad = ((m + 3) / 4) * 4 + 4;
    if ((e = cudaMallocAsync(d_off, sizeof(int64_t) * (size_t)(n + 1), st)) != cudaSuccess) break;
    if ((e = cudaMallocAsync(d_edge, sizeof(uint2) * (size_t)m_pad, st)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(*d_edge, 0, sizeof(uint2) * (size_t)m_pad, st)) != cudaSuccess) break;
    if (m == 0) {
      e = cudaMemsetAsync(*d_off, 0, sizeof(int64_t) * (size_t)(n + 1), st);
    } else {
      // the unique keys are the CSR order (dst, src): offsets and records as for a loaded graph
      k_offsets<<<grid_for(m + 1, 256), 256, 0, st>>>(k_in, n, m, scale, *d_off);
      k_fill_edges<<<grid_for(m, 256), 256, 0, st>>>(k_in, nullptr, *d_off, m, scale, weighting, weight_seed,
                                                     nullptr, *d_edge);
      *launches += 2;
      e = cudaGetLastError();
    }
    *m_out = m;
  } while (false);
  if (k_in) cudaFreeAsync(k_in, st);
  if (k_out) cudaFreeAsync(k_out, st);
  if (d_count) cudaFreeAsync(d_count, st);
  if (tmp) cudaFreeAsync(tmp, st);
  if (e != cudaSuccess) {
    if (*d_off) cudaFreeAsync(*d_off, st);
    if (*d_edge) cudaFreeAsync(*d_edge, st);
    *d_off = nullptr;
    *d_edge = nullptr;
  }
  return e;
}

cudaError_t build_graph(int64_t n, int64_t m, const int32_t* d_src, const int32_t* d_dst, const uint32_t* d_thr_in,
                        int weighting, uint64_t weight_seed, int64_t* d_off, uint2* d_edge, unsigned int* d_err,
                        cudaStream_t st, int* launches) {
  int bits = 1;
  while ((1ll << bits) < n) ++bits;
  cudaError_t e = cudaSuccess;
  if (m == 0) {
    e = cudaMemsetAsync(d_off, 0, sizeof(int64_t) * (size_t)(n + 1), st);
    return e;
  }
  unsigned long long *k_in = nullptr, *k_out = nullptr;
  int32_t *v_in = nullptr, *v_out = nullptr;
  void* tmp = nullptr;
  size_t tmp_bytes = 0;
  do {
    if ((e = cudaMallocAsync(&k_in, sizeof(unsigned long long) * (size_t)m, st)) != cudaSuccess) break;
    if ((e = cudaMallocAsync(&k_out, sizeof(unsigned long long) * (size_t)m, st)) != cudaSuccess) break;
    if ((e = cudaMallocAsync(&v_in, sizeof(int32_t) * (size_t)m, st)) != cudaSuccess) break;
    if ((e = cudaMallocAsync(&v_out, sizeof(int32_t) * (size_t)m, st)) != cudaSuccess) break;
    k_make_keys<<<grid_for(m, 256), 256, 0, st>>>(d_src, d_dst, n, m, bits, k_in, v_in, d_err);
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, k_in, k_out, v_in, v_out, (int64_t)m, 0, 2 * bits,
                                             st)) != cudaSuccess)
      break;
    if ((e = cudaMallocAsync(&tmp, tmp_bytes, st)) != cudaSuccess) break;
    if ((e = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, k_in, k_out, v_in, v_out, (int64_t)m, 0, 2 * bits,
                                             st)) != cudaSuccess)
      break;
    *launches += 2 * ((2 * bits + 7) / 8) + 1;
    k_offsets<<<grid_for(m + 1, 256), 256, 0, st>>>(k_out, n, m, bits, d_off);
    ++*launches;
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    k_fill_edges<<<grid_for(m, 256), 256, 0, st>>>(k_out, v_out, d_off, m, bits, weighting, weight_seed, d_thr_in,
                                                   d_edge);
    ++*launches;
    e = cudaGetLastError();
  } while (false);
  if (k_in) cudaFreeAsync(k_in, st);
  if (k_out) cudaFreeAsync(k_out, st);
  if (v_in) cudaFreeAsync(v_in, st);
  if (v_out) cudaFreeAsync(v_out, st);
  if (tmp) cudaFreeAsync(tmp, st);
  return e;
}

namespace {
__global__ void k_max_in_degree(const int64_t* off, int64_t n, unsigned long long* out) {
  unsigned long long best = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long d = (unsigned long long)(off[v + 1] - off[v]);
    best = d > best ? d : best;
  }
  for (int s = 16; s; s >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, s);
    best = o > best ? o : best;
  }
  if ((threadIdx.x & 31) == 0 && best) atomicMax(out, best);
}

// Row of in-degree d (1 <= d < 2^K): the powers q^(2^i), i < bit length of d,
// of the weighted-cascade gap form (Q = (2^32 - t) << 32 with t = floor(2^32/d),
// 0xFFFFFFFF for d = 1; each power the high 64 bits of the previous one squared).
__global__ void k_wc_pow_rows(uint64_t* tab, int K) {
  const int64_t rows = int64_t(1) << K;
  for (int64_t d = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < rows;
       d += (int64_t)gridDim.x * blockDim.x) {
    const int k = 63 - __clzll(d);
    const uint64_t base = k == 0 ? 0ull : (uint64_t)(k - 1) * (1ull << k) + 1ull;
    uint64_t* row = tab + base + (uint64_t)(d - (int64_t(1) << k)) * (uint64_t)(k + 1);
    const uint32_t t = d == 1 ? 0xFFFFFFFFu : (uint32_t)(0x100000000ull / (uint64_t)d);
    uint64_t p = (0x100000000ull - t) << 32;
    for (int i = 0; i <= k; ++i) {
      row[i] = p;
      p = __umul64hi(p, p);
    }
  }
}
}  // namespace

cudaError_t build_wc_pow(const int64_t* d_off, int64_t n, uint64_t** tab, int* k_out, cudaStream_t st) {
  *tab = nullptr;
  *k_out = 0;
  unsigned long long* d_max = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d_max), sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  unsigned long long maxd = 0;
  cudaMemsetAsync(d_max, 0, sizeof(unsigned long long), st);
  k_max_in_degree<<<grid_for(n, 256), 256, 0, st>>>(d_off, n, d_max);
  cudaMemcpyAsync(&maxd, d_max, sizeof(maxd), cudaMemcpyDeviceToHost, st);
  e = cudaStreamSynchronize(st);
  cudaFree(d_max);
  if (e != cudaSuccess) return e;
  int K = 0;
  while (K < WC_POW_K && (1ull << K) <= maxd) ++K;  // rows for every d < 2^K that occurs
  if (K < 2) return cudaSuccess;                     // no in-list of 2 or more edges
  const size_t entries = (size_t)(K - 1) * ((size_t)1 << K) + 1;
  if ((e = cudaMallocAsync(reinterpret_cast<void**>(tab), sizeof(uint64_t) * entries, st)) != cudaSuccess) return e;
  k_wc_pow_rows<<<grid_for((int64_t)1 << K, 256), 256, 0, st>>>(*tab, K);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  *k_out = K;
  return cudaSuccess;
}

}  // namespace ssa
