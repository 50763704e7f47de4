// Allocation-free coverage count: ssa_coverage_noalloc (see include/ssa.h).
//
// Some callers cannot allocate device memory at call time: a serving loop
// that reserved all of its device memory up front and must not trigger an
// allocation (or the implicit synchronisation of cudaMalloc) in its request
// path, or a host runtime whose allocator owns the device.  This entry point
// computes the same Cov (Eq. 1) as ssa_coverage, over a flat RR pool the
// caller already holds in device memory, with all of its scratch in one
// file-scope device array of fixed size.  The array lives as long as the
// library is loaded, on every device that loads it; every call shares it and
// it keeps the last call's contents, so each call clears the part it uses,
// and calls whose work overlaps on the GPU (different streams, or threads)
// race on it.
#include "../../include/ssa.h"
#include "device.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr size_t kHeaderBytes = 256;                // counter + error flag

static __device__ __align__(256) unsigned char g_cov_scratch[kScratchBytes];

struct ScratchHeader {
  unsigned long long cov;
  unsigned int bad_id;
};

// Device address of the scratch array on the current device.  Host code must
// not use the symbol itself as an address.  It is looked up on every call (a
// lookup allocates nothing and is cheap), so an address never outlives the
// context it came from, e.g. across a cudaDeviceReset.
cudaError_t scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_cov_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

__global__ void k_na_seed_bits(const int32_t* seeds, int k, int64_t n, uint32_t* bits, ScratchHeader* h) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
    const int32_t v = seeds[i];
    if (v < 0 || v >= n) {
      atomicExch(&h->bad_id, 1u);
      continue;
    }
    atomicOr(bits + (v >> 5), 1u << (v & 31));
  }
}

// hit bit of sample s - first for every entry (node, s) with a seed node
__global__ void k_na_mark(const int32_t* __restrict__ nodes, const int32_t* __restrict__ samp, int64_t entries,
                          int64_t n, int64_t first, int64_t count, const uint32_t* __restrict__ seed_bits,
                          uint32_t* hit_bits, ScratchHeader* h) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < entries;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = samp[q];
    if (s < first || s >= first + count) continue;
    const int32_t v = nodes[q];
    if (v < 0 || v >= n) {
      atomicExch(&h->bad_id, 1u);
      continue;
    }
    if ((seed_bits[v >> 5] >> (v & 31)) & 1u) {
      const int64_t i = s - first;
      atomicOr(hit_bits + (i >> 5), 1u << (i & 31));
    }
  }
}

__global__ void k_na_count(const uint32_t* __restrict__ hit_bits, int64_t words, ScratchHeader* h) {
  unsigned long long c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x)
    c += (unsigned long long)__popc(hit_bits[i]);
  c = ssa::warp_sum(c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&h->cov, c);
}

int blocks_for(int64_t work) {
  int64_t b = (work + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  return (int)(b < 1 ? 1 : b);
}

ssa_status fail_msg(ssa_status s, const char* msg) {
  ssa::set_last_error(msg);
  return s;
}

}  // namespace

extern "C" ssa_status ssa_coverage_noalloc(int64_t n, const int32_t* nodes, const int32_t* samp, int64_t entries,
                                           int64_t first, int64_t count, const int32_t* seeds, int32_t k,
                                           int64_t* cov, void* stream) {
  if (!cov) return fail_msg(SSA_E_ARG, "ssa_coverage_noalloc: null cov");
  if (n < 1 || entries < 0 || first < 0 || count < 0 || k < 0)
    return fail_msg(SSA_E_ARG, "ssa_coverage_noalloc: negative size or n < 1");
  if ((entries > 0 && (!nodes || !samp)) || (k > 0 && !seeds))
    return fail_msg(SSA_E_ARG, "ssa_coverage_noalloc: null device array");
  const size_t seed_words = (size_t)((n + 31) / 32);
  const size_t hit_words = (size_t)((count + 31) / 32);
  const size_t need = kHeaderBytes + 4 * seed_words + 4 * hit_words;
  if (need > kScratchBytes)
    return fail_msg(SSA_E_ARG,
                    "ssa_coverage_noalloc: n/32 + count/32 words exceed the 16 MiB scratch "
                    "(n + count must stay below about 134 million)");
  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return fail_msg(SSA_E_CUDA, "ssa_coverage_noalloc: cudaGetSymbolAddress failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ScratchHeader* h = static_cast<ScratchHeader*>(base);
  uint32_t* seed_bits = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(base) + kHeaderBytes);
  uint32_t* hit_bits = seed_bits + seed_words;
  // the array keeps the previous call's contents: clear what this call uses
  if ((e = cudaMemsetAsync(base, 0, need, st)) != cudaSuccess)
    return fail_msg(SSA_E_CUDA, "ssa_coverage_noalloc: clearing scratch failed");
  if (k > 0) k_na_seed_bits<<<blocks_for(k), 256, 0, st>>>(seeds, k, n, seed_bits, h);
  if (entries > 0 && count > 0)
    k_na_mark<<<blocks_for(entries), 256, 0, st>>>(nodes, samp, entries, n, first, count, seed_bits, hit_bits, h);
  if (hit_words > 0) k_na_count<<<blocks_for((int64_t)hit_words), 256, 0, st>>>(hit_bits, (int64_t)hit_words, h);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail_msg(SSA_E_CUDA, "ssa_coverage_noalloc: launch failed");
  ScratchHeader out{};
  if ((e = cudaMemcpyAsync(&out, h, sizeof(out), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail_msg(SSA_E_CUDA, "ssa_coverage_noalloc: reading the count failed");
  if (out.bad_id) return fail_msg(SSA_E_ARG, "ssa_coverage_noalloc: a node or seed id lies outside [0, n)");
  *cov = (int64_t)out.cov;
  return SSA_OK;
}
