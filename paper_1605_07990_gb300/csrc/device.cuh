// Device-side helpers shared by the sm_103a kernels: the Philox4x32-10
// generator and the sample keying, warp scans and bit tests.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.h"

namespace ssa {

constexpr unsigned FULL_MASK = 0xffffffffu;
constexpr uint32_t NO_NODE = 0xffffffffu;

enum : uint32_t { PURPOSE_ROOT = 1, PURPOSE_IC = 2, PURPOSE_LT = 3, PURPOSE_SKIP = 4, PURPOSE_WEIGHT = 5 };

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of the 4x32 S-box
// (two 32x32->64 products, the high halves xored into the other words), the
// key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ uint2 philox_key(uint64_t seed) {
  return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
}

// High word of the counter: purpose | stream | bits 32..51 of the sample id.
__device__ __forceinline__ uint32_t ctr_word3(uint32_t purpose, uint32_t stream, int64_t j) {
  return (purpose << 28) | ((stream & 0xFFu) << 20) | ((uint32_t)((uint64_t)j >> 32) & 0xFFFFFu);
}

__device__ __forceinline__ uint4 keyed_draw(uint64_t seed, uint32_t purpose, uint32_t stream, int64_t j,
                                            uint64_t x) {
  return philox4x32_10(make_uint4((uint32_t)x, (uint32_t)(x >> 32), (uint32_t)j, ctr_word3(purpose, stream, j)),
                       philox_key(seed));
}

// An edge is live when its draw is below the threshold; 0xFFFFFFFF = always.
__device__ __forceinline__ bool edge_live(uint32_t r, uint32_t thr) {
  return thr == 0xFFFFFFFFu || r < thr;
}

__device__ __forceinline__ bool test_bit(const uint32_t* bits, uint32_t v) {
  return (__ldg(bits + (v >> 5)) >> (v & 31)) & 1u;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int d = 16; d; d >>= 1) x += __shfl_xor_sync(FULL_MASK, x, d);
  return x;
}

__device__ __forceinline__ int warp_inclusive_scan(int x, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(FULL_MASK, x, d);
    if (lane >= d) x += t;
  }
  return x;
}

}  // namespace ssa
