// afc_device.cuh -- device-side building blocks shared by the library's kernels:
// the Philox4x32-10 counter-based generator, thread-group primitives and small helpers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace afc {

constexpr uint32_t kFull = 0xFFFFFFFFu;

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the multiply-hi/lo
// bijection on a 4 x 32-bit counter with a Weyl key schedule.  Realization draws use the
// counter (edge, realization, graph, 0); perturbation draws use (column, row, index, 1).
__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, x.x), lo0 = 0xD2511F53u * x.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, x.z), lo1 = 0xCD9E8D57u * x.z;
    x = make_uint4(hi1 ^ x.y ^ k0, lo1, hi0 ^ x.w ^ k1, lo0);
  }
  return x;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Warp-aggregated append: returns a unique slot from *counter for every calling lane.
__device__ __forceinline__ uint32_t warp_append(uint32_t *counter) {
  const uint32_t mask = __activemask();
  const uint32_t leader = __ffs(mask) - 1;
  uint32_t base = 0;
  if (lane_id() == leader) base = atomicAdd(counter, (uint32_t)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  return base + (uint32_t)__popc(mask & lanemask_lt());
}

// Warp-aggregated append keyed by `key`: lanes with equal keys share one atomicAdd on the
// counter they all pass (lanes with different keys must pass different counters).
__device__ __forceinline__ uint32_t warp_append_keyed(uint32_t *counter, uint32_t key) {
  const uint32_t peers = __match_any_sync(__activemask(), key);
  const uint32_t leader = __ffs(peers) - 1;
  uint32_t base = 0;
  if (lane_id() == leader) base = atomicAdd(counter, (uint32_t)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  return base + (uint32_t)__popc(peers & lanemask_lt());
}

}  // namespace afc
