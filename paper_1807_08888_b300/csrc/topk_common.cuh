// Device helpers shared by the query engines: the global k-th-best threshold and result
// appends (Algorithm 1's result-set update and its dominated() test).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace nuri {

__device__ __forceinline__ int32_t ld_volatile(const int32_t* p) {
  return *(const volatile int32_t*)p;
}
__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
  return *(const volatile unsigned long long*)p;
}

// One value for the whole warp: lane 0 loads, the others take its value.  Warp-wide code
// (shuffles, ballots, __syncwarp with a full mask) may only branch on values every lane
// agrees on; a location other warps update (a threshold, a domain bitmap, a counter) read by
// each lane on its own can differ between lanes, which would part the warp before a warp-wide
// operation that the departed lanes never reach.
template <class T>
__device__ __forceinline__ T warp_load(const T* p) {
  T v{};
  if ((threadIdx.x & 31) == 0) v = *(const volatile T*)p;
  return __shfl_sync(0xffffffffu, v, 0);
}

// The deadline test of warp-wide code, decided by lane 0 for the whole warp.
__device__ __forceinline__ bool warp_past(const uint64_t* deadline) {
  int late = 0;
  if ((threadIdx.x & 31) == 0) {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    late = t > *(const volatile uint64_t*)deadline;
  }
  return __shfl_sync(0xffffffffu, late, 0) != 0;
}

// Threshold from a histogram: tau = max t with sum_{s >= t} hist[s] >= k, or INT32_MIN
// when fewer than k results exist.  Bins may be coarse (score >> shift): the value returned
// is then the lower edge of the bin, still a valid lower bound of the exact k-th score.
// Any snapshot of the counters undercounts the final histogram, so every value computed
// here is <= the final k-th score; publishing it with atomicMax keeps tau monotone.
// The scan starts at `top` (the highest non-empty bin) and stops at the current tau.
__device__ __forceinline__ void publish_threshold(const int32_t* hist, int32_t top,
                                                  int32_t shift, int64_t k, int32_t* tau) {
  int32_t cur = ld_volatile(tau);
  int32_t floor_bin = cur > 0 ? (cur >> shift) : 0;
  int64_t acc = 0;
  for (int32_t b = top; b >= floor_bin; --b) {
    acc += ld_volatile(hist + b);
    if (acc >= k) {
      int32_t t = b << shift;
      if (t > cur) atomicMax(tau, t);
      return;
    }
  }
}

}  // namespace nuri
