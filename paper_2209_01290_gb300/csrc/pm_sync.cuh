// pm_sync.cuh -- the bounded dependency waits of the persistent launches
// (pm_persist.cu, pm_wpersist.cu): per-unit counters published with release
// reductions and read with acquire loads at GPU scope.  Every wait gives up
// after about a second (by %globaltimer, with a poll-count backstop) and
// records that in the launch's error flag instead of hanging.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace pm {
namespace {

constexpr uint64_t kWaitNs = 1000000000ull;  // give up a wait after one second
constexpr long kWaitIters = 1L << 26;        // backstop on the number of polls

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(uint32_t* p, uint32_t v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0 waits until *ctr >= target, for at most about a second; on
// giving up it sets the error flag and the CTA proceeds (its result is then
// invalid, which the host learns from the flag).
__device__ __forceinline__ void cta_wait(const uint32_t* ctr, uint32_t target, int* err) {
  if (threadIdx.x == 0 && ld_acquire(ctr) < target) {
    const uint64_t t0 = global_ns();
    long it = 0;
    while (ld_acquire(ctr) < target) {
      if (++it > kWaitIters || global_ns() - t0 > kWaitNs) {
        atomicOr(err, 1);
        break;
      }
      __nanosleep(128);
    }
  }
  __syncthreads();
}

// All threads' global writes are complete; thread 0 publishes them.
__device__ __forceinline__ void cta_signal(uint32_t* ctr) {
  __syncthreads();
  if (threadIdx.x == 0) red_release_add(ctr, 1);
}

}  // namespace
}  // namespace pm
