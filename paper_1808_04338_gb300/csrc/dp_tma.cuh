// Bulk asynchronous copies (the untiled form of the tensor memory
// accelerator: cp.async.bulk global -> shared) completing on shared-memory
// mbarriers, and bounded waits on those barriers.  A wait that has not seen
// its phase complete after kWaitNs of global time gives up and returns
// false; the kernel then records the failure in a device flag and returns,
// so a lost copy ends as an error status on the host instead of a hung GPU.
#pragma once
#include <cstdint>

namespace dp {

constexpr uint64_t kWaitNs = 1000000000ull;   // 1 s

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// makes the initialised barriers visible to the async proxy and the CTA
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one arrival that also raises the phase's expected transaction bytes
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// waits for the completion of the barrier's phase of the given parity;
// false after kWaitNs without it
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_test(bar, parity)) return true;
  uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_test(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

// bytes (a multiple of 16) from global src to shared dst (both 16-byte
// aligned), counted on bar's transaction bytes when they have landed
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier of all threads of a cooperative launch: the k-th barrier of
// the launch is passed when cnt[0] reaches k * gridDim.x arrivals (target);
// false, for every thread of the CTA, when the wait gave up or *err is set.
// The launch's last CTA resets the count (grid_exit).
__device__ __forceinline__ bool grid_sync_all(unsigned *cnt, unsigned target, int *err) {
  __shared__ int gave_up;
  __syncthreads();
  if (threadIdx.x == 0) {
    gave_up = 0;
    __threadfence();
    atomicAdd(cnt, 1u);
    uint64_t t0 = global_ns();
    while (ld_acquire_u32(cnt) < target) {
      if (*(volatile int *)err || global_ns() - t0 > kWaitNs) {
        atomicExch(err, 1);
        gave_up = 1;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
  return !gave_up;
}

// called by every CTA when it leaves: the last one resets cnt[0] and cnt[1]
__device__ __forceinline__ void grid_exit(unsigned *cnt) {
  __syncthreads();
  if (threadIdx.x == 0 && atomicAdd(cnt + 1, 1u) == gridDim.x - 1) {
    cnt[0] = 0;
    cnt[1] = 0;
    __threadfence();
  }
}

}  // namespace dp
