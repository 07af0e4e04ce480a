// Bulk asynchronous copies into shared memory and the mbarriers they complete on (PTX
// cp.async.bulk / mbarrier), with waits bounded by the global timer.
#pragma once

#include <cstdint>

namespace lpk {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Global-memory -> shared-memory bulk copy completing on an mbarrier.  dst, src 16-byte
// aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Ends an mbarrier's life (no pending arrivals or copies), so its shared memory may be reused.
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Makes mbarrier initialisations visible to the other threads and to the async proxy.
__device__ __forceinline__ void fence_mbarrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr uint64_t kWaitLimitNs = 1000000000ull;   // 1 s per wait unless ColArgs::wait_ns

// Bounded wait for phase `parity` of bar.  Returns false (after limit_ns) if it never came.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity,
                                                  uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (unsigned spin = 1;; ++spin) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((spin & 255u) == 0 && global_ns() - t0 > limit_ns) return false;
  }
}

// Barrier over all CTAs of a cooperative launch (every CTA resident), in two levels so that no
// single counter takes every arrival: CTA b arrives on counter 2 + (b % kBarFan); the last of
// each group arrives on bar[0]; the last of those bumps the generation word bar[1], on which
// the others wait (polling with a short back-off).  bar holds 2 + kBarFan zeroed words at
// launch.  The wait is bounded by the global timer; false when it gave up (the caller reports
// a timeout and stops).
constexpr int kBarFan = 16;

__device__ __forceinline__ bool grid_sync_bounded(unsigned* bar, uint64_t limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    s_ok = 1;
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    const unsigned nb = gridDim.x, b = blockIdx.x;
    const unsigned grp = b % kBarFan;
    const unsigned ngrp = nb < (unsigned)kBarFan ? nb : (unsigned)kBarFan;
    const unsigned in_grp = nb / kBarFan + (grp < nb % kBarFan ? 1u : 0u);
    __threadfence();
    bool last = false;
    if (atomicAdd(&bar[2 + grp], 1u) == in_grp - 1) {
      atomicExch(&bar[2 + grp], 0u);
      __threadfence();
      last = atomicAdd(&bar[0], 1u) == ngrp - 1;
    }
    if (last) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    } else {
      const uint64_t t0 = global_ns();
      for (unsigned spin = 1; *gen == g; ++spin) {
        __nanosleep(32);
        if ((spin & 63u) == 0 && global_ns() - t0 > limit_ns) {
          s_ok = 0;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace lpk
