// kt_tma.cuh -- Tensor Memory Accelerator loads into shared memory, completed on mbarriers.
//
// One elected thread arms an mbarrier with the expected byte count and issues a tiled
// cp.async.bulk.tensor copy of a box of a field array; every thread then waits on the barrier's
// phase.  Every wait is bounded: it gives up after max_tries polls and reports failure, so a copy
// that never completes becomes an error status instead of a hang.
#pragma once
#include <cuda.h>
#include <stdint.h>

namespace kt {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make initialised barriers visible to the asynchronous (TMA) proxy
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier generic-proxy shared-memory accesses before later async-proxy ones
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// acquire a tensor map in global memory that was (re)written before this kernel started
__device__ __forceinline__ void fence_tensormap_acquire(const CUtensorMap* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// box at coordinates (x, y, z, w) of a 4-d tensor map into shared memory; completes on bar.
// x times the element size must be a multiple of 16 bytes; dst must be 128-byte aligned.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
      : "memory");
}

// wait until the barrier completes the phase with the given parity; false after max_tries polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned max_tries) {
  const uint32_t a = smem_u32(bar);
  for (unsigned i = 0; i < max_tries; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

}  // namespace kt
