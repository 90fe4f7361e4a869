// iwpp_tma.cuh -- Tensor Memory Accelerator (TMA) staging of tile boxes and
// the mbarrier that tracks them, as inline PTX for sm_103a.
//
// A tile visit stages a 2-D box (tile + halo, widened so that the box's
// first column is 16-byte aligned) with one cp.async.bulk.tensor per image;
// the transaction count on the CTA's mbarrier completes when all bytes have
// landed.  Out-of-image parts of a box are zero-filled by the hardware.
// Every wait is bounded by a deadline on %globaltimer.
#pragma once

#include <cuda.h>
#include <cstdint>

#include "iwpp_device.cuh"

namespace iwpp {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
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

// Waits for phase `parity` of the barrier; false if `deadline` passed first.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned long long deadline) {
    while (!mbar_try_wait(bar, parity)) {
        if (globaltimer_ns() > deadline) return false;
    }
    return true;
}

// Orders this thread's earlier generic-proxy shared-memory accesses (made
// visible to it by a barrier) before later async-proxy (TMA) writes.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 2-D tiled bulk tensor load of the box at element coordinates (x, y) into
// shared memory, completing `bytes` transactions on `bar`.  x must make the
// box start 16-byte aligned (multiple of 16 for u8, of 4 for int32).
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace iwpp
