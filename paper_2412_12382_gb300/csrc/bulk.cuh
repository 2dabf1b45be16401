// Bulk global -> shared copies completed on a shared-memory mbarrier (the
// Hopper/Blackwell async copy engine, PTX cp.async.bulk + mbarrier), for the
// streaming passes: one thread moves a whole tile of a per-edge array into
// shared memory, so a block keeps tens of kilobytes in flight without
// spending registers on them.
//
// Rules kept by every caller: source and destination 16-byte aligned, sizes a
// multiple of 16 bytes; a shared buffer that threads have read is refilled
// only after a __syncthreads() and fence_proxy_async() (the generic reads
// must be ordered before the copy engine's writes); every wait is bounded.
#pragma once

#include <stdint.h>

namespace tec {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Makes initialised barriers visible to the copy engine.
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Orders this thread's earlier generic shared-memory accesses before later
// async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Arrives once on the barrier and adds `bytes` to the transaction count the
// current phase waits for.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Copies `bytes` from global `src` to shared `dst`; completion is counted on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
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

// Each try_wait suspends the thread for a bounded, hardware-chosen time, so
// this cap (about a second or more in total) only ends a wait that can never
// complete.
constexpr int MBAR_WAIT_CAP = 1 << 22;

// Waits for the phase of `bar` with the given parity; false once the cap ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (int i = 0; i < MBAR_WAIT_CAP; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

}  // namespace tec
