// Bulk global -> shared copies completed on a shared-memory mbarrier (the
// Hopper/Blackwell async copy engine, PTX cp.async.bulk + mbarrier), for the
// streaming passes: one thread moves a whole tile of a per-edge array into
// shared memory, so a block keeps tens of kilobytes in flight without
// spending registers on them.
//
// bulk_tiles runs the double-buffered persistent loop the streaming kernels
// share.  Rules kept by every caller: source and destination 16-byte aligned, sizes a
// multiple of 16 bytes; a shared buffer that threads have read is refilled
// only after a __syncthreads() and fence_proxy_async() (the generic reads
// must be ordered before the copy engine's writes); every wait is bounded.
#pragma once

#include <stdint.h>

#include "tec_internal.cuh"

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

constexpr int BULK_STAGES = 2;

// Initialises the two stage barriers and the block's abort flag.
__device__ __forceinline__ void bulk_init(uint64_t *bar, int *s_flag) {
    if (threadIdx.x == 0) {
        for (int x = 0; x < BULK_STAGES; ++x) mbar_init(&bar[x], 1);
        fence_mbar_init();
        *s_flag = 0;
    }
    __syncthreads();
}

// Persistent walk over the tiles blockIdx.x, + gridDim.x, ... below `full`
// with a two-stage copy pipeline: while body(tile, stage) (all threads) works
// on one tile, the copies of the next one, started by issue(tile, stage)
// (thread 0 only; it must arm bar[stage] with mbar_arrive_expect_tx before
// its copies), land in the other stage.  Returns false when a wait ran out:
// ST_TIMEOUT is then set and the copies still in flight have been waited for
// (bounded) so that the block can exit.
template <class Issue, class Body>
__device__ __forceinline__ bool bulk_tiles(int64_t full, uint64_t *bar, int *s_flag, unsigned long long *ctr,
                                           Issue &&issue, Body &&body) {
    int64_t tile = blockIdx.x;
    if (threadIdx.x == 0 && tile < full) issue(tile, 0);
    uint32_t phase = 0;                        // bit x: parity of stage x's next phase
    uint32_t pending = tile < full ? 1u : 0u;  // bit x: a copy into stage x not yet waited for
    for (int it = 0; tile < full; ++it, tile += gridDim.x) {
        const int stage = it & 1;
        const int64_t nxt = tile + gridDim.x;
        if (nxt < full) {
            if (threadIdx.x == 0) issue(nxt, stage ^ 1);
            pending |= 1u << (stage ^ 1);
        }
        if (!mbar_wait(&bar[stage], (phase >> stage) & 1u)) *s_flag = 1;
        phase ^= 1u << stage;
        pending &= ~(1u << stage);
        __syncthreads();
        if (*s_flag) break;
        body(tile, stage);
        fence_proxy_async();                   // the stage is read before the copy engine refills it
        __syncthreads();
    }
    if (*s_flag) {
        if (threadIdx.x == 0) {
            flag_status(ctr, ST_TIMEOUT);
            for (int x = 0; x < BULK_STAGES; ++x)
                if ((pending >> x) & 1u) mbar_wait(&bar[x], (phase >> x) & 1u);
        }
        return false;
    }
    return true;
}

// Blocks of a persistent launch: as many as fit on the device at once, at
// most one per full tile, at least one.
template <class K>
cudaError_t persistent_grid(K kernel, int threads, size_t dyn_smem, int64_t full, unsigned *grid) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, dyn_smem);
    if (e != cudaSuccess) return e;
    const int64_t want = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    *grid = (unsigned)(full < 1 ? 1 : (want < full ? want : full));
    return cudaSuccess;
}

}  // namespace tec
