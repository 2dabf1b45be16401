// Per-edge triangle counts t(u,v) = |N(u) n N(v)| (Sec. I) on the oriented CSR.
//
// Every triangle {u, v, w} with (deg, id)-rank u < v < w is listed exactly once,
// from u: v runs over N+(u) and w over N+(v) n N+(u).  It is credited to its
// three edges: u->v and u->w live in row u (accumulated by the owning warp or
// block in shared memory, one global add per edge), v->w lives in row v (one
// global atomic add per triangle).  Integer sums do not depend on the order of
// the adds, so the counts are exact and deterministic.
//
// Work is binned by out-degree d+(u):
//   d+(u) <= 32   one warp per u, N+(u) held one id per lane, membership of
//                 each w by a 5-step lane-shuffle binary search;
//   d+(u) >  32   one block per u, N+(u) staged in shared memory in chunks of
//                 8192 ids, membership by binary search in shared memory,
//                 blocks take vertices from a global work counter.
// Reads of N+(v) are coalesced: a warp reads consecutive ids of one row.
#include <climits>

#include "tec_internal.cuh"

namespace tec {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int SUP_THREADS = 256;
constexpr int SUP_WARPS = SUP_THREADS / 32;

__global__ void k_classify(const int64_t *ooff, int64_t n, int32_t *vlist, unsigned long long *ctr) {
    if (graph_bad(ctr)) return;
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t u = base + threadIdx.x;
        const int64_t d = u < n ? ooff[u + 1] - ooff[u] : 0;
        const bool small = d > 0 && d <= SMALL_ROW;
        const bool large = d > SMALL_ROW;
        const unsigned ms = __ballot_sync(FULL, small);
        const unsigned ml = __ballot_sync(FULL, large);
        unsigned long long bs = 0, bl = 0;
        if (lane == 0) {
            if (ms) bs = atomicAdd(&ctr[C_NSMALL], (unsigned long long)__popc(ms));
            if (ml) bl = atomicAdd(&ctr[C_NLARGE], (unsigned long long)__popc(ml));
        }
        bs = __shfl_sync(FULL, bs, 0);
        bl = __shfl_sync(FULL, bl, 0);
        if (small) vlist[bs + __popc(ms & lt)] = (int32_t)u;
        if (large) vlist[n - 1 - (int64_t)(bl + __popc(ml & lt))] = (int32_t)u;
    }
}

__global__ void __launch_bounds__(SUP_THREADS)
k_support_small(const int64_t *ooff, const int32_t *ocol, uint32_t *t, const int32_t *vlist,
                const unsigned long long *ctr) {
    __shared__ uint32_t s_cnt[SUP_WARPS][32];
    if (graph_bad(ctr)) return;
    const unsigned lane = lane_id();
    const int w = threadIdx.x >> 5;
    const int64_t nsmall = (int64_t)ctr[C_NSMALL];
    for (int64_t it = (int64_t)blockIdx.x * SUP_WARPS + w; it < nsmall; it += (int64_t)gridDim.x * SUP_WARPS) {
        const int32_t u = vlist[it];
        const int64_t ub = ooff[u];
        const int du = (int)(ooff[u + 1] - ub);
        const int32_t a = (int)lane < du ? ocol[ub + lane] : INT_MAX;   // ascending over lanes
        s_cnt[w][lane] = 0u;
        __syncwarp();
        for (int j = 0; j < du; ++j) {
            const int32_t v = __shfl_sync(FULL, a, j);
            const int64_t vb = ooff[v], ve = ooff[v + 1];
            int hits = 0;
            for (int64_t kb = vb; kb < ve; kb += 32) {
                const int64_t k = kb + lane;
                const int32_t x = k < ve ? ocol[k] : -1;
                int p = 0;
#pragma unroll
                for (int st = 16; st >= 1; st >>= 1) {
                    const int32_t c = __shfl_sync(FULL, a, p + st - 1);
                    if (c < x) p += st;
                }
                const int32_t ap = __shfl_sync(FULL, a, p);
                if (x >= 0 && ap == x) {
                    ++hits;
                    atomicAdd(&s_cnt[w][p], 1u);      // edge u -> x
                    atomicAdd(&t[k], 1u);             // edge v -> x
                }
            }
            hits = warp_sum(hits);
            if (lane == 0 && hits) atomicAdd(&s_cnt[w][j], (uint32_t)hits);   // edge u -> v
        }
        __syncwarp();
        if ((int)lane < du) {
            const uint32_t c = s_cnt[w][lane];
            if (c) atomicAdd(&t[ub + lane], c);
        }
        __syncwarp();
    }
}

__device__ __forceinline__ int64_t lower_bound_g(const int32_t *a, int64_t lo, int64_t hi, int32_t x) {
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(SUP_THREADS)
k_support_large(const int64_t *ooff, const int32_t *ocol, int64_t n, uint32_t *t, const int32_t *vlist,
                unsigned long long *ctr) {
    extern __shared__ int32_t smem[];
    int32_t *s_a = smem;
    uint32_t *s_cnt = reinterpret_cast<uint32_t *>(smem + LARGE_CHUNK);
    __shared__ long long s_item;
    if (graph_bad(ctr)) return;
    const unsigned lane = lane_id();
    const int w = threadIdx.x >> 5;
    const int64_t nlarge = (int64_t)ctr[C_NLARGE];
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(&ctr[C_NEXT], 1ull);
        __syncthreads();
        const int64_t it = s_item;
        __syncthreads();
        if (it >= nlarge) break;
        const int32_t u = vlist[n - 1 - it];
        const int64_t ub = ooff[u];
        const int64_t du = ooff[u + 1] - ub;
        const bool chunked = du > LARGE_CHUNK;
        for (int64_t c0 = 0; c0 < du; c0 += LARGE_CHUNK) {
            const int cl = (int)(du - c0 < LARGE_CHUNK ? du - c0 : LARGE_CHUNK);
            for (int i = threadIdx.x; i < cl; i += SUP_THREADS) {
                s_a[i] = ocol[ub + c0 + i];
                s_cnt[i] = 0u;
            }
            __syncthreads();
            const int32_t lo_val = s_a[0], hi_val = s_a[cl - 1];
            for (int64_t j = w; j < du; j += SUP_WARPS) {
                const int32_t v = ocol[ub + j];
                int64_t vb = ooff[v], ve = ooff[v + 1];
                if (chunked) {
                    vb = lower_bound_g(ocol, vb, ve, lo_val);
                    ve = lower_bound_g(ocol, vb, ve, hi_val == INT_MAX ? hi_val : hi_val + 1);
                }
                int hits = 0;
                for (int64_t k = vb + lane; k < ve; k += 32) {
                    const int32_t x = ocol[k];
                    int lo = 0, hi = cl;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (s_a[mid] < x) lo = mid + 1; else hi = mid;
                    }
                    if (lo < cl && s_a[lo] == x) {
                        ++hits;
                        atomicAdd(&s_cnt[lo], 1u);     // edge u -> x
                        atomicAdd(&t[k], 1u);          // edge v -> x
                    }
                }
                hits = warp_sum(hits);
                if (lane == 0 && hits) atomicAdd(&t[ub + j], (uint32_t)hits);   // edge u -> v
            }
            __syncthreads();
            for (int i = threadIdx.x; i < cl; i += SUP_THREADS) {
                const uint32_t c = s_cnt[i];
                if (c) atomicAdd(&t[ub + c0 + i], c);
            }
            __syncthreads();
        }
    }
}

__global__ void k_reset_support_counters(unsigned long long *ctr) {
    ctr[C_NSMALL] = 0;
    ctr[C_NLARGE] = 0;
    ctr[C_NEXT] = 0;
}

}  // namespace

cudaError_t launch_support(const int64_t *ooff, const int32_t *ocol, int64_t n, int64_t m, uint32_t *t,
                           int32_t *vlist, unsigned long long *ctr, int num_sms, cudaStream_t s) {
    const int large_smem = 2 * LARGE_CHUNK * (int)sizeof(int32_t);
    {
        cudaError_t e = cudaFuncSetAttribute(k_support_large, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             large_smem);
        if (e != cudaSuccess) return e;
    }
    if (m > 0) {
        cudaError_t e = cudaMemsetAsync(t, 0, (size_t)m * sizeof(uint32_t), s);
        if (e != cudaSuccess) return e;
    }
    if (n <= 0 || m <= 0) return cudaSuccess;
    k_reset_support_counters<<<1, 1, 0, s>>>(ctr);
    {
        int64_t g = ceil_div(n, 256);
        k_classify<<<(unsigned)(g < 65536 ? g : 65536), 256, 0, s>>>(ooff, n, vlist, ctr);
    }
    k_support_small<<<(unsigned)(num_sms * 8), SUP_THREADS, 0, s>>>(ooff, ocol, t, vlist, ctr);
    k_support_large<<<(unsigned)(num_sms * 2), SUP_THREADS, large_smem, s>>>(ooff, ocol, n, t, vlist, ctr);
    count_launches(4);
    return cudaGetLastError();
}

}  // namespace tec
