// K4 participation (Table 1, kappa = 4): for every oriented edge x -> y the
// number of 4-cliques containing it, i.e. the number of edges {c, d} with both
// ends in the common neighbourhood C = N(x) n N(y) (|C| = t(x, y)).
//
// One warp per edge; warps take edges 4 at a time from a counter.  When |C|
// fits the warp's shared slice, C is built there in sorted order (each id of
// the shorter row is binary-searched in the longer one; a ballot keeps the
// order) and every c in C then counts the d of its oriented row N+(c) that
// lie in C, by binary search in the slice.  Each edge {c, d} of C is oriented
// one way only, so it is counted once.  A larger C is walked the same way
// without being stored, membership tested by binary search in both rows.
// Counts saturate at 2^32 - 1.
#include "tec_internal.cuh"

namespace tec {
namespace {

constexpr int K4_CAP = 3072;       // ids of C per warp slice (dynamic shared memory, 12 KB)
constexpr int K4_WARPS = 8;
constexpr int K4_GRAB = 4;         // edges per counter bump: heavy edges of one row spread over warps
constexpr size_t K4_SMEM = (size_t)K4_WARPS * K4_CAP * sizeof(int32_t);

__device__ __forceinline__ bool in_row(const int32_t *a, int64_t lo, int64_t hi, int32_t x) {
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        const int32_t v = a[mid];
        if (v == x) return true;
        if (v < x) lo = mid + 1; else hi = mid;
    }
    return false;
}

__device__ __forceinline__ bool in_slice(const int32_t *a, int n, int32_t x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int32_t v = a[mid];
        if (v == x) return true;
        if (v < x) lo = mid + 1; else hi = mid;
    }
    return false;
}

// Edges {c, d} with c the id c (in C) and d in N+(c) n C, C given either as
// the warp's slice (n_c >= 0) or as the two rows [ax, ax_end) and [ay, ay_end).
__device__ __forceinline__ unsigned long long count_from(const int64_t *ooff, const int32_t *ocol,
                                                         const int32_t *col, int32_t c, const int32_t *slice,
                                                         int n_c, int64_t ax, int64_t ax_end, int64_t ay,
                                                         int64_t ay_end) {
    const unsigned lane = lane_id();
    unsigned long long cnt = 0;
    const int64_t r0 = ooff[c], r1 = ooff[c + 1];
    for (int64_t i = r0; i < r1; i += 32) {
        const int64_t k = i + lane;
        bool hit = false;
        if (k < r1) {
            const int32_t d = ocol[k];
            hit = n_c >= 0 ? in_slice(slice, n_c, d) : (in_row(col, ax, ax_end, d) && in_row(col, ay, ay_end, d));
        }
        cnt += __popc(__ballot_sync(0xffffffffu, hit));
    }
    return cnt;
}

__global__ void __launch_bounds__(K4_WARPS * 32)
k_edge_k4(const int64_t *off, const int32_t *col, const int64_t *ooff, const int32_t *ocol, const uint32_t *t,
          int64_t n, int64_t m, unsigned long long *next, uint32_t *k4, unsigned long long *ctr) {
    extern __shared__ int32_t s_c[];
    if (graph_bad(ctr)) return;
    const unsigned lane = lane_id();
    int32_t *slice = s_c + (threadIdx.x >> 5) * K4_CAP;
    for (;;) {
        unsigned long long g0 = 0;
        if (lane == 0) g0 = atomicAdd(next, (unsigned long long)K4_GRAB);
        g0 = __shfl_sync(0xffffffffu, g0, 0);
        if ((int64_t)g0 >= m) break;
        const int64_t j1 = min(m, (int64_t)g0 + K4_GRAB);
        int64_t x = row_search(ooff, 0, n - 1, (int64_t)g0);
        for (int64_t j = (int64_t)g0; j < j1; ++j) {
            while (ooff[x + 1] <= j) ++x;          // row of edge j (rows may be empty)
            const int32_t y = ocol[j];
            const uint32_t tc = t[j];
            unsigned long long total = 0;
            if (tc >= 2) {
                int64_t ax = off[x], ax_end = off[x + 1], ay = off[y], ay_end = off[y + 1];
                // probe the shorter row against the longer
                int64_t s0 = ax, s1 = ax_end, l0 = ay, l1 = ay_end;
                if (s1 - s0 > l1 - l0) {
                    s0 = ay; s1 = ay_end; l0 = ax; l1 = ax_end;
                }
                const bool stored = tc <= (uint32_t)K4_CAP;
                int nc = 0;
                for (int64_t i = s0; i < s1; i += 32) {
                    const int64_t k = i + lane;
                    int32_t v = -1;
                    bool found = false;
                    if (k < s1) {
                        v = col[k];
                        found = in_row(col, l0, l1, v);
                    }
                    const unsigned fm = __ballot_sync(0xffffffffu, found);
                    if (stored) {
                        if (found) slice[nc + __popc(fm & ((1u << lane) - 1u))] = v;
                        nc += __popc(fm);
                    } else {
                        for (unsigned mm = fm; mm; mm &= mm - 1) {   // walk C without storing it
                            const int32_t c = __shfl_sync(0xffffffffu, v, __ffs(mm) - 1);
                            total += count_from(ooff, ocol, col, c, nullptr, -1, ax, ax_end, ay, ay_end);
                        }
                    }
                }
                if (stored) {
                    __syncwarp();
                    for (int a = 0; a < nc; ++a)
                        total += count_from(ooff, ocol, col, slice[a], slice, nc, ax, ax_end, ay, ay_end);
                    __syncwarp();
                }
            }
            if (lane == 0) k4[j] = total > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)total;
        }
    }
}

}  // namespace

cudaError_t launch_k4(const int64_t *off, const int32_t *col, const int64_t *ooff, const int32_t *ocol,
                      const uint32_t *t, int64_t n, int64_t m, unsigned long long *next, uint32_t *k4,
                      unsigned long long *ctr, int num_sms, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_edge_k4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K4_SMEM);
    if (e != cudaSuccess) return e;
    k_edge_k4<<<(unsigned)(num_sms * 2), K4_WARPS * 32, K4_SMEM, s>>>(off, col, ooff, ocol, t, n, m, next, k4, ctr);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace tec
