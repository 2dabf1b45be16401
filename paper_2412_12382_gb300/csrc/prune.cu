// Similarity, pruning and per-edge exports.
//
// Tectonic (Table 1) keeps oriented edge u->v iff t*q >= p*(deg u + deg v);
// TW (Eq. 1) keeps it iff (3t + 2 - deg u - deg v)*q >= p, since
// wedge = |N(u) u N(v)| - t - 2 = deg u + deg v - 2t - 2; Jaccard iff
// t*q >= p*(deg u + deg v - t); K3 iff t*q >= p; K4 is the K3 test on the
// 4-clique counts (keep_edge in tec_internal.cuh).  Algorithm 1 removes only
// edges with sim < p/q, so equality keeps the edge.  Products fit int64 when
// |p|, q < 2^28; larger thresholds take the 128-bit path.
//
// The prune kernel streams the oriented edges in tiles of 2048, reads each
// edge's source row from the per-edge source table (or finds it by binary
// search in the tile's row range), writes one keep
// bit per edge and, fused, can hook the endpoints of kept edges in the
// union-find forest (the first phase of the components step).
#include "bulk.cuh"
#include "tec_internal.cuh"
#include "uf.cuh"

namespace tec {
namespace {


// The orientation puts the lower-ranked endpoint first, so deg v >= deg u and
// s = deg u + deg v >= 2 deg u.  Every survival test is non-increasing in s
// (Tectonic and Jaccard for p >= 0, TW always; for p < 0 the first two keep
// every edge; K3 ignores s), so an edge that fails it at s = 2 deg u is pruned
// without gathering deg v, which most edges of a selective threshold do.
//
// Loads of all eight items of a thread are issued before any is used (the
// row of each edge, then the degree gathers), so every thread keeps several
// loads in flight.
template <bool HOOK, bool WIDE>
__global__ void __launch_bounds__(TILE_THREADS)
k_prune(const int64_t *__restrict__ ooff, const int32_t *__restrict__ ocol, const int32_t *__restrict__ deg,
        const uint32_t *__restrict__ t, int64_t n, int64_t m, const int32_t *__restrict__ orows,
        const int32_t *__restrict__ osrc, int measure, int64_t p, int64_t q, uint32_t *__restrict__ keep,
        int32_t *parent, unsigned long long *ctr) {
    __shared__ int ws[TILE_THREADS / 32];
    if (graph_bad(ctr)) return;
    const int64_t k0 = (int64_t)blockIdx.x * TILE;
    int64_t r0, r1;
    tile_row_range(orows, ooff, n, m, r0, r1);
    const unsigned lane = lane_id();
    int32_t u[TILE_ITEMS], v[TILE_ITEMS];
    uint32_t tt[TILE_ITEMS];
#pragma unroll
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int64_t j = k0 + (int64_t)i * TILE_THREADS + threadIdx.x;
        const bool in = j < m;
        u[i] = in ? (int32_t)edge_source(osrc, ooff, r0, r1, j) : 0;
        v[i] = in ? ocol[j] : 0;
        tt[i] = in ? t[j] : 0u;
    }
    uint32_t sd[TILE_ITEMS];                   // deg u, then deg u + deg v (< 2^32)
#pragma unroll
    for (int i = 0; i < TILE_ITEMS; ++i)
        sd[i] = k0 + (int64_t)i * TILE_THREADS + threadIdx.x < m ? (uint32_t)deg[u[i]] : 0u;
    unsigned pre = 0;                          // bit i: item i passes at s = 2 deg u
#pragma unroll
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int64_t j = k0 + (int64_t)i * TILE_THREADS + threadIdx.x;
        if (j < m && keep_edge<WIDE>(measure, tt[i], 2 * (int64_t)sd[i], p, q)) {
            pre |= 1u << i;
            sd[i] += (uint32_t)deg[v[i]];
        }
    }
    int kept = 0;
#pragma unroll
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int64_t jw = k0 + (int64_t)i * TILE_THREADS + (threadIdx.x & ~31u);
        const bool kp = ((pre >> i) & 1u) && keep_edge<WIDE>(measure, tt[i], (int64_t)sd[i], p, q);
        if (HOOK && kp) uf_link(parent, u[i], v[i], ctr);
        const unsigned b = __ballot_sync(0xffffffffu, kp);
        if (lane == 0 && jw < m) keep[jw >> 5] = b;
        kept += kp ? 1 : 0;
    }
    kept = warp_sum(kept);
    if (lane == 0) ws[threadIdx.x >> 5] = kept;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < TILE_THREADS / 32; ++w) tot += ws[w];
        if (tot) atomicAdd(&ctr[C_KEPT], (unsigned long long)tot);
    }
}

// The prune test of one tile of `cnt` (<= TILE) oriented edges starting at
// j0, read from su / sv / st (shared or global memory): keep words written,
// kept edges hooked (HOOK), kept count of this thread returned.  Same load
// order and s >= 2 deg u pre-test as k_prune.
template <bool HOOK, bool WIDE>
__device__ __forceinline__ int prune_tile(const int32_t *su, const int32_t *sv, const uint32_t *st, int64_t j0,
                                          int cnt, const int32_t *__restrict__ deg, int measure, int64_t p,
                                          int64_t q, uint32_t *__restrict__ keep, int32_t *parent,
                                          unsigned long long *ctr) {
    int32_t u[TILE_ITEMS], v[TILE_ITEMS];
    uint32_t tt[TILE_ITEMS];
#pragma unroll
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int x = i * TILE_THREADS + (int)threadIdx.x;
        const bool in = x < cnt;
        u[i] = in ? su[x] : 0;
        v[i] = in ? sv[x] : 0;
        tt[i] = in ? st[x] : 0u;
    }
    uint32_t sd[TILE_ITEMS];                   // deg u, then deg u + deg v (< 2^32)
#pragma unroll
    for (int i = 0; i < TILE_ITEMS; ++i) sd[i] = i * TILE_THREADS + (int)threadIdx.x < cnt ? (uint32_t)deg[u[i]] : 0u;
    unsigned pre = 0;
#pragma unroll
    for (int i = 0; i < TILE_ITEMS; ++i) {
        if (i * TILE_THREADS + (int)threadIdx.x < cnt && keep_edge<WIDE>(measure, tt[i], 2 * (int64_t)sd[i], p, q)) {
            pre |= 1u << i;
            sd[i] += (uint32_t)deg[v[i]];
        }
    }
    const unsigned lane = lane_id();
    int kept = 0;
#pragma unroll
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int xw = i * TILE_THREADS + (int)(threadIdx.x & ~31u);
        const bool kp = ((pre >> i) & 1u) && keep_edge<WIDE>(measure, tt[i], (int64_t)sd[i], p, q);
        if (HOOK && kp) uf_link(parent, u[i], v[i], ctr);
        const unsigned b = __ballot_sync(0xffffffffu, kp);
        if (lane == 0 && xw < cnt) keep[(j0 + xw) >> 5] = b;
        kept += kp ? 1 : 0;
    }
    return kept;
}

constexpr uint32_t PB_ARRAY_BYTES = TILE * 4;                  // one array's share of a tile
constexpr size_t PB_SMEM = (size_t)BULK_STAGES * 3 * PB_ARRAY_BYTES;

// k_prune for graphs with a per-edge source table, as a persistent kernel:
// each block walks tiles blockIdx.x, + gridDim.x, ..., and while it tests one
// tile the copy engine brings the source rows, column ids and counts of its
// next tile (3 x 8 KB) into the other shared-memory stage.  A partial last
// tile is read from global memory directly.  Needs osrc, ocol and t 16-byte
// aligned.  A copy that does not land within the wait cap sets ST_TIMEOUT.
template <bool HOOK, bool WIDE>
__global__ void __launch_bounds__(TILE_THREADS)
k_prune_bulk(const int32_t *__restrict__ ocol, const int32_t *__restrict__ deg, const uint32_t *__restrict__ t,
             int64_t m, const int32_t *__restrict__ osrc, int measure, int64_t p, int64_t q,
             uint32_t *__restrict__ keep, int32_t *parent, unsigned long long *ctr) {
    extern __shared__ __align__(16) unsigned char pb_smem[];
    int32_t *buf = reinterpret_cast<int32_t *>(pb_smem);
    __shared__ uint64_t bar[BULK_STAGES];
    __shared__ int ws[TILE_THREADS / 32];
    __shared__ int s_flag;
    const int64_t full = m / TILE;
    bulk_init(bar, &s_flag);
    if (graph_bad(ctr)) return;              // uniform: nothing in this launch sets the bit
    int kept = 0;
    const bool ok = bulk_tiles(
        full, bar, &s_flag, ctr,
        [&](int64_t tile, int stage) {
            int32_t *dst = buf + (size_t)stage * 3 * TILE;
            const int64_t j0 = tile * TILE;
            fence_proxy_async();
            mbar_arrive_expect_tx(&bar[stage], 3 * PB_ARRAY_BYTES);
            bulk_g2s(dst, osrc + j0, PB_ARRAY_BYTES, &bar[stage]);
            bulk_g2s(dst + TILE, ocol + j0, PB_ARRAY_BYTES, &bar[stage]);
            bulk_g2s(dst + 2 * TILE, t + j0, PB_ARRAY_BYTES, &bar[stage]);
        },
        [&](int64_t tile, int stage) {
            const int32_t *su = buf + (size_t)stage * 3 * TILE;
            kept += prune_tile<HOOK, WIDE>(su, su + TILE, reinterpret_cast<const uint32_t *>(su + 2 * TILE),
                                           tile * TILE, TILE, deg, measure, p, q, keep, parent, ctr);
        });
    if (!ok) return;
    if (full * TILE < m && blockIdx.x == (unsigned)(full % gridDim.x)) {
        const int64_t j0 = full * TILE;
        kept += prune_tile<HOOK, WIDE>(osrc + j0, ocol + j0, t + j0, j0, (int)(m - j0), deg, measure, p, q, keep,
                                       parent, ctr);
    }
    kept = warp_sum(kept);
    if (lane_id() == 0) ws[threadIdx.x >> 5] = kept;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < TILE_THREADS / 32; ++w) tot += ws[w];
        if (tot) atomicAdd(&ctr[C_KEPT], (unsigned long long)tot);
    }
}

// Per-graph thresholds: the edge's graph is the segment of its source row.
// One block per tile; used without a per-edge source table (the persistent
// k_prune_seg_warps below is the default otherwise).
// With a third or more of the edges kept the hooks dominate and want
// occupancy: loading all eight items ahead (116 registers) took the
// 500-graph batch from 1.95 to 4.2 ms.  Items in flight per group, chosen by
// the autotuner:
constexpr int PRUNE_SEG_ITEMS = 1;

template <bool HOOK>
__global__ void __launch_bounds__(TILE_THREADS)
k_prune_seg(const int64_t *ooff, const int32_t *ocol, const int32_t *deg, const uint32_t *t, int64_t n, int64_t m,
            const int32_t *orows, const int32_t *osrc, int measure, const int64_t *sp, const int64_t *sq,
            const int64_t *seg_off, int nseg, uint32_t *keep, int32_t *parent, unsigned long long *ctr) {
    __shared__ int ws[TILE_THREADS / 32];
    if (graph_bad(ctr)) return;
    const int64_t k0 = (int64_t)blockIdx.x * TILE;
    int64_t r0, r1;
    tile_row_range(orows, ooff, n, m, r0, r1);
    // the segments of the tile's rows: one search per tile, and per edge only
    // when the tile spans several graphs
    int s0 = 0, s1 = nseg - 1;
    while (s0 < s1) {
        const int mid = (s0 + s1 + 1) >> 1;
        if (seg_off[mid] <= r0) s0 = mid; else s1 = mid - 1;
    }
    {
        int lo = s0, hi = nseg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (seg_off[mid] <= r1) lo = mid; else hi = mid - 1;
        }
        s1 = lo;
    }
    const unsigned lane = lane_id();
    int kept = 0;
    // PRUNE_SEG_ITEMS items at a time: their loads are issued together, then
    // their kept edges are hooked
    static_assert(TILE_ITEMS % PRUNE_SEG_ITEMS == 0, "whole groups of items");
    for (int i0 = 0; i0 < TILE_ITEMS; i0 += PRUNE_SEG_ITEMS) {
        int32_t u[PRUNE_SEG_ITEMS], v[PRUNE_SEG_ITEMS];
        bool kp[PRUNE_SEG_ITEMS];
#pragma unroll
        for (int b = 0; b < PRUNE_SEG_ITEMS; ++b) {
            const int64_t j = k0 + (int64_t)(i0 + b) * TILE_THREADS + threadIdx.x;
            kp[b] = false;
            u[b] = v[b] = 0;
            if (j < m) {
                u[b] = (int32_t)edge_source(osrc, ooff, r0, r1, j);
                int lo = s0, hi = s1;                // segment of u
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (seg_off[mid] <= u[b]) lo = mid; else hi = mid - 1;
                }
                v[b] = ocol[j];
                const int64_t s = (int64_t)deg[u[b]] + deg[v[b]];
                const int64_t p = sp[lo], q = sq[lo];
                kp[b] = q > 0 && (needs_wide_dev(p, q) ? keep_edge<true>(measure, t[j], s, p, q)
                                                       : keep_edge<false>(measure, t[j], s, p, q));
            }
        }
#pragma unroll
        for (int b = 0; b < PRUNE_SEG_ITEMS; ++b) {
            const int64_t jw = k0 + (int64_t)(i0 + b) * TILE_THREADS + (threadIdx.x & ~31u);
            if (HOOK && kp[b]) uf_link(parent, u[b], v[b], ctr);
            const unsigned w = __ballot_sync(0xffffffffu, kp[b]);
            if (lane == 0 && jw < m) keep[jw >> 5] = w;
            kept += kp[b] ? 1 : 0;
        }
    }
    kept = warp_sum(kept);
    if (lane == 0) ws[threadIdx.x >> 5] = kept;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < TILE_THREADS / 32; ++w) tot += ws[w];
        if (tot) atomicAdd(&ctr[C_KEPT], (unsigned long long)tot);
    }
}

// k_prune_seg as a persistent kernel of independent warps: each warp walks
// chunks of 256 consecutive edges (8 rounds of 32), chunk c, c + total warps,
// ...; it finds the graphs of its chunk's first and last edge itself, so no
// block barrier stands between chunks and a warp held up by long union-find
// walks keeps only itself waiting, not the other warps of a block.  Needs the
// per-edge source table.  Chosen by the autotuner (PRUNE_SEG_PERSISTENT).
constexpr int PRUNE_SEG_PERSISTENT = 1;
constexpr int PS_CHUNK = 256;

__device__ __forceinline__ int seg_search(const int64_t *seg_off, int lo, int hi, int64_t x) {
    while (lo < hi) {                            // last segment in [lo, hi] starting at or before x
        const int mid = (lo + hi + 1) >> 1;
        if (seg_off[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <bool HOOK>
__global__ void __launch_bounds__(TILE_THREADS)
k_prune_seg_warps(const int32_t *__restrict__ ocol, const int32_t *__restrict__ deg, const uint32_t *__restrict__ t,
                  int64_t m, const int32_t *__restrict__ osrc, int measure, const int64_t *__restrict__ sp,
                  const int64_t *__restrict__ sq, const int64_t *__restrict__ seg_off, int nseg,
                  uint32_t *__restrict__ keep, int32_t *parent, unsigned long long *ctr) {
    __shared__ int ws[TILE_THREADS / 32];
    if (graph_bad(ctr)) return;
    const unsigned lane = lane_id();
    const int64_t warps = (int64_t)gridDim.x * (TILE_THREADS / 32);
    const int64_t nchunks = ceil_div(m, PS_CHUNK);
    int kept = 0;
    for (int64_t c = (int64_t)blockIdx.x * (TILE_THREADS / 32) + (threadIdx.x >> 5); c < nchunks; c += warps) {
        const int64_t j0 = c * PS_CHUNK;
        const int64_t jl = (j0 + PS_CHUNK < m ? j0 + PS_CHUNK : m) - 1;
        // lane 0 finds the graph of the first edge, lane 1 that of the last
        const int mine = lane < 2 ? seg_search(seg_off, 0, nseg - 1, osrc[lane == 0 ? j0 : jl]) : 0;
        const int s0 = __shfl_sync(0xffffffffu, mine, 0), s1 = __shfl_sync(0xffffffffu, mine, 1);
        for (int i = 0; i < PS_CHUNK / 32; ++i) {
            const int64_t jw = j0 + i * 32;
            const int64_t j = jw + lane;
            bool kp = false;
            if (j < m) {
                const int32_t u = osrc[j];
                const int lo = seg_search(seg_off, s0, s1, u);
                const int32_t v = ocol[j];
                const int64_t s = (int64_t)deg[u] + deg[v];
                const int64_t p = sp[lo], q = sq[lo];
                kp = q > 0 && (needs_wide_dev(p, q) ? keep_edge<true>(measure, t[j], s, p, q)
                                                    : keep_edge<false>(measure, t[j], s, p, q));
                if (HOOK && kp) uf_link(parent, u, v, ctr);
            }
            const unsigned b = __ballot_sync(0xffffffffu, kp);
            if (lane == 0 && jw < m) keep[jw >> 5] = b;
            kept += kp ? 1 : 0;
        }
    }
    kept = warp_sum(kept);
    if (lane == 0) ws[threadIdx.x >> 5] = kept;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < TILE_THREADS / 32; ++w) tot += ws[w];
        if (tot) atomicAdd(&ctr[C_KEPT], (unsigned long long)tot);
    }
}

// Number of neighbours greater than u in each row (the canonical edges the row owns).
__global__ void k_upper_counts(const int64_t *off, const int32_t *col, int64_t n, int32_t *cnt) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = off[u], hi = off[u + 1];
        const int64_t end = hi;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (col[mid] <= u) lo = mid + 1; else hi = mid;
        }
        cnt[u] = (int32_t)(end - lo);
    }
}

// One thread per symmetric entry (u, v) with u < v: canonical id
// e = uoff[u+1] - (off[u+1] - k); the oriented copy of the edge sits in the row
// of the lower-ranked endpoint, found by binary search (rows are sorted).
__global__ void __launch_bounds__(TILE_THREADS)
k_export(const int64_t *off, const int32_t *col, const int32_t *deg, const int64_t *ooff,
         const int32_t *ocol, const uint32_t *t, const uint32_t *keep, int64_t n, int64_t nnz,
         const int64_t *uoff, int32_t *u_out, int32_t *v_out, uint32_t *t_out, uint32_t *wedge_out,
         double *w_out, int w_measure, uint8_t *keep_out, unsigned long long *ctr) {
    if (graph_bad(ctr)) return;
    const int64_t k0 = (int64_t)blockIdx.x * TILE;
    const int64_t klast = min(k0 + TILE, nnz) - 1;
    const int64_t r0 = row_search(off, 0, n - 1, k0);
    const int64_t r1 = row_search(off, r0, n - 1, klast);
    const bool need_pos = t_out || wedge_out || w_out || keep_out;
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int64_t k = k0 + (int64_t)i * TILE_THREADS + threadIdx.x;
        if (k >= nnz) break;
        const int64_t u = row_search(off, r0, r1, k);
        const int32_t v = col[k];
        if (v <= u) continue;
        const int64_t e = uoff[u + 1] - (off[u + 1] - k);
        if (u_out) u_out[e] = (int32_t)u;
        if (v_out) v_out[e] = v;
        if (!need_pos) continue;
        const int32_t du = deg[u], dv = deg[v];
        const bool u_first = rank_less(du, u, dv, v);
        const int64_t x = u_first ? u : v;
        const int32_t y = u_first ? v : (int32_t)u;
        int64_t lo = ooff[x], hi = ooff[x + 1];
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (ocol[mid] < y) lo = mid + 1; else hi = mid;
        }
        const int64_t pos = lo;
        const uint32_t tt = t ? t[pos] : 0u;
        const int64_t s = (int64_t)du + dv;
        if (t_out) t_out[e] = tt;
        if (wedge_out) wedge_out[e] = (uint32_t)(s - 2 * (int64_t)tt - 2);
        if (w_out) {
            if (w_measure == TEC_TECTONIC) w_out[e] = __ddiv_rn((double)tt, (double)s);
            else if (w_measure == TEC_JACCARD) w_out[e] = __ddiv_rn((double)tt, (double)(s - (int64_t)tt));
            else if (w_measure == TEC_K3) w_out[e] = (double)tt;
            else w_out[e] = (double)(3 * (int64_t)tt + 2 - s);
        }
        if (keep_out) keep_out[e] = (uint8_t)((keep[pos >> 5] >> (pos & 31)) & 1u);
    }
}

}  // namespace

// Persistent launch of k_prune_bulk: as many blocks as fit on the device at
// once (48 KB of stages each), at most one per full tile.
template <bool HOOK, bool WIDE>
cudaError_t launch_bulk(const int32_t *ocol, const int32_t *deg, const uint32_t *t, int64_t m, const int32_t *osrc,
                        const PruneArgs &a, uint32_t *keep, int32_t *parent, unsigned long long *ctr,
                        cudaStream_t s) {
    cudaError_t e =
        cudaFuncSetAttribute(k_prune_bulk<HOOK, WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PB_SMEM);
    unsigned grid = 1;
    if (e == cudaSuccess) e = persistent_grid(k_prune_bulk<HOOK, WIDE>, TILE_THREADS, PB_SMEM, m / TILE, &grid);
    if (e != cudaSuccess) return e;
    k_prune_bulk<HOOK, WIDE><<<grid, TILE_THREADS, PB_SMEM, s>>>(ocol, deg, t, m, osrc, a.measure, a.p, a.q, keep,
                                                                 parent, ctr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_prune(const int64_t *ooff, const int32_t *ocol, const int32_t *deg, const uint32_t *t,
                         int64_t n, int64_t m, const int32_t *orows, const int32_t *osrc, PruneArgs a, uint32_t *keep,
                         int32_t *parent,
                         unsigned long long *ctr, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)ceil_div(m, TILE);
    const bool wide = needs_wide(a.p, a.q);
    const bool aligned = ((uintptr_t)osrc | (uintptr_t)ocol | (uintptr_t)t) % 16 == 0;
    if (osrc && aligned && m >= 2 * TILE) {
        if (a.hook) return wide ? launch_bulk<true, true>(ocol, deg, t, m, osrc, a, keep, parent, ctr, s)
                                : launch_bulk<true, false>(ocol, deg, t, m, osrc, a, keep, parent, ctr, s);
        return wide ? launch_bulk<false, true>(ocol, deg, t, m, osrc, a, keep, parent, ctr, s)
                    : launch_bulk<false, false>(ocol, deg, t, m, osrc, a, keep, parent, ctr, s);
    }
    if (a.hook) {
        if (wide) k_prune<true, true><<<grid, TILE_THREADS, 0, s>>>(ooff, ocol, deg, t, n, m, orows, osrc, a.measure, a.p, a.q, keep, parent, ctr);
        else k_prune<true, false><<<grid, TILE_THREADS, 0, s>>>(ooff, ocol, deg, t, n, m, orows, osrc, a.measure, a.p, a.q, keep, parent, ctr);
    } else {
        if (wide) k_prune<false, true><<<grid, TILE_THREADS, 0, s>>>(ooff, ocol, deg, t, n, m, orows, osrc, a.measure, a.p, a.q, keep, parent, ctr);
        else k_prune<false, false><<<grid, TILE_THREADS, 0, s>>>(ooff, ocol, deg, t, n, m, orows, osrc, a.measure, a.p, a.q, keep, parent, ctr);
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_prune_seg(const int64_t *ooff, const int32_t *ocol, const int32_t *deg, const uint32_t *t,
                             int64_t n, int64_t m, const int32_t *orows, const int32_t *osrc, int measure,
                             const int64_t *sp, const int64_t *sq,
                             const int64_t *seg_off, int nseg, bool hook, uint32_t *keep, int32_t *parent,
                             unsigned long long *ctr, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    if (PRUNE_SEG_PERSISTENT && osrc) {
        unsigned pgrid = 1;
        cudaError_t e = hook ? persistent_grid(k_prune_seg_warps<true>, TILE_THREADS, 0, ceil_div(m, PS_CHUNK), &pgrid)
                             : persistent_grid(k_prune_seg_warps<false>, TILE_THREADS, 0, ceil_div(m, PS_CHUNK), &pgrid);
        if (e != cudaSuccess) return e;
        if (hook) k_prune_seg_warps<true><<<pgrid, TILE_THREADS, 0, s>>>(ocol, deg, t, m, osrc, measure, sp, sq, seg_off, nseg, keep, parent, ctr);
        else k_prune_seg_warps<false><<<pgrid, TILE_THREADS, 0, s>>>(ocol, deg, t, m, osrc, measure, sp, sq, seg_off, nseg, keep, parent, ctr);
        count_launches(1);
        return cudaGetLastError();
    }
    const unsigned grid = (unsigned)ceil_div(m, TILE);
    if (hook) k_prune_seg<true><<<grid, TILE_THREADS, 0, s>>>(ooff, ocol, deg, t, n, m, orows, osrc, measure, sp, sq, seg_off, nseg, keep, parent, ctr);
    else k_prune_seg<false><<<grid, TILE_THREADS, 0, s>>>(ooff, ocol, deg, t, n, m, orows, osrc, measure, sp, sq, seg_off, nseg, keep, parent, ctr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_upper_counts(const int64_t *off, const int32_t *col, int64_t n, int32_t *cnt, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t g = ceil_div(n, 256);
    k_upper_counts<<<(unsigned)(g < 65536 ? g : 65536), 256, 0, s>>>(off, col, n, cnt);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_export(const int64_t *off, const int32_t *col, const int32_t *deg, const int64_t *ooff,
                          const int32_t *ocol, const uint32_t *t, const uint32_t *keep, int64_t n,
                          int64_t nnz, const int64_t *uoff, int32_t *u_out, int32_t *v_out,
                          uint32_t *t_out, uint32_t *wedge_out, double *w_out, int w_measure,
                          uint8_t *keep_out, unsigned long long *ctr, cudaStream_t s) {
    if (nnz <= 0) return cudaSuccess;
    k_export<<<(unsigned)ceil_div(nnz, TILE), TILE_THREADS, 0, s>>>(off, col, deg, ooff, ocol, t, keep, n, nnz,
                                                                   uoff, u_out, v_out, t_out, wedge_out,
                                                                   w_out, w_measure, keep_out, ctr);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace tec
