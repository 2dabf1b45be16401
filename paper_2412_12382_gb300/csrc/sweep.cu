// Components at many thresholds at once (tec_sweep).
//
// For thresholds theta_1 <= ... <= theta_k (sorted ascending), the graph kept
// at theta_i is G_i = {e : sim(e) >= theta_i} (Algorithm 1), and
// G_k c ... c G_1.  Each edge gets its level L(e) = #{i : sim(e) >= theta_i},
// decided exactly like tec_prune, so e is in G_i iff L(e) >= i.
//
// 1. Boruvka maximum spanning forest F under the key (L(e), -edge index),
//    edges with L >= 1 only: every round each component picks its heaviest
//    incident edge (64-bit atomicMax of the packed key at both roots) and the
//    picked edges are hooked with the union-find; a pick that joins two trees
//    is a forest edge (bit 7 of the level byte).  By the cut property, G_i and
//    F_i = {e in F : L(e) >= i} have the same components for every i.  The
//    first round runs inside the level pass; later rounds read a list of the
//    edges that still join two trees, compacted in place every round.
// 2. Offline sweep: forest edges are bucketed by level; starting from
//    singletons, level i = k .. 1 unions bucket i and then snapshots every
//    vertex's root (the component minimum) as the labels at theta_i.
// A batch of graphs is one disjoint union: with a segment table the snapshot
// writes labels relative to each graph's first vertex and counts components
// per graph.
#include <algorithm>
#include <atomic>

#include "msf_key.h"
#include "tec_internal.cuh"
#include "uf.cuh"

namespace tec {
namespace {

constexpr uint8_t FOREST_BIT = 0x80;

__device__ __forceinline__ uint64_t msf_key(uint8_t L, int64_t j) { return msf_key_pack(L, j); }

// Exclusive prefix of per-thread counts over a TILE_THREADS block; *total gets the block sum.
__device__ __forceinline__ int block_excl_prefix(int c, int *total) {
    __shared__ int s_w[TILE_THREADS / 32];
    const unsigned lane = lane_id();
    const int w = (int)(threadIdx.x >> 5);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += y;
    }
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    int base = 0, all = 0;
#pragma unroll
    for (int i = 0; i < TILE_THREADS / 32; ++i) {
        base += i < w ? s_w[i] : 0;
        all += s_w[i];
    }
    *total = all;
    return base + incl - c;
}

// Edge levels and the first Boruvka round in one pass.  Every vertex is
// still its own tree, so each edge with L >= 1 offers itself to both
// endpoints.  With COMPACT the tile's offered edges are also written to its
// region of the live-edge list (lu, lv, lk at [tile * TILE, + rcnt[tile])).
template <bool WIDE, bool COMPACT>
__global__ void __launch_bounds__(TILE_THREADS)
k_levels(const int64_t *ooff, const int32_t *ocol, const int32_t *deg, const uint32_t *t, int64_t n, int64_t m,
         const int32_t *orows, const int32_t *osrc, int measure, const int64_t *tp, const int64_t *tq, int k,
         uint8_t *lvl, unsigned long long *best, int32_t *lu, int32_t *lv, unsigned long long *lk, int32_t *rcnt,
         unsigned long long *ctr) {
    if (graph_bad(ctr)) return;                  // uniform over the grid
    const int64_t k0 = (int64_t)blockIdx.x * TILE;
    int64_t r0 = 0, r1 = 0;
    if (!osrc) tile_row_range(orows, ooff, n, m, r0, r1);
    int32_t eu[TILE_ITEMS], ev[TILE_ITEMS];
    uint8_t el[TILE_ITEMS];
    int c = 0;
#pragma unroll
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int64_t j = k0 + (int64_t)i * TILE_THREADS + threadIdx.x;
        el[i] = 0;
        eu[i] = ev[i] = 0;
        if (j >= m) continue;
        const int64_t u = edge_source(osrc, ooff, r0, r1, j);
        const int32_t v = ocol[j];
        const int64_t s = (int64_t)deg[u] + deg[v];
        const uint32_t tt = t[j];
        int lo = 0, hi = k;                      // first threshold the edge does not survive
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (keep_edge<WIDE>(measure, tt, s, tp[mid], tq[mid])) lo = mid + 1; else hi = mid;
        }
        lvl[j] = (uint8_t)lo;
        el[i] = (uint8_t)lo;
        eu[i] = (int32_t)u;
        ev[i] = v;
        if (lo) {
            const unsigned long long key = msf_key((uint8_t)lo, j);
            atomicMax(&best[u], key);
            atomicMax(&best[v], key);
            ++c;
        }
    }
    if (!COMPACT) return;
    int total;
    int at = block_excl_prefix(c, &total);
#pragma unroll
    for (int i = 0; i < TILE_ITEMS; ++i) {
        if (!el[i]) continue;
        const int64_t j = k0 + (int64_t)i * TILE_THREADS + threadIdx.x;
        lu[k0 + at] = eu[i];
        lv[k0 + at] = ev[i];
        lk[k0 + at] = msf_key(el[i], j);
        ++at;
    }
    if (threadIdx.x == 0) rcnt[blockIdx.x] = total;
}

// A later Boruvka round over the live-edge list: each entry (tree roots of
// both ends as of an earlier round, and the edge key) whose ends are still in
// different trees offers itself to both current roots and stays in its
// tile's region, stored by those roots; the others leave the list (trees
// only merge, so such an edge never joins two trees again).  Every entry of
// the region is read before the block's barrier and written after it.
__global__ void __launch_bounds__(TILE_THREADS)
k_msf_offer_list(int32_t *lu, int32_t *lv, unsigned long long *lk, int32_t *rcnt, int64_t ntiles, int32_t *parent,
                 unsigned long long *best, const unsigned long long *prev_changed) {
    if (*prev_changed == 0ull) return;           // forest complete; uniform over the grid
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {   // persistent over tile regions
        const int64_t base = tile * TILE;
        const int cnt = rcnt[tile];
        if (cnt == 0) continue;                  // uniform over the block
        int32_t ru[TILE_ITEMS], rv[TILE_ITEMS];
        unsigned long long key[TILE_ITEMS];
        unsigned live = 0;
        int c = 0;
#pragma unroll
        for (int i = 0; i < TILE_ITEMS; ++i) {
            const int idx = i * TILE_THREADS + (int)threadIdx.x;
            ru[i] = rv[i] = 0;
            key[i] = 0;
            if (idx >= cnt) continue;
            int32_t a, b;
            uf_find2(parent, lu[base + idx], lv[base + idx], a, b);
            if (a == b) continue;
            key[i] = lk[base + idx];
            ru[i] = a;
            rv[i] = b;
            atomicMax(&best[a], key[i]);
            atomicMax(&best[b], key[i]);
            live |= 1u << i;
            ++c;
        }
        int total;
        int at = block_excl_prefix(c, &total);
#pragma unroll
        for (int i = 0; i < TILE_ITEMS; ++i) {
            if (!((live >> i) & 1u)) continue;
            lu[base + at] = ru[i];
            lv[base + at] = rv[i];
            lk[base + at] = key[i];
            ++at;
        }
        if (threadIdx.x == 0) rcnt[tile] = total;
        __syncthreads();                         // the prefix scratch is reused by the next tile
    }
}

// Every edge with L >= 1 between two different trees offers itself to both roots.
__global__ void __launch_bounds__(TILE_THREADS)
k_msf_offer(const int64_t *ooff, const int32_t *ocol, const uint8_t *lvl, int64_t n, int64_t m, const int32_t *osrc,
            int32_t *parent, unsigned long long *best, const unsigned long long *prev_changed,
            unsigned long long *ctr) {
    if (*prev_changed == 0ull) return;           // forest complete; uniform over the grid
    const int64_t ntiles = ceil_div(m, (int64_t)TILE);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t k0 = tile * TILE;
        const int64_t klast = min(k0 + TILE, m) - 1;
        int64_t r0 = 0, r1 = 0;
        if (!osrc) {
            r0 = row_search(ooff, 0, n - 1, k0);
            r1 = row_search(ooff, r0, n - 1, klast);
        }
        for (int i = 0; i < TILE_ITEMS; ++i) {
            const int64_t j = k0 + (int64_t)i * TILE_THREADS + threadIdx.x;
            if (j >= m) break;
            const uint8_t L = lvl[j] & (uint8_t)~FOREST_BIT;
            if (L == 0) continue;
            const int32_t u = (int32_t)edge_source(osrc, ooff, r0, r1, j);
            int32_t ru, rv;
            uf_find2(parent, u, ocol[j], ru, rv);
            if (ru == rv) continue;
            const uint64_t key = msf_key(L, j);
            atomicMax(&best[ru], (unsigned long long)key);
            atomicMax(&best[rv], (unsigned long long)key);
        }
    }
}

// Each root hooks along its heaviest offer; a hook that joins two trees marks a
// forest edge and sets this round's changed flag (one store per block).
// Clears the offers for the next round.  Skipped when the previous round
// joined nothing (the forest is complete).
__global__ void k_msf_hook(const int64_t *ooff, const int32_t *ocol, const int32_t *osrc, uint8_t *lvl, int64_t n,
                           int32_t *parent, unsigned long long *best, const unsigned long long *prev_changed,
                           unsigned long long *changed, unsigned long long *ctr) {
    if (prev_changed && *prev_changed == 0ull) return;   // uniform over the grid
    int did = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = best[r];
        if (!key) continue;
        best[r] = 0ull;
        const int64_t j = msf_key_edge(key);
        const int32_t u = osrc ? osrc[j] : (int32_t)row_search(ooff, 0, n - 1, j);
        if (uf_link_merged(parent, u, ocol[j], ctr)) {
            lvl[j] |= FOREST_BIT;
            did = 1;
        }
    }
    if (__syncthreads_or(did) && threadIdx.x == 0) *changed = 1ull;
}

// Flags a forest that was still growing in the last round the sweep allows.
__global__ void k_msf_check(const unsigned long long *last_changed, unsigned long long *ctr) {
    if (*last_changed) flag_status(ctr, ST_TIMEOUT);
}

// Writes the sorted thresholds (p then q, 127 each) from the launch
// parameters, so a sweep needs no host-to-device copy.
struct SweepThresholds {
    int64_t v[2 * 127];
};
__global__ void k_store_thresholds(SweepThresholds th, int count, int64_t *dst) {
    for (int i = threadIdx.x; i < count; i += blockDim.x) dst[i] = th.v[i];
}

// Per-level forest-edge counts: a block histogram in shared memory, merged
// into bucket[0 .. k] with one atomic per non-empty level per block.
__global__ void k_forest_count(const uint8_t *lvl, int64_t m, int k, unsigned long long *bucket) {
    __shared__ unsigned int hist[128];
    for (int b = threadIdx.x; b <= k; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        if (lvl[j] & FOREST_BIT) atomicAdd(&hist[lvl[j] & (uint8_t)~FOREST_BIT], 1u);
    __syncthreads();
    for (int b = threadIdx.x; b <= k; b += blockDim.x)
        if (hist[b]) atomicAdd(&bucket[b], (unsigned long long)hist[b]);
}

// bucket[0 .. k] are the counts per level; this writes their exclusive scan
// to bucket[k+1 .. 2k+2] (k+2 offsets, the last one the total) and a copy used
// as fill cursors to bucket[2k+3 .. 3k+3] (one thread; k <= 127).
__global__ void k_forest_offsets(unsigned long long *bucket, int k, int64_t n, unsigned long long *ctr) {
    unsigned long long acc = 0;
    for (int b = 0; b <= k; ++b) {
        bucket[k + 1 + b] = acc;
        bucket[2 * k + 3 + b] = acc;
        acc += bucket[b];
    }
    bucket[2 * k + 2] = acc;
    if (acc > (unsigned long long)(n > 0 ? n - 1 : 0)) flag_status(ctr, ST_BADGRAPH);   // a forest has < n edges
}

// Writes the forest edges of one tile to their level buckets: the tile's
// per-level counts are reserved with one global atomic per level, then each
// edge takes a slot from a shared-memory cursor.
__global__ void __launch_bounds__(TILE_THREADS)
k_forest_scatter(const int64_t *ooff, const int32_t *ocol, const uint8_t *lvl, int64_t n, int64_t m,
                 const int32_t *orows, const int32_t *osrc, int k, unsigned long long *bucket, int32_t *fu,
                 int32_t *fv) {
    __shared__ unsigned int cnt[128];
    __shared__ unsigned long long base[128];
    for (int b = threadIdx.x; b <= k; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    const int64_t k0 = (int64_t)blockIdx.x * TILE;
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int64_t j = k0 + (int64_t)i * TILE_THREADS + threadIdx.x;
        if (j >= m) break;
        if (lvl[j] & FOREST_BIT) atomicAdd(&cnt[lvl[j] & (uint8_t)~FOREST_BIT], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b <= k; b += blockDim.x) {
        base[b] = cnt[b] ? atomicAdd(&bucket[2 * k + 3 + b], (unsigned long long)cnt[b]) : 0ull;
        cnt[b] = 0;
    }
    __syncthreads();
    int64_t r0 = 0, r1 = 0;
    if (!osrc) tile_row_range(orows, ooff, n, m, r0, r1);
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int64_t j = k0 + (int64_t)i * TILE_THREADS + threadIdx.x;
        if (j >= m) break;
        if (!(lvl[j] & FOREST_BIT)) continue;
        const int L = lvl[j] & (uint8_t)~FOREST_BIT;
        const unsigned long long at = base[L] + atomicAdd(&cnt[L], 1u);
        if (at >= (unsigned long long)n) continue;   // a forest has < n edges; the host checks the total
        fu[at] = (int32_t)edge_source(osrc, ooff, r0, r1, j);
        fv[at] = ocol[j];
    }
}

// Unions level L's bucket of forest edges; the bounds are read on the device.
__global__ void k_union_bucket(const int32_t *fu, const int32_t *fv, const unsigned long long *bucket, int k, int L,
                               int32_t *parent, unsigned long long *ctr) {
    const int64_t b0 = (int64_t)bucket[k + 1 + L], b1 = (int64_t)bucket[k + 1 + L + 1];
    for (int64_t e = b0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < b1; e += (int64_t)gridDim.x * blockDim.x)
        uf_link(parent, fu[e], fv[e], ctr);
}

// labels[x] = root of x (minus the first vertex of x's segment when a segment
// table is given); ncomp[s] counts the roots of segment s.  Each warp takes
// chunks of VCHUNK consecutive vertices: the first parent loads of the whole
// chunk are issued together, the segment is looked up once, and root counts
// are summed per warp and added with one atomic whenever the segment changes
// (per vertex only in the rare chunk that straddles a segment boundary).
__global__ void __launch_bounds__(256) k_snapshot(int32_t *parent, int64_t n, int32_t *labels,
                                                  const int64_t *seg_off, int nseg, unsigned long long *ncomp) {
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const unsigned lane = lane_id();
    int pend_s = -1;
    unsigned long long pend = 0;                 // roots counted for segment pend_s (lane 0)
    for (int64_t c0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * VCHUNK; c0 < n;
         c0 += nw * VCHUNK) {
        int32_t r[VCHUNK_V];
#pragma unroll
        for (int v = 0; v < VCHUNK_V; ++v) {
            const int64_t x = c0 + v * 32 + lane;
            r[v] = x < n ? __ldcg(&parent[x]) : -1;
        }
#pragma unroll
        for (int v = 0; v < VCHUNK_V; ++v) {
            const int64_t x = c0 + v * 32 + lane;
            if (x < n) r[v] = uf_find_from(parent, (int32_t)x, r[v]);
        }
        const int64_t cend = c0 + VCHUNK < n ? c0 + VCHUNK : n;
        int sg = 0;
        bool uniform = true;
        if (seg_off) {
            sg = warp_seg_of(seg_off, nseg, c0, c0);
            uniform = sg + 1 >= nseg || seg_off[sg + 1] >= cend;
        }
        if (uniform) {
            const int64_t base = seg_off ? seg_off[sg] : 0;
            int cnt = 0;
#pragma unroll
            for (int v = 0; v < VCHUNK_V; ++v) {
                const int64_t x = c0 + v * 32 + lane;
                if (x < n) {
                    labels[x] = (int32_t)(r[v] - base);
                    cnt += r[v] == x ? 1 : 0;
                }
            }
            cnt = warp_sum(cnt);
            if (sg != pend_s) {
                if (lane == 0 && pend) atomicAdd(&ncomp[pend_s], pend);
                pend_s = sg;
                pend = 0;
            }
            pend += (unsigned long long)cnt;
        } else {
#pragma unroll
            for (int v = 0; v < VCHUNK_V; ++v) {
                const int64_t x0 = c0 + v * 32, x = x0 + lane;
                const bool valid = x < n;
                const int s = warp_seg_of(seg_off, nseg, x0 < n ? x0 : n - 1, valid ? x : n - 1);
                if (valid) labels[x] = (int32_t)(r[v] - seg_off[s]);
                const unsigned same = __match_any_sync(0xffffffffu, valid ? s : -1);
                const unsigned rm = __ballot_sync(0xffffffffu, valid && r[v] == x) & same;
                if (valid && rm && lane == (unsigned)(__ffs(same) - 1))
                    atomicAdd(&ncomp[s], (unsigned long long)__popc(rm));
            }
        }
    }
    if (lane == 0 && pend) atomicAdd(&ncomp[pend_s], pend);
}

inline unsigned grid_for(int64_t work) {
    const int64_t g = ceil_div(work > 0 ? work : 1, 256);
    return (unsigned)(g < 65536 ? g : 65536);
}

}  // namespace

unsigned vertex_pass_grid(int64_t n) {
    static std::atomic<int> sms[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    int c = dev >= 0 && dev < 64 ? sms[dev].load(std::memory_order_relaxed) : 0;
    if (c <= 0) {
        if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0) c = 1;
        if (dev >= 0 && dev < 64) sms[dev].store(c, std::memory_order_relaxed);
    }
    const int64_t blocks = ceil_div(ceil_div(n > 0 ? n : 1, VCHUNK), 8);
    const int64_t cap = (int64_t)c * 16;
    return (unsigned)(blocks < cap ? blocks : cap);
}

cudaError_t launch_levels(const int64_t *ooff, const int32_t *ocol, const int32_t *deg, const uint32_t *t,
                          int64_t n, int64_t m, const int32_t *orows, const int32_t *osrc, int measure,
                          const int64_t *tp, const int64_t *tq, int k, bool wide,
                          uint8_t *lvl, unsigned long long *best, int32_t *lu, int32_t *lv, unsigned long long *lk,
                          int32_t *rcnt, unsigned long long *ctr, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)ceil_div(m, TILE);
    const bool compact = lu != nullptr;
#define TEC_LEVELS(W, C) \
    k_levels<W, C><<<grid, TILE_THREADS, 0, s>>>(ooff, ocol, deg, t, n, m, orows, osrc, measure, tp, tq, k, lvl, \
                                                 best, lu, lv, lk, rcnt, ctr)
    if (wide) {
        if (compact) TEC_LEVELS(true, true); else TEC_LEVELS(true, false);
    } else {
        if (compact) TEC_LEVELS(false, true); else TEC_LEVELS(false, false);
    }
#undef TEC_LEVELS
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_msf_offer(const int64_t *ooff, const int32_t *ocol, uint8_t *lvl, int64_t n, int64_t m,
                             const int32_t *osrc, int32_t *parent, unsigned long long *best, int32_t *lu, int32_t *lv,
                             unsigned long long *lk, int32_t *rcnt, const unsigned long long *prev_changed,
                             unsigned long long *ctr, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    // persistent grids: a round after the forest is complete costs one tiny launch
    const int64_t ntiles = ceil_div(m, (int64_t)TILE);
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)vertex_pass_grid(int64_t(1) << 40) / 2);
    if (lu)
        k_msf_offer_list<<<grid, TILE_THREADS, 0, s>>>(lu, lv, lk, rcnt, ntiles, parent, best, prev_changed);
    else
        k_msf_offer<<<grid, TILE_THREADS, 0, s>>>(ooff, ocol, lvl, n, m, osrc, parent, best, prev_changed, ctr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_msf_hook(const int64_t *ooff, const int32_t *ocol, const int32_t *osrc, uint8_t *lvl, int64_t n,
                            int32_t *parent, unsigned long long *best, const unsigned long long *prev_changed,
                            unsigned long long *changed, unsigned long long *ctr, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_msf_hook<<<vertex_pass_grid(n), 256, 0, s>>>(ooff, ocol, osrc, lvl, n, parent, best, prev_changed, changed, ctr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_msf_check(const unsigned long long *last_changed, unsigned long long *ctr, cudaStream_t s) {
    k_msf_check<<<1, 1, 0, s>>>(last_changed, ctr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_store_thresholds(const int64_t *sorted_pq, int count, int64_t *dst, cudaStream_t s) {
    SweepThresholds th{};
    for (int i = 0; i < count && i < 2 * 127; ++i) th.v[i] = sorted_pq[i];
    k_store_thresholds<<<1, 256, 0, s>>>(th, count, dst);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_forest_buckets(const int64_t *ooff, const int32_t *ocol, const uint8_t *lvl, int64_t n, int64_t m,
                                  const int32_t *orows, const int32_t *osrc, int k, unsigned long long *bucket, int32_t *fu, int32_t *fv, unsigned long long *ctr,
                                  cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bucket, 0, (size_t)(k + 1) * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int64_t cblocks = ceil_div(m, 4096);
    if (m > 0) k_forest_count<<<(unsigned)(cblocks < 152 * 16 ? cblocks : 152 * 16), 256, 0, s>>>(lvl, m, k, bucket);
    k_forest_offsets<<<1, 1, 0, s>>>(bucket, k, n, ctr);
    if (m > 0)
        k_forest_scatter<<<(unsigned)ceil_div(m, TILE), TILE_THREADS, 0, s>>>(ooff, ocol, lvl, n, m, orows, osrc, k, bucket,
                                                                                    fu, fv);
    count_launches(m > 0 ? 3 : 1);
    return cudaGetLastError();
}

cudaError_t launch_snapshot(int32_t *parent, int64_t n, int32_t *labels, const int64_t *seg_off, int nseg,
                            unsigned long long *ncomp, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_snapshot<<<vertex_pass_grid(n), 256, 0, s>>>(parent, n, labels, seg_off, nseg, ncomp);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_sweep_level(const int32_t *fu, const int32_t *fv, const unsigned long long *bucket, int k, int L,
                               int64_t n, int32_t *parent, int32_t *labels, const int64_t *seg_off, int nseg,
                               unsigned long long *ncomp, unsigned long long *ctr, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_union_bucket<<<vertex_pass_grid(n), 256, 0, s>>>(fu, fv, bucket, k, L, parent, ctr);
    k_snapshot<<<vertex_pass_grid(n), 256, 0, s>>>(parent, n, labels, seg_off, nseg, ncomp);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace tec
