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
//    F_i = {e in F : L(e) >= i} have the same components for every i.
// 2. Offline sweep: forest edges are bucketed by level; starting from
//    singletons, level i = k .. 1 unions bucket i and then snapshots every
//    vertex's root (the component minimum) as the labels at theta_i.
// A batch of graphs is one disjoint union: with a segment table the snapshot
// writes labels relative to each graph's first vertex and counts components
// per graph.
#include "tec_internal.cuh"
#include "uf.cuh"

namespace tec {
namespace {

constexpr uint8_t FOREST_BIT = 0x80;

template <bool WIDE>
__global__ void __launch_bounds__(TILE_THREADS)
k_levels(const int64_t *ooff, const int32_t *ocol, const int32_t *deg, const uint32_t *t, int64_t n, int64_t m,
         int measure, const int64_t *tp, const int64_t *tq, int k, uint8_t *lvl, unsigned long long *ctr) {
    if (graph_bad(ctr)) return;
    const int64_t k0 = (int64_t)blockIdx.x * TILE;
    const int64_t klast = min(k0 + TILE, m) - 1;
    const int64_t r0 = row_search(ooff, 0, n - 1, k0);
    const int64_t r1 = row_search(ooff, r0, n - 1, klast);
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int64_t j = k0 + (int64_t)i * TILE_THREADS + threadIdx.x;
        if (j >= m) break;
        const int64_t u = row_search(ooff, r0, r1, j);
        const int64_t s = (int64_t)deg[u] + deg[ocol[j]];
        const uint32_t tt = t[j];
        int lo = 0, hi = k;                      // first threshold the edge does not survive
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (keep_edge<WIDE>(measure, tt, s, tp[mid], tq[mid])) lo = mid + 1; else hi = mid;
        }
        lvl[j] = (uint8_t)lo;
    }
}

__device__ __forceinline__ uint64_t msf_key(uint8_t L, int64_t j) {
    return ((uint64_t)L << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)j);
}

// Every edge with L >= 1 between two different trees offers itself to both roots.
__global__ void __launch_bounds__(TILE_THREADS)
k_msf_offer(const int64_t *ooff, const int32_t *ocol, const uint8_t *lvl, int64_t n, int64_t m,
            int32_t *parent, unsigned long long *best, unsigned long long *ctr) {
    const int64_t k0 = (int64_t)blockIdx.x * TILE;
    const int64_t klast = min(k0 + TILE, m) - 1;
    const int64_t r0 = row_search(ooff, 0, n - 1, k0);
    const int64_t r1 = row_search(ooff, r0, n - 1, klast);
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int64_t j = k0 + (int64_t)i * TILE_THREADS + threadIdx.x;
        if (j >= m) break;
        const uint8_t L = lvl[j] & (uint8_t)~FOREST_BIT;
        if (L == 0) continue;
        const int32_t u = (int32_t)row_search(ooff, r0, r1, j);
        const int32_t ru = uf_find(parent, u), rv = uf_find(parent, ocol[j]);
        if (ru == rv) continue;
        const uint64_t key = msf_key(L, j);
        atomicMax(&best[ru], (unsigned long long)key);
        atomicMax(&best[rv], (unsigned long long)key);
    }
}

// Each root hooks along its heaviest offer; a hook that joins two trees marks a
// forest edge.  Clears the offers for the next round.
__global__ void k_msf_hook(const int64_t *ooff, const int32_t *ocol, uint8_t *lvl, int64_t n, int32_t *parent,
                           unsigned long long *best, unsigned long long *ctr) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = best[r];
        if (!key) continue;
        best[r] = 0ull;
        const int64_t j = (int64_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull));
        const int32_t u = (int32_t)row_search(ooff, 0, n - 1, j);
        if (uf_link_merged(parent, u, ocol[j], ctr)) {
            lvl[j] |= FOREST_BIT;
            atomicAdd(&ctr[C_CHANGED], 1ull);
        }
    }
}

__global__ void k_forest_count(const uint8_t *lvl, int64_t m, unsigned long long *bucket) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        if (lvl[j] & FOREST_BIT) atomicAdd(&bucket[lvl[j] & (uint8_t)~FOREST_BIT], 1ull);
}

// bucket[0 .. k] are the counts per level; this writes their exclusive scan
// to bucket[k+1 .. 2k+2] (k+2 offsets, the last one the total) and a copy used
// as fill cursors to bucket[2k+3 .. 3k+3] (one thread; k <= 127).
__global__ void k_forest_offsets(unsigned long long *bucket, int k) {
    unsigned long long acc = 0;
    for (int b = 0; b <= k; ++b) {
        bucket[k + 1 + b] = acc;
        bucket[2 * k + 3 + b] = acc;
        acc += bucket[b];
    }
    bucket[2 * k + 2] = acc;
}

__global__ void __launch_bounds__(TILE_THREADS)
k_forest_scatter(const int64_t *ooff, const int32_t *ocol, const uint8_t *lvl, int64_t n, int64_t m, int k,
                 unsigned long long *bucket, int32_t *fu, int32_t *fv) {
    const int64_t k0 = (int64_t)blockIdx.x * TILE;
    const int64_t klast = min(k0 + TILE, m) - 1;
    const int64_t r0 = row_search(ooff, 0, n - 1, k0);
    const int64_t r1 = row_search(ooff, r0, n - 1, klast);
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int64_t j = k0 + (int64_t)i * TILE_THREADS + threadIdx.x;
        if (j >= m) break;
        if (!(lvl[j] & FOREST_BIT)) continue;
        const int L = lvl[j] & (uint8_t)~FOREST_BIT;
        const unsigned long long at = atomicAdd(&bucket[2 * k + 3 + L], 1ull);
        fu[at] = (int32_t)row_search(ooff, r0, r1, j);
        fv[at] = ocol[j];
    }
}

__global__ void k_union_bucket(const int32_t *fu, const int32_t *fv, const unsigned long long *bucket, int k, int L,
                               int32_t *parent, unsigned long long *ctr) {
    const int64_t b0 = (int64_t)bucket[k + 1 + L], b1 = (int64_t)bucket[k + 1 + L + 1];
    for (int64_t e = b0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < b1; e += (int64_t)gridDim.x * blockDim.x)
        uf_link(parent, fu[e], fv[e], ctr);
}

// labels[x] = root of x (minus the first vertex of x's segment when a segment
// table is given); ncomp[s] counts the roots of segment s.
__global__ void k_snapshot(int32_t *parent, int64_t n, int32_t *labels, const int64_t *seg_off, int nseg,
                           unsigned long long *ncomp) {
    int roots = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = uf_find(parent, (int32_t)x);
        int64_t base = 0;
        if (seg_off) {
            int lo = 0, hi = nseg - 1;           // last segment starting at or before x
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (seg_off[mid] <= x) lo = mid; else hi = mid - 1;
            }
            base = seg_off[lo];
            if (r == x) atomicAdd(&ncomp[lo], 1ull);
        } else {
            roots += (r == x) ? 1 : 0;
        }
        labels[x] = (int32_t)(r - base);
    }
    if (!seg_off) {
        roots = warp_sum(roots);
        if (lane_id() == 0 && roots) atomicAdd(&ncomp[0], (unsigned long long)roots);
    }
}

inline unsigned grid_for(int64_t work) {
    const int64_t g = ceil_div(work > 0 ? work : 1, 256);
    return (unsigned)(g < 65536 ? g : 65536);
}

}  // namespace

cudaError_t launch_levels(const int64_t *ooff, const int32_t *ocol, const int32_t *deg, const uint32_t *t,
                          int64_t n, int64_t m, int measure, const int64_t *tp, const int64_t *tq, int k, bool wide,
                          uint8_t *lvl, unsigned long long *ctr, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)ceil_div(m, TILE);
    if (wide) k_levels<true><<<grid, TILE_THREADS, 0, s>>>(ooff, ocol, deg, t, n, m, measure, tp, tq, k, lvl, ctr);
    else k_levels<false><<<grid, TILE_THREADS, 0, s>>>(ooff, ocol, deg, t, n, m, measure, tp, tq, k, lvl, ctr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_msf_round(const int64_t *ooff, const int32_t *ocol, uint8_t *lvl, int64_t n, int64_t m,
                             int32_t *parent, unsigned long long *best, unsigned long long *ctr, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    k_msf_offer<<<(unsigned)ceil_div(m, TILE), TILE_THREADS, 0, s>>>(ooff, ocol, lvl, n, m, parent, best, ctr);
    k_msf_hook<<<grid_for(n), 256, 0, s>>>(ooff, ocol, lvl, n, parent, best, ctr);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_forest_buckets(const int64_t *ooff, const int32_t *ocol, const uint8_t *lvl, int64_t n, int64_t m,
                                  int k, unsigned long long *bucket, int32_t *fu, int32_t *fv, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bucket, 0, (size_t)(k + 1) * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (m > 0) k_forest_count<<<grid_for(m), 256, 0, s>>>(lvl, m, bucket);
    k_forest_offsets<<<1, 1, 0, s>>>(bucket, k);
    if (m > 0)
        k_forest_scatter<<<(unsigned)ceil_div(m, TILE), TILE_THREADS, 0, s>>>(ooff, ocol, lvl, n, m, k, bucket, fu, fv);
    count_launches(m > 0 ? 3 : 1);
    return cudaGetLastError();
}

cudaError_t launch_snapshot(int32_t *parent, int64_t n, int32_t *labels, const int64_t *seg_off, int nseg,
                            unsigned long long *ncomp, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_snapshot<<<grid_for(n), 256, 0, s>>>(parent, n, labels, seg_off, nseg, ncomp);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_sweep_level(const int32_t *fu, const int32_t *fv, const unsigned long long *bucket, int k, int L,
                               int64_t n, int32_t *parent, int32_t *labels, const int64_t *seg_off, int nseg,
                               unsigned long long *ncomp, unsigned long long *ctr, cudaStream_t s) {
    k_union_bucket<<<grid_for(n), 256, 0, s>>>(fu, fv, bucket, k, L, parent, ctr);
    if (n > 0) k_snapshot<<<grid_for(n), 256, 0, s>>>(parent, n, labels, seg_off, nseg, ncomp);
    count_launches(n > 0 ? 2 : 1);
    return cudaGetLastError();
}

}  // namespace tec
