// Per-graph features for the threshold picker, the adjusted Rand index, and
// precision / recall / F1 (Sec. IV-A) of labelings against planted blocks.
//
// Features (tec_features): the 64-bin histogram of Tectonic weights on the
// grid i/128 -- bin = min(63, floor(128 t / (deg u + deg v))), the level an
// edge reaches in a sweep of thresholds i/128 -- divided by m, then
// ln(2m / n) and ln(m); one row of 66 floats per graph of a batch.
//
// ARI (tec_ari, Hubert & Arabie 1985): for component labels c and reference
// blocks b of one graph with n vertices,
//   S_ab = sum over cells (c, b) of C(n_cb, 2), S_a = sum over components of
//   C(size, 2), S_b = sum over blocks of C(size, 2), T = C(n, 2),
//   ARI = (2 T S_ab - 2 S_a S_b) / (T (S_a + S_b) - 2 S_a S_b),
// with ARI = 1 when the denominator is 0 (both partitions all singletons or
// both one cluster) or n < 2.  All sums are exact 64-bit integers and the
// ratio is formed from exact 128-bit numerator and denominator.
//
// Per level, two passes over the vertices.  Sizes: each component's size is
// a counter at its root.  Cells: each (component root, block) pair of a
// component with at least two vertices is a counter in an open-addressing
// hash table (singleton components add nothing to either sum).  The sums
// are built incrementally: adding c to a counter that held o raises
// C(count, 2) by o c + C(c, 2), so no pass over the counters is needed.
// Lanes of a warp with the same root or cell add once for all of them.
// Cell counters and keys carry the level's tag in their top 24 bits; a word
// with an older tag reads as empty, so the table is zeroed only when the tag
// wraps, not per level.  Sizes use two plain counter arrays in turn: each
// level's first pass zeroes the array the next level will use.
#include "bulk.cuh"
#include "tec_internal.cuh"

namespace tec {
namespace {

constexpr int NBINS = 64;

__device__ __forceinline__ int seg_of(const int64_t *seg_off, int nseg, int64_t x) {
    int lo = 0, hi = nseg - 1;                   // last segment starting at or before x
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg_off[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// floor(128 t / s) clamped to the last bin: an approximate float quotient
// (__fdividef: a few ulp of a value below 64, so off by at most one)
// corrected by exact integer comparisons.
__device__ __forceinline__ int weight_bin(uint32_t tt, int64_t s) {
    const int64_t num = 128 * (int64_t)tt;
    int64_t b = (int64_t)__fdividef((float)num, (float)s);
    if (b * s > num) --b;
    else if ((b + 1) * s <= num) ++b;
    return b > NBINS - 1 ? NBINS - 1 : (int)b;
}

__global__ void __launch_bounds__(TILE_THREADS)
k_feat_hist(const int64_t *ooff, const int32_t *ocol, const int32_t *deg, const uint32_t *t, int64_t n, int64_t m,
            const int32_t *orows, const int32_t *osrc, const int64_t *seg_off, int nseg, unsigned int *hist,
            unsigned long long *ctr) {
    __shared__ unsigned int s_h[NBINS];
    if (graph_bad(ctr)) return;
    const int64_t k0 = (int64_t)blockIdx.x * TILE;
    int64_t r0, r1;
    tile_row_range(orows, ooff, n, m, r0, r1);
    const int s0 = seg_off ? seg_of(seg_off, nseg, r0) : 0;
    const int s1 = seg_off ? seg_of(seg_off, nseg, r1) : 0;
    const bool one = s0 == s1;                   // the common case: aggregate in shared memory
    if (threadIdx.x < NBINS) s_h[threadIdx.x] = 0u;
    __syncthreads();
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int64_t j = k0 + (int64_t)i * TILE_THREADS + threadIdx.x;
        const bool valid = j < m;
        int64_t b = -1, u = 0;
        if (valid) {
            u = edge_source(osrc, ooff, r0, r1, j);
            b = weight_bin(t[j], (int64_t)deg[u] + deg[ocol[j]]);
        }
        // bin 0 (edges in no triangle, most of a sparse graph) is counted with
        // one shared add per warp: lane-by-lane adds to one word serialise
        const unsigned zero = __ballot_sync(0xffffffffu, valid && b == 0);
        if (one) {
            if (lane_id() == 0 && zero) atomicAdd(&s_h[0], (unsigned)__popc(zero));
            if (valid && b > 0) atomicAdd(&s_h[b], 1u);
        } else if (valid) {
            atomicAdd(&hist[(int64_t)seg_of(seg_off, nseg, u) * NBINS + b], 1u);
        }
    }
    __syncthreads();
    if (one && threadIdx.x < NBINS && s_h[threadIdx.x]) atomicAdd(&hist[(int64_t)s0 * NBINS + threadIdx.x], s_h[threadIdx.x]);
}

// k_feat_hist as a persistent grid of independent warps, each with its own
// shared-memory histogram and a contiguous share of 256-edge chunks: a warp
// adds into its histogram while its chunks stay in one graph and flushes it
// (64 global adds) when the graph changes, so there is no block barrier and
// no contention between warps.  Needs the per-edge source table.  Chosen by
// the autotuner (FEAT_PERSISTENT).
constexpr int FEAT_PERSISTENT = 1;
constexpr int FH_CHUNK = 256;

__device__ __forceinline__ int seg_in(const int64_t *seg_off, int lo, int hi, int64_t x) {
    while (lo < hi) {                            // last segment in [lo, hi] starting at or before x
        const int mid = (lo + hi + 1) >> 1;
        if (seg_off[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(TILE_THREADS)
k_feat_hist_warps(const int32_t *__restrict__ ocol, const int32_t *__restrict__ deg, const uint32_t *__restrict__ t,
                  int64_t m, const int32_t *__restrict__ osrc, const int64_t *__restrict__ seg_off, int nseg,
                  unsigned int *hist, unsigned long long *ctr) {
    __shared__ unsigned int s_h[TILE_THREADS / 32][NBINS];
    if (graph_bad(ctr)) return;
    const unsigned lane = lane_id();
    unsigned int *h = s_h[threadIdx.x >> 5];
    h[lane] = 0u;
    h[lane + 32] = 0u;
    __syncwarp();
    const int64_t nchunks = ceil_div(m, FH_CHUNK);
    const int64_t warps = (int64_t)gridDim.x * (TILE_THREADS / 32);
    const int64_t per = ceil_div(nchunks, warps);
    const int64_t c0 = ((int64_t)blockIdx.x * (TILE_THREADS / 32) + (threadIdx.x >> 5)) * per;
    const int64_t c1 = c0 + per < nchunks ? c0 + per : nchunks;
    int cur = -1;                                // the graph whose counts h holds
    auto flush = [&]() {
        __syncwarp();
        if (cur >= 0) {
            for (int b = (int)lane; b < NBINS; b += 32)
                if (h[b]) {
                    atomicAdd(&hist[(int64_t)cur * NBINS + b], h[b]);
                    h[b] = 0u;
                }
        }
        __syncwarp();
    };
    for (int64_t c = c0; c < c1; ++c) {
        const int64_t j0 = c * FH_CHUNK;
        const int64_t jl = (j0 + FH_CHUNK < m ? j0 + FH_CHUNK : m) - 1;
        int s0 = 0, s1 = 0;
        if (seg_off) {                           // lane 0: graph of the first edge, lane 1: of the last
            const int mine = lane < 2 ? seg_in(seg_off, 0, nseg - 1, osrc[lane == 0 ? j0 : jl]) : 0;
            s0 = __shfl_sync(0xffffffffu, mine, 0);
            s1 = __shfl_sync(0xffffffffu, mine, 1);
        }
        const bool one = s0 == s1;
        if (one && s0 != cur) {
            flush();
            cur = s0;
        }
        for (int i = 0; i < FH_CHUNK / 32; ++i) {
            const int64_t j = j0 + i * 32 + lane;
            const bool valid = j < m;
            int b = -1;
            int32_t u = 0;
            if (valid) {
                u = osrc[j];
                b = weight_bin(t[j], (int64_t)deg[u] + deg[ocol[j]]);
            }
            // bin 0 (edges in no triangle) is added once per warp
            const unsigned zero = __ballot_sync(0xffffffffu, valid && b == 0);
            if (one) {
                if (lane == 0 && zero) atomicAdd(&h[0], (unsigned)__popc(zero));
                if (valid && b > 0) atomicAdd(&h[b], 1u);
            } else if (valid) {
                atomicAdd(&hist[(int64_t)seg_in(seg_off, s0, s1, u) * NBINS + b], 1u);
            }
        }
    }
    flush();
}

// One warp per graph: 64 normalised bins, ln(2m/n), ln(m).
__global__ void k_feat_final(const unsigned int *hist, const int64_t *seg_off, int nseg, int64_t n_all,
                             float *feat) {
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (w >= nseg) return;
    const int lane = (int)lane_id();
    const unsigned int h0 = hist[(int64_t)w * NBINS + lane], h1 = hist[(int64_t)w * NBINS + 32 + lane];
    unsigned long long mm = (unsigned long long)h0 + h1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mm += __shfl_xor_sync(0xffffffffu, mm, o);
    const int64_t nv = seg_off ? seg_off[w + 1] - seg_off[w] : n_all;
    float *f = feat + (int64_t)w * (NBINS + 2);
    const float mf = (float)mm;
    f[lane] = mm ? (float)h0 / mf : 0.f;
    f[32 + lane] = mm ? (float)h1 / mf : 0.f;
    if (lane == 0) {
        f[NBINS] = (mm && nv) ? logf(2.f * mf / (float)nv) : 0.f;
        f[NBINS + 1] = mm ? logf(mf) : 0.f;
    }
}

// ---------------------------------------------------------------- ARI

constexpr int TAG_SHIFT = 40;
constexpr unsigned long long CNT_MASK = (1ull << TAG_SHIFT) - 1ull;
constexpr unsigned long long TAG_LIMIT = (1ull << (64 - TAG_SHIFT)) - 1ull;
constexpr int BS_CHUNK = 8192;                   // vertices per block in k_block_sizes

__device__ __forceinline__ uint64_t hkey(uint64_t key, int bits) {
    return (key * 0x9E3779B97F4A7C15ull) >> (64 - bits);
}

__device__ __forceinline__ unsigned long long c2(unsigned long long x) { return x * (x - (x > 0)) / 2; }

// Adds c to a level-tagged counter and returns the count it held at this
// level (0 if the word carried an older tag).  Within a level a word only
// goes from an older tag to the current one (by the compare-and-swap here)
// and then grows, so a failed swap always leaves a current word and the
// second iteration adds.
__device__ __forceinline__ unsigned long long tagged_add(unsigned long long *w, unsigned long long tag,
                                                         unsigned long long c) {
    unsigned long long cur = __ldcg(w);
    for (int it = 0; it < 2; ++it) {
        if ((cur >> TAG_SHIFT) == tag) break;
        const unsigned long long old = atomicCAS(w, cur, (tag << TAG_SHIFT) | c);
        if (old == cur) return 0ull;
        cur = old;
    }
    return atomicAdd(w, c) & CNT_MASK;
}

// Slot of cell key ck (< 2^40) at this level: linear probing from its hash,
// claiming the first slot with an older tag.  Slots of this level are never
// re-claimed, so a key is found wherever its first claim put it.  -1 if the
// table is full (it holds 2n slots and at most n cells per level).
__device__ __forceinline__ int64_t cell_slot(unsigned long long *keys, int bits, unsigned long long tag,
                                             unsigned long long ck) {
    const uint64_t mask = (1ull << bits) - 1ull;
    const unsigned long long want = (tag << TAG_SHIFT) | ck;
    uint64_t h = hkey(ck, bits);
    for (uint64_t probe = 0; probe <= mask; ++probe, h = (h + 1) & mask) {
        unsigned long long cur = __ldcg(&keys[h]);
        for (int it = 0; it < 2; ++it) {         // a failed claim leaves a key of this level
            if (cur == want) return (int64_t)h;
            if ((cur >> TAG_SHIFT) == tag) break;
            const unsigned long long old = atomicCAS(&keys[h], cur, want);
            if (old == cur) return (int64_t)h;
            cur = old;
        }
        if (cur == want) return (int64_t)h;
    }
    return -1;
}

// Adds the per-lane pair-count increments of a warp to sums[2 s + which]:
// one atomic per warp when every valid lane is in the same segment.
__device__ __forceinline__ void add_pairs(unsigned long long *sums, int which, int s, bool valid,
                                          unsigned long long d) {
    const int s0 = __shfl_sync(0xffffffffu, s, 0);
    if (__all_sync(0xffffffffu, !valid || s == s0)) {
        d = warp_sum64(d);
        if (lane_id() == 0 && d) atomicAdd(&sums[2 * s0 + which], d);
    } else if (d) {
        atomicAdd(&sums[2 * s + which], d);
    }
}

// Block sizes per graph: each block counts a contiguous chunk of vertices in
// shared memory when the chunk lies in one graph.
__global__ void k_block_sizes(const int32_t *truth, int64_t n, const int64_t *seg_off, int nseg, unsigned int *bsz,
                              unsigned long long *ctr) {
    __shared__ unsigned int s_h[NBINS];
    const int64_t c0 = (int64_t)blockIdx.x * BS_CHUNK;
    const int64_t c1 = min(c0 + BS_CHUNK, n);
    const int s0 = seg_off ? seg_of(seg_off, nseg, c0) : 0;
    const bool one = !seg_off || seg_of(seg_off, nseg, c1 - 1) == s0;
    if (threadIdx.x < NBINS) s_h[threadIdx.x] = 0u;
    __syncthreads();
    for (int64_t x = c0 + threadIdx.x; x < c1; x += blockDim.x) {
        const int b = truth[x];
        if (b < 0 || b >= NBINS) { flag_status(ctr, ST_BADGRAPH); continue; }
        if (one) atomicAdd(&s_h[b], 1u);
        else atomicAdd(&bsz[(int64_t)seg_of(seg_off, nseg, x) * NBINS + b], 1u);
    }
    __syncthreads();
    if (one && threadIdx.x < NBINS && s_h[threadIdx.x])
        atomicAdd(&bsz[(int64_t)s0 * NBINS + threadIdx.x], s_h[threadIdx.x]);
}

// Pass 1 of a level: component sizes into cur (zeroed), S_a into
// sums[2 s + 1]; zeroes prev (the other buffer) for the next level.  Chunks
// of VCHUNK vertices per warp, as in the snapshot; lanes grouped by
// key_group; each warp adds its pair increments with one atomic per segment
// change.
__global__ void __launch_bounds__(256) k_ari_sizes(const int32_t *labels, int64_t n, const int64_t *seg_off, int nseg,
                                                   unsigned int *cur, unsigned int *prev, unsigned long long *sums,
                                                   unsigned long long *ctr) {
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const unsigned lane = lane_id();
    int pend_s = -1;
    unsigned long long pend = 0;
    for (int64_t c0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * VCHUNK; c0 < n;
         c0 += nw * VCHUNK) {
        int32_t lab[VCHUNK_V];
#pragma unroll
        for (int v = 0; v < VCHUNK_V; ++v) {
            const int64_t x = c0 + v * 32 + lane;
            lab[v] = x < n ? labels[x] : 0;
            if (x < n) prev[x] = 0u;
        }
        const int64_t cend = c0 + VCHUNK < n ? c0 + VCHUNK : n;
        int sg = seg_off ? warp_seg_of(seg_off, nseg, c0, c0) : 0;
        const bool uniform = !seg_off || sg + 1 >= nseg || seg_off[sg + 1] >= cend;
        unsigned long long d = 0;
#pragma unroll
        for (int v = 0; v < VCHUNK_V; ++v) {
            const int64_t x0 = c0 + v * 32, x = x0 + lane;
            bool valid = x < n;
            int s = sg;
            if (!uniform) s = warp_seg_of(seg_off, nseg, x0 < n ? x0 : n - 1, valid ? x : n - 1);
            int32_t root = -1;
            if (valid) {
                const int64_t r = (seg_off ? seg_off[s] : 0) + lab[v];
                if (r < 0 || r >= n) {
                    flag_status(ctr, ST_BADGRAPH);
                    valid = false;
                } else {
                    root = (int32_t)r;
                }
            }
            const unsigned same = key_group(valid, root);
            unsigned long long dv = 0;
            if (valid && lane == (unsigned)(__ffs(same) - 1)) {
                const unsigned long long c = (unsigned long long)__popc(same);
                dv = (unsigned long long)atomicAdd(&cur[root], (unsigned int)c) * c + c2(c);
            }
            if (uniform) d += dv;
            else add_pairs(sums, 1, s, valid, dv);
        }
        if (uniform) {
            d = warp_sum64(d);
            if (sg != pend_s) {
                if (lane == 0 && pend) atomicAdd(&sums[2 * pend_s + 1], pend);
                pend_s = sg;
                pend = 0;
            }
            pend += d;
        }
    }
    if (lane == 0 && pend) atomicAdd(&sums[2 * pend_s + 1], pend);
}

// Pass 2 of a level: (root, block) cells of components with two or more
// vertices, and S_ab into sums[2 s].
__global__ void __launch_bounds__(256) k_ari_cells(const int32_t *labels, const int32_t *truth, int64_t n,
                                                   const int64_t *seg_off, int nseg, unsigned long long tag,
                                                   const unsigned int *size, unsigned long long *keys,
                                                   unsigned long long *cnt, int bits, unsigned long long *sums,
                                                   unsigned long long *ctr) {
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const unsigned lane = lane_id();
    int pend_s = -1;
    unsigned long long pend = 0;
    for (int64_t c0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * VCHUNK; c0 < n;
         c0 += nw * VCHUNK) {
        const int64_t cend = c0 + VCHUNK < n ? c0 + VCHUNK : n;
        int sg = seg_off ? warp_seg_of(seg_off, nseg, c0, c0) : 0;
        const bool uniform = !seg_off || sg + 1 >= nseg || seg_off[sg + 1] >= cend;
        int64_t root[VCHUNK_V];
        int blk[VCHUNK_V];
#pragma unroll
        for (int v = 0; v < VCHUNK_V; ++v) {
            const int64_t x = c0 + v * 32 + lane;
            root[v] = -1;
            blk[v] = -1;
            if (x < n) {
                const int s = uniform ? sg : warp_seg_of(seg_off, nseg, c0, x);
                root[v] = (seg_off ? seg_off[s] : 0) + labels[x];
                blk[v] = truth[x];
            }
        }
        unsigned int sz[VCHUNK_V];
#pragma unroll
        for (int v = 0; v < VCHUNK_V; ++v) sz[v] = (root[v] >= 0 && root[v] < n) ? size[root[v]] : 0u;
        unsigned long long d = 0;
#pragma unroll
        for (int v = 0; v < VCHUNK_V; ++v) {
            const int64_t x0 = c0 + v * 32, x = x0 + lane;
            // invalid roots and blocks are reported by the other passes
            const bool valid = x < n && sz[v] >= 2 && blk[v] >= 0 && blk[v] < NBINS;
            const unsigned long long key =
                valid ? ((unsigned long long)root[v] << 6) | (unsigned long long)blk[v] : ~0ull;
            const unsigned same = key_group(valid, key);
            unsigned long long dv = 0;
            if (valid && lane == (unsigned)(__ffs(same) - 1)) {
                const int64_t slot = cell_slot(keys, bits, tag, key);
                if (slot < 0) {
                    flag_status(ctr, ST_BADGRAPH);
                } else {
                    const unsigned long long c = (unsigned long long)__popc(same);
                    dv = tagged_add(&cnt[slot], tag, c) * c + c2(c);
                }
            }
            if (uniform) {
                d += dv;
            } else {
                const int s = warp_seg_of(seg_off, nseg, x0 < n ? x0 : n - 1, x < n ? x : n - 1);
                add_pairs(sums, 0, s, x < n, dv);
            }
        }
        if (uniform) {
            d = warp_sum64(d);
            if (sg != pend_s) {
                if (lane == 0 && pend) atomicAdd(&sums[2 * pend_s], pend);
                pend_s = sg;
                pend = 0;
            }
            pend += d;
        }
    }
    if (lane == 0 && pend) atomicAdd(&sums[2 * pend_s], pend);
}

// ---------------------------------------------------------------- P/R/F1
//
// Sec. IV-A: each found community S (a component) is matched to the reference
// block C of largest Jaccard |C n S| / |C u S| (the lowest block id on ties),
// p = |C n S| / |S|, r = |C n S| / |C|, and precision, recall and F1 are the
// size-weighted means of p, r and 2pr/(p + r).  Per level: component sizes
// (the ARI sizes pass), every (root, block) cell counted (singletons
// included), each vertex raising its root's best Jaccard (the double of the
// same division the definition writes, so ties are exact), the lowest block
// reaching it, and one term per community.

// Slot of cell key ck at this level, or -1 (no claim: a cell is found at or
// before the first slot of an older level along its probe sequence).
__device__ __forceinline__ int64_t cell_find(const unsigned long long *keys, int bits, unsigned long long tag,
                                             unsigned long long ck) {
    const uint64_t mask = (1ull << bits) - 1ull;
    const unsigned long long want = (tag << TAG_SHIFT) | ck;
    uint64_t h = hkey(ck, bits);
    for (uint64_t probe = 0; probe <= mask; ++probe, h = (h + 1) & mask) {
        const unsigned long long cur = __ldcg(&keys[h]);
        if (cur == want) return (int64_t)h;
        if ((cur >> TAG_SHIFT) != tag) return -1;
    }
    return -1;
}

struct PrfVertex {
    bool valid;
    int s;
    int32_t root;
    int b;
};

// Root and block of vertex x (x0 the warp's first vertex), for the P/R/F1 passes.
__device__ __forceinline__ PrfVertex prf_vertex(const int32_t *labels, const int32_t *truth, int64_t n,
                                                const int64_t *seg_off, int nseg, int64_t x0, int64_t x) {
    PrfVertex v{false, 0, -1, -1};
    if (x >= n) return v;
    v.s = seg_off ? warp_seg_of(seg_off, nseg, x0, x) : 0;
    const int64_t r = (seg_off ? seg_off[v.s] : 0) + labels[x];
    const int b = truth[x];
    if (r < 0 || r >= n || b < 0 || b >= NBINS) return v;   // reported by the sizes pass / block sizes
    v.valid = true;
    v.root = (int32_t)r;
    v.b = b;
    return v;
}

__device__ __forceinline__ double prf_jaccard(unsigned long long inter, unsigned int size, unsigned int csize) {
    return (double)inter / (double)((unsigned long long)size + csize - inter);
}

__global__ void __launch_bounds__(256) k_prf_cells(const int32_t *labels, const int32_t *truth, int64_t n,
                                                   const int64_t *seg_off, int nseg, unsigned long long tag,
                                                   unsigned long long *keys, unsigned long long *cnt, int bits,
                                                   unsigned long long *ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const unsigned lane = lane_id();
    for (int64_t x0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); x0 < n; x0 += stride) {
        const int64_t x = x0 + lane;
        const PrfVertex v = prf_vertex(labels, truth, n, seg_off, nseg, x0 < n ? x0 : n - 1, x);
        const unsigned long long key = v.valid ? ((unsigned long long)v.root << 6) | (unsigned long long)v.b : ~0ull;
        const unsigned same = key_group(v.valid, key);
        if (v.valid && lane == (unsigned)(__ffs(same) - 1)) {
            const int64_t slot = cell_slot(keys, bits, tag, key);
            if (slot < 0) flag_status(ctr, ST_BADGRAPH);
            else tagged_add(&cnt[slot], tag, (unsigned long long)__popc(same));
        }
    }
}

// PICK = false: best[root] = max over its cells of the Jaccard bits;
// PICK = true: bestb[root] = lowest block whose cell reaches best[root].
template <bool PICK>
__global__ void __launch_bounds__(256) k_prf_best(const int32_t *labels, const int32_t *truth, int64_t n,
                                                  const int64_t *seg_off, int nseg, unsigned long long tag,
                                                  const unsigned long long *keys, const unsigned long long *cnt,
                                                  int bits, const unsigned int *size, const unsigned int *bsz,
                                                  unsigned long long *best, unsigned int *bestb) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const unsigned lane = lane_id();
    for (int64_t x0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); x0 < n; x0 += stride) {
        const int64_t x = x0 + lane;
        const PrfVertex v = prf_vertex(labels, truth, n, seg_off, nseg, x0 < n ? x0 : n - 1, x);
        if (!v.valid) continue;
        const unsigned long long key = ((unsigned long long)v.root << 6) | (unsigned long long)v.b;
        const int64_t slot = cell_find(keys, bits, tag, key);
        if (slot < 0) continue;
        const unsigned long long inter = __ldcg(&cnt[slot]) & CNT_MASK;
        const double j = prf_jaccard(inter, size[v.root], bsz[(int64_t)v.s * NBINS + v.b]);
        const unsigned long long jb = (unsigned long long)__double_as_longlong(j);   // j >= 0: bits order as values
        if (!PICK) atomicMax(&best[v.root], jb);
        else if (jb == __ldcg(&best[v.root])) atomicMin(&bestb[v.root], (unsigned int)v.b);
    }
}

// One term per community (every label value r with size[r] > 0; r indexes
// the graph the labels are relative to): sums[3 s] += |C n S| (integer),
// sums[3 s + 1] += r |S|, sums[3 s + 2] += 2pr/(p + r) |S| (doubles, as bit
// patterns).
__global__ void __launch_bounds__(256) k_prf_sum(int64_t n, const int64_t *seg_off, int nseg,
                                                 unsigned long long tag, const unsigned long long *keys,
                                                 const unsigned long long *cnt, int bits, const unsigned int *size,
                                                 const unsigned int *bsz, const unsigned int *bestb,
                                                 unsigned long long *sums) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const unsigned lane = lane_id();
    for (int64_t x0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); x0 < n; x0 += stride) {
        const int64_t x = x0 + lane;
        if (x >= n || size[x] == 0u) continue;                             // communities only
        const int s = seg_off ? warp_seg_of(seg_off, nseg, x0, x) : 0;
        const unsigned int b = bestb[x];
        if (b >= (unsigned)NBINS) continue;
        const int64_t slot = cell_find(keys, bits, tag, ((unsigned long long)x << 6) | b);
        if (slot < 0) continue;
        const unsigned long long inter = __ldcg(&cnt[slot]) & CNT_MASK;
        const unsigned int sz = size[x], cs = bsz[(int64_t)s * NBINS + b];
        const double p = (double)inter / (double)sz, r = (double)inter / (double)cs;
        atomicAdd(&sums[3 * s], inter);
        atomicAdd(reinterpret_cast<double *>(&sums[3 * s + 1]), r * (double)sz);
        atomicAdd(reinterpret_cast<double *>(&sums[3 * s + 2]), (2.0 * p * r / (p + r)) * (double)sz);
    }
}

__global__ void k_prf_final(const unsigned long long *sums, const int64_t *seg_off, int nseg, int levels,
                            int64_t n_all, double *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)levels * nseg) return;
    const int s = (int)(i % nseg);
    const int64_t nv = seg_off ? seg_off[s + 1] - seg_off[s] : n_all;
    const double inv = nv > 0 ? 1.0 / (double)nv : 0.0;
    out[3 * i] = nv > 0 ? (double)sums[3 * i] / (double)nv : 0.0;
    out[3 * i + 1] = __longlong_as_double((long long)sums[3 * i + 1]) * inv;
    out[3 * i + 2] = __longlong_as_double((long long)sums[3 * i + 2]) * inv;
}

__device__ double i128_to_double(__int128 v) {
    const bool neg = v < 0;
    unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const double d = (double)(uint64_t)(u >> 64) * 18446744073709551616.0 + (double)(uint64_t)u;
    return neg ? -d : d;
}

// ARI of `levels` consecutive levels: sums is levels x nseg x (S_ab, S_a),
// out is levels x nseg.
__global__ void k_ari_final(const unsigned long long *sums, const unsigned int *bsz, const int64_t *seg_off, int nseg,
                            int levels, int64_t n_all, double *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)levels * nseg) return;
    const int s = (int)(i % nseg);
    const int64_t nv = seg_off ? seg_off[s + 1] - seg_off[s] : n_all;
    unsigned long long sb = 0;
    for (int b = 0; b < NBINS; ++b) sb += c2(bsz[(int64_t)s * NBINS + b]);
    const unsigned long long sab = sums[2 * i], sa = sums[2 * i + 1];
    const unsigned long long T = (unsigned long long)nv * (unsigned long long)(nv > 0 ? nv - 1 : 0) / 2;
    const __int128 num = 2 * (__int128)T * sab - 2 * (__int128)sa * sb;
    const __int128 den = (__int128)T * (sa + sb) - 2 * (__int128)sa * sb;
    out[i] = (nv < 2 || den == 0) ? 1.0 : i128_to_double(num) / i128_to_double(den);
}

// Per graph: the first level of highest ARI (ari is k x nseg).
__global__ void k_best_level(const double *ari, int k, int nseg, int32_t *best, double *best_ari) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    int bi = 0;
    double bv = ari[s];
    for (int L = 1; L < k; ++L) {
        const double v = ari[(int64_t)L * nseg + s];
        if (v > bv) { bv = v; bi = L; }
    }
    best[s] = bi;
    if (best_ari) best_ari[s] = bv;
}

inline unsigned grid_for(int64_t work) {
    const int64_t g = ceil_div(work > 0 ? work : 1, 256);
    return (unsigned)(g < 65536 ? g : 65536);
}

}  // namespace

cudaError_t launch_features(const int64_t *ooff, const int32_t *ocol, const int32_t *deg, const uint32_t *t,
                            int64_t n, int64_t m, const int32_t *orows, const int32_t *osrc, const int64_t *seg_off,
                            int nseg, unsigned int *hist, float *feat, unsigned long long *ctr, cudaStream_t s) {
    const int ns = seg_off ? nseg : 1;
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)ns * NBINS * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    if (m > 0 && FEAT_PERSISTENT && osrc) {
        unsigned grid = 1;
        e = persistent_grid(k_feat_hist_warps, TILE_THREADS, 0, ceil_div(m, FH_CHUNK), &grid);
        if (e != cudaSuccess) return e;
        k_feat_hist_warps<<<grid, TILE_THREADS, 0, s>>>(ocol, deg, t, m, osrc, seg_off, ns, hist, ctr);
    } else if (m > 0) {
        k_feat_hist<<<(unsigned)ceil_div(m, TILE), TILE_THREADS, 0, s>>>(ooff, ocol, deg, t, n, m, orows, osrc, seg_off, ns,
                                                                         hist, ctr);
    }
    k_feat_final<<<(unsigned)ceil_div((int64_t)ns * 32, 256), 256, 0, s>>>(hist, seg_off, ns, n, feat);
    count_launches(m > 0 ? 2 : 1);
    return cudaGetLastError();
}

cudaError_t launch_best_level(const double *ari, int k, int nseg, int32_t *best, double *best_ari, cudaStream_t s) {
    if (nseg <= 0) return cudaSuccess;
    k_best_level<<<(unsigned)ceil_div(nseg, 128), 128, 0, s>>>(ari, k, nseg, best, best_ari);
    count_launches(1);
    return cudaGetLastError();
}

int ari_table_bits(int64_t n) {
    int bits = 6;
    while (((int64_t)1 << bits) < 2 * n) ++bits;
    return bits;
}

cudaError_t launch_ari(const int32_t *labels, int k, const int32_t *truth, int64_t n, const int64_t *seg_off, int nseg,
                       unsigned int *bsz, unsigned int *size, int64_t size_len, unsigned long long *keys,
                       unsigned long long *cnt, int64_t tsize, unsigned long long *sums, double *out,
                       unsigned long long *tag, unsigned long long *ctr, cudaStream_t s) {
    const int ns = seg_off ? nseg : 1;
    const int bits = ari_table_bits(n);
    cudaError_t e = cudaMemsetAsync(bsz, 0, (size_t)ns * NBINS * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    int launched = 0;
    if (n > 0) {
        k_block_sizes<<<(unsigned)ceil_div(n, BS_CHUNK), 256, 0, s>>>(truth, n, seg_off, ns, bsz, ctr);
        ++launched;
    }
    for (int L0 = 0; L0 < k; L0 += ARI_CHUNK) {
        const int levels = k - L0 < ARI_CHUNK ? k - L0 : ARI_CHUNK;
        if ((e = cudaMemsetAsync(sums, 0, (size_t)2 * ns * levels * sizeof(unsigned long long), s)) != cudaSuccess)
            return e;
        for (int L = L0; L < L0 + levels && n > 0; ++L) {
            if (*tag >= TAG_LIMIT) {             // first use, or the tag would wrap: zero every word
                if ((e = cudaMemsetAsync(size, 0, (size_t)2 * size_len * sizeof(unsigned int), s)) != cudaSuccess)
                    return e;
                if ((e = cudaMemsetAsync(keys, 0, (size_t)tsize * sizeof(unsigned long long), s)) != cudaSuccess)
                    return e;
                if ((e = cudaMemsetAsync(cnt, 0, (size_t)tsize * sizeof(unsigned long long), s)) != cudaSuccess)
                    return e;
                *tag = 0;
            }
            const unsigned long long t = ++*tag;
            unsigned long long *ls = sums + (int64_t)2 * ns * (L - L0);
            const int32_t *lab = labels + (int64_t)L * n;
            unsigned int *cur = size + (t & 1ull) * size_len, *prev = size + ((t & 1ull) ^ 1ull) * size_len;
            k_ari_sizes<<<vertex_pass_grid(n), 256, 0, s>>>(lab, n, seg_off, ns, cur, prev, ls, ctr);
            k_ari_cells<<<vertex_pass_grid(n), 256, 0, s>>>(lab, truth, n, seg_off, ns, t, cur, keys, cnt, bits, ls,
                                                            ctr);
            launched += 2;
        }
        const int64_t cells = (int64_t)levels * ns;
        k_ari_final<<<(unsigned)ceil_div(cells, 128), 128, 0, s>>>(sums, bsz, seg_off, ns, levels, n,
                                                                   out + (int64_t)L0 * ns);
        ++launched;
    }
    count_launches(launched);
    return cudaGetLastError();
}

cudaError_t launch_prf(const int32_t *labels, int k, const int32_t *truth, int64_t n, const int64_t *seg_off, int nseg,
                       unsigned int *bsz, unsigned int *size, int64_t size_len, unsigned long long *keys,
                       unsigned long long *cnt, int64_t tsize, unsigned long long *scratch_sums,
                       unsigned long long *best, unsigned int *bestb, unsigned long long *sums, double *out,
                       unsigned long long *tag, unsigned long long *ctr, cudaStream_t s) {
    const int ns = seg_off ? nseg : 1;
    const int bits = ari_table_bits(n);
    cudaError_t e = cudaMemsetAsync(bsz, 0, (size_t)ns * NBINS * sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    int launched = 0;
    if (n > 0) {
        k_block_sizes<<<(unsigned)ceil_div(n, BS_CHUNK), 256, 0, s>>>(truth, n, seg_off, ns, bsz, ctr);
        ++launched;
    }
    for (int L0 = 0; L0 < k; L0 += ARI_CHUNK) {
        const int levels = k - L0 < ARI_CHUNK ? k - L0 : ARI_CHUNK;
        if ((e = cudaMemsetAsync(sums, 0, (size_t)3 * ns * levels * sizeof(unsigned long long), s)) != cudaSuccess)
            return e;
        for (int L = L0; L < L0 + levels && n > 0; ++L) {
            if (*tag >= TAG_LIMIT) {             // first use, or the tag would wrap: zero every word
                if ((e = cudaMemsetAsync(size, 0, (size_t)2 * size_len * sizeof(unsigned int), s)) != cudaSuccess)
                    return e;
                if ((e = cudaMemsetAsync(keys, 0, (size_t)tsize * sizeof(unsigned long long), s)) != cudaSuccess)
                    return e;
                if ((e = cudaMemsetAsync(cnt, 0, (size_t)tsize * sizeof(unsigned long long), s)) != cudaSuccess)
                    return e;
                *tag = 0;
            }
            const unsigned long long t = ++*tag;
            unsigned int *cur = size + (t & 1ull) * size_len, *prev = size + ((t & 1ull) ^ 1ull) * size_len;
            const int32_t *lab = labels + (int64_t)L * n;
            if ((e = cudaMemsetAsync(best, 0, (size_t)n * sizeof(unsigned long long), s)) != cudaSuccess) return e;
            if ((e = cudaMemsetAsync(bestb, 0xFF, (size_t)n * sizeof(unsigned int), s)) != cudaSuccess) return e;
            if ((e = cudaMemsetAsync(scratch_sums, 0, (size_t)2 * ns * sizeof(unsigned long long), s)) != cudaSuccess)
                return e;
            const unsigned grid = vertex_pass_grid(n), gv = grid_for(n);
            unsigned long long *ls = sums + (int64_t)3 * ns * (L - L0);
            k_ari_sizes<<<grid, 256, 0, s>>>(lab, n, seg_off, ns, cur, prev, scratch_sums, ctr);
            k_prf_cells<<<gv, 256, 0, s>>>(lab, truth, n, seg_off, ns, t, keys, cnt, bits, ctr);
            k_prf_best<false><<<gv, 256, 0, s>>>(lab, truth, n, seg_off, ns, t, keys, cnt, bits, cur, bsz, best, bestb);
            k_prf_best<true><<<gv, 256, 0, s>>>(lab, truth, n, seg_off, ns, t, keys, cnt, bits, cur, bsz, best, bestb);
            k_prf_sum<<<gv, 256, 0, s>>>(n, seg_off, ns, t, keys, cnt, bits, cur, bsz, bestb, ls);
            launched += 5;
        }
        const int64_t cells = (int64_t)levels * ns;
        k_prf_final<<<(unsigned)ceil_div(cells, 128), 128, 0, s>>>(sums, seg_off, ns, levels, n,
                                                                   out + (int64_t)3 * L0 * ns);
        ++launched;
    }
    count_launches(launched);
    return cudaGetLastError();
}

}  // namespace tec
