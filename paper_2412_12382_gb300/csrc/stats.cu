// Sweep statistics and the threshold rules of thumb (Sec. IV-D, Fig. 6).
//
// For k labelings of a batch of graphs (rows of a sweep over thresholds
// theta_r = p[r]/q[r]) and every graph s of the batch:
//   ncomp    components (roots: vertices whose label is themselves),
//   kept     edges with sim >= theta_r (Algorithm 1's survivors),
//   largest  vertices of the largest component,
//   intra    edges of the input graph whose ends share a component,
//   Q        modularity (Sec. II) of the components as communities:
//            Q = intra/m - sum_c vol(c)^2 / (2m)^2, vol(c) the degree sum,
//            from exact integers: Q = (4 m intra - sum vol^2) / (4 m^2).
// Edge pass (k_stat_edges): each edge's level L (thresholds survived, the
// binary search of the sweep) and its join level J (sorted thresholds at
// which both ends share a component: a prefix, because the labelings of a
// sweep are nested; J by binary search over the rows) go into per-graph
// histograms; kept and intra are their suffix sums.  Vertex passes, per
// level: sizes and volumes at the roots (two alternating counter arrays,
// each pass zeroing the other), then the roots' counts, maximum and squared
// volumes.
//
// Rules (k_rules, one thread per graph): R1 visits the thresholds in
// decreasing order and takes the one just above the largest increase of the
// largest component (the highest on ties), falling back to R2 where the
// largest component never grows; R2 takes the largest modularity (the lowest
// threshold on ties).
#include "tec_internal.cuh"

namespace tec {
namespace {

constexpr int MAXK = 127;

struct SortedRows {
    int order[MAXK];         // order[i] = row of the i-th smallest threshold
};

__device__ __forceinline__ unsigned long long c_sq(unsigned long long v) { return v * v; }

template <bool WIDE>
__global__ void __launch_bounds__(TILE_THREADS)
k_stat_edges(const int64_t *ooff, const int32_t *ocol, const int32_t *deg, const uint32_t *t, int64_t n, int64_t m,
             const int32_t *orows, const int32_t *osrc, int measure, const int64_t *tp, const int64_t *tq, int k,
             SortedRows rows, const int32_t *labels, const int64_t *seg_off, int nseg, unsigned long long *hist,
             unsigned long long *ctr) {
    __shared__ unsigned int s_h[2 * (MAXK + 1)];
    if (graph_bad(ctr)) return;                  // uniform over the grid
    const int64_t k0 = (int64_t)blockIdx.x * TILE;
    int64_t r0, r1;
    tile_row_range(orows, ooff, n, m, r0, r1);
    int s0 = 0;
    bool one = true;
    if (seg_off) {
        s0 = row_search(seg_off, 0, nseg - 1, r0);
        one = row_search(seg_off, s0, nseg - 1, r1) == s0;
    }
    for (int i = threadIdx.x; i < 2 * (k + 1); i += blockDim.x) s_h[i] = 0u;
    __syncthreads();
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int64_t j = k0 + (int64_t)i * TILE_THREADS + threadIdx.x;
        if (j >= m) break;
        const int64_t u = edge_source(osrc, ooff, r0, r1, j);
        const int32_t v = ocol[j];
        const int64_t s = (int64_t)deg[u] + deg[v];
        const uint32_t tt = t[j];
        int lo = 0, hi = k;                      // level: thresholds survived
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (keep_edge<WIDE>(measure, tt, s, tp[mid], tq[mid])) lo = mid + 1; else hi = mid;
        }
        const int L = lo;
        lo = 0;
        hi = k;                                  // join level: sorted rows with both ends together
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            const int32_t *lab = labels + (int64_t)rows.order[mid] * n;
            if (lab[u] == lab[v]) lo = mid + 1; else hi = mid;
        }
        const int J = lo;
        if (one) {
            atomicAdd(&s_h[L], 1u);
            atomicAdd(&s_h[k + 1 + J], 1u);
        } else {
            const int sg = row_search(seg_off, 0, nseg - 1, u);
            atomicAdd(&hist[(int64_t)sg * 2 * (k + 1) + L], 1ull);
            atomicAdd(&hist[(int64_t)sg * 2 * (k + 1) + k + 1 + J], 1ull);
        }
    }
    __syncthreads();
    if (one)
        for (int i = threadIdx.x; i < 2 * (k + 1); i += blockDim.x)
            if (s_h[i]) atomicAdd(&hist[(int64_t)s0 * 2 * (k + 1) + i], (unsigned long long)s_h[i]);
}

// Pass 1 of a level: vertices and degree volume per root into cur_n / cur_v
// (zeroed); zeroes prev_n / prev_v for the next level.  Chunks of VCHUNK
// vertices per warp, one segment lookup per chunk.
__global__ void __launch_bounds__(256) k_stat_sizes(const int32_t *labels, const int32_t *deg, int64_t n,
                                                    const int64_t *seg_off, int nseg, unsigned int *cur_n,
                                                    unsigned long long *cur_v, unsigned int *prev_n,
                                                    unsigned long long *prev_v, unsigned long long *ctr) {
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const unsigned lane = lane_id();
    for (int64_t c0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * VCHUNK; c0 < n;
         c0 += nw * VCHUNK) {
        int32_t lab[VCHUNK_V];
        int32_t dg[VCHUNK_V];
#pragma unroll
        for (int v = 0; v < VCHUNK_V; ++v) {
            const int64_t x = c0 + v * 32 + lane;
            lab[v] = x < n ? labels[x] : 0;
            dg[v] = x < n ? deg[x] : 0;
            if (x < n) {
                prev_n[x] = 0u;
                prev_v[x] = 0ull;
            }
        }
        const int64_t cend = c0 + VCHUNK < n ? c0 + VCHUNK : n;
        const int sg = seg_off ? warp_seg_of(seg_off, nseg, c0, c0) : 0;
        const bool uniform = !seg_off || sg + 1 >= nseg || seg_off[sg + 1] >= cend;
#pragma unroll
        for (int v = 0; v < VCHUNK_V; ++v) {
            const int64_t x0 = c0 + v * 32, x = x0 + lane;
            bool valid = x < n;
            int32_t root = -1;
            if (valid) {
                const int s = uniform ? sg : warp_seg_of(seg_off, nseg, x0, x);
                const int64_t r = (seg_off ? seg_off[s] : 0) + lab[v];
                if (r < 0 || r >= n) {
                    flag_status(ctr, ST_BADGRAPH);
                    valid = false;
                } else {
                    root = (int32_t)r;
                }
            }
            // one root for the whole warp (a large component over consecutive
            // vertices): one add each; otherwise every lane adds its own
            const unsigned vm = __ballot_sync(0xffffffffu, valid);
            const int32_t r0 = vm ? __shfl_sync(0xffffffffu, root, __ffs(vm) - 1) : -1;
            const unsigned long long vol = valid ? (unsigned long long)dg[v] : 0ull;
            if (__all_sync(0xffffffffu, !valid || root == r0)) {
                const unsigned long long gv = warp_sum64(vol);
                if (vm && lane == (unsigned)(__ffs(vm) - 1)) {
                    atomicAdd(&cur_n[root], (unsigned int)__popc(vm));
                    atomicAdd(&cur_v[root], gv);
                }
            } else if (valid) {
                atomicAdd(&cur_n[root], 1u);
                atomicAdd(&cur_v[root], vol);
            }
        }
    }
}

// Pass 2 of a level: for every root x (label of x is x), its component's size
// and volume: count, maximum and squared volume per graph into sums[3 s ..].
__global__ void __launch_bounds__(256) k_stat_roots(const int32_t *labels, int64_t n, const int64_t *seg_off,
                                                    int nseg, const unsigned int *cur_n,
                                                    const unsigned long long *cur_v, unsigned long long *sums) {
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const unsigned lane = lane_id();
    int pend_s = -1;
    unsigned long long p_cnt = 0, p_max = 0, p_sq = 0;
    for (int64_t c0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * VCHUNK; c0 < n;
         c0 += nw * VCHUNK) {
        const int64_t cend = c0 + VCHUNK < n ? c0 + VCHUNK : n;
        const int sg = seg_off ? warp_seg_of(seg_off, nseg, c0, c0) : 0;
        const bool uniform = !seg_off || sg + 1 >= nseg || seg_off[sg + 1] >= cend;
        unsigned long long cnt = 0, mx = 0, sq = 0;
#pragma unroll
        for (int v = 0; v < VCHUNK_V; ++v) {
            const int64_t x0 = c0 + v * 32, x = x0 + lane;
            bool is_root = false;
            int s = sg;
            unsigned long long sz = 0, vol = 0;
            if (x < n) {
                if (!uniform) s = warp_seg_of(seg_off, nseg, x0, x);
                const int64_t base = seg_off ? seg_off[s] : 0;
                is_root = base + labels[x] == x;
                if (is_root) {
                    sz = cur_n[x];
                    vol = cur_v[x];
                }
            }
            if (uniform) {
                cnt += is_root ? 1ull : 0ull;
                mx = sz > mx ? sz : mx;
                sq += c_sq(vol);
            } else if (is_root) {
                atomicAdd(&sums[3 * s], 1ull);
                atomicMax(&sums[3 * s + 1], sz);
                atomicAdd(&sums[3 * s + 2], c_sq(vol));
            }
        }
        if (uniform) {
            cnt = warp_sum64(cnt);
            sq = warp_sum64(sq);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
                mx = y > mx ? y : mx;
            }
            if (sg != pend_s) {
                if (lane == 0 && pend_s >= 0) {
                    atomicAdd(&sums[3 * pend_s], p_cnt);
                    atomicMax(&sums[3 * pend_s + 1], p_max);
                    atomicAdd(&sums[3 * pend_s + 2], p_sq);
                }
                pend_s = sg;
                p_cnt = p_max = p_sq = 0;
            }
            p_cnt += cnt;
            p_max = mx > p_max ? mx : p_max;
            p_sq += sq;
        }
    }
    if (lane == 0 && pend_s >= 0) {
        atomicAdd(&sums[3 * pend_s], p_cnt);
        atomicMax(&sums[3 * pend_s + 1], p_max);
        atomicAdd(&sums[3 * pend_s + 2], p_sq);
    }
}

__device__ double i128_double(__int128 v) {
    const bool neg = v < 0;
    unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const double d = (double)(uint64_t)(u >> 64) * 18446744073709551616.0 + (double)(uint64_t)u;
    return neg ? -d : d;
}

// One thread per (row, graph): stats_out[row * nseg + s].  sums holds the
// vertex-pass results of every row (3 per graph), hist the edge histograms.
__global__ void k_stat_final(const unsigned long long *hist, const unsigned long long *sums, int k, int nseg,
                             SortedRows rows, tec_sweep_stat *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)k * nseg) return;
    const int r = (int)(i / nseg), s = (int)(i % nseg);
    int pos = 0;                                 // sorted position of row r
    while (rows.order[pos] != r) ++pos;
    const unsigned long long *h = hist + (int64_t)s * 2 * (k + 1);
    unsigned long long kept = 0, intra = 0, ms = 0;
    for (int L = 0; L <= k; ++L) {
        ms += h[L];
        if (L >= pos + 1) kept += h[L];
        if (L >= pos + 1) intra += h[k + 1 + L];
    }
    // ms: edges of graph s (every edge has exactly one level)
    const unsigned long long *sm = sums + ((int64_t)r * nseg + s) * 3;
    tec_sweep_stat st;
    st.ncomp = (int64_t)sm[0];
    st.kept = (int64_t)kept;
    st.largest = (int64_t)sm[1];
    st.intra = (int64_t)intra;
    if (ms == 0) {
        st.modularity = 0.0;
    } else {
        const __int128 num = 4 * (__int128)ms * (__int128)intra - (__int128)sm[2];
        const __int128 den = 4 * (__int128)ms * (__int128)ms;
        st.modularity = i128_double(num) / i128_double(den);
    }
    out[i] = st;
}

__global__ void k_rules(const tec_sweep_stat *stats, int k, int nseg, SortedRows rows, int rule, int32_t *best) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    int r2 = rows.order[0];                      // R2: largest modularity, lowest threshold on ties
    for (int i = 1; i < k; ++i) {
        const int r = rows.order[i];
        if (stats[(int64_t)r * nseg + s].modularity > stats[(int64_t)r2 * nseg + s].modularity) r2 = r;
    }
    int r1 = -1;                                 // R1: just above the largest increase of the largest component
    long long best_jump = 0;
    if (rule == TEC_RULE_LARGEST_JUMP) {
        for (int i = k - 2; i >= 0; --i) {
            const long long jump = (long long)stats[(int64_t)rows.order[i] * nseg + s].largest -
                                   (long long)stats[(int64_t)rows.order[i + 1] * nseg + s].largest;
            if (jump > best_jump) {
                best_jump = jump;
                r1 = rows.order[i + 1];
            }
        }
    }
    best[s] = r1 >= 0 ? r1 : r2;
}

inline unsigned grid_for(int64_t work) {
    const int64_t g = ceil_div(work > 0 ? work : 1, 256);
    return (unsigned)(g < 65536 ? g : 65536);
}

SortedRows make_rows(const int *order, int k) {
    SortedRows r{};
    for (int i = 0; i < k && i < MAXK; ++i) r.order[i] = order[i];
    return r;
}

}  // namespace

cudaError_t launch_sweep_stats(const int64_t *ooff, const int32_t *ocol, const int32_t *deg, const uint32_t *t,
                               int64_t n, int64_t m, const int32_t *orows, const int32_t *osrc, int measure, const int64_t *tp, const int64_t *tq, int k,
                               const int *order, bool wide, const int32_t *labels, const int64_t *seg_off, int nseg,
                               unsigned long long *hist, unsigned int *cnt_n, unsigned long long *cnt_v,
                               int64_t cnt_len, unsigned long long *sums, tec_sweep_stat *out,
                               unsigned long long *ctr, cudaStream_t s) {
    const int ns = seg_off ? nseg : 1;
    const SortedRows rows = make_rows(order, k);
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)ns * 2 * (k + 1) * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sums, 0, (size_t)k * ns * 3 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt_n, 0, (size_t)2 * cnt_len * sizeof(unsigned int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt_v, 0, (size_t)2 * cnt_len * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    int launched = 0;
    if (m > 0) {
        const unsigned grid = (unsigned)ceil_div(m, TILE);
        if (wide)
            k_stat_edges<true><<<grid, TILE_THREADS, 0, s>>>(ooff, ocol, deg, t, n, m, orows, osrc, measure, tp, tq, k,
                                                             rows, labels, seg_off, ns, hist, ctr);
        else
            k_stat_edges<false><<<grid, TILE_THREADS, 0, s>>>(ooff, ocol, deg, t, n, m, orows, osrc, measure, tp, tq,
                                                              k, rows, labels, seg_off, ns, hist, ctr);
        ++launched;
    }
    for (int r = 0; r < k && n > 0; ++r) {
        unsigned int *cn = cnt_n + (r & 1) * cnt_len, *pn = cnt_n + ((r & 1) ^ 1) * cnt_len;
        unsigned long long *cv = cnt_v + (r & 1) * cnt_len, *pv = cnt_v + ((r & 1) ^ 1) * cnt_len;
        const int32_t *lab = labels + (int64_t)r * n;
        k_stat_sizes<<<vertex_pass_grid(n), 256, 0, s>>>(lab, deg, n, seg_off, ns, cn, cv, pn, pv, ctr);
        k_stat_roots<<<vertex_pass_grid(n), 256, 0, s>>>(lab, n, seg_off, ns, cn, cv, sums + (int64_t)r * ns * 3);
        launched += 2;
    }
    k_stat_final<<<(unsigned)ceil_div((int64_t)k * ns, 128), 128, 0, s>>>(hist, sums, k, ns, rows, out);
    count_launches(launched + 1);
    return cudaGetLastError();
}

cudaError_t launch_rules(const tec_sweep_stat *stats, int k, int nseg, const int *order, int rule, int32_t *best,
                         cudaStream_t s) {
    if (nseg <= 0) return cudaSuccess;
    k_rules<<<(unsigned)ceil_div(nseg, 128), 128, 0, s>>>(stats, k, nseg, make_rows(order, k), rule, best);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace tec
