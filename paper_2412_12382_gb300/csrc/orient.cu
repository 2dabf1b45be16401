// Degrees, CSR validation and the degree-ordered orientation.
//
// The oriented CSR is the stream compaction of the symmetric CSR that keeps
// entry (u, v) iff (deg u, u) < (deg v, v).  Compaction preserves order, so
// every oriented row stays sorted, and the oriented offset of row u is the
// number of kept entries before off[u].  Two streaming passes over tiles of
// 2048 entries: (1) keep bits + per-tile counts, (2) after a scan of the tile
// counts, scatter of the kept ids and of the row offsets.  Each tile learns
// the row of its entries from one coalesced read of its rows' offsets
// (tile_entry_rows).
#include "bulk.cuh"
#include "tec_internal.cuh"

namespace tec {
namespace {

// One thread per row u: the tiles whose first entry lies in u's entries
// [off[u], off[u+1]) get u (tiles outside [0, ntiles) are skipped, so a bad
// offset array writes nothing out of range).
__global__ void k_tile_rows(const int64_t *off, int64_t n, int64_t ntiles, int32_t *trow) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = off[u], b = off[u + 1];
        if (a >= b || a < 0) continue;
        for (int64_t t = (a + TILE - 1) / TILE; t * TILE < b && t < ntiles; ++t) trow[t] = (int32_t)u;
    }
}

__global__ void k_widen(const int32_t *in, int64_t count, int64_t *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i];
}

__global__ void k_degrees(const int64_t *off, int64_t n, int32_t *deg) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x)
        deg[u] = (int32_t)(off[u + 1] - off[u]);
}

__global__ void k_validate_rows(const int64_t *off, int64_t n, int64_t nnz, unsigned long long *ctr) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        int64_t a = off[u], b = off[u + 1];
        if (a > b || b - a >= n) flag_status(ctr, ST_BADGRAPH);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (off[0] != 0 || off[n] != nnz))
        flag_status(ctr, ST_BADGRAPH);
}

// Needs valid offsets (k_validate_rows passed).  Checks ids in range, no
// self-loop, strictly increasing rows, and that u is in N(v) for every v in N(u).
__global__ void __launch_bounds__(TILE_THREADS)
k_validate_entries(const int64_t *off, const int32_t *col, int64_t n, int64_t nnz, const int32_t *trow,
                   unsigned long long *ctr) {
    __shared__ __align__(16) int32_t s_row[TILE];
    __shared__ int32_t s_warp[TILE_THREADS / 32];
    const int64_t k0 = (int64_t)blockIdx.x * TILE;
    int64_t r0, r1;
    tile_row_range(trow, off, n, nnz, r0, r1);
    tile_entry_rows(off, nnz, (int64_t)blockIdx.x, r0, r1, s_row, s_warp);
    for (int i = 0; i < TILE_ITEMS; ++i) {
        int64_t k = k0 + (int64_t)i * TILE_THREADS + threadIdx.x;
        if (k >= nnz) break;
        int64_t u = r0 + s_row[i * TILE_THREADS + threadIdx.x];
        int64_t v = col[k];
        bool bad = v < 0 || v >= n || v == u || (k > off[u] && col[k - 1] >= v);
        if (!bad) {
            int64_t lo = off[v], hi = off[v + 1];
            while (lo < hi) {
                int64_t mid = lo + (hi - lo) / 2;
                if (col[mid] < u) lo = mid + 1; else hi = mid;
            }
            bad = lo >= off[v + 1] || col[lo] != u;
        }
        if (bad) flag_status(ctr, ST_BADGRAPH);
    }
}

__device__ __forceinline__ int block_sum_int(int x) {
    __shared__ int ws[TILE_THREADS / 32];
    x = warp_sum(x);
    if (lane_id() == 0) ws[threadIdx.x >> 5] = x;
    __syncthreads();
    int tot = 0;
#pragma unroll
    for (int w = 0; w < TILE_THREADS / 32; ++w) tot += ws[w];
    __syncthreads();
    return tot;
}

// Whether each orientation pass runs as the persistent bulk-copy kernel (1)
// or as one block per tile reading global memory (0), the blocks per SM the
// one-block-per-tile flag pass is compiled for (register budget), and whether
// its degree gathers bypass L1; chosen by the autotuner.
constexpr int ORIENT_FLAGS_PERSISTENT = 0;
constexpr int ORIENT_FILL_PERSISTENT = 0;
constexpr int ORIENT_FLAGS_MIN_BLOCKS = 1;
constexpr int ORIENT_GATHER_CG = 1;

// Pass 1 on one tile of `cnt` symmetric entries whose column ids are read
// from sc (shared or global memory): keep bit per entry (bit k of flags) and
// the tile's kept count.  The degree gathers of the eight items' columns are
// issued first and stay in flight while the tile's rows are worked out.
__device__ __forceinline__ void flags_tile(const int32_t *sc, int64_t tile, int cnt, const int64_t *__restrict__ off,
                                           const int32_t *__restrict__ deg, int64_t n, int64_t nnz,
                                           const int32_t *__restrict__ trow, uint32_t *__restrict__ flags,
                                           int64_t *__restrict__ tile_cnt, int32_t *s_row, int32_t *s_warp,
                                           unsigned long long *ctr) {
    int32_t v[TILE_ITEMS], dv[TILE_ITEMS];
    bool bad = false;
#pragma unroll
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int x = i * TILE_THREADS + (int)threadIdx.x;
        v[i] = x < cnt ? sc[x] : -1;
        const bool in = v[i] >= 0 && (int64_t)v[i] < n;
        bad |= x < cnt && !in;
        if (!in) v[i] = -1;
        dv[i] = in ? (ORIENT_GATHER_CG ? __ldcg(&deg[v[i]]) : deg[v[i]]) : 0;
    }
    if (bad) flag_status(ctr, ST_BADGRAPH);
    int64_t r0, r1;
    tile_row_range(trow, off, n, nnz, tile, r0, r1);
    tile_entry_rows(off, nnz, tile, r0, r1, s_row, s_warp);
    const unsigned lane = lane_id();
    int c = 0;
#pragma unroll
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int x = i * TILE_THREADS + (int)threadIdx.x;
        const int xw = x - (int)lane;
        const int64_t u = r0 + s_row[x];
        const bool f = v[i] >= 0 && rank_less(deg[u], u, dv[i], v[i]);
        const unsigned b = __ballot_sync(0xffffffffu, f);
        if (lane == 0 && xw < cnt) flags[(tile * TILE + xw) >> 5] = b;
        c += f ? 1 : 0;
    }
    const int tot = block_sum_int(c);
    if (threadIdx.x == 0) tile_cnt[tile] = tot;
}

// Pass 2 on one tile of `cnt` entries, column ids from sc and its flag words
// from sw (shared or global memory): scatter of the kept ids to
// ocol[global rank of the keep bit] (and of the source row to osrc), and
// ooff[u] for every row that starts (or, if empty, sits) at an entry of the
// tile.  The rank of a keep bit is the tile's base plus a popcount prefix of
// the tile's flag words.
__device__ __forceinline__ void fill_tile(const int32_t *sc, const uint32_t *sw, int64_t tile, int cnt,
                                          const int64_t *__restrict__ off, int64_t n, int64_t nnz,
                                          const int32_t *__restrict__ trow, const int64_t *__restrict__ tile_base,
                                          int64_t *__restrict__ ooff, int32_t *__restrict__ ocol,
                                          int32_t *__restrict__ osrc, int64_t m, int32_t *s_row, int32_t *s_warp,
                                          int32_t *s_wpre, uint32_t *s_word, unsigned long long *ctr) {
    constexpr int WORDS = TILE / 32;
    static_assert(WORDS == 64, "two flag words per lane of warp 0");
    int64_t r0, r1;
    tile_row_range(trow, off, n, nnz, tile, r0, r1);
    const int64_t base = tile_base[tile];
    int32_t c[TILE_ITEMS];
#pragma unroll
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int x = i * TILE_THREADS + (int)threadIdx.x;
        c[i] = x < cnt ? sc[x] : 0;
    }
    if (threadIdx.x < WORDS) s_word[threadIdx.x] = 32 * (int)threadIdx.x < cnt ? sw[threadIdx.x] : 0u;
    tile_entry_rows(off, nnz, tile, r0, r1, s_row, s_warp);    // its barriers publish s_word
    if (threadIdx.x < 32) {
        const int a = __popc(s_word[2 * threadIdx.x]), b = __popc(s_word[2 * threadIdx.x + 1]);
        int inc = a + b;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, inc, d);
            if (threadIdx.x >= (unsigned)d) inc += x;
        }
        s_wpre[2 * threadIdx.x] = inc - a - b;
        s_wpre[2 * threadIdx.x + 1] = inc - b;
    }
    __syncthreads();
    const int64_t k0 = tile * TILE, k1 = k0 + cnt;
    // oriented offsets of the rows whose first entry lies in the tile
    for (int64_t r = r0 + threadIdx.x; r <= r1; r += TILE_THREADS) {
        const int64_t a = off[r];
        if (a >= k0 && a < k1) {
            const int p = (int)(a - k0);
            ooff[r] = base + s_wpre[p >> 5] + __popc(s_word[p >> 5] & ((1u << (p & 31)) - 1u));
        }
    }
    // empty rows just before r0 that sit at the tile's first entry
    if (threadIdx.x == 0 && off[r0] == k0)
        for (int64_t x = r0 - 1; x >= 0 && off[x] == k0; --x) ooff[x] = base;
    const unsigned lane = lane_id();
#pragma unroll
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int p = i * TILE_THREADS + (int)threadIdx.x;
        const uint32_t word = s_word[p >> 5];
        if (p < cnt && ((word >> lane) & 1u)) {
            const int64_t pos = base + s_wpre[p >> 5] + __popc(word & ((1u << lane) - 1u));
            if (pos < m) {
                ocol[pos] = c[i];
                if (osrc) osrc[pos] = (int32_t)(r0 + s_row[p]);
            } else {
                flag_status(ctr, ST_BADGRAPH);
            }
        }
    }
}

constexpr uint32_t OB_COL_BYTES = TILE * 4;
constexpr uint32_t OB_WORD_BYTES = TILE / 8;

// Both passes run as persistent kernels: each block walks tiles blockIdx.x,
// + gridDim.x, ..., and while it works on one tile the copy engine brings the
// column ids (and, in pass 2, the flag words) of its next tile into the other
// shared-memory stage.  A partial last tile is read from global memory.  A
// copy that does not land within the wait cap sets ST_TIMEOUT.
template <bool FILL, bool BULK>
__global__ void __launch_bounds__(TILE_THREADS, (BULK || FILL) ? 1 : ORIENT_FLAGS_MIN_BLOCKS)
k_orient_pass(const int64_t *__restrict__ off, const int32_t *__restrict__ col, const int32_t *__restrict__ deg,
              int64_t n, int64_t nnz, const int32_t *__restrict__ trow,
              uint32_t *__restrict__ flags, int64_t *__restrict__ tile_cnt, const int64_t *__restrict__ tile_base,
              int64_t *__restrict__ ooff, int32_t *__restrict__ ocol, int32_t *__restrict__ osrc, int64_t m,
              unsigned long long *ctr) {
    __shared__ __align__(16) int32_t s_col[BULK_STAGES * TILE];
    __shared__ __align__(16) uint32_t s_w[FILL ? BULK_STAGES * (TILE / 32) : 4];
    __shared__ __align__(16) int32_t s_row[TILE];
    __shared__ int32_t s_warp[TILE_THREADS / 32];
    __shared__ int32_t s_wpre[TILE / 32];
    __shared__ uint32_t s_word[TILE / 32];
    __shared__ uint64_t bar[BULK_STAGES];
    __shared__ int s_flag;
    if (!BULK) {                                 // one tile per block, read from global memory
        const int64_t tile = blockIdx.x;
        const int cnt = (int)(nnz - tile * TILE < TILE ? nnz - tile * TILE : TILE);
        if (FILL)
            fill_tile(col + tile * TILE, flags + tile * (TILE / 32), tile, cnt, off, n, nnz, trow, tile_base, ooff,
                      ocol, osrc, m, s_row, s_warp, s_wpre, s_word, ctr);
        else
            flags_tile(col + tile * TILE, tile, cnt, off, deg, n, nnz, trow, flags, tile_cnt, s_row, s_warp, ctr);
        return;
    }
    const int64_t full = nnz / TILE;
    bulk_init(bar, &s_flag);
    const bool ok = bulk_tiles(
        full, bar, &s_flag, ctr,
        [&](int64_t tile, int stage) {
            fence_proxy_async();
            mbar_arrive_expect_tx(&bar[stage], OB_COL_BYTES + (FILL ? OB_WORD_BYTES : 0u));
            bulk_g2s(s_col + stage * TILE, col + tile * TILE, OB_COL_BYTES, &bar[stage]);
            if (FILL) bulk_g2s(s_w + stage * (TILE / 32), flags + tile * (TILE / 32), OB_WORD_BYTES, &bar[stage]);
        },
        [&](int64_t tile, int stage) {
            if (FILL)
                fill_tile(s_col + stage * TILE, s_w + stage * (TILE / 32), tile, TILE, off, n, nnz, trow, tile_base,
                          ooff, ocol, osrc, m, s_row, s_warp, s_wpre, s_word, ctr);
            else
                flags_tile(s_col + stage * TILE, tile, TILE, off, deg, n, nnz, trow, flags, tile_cnt, s_row, s_warp,
                           ctr);
        });
    if (!ok) return;
    if (full * TILE < nnz && blockIdx.x == (unsigned)(full % gridDim.x)) {
        const int cnt = (int)(nnz - full * TILE);
        if (FILL)
            fill_tile(col + full * TILE, flags + full * (TILE / 32), full, cnt, off, n, nnz, trow, tile_base, ooff,
                      ocol, osrc, m, s_row, s_warp, s_wpre, s_word, ctr);
        else
            flags_tile(col + full * TILE, full, cnt, off, deg, n, nnz, trow, flags, tile_cnt, s_row, s_warp, ctr);
    }
}

// Rows whose offset equals nnz (trailing empty rows and the sentinel n) get the
// total; a total other than m means the CSR was not symmetric.
__global__ void k_orient_tail(const int64_t *off, int64_t n, int64_t nnz, const int64_t *total_p,
                              int64_t *ooff, int64_t m, unsigned long long *ctr) {
    const int64_t total = *total_p;
    if (blockIdx.x == 0 && threadIdx.x == 0 && total != m) flag_status(ctr, ST_BADGRAPH);
    // first x with off[x] == nnz
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (off[mid] < nnz) lo = mid + 1; else hi = mid;
    }
    for (int64_t x = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= n;
         x += (int64_t)gridDim.x * blockDim.x)
        ooff[x] = total < m ? total : m;
}

inline unsigned grid_for(int64_t work, int threads, int64_t cap = 65536) {
    int64_t g = ceil_div(work > 0 ? work : 1, threads);
    return (unsigned)(g < cap ? g : cap);
}

}  // namespace

int64_t tile_rows_size(int64_t len) { return ceil_div(len > 0 ? len : 1, (int64_t)TILE) + 1; }

cudaError_t launch_tile_rows(const int64_t *off, int64_t n, int64_t len, int32_t *trow, cudaStream_t s) {
    if (n <= 0 || len <= 0) return cudaSuccess;
    // every tile of a valid CSR is written; zeros keep a bad one in range
    cudaError_t e = cudaMemsetAsync(trow, 0, (size_t)tile_rows_size(len) * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    k_tile_rows<<<grid_for(n, 256), 256, 0, s>>>(off, n, ceil_div(len, TILE), trow);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_widen_offsets(const int32_t *in, int64_t count, int64_t *out, cudaStream_t s) {
    k_widen<<<grid_for(count, 256), 256, 0, s>>>(in, count, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_degrees(const int64_t *off, int64_t n, int32_t *deg, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_degrees<<<grid_for(n, 256), 256, 0, s>>>(off, n, deg);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_validate(const int64_t *off, const int32_t *col, int64_t n, int64_t nnz,
                            unsigned long long *ctr, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_validate_rows<<<grid_for(n, 256), 256, 0, s>>>(off, n, nnz, ctr);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // entry checks need sane offsets: the caller syncs and checks between the two
    return cudaSuccess;
}

cudaError_t launch_validate_entries(const int64_t *off, const int32_t *col, int64_t n, int64_t nnz,
                                    const int32_t *trow, unsigned long long *ctr, cudaStream_t s) {
    if (nnz <= 0) return cudaSuccess;
    k_validate_entries<<<(unsigned)ceil_div(nnz, TILE), TILE_THREADS, 0, s>>>(off, col, n, nnz, trow, ctr);
    count_launches(1);
    return cudaGetLastError();
}


template <bool FILL>
cudaError_t launch_orient_pass(const int64_t *off, const int32_t *col, const int32_t *deg, int64_t n, int64_t nnz,
                               const int32_t *trow, uint32_t *flags, int64_t *tile_cnt, const int64_t *tile_base,
                               int64_t *ooff, int32_t *ocol, int32_t *osrc, int64_t m, unsigned long long *ctr,
                               cudaStream_t s) {
    constexpr bool BULK = FILL ? ORIENT_FILL_PERSISTENT != 0 : ORIENT_FLAGS_PERSISTENT != 0;
    unsigned grid = (unsigned)ceil_div(nnz, TILE);
    if (BULK) {
        cudaError_t e = persistent_grid(k_orient_pass<FILL, BULK>, TILE_THREADS, 0, nnz / TILE, &grid);
        if (e != cudaSuccess) return e;
    }
    k_orient_pass<FILL, BULK><<<grid, TILE_THREADS, 0, s>>>(off, col, deg, n, nnz, trow, flags, tile_cnt, tile_base,
                                                            ooff, ocol, osrc, m, ctr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_orient(const int64_t *off, const int32_t *col, const int32_t *deg, int64_t n,
                          int64_t nnz, const int32_t *trow, uint32_t *flags, int64_t *tile_cnt, int64_t *tile_base,
                          int64_t *bsum, int64_t *ooff, int32_t *ocol, int32_t *osrc, int64_t m,
                          unsigned long long *ctr, cudaStream_t s) {
    const int64_t ntiles = ceil_div(nnz, TILE);
    if (((uintptr_t)col | (uintptr_t)flags) % 16 != 0) return cudaErrorInvalidValue;
    if (ntiles > 0) {
        cudaError_t e = launch_orient_pass<false>(off, col, deg, n, nnz, trow, flags, tile_cnt, tile_base, ooff,
                                                  ocol, osrc, m, ctr, s);
        if (e != cudaSuccess) return e;
        e = scan_exclusive_i64(tile_cnt, ntiles, tile_base, bsum, s);
        if (e != cudaSuccess) return e;
        e = launch_orient_pass<true>(off, col, deg, n, nnz, trow, flags, tile_cnt, tile_base, ooff, ocol, osrc,
                                     m, ctr, s);
        if (e != cudaSuccess) return e;
    } else {
        cudaError_t e = scan_exclusive_i64(tile_cnt, 0, tile_base, bsum, s);
        if (e != cudaSuccess) return e;
    }
    k_orient_tail<<<grid_for(n + 1, 256, 1024), 256, 0, s>>>(off, n, nnz, tile_base + ntiles, ooff, m, ctr);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace tec
