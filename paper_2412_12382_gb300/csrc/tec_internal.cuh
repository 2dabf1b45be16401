// Internal declarations of the tectonic library (not part of the C ABI).
//
// Device data layout of one loaded graph (all in HBM, owned by tec_graph):
//   off   int64[n+1]   symmetric CSR row offsets (input copy)
//   col   int32[nnz]   symmetric CSR column ids, rows ascending (input copy)
//   deg   int32[n]     deg(u) = off[u+1] - off[u]
//   ooff  int64[n+1]   oriented CSR offsets: row u holds N+(u) = {v in N(u) : (deg u, u) < (deg v, v)}
//   ocol  int32[m]     oriented column ids, each row still ascending
//   t     uint32[m]    triangle count of oriented edge j (same index as ocol)
//   keep  uint32[ceil(m/32)] keep bit of oriented edge j after the last prune
//   parent int32[n]    union-find forest; parent[x] <= x, roots are component minima
// Every per-edge array is indexed by the oriented position j; exports map it to
// the canonical (u < v, lexicographic) order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tectonic.h"

namespace tec {

// Device status bits (status word in the graph's counter block).
constexpr uint32_t ST_TIMEOUT = 1u;   // a capped loop ran out
constexpr uint32_t ST_BADGRAPH = 2u;  // the CSR violated an invariant

// Counter block layout (unsigned long long each).
enum Ctr : int {
    C_STATUS = 0,
    C_KEPT = 1,
    C_NCOMP = 2,
    C_NWTASK = 3,
    C_NBTASK = 4,
    C_NEXT = 5,
    C_NEXTW = 6,
    C_CHANGED = 7,
    C_NCTASK = 8,       // core block visits
    C_NEXTC = 9,        // next core block visit
    C_NHEAVY = 10,      // core centres whose candidates are tiled by probe-row group
    C_NEXTT = 11,       // next tiled (group, centre) item
    C_DEBUG_LINK_CAP = 12,  // debug builds: 1 + a lowered union-find retry cap (0: the normal cap)
    C_COUNT = 16
};

// Tile of CSR entries handled by one 256-thread block in the streaming passes.
constexpr int TILE_THREADS = 256;
constexpr int TILE_ITEMS = 8;
constexpr int TILE = TILE_THREADS * TILE_ITEMS;   // 2048 entries, a multiple of 32

// Centres with at most this many oriented neighbours are handled by one warp
// in the support kernels; larger ones by a whole block.
constexpr int SMALL_ROW = 32;
// Candidates (probe rows) per support task.
constexpr int64_t TASK_C = 256;

// Retry cap of one union-find link (each retry strictly lowers a root id, so a
// correct run never needs more than n).
constexpr int LINK_RETRY_CAP = 1 << 24;

tec_status set_error(tec_status s, const char *fmt, ...);
void clear_error();

// Process-wide count of kernels this library has launched (tec_launch_count).
void count_launches(int k);

#define TEC_CUDA(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return ::tec::set_error(TEC_ECUDA, "%s failed: %s (%s:%d)", #call,                \
                                    cudaGetErrorString(e_), __FILE__, __LINE__);             \
    } while (0)

#define TEC_TRY(expr)                                                                         \
    do {                                                                                      \
        tec_status s_ = (expr);                                                               \
        if (s_ != TEC_OK) return s_;                                                          \
    } while (0)

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------- launchers
// Each returns cudaGetLastError() of its launches; all run on `s`.

// scan.cu: exclusive prefix sum of `in[0..N)` into `out[0..N]` (out[N] = total).
// `bsum` needs ceil(N / 2048) + 1 entries.
cudaError_t scan_exclusive_i64(const int64_t *in, int64_t N, int64_t *out, int64_t *bsum, cudaStream_t s);
cudaError_t scan_exclusive_i32(const int32_t *in, int64_t N, int64_t *out, int64_t *bsum, cudaStream_t s);
int64_t scan_bsum_size(int64_t N);

// orient.cu
// trow[t] = the row of entry t * TILE (the last r with off[r] <= t * TILE) for
// the ceil(len / TILE) tiles of a CSR with n rows and len entries.
cudaError_t launch_tile_rows(const int64_t *off, int64_t n, int64_t len, int32_t *trow, cudaStream_t s);
int64_t tile_rows_size(int64_t len);
cudaError_t launch_widen_offsets(const int32_t *in, int64_t count, int64_t *out, cudaStream_t s);
cudaError_t launch_degrees(const int64_t *off, int64_t n, int32_t *deg, cudaStream_t s);
cudaError_t launch_validate(const int64_t *off, const int32_t *col, int64_t n, int64_t nnz,
                            unsigned long long *ctr, cudaStream_t s);
cudaError_t launch_validate_entries(const int64_t *off, const int32_t *col, int64_t n, int64_t nnz,
                                    const int32_t *trow, unsigned long long *ctr, cudaStream_t s);
// osrc (m entries, or nullptr) receives the source row of every oriented edge.
// col and flags 16-byte aligned (cudaInvalidValue otherwise).
cudaError_t launch_orient(const int64_t *off, const int32_t *col, const int32_t *deg, int64_t n,
                          int64_t nnz, const int32_t *trow, uint32_t *flags, int64_t *tile_cnt, int64_t *tile_base,
                          int64_t *bsum, int64_t *ooff, int32_t *ocol, int32_t *osrc, int64_t m,
                          unsigned long long *ctr, cudaStream_t s);

// support.cu: t[j] for every oriented edge (zeroed inside).  `flags` are the
// orientation bits of the symmetric entries; `tasks` holds task_cap entries.
int64_t support_task_capacity(int64_t n, int64_t nnz);
// Core labels for the support kernel: degree >= D vertices numbered in id
// order (core_of, -1 otherwise; D the smallest power of two with at most 2^20
// of them, meta = {D, K}) and pv2[j] = core_of[ocol[j]].  hist: 33 entries;
// tcnt / tbase: ceil(n / TILE) entries each; bsum: scan scratch.
cudaError_t launch_core_labels(const int32_t *deg, int64_t n, const int32_t *ocol, int64_t m,
                               unsigned long long *hist, long long *meta, int64_t *tcnt, int64_t *tbase,
                               int64_t *bsum, int32_t *core_of, int32_t *pv2, cudaStream_t s);
// Probe-row tiling of the core centres with the most candidates (support.cu):
// the vertex ids are split into `groups` ranges of about equal oriented-row
// volume, and each such centre is visited once per range that holds some of
// its candidates, all visits of range 0 first, then range 1, ...  The probe
// rows and counters of one range fit in L2, so centres visited at the same
// time share them.  groups = 0: no tiling.
struct SupportTiling {
    int groups = 0;
    int32_t *gb = nullptr;          // groups + 1 range starts (vertex ids)
    int32_t *heavy = nullptr;       // heavy_cap tiled centres
    int64_t heavy_cap = 0;
    int32_t *bu = nullptr;          // (groups + 1) x heavy_cap: first position of each range in N+(c)
    int32_t *bv = nullptr;          // (groups + 1) x heavy_cap: first position of each range in N(c)
    uint32_t *items = nullptr;      // item_cap (range << 20 | heavy index) items, range-major
    int64_t item_cap = 0;
    int64_t *icnt = nullptr;        // groups + 1 items per range, then their prefix (groups + 1)
    int64_t *ioff = nullptr;
    int64_t *bsum = nullptr;        // scan scratch for groups entries
};
// Buffers of the d+ order of the core visits: ORDER_CLASSES + 1 counts and
// offsets, scan scratch, and the reordered visit list (task_cap entries).
struct CoreOrder {
    int64_t *hist = nullptr;
    int64_t *base = nullptr;
    int64_t *bsum = nullptr;
    uint64_t *sorted = nullptr;
};
int64_t core_order_classes();
// Ranges the automatic rule gives a graph of m oriented edges (0: no tiling).
int support_auto_groups(int64_t m);
// Largest number of ranges, and the buffer sizes for a graph of n vertices,
// nnz symmetric entries and `groups` ranges.
constexpr int SUPPORT_MAX_GROUPS = 4095;
int64_t support_heavy_capacity(int64_t n);
int64_t support_item_capacity(int64_t nnz, int groups, int64_t heavy_cap);

// Triangle counts; with pv2 / core_of / ctasks (capacity task_cap) block
// visits of core centres run in the bitmap kernel, and with tiling.groups > 0
// (which needs the core staging) the heaviest core centres are tiled.
cudaError_t launch_support(const int64_t *off, const int32_t *col, const uint32_t *flags, const int64_t *ooff,
                           const int32_t *ocol, int64_t n, int64_t m, uint32_t *t, uint64_t *tasks,
                           int64_t task_cap, unsigned long long *ctr, int num_sms, cudaStream_t s,
                           const int32_t *pv2, const int32_t *core_of, uint64_t *ctasks,
                           const SupportTiling &tiling, const CoreOrder &order);

// prune.cu
struct PruneArgs {
    int measure;
    int64_t p, q;
    bool hook;          // also union the endpoints of every kept edge into `parent`
};
// orows: the tile-row table of the oriented CSR, osrc its per-edge source
// rows (either may be nullptr).
cudaError_t launch_prune(const int64_t *ooff, const int32_t *ocol, const int32_t *deg,
                         const uint32_t *t, int64_t n, int64_t m, const int32_t *orows, const int32_t *osrc,
                         PruneArgs a, uint32_t *keep,
                         int32_t *parent, unsigned long long *ctr, cudaStream_t s);
cudaError_t launch_prune_seg(const int64_t *ooff, const int32_t *ocol, const int32_t *deg, const uint32_t *t,
                             int64_t n, int64_t m, const int32_t *orows, const int32_t *osrc, int measure,
                             const int64_t *sp,
                             const int64_t *sq, const int64_t *seg_off, int nseg, bool hook, uint32_t *keep,
                             int32_t *parent, unsigned long long *ctr, cudaStream_t s);
cudaError_t launch_export(const int64_t *off, const int32_t *col, const int32_t *deg,
                          const int64_t *ooff, const int32_t *ocol, const uint32_t *t,
                          const uint32_t *keep, int64_t n, int64_t nnz, const int64_t *uoff,
                          int32_t *u_out, int32_t *v_out, uint32_t *t_out, uint32_t *wedge_out,
                          double *w_out, int w_measure, uint8_t *keep_out,
                          unsigned long long *ctr, cudaStream_t s);
cudaError_t launch_upper_counts(const int64_t *off, const int32_t *col, int64_t n, int32_t *cnt,
                                cudaStream_t s);

// sweep.cu: levels (number of sorted thresholds each edge survives), Boruvka
// rounds of the maximum spanning forest (forest edges get bit 7 of lvl), the
// level buckets of the forest edges, and one union + snapshot step per level.
// Levels of every edge plus the first Boruvka round (offers into best, which
// must be zero); with lu != nullptr also the live-edge list for later rounds
// (lu, lv, lk with ceil(m / TILE) * TILE entries, rcnt one count per tile).
cudaError_t launch_levels(const int64_t *ooff, const int32_t *ocol, const int32_t *deg, const uint32_t *t,
                          int64_t n, int64_t m, const int32_t *orows, const int32_t *osrc, int measure,
                          const int64_t *tp, const int64_t *tq, int k, bool wide,
                          uint8_t *lvl, unsigned long long *best, int32_t *lu, int32_t *lv, unsigned long long *lk,
                          int32_t *rcnt, unsigned long long *ctr, cudaStream_t s);
// A later Boruvka round's offers: from the live-edge list if lu != nullptr,
// else from the CSR; nothing when *prev_changed is 0 (the forest is complete).
cudaError_t launch_msf_offer(const int64_t *ooff, const int32_t *ocol, uint8_t *lvl, int64_t n, int64_t m,
                             const int32_t *osrc, int32_t *parent, unsigned long long *best, int32_t *lu, int32_t *lv,
                             unsigned long long *lk, int32_t *rcnt, const unsigned long long *prev_changed,
                             unsigned long long *ctr, cudaStream_t s);
// Hooks every root along its heaviest offer, clears the offers and sets
// *changed when a tree grew; nothing when prev_changed is set and 0.
cudaError_t launch_msf_hook(const int64_t *ooff, const int32_t *ocol, const int32_t *osrc, uint8_t *lvl, int64_t n,
                            int32_t *parent,
                            unsigned long long *best, const unsigned long long *prev_changed,
                            unsigned long long *changed, unsigned long long *ctr, cudaStream_t s);
// Flags TEC_ETIMEOUT if the last allowed round still grew the forest.
cudaError_t launch_msf_check(const unsigned long long *last_changed, unsigned long long *ctr, cudaStream_t s);
// Stores count int64 values (sorted p then q) to dst from the launch parameters.
cudaError_t launch_store_thresholds(const int64_t *sorted_pq, int count, int64_t *dst, cudaStream_t s);
cudaError_t launch_forest_buckets(const int64_t *ooff, const int32_t *ocol, const uint8_t *lvl, int64_t n, int64_t m,
                                  const int32_t *orows, const int32_t *osrc, int k, unsigned long long *bucket, int32_t *fu, int32_t *fv, unsigned long long *ctr,
                                  cudaStream_t s);
// Unions level L's bucket (bounds read on the device), then snapshots the labels.
cudaError_t launch_sweep_level(const int32_t *fu, const int32_t *fv, const unsigned long long *bucket, int k, int L,
                               int64_t n, int32_t *parent, int32_t *labels, const int64_t *seg_off, int nseg,
                               unsigned long long *ncomp, unsigned long long *ctr, cudaStream_t s);

cudaError_t launch_snapshot(int32_t *parent, int64_t n, int32_t *labels, const int64_t *seg_off, int nseg,
                            unsigned long long *ncomp, cudaStream_t s);

// eval.cu: picker features per graph and adjusted Rand index per (level, graph).
cudaError_t launch_features(const int64_t *ooff, const int32_t *ocol, const int32_t *deg, const uint32_t *t,
                            int64_t n, int64_t m, const int32_t *orows, const int32_t *osrc, const int64_t *seg_off,
                            int nseg, unsigned int *hist, float *feat, unsigned long long *ctr, cudaStream_t s);
int ari_table_bits(int64_t n);
cudaError_t launch_best_level(const double *ari, int k, int nseg, int32_t *best, double *best_ari, cudaStream_t s);
// ARI_CHUNK levels share one zeroing of the pair sums (sums holds 2 x nseg x ARI_CHUNK).
constexpr int ARI_CHUNK = 64;
// size holds two arrays of size_len >= n counters used in turn (by the
// parity of the level tag); keys / cnt (tsize = 2^ari_table_bits(n_cap)
// slots) are level-tagged.  *tag advances by one per level; a *tag of
// ~0 (or one about to wrap) zeroes all three first.
cudaError_t launch_ari(const int32_t *labels, int k, const int32_t *truth, int64_t n, const int64_t *seg_off, int nseg,
                       unsigned int *bsz, unsigned int *size, int64_t size_len, unsigned long long *keys,
                       unsigned long long *cnt, int64_t tsize, unsigned long long *sums, double *out,
                       unsigned long long *tag, unsigned long long *ctr, cudaStream_t s);

// stats.cu: sweep statistics (thresholds sorted ascending in tp/tq, order[i]
// = row of the i-th; hist 2 (k+1) per graph, sums 3 per row and graph,
// cnt_n / cnt_v two arrays of cnt_len >= n each).
cudaError_t launch_sweep_stats(const int64_t *ooff, const int32_t *ocol, const int32_t *deg, const uint32_t *t,
                               int64_t n, int64_t m, const int32_t *orows, const int32_t *osrc, int measure, const int64_t *tp, const int64_t *tq, int k,
                               const int *order, bool wide, const int32_t *labels, const int64_t *seg_off, int nseg,
                               unsigned long long *hist, unsigned int *cnt_n, unsigned long long *cnt_v,
                               int64_t cnt_len, unsigned long long *sums, tec_sweep_stat *out,
                               unsigned long long *ctr, cudaStream_t s);
cudaError_t launch_rules(const tec_sweep_stat *stats, int k, int nseg, const int *order, int rule, int32_t *best,
                         cudaStream_t s);

// k4.cu: K4 participation per oriented edge (t = triangle counts, next = one
// work counter), saturating at 2^32 - 1.
cudaError_t launch_k4(const int64_t *off, const int32_t *col, const int64_t *ooff, const int32_t *ocol,
                      const uint32_t *t, int64_t n, int64_t m, unsigned long long *next, uint32_t *k4,
                      unsigned long long *ctr, int num_sms, cudaStream_t s);

// P/R/F1 of Sec. IV-A (shares the ARI counters, tables and tag; best / bestb:
// n each; scratch_sums: 2 x nseg; sums: 3 x nseg x ARI_CHUNK; out: k x nseg x 3).
cudaError_t launch_prf(const int32_t *labels, int k, const int32_t *truth, int64_t n, const int64_t *seg_off, int nseg,
                       unsigned int *bsz, unsigned int *size, int64_t size_len, unsigned long long *keys,
                       unsigned long long *cnt, int64_t tsize, unsigned long long *scratch_sums,
                       unsigned long long *best, unsigned int *bestb, unsigned long long *sums, double *out,
                       unsigned long long *tag, unsigned long long *ctr, cudaStream_t s);

// cc.cu
cudaError_t launch_cc_init(int32_t *parent, int64_t n, cudaStream_t s);
cudaError_t launch_cc_hook(const int64_t *ooff, const int32_t *ocol, const uint32_t *keep,
                           int64_t n, int64_t m, const int32_t *orows, const int32_t *osrc, int32_t *parent,
                           unsigned long long *ctr, cudaStream_t s);
cudaError_t launch_cc_finish(int32_t *parent, int64_t n, int32_t *labels,
                             unsigned long long *ctr, cudaStream_t s);

// ---------------------------------------------------------------- device helpers

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ int warp_sum(int x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Segment of vertex x (the last s with seg_off[s] <= x) for lanes that hold
// x = x0 + lane with x0 warp-uniform: every lane runs the same binary search
// for x0 (broadcast loads), then walks forward over at most 31 segment starts.
__device__ __forceinline__ int warp_seg_of(const int64_t *seg_off, int nseg, int64_t x0, int64_t x) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg_off[mid] <= x0) lo = mid; else hi = mid - 1;
    }
    while (lo + 1 < nseg && seg_off[lo + 1] <= x) ++lo;
    return lo;
}

// Vertex passes (snapshot, ARI) hand each warp chunks of VCHUNK_V x 32
// consecutive vertices: one segment lookup per chunk, VCHUNK_V independent
// loads in flight per lane.
constexpr int VCHUNK_V = 4;
constexpr int VCHUNK = 32 * VCHUNK_V;

// Grid for a persistent vertex pass of 256-thread blocks: enough warps for
// every chunk, at most 16 blocks per SM.
unsigned vertex_pass_grid(int64_t n);

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Groups the valid lanes of a warp by key for one atomic per group: returns
// a mask of lanes that hold this lane's key (the lane itself at least).  Any
// grouping by equal keys is exact, because every group computes its pair
// increment from the count its own atomic returns; so the full (slow) match
// runs only when neighbouring lanes repeat keys often.  All keys equal
// (a large component over consecutive vertices) costs one shuffle; mostly
// distinct keys (singletons, interleaved components) add lane by lane.
template <typename K>
__device__ __forceinline__ unsigned key_group(bool valid, K key) {
    const unsigned lane = lane_id();
    const unsigned vm = __ballot_sync(0xffffffffu, valid);
    if (!vm) return 0u;
    const K k0 = __shfl_sync(0xffffffffu, key, __ffs(vm) - 1);
    if (__all_sync(0xffffffffu, !valid || key == k0)) return vm;
    const K up = __shfl_up_sync(0xffffffffu, key, 1);
    const bool rep = valid && lane > 0 && ((vm >> (lane - 1)) & 1u) && key == up;
    if (__popc(__ballot_sync(0xffffffffu, rep)) >= 8) return __match_any_sync(0xffffffffu, key) & vm;
    return 1u << lane;
}

// Largest r in [lo, hi] with off[r] <= k (off non-decreasing, off[lo] <= k).
__device__ __forceinline__ int64_t row_search(const int64_t *off, int64_t lo, int64_t hi, int64_t k) {
    while (lo < hi) {
        int64_t mid = lo + (hi - lo + 1) / 2;
        if (off[mid] <= k) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Rows of tile `tile` (entries [tile * TILE, + TILE) of a CSR with `len`
// entries): r0 = the row of its first entry, r1 >= the row of its last.
// From the tile-row table trow of launch_tile_rows when given (two loads),
// else by binary search over all n rows.
__device__ __forceinline__ void tile_row_range(const int32_t *trow, const int64_t *off, int64_t n, int64_t len,
                                               int64_t tile, int64_t &r0, int64_t &r1) {
    const int64_t k0 = tile * TILE;
    if (trow) {
        r0 = trow[tile];
        r0 = r0 < 0 ? 0 : (r0 > n - 1 ? n - 1 : r0);      // in range even for a bad CSR
        // the last tile ends at the row of the last entry, not at the trailing empty rows
        r1 = k0 + TILE < len ? (int64_t)trow[tile + 1] : row_search(off, r0, n - 1, len - 1);
        r1 = r1 < r0 ? r0 : (r1 > n - 1 ? n - 1 : r1);
    } else {
        const int64_t klast = (k0 + TILE < len ? k0 + TILE : len) - 1;
        r0 = row_search(off, 0, n - 1, k0);
        r1 = row_search(off, r0, n - 1, klast);
    }
}

__device__ __forceinline__ void tile_row_range(const int32_t *trow, const int64_t *off, int64_t n, int64_t len,
                                               int64_t &r0, int64_t &r1) {
    tile_row_range(trow, off, n, len, (int64_t)blockIdx.x, r0, r1);
}

constexpr int64_t ROW_MARK_CAP = 4 * TILE;

// Row of every entry of tile `tile`, into shared memory: s_row[p] =
// row(k0 + p) - r0 for p < TILE, where row(k) is the last nonempty row whose
// first entry is at or before k and r0 = row(k0) (tile_row_range).  Each
// nonempty row of [r0 + 1, r1] marks its first entry, then a block-wide
// running maximum spreads the marks (marks grow with position), so the rows
// are read once, coalesced, instead of one binary search per entry (kept for
// tiles spanning more than ROW_MARK_CAP rows, i.e. long runs of empty rows).  Every
// write stays in s_row whatever off holds, and every result lies in
// [0, r1 - r0].  Needs blockDim.x == TILE_THREADS, s_row 16-byte aligned,
// s_warp of TILE_THREADS / 32 ints; ends with __syncthreads().
__device__ __forceinline__ void tile_entry_rows(const int64_t *__restrict__ off, int64_t len, int64_t tile, int64_t r0,
                                                int64_t r1, int32_t *s_row, int32_t *s_warp) {
    const int64_t k0 = tile * TILE;
    const int64_t k1 = k0 + TILE < len ? k0 + TILE : len;
    if (r1 - r0 > ROW_MARK_CAP) {          // a long run of empty rows: search per entry
        for (int p = threadIdx.x; p < TILE; p += TILE_THREADS)
            s_row[p] = k0 + p < k1 ? (int32_t)(row_search(off, r0, r1, k0 + p) - r0) : 0;
        __syncthreads();
        return;
    }
    for (int p = threadIdx.x; p < TILE; p += TILE_THREADS) s_row[p] = 0;
    __syncthreads();
    for (int64_t r = r0 + 1 + threadIdx.x; r <= r1; r += TILE_THREADS) {
        const int64_t a = off[r];
        if (a >= k0 && a < k1 && a < off[r + 1]) s_row[a - k0] = (int32_t)(r - r0);
    }
    __syncthreads();
    static_assert(TILE_ITEMS == 8, "two int4 per thread");
    int4 *s4 = reinterpret_cast<int4 *>(s_row) + 2 * threadIdx.x;
    int4 a = s4[0], b = s4[1];
    a.y = max(a.y, a.x); a.z = max(a.z, a.y); a.w = max(a.w, a.z);
    b.x = max(b.x, a.w); b.y = max(b.y, b.x); b.z = max(b.z, b.y); b.w = max(b.w, b.z);
    const unsigned lane = threadIdx.x & 31u;
    int32_t inc = b.w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t x = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= (unsigned)d) inc = max(inc, x);
    }
    int32_t pre = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) pre = 0;
    if (lane == 31) s_warp[threadIdx.x >> 5] = inc;
    __syncthreads();
    for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) pre = max(pre, s_warp[w]);
    a.x = max(a.x, pre); a.y = max(a.y, pre); a.z = max(a.z, pre); a.w = max(a.w, pre);
    b.x = max(b.x, pre); b.y = max(b.y, pre); b.z = max(b.z, pre); b.w = max(b.w, pre);
    s4[0] = a;
    s4[1] = b;
    __syncthreads();
}

// Source row of oriented edge j: from the per-edge source table osrc when
// given (one coalesced load), else by binary search over the tile's rows.
__device__ __forceinline__ int64_t edge_source(const int32_t *osrc, const int64_t *ooff, int64_t r0, int64_t r1,
                                               int64_t j) {
    return osrc ? (int64_t)__ldg(&osrc[j]) : row_search(ooff, r0, r1, j);
}

// Orientation order: u before v iff (deg u, u) < (deg v, v).
__device__ __forceinline__ bool rank_less(int32_t du, int64_t u, int32_t dv, int64_t v) {
    return du < dv || (du == dv && u < v);
}

// Algorithm 1's survival test sim(e) >= p/q in exact integers, given
// t = t(u,v) and s = deg u + deg v (q > 0):
//   Tectonic (Table 1): t*q >= p*s;   TW (Eq. 1): (3t + 2 - s)*q >= p;
//   Jaccard (Table 1): t*q >= p*(s - t), s - t = |N(u) u N(v)| > 0;
//   K3 (Table 1): t*q >= p.
// All products fit int64 when |p|, q < 2^28; WIDE uses 128-bit products.
template <bool WIDE>
__device__ __forceinline__ bool keep_edge(int measure, uint32_t tt, int64_t s, int64_t p, int64_t q) {
    if (measure == TEC_TECTONIC) {
        if (WIDE) return (__int128)tt * q >= (__int128)p * s;
        return (int64_t)tt * q >= p * s;
    }
    if (measure == TEC_JACCARD) {
        const int64_t uni = s - (int64_t)tt;
        if (WIDE) return (__int128)tt * q >= (__int128)p * uni;
        return (int64_t)tt * q >= p * uni;
    }
    if (measure == TEC_K3) {
        if (WIDE) return (__int128)tt * q >= (__int128)p;
        return (int64_t)tt * q >= p;
    }
    const int64_t tw = 3 * (int64_t)tt + 2 - s;
    if (WIDE) return (__int128)tw * q >= (__int128)p;
    return tw * q >= p;
}

__device__ __forceinline__ bool needs_wide_dev(int64_t p, int64_t q) {
    const int64_t lim = (int64_t)1 << 28;
    return !(p > -lim && p < lim && q < lim);
}

inline bool needs_wide(int64_t p, int64_t q) {
    const int64_t lim = (int64_t)1 << 28;
    return !(p > -lim && p < lim && q < lim);
}

__device__ __forceinline__ void flag_status(unsigned long long *ctr, uint32_t bit) {
    atomicOr(&ctr[C_STATUS], (unsigned long long)bit);
}

__device__ __forceinline__ bool graph_bad(const unsigned long long *ctr) {
    return (*(volatile const unsigned long long *)&ctr[C_STATUS] & ST_BADGRAPH) != 0;
}

}  // namespace tec

// The opaque handle of the C ABI.
struct tec_graph {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    int64_t n_cap = 0, nnz_cap = 0, m_cap = 0;
    int64_t n = 0, nnz = 0, m = 0;

    int64_t *off = nullptr;
    int32_t *col = nullptr;
    int32_t *deg = nullptr;
    int64_t *ooff = nullptr;
    int32_t *ocol = nullptr;
    uint32_t *t = nullptr;
    uint32_t *keep = nullptr;
    int32_t *parent = nullptr;
    uint64_t *tasks = nullptr;      // support work list
    int64_t task_cap = 0;
    uint32_t *flags = nullptr;
    int32_t *sym_rows = nullptr;    // tile-row table of the symmetric CSR
    int32_t *or_rows = nullptr;     // tile-row table of the oriented CSR
    int32_t *osrc = nullptr;        // m: source row of every oriented edge (written by the orientation)
    int64_t *tile_cnt = nullptr;
    int64_t *tile_base = nullptr;
    int64_t *bsum = nullptr;
    int64_t *uoff = nullptr;        // export only, allocated on first export
    int32_t *ucnt = nullptr;        // export only
    int32_t *labels = nullptr;      // host-buffer pass only, allocated on first use
    // sweep scratch, allocated on first sweep
    uint8_t *lvl = nullptr;         // m: level of each oriented edge, bit 7 = forest edge
    unsigned long long *best = nullptr;   // n: Boruvka offers
    int32_t *msf_u = nullptr, *msf_v = nullptr;  // live-edge list: tree roots of both ends
    unsigned long long *msf_k = nullptr;  // live-edge list: edge keys
    int32_t *msf_cnt = nullptr;           // live entries per tile region
    int64_t msf_cap = 0;                  // entries allocated (0: no list, rounds rescan the CSR)
    // core staging of the support kernel (optional: without it all block visits hash)
    int32_t *core_of = nullptr;           // n: core code or -1
    int32_t *pv2 = nullptr;               // m + 4: core codes of ocol
    uint64_t *ctasks = nullptr;           // task_cap core block visits
    tec::CoreOrder corder;                // the core visits reordered by out-degree (optional)
    int64_t *core_tc = nullptr;           // 2 x ceil(n_cap / TILE) + 64: tile counts and bases
    unsigned long long *core_hist = nullptr;  // 33 degree bins + 2 meta words
    int core_state = 0;                   // 0 untried, 1 available, -1 unavailable
    bool core_enabled = true;             // tec_set_core_staging
    // probe-row tiling of the heaviest core centres (buffers for tile.groups ranges)
    tec::SupportTiling tile;
    int tile_request = 0;                 // tec_set_support_tiling: 0 automatic, -1 off, > 0 ranges
    int tile_failed_groups = 0;           // range count whose buffers could not be allocated
    // K4 participation per oriented edge (saturating), allocated on first use
    uint32_t *k4 = nullptr;
    unsigned long long *k4_next = nullptr;
    unsigned long long support_epoch = 0; // bumped whenever the triangle counts are recomputed
    unsigned long long k4_epoch = ~0ull;  // support_epoch the K4 counts belong to
    unsigned long long *msf_changed = nullptr;  // 64 per-round "a tree grew" flags
    int32_t *fu = nullptr, *fv = nullptr; // n: forest edges bucketed by level
    unsigned long long *bucket = nullptr; // 3k+4 bucket counts / offsets / cursors
    int64_t *thr = nullptr;         // 2 * 128 sorted thresholds (p then q)
    unsigned long long *sw_ncomp = nullptr;  // components per level and segment
    int64_t sw_ncomp_cap = 0;
    // features / ARI scratch, grown on demand
    unsigned int *seg_hist = nullptr;      // nseg x 64 (histogram, block sizes)
    int64_t seg_cap = 0;
    unsigned long long *ari_sums = nullptr; // 2 x nseg x ARI_CHUNK pair sums
    unsigned int *ari_size = nullptr;      // 2 x n_cap component sizes (two levels in turn)
    int64_t ari_n = -1;                     // vertex count the ARI counters were last used with
    unsigned long long *ari_keys = nullptr; // 2^bits level-tagged cell keys
    unsigned long long *ari_cnt = nullptr;  // 2^bits level-tagged cell counts
    unsigned long long ari_tag = 0;         // last level tag used in the arrays above
    // P/R/F1 scratch
    unsigned long long *prf_best = nullptr;     // n_cap best Jaccard bits per root
    unsigned int *prf_bestb = nullptr;          // n_cap matched block per root
    unsigned long long *prf_sums = nullptr;     // 3 x nseg x ARI_CHUNK
    int64_t prf_sums_cap = 0;
    // sweep statistics scratch, grown on demand
    unsigned long long *st_hist = nullptr;  // nseg x 2 (k + 1) level / join-level histograms
    int64_t st_hist_cap = 0;
    unsigned long long *st_sums = nullptr;  // k x nseg x 3 root counts, maxima, squared volumes
    int64_t st_sums_cap = 0;
    unsigned int *st_cnt_n = nullptr;       // 2 x n_cap vertices per root (two levels in turn)
    unsigned long long *st_cnt_v = nullptr; // 2 x n_cap degree volume per root
    unsigned long long *ctr = nullptr;      // device counter block
    unsigned long long *ctr_host = nullptr; // pinned mirror for reads

    // pipeline state
    bool oriented = false;
    bool supported = false;
    bool pruned = false;
    bool hooked = false;            // parent already holds the kept-edge forest
    bool uoff_valid = false;
    cudaEvent_t stage_ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int n_stage_ev = 0;
    int last_measure = 0;
    int64_t last_p = 0, last_q = 1;
};
