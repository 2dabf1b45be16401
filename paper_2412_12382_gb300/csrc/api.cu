// C ABI entry points (include/tectonic.h): argument checks, graph memory,
// step ordering and status reporting.  All device work is in the kernels of
// the other .cu files (orientation, triangle counts, K4, pruning, components,
// sweep, statistics, evaluation, picker).
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <algorithm>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "tec_internal.cuh"

namespace tec {

// Names the host-side span of an entry point for profilers (Nsight can then
// select the kernels one call launched).  Without a tool attached NVTX calls
// return at once.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define TEC_RANGE() ::tec::NvtxRange tec_nvtx_range_(__func__)

static thread_local char g_err[1024];

tec_status set_error(tec_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

void clear_error() { g_err[0] = '\0'; }

static std::atomic<long long> g_launches{0};
void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

namespace {

constexpr int64_t MAX_N = ((int64_t)1 << 31) - 1;
constexpr int64_t THRESH_LIMIT = (int64_t)1 << 62;

// Makes the graph's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

#ifdef TEC_DEBUG
// Debug builds (-DTEC_DEBUG): every graph-owned device buffer is followed by
// CANARY_BYTES bytes of 0xA5, and tec_sync checks them all; a kernel that
// wrote past the end of a buffer is reported with the buffer's name.  This
// stands in for a memory checker where none can be run.
constexpr size_t CANARY_BYTES = 256;
constexpr unsigned char CANARY = 0xA5;
struct CanaryEntry {
    void *p;
    size_t bytes;
    const char *what;
};
std::mutex g_canary_mu;
std::vector<CanaryEntry> g_canaries;

tec_status check_canaries() {
    TEC_CUDA(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> lock(g_canary_mu);
    std::vector<unsigned char> h(CANARY_BYTES);
    for (const CanaryEntry &c : g_canaries) {
        TEC_CUDA(cudaMemcpy(h.data(), (char *)c.p + c.bytes, CANARY_BYTES, cudaMemcpyDeviceToHost));
        for (unsigned char v : h)
            if (v != CANARY)
                return set_error(TEC_ECUDA, "debug build: the %zu bytes after %s (%zu bytes) were overwritten",
                                 CANARY_BYTES, c.what, c.bytes);
    }
    return TEC_OK;
}

// Lowered iteration caps: TEC_DEBUG_LINK_CAP=<k> allows every union-find
// link k retries (0: a link between two different roots gives up at once),
// TEC_DEBUG_MSF_ROUNDS=<r> at most r Boruvka rounds in a sweep.  Both are read
// again by every call that runs the union-find, so a test can lower a cap,
// see TEC_ETIMEOUT, restore it and call again on the same graph.
tec_status debug_refresh_caps(tec_graph *g) {
    const char *s = getenv("TEC_DEBUG_LINK_CAP");
    const unsigned long long v = (s && *s) ? std::strtoull(s, nullptr, 10) + 1ull : 0ull;
    TEC_CUDA(cudaMemcpy(&g->ctr[C_DEBUG_LINK_CAP], &v, sizeof(v), cudaMemcpyHostToDevice));
    return TEC_OK;
}

int debug_msf_rounds(int rounds) {
    const char *s = getenv("TEC_DEBUG_MSF_ROUNDS");
    if (!s || !*s) return rounds;
    const long r = std::strtol(s, nullptr, 10);
    return r >= 1 && r < rounds ? (int)r : rounds;
}

// Failure injection: with TEC_DEBUG_FAIL_ALLOC set, every allocation whose
// name contains that text fails as if the device were out of memory, so the
// fallback and retry paths can be driven on purpose.
bool injected_alloc_failure(const char *what) {
    const char *pat = getenv("TEC_DEBUG_FAIL_ALLOC");
    return pat && *pat && strstr(what, pat) != nullptr;
}
#else
inline tec_status debug_refresh_caps(tec_graph *) { return TEC_OK; }
inline int debug_msf_rounds(int rounds) { return rounds; }
#endif

template <typename T>
tec_status dalloc(T **p, int64_t count, const char *what) {
    *p = nullptr;
    size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
#ifdef TEC_DEBUG
    if (injected_alloc_failure(what))
        return set_error(TEC_ENOMEM, "cudaMalloc of %zu bytes for %s failed: injected by TEC_DEBUG_FAIL_ALLOC",
                         bytes, what);
    cudaError_t e = cudaMalloc((void **)p, bytes + CANARY_BYTES);
    if (e == cudaSuccess) e = cudaMemset((char *)*p + bytes, CANARY, CANARY_BYTES);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lock(g_canary_mu);
        g_canaries.push_back({(void *)*p, bytes, what});
    } else if (*p) {
        cudaFree(*p);
    }
#else
    cudaError_t e = cudaMalloc((void **)p, bytes);
#endif
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(e == cudaErrorMemoryAllocation ? TEC_ENOMEM : TEC_ECUDA,
                         "cudaMalloc of %zu bytes for %s failed: %s", bytes, what, cudaGetErrorString(e));
    }
    return TEC_OK;
}

// Frees a buffer from dalloc (NULL is ignored).
void dfree(void *p) {
    if (!p) return;
#ifdef TEC_DEBUG
    {
        std::lock_guard<std::mutex> lock(g_canary_mu);
        for (size_t i = 0; i < g_canaries.size(); ++i)
            if (g_canaries[i].p == p) {
                g_canaries.erase(g_canaries.begin() + (long)i);
                break;
            }
    }
#endif
    cudaFree(p);
}

void free_tiling(tec_graph *g) {
    SupportTiling &t = g->tile;
    void *ptrs[] = {t.gb, t.heavy, t.bu, t.bv, t.items, t.icnt, t.ioff, t.bsum};
    for (void *p : ptrs) dfree(p);
    t = SupportTiling();
}

// Buffers of the probe-row tiling for `groups` ranges; false (tiling off for
// this count, no error) when they cannot be allocated.
bool ensure_tiling(tec_graph *g, int groups) {
    if (g->tile.groups == groups && g->tile.items) return true;
    if (g->tile_failed_groups == groups) return false;
    free_tiling(g);
    SupportTiling t;
    t.groups = groups;
    t.heavy_cap = support_heavy_capacity(g->n_cap);
    t.item_cap = support_item_capacity(g->nnz_cap, groups, t.heavy_cap);
    const int64_t bsz = (int64_t)(groups + 1) * t.heavy_cap;
    if (dalloc(&t.gb, groups + 1, "tiling ranges") != TEC_OK || dalloc(&t.heavy, t.heavy_cap, "tiling centres") != TEC_OK ||
        dalloc(&t.bu, bsz, "tiling row bounds") != TEC_OK || dalloc(&t.bv, bsz, "tiling row bounds") != TEC_OK ||
        dalloc(&t.items, t.item_cap, "tiling items") != TEC_OK || dalloc(&t.icnt, groups + 1, "tiling counts") != TEC_OK ||
        dalloc(&t.ioff, groups + 1, "tiling counts") != TEC_OK ||
        dalloc(&t.bsum, scan_bsum_size(groups), "tiling counts") != TEC_OK) {
        g->tile = t;
        free_tiling(g);
        g->tile_failed_groups = groups;
        clear_error();
        return false;
    }
    g->tile = t;
    return true;
}

void free_graph_memory(tec_graph *g) {
    void *ptrs[] = {g->off, g->col, g->deg, g->ooff, g->ocol, g->t, g->keep, g->parent, g->tasks, g->sym_rows, g->or_rows, g->osrc,
                    g->flags, g->tile_cnt, g->tile_base, g->bsum, g->uoff, g->ucnt, g->labels, g->lvl, g->best,
                    g->fu, g->fv, g->bucket, g->thr, g->sw_ncomp, g->seg_hist, g->ari_sums,
                    g->ari_size, g->ari_keys, g->ari_cnt, g->msf_u, g->msf_v, g->msf_k, g->msf_cnt, g->msf_changed,
                    g->core_of, g->pv2, g->ctasks, g->core_tc, g->core_hist, g->k4, g->k4_next,
                    g->prf_best, g->prf_bestb, g->prf_sums,
                    g->st_hist, g->st_sums, g->st_cnt_n, g->st_cnt_v, g->ctr};
    for (void *p : ptrs) dfree(p);
    free_tiling(g);
    void *order[] = {g->corder.hist, g->corder.base, g->corder.bsum, g->corder.sorted};
    for (void *p : order) dfree(p);
    g->corder = CoreOrder();
    if (g->ctr_host) cudaFreeHost(g->ctr_host);
}

// Copies the counter block to the host and turns status bits into an error.
tec_status read_counters(tec_graph *g) {
    TEC_CUDA(cudaMemcpyAsync(g->ctr_host, g->ctr, C_COUNT * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, g->stream));
    TEC_CUDA(cudaStreamSynchronize(g->stream));
    const unsigned long long st = g->ctr_host[C_STATUS];
    if (st) {
        TEC_CUDA(cudaMemsetAsync(&g->ctr[C_STATUS], 0, sizeof(unsigned long long), g->stream));
        TEC_CUDA(cudaStreamSynchronize(g->stream));
        if (st & ST_BADGRAPH) {
            g->oriented = g->supported = g->pruned = g->hooked = false;
            return set_error(TEC_EBADGRAPH, "invalid input on the device: a CSR that is not a simple undirected graph "
                                            "with sorted rows, or a label or block id out of range");
        }
        g->pruned = g->hooked = false;
        return set_error(TEC_ETIMEOUT, "a bounded device loop reached its iteration cap");
    }
    return TEC_OK;
}

tec_status reset_counter(tec_graph *g, int which) {
    TEC_CUDA(cudaMemsetAsync(&g->ctr[which], 0, sizeof(unsigned long long), g->stream));
    return TEC_OK;
}

tec_status ensure_oriented(tec_graph *g) {
    if (g->oriented) return TEC_OK;
    TEC_CUDA(launch_orient(g->off, g->col, g->deg, g->n, g->nnz, g->sym_rows, g->flags, g->tile_cnt, g->tile_base,
                           g->bsum, g->ooff, g->ocol, g->osrc, g->m, g->ctr, g->stream));
    TEC_CUDA(launch_tile_rows(g->ooff, g->n, g->m, g->or_rows, g->stream));
    g->oriented = true;
    g->supported = g->pruned = g->hooked = false;
    return TEC_OK;
}

tec_status ensure_support(tec_graph *g) {
    TEC_TRY(ensure_oriented(g));
    if (g->supported) return TEC_OK;
    // core staging buffers: allocated once; without the memory the bitmap
    // kernel is skipped and every block visit uses the hashed staging
    if (g->core_state == 0 && g->core_enabled) {
        const int64_t tiles = ceil_div(std::max<int64_t>(g->n_cap, 1), (int64_t)TILE);
        if (dalloc(&g->core_of, std::max<int64_t>(g->n_cap, 1), "core codes") != TEC_OK ||
            dalloc(&g->pv2, g->m_cap + 4, "core-coded columns") != TEC_OK ||
            dalloc(&g->ctasks, g->task_cap, "core visits") != TEC_OK ||
            dalloc(&g->core_tc, 2 * tiles + 64, "core tile counts") != TEC_OK ||
            dalloc(&g->core_hist, 36, "degree histogram") != TEC_OK) {
            void *part[] = {g->core_of, g->pv2, g->ctasks, g->core_tc, g->core_hist};
            for (void *q2 : part) dfree(q2);
            g->core_of = nullptr;
            g->pv2 = nullptr;
            g->ctasks = nullptr;
            g->core_tc = nullptr;
            g->core_hist = nullptr;
            g->core_state = -1;
            clear_error();
        } else {
            g->core_state = 1;
            // optional: the visit order by out-degree (without it, the visits run as emitted)
            const int64_t oc = core_order_classes();
            CoreOrder o;
            if (oc > 0 && (dalloc(&o.hist, oc + 1, "core visit order") != TEC_OK ||
                           dalloc(&o.base, oc + 1, "core visit order") != TEC_OK ||
                           dalloc(&o.bsum, scan_bsum_size(oc), "core visit order") != TEC_OK ||
                           dalloc(&o.sorted, g->task_cap, "core visit order") != TEC_OK)) {
                void *part[] = {o.hist, o.base, o.bsum, o.sorted};
                for (void *q2 : part) dfree(q2);
                o = CoreOrder();
                clear_error();
            }
            g->corder = o;
        }
    }
    const bool core = g->core_state > 0 && g->core_enabled;
    if (core) {
        const int64_t tiles = ceil_div(std::max<int64_t>(g->n, 1), (int64_t)TILE);
        TEC_CUDA(launch_core_labels(g->deg, g->n, g->ocol, g->m, g->core_hist,
                                    reinterpret_cast<long long *>(g->core_hist + 33), g->core_tc,
                                    g->core_tc + tiles + 32, g->bsum, g->core_of, g->pv2, g->stream));
    }
    // probe-row tiling (needs the core staging): automatic range count unless set
    int groups = g->tile_request < 0 ? 0 : g->tile_request > 0 ? g->tile_request : support_auto_groups(g->m);
    if (!core || (groups > 0 && !ensure_tiling(g, groups))) groups = 0;
    SupportTiling tl = g->tile;
    if (!groups) tl.groups = 0;
    TEC_CUDA(launch_support(g->off, g->col, g->flags, g->ooff, g->ocol, g->n, g->m, g->t, g->tasks, g->task_cap,
                            g->ctr, g->num_sms, g->stream, core ? g->pv2 : nullptr, core ? g->core_of : nullptr,
                            core ? g->ctasks : nullptr, tl, g->corder));
    ++g->support_epoch;
    g->supported = true;
    g->pruned = g->hooked = false;
    return TEC_OK;
}

// K4 participation of the current triangle counts.
tec_status ensure_k4(tec_graph *g) {
    TEC_TRY(ensure_support(g));
    if (g->k4 && g->k4_epoch == g->support_epoch) return TEC_OK;
    if (!g->k4) TEC_TRY(dalloc(&g->k4, std::max<int64_t>(g->m_cap, 1), "K4 counts"));
    if (!g->k4_next) TEC_TRY(dalloc(&g->k4_next, 1, "K4 work counter"));
    TEC_CUDA(launch_k4(g->off, g->col, g->ooff, g->ocol, g->t, g->n, g->m, g->k4_next, g->k4, g->ctr, g->num_sms,
                       g->stream));
    g->k4_epoch = g->support_epoch;
    return TEC_OK;
}

// The per-edge counts a measure compares and the comparison it uses: K4 is the
// K3 test on the K4 counts; every other measure works on the triangle counts.
tec_status measure_counts(tec_graph *g, int measure, const uint32_t **counts, int *cmp) {
    if (measure == TEC_K4) {
        TEC_TRY(ensure_k4(g));
        *counts = g->k4;
        *cmp = TEC_K3;
    } else {
        TEC_TRY(ensure_support(g));
        *counts = g->t;
        *cmp = measure;
    }
    return TEC_OK;
}

tec_status ensure_uoff(tec_graph *g) {
    if (g->uoff_valid) return TEC_OK;
    if (!g->uoff) TEC_TRY(dalloc(&g->uoff, g->n_cap + 1, "canonical row offsets"));
    if (!g->ucnt) TEC_TRY(dalloc(&g->ucnt, g->n_cap, "canonical row counts"));
    TEC_CUDA(launch_upper_counts(g->off, g->col, g->n, g->ucnt, g->stream));
    TEC_CUDA(scan_exclusive_i32(g->ucnt, g->n, g->uoff, g->bsum, g->stream));
    g->uoff_valid = true;
    return TEC_OK;
}

tec_status check_threshold(int measure, int64_t p, int64_t q) {
    if (measure < TEC_TECTONIC || measure > TEC_K4) return set_error(TEC_EINVAL, "unknown measure %d", measure);
    if (q <= 0) return set_error(TEC_EINVAL, "threshold denominator q must be positive (got %lld)", (long long)q);
    if (q >= THRESH_LIMIT || p >= THRESH_LIMIT || p <= -THRESH_LIMIT)
        return set_error(TEC_EOVERFLOW, "|p| and q must be below 2^62");
    // K4 counts saturate at 2^32 - 1: comparisons stay exact for thresholds up to that
    if (measure == TEC_K4 && (__int128)p > (__int128)0xFFFFFFFFll * q)
        return set_error(TEC_EOVERFLOW, "K4 thresholds must not exceed 2^32 - 1");
    return TEC_OK;
}

tec_status stage_mark(tec_graph *g, int i) {
    if (i < g->n_stage_ev && g->stage_ev[i]) TEC_CUDA(cudaEventRecord(g->stage_ev[i], g->stream));
    return TEC_OK;
}

tec_status run_full_pass(tec_graph *g, int measure, int64_t p, int64_t q, int32_t *labels) {
    g->oriented = g->supported = false;
    TEC_TRY(stage_mark(g, 0));
    TEC_TRY(ensure_oriented(g));
    TEC_TRY(stage_mark(g, 1));
    TEC_TRY(ensure_support(g));
    const uint32_t *cts = nullptr;
    int cmp = measure;
    TEC_TRY(measure_counts(g, measure, &cts, &cmp));
    TEC_TRY(stage_mark(g, 2));
    TEC_TRY(reset_counter(g, C_KEPT));
    TEC_TRY(reset_counter(g, C_NCOMP));
    TEC_CUDA(launch_cc_init(g->parent, g->n, g->stream));
    PruneArgs a{cmp, p, q, true};
    TEC_CUDA(launch_prune(g->ooff, g->ocol, g->deg, cts, g->n, g->m, g->or_rows, g->osrc, a, g->keep, g->parent, g->ctr, g->stream));
    g->pruned = g->hooked = true;
    g->last_measure = measure;
    g->last_p = p;
    g->last_q = q;
    TEC_TRY(stage_mark(g, 3));
    TEC_CUDA(launch_cc_finish(g->parent, g->n, labels, g->ctr, g->stream));
    TEC_TRY(stage_mark(g, 4));
    return TEC_OK;
}

}  // namespace
}  // namespace tec

using namespace tec;

namespace tec {
namespace {
tec_status ensure_seg_scratch(tec_graph *g, int ns) {
    if (g->seg_cap >= ns) return TEC_OK;
    dfree(g->seg_hist);
    dfree(g->ari_sums);
    g->seg_hist = nullptr;
    g->ari_sums = nullptr;
    g->seg_cap = 0;
    TEC_TRY(dalloc(&g->seg_hist, (int64_t)ns * 64, "per-graph histograms"));
    TEC_TRY(dalloc(&g->ari_sums, (int64_t)ns * 2 * ARI_CHUNK, "per-graph pair sums"));
    g->seg_cap = ns;
    return TEC_OK;
}

// Rows sorted by ascending threshold p/q (exact 128-bit comparison), equal
// thresholds in input order.
std::vector<int> ascending_rows(const int64_t *p, const int64_t *q, int k) {
    std::vector<int> order(k);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return (__int128)p[a] * q[b] < (__int128)p[b] * q[a]; });
    return order;
}

// Size counters and the level-tagged cell table shared by tec_ari and tec_prf.
// Each buffer is allocated on its own, so one whose allocation failed is
// retried by the next call; a fresh buffer, or a new vertex count (counters
// beyond the old n may be stale), forces the zeroing of all three.
tec_status ensure_cell_tables(tec_graph *g, int64_t tsize) {
    const int64_t ncap = std::max<int64_t>(g->n_cap, 1);
    if (!g->ari_size || !g->ari_keys || !g->ari_cnt) g->ari_tag = ~0ull;
    if (!g->ari_size) TEC_TRY(dalloc(&g->ari_size, 2 * ncap, "component sizes"));
    if (!g->ari_keys) TEC_TRY(dalloc(&g->ari_keys, tsize, "cell keys"));
    if (!g->ari_cnt) TEC_TRY(dalloc(&g->ari_cnt, tsize, "cell counts"));
    if (g->ari_n != g->n) g->ari_tag = ~0ull;
    g->ari_n = g->n;
    return TEC_OK;
}

template <class T>
tec_status grow(T **buf, int64_t *cap, int64_t need, const char *what) {
    if (*cap >= need) return TEC_OK;
    dfree(*buf);
    *buf = nullptr;
    *cap = 0;
    TEC_TRY(dalloc(buf, need, what));
    *cap = need;
    return TEC_OK;
}
}  // namespace
}  // namespace tec

extern "C" {

tec_status tec_features(tec_graph *g, const int64_t *seg_off, int nseg, float *feat_out) {
    clear_error();
    TEC_RANGE();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    if (!feat_out) return set_error(TEC_EINVAL, "feat_out is NULL");
    if (seg_off && nseg < 1) return set_error(TEC_EINVAL, "nseg must be >= 1 with a segment table");
    DeviceGuard dg(g->device);
    const int ns = seg_off ? nseg : 1;
    TEC_TRY(ensure_seg_scratch(g, ns));
    TEC_TRY(ensure_support(g));
    TEC_CUDA(launch_features(g->ooff, g->ocol, g->deg, g->t, g->n, g->m, g->or_rows, g->osrc, seg_off, nseg, g->seg_hist, feat_out, g->ctr,
                             g->stream));
    return TEC_OK;
}

tec_status tec_ari(tec_graph *g, int k, const int32_t *labels, const int32_t *truth, const int64_t *seg_off, int nseg,
                   double *ari_out) {
    clear_error();
    TEC_RANGE();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    if (k < 1) return set_error(TEC_EINVAL, "k must be >= 1");
    if ((!labels || !truth) && g->n > 0) return set_error(TEC_EINVAL, "labels or truth is NULL");
    if (!ari_out) return set_error(TEC_EINVAL, "ari_out is NULL");
    if (seg_off && nseg < 1) return set_error(TEC_EINVAL, "nseg must be >= 1 with a segment table");
    DeviceGuard dg(g->device);
    const int ns = seg_off ? nseg : 1;
    TEC_TRY(ensure_seg_scratch(g, ns));
    const int64_t tsize = (int64_t)1 << ari_table_bits(g->n_cap);
    TEC_TRY(ensure_cell_tables(g, tsize));
    TEC_CUDA(launch_ari(labels, k, truth, g->n, seg_off, nseg, g->seg_hist, g->ari_size, std::max<int64_t>(g->n_cap, 1),
                        g->ari_keys, g->ari_cnt, tsize, g->ari_sums, ari_out, &g->ari_tag, g->ctr, g->stream));
    return TEC_OK;
}

tec_status tec_prf(tec_graph *g, int k, const int32_t *labels, const int32_t *truth, const int64_t *seg_off, int nseg,
                   double *prf_out) {
    clear_error();
    TEC_RANGE();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    if (k < 1) return set_error(TEC_EINVAL, "k must be >= 1");
    if ((!labels || !truth) && g->n > 0) return set_error(TEC_EINVAL, "labels or truth is NULL");
    if (!prf_out) return set_error(TEC_EINVAL, "prf_out is NULL");
    if (seg_off && nseg < 1) return set_error(TEC_EINVAL, "nseg must be >= 1 with a segment table");
    DeviceGuard dg(g->device);
    const int ns = seg_off ? nseg : 1;
    TEC_TRY(ensure_seg_scratch(g, ns));
    const int64_t tsize = (int64_t)1 << ari_table_bits(g->n_cap);
    const int64_t ncap = std::max<int64_t>(g->n_cap, 1);
    if (!g->prf_best) TEC_TRY(dalloc(&g->prf_best, ncap, "best matches"));
    if (!g->prf_bestb) TEC_TRY(dalloc(&g->prf_bestb, ncap, "matched blocks"));
    TEC_TRY(grow(&g->prf_sums, &g->prf_sums_cap, (int64_t)3 * ns * ARI_CHUNK, "P/R/F1 sums"));
    TEC_TRY(ensure_cell_tables(g, tsize));
    TEC_CUDA(launch_prf(labels, k, truth, g->n, seg_off, nseg, g->seg_hist, g->ari_size, ncap, g->ari_keys, g->ari_cnt,
                        tsize, g->ari_sums, g->prf_best, g->prf_bestb, g->prf_sums, prf_out, &g->ari_tag, g->ctr,
                        g->stream));
    return TEC_OK;
}

tec_status tec_ari_best(const double *ari, int k, int nseg, int32_t *best, double *best_ari, void *stream) {
    clear_error();
    if (k < 1 || nseg < 0 || (nseg > 0 && (!ari || !best))) return set_error(TEC_EINVAL, "bad argument");
    TEC_CUDA(launch_best_level(ari, k, nseg, best, best_ari, (cudaStream_t)stream));
    return TEC_OK;
}

}  // extern "C"

extern "C" {

int tec_version(void) { return 100; }

size_t tec_last_error(char *buf, size_t len) {
    size_t full = strlen(g_err);
    if (buf && len) {
        size_t c = full < len - 1 ? full : len - 1;
        memcpy(buf, g_err, c);
        buf[c] = '\0';
    }
    return full;
}

tec_status tec_graph_create(int64_t n_cap, int64_t nnz_cap, void *stream, tec_graph **out) {
    clear_error();
    if (!out) return set_error(TEC_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_cap < 0 || n_cap > MAX_N) return set_error(TEC_EINVAL, "n_cap must be in [0, 2^31-1]");
    if (nnz_cap < 0 || nnz_cap > (int64_t)1 << 40) return set_error(TEC_EINVAL, "nnz_cap out of range");
    tec_graph *g = new (std::nothrow) tec_graph();
    if (!g) return set_error(TEC_ENOMEM, "host allocation failed");
    g->stream = (cudaStream_t)stream;
    g->n_cap = n_cap;
    g->nnz_cap = nnz_cap;
    g->m_cap = nnz_cap / 2;
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e != cudaSuccess) {
        delete g;
        return set_error(TEC_ECUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
    }
    const int64_t ntiles = ceil_div(nnz_cap, TILE);
    const int64_t mwords = ceil_div(g->m_cap, TILE) * (TILE / 32);
    const int64_t scan_len = (n_cap + 1 > ntiles ? n_cap + 1 : ntiles);
    tec_status s = TEC_OK;
    if (s == TEC_OK) s = dalloc(&g->off, n_cap + 1, "row offsets");
    if (s == TEC_OK) s = dalloc(&g->col, nnz_cap, "column ids");
    if (s == TEC_OK) s = dalloc(&g->deg, n_cap, "degrees");
    if (s == TEC_OK) s = dalloc(&g->ooff, n_cap + 1, "oriented offsets");
    if (s == TEC_OK) s = dalloc(&g->ocol, g->m_cap + 4, "oriented column ids");   // 16-byte padded for bulk prefetches
    if (s == TEC_OK) s = dalloc(&g->t, g->m_cap, "triangle counts");
    if (s == TEC_OK) s = dalloc(&g->keep, mwords, "keep mask");
    if (s == TEC_OK) s = dalloc(&g->parent, n_cap, "union-find parents");
    g->task_cap = support_task_capacity(n_cap, nnz_cap);
    if (s == TEC_OK) s = dalloc(&g->tasks, g->task_cap, "support task list");
    if (s == TEC_OK) s = dalloc(&g->flags, ntiles * (TILE / 32), "orientation bits");
    if (s == TEC_OK) s = dalloc(&g->sym_rows, tile_rows_size(nnz_cap), "tile rows");
    if (s == TEC_OK) s = dalloc(&g->or_rows, tile_rows_size(g->m_cap), "tile rows");
    if (s == TEC_OK) s = dalloc(&g->osrc, g->m_cap, "edge sources");
    if (s == TEC_OK) s = dalloc(&g->tile_cnt, ntiles + 1, "tile counts");
    if (s == TEC_OK) s = dalloc(&g->tile_base, ntiles + 1, "tile offsets");
    if (s == TEC_OK) s = dalloc(&g->bsum, scan_bsum_size(scan_len), "scan partials");
    if (s == TEC_OK) s = dalloc(&g->ctr, C_COUNT, "counters");
    if (s == TEC_OK) {
        e = cudaMallocHost((void **)&g->ctr_host, C_COUNT * sizeof(unsigned long long));
        if (e != cudaSuccess) s = set_error(TEC_ENOMEM, "pinned host allocation failed: %s", cudaGetErrorString(e));
    }
    if (s == TEC_OK) {
        e = cudaMemsetAsync(g->ctr, 0, C_COUNT * sizeof(unsigned long long), g->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(g->off, 0, sizeof(int64_t), g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) s = set_error(TEC_ECUDA, "initialisation failed: %s", cudaGetErrorString(e));
    }
    if (s != TEC_OK) {
        free_graph_memory(g);
        delete g;
        return s;
    }
    *out = g;
    return TEC_OK;
}

tec_status tec_graph_load(tec_graph *g, const void *row_off, int off_is_i64, const int32_t *col, int64_t n,
                          int64_t nnz, uint32_t flags) {
    clear_error();
    TEC_RANGE();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    if (n < 0 || n > g->n_cap) return set_error(TEC_EINVAL, "n=%lld exceeds the capacity %lld", (long long)n, (long long)g->n_cap);
    if (nnz < 0 || nnz > g->nnz_cap) return set_error(TEC_EINVAL, "nnz=%lld exceeds the capacity %lld", (long long)nnz, (long long)g->nnz_cap);
    if (nnz % 2) return set_error(TEC_EINVAL, "nnz must be even (both directions of every edge)");
    if (n == 0 && nnz != 0) return set_error(TEC_EINVAL, "a graph without vertices has no edges");
    if (!row_off && n > 0) return set_error(TEC_EINVAL, "row_off is NULL");
    if (!col && nnz > 0) return set_error(TEC_EINVAL, "col is NULL");
    if (!off_is_i64 && nnz > INT32_MAX) return set_error(TEC_EOVERFLOW, "int32 offsets cannot index %lld entries", (long long)nnz);
    DeviceGuard dg(g->device);
    cudaStream_t s = g->stream;
    const bool host = (flags & TEC_HOST_PTR) != 0;
    g->oriented = g->supported = g->pruned = g->hooked = g->uoff_valid = false;
    g->n = g->nnz = g->m = 0;
    if (n > 0) {
        if (off_is_i64) {
            TEC_CUDA(cudaMemcpyAsync(g->off, row_off, (size_t)(n + 1) * sizeof(int64_t),
                                     host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
        } else if (host) {
            const int32_t *o32 = (const int32_t *)row_off;
            std::vector<int64_t> wide(o32, o32 + n + 1);
            TEC_CUDA(cudaMemcpyAsync(g->off, wide.data(), wide.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
            TEC_CUDA(cudaStreamSynchronize(s));
        } else {
            TEC_CUDA(launch_widen_offsets((const int32_t *)row_off, n + 1, g->off, s));
        }
    } else {
        TEC_CUDA(cudaMemsetAsync(g->off, 0, sizeof(int64_t), s));
    }
    if (nnz > 0)
        TEC_CUDA(cudaMemcpyAsync(g->col, col, (size_t)nnz * sizeof(int32_t),
                                 host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    TEC_CUDA(cudaMemsetAsync(g->ctr, 0, C_COUNT * sizeof(unsigned long long), s));
    g->n = n;
    g->nnz = nnz;
    g->m = nnz / 2;
    TEC_CUDA(launch_tile_rows(g->off, n, nnz, g->sym_rows, s));
    if (flags & TEC_VALIDATE) {
        TEC_CUDA(launch_validate(g->off, g->col, n, nnz, g->ctr, s));
        tec_status st = read_counters(g);
        if (st == TEC_OK) {
            TEC_CUDA(launch_validate_entries(g->off, g->col, n, nnz, g->sym_rows, g->ctr, s));
            st = read_counters(g);
        }
        if (st != TEC_OK) {
            g->n = g->nnz = g->m = 0;
            return st;
        }
    }
    TEC_CUDA(launch_degrees(g->off, n, g->deg, s));
    if (host) TEC_CUDA(cudaStreamSynchronize(s));
    return TEC_OK;
}

tec_status tec_graph_upload(const void *row_off, int off_is_i64, const int32_t *col, int64_t n, int64_t nnz,
                            uint32_t flags, void *stream, tec_graph **out) {
    clear_error();
    if (!out) return set_error(TEC_EINVAL, "out is NULL");
    *out = nullptr;
    tec_graph *g = nullptr;
    TEC_TRY(tec_graph_create(n, nnz, stream, &g));
    tec_status s = tec_graph_load(g, row_off, off_is_i64, col, n, nnz, flags);
    if (s != TEC_OK) {
        char keep_msg[sizeof(g_err)];
        memcpy(keep_msg, g_err, sizeof(g_err));
        tec_graph_free(g);
        memcpy(g_err, keep_msg, sizeof(g_err));
        return s;
    }
    *out = g;
    return TEC_OK;
}

tec_status tec_graph_free(tec_graph *g) {
    clear_error();
    if (!g) return TEC_OK;
    DeviceGuard dg(g->device);
    cudaStreamSynchronize(g->stream);
    free_graph_memory(g);
    delete g;
    return TEC_OK;
}

tec_status tec_graph_info(const tec_graph *g, int64_t *n, int64_t *m) {
    clear_error();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    if (n) *n = g->n;
    if (m) *m = g->m;
    return TEC_OK;
}

tec_status tec_sync(tec_graph *g) {
    clear_error();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    DeviceGuard dg(g->device);
#ifdef TEC_DEBUG
    TEC_TRY(read_counters(g));
    return check_canaries();
#else
    return read_counters(g);
#endif
}

tec_status tec_orient(tec_graph *g) {
    clear_error();
    TEC_RANGE();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    DeviceGuard dg(g->device);
    g->oriented = false;
    return ensure_oriented(g);
}

tec_status tec_support(tec_graph *g) {
    clear_error();
    TEC_RANGE();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    DeviceGuard dg(g->device);
    g->supported = false;
    return ensure_support(g);
}

tec_status tec_edge_list(tec_graph *g, int32_t *u_out, int32_t *v_out) {
    clear_error();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    if ((!u_out || !v_out) && g->m > 0) return set_error(TEC_EINVAL, "output is NULL");
    DeviceGuard dg(g->device);
    TEC_TRY(ensure_uoff(g));
    TEC_CUDA(launch_export(g->off, g->col, g->deg, g->ooff, g->ocol, nullptr, g->keep, g->n, g->nnz, g->uoff,
                           u_out, v_out, nullptr, nullptr, nullptr, 0, nullptr, g->ctr, g->stream));
    return TEC_OK;
}

tec_status tec_edge_support(tec_graph *g, uint32_t *t_out, uint32_t *wedge_out) {
    clear_error();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    if (!t_out && g->m > 0) return set_error(TEC_EINVAL, "t_out is NULL");
    DeviceGuard dg(g->device);
    TEC_TRY(ensure_support(g));
    TEC_TRY(ensure_uoff(g));
    TEC_CUDA(launch_export(g->off, g->col, g->deg, g->ooff, g->ocol, g->t, g->keep, g->n, g->nnz, g->uoff,
                           nullptr, nullptr, t_out, wedge_out, nullptr, 0, nullptr, g->ctr, g->stream));
    return TEC_OK;
}

tec_status tec_edge_k4(tec_graph *g, uint32_t *k4_out) {
    clear_error();
    TEC_RANGE();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    if (!k4_out && g->m > 0) return set_error(TEC_EINVAL, "k4_out is NULL");
    DeviceGuard dg(g->device);
    TEC_TRY(ensure_k4(g));
    TEC_TRY(ensure_uoff(g));
    TEC_CUDA(launch_export(g->off, g->col, g->deg, g->ooff, g->ocol, g->k4, g->keep, g->n, g->nnz, g->uoff,
                           nullptr, nullptr, k4_out, nullptr, nullptr, 0, nullptr, g->ctr, g->stream));
    return TEC_OK;
}

tec_status tec_edge_weights(tec_graph *g, tec_measure measure, double *w_out) {
    clear_error();
    TEC_RANGE();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    if (measure < TEC_TECTONIC || measure > TEC_K4) return set_error(TEC_EINVAL, "unknown measure %d", (int)measure);
    if (!w_out && g->m > 0) return set_error(TEC_EINVAL, "w_out is NULL");
    DeviceGuard dg(g->device);
    const uint32_t *cts = nullptr;
    int cmp = (int)measure;
    TEC_TRY(measure_counts(g, (int)measure, &cts, &cmp));
    TEC_TRY(ensure_uoff(g));
    TEC_CUDA(launch_export(g->off, g->col, g->deg, g->ooff, g->ocol, cts, g->keep, g->n, g->nnz, g->uoff,
                           nullptr, nullptr, nullptr, nullptr, w_out, cmp, nullptr, g->ctr, g->stream));
    return TEC_OK;
}

tec_status tec_prune(tec_graph *g, tec_measure measure, int64_t p, int64_t q, uint8_t *keep_out,
                     int64_t *kept_out) {
    clear_error();
    TEC_RANGE();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    TEC_TRY(check_threshold((int)measure, p, q));
    DeviceGuard dg(g->device);
    TEC_TRY(debug_refresh_caps(g));
    const uint32_t *cts = nullptr;
    int cmp = (int)measure;
    TEC_TRY(measure_counts(g, (int)measure, &cts, &cmp));
    TEC_TRY(reset_counter(g, C_KEPT));
    PruneArgs a{cmp, p, q, false};
    TEC_CUDA(launch_prune(g->ooff, g->ocol, g->deg, cts, g->n, g->m, g->or_rows, g->osrc, a, g->keep, g->parent, g->ctr, g->stream));
    g->pruned = true;
    g->hooked = false;
    g->last_measure = (int)measure;
    g->last_p = p;
    g->last_q = q;
    if (keep_out) {
        TEC_TRY(ensure_uoff(g));
        TEC_CUDA(launch_export(g->off, g->col, g->deg, g->ooff, g->ocol, g->t, g->keep, g->n, g->nnz, g->uoff,
                               nullptr, nullptr, nullptr, nullptr, nullptr, 0, keep_out, g->ctr, g->stream));
    }
    if (kept_out) {
        TEC_TRY(read_counters(g));
        *kept_out = (int64_t)g->ctr_host[C_KEPT];
    }
    return TEC_OK;
}

tec_status tec_components(tec_graph *g, int32_t *labels_out, int64_t *ncomp_out) {
    clear_error();
    TEC_RANGE();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    if (!g->pruned) return set_error(TEC_ESTATE, "tec_components needs a tec_prune first");
    if (!labels_out && g->n > 0) return set_error(TEC_EINVAL, "labels_out is NULL");
    DeviceGuard dg(g->device);
    TEC_TRY(debug_refresh_caps(g));
    if (!g->hooked) {
        TEC_CUDA(launch_cc_init(g->parent, g->n, g->stream));
        TEC_CUDA(launch_cc_hook(g->ooff, g->ocol, g->keep, g->n, g->m, g->or_rows, g->osrc, g->parent, g->ctr, g->stream));
        g->hooked = true;
    }
    TEC_TRY(reset_counter(g, C_NCOMP));
    TEC_CUDA(launch_cc_finish(g->parent, g->n, labels_out, g->ctr, g->stream));
    if (ncomp_out) {
        TEC_TRY(read_counters(g));
        *ncomp_out = (int64_t)g->ctr_host[C_NCOMP];
    }
    return TEC_OK;
}

tec_status tec_full_pass(tec_graph *g, tec_measure measure, int64_t p, int64_t q, int32_t *labels_out,
                         int64_t *ncomp_out) {
    clear_error();
    TEC_RANGE();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    TEC_TRY(check_threshold((int)measure, p, q));
    if (!labels_out && g->n > 0) return set_error(TEC_EINVAL, "labels_out is NULL");
    DeviceGuard dg(g->device);
    TEC_TRY(debug_refresh_caps(g));
    TEC_TRY(run_full_pass(g, (int)measure, p, q, labels_out));
    if (ncomp_out) {
        TEC_TRY(read_counters(g));
        *ncomp_out = (int64_t)g->ctr_host[C_NCOMP];
    }
    return TEC_OK;
}

tec_status tec_full_pass_host(tec_graph *g, const int64_t *row_off_host, const int32_t *col_host, int64_t n,
                              int64_t nnz, tec_measure measure, int64_t p, int64_t q, int32_t *labels_host,
                              int64_t *ncomp_out) {
    clear_error();
    TEC_RANGE();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    if (!labels_host && n > 0) return set_error(TEC_EINVAL, "labels_host is NULL");
    TEC_TRY(check_threshold((int)measure, p, q));
    DeviceGuard dg(g->device);
    TEC_TRY(tec_graph_load(g, row_off_host, 1, col_host, n, nnz, TEC_HOST_PTR));
    TEC_TRY(debug_refresh_caps(g));   // loading clears the counter block
    // Labels need their own buffer: while the finishing kernel resolves roots,
    // path compression may still re-point parent[x] at an intermediate ancestor.
    if (!g->labels) TEC_TRY(dalloc(&g->labels, g->n_cap, "label buffer"));
    TEC_TRY(run_full_pass(g, (int)measure, p, q, g->labels));
    if (n > 0)
        TEC_CUDA(cudaMemcpyAsync(labels_host, g->labels, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                 g->stream));
    TEC_TRY(read_counters(g));
    if (ncomp_out) *ncomp_out = (int64_t)g->ctr_host[C_NCOMP];
    return TEC_OK;
}

tec_status tec_sweep(tec_graph *g, tec_measure measure, const int64_t *p, const int64_t *q, int k,
                     const int64_t *seg_off, int nseg, int32_t *labels_out, int64_t *ncomp_out) {
    clear_error();
    TEC_RANGE();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    if (k < 1 || k > 127) return set_error(TEC_EINVAL, "k must be in [1, 127] (got %d)", k);
    if (!p || !q) return set_error(TEC_EINVAL, "threshold arrays are NULL");
    if (!labels_out && g->n > 0) return set_error(TEC_EINVAL, "labels_out is NULL");
    if (seg_off && nseg < 1) return set_error(TEC_EINVAL, "nseg must be >= 1 with a segment table");
    bool wide = false;
    for (int i = 0; i < k; ++i) {
        TEC_TRY(check_threshold((int)measure, p[i], q[i]));
        wide = wide || needs_wide(p[i], q[i]);
    }
    DeviceGuard dg(g->device);
    TEC_TRY(debug_refresh_caps(g));
    const int nsl = seg_off ? nseg : 1;
    const std::vector<int> order = ascending_rows(p, q, k);
    std::vector<int64_t> hthr(2 * k);
    for (int i = 0; i < k; ++i) {
        hthr[i] = p[order[i]];
        hthr[k + i] = q[order[i]];
    }
    if (!g->lvl) TEC_TRY(dalloc(&g->lvl, g->m_cap, "edge levels"));
    if (!g->best) TEC_TRY(dalloc(&g->best, g->n_cap, "forest offers"));
    if (!g->fu) TEC_TRY(dalloc(&g->fu, g->n_cap, "forest edges"));
    if (!g->fv) TEC_TRY(dalloc(&g->fv, g->n_cap, "forest edges"));
    if (!g->bucket) TEC_TRY(dalloc(&g->bucket, 3 * 127 + 4, "level buckets"));
    if (!g->thr) TEC_TRY(dalloc(&g->thr, 2 * 127, "thresholds"));
    if (g->sw_ncomp_cap < (int64_t)k * nsl) {
        dfree(g->sw_ncomp);
        g->sw_ncomp = nullptr;
        g->sw_ncomp_cap = 0;
        TEC_TRY(dalloc(&g->sw_ncomp, (int64_t)k * nsl, "component counts"));
        g->sw_ncomp_cap = (int64_t)k * nsl;
    }
    cudaStream_t s = g->stream;
    // live-edge list of the later Boruvka rounds (16 bytes per edge); without
    // the memory for it those rounds rescan the CSR instead
    if (g->msf_cap == 0 && g->m_cap > 0) {
        const int64_t tiles = ceil_div(g->m_cap, (int64_t)TILE), cap = tiles * TILE;
        if (dalloc(&g->msf_u, cap, "live edges") != TEC_OK || dalloc(&g->msf_v, cap, "live edges") != TEC_OK ||
            dalloc(&g->msf_k, cap, "live edge keys") != TEC_OK || dalloc(&g->msf_cnt, tiles, "live edge counts") != TEC_OK) {
            void *part[] = {g->msf_u, g->msf_v, g->msf_k, g->msf_cnt};
            for (void *q2 : part) dfree(q2);
            g->msf_u = g->msf_v = g->msf_cnt = nullptr;
            g->msf_k = nullptr;
            g->msf_cap = -1;
            clear_error();
        } else {
            g->msf_cap = cap;
        }
    }
    const bool list = g->msf_cap > 0;
    int32_t *lu = list ? g->msf_u : nullptr, *lv = list ? g->msf_v : nullptr, *lc = list ? g->msf_cnt : nullptr;
    unsigned long long *lk = list ? g->msf_k : nullptr;
    if (!g->msf_changed) TEC_TRY(dalloc(&g->msf_changed, 64, "forest round flags"));
    const uint32_t *cts = nullptr;
    int cmp = (int)measure;
    TEC_TRY(measure_counts(g, (int)measure, &cts, &cmp));
    // From here on only kernels and memsets on the graph's stream: with the
    // buffers above allocated and ncomp_out NULL, a caller can capture the
    // whole sweep in a CUDA graph.
    TEC_CUDA(launch_store_thresholds(hthr.data(), 2 * k, g->thr, s));
    // Boruvka rounds of the maximum spanning forest.  The first runs in the
    // level pass; every round merges each tree that still has a live edge, so
    // ceil(log2 n) + 1 rounds complete the forest and one more finds nothing.
    // Rounds after a round that joined nothing return at once.
    int rounds = 2;
    while (rounds < 64 && ((int64_t)1 << (rounds - 2)) < g->n) ++rounds;
    rounds = debug_msf_rounds(rounds);
    g->pruned = g->hooked = false;
    TEC_CUDA(launch_cc_init(g->parent, g->n, s));
    if (g->n > 0) TEC_CUDA(cudaMemsetAsync(g->best, 0, (size_t)g->n * sizeof(unsigned long long), s));
    TEC_CUDA(cudaMemsetAsync(g->msf_changed, 0, 64 * sizeof(unsigned long long), s));
    TEC_CUDA(launch_levels(g->ooff, g->ocol, g->deg, cts, g->n, g->m, g->or_rows, g->osrc, cmp, g->thr, g->thr + k, k, wide,
                           g->lvl, g->best, lu, lv, lk, lc, g->ctr, s));
    for (int round = 0; round < rounds; ++round) {
        const unsigned long long *prev = round > 0 ? g->msf_changed + round - 1 : nullptr;
        if (round > 0)
            TEC_CUDA(launch_msf_offer(g->ooff, g->ocol, g->lvl, g->n, g->m, g->osrc, g->parent, g->best, lu, lv, lk, lc, prev,
                                      g->ctr, s));
        TEC_CUDA(launch_msf_hook(g->ooff, g->ocol, g->osrc, g->lvl, g->n, g->parent, g->best, prev, g->msf_changed + round,
                                 g->ctr, s));
    }
    TEC_CUDA(launch_msf_check(g->msf_changed + rounds - 1, g->ctr, s));
    // offline sweep over the forest edges, highest level first
    TEC_CUDA(launch_forest_buckets(g->ooff, g->ocol, g->lvl, g->n, g->m, g->or_rows, g->osrc, k, g->bucket, g->fu, g->fv, g->ctr, s));
    TEC_CUDA(launch_cc_init(g->parent, g->n, s));
    TEC_CUDA(cudaMemsetAsync(g->sw_ncomp, 0, (size_t)k * nsl * sizeof(unsigned long long), s));
    for (int L = k; L >= 1; --L) {
        const int dst = order[L - 1];
        TEC_CUDA(launch_sweep_level(g->fu, g->fv, g->bucket, k, L, g->n, g->parent, labels_out + (int64_t)dst * g->n,
                                    seg_off, nseg, g->sw_ncomp + (int64_t)dst * nsl, g->ctr, s));
    }
    if (ncomp_out) {
        std::vector<unsigned long long> hn((size_t)k * nsl);
        TEC_CUDA(cudaMemcpyAsync(hn.data(), g->sw_ncomp, hn.size() * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, s));
        TEC_TRY(read_counters(g));
        for (size_t i = 0; i < hn.size(); ++i) ncomp_out[i] = (int64_t)hn[i];
    }
    return TEC_OK;
}

tec_status tec_sweep_stats(tec_graph *g, tec_measure measure, const int64_t *p, const int64_t *q, int k,
                           const int32_t *labels, const int64_t *seg_off, int nseg, tec_sweep_stat *stats_out) {
    clear_error();
    TEC_RANGE();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    if (k < 1 || k > 127) return set_error(TEC_EINVAL, "k must be in [1, 127] (got %d)", k);
    if (!p || !q || !stats_out) return set_error(TEC_EINVAL, "NULL argument");
    if (!labels && g->n > 0) return set_error(TEC_EINVAL, "labels is NULL");
    if (seg_off && nseg < 1) return set_error(TEC_EINVAL, "nseg must be >= 1 with a segment table");
    bool wide = false;
    for (int i = 0; i < k; ++i) {
        TEC_TRY(check_threshold((int)measure, p[i], q[i]));
        wide = wide || needs_wide(p[i], q[i]);
    }
    DeviceGuard dg(g->device);
    const int ns = seg_off ? nseg : 1;
    const std::vector<int> order = ascending_rows(p, q, k);
    std::vector<int64_t> hthr(2 * 127);
    for (int i = 0; i < k; ++i) {
        hthr[i] = p[order[i]];
        hthr[127 + i] = q[order[i]];
    }
    if (!g->thr) TEC_TRY(dalloc(&g->thr, 2 * 127, "thresholds"));
    TEC_TRY(grow(&g->st_hist, &g->st_hist_cap, (int64_t)ns * 2 * (k + 1), "statistics histograms"));
    TEC_TRY(grow(&g->st_sums, &g->st_sums_cap, (int64_t)k * ns * 3, "statistics sums"));
    const int64_t cl = std::max<int64_t>(g->n_cap, 1);
    if (!g->st_cnt_n) TEC_TRY(dalloc(&g->st_cnt_n, 2 * cl, "component sizes"));
    if (!g->st_cnt_v) TEC_TRY(dalloc(&g->st_cnt_v, 2 * cl, "component volumes"));
    TEC_CUDA(cudaMemcpyAsync(g->thr, hthr.data(), hthr.size() * sizeof(int64_t), cudaMemcpyHostToDevice, g->stream));
    const uint32_t *cts = nullptr;
    int cmp = (int)measure;
    TEC_TRY(measure_counts(g, (int)measure, &cts, &cmp));
    TEC_CUDA(launch_sweep_stats(g->ooff, g->ocol, g->deg, cts, g->n, g->m, g->or_rows, g->osrc, cmp, g->thr, g->thr + 127, k,
                                order.data(), wide, labels, seg_off, nseg, g->st_hist, g->st_cnt_n, g->st_cnt_v, cl,
                                g->st_sums, stats_out, g->ctr, g->stream));
    return TEC_OK;
}

tec_status tec_rule_of_thumb(const tec_sweep_stat *stats, const int64_t *p, const int64_t *q, int k, int nseg,
                             tec_rule rule, int32_t *best_out, void *stream) {
    clear_error();
    if (k < 1 || k > 127 || nseg < 0) return set_error(TEC_EINVAL, "k must be in [1, 127], nseg >= 0");
    if (!p || !q || (nseg > 0 && (!stats || !best_out))) return set_error(TEC_EINVAL, "NULL argument");
    if (rule != TEC_RULE_LARGEST_JUMP && rule != TEC_RULE_MODULARITY) return set_error(TEC_EINVAL, "unknown rule");
    for (int i = 0; i < k; ++i)
        if (q[i] <= 0) return set_error(TEC_EINVAL, "threshold denominators must be positive");
    const std::vector<int> order = ascending_rows(p, q, k);
    TEC_CUDA(launch_rules(stats, k, nseg, order.data(), (int)rule, best_out, (cudaStream_t)stream));
    return TEC_OK;
}

tec_status tec_prune_components_batch(tec_graph *g, tec_measure measure, const int64_t *p, const int64_t *q,
                                      const int64_t *seg_off, int nseg, int32_t *labels_out, int64_t *ncomp_out) {
    clear_error();
    TEC_RANGE();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    if (measure < TEC_TECTONIC || measure > TEC_K4) return set_error(TEC_EINVAL, "unknown measure %d", (int)measure);
    if (!p || !q || !seg_off || nseg < 1) return set_error(TEC_EINVAL, "thresholds and segment table are required");
    if (!labels_out && g->n > 0) return set_error(TEC_EINVAL, "labels_out is NULL");
    DeviceGuard dg(g->device);
    TEC_TRY(debug_refresh_caps(g));
    if (g->sw_ncomp_cap < nseg) {
        dfree(g->sw_ncomp);
        g->sw_ncomp = nullptr;
        g->sw_ncomp_cap = 0;
        TEC_TRY(dalloc(&g->sw_ncomp, nseg, "component counts"));
        g->sw_ncomp_cap = nseg;
    }
    const uint32_t *cts = nullptr;
    int cmp = (int)measure;
    TEC_TRY(measure_counts(g, (int)measure, &cts, &cmp));
    TEC_TRY(reset_counter(g, C_KEPT));
    TEC_CUDA(launch_cc_init(g->parent, g->n, g->stream));
    TEC_CUDA(launch_prune_seg(g->ooff, g->ocol, g->deg, cts, g->n, g->m, g->or_rows, g->osrc, cmp, p, q, seg_off, nseg, true,
                              g->keep, g->parent, g->ctr, g->stream));
    g->pruned = g->hooked = true;
    TEC_CUDA(cudaMemsetAsync(g->sw_ncomp, 0, (size_t)nseg * sizeof(unsigned long long), g->stream));
    TEC_CUDA(launch_snapshot(g->parent, g->n, labels_out, seg_off, nseg, g->sw_ncomp, g->stream));
    if (ncomp_out) {
        std::vector<unsigned long long> hn((size_t)nseg);
        TEC_CUDA(cudaMemcpyAsync(hn.data(), g->sw_ncomp, hn.size() * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, g->stream));
        TEC_TRY(read_counters(g));
        for (int i = 0; i < nseg; ++i) ncomp_out[i] = (int64_t)hn[i];
    }
    return TEC_OK;
}

tec_status tec_set_core_staging(tec_graph *g, int enable) {
    clear_error();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    if ((enable != 0) != g->core_enabled) {
        g->core_enabled = enable != 0;
        g->supported = g->pruned = g->hooked = false;   // counts are recomputed by the other path
    }
    return TEC_OK;
}

tec_status tec_set_support_tiling(tec_graph *g, int groups) {
    clear_error();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    if (groups < -1 || groups > SUPPORT_MAX_GROUPS)
        return set_error(TEC_EINVAL, "groups must be -1 (off), 0 (automatic) or 1..%d", SUPPORT_MAX_GROUPS);
    if (groups != g->tile_request) {
        g->tile_request = groups;
        g->supported = g->pruned = g->hooked = false;   // counts are recomputed on the next use
    }
    return TEC_OK;
}

long long tec_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

tec_status tec_set_stage_events(tec_graph *g, void *const *events, int count) {
    clear_error();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    if (count < 0 || count > 5 || (count > 0 && !events)) return set_error(TEC_EINVAL, "0..5 events");
    for (int i = 0; i < 5; ++i) g->stage_ev[i] = i < count ? (cudaEvent_t)events[i] : nullptr;
    g->n_stage_ev = count;
    return TEC_OK;
}

tec_status tec_oriented_csr(tec_graph *g, int64_t *ooff_out, int32_t *ocol_out) {
    clear_error();
    if (!g) return set_error(TEC_EINVAL, "graph is NULL");
    DeviceGuard dg(g->device);
    TEC_TRY(ensure_oriented(g));
    if (ooff_out)
        TEC_CUDA(cudaMemcpyAsync(ooff_out, g->ooff, (size_t)(g->n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice,
                                 g->stream));
    if (ocol_out && g->m > 0)
        TEC_CUDA(cudaMemcpyAsync(ocol_out, g->ocol, (size_t)g->m * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                 g->stream));
    return TEC_OK;
}

}  // extern "C"
