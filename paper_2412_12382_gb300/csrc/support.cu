// Per-edge triangle counts t(u,v) = |N(u) n N(v)| (Sec. I) on the oriented CSR.
//
// Every triangle {a, b, c} with (deg, id)-rank a < b < c is found exactly once,
// as the element c of N+(a) n N+(b) for the oriented edge a -> b, and is
// credited to its three oriented edges a->b, a->c, b->c.  Integer sums do not
// depend on the order of the adds, so the counts are exact and deterministic.
//
// Each oriented edge x -> y is intersected from the side with the shorter
// out-row, so the probe work is the sum over edges of min(d+(x), d+(y)):
//   U-mode, centre c = x, when d+(y) <= d+(x): the ids of N+(y) are probed
//     against the staged set N+(c);
//   V-mode, centre c = y, when d+(x) <  d+(y): the ids of N+(x) are probed
//     against the staged set N+(c).  The in-neighbours x of c are the entries
//     of c's symmetric row whose orientation bit is clear, so no transposed
//     graph is needed.
// A probe row is never longer than the staged set.
//
// The candidates of centre c are indexed 0 .. d+(c) + deg(c) - 1: first the
// U-mode candidates N+(c), then the entries of c's symmetric row (V-mode).  A
// visit is a contiguous slice of them, sized by probes:
//   core visits   centres of degree >= D (a core of at most 2^20 vertices, see
//                 "core staging" below) with enough work: N+(c) staged per
//                 block as an exact bitmap over core codes, 2^25 probes;
//   warp visits   other centres with d+(c) <= 256: N+(c) staged in the warp's
//                 own slice of shared memory (sorted ids, bitmap filter,
//                 bucket directory), 2^20 probes;
//   block visits  the rest: N+(c) staged per block in chunks of 4096 ids
//                 (sorted ids, bitmap filter, bucket directory), 2^25 probes.
// In a block or core visit the block's warps take batches of 8 candidates
// from a shared counter; a warp visit walks its candidates 32 at a time.  Each
// lane loads one candidate's row bounds (one round of latency per batch); long
// rows are then read one after another by the whole warp, coalesced, with 4
// (hashed staging) or 16 (core staging) ids per lane in flight, and short
// rows are packed end to end over the lanes.  Two persistent kernels: one
// 1024-thread block per SM for the core visits, then two 512-thread blocks per
// SM that drain the block visits and reuse the same shared memory for warp
// visits.
#include <algorithm>
#include <climits>

#include "tec_internal.cuh"

namespace tec {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int W_MAX = 256;                      // largest d+(c) of a warp visit
constexpr int B_THREADS = 512;                  // block-visit kernel block
constexpr int B_WARPS = B_THREADS / 32;
constexpr int S_CHUNK = 4096;                   // staged ids per block chunk
constexpr int64_t VISIT_PROBES_W = 1 << 20;     // target probes per warp visit
// Target probes per block (and core) visit.  A block visit ends at a block
// barrier, so its warps idle for up to one batch at the end: the visit must
// hold many batches per warp for that tail to stay small.
constexpr int64_t VISIT_PROBES_B = 1 << 25;
constexpr int W_GRAB = 16;                      // warp visits taken per counter bump
constexpr int64_t CORE_MIN_WORK = 1 << 16;      // probes (about) for a small core centre to get a block visit
// Candidates per batch of a block visit.  A visit ends at a block barrier, and
// one batch of long rows can hold many times the average batch's probes, so
// batches smaller than a warp keep the barrier tail short.
constexpr int B_BATCH = 8;
constexpr int C_BATCH = 16;                     // candidates per batch in core visits (bitmap tests are short)
constexpr uint64_t VIS_MASK = (1ull << 32) - 1;
// Probe-row tiling (when a range count is set): the candidates per range a
// core centre needs to be tiled (each range's visit restages the centre's row).
constexpr int HEAVY_CAND = 8;
constexpr int T_BATCH = 2;                      // candidates per batch of a tiled visit (few per range)
// Order of the core visits: 0 as emitted (about id order), 1 by d+(c)
// descending, 2 by d+(c) ascending (a counting sort over d+ clamped to
// ORDER_CLASSES - 1), meant to let visits running at the same time share
// probe rows in L2.  Measured on R-MAT scale 26: 2571 ms (0), 2592 ms (1),
// 2595 ms (2), so the visits run as emitted.
constexpr int CORE_ORDER = 0;
constexpr int ORDER_CLASSES = 1 << 16;

__device__ __forceinline__ bool out_bit(const uint32_t *flags, int64_t e) {
    return (flags[e >> 5] >> (e & 31)) & 1u;
}

__device__ __forceinline__ int64_t lower_bound_g(const int32_t *a, int64_t lo, int64_t hi, int32_t x) {
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Candidates of one visit: du + deg candidates split into slices of vlen
// (block = a visit run by a whole block: the hashed block visits and all
// core visits).
__device__ __forceinline__ int64_t visit_len(int64_t du, bool block) {
    int64_t v = (block ? VISIT_PROBES_B : VISIT_PROBES_W) / (du > 0 ? du : 1);
    return v < 256 ? 256 : (v > 65536 ? 65536 : v);
}

// One thread per vertex: emits the visits of centre c: the warp list from the
// front of tasks[], the block list from its back, and the visits of core
// centres (core_of[c] >= 0, when core_of is given) to ctasks[]: all with
// d+(c) > W_MAX, and smaller ones with at least CORE_MIN_WORK probes.
__global__ void k_make_visits(const int64_t *off, const int64_t *ooff, int64_t n, uint64_t *tasks, int64_t cap,
                              const int32_t *core_of, uint64_t *ctasks, int groups, int32_t *heavy,
                              int64_t heavy_cap, unsigned long long *ctr) {
    if (graph_bad(ctr)) return;
    const unsigned lane = lane_id();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t c = base + threadIdx.x;
        int64_t du = 0, deg = 0;
        bool core = false;
        if (c < n) {
            du = ooff[c + 1] - ooff[c];
            deg = off[c + 1] - off[c];
            core = core_of && core_of[c] >= 0;
        }
        // V-mode candidates exist only if c has in-neighbours
        const int64_t ncand = du > 0 ? du + (deg > du ? deg : 0) : 0;
        // a core centre with enough candidates per probe-row range is tiled:
        // it goes to the heavy list and gets no visits here
        const bool tiled = core && groups > 0 && ncand >= (int64_t)HEAVY_CAND * groups;
        {
            const unsigned hm = __ballot_sync(FULL, tiled);
            unsigned long long hb = 0;
            if (lane == 0 && hm) hb = atomicAdd(&ctr[C_NHEAVY], (unsigned long long)__popc(hm));
            hb = __shfl_sync(FULL, hb, 0);
            if (tiled) {
                const int64_t slot = (int64_t)hb + __popc(hm & ((1u << lane) - 1u));
                if (slot < heavy_cap) heavy[slot] = (int32_t)c;
                else flag_status(ctr, ST_BADGRAPH);
            }
        }
        if (tiled) core = false;
        // a core centre with little work stays a warp visit: a block visit
        // costs a few block barriers however small it is
        if (core && du <= W_MAX && ncand * du < CORE_MIN_WORK) core = false;
        const bool small = du <= W_MAX && !core;
        const int64_t cnt = (ncand > 0 && !tiled) ? ceil_div(ncand, visit_len(du, !small)) : 0;
        const int64_t my_w = small ? cnt : 0, my_b = (small || core) ? 0 : cnt, my_c = core ? cnt : 0;
        int64_t sw = my_w, sb = my_b, sc = my_c;   // inclusive warp scans
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t yw = __shfl_up_sync(FULL, sw, o), yb = __shfl_up_sync(FULL, sb, o);
            const int64_t yc = __shfl_up_sync(FULL, sc, o);
            if ((int)lane >= o) { sw += yw; sb += yb; sc += yc; }
        }
        unsigned long long bw = 0, bb = 0, bc = 0;
        if (lane == 31) {
            if (sw) bw = atomicAdd(&ctr[C_NWTASK], (unsigned long long)sw);
            if (sb) bb = atomicAdd(&ctr[C_NBTASK], (unsigned long long)sb);
            if (sc) bc = atomicAdd(&ctr[C_NCTASK], (unsigned long long)sc);
        }
        bw = __shfl_sync(FULL, bw, 31);
        bb = __shfl_sync(FULL, bb, 31);
        bc = __shfl_sync(FULL, bc, 31);
        int64_t at = small ? (int64_t)bw + sw - my_w : core ? (int64_t)bc + sc - my_c : (int64_t)bb + sb - my_b;
        for (int64_t i = 0; i < cnt; ++i, ++at) {
            const int64_t slot = (small || core) ? at : cap - 1 - at;
            if (slot >= 0 && slot < cap) (core ? ctasks : tasks)[slot] = ((uint64_t)c << 32) | (uint64_t)i;
            else flag_status(ctr, ST_BADGRAPH);
        }
    }
}

// Row bounds of candidate q of centre c (q < du: U-mode, else V-mode entry
// off[c] + q - du).  len = 0 when the edge is not intersected from c.
struct Cand {
    int64_t rs;     // first probe position (in ocol)
    int64_t jpos;   // V-mode with a chunked centre: position of c in N+(x), else -1
    int len;
    bool vmode;
};

__device__ __forceinline__ Cand load_cand(const int64_t *off, const int32_t *col, const uint32_t *flags,
                                          const int64_t *ooff, const int32_t *ocol, int32_t c, int64_t cb,
                                          int64_t du, int64_t q, bool chunked, int32_t lo_val, int32_t hi_val) {
    Cand r{0, -1, 0, q >= du};
    int32_t x = -1;
    int64_t lim = du;
    if (q < du) {
        x = ocol[cb + q];
    } else {
        const int64_t e = off[c] + (q - du);
        if (!out_bit(flags, e)) x = col[e];
        lim = du - 1;
    }
    if (x < 0) return r;
    int64_t rs = ooff[x], re = ooff[x + 1];
    if (re - rs <= 0 || re - rs > lim) return r;
    if (chunked) {
        const int64_t r0 = rs, r1 = re;
        rs = lower_bound_g(ocol, r0, r1, lo_val);
        re = lower_bound_g(ocol, rs, r1, hi_val == INT_MAX ? hi_val : hi_val + 1);
        if (r.vmode) r.jpos = lower_bound_g(ocol, r0, r1, c);
    }
    r.rs = rs;
    r.len = (int)(re - rs);
    return r;
}

// ------------------------------------------------------------------ membership
//
// The staged set S (sorted ids a[0..cl)) is tested through a one-hash bitmap
// filter of 2^fb bits (2^fb >= 64 cl where shared memory allows, so a miss is
// a false positive with probability <= 1/64).  The filter test is loop-free;
// the positives (triangles plus false positives) are pushed to a per-warp
// queue and resolved 32 at a time through a bucket directory over S: bucket
// b = (id >> shift) - base holds the positions dir[b] .. dir[b+1]-1 of its ids
// in a, about one id per bucket, so a lookup is two shared loads and a short
// scan.

constexpr int QCAP = 64;                 // per-warp queue of filter positives
constexpr int UNROLL = 4;                // ids loaded per lane before the first is probed
constexpr int SHORT_ROW = 96;            // rows up to this length are packed across lanes

struct WarpScratch {
    int64_t qk[QCAP];      // position of the probed id in ocol
    int32_t qw[QCAP];      // probed id
    int32_t qs[QCAP];      // batch slot (candidate lane) of the probe row
    uint32_t rowhits[32];  // hits per candidate of the batch
    int64_t jpos[32];      // V-mode: position of c in the candidate's row
};

// One staged chunk of N+(c) with its filter and directory (shared memory).
struct Staged {
    const int32_t *a;      // sorted ids
    int cl;                // number of ids
    uint32_t *cnt;         // per-id triangle counters (edge c -> a[i])
    const uint32_t *filt;  // 2^fb-bit filter
    int fb;
    const uint16_t *dir;   // nb + 1 bucket starts
    int shift;
    int32_t base;
    int nb;
};

// Bulk prefetch of ids [start, start + count) of a (16-byte aligned, padded to
// a multiple of 16 bytes) id array into L2: one instruction per row, issued
// by one lane; the range is widened to 16-byte boundaries.
__device__ __forceinline__ void l2_prefetch_ids(const int32_t *a, int64_t start, int64_t count) {
    const int64_t a0 = start & ~(int64_t)3, a1 = (start + count + 3) & ~(int64_t)3;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a + a0), "r"((uint32_t)((a1 - a0) * 4))
                 : "memory");
}

__device__ __forceinline__ uint32_t fhash(int32_t w, int fb) {
    return ((uint32_t)w * 0x9E3779B1u) >> (32 - fb);
}

__device__ __forceinline__ int filter_bits(int cl, int fb_max) {
    int fb = 10;
    while (fb < fb_max && (1 << fb) < 64 * cl) ++fb;
    return fb;
}

// Stages a[0..cl) (already in shared memory) into filter and directory with
// threads tid, tid + nthr, ...; the caller clears the filter first and
// synchronises before and after.
__device__ __forceinline__ void index_staged(Staged &S, uint32_t *filt, uint16_t *dir, int nb_max, int tid,
                                             int nthr) {
    const int32_t lo = S.a[0], hi = S.a[S.cl - 1];
    int sh = 0;
    while (((hi >> sh) - (lo >> sh)) >= nb_max) ++sh;
    S.shift = sh;
    S.base = lo >> sh;
    S.nb = (hi >> sh) - S.base + 1;
    for (int i = tid; i < S.cl; i += nthr) {
        const int32_t v = S.a[i];
        const uint32_t h = fhash(v, S.fb);
        atomicOr(&filt[h >> 5], 1u << (h & 31));
        const int b = (v >> sh) - S.base;
        const int bp = i == 0 ? -1 : (S.a[i - 1] >> sh) - S.base;
        for (int x = bp + 1; x <= b; ++x) dir[x] = (uint16_t)i;
        if (i == S.cl - 1)
            for (int x = b + 1; x <= S.nb; ++x) dir[x] = (uint16_t)S.cl;
    }
}

// Position of w in S.a, or -1.
__device__ __forceinline__ int staged_find(const Staged &S, int32_t w) {
    const int b = (w >> S.shift) - S.base;
    if (b < 0 || b >= S.nb) return -1;
    for (int i = S.dir[b], e = S.dir[b + 1]; i < e; ++i) {
        const int32_t v = S.a[i];
        if (v >= w) return v == w ? i : -1;
    }
    return -1;
}

// Resolves queue entries [0, cnt) (cnt <= 32), one per lane.
__device__ __forceinline__ void drain(WarpScratch &ws, int cnt, const Staged &S, uint32_t *t) {
    const int lane = (int)lane_id();
    if (lane < cnt) {
        const int p = staged_find(S, ws.qw[lane]);
        if (p >= 0) {
            atomicAdd(&S.cnt[p], 1u);                 // c -> w
            atomicAdd(&t[ws.qk[lane]], 1u);           // x -> w
            atomicAdd(&ws.rowhits[ws.qs[lane]], 1u);  // x -> c or c -> x, credited per row below
        }
    }
    __syncwarp();
}

// One filter test per lane (w < 0: no id) and the push of the positives to the
// warp's queue, which is drained 32 at a time.  Called by every lane.  An id
// equal to c can only occur in a V-mode row N+(x), where it is the edge x -> c.
__device__ __forceinline__ void probe_step(int32_t w, int64_t k, int slot, int32_t c, const Staged &S,
                                           uint32_t *t, WarpScratch &ws, int &qn) {
    const unsigned lane = lane_id();
    bool pos = false;
    if (w >= 0) {
        if (w == c) ws.jpos[slot] = k;
        const uint32_t h = fhash(w, S.fb);
        pos = (S.filt[h >> 5] >> (h & 31)) & 1u;
    }
    const unsigned pm = __ballot_sync(FULL, pos);
    if (pos) {
        const int at = qn + __popc(pm & ((1u << lane) - 1u));
        ws.qw[at] = w;
        ws.qk[at] = k;
        ws.qs[at] = slot;
    }
    qn += __popc(pm);
    if (qn >= 32) {
        __syncwarp();
        drain(ws, 32, S, t);
        if ((int)lane < qn - 32) {
            ws.qw[lane] = ws.qw[32 + lane];
            ws.qk[lane] = ws.qk[32 + lane];
            ws.qs[lane] = ws.qs[32 + lane];
        }
        qn -= 32;
        __syncwarp();
    }
}

// Membership policy of the hashed staging: filter test, queue, directory.
struct FilterSet {
    static constexpr int ROW_LOADS = UNROLL;   // ids per lane in flight along a long row
    static constexpr int SHORT_LOADS = UNROLL; // ids per lane in flight over packed short rows
    static constexpr int PF_AHEAD = 2;         // long rows pulled into L2 this many rows ahead
    Staged S;
    __device__ __forceinline__ void probe(int32_t w, int64_t k, int slot, int32_t cval, uint32_t *t,
                                          WarpScratch &ws, int &qn) const {
        probe_step(w, k, slot, cval, S, t, ws, qn);
    }
    __device__ __forceinline__ void finish(uint32_t *t, WarpScratch &ws, int &qn) const {
        if (qn) drain(ws, qn, S, t);
        qn = 0;
    }
};

// ------------------------------------------------------------------ core staging
//
// Vertices of degree >= D are numbered 0 .. K-1 in id order (core codes; D is
// the smallest power of two with K <= 2^20), and pv2[j] is the code of ocol[j]
// or -1.  Every id of N+(c) ranks above c, so has degree >= deg(c): for a
// centre of degree >= D all of N+(c) is core, and a chunk of it is staged as
// an exact bitmap over core codes.  A probe is then one shared load and a bit
// test (a non-core id misses at once); a hit's position in the chunk is the
// position of its word's first member, pref[word], plus the members below it
// in the word (codes follow ids, so bit order is position order).  There are
// no false positives and no queue: hits are credited where they are found.
constexpr int CORE_BITS = 20;
constexpr int64_t CORE_CAP = int64_t(1) << CORE_BITS;
constexpr int C_WORDS = (int)(CORE_CAP / 64);        // bitmap words
constexpr int C_CHUNK = 8192;                          // staged ids per chunk (positions fit 16 bits)
constexpr int C_THREADS = 1024;
constexpr int C_WARPS = C_THREADS / 32;
constexpr size_t C_SMEM = (size_t)C_WORDS * 8 + (size_t)C_WORDS * 2 + (size_t)C_CHUNK * 4;

struct CoreScratch {
    uint32_t rowhits[32];  // hits per candidate of the batch
    int64_t jpos[32];      // V-mode: position of c in the candidate's row
};

// Ids per lane in flight along a long row of a core visit: the bitmap test
// is short, so more loads per lane are needed to cover memory latency.  With
// that many in flight, prefetching rows ahead costs; one bulk prefetch of
// the row about to be read still pays (measured on R-MAT scale 26).
constexpr int C_ROW_LOADS = 16;
constexpr int C_SHORT_LOADS = 4;

struct CoreSet {
    static constexpr int ROW_LOADS = C_ROW_LOADS;
    static constexpr int SHORT_LOADS = C_SHORT_LOADS;
    static constexpr int PF_AHEAD = 0;
    const unsigned long long *bm;   // C_WORDS words, members of the staged chunk
    const uint16_t *pref;           // per word holding members: position of its first member
    uint32_t *cnt;                  // per position: triangles on c -> member
    __device__ __forceinline__ void probe(int32_t w, int64_t k, int slot, int32_t cval, uint32_t *t,
                                          CoreScratch &ws, int &) const {
        if (w < 0) return;
        if (w == cval) ws.jpos[slot] = k;
        const unsigned long long word = bm[w >> 6];
        const unsigned sh = (unsigned)w & 63u;
        if ((word >> sh) & 1ull) {
            const int p = (int)pref[w >> 6] + __popcll(word & ((1ull << sh) - 1ull));
            atomicAdd(&cnt[p], 1u);                   // c -> w
            atomicAdd(&t[k], 1u);                     // x -> w
            atomicAdd(&ws.rowhits[slot], 1u);         // x -> c or c -> x, credited per row
        }
    }
    __device__ __forceinline__ void finish(uint32_t *, CoreScratch &, int &) const {}
};

// One warp processes candidates q0 .. min(q0 + 32, qend) - 1 of centre c (a batch)
// against the staged chunk S.  Rows longer than SHORT_ROW are read one at a
// time by the whole warp; the shorter ones are laid end to end over the lanes
// (each lane finds the row of its id by a 5-step shuffle search over the
// rows' start offsets).  U-mode row hits are credited to c -> x through
// S.cnt[q] when uv_local (the whole N+(c) is staged) or through t otherwise;
// V-mode row hits to x -> c at the position of c in N+(x).
template <class Set, class Scratch>
__device__ __forceinline__ void process_batch(const int64_t *off, const int32_t *col, const uint32_t *flags,
                                              const int64_t *ooff, const int32_t *ocol, const int32_t *pv,
                                              uint32_t *t, int32_t c, int32_t cval, int64_t cb, int64_t du,
                                              int64_t q0, int64_t qend, bool chunked, int32_t lo_id, int32_t hi_id,
                                              const Set &S, uint32_t *scnt, bool uv_local, Scratch &ws,
                                              unsigned long long *ctr) {
    const unsigned lane = lane_id();
    const int64_t q = q0 + lane;
    Cand cd{0, -1, 0, false};
    if (q < qend) cd = load_cand(off, col, flags, ooff, ocol, c, cb, du, q, chunked, lo_id, hi_id);
    ws.rowhits[lane] = 0u;
    ws.jpos[lane] = cd.jpos;
    __syncwarp();
    int qn = 0;
    // long rows, one after another; the first PF_AHEAD are pulled into L2 now
    // and each row started pulls the one PF_AHEAD rows later (with PF_AHEAD
    // = 0, itself: one bulk request for the row the warp is about to read)
    unsigned todo = __ballot_sync(FULL, cd.len > SHORT_ROW);
    unsigned pf = todo;
    {
        constexpr int AHEAD = Set::PF_AHEAD;
        const unsigned rank = __popc(todo & ((1u << lane) - 1u));
        if (((todo >> lane) & 1u) && rank < AHEAD) l2_prefetch_ids(pv, cd.rs, cd.len);
        for (int i = 0; i < AHEAD && pf; ++i) pf &= pf - 1;
    }
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        if (pf) {
            if ((int)lane == __ffs(pf) - 1) l2_prefetch_ids(pv, cd.rs, cd.len);
            pf &= pf - 1;
        }
        const int64_t rs = __shfl_sync(FULL, cd.rs, src);
        const int len = __shfl_sync(FULL, cd.len, src);
        constexpr int LOADS = Set::ROW_LOADS;
        for (int base = 0; base < len; base += 32 * LOADS) {
            int32_t w[LOADS];
#pragma unroll
            for (int j = 0; j < LOADS; ++j) {    // all loads issued before any is used
                const int i = base + 32 * j + (int)lane;
                w[j] = i < len ? __ldg(&pv[rs + i]) : -1;
            }
#pragma unroll
            for (int j = 0; j < LOADS; ++j) S.probe(w[j], rs + base + 32 * j + (int)lane, src, cval, t, ws, qn);
        }
    }
    // short rows, packed end to end
    const int slen = (cd.len > 0 && cd.len <= SHORT_ROW) ? cd.len : 0;
    int incl = slen;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if ((int)lane >= o) incl += y;
    }
    const int sstart = incl - slen;
    const int stotal = __shfl_sync(FULL, incl, 31);
    constexpr int SLOADS = Set::SHORT_LOADS;
    for (int e0 = 0; e0 < stotal; e0 += 32 * SLOADS) {
        int32_t w[SLOADS];
        int64_t kk[SLOADS];
        int own[SLOADS];
#pragma unroll
        for (int j = 0; j < SLOADS; ++j) {
            const int e = e0 + 32 * j + (int)lane;
            int p = 0;                           // last lane whose row starts at or before e
#pragma unroll
            for (int st = 16; st >= 1; st >>= 1) {
                const int sp = __shfl_sync(FULL, sstart, p + st);
                if (sp <= e) p += st;
            }
            const int64_t prs = __shfl_sync(FULL, cd.rs, p);
            const int pst = __shfl_sync(FULL, sstart, p);
            own[j] = p;
            kk[j] = prs + (e - pst);
            w[j] = e < stotal ? __ldg(&pv[kk[j]]) : -1;
        }
#pragma unroll
        for (int j = 0; j < SLOADS; ++j) S.probe(w[j], kk[j], own[j], cval, t, ws, qn);
    }
    __syncwarp();
    S.finish(t, ws, qn);
    const uint32_t hits = ws.rowhits[lane];
    if (hits) {
        if (q < du) {
            if (uv_local) atomicAdd(&scnt[q], hits);        // c -> x (whole N+(c) staged)
            else atomicAdd(&t[cb + q], hits);               // c -> x
        } else {
            const int64_t jp = ws.jpos[lane];
            if (jp >= 0) atomicAdd(&t[jp], hits);           // x -> c
            else flag_status(ctr, ST_BADGRAPH);
        }
    }
    __syncwarp();
}

// ------------------------------------------------------------------ warp visits

constexpr int W_FB = 14;                             // warp filter: 2^14 bits = 2 KB
constexpr int W_DIR = 128;                           // warp directory buckets
constexpr int W_SLICE = (1 << W_FB) / 32 + 2 * W_MAX + (W_DIR + 2) / 2;   // words per warp

// One warp, one visit of a centre with d+(c) <= W_MAX, on the warp's own
// slice of shared memory: filter, ids, counters, directory.
__device__ __forceinline__ void warp_visit(const int64_t *off, const int32_t *col, const uint32_t *flags,
                                           const int64_t *ooff, const int32_t *ocol, uint32_t *t, uint64_t task,
                                           int32_t *slice, WarpScratch &ws, unsigned long long *ctr) {
    const unsigned lane = lane_id();
    uint32_t *filt = reinterpret_cast<uint32_t *>(slice);
    int32_t *s_a = slice + (1 << W_FB) / 32;
    uint32_t *s_cnt = reinterpret_cast<uint32_t *>(s_a + W_MAX);
    uint16_t *dir = reinterpret_cast<uint16_t *>(s_a + 2 * W_MAX);
    const int32_t c = (int32_t)(task >> 32);
    const int64_t vis = (int64_t)(task & VIS_MASK);
    const int64_t cb = ooff[c];
    const int du = (int)(ooff[c + 1] - cb);
    const int64_t deg = off[c + 1] - off[c];
    const int64_t ncand = du + (deg > du ? deg : 0);
    const int64_t vl = visit_len(du, false);
    const int64_t qbeg = vis * vl, qend = min(ncand, qbeg + vl);
    Staged S{s_a, du, s_cnt, filt, filter_bits(du, W_FB), dir, 0, 0, 0};
    for (int i = (int)lane; i < (1 << S.fb) / 32; i += 32) filt[i] = 0u;
    for (int i = (int)lane; i < du; i += 32) {
        s_a[i] = ocol[cb + i];
        s_cnt[i] = 0u;
    }
    __syncwarp();
    index_staged(S, filt, dir, W_DIR, (int)lane, 32);
    __syncwarp();
    for (int64_t q0 = qbeg; q0 < qend; q0 += 32)
        process_batch(off, col, flags, ooff, ocol, ocol, t, c, c, cb, du, q0, qend, false, S.a[0], S.a[S.cl - 1],
                      FilterSet{S}, S.cnt, true, ws, ctr);
    __syncwarp();
    for (int i = (int)lane; i < du; i += 32) {
        const uint32_t cv = s_cnt[i];
        if (cv) atomicAdd(&t[cb + i], cv);
    }
    __syncwarp();
}

// ------------------------------------------------------------------ block visits

constexpr int B_FB = 18;                             // block filter: 2^18 bits = 32 KB
constexpr int B_DIR = S_CHUNK;                       // block directory buckets
constexpr int B_WORDS = (1 << B_FB) / 32 + 2 * S_CHUNK + (B_DIR + 2) / 2;
static_assert(B_WARPS * W_SLICE <= B_WORDS, "warp slices must fit the block buffer");

// Persistent kernel: every block first drains the block-visit list (pulled
// from a global counter, the block's warps taking batches of 32 candidates
// from a shared counter), then its warps take warp visits in groups of W_GRAB.
__global__ void __launch_bounds__(B_THREADS, 2)
k_support(const int64_t *off, const int32_t *col, const uint32_t *flags, const int64_t *ooff,
          const int32_t *ocol, uint32_t *t, const uint64_t *tasks, int64_t cap, unsigned long long *ctr) {
    extern __shared__ int32_t smem[];
    uint32_t *filt = reinterpret_cast<uint32_t *>(smem);              // 2^B_FB bits
    int32_t *s_a = smem + (1 << B_FB) / 32;                           // S_CHUNK ids
    uint32_t *s_cnt = reinterpret_cast<uint32_t *>(s_a + S_CHUNK);      // S_CHUNK counters
    uint16_t *dir = reinterpret_cast<uint16_t *>(s_a + 2 * S_CHUNK);    // B_DIR + 1 bucket starts
    __shared__ WarpScratch s_ws[B_WARPS];
    __shared__ long long s_item;
    __shared__ int s_next;
    if (graph_bad(ctr)) return;
    const unsigned lane = lane_id();
    const int wi = threadIdx.x >> 5;
    WarpScratch &ws = s_ws[wi];
    const int64_t ntasks = (int64_t)ctr[C_NBTASK];
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(&ctr[C_NEXT], 1ull);
        __syncthreads();
        const int64_t it = s_item;
        __syncthreads();
        if (it >= ntasks) break;
        const uint64_t task = tasks[cap - 1 - it];
        const int32_t c = (int32_t)(task >> 32);
        const int64_t vis = (int64_t)(task & VIS_MASK);
        const int64_t cb = ooff[c];
        const int64_t du = ooff[c + 1] - cb;
        const int64_t deg = off[c + 1] - off[c];
        const int64_t ncand = du + (deg > du ? deg : 0);
        const int64_t vl = visit_len(du, true);
        const int64_t qbeg = vis * vl, qend = min(ncand, qbeg + vl);
        const bool chunked = du > S_CHUNK;
        for (int64_t c0 = 0; c0 < du; c0 += S_CHUNK) {
            const int cl = (int)min((int64_t)S_CHUNK, du - c0);
            Staged S{s_a, cl, s_cnt, filt, filter_bits(cl, B_FB), dir, 0, 0, 0};
            for (int i = threadIdx.x; i < (1 << S.fb) / 32; i += B_THREADS) filt[i] = 0u;
            for (int i = threadIdx.x; i < cl; i += B_THREADS) {
                s_a[i] = ocol[cb + c0 + i];
                s_cnt[i] = 0u;
            }
            if (threadIdx.x == 0) s_next = 0;
            __syncthreads();
            index_staged(S, filt, dir, B_DIR, threadIdx.x, B_THREADS);
            __syncthreads();
            for (;;) {
                int b = 0;
                if (lane == 0) b = atomicAdd(&s_next, B_BATCH);
                b = __shfl_sync(FULL, b, 0);
                if (qbeg + b >= qend) break;
                process_batch(off, col, flags, ooff, ocol, ocol, t, c, c, cb, du, qbeg + b,
                              min(qend, qbeg + b + B_BATCH), chunked, S.a[0],
                              S.a[S.cl - 1], FilterSet{S}, S.cnt, false, ws, ctr);
            }
            __syncthreads();
            for (int i = threadIdx.x; i < cl; i += B_THREADS) {
                const uint32_t cv = s_cnt[i];
                if (cv) atomicAdd(&t[cb + c0 + i], cv);
            }
            __syncthreads();
        }
    }
    // phase 2: warp visits on per-warp slices of the same shared memory
    int32_t *slice = smem + wi * W_SLICE;
    const int64_t nw = (int64_t)ctr[C_NWTASK];
    for (;;) {
        unsigned long long g0 = 0;
        if (lane == 0) g0 = atomicAdd(&ctr[C_NEXTW], (unsigned long long)W_GRAB);
        g0 = __shfl_sync(FULL, g0, 0);
        if ((int64_t)g0 >= nw) break;
        const int64_t g1 = min(nw, (int64_t)g0 + W_GRAB);
        for (int64_t it = (int64_t)g0; it < g1; ++it)
            warp_visit(off, col, flags, ooff, ocol, t, tasks[it], slice, ws, ctr);
    }
}

__global__ void k_reset_support_counters(unsigned long long *ctr) {
    ctr[C_NWTASK] = 0;
    ctr[C_NBTASK] = 0;
    ctr[C_NEXT] = 0;
    ctr[C_NEXTW] = 0;
    ctr[C_NCTASK] = 0;
    ctr[C_NEXTC] = 0;
    ctr[C_NHEAVY] = 0;
    ctr[C_NEXTT] = 0;
}

// ------------------------------------------------------------------ core labels

// hist[b] = vertices of degree in [2^b, 2^(b+1)) (b < 32); hist[32] = degree 0.
__global__ void k_degree_log_hist(const int32_t *deg, int64_t n, unsigned long long *hist) {
    __shared__ unsigned int h[33];
    if (threadIdx.x < 33) h[threadIdx.x] = 0u;
    __syncthreads();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int d = deg[v];
        atomicAdd(&h[d > 0 ? 31 - __clz(d) : 32], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 33 && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], (unsigned long long)h[threadIdx.x]);
}

// meta[0] = D, the smallest power of two with at most CORE_CAP vertices of
// degree >= D (0: no core); meta[1] = that count K.
__global__ void k_core_pick(const unsigned long long *hist, long long *meta) {
    unsigned long long k = 0;
    int best = -1;
    unsigned long long kb = 0;
    for (int b = 31; b >= 0; --b) {
        k += hist[b];
        if (k > (unsigned long long)CORE_CAP) break;
        best = b;
        kb = k;
    }
    meta[0] = (best >= 0 && kb > 0) ? (1ll << best) : 0ll;
    meta[1] = (best >= 0) ? (long long)kb : 0ll;
}

// Per TILE of vertices: the number of core vertices (degree >= D).
__global__ void k_core_count(const int32_t *deg, int64_t n, const long long *meta, int64_t *tcnt) {
    const long long D = meta[0];
    const int64_t v0 = (int64_t)blockIdx.x * TILE;
    int c = 0;
    for (int i = 0; i < TILE_ITEMS; ++i) {
        const int64_t v = v0 + (int64_t)i * TILE_THREADS + threadIdx.x;
        if (v < n && D > 0 && deg[v] >= D) ++c;
    }
    c = warp_sum(c);
    __shared__ int s_c[TILE_THREADS / 32];
    if (lane_id() == 0) s_c[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < TILE_THREADS / 32; ++w) t += s_c[w];
        tcnt[blockIdx.x] = t;
    }
}

// core_of[v] = rank of v among the core vertices in id order, or -1.
__global__ void k_core_fill(const int32_t *deg, int64_t n, const long long *meta, const int64_t *tbase,
                            int32_t *core_of) {
    const long long D = meta[0];
    const int64_t v0 = (int64_t)blockIdx.x * TILE;
    __shared__ int s_w[TILE_THREADS / 32];
    int64_t run = tbase[blockIdx.x];
    for (int i = 0; i < TILE_ITEMS; ++i) {     // one row of TILE_THREADS vertices at a time, in id order
        const int64_t v = v0 + (int64_t)i * TILE_THREADS + threadIdx.x;
        const bool is_core = v < n && D > 0 && deg[v] >= D;
        const unsigned b = __ballot_sync(FULL, is_core);
        if (lane_id() == 0) s_w[threadIdx.x >> 5] = __popc(b);
        __syncthreads();
        int before = 0, row = 0;
        for (int w = 0; w < TILE_THREADS / 32; ++w) {
            before += w < (int)(threadIdx.x >> 5) ? s_w[w] : 0;
            row += s_w[w];
        }
        if (v < n) core_of[v] = is_core ? (int32_t)(run + before + __popc(b & ((1u << lane_id()) - 1u))) : -1;
        run += row;
        __syncthreads();
    }
}

// pv2[j] = core code of ocol[j], or -1.
__global__ void k_core_codes(const int32_t *ocol, int64_t m, const int32_t *core_of, int32_t *pv2) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        pv2[j] = core_of[ocol[j]];
}

// ------------------------------------------------------------------ core visits

// Persistent kernel, one 1024-thread block per SM: block visits of core
// centres.  Per chunk of N+(c): set the members' bits and their words' first
// positions, run the batches, flush the counters and clear the bits again.
__global__ void __launch_bounds__(C_THREADS, 1)
k_support_core(const int64_t *off, const int32_t *col, const uint32_t *flags, const int64_t *ooff,
               const int32_t *ocol, const int32_t *pv2, const int32_t *core_of, uint32_t *t, const uint64_t *ctasks,
               unsigned long long *ctr) {
    extern __shared__ unsigned long long csm[];
    unsigned long long *bm = csm;                                           // C_WORDS
    uint16_t *pref = reinterpret_cast<uint16_t *>(bm + C_WORDS);            // C_WORDS
    uint32_t *s_cnt = reinterpret_cast<uint32_t *>(pref + C_WORDS);         // C_CHUNK
    __shared__ CoreScratch s_cws[C_WARPS];
    __shared__ long long s_item;
    __shared__ int s_next;
    if (graph_bad(ctr)) return;
    const unsigned lane = lane_id();
    CoreScratch &ws = s_cws[threadIdx.x >> 5];
    for (int i = threadIdx.x; i < C_WORDS; i += C_THREADS) bm[i] = 0ull;
    for (int i = threadIdx.x; i < C_CHUNK; i += C_THREADS) s_cnt[i] = 0u;
    __syncthreads();
    const int64_t ntasks = (int64_t)ctr[C_NCTASK];
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(&ctr[C_NEXTC], 1ull);
        __syncthreads();
        const int64_t it = s_item;
        __syncthreads();
        if (it >= ntasks) break;
        const uint64_t task = ctasks[it];
        const int32_t c = (int32_t)(task >> 32);
        const int64_t vis = (int64_t)(task & VIS_MASK);
        const int64_t cb = ooff[c];
        const int64_t du = ooff[c + 1] - cb;
        const int64_t deg = off[c + 1] - off[c];
        const int64_t ncand = du + (deg > du ? deg : 0);
        const int64_t vl = visit_len(du, true);
        const int64_t qbeg = vis * vl, qend = min(ncand, qbeg + vl);
        const bool chunked = du > C_CHUNK;
        const int32_t cval = core_of[c];
        for (int64_t c0 = 0; c0 < du; c0 += C_CHUNK) {
            const int cl = (int)min((int64_t)C_CHUNK, du - c0);
            for (int i = threadIdx.x; i < cl; i += C_THREADS) {
                const int32_t w = pv2[cb + c0 + i];
                if (w >= 0) atomicOr(&bm[w >> 6], 1ull << (w & 63));
                else flag_status(ctr, ST_BADGRAPH);   // a core centre has only core out-neighbours
            }
            if (threadIdx.x == 0) s_next = 0;
            __syncthreads();
            for (int i = threadIdx.x; i < cl; i += C_THREADS) {
                const int32_t w = pv2[cb + c0 + i];
                if (w >= 0 && !(i > 0 && (pv2[cb + c0 + i - 1] >> 6) == (w >> 6)))   // the word's first member
                    pref[w >> 6] = (uint16_t)i;
            }
            __syncthreads();
            const CoreSet S{bm, pref, s_cnt};
            const int32_t lo_id = ocol[cb + c0], hi_id = ocol[cb + c0 + cl - 1];
            for (;;) {
                int b = 0;
                if (lane == 0) b = atomicAdd(&s_next, C_BATCH);
                b = __shfl_sync(FULL, b, 0);
                if (qbeg + b >= qend) break;
                process_batch(off, col, flags, ooff, ocol, pv2, t, c, cval, cb, du, qbeg + b,
                              min(qend, qbeg + b + C_BATCH), chunked, lo_id, hi_id, S, s_cnt, false, ws, ctr);
            }
            __syncthreads();
            for (int i = threadIdx.x; i < cl; i += C_THREADS) {
                const uint32_t cv = s_cnt[i];
                if (cv) {
                    atomicAdd(&t[cb + c0 + i], cv);
                    s_cnt[i] = 0u;
                }
                const int32_t w = pv2[cb + c0 + i];
                if (w >= 0) bm[w >> 6] = 0ull;
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------ core visit order

__device__ __forceinline__ int order_class(const int64_t *ooff, uint64_t task) {
    const int32_t c = (int32_t)(task >> 32);
    const int64_t d = min(ooff[c + 1] - ooff[c], (int64_t)ORDER_CLASSES - 1);
    return CORE_ORDER == 1 ? ORDER_CLASSES - 1 - (int)d : (int)d;
}

__global__ void k_order_count(const uint64_t *ctasks, const int64_t *ooff, unsigned long long *hist,
                              const unsigned long long *ctr) {
    const int64_t nt = (int64_t)ctr[C_NCTASK];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&hist[order_class(ooff, ctasks[i])], 1ull);
}

// out[base[class] + cursor]: the visits grouped by class, classes ascending.
__global__ void k_order_fill(const uint64_t *ctasks, const int64_t *ooff, const int64_t *base,
                             unsigned long long *cursor, uint64_t *out, int64_t cap, unsigned long long *ctr) {
    const int64_t nt = (int64_t)ctr[C_NCTASK];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t task = ctasks[i];
        const int cls = order_class(ooff, task);
        const int64_t pos = base[cls] + (int64_t)atomicAdd(&cursor[cls], 1ull);
        if (pos < cap) out[pos] = task;
        else flag_status(ctr, ST_BADGRAPH);
    }
}

// ------------------------------------------------------------------ probe-row tiling
//
// The core kernel above reads a centre's candidate rows wherever they lie, so
// every probe row is fetched from DRAM once per centre probing it, and every
// third-edge credit is a random read-modify-write of a DRAM-resident counter.
// The tiled kernel visits a heavy centre once per vertex-id range ("group")
// of about equal probe-id volume (set by tec_set_support_tiling), all visits of group 0
// first: the centres visited at the same time probe only the rows of one
// group, which stay in L2 with their counters.  A visit covers the candidates
// of one group, which are a contiguous slice of the centre's oriented row
// (U-mode) and of its symmetric row (V-mode), both sorted by id.  The counts
// do not change: every oriented edge is still intersected exactly once, from
// the same side.

// gb[g] = first vertex of group g: the smallest v with ooff[v] >= g m / groups
// (gb[0] = 0, gb[groups] = n).
__global__ void k_tile_groups(const int64_t *ooff, int64_t n, int64_t m, int groups, int32_t *gb) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g > groups) return;
    if (g == 0 || g == groups) {
        gb[g] = g == 0 ? 0 : (int32_t)n;
        return;
    }
    const int64_t target = (int64_t)((__int128)m * g / groups);
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (ooff[mid] < target) lo = mid + 1; else hi = mid;
    }
    gb[g] = (int32_t)lo;
}

// One warp per tiled centre h: bu[g * hcap + h] = first position of N+(c)
// holding an id >= gb[g], bv[...] the same in c's symmetric row (g = 0..groups).
__global__ void k_tile_bounds(const int64_t *off, const int32_t *col, const int64_t *ooff, const int32_t *ocol,
                              const int32_t *heavy, int64_t hcap, int groups, const int32_t *gb, int32_t *bu,
                              int32_t *bv, const unsigned long long *ctr) {
    const int64_t H = (int64_t)ctr[C_NHEAVY];
    const int64_t warps = (int64_t)gridDim.x * blockDim.x / 32;
    for (int64_t h = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; h < H && h < hcap; h += warps) {
        const int32_t c = heavy[h];
        const int64_t cb = ooff[c], ce = ooff[c + 1], sb = off[c], se = off[c + 1];
        for (int g = (int)lane_id(); g <= groups; g += 32) {
            const int32_t x = gb[g];
            bu[(int64_t)g * hcap + h] = (int32_t)(lower_bound_g(ocol, cb, ce, x) - cb);
            bv[(int64_t)g * hcap + h] = (int32_t)(lower_bound_g(col, sb, se, x) - sb);
        }
    }
}

__device__ __forceinline__ bool tile_item_nonempty(const int32_t *bu, const int32_t *bv, int64_t hcap, int g,
                                                   int64_t h) {
    const int64_t a = (int64_t)g * hcap + h, b = a + hcap;
    return bu[b] > bu[a] || bv[b] > bv[a];
}

// icnt[g] = number of tiled centres with candidates in group g.  Grid: x over
// centres, y over groups.
__global__ void k_tile_count(const int32_t *bu, const int32_t *bv, int64_t hcap, int groups, int64_t *icnt,
                             const unsigned long long *ctr) {
    const int64_t H = min((int64_t)ctr[C_NHEAVY], hcap);
    for (int g = blockIdx.y; g < groups; g += gridDim.y) {
        int c = 0;
        for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < H; h += (int64_t)gridDim.x * blockDim.x)
            c += tile_item_nonempty(bu, bv, hcap, g, h) ? 1 : 0;
        c = warp_sum(c);
        if (lane_id() == 0 && c) atomicAdd((unsigned long long *)&icnt[g], (unsigned long long)c);
    }
}

// Writes the items of group g at ioff[g] + (a per-group cursor), range-major.
__global__ void k_tile_fill(const int32_t *bu, const int32_t *bv, int64_t hcap, int groups, const int64_t *ioff,
                            int64_t *cursor, uint32_t *items, int64_t item_cap, unsigned long long *ctr) {
    const int64_t H = min((int64_t)ctr[C_NHEAVY], hcap);
    const unsigned lane = lane_id();
    for (int g = blockIdx.y; g < groups; g += gridDim.y) {
        for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < H; base += (int64_t)gridDim.x * blockDim.x) {
            const int64_t h = base + threadIdx.x;
            const bool ne = h < H && tile_item_nonempty(bu, bv, hcap, g, h);
            const unsigned bm = __ballot_sync(FULL, ne);
            unsigned long long at = 0;
            if (lane == 0 && bm) at = atomicAdd((unsigned long long *)&cursor[g], (unsigned long long)__popc(bm));
            at = __shfl_sync(FULL, at, 0);
            if (ne) {
                const int64_t slot = ioff[g] + (int64_t)at + __popc(bm & ((1u << lane) - 1u));
                if (slot < item_cap) items[slot] = ((uint32_t)g << CORE_BITS) | (uint32_t)h;
                else flag_status(ctr, ST_BADGRAPH);
            }
        }
    }
}

// Persistent kernel, one 1024-thread block per SM: the tiled items in order.
// Per item (group g, centre c): per chunk of N+(c), stage the bitmap as the
// core kernel does, run the batches of the group's U-mode slice [u0, u1) and
// V-mode slice [v0, v1) of the candidates, flush the centre's counters and
// clear the bits.
__global__ void __launch_bounds__(C_THREADS, 1)
k_support_tiled(const int64_t *off, const int32_t *col, const uint32_t *flags, const int64_t *ooff,
                const int32_t *ocol, const int32_t *pv2, const int32_t *core_of, uint32_t *t, const int32_t *heavy,
                int64_t hcap, const int32_t *bu, const int32_t *bv, const uint32_t *items, const int64_t *ioff,
                int groups, unsigned long long *ctr) {
    extern __shared__ unsigned long long csm[];
    unsigned long long *bm = csm;                                           // C_WORDS
    uint16_t *pref = reinterpret_cast<uint16_t *>(bm + C_WORDS);            // C_WORDS
    uint32_t *s_cnt = reinterpret_cast<uint32_t *>(pref + C_WORDS);         // C_CHUNK
    __shared__ CoreScratch s_cws[C_WARPS];
    __shared__ long long s_item;
    __shared__ int s_next;
    if (graph_bad(ctr)) return;
    const unsigned lane = lane_id();
    CoreScratch &ws = s_cws[threadIdx.x >> 5];
    for (int i = threadIdx.x; i < C_WORDS; i += C_THREADS) bm[i] = 0ull;
    for (int i = threadIdx.x; i < C_CHUNK; i += C_THREADS) s_cnt[i] = 0u;
    __syncthreads();
    const int64_t nitems = ioff[groups];
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(&ctr[C_NEXTT], 1ull);
        __syncthreads();
        const int64_t it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const uint32_t code = items[it];
        const int g = (int)(code >> CORE_BITS);
        const int64_t h = (int64_t)(code & (uint32_t)(CORE_CAP - 1));
        const int32_t c = heavy[h];
        const int64_t cb = ooff[c];
        const int64_t du = ooff[c + 1] - cb;
        const int64_t a = (int64_t)g * hcap + h;
        const int64_t u0 = bu[a], u1 = bu[a + hcap], v0 = bv[a], v1 = bv[a + hcap];
        const int64_t nbu = ceil_div(u1 - u0, (int64_t)T_BATCH), nb = nbu + ceil_div(v1 - v0, (int64_t)T_BATCH);
        const bool chunked = du > C_CHUNK;
        const int32_t cval = core_of[c];
        for (int64_t c0 = 0; c0 < du; c0 += C_CHUNK) {
            const int cl = (int)min((int64_t)C_CHUNK, du - c0);
            for (int i = threadIdx.x; i < cl; i += C_THREADS) {
                const int32_t w = pv2[cb + c0 + i];
                if (w >= 0) atomicOr(&bm[w >> 6], 1ull << (w & 63));
                else flag_status(ctr, ST_BADGRAPH);   // a core centre has only core out-neighbours
            }
            if (threadIdx.x == 0) s_next = 0;
            __syncthreads();
            for (int i = threadIdx.x; i < cl; i += C_THREADS) {
                const int32_t w = pv2[cb + c0 + i];
                if (w >= 0 && !(i > 0 && (pv2[cb + c0 + i - 1] >> 6) == (w >> 6)))   // the word's first member
                    pref[w >> 6] = (uint16_t)i;
            }
            __syncthreads();
            const CoreSet S{bm, pref, s_cnt};
            const int32_t lo_id = ocol[cb + c0], hi_id = ocol[cb + c0 + cl - 1];
            for (;;) {
                int b = 0;
                if (lane == 0) b = atomicAdd(&s_next, 1);
                b = __shfl_sync(FULL, b, 0);
                if (b >= nb) break;
                // batch b: of the U-mode slice first, then of the V-mode slice
                // (candidate q >= du is entry q - du of the symmetric row)
                const int64_t q0 = b < nbu ? u0 + (int64_t)b * T_BATCH : du + v0 + (int64_t)(b - nbu) * T_BATCH;
                const int64_t qe = b < nbu ? u1 : du + v1;
                process_batch(off, col, flags, ooff, ocol, pv2, t, c, cval, cb, du, q0, min(qe, q0 + T_BATCH),
                              chunked, lo_id, hi_id, S, s_cnt, false, ws, ctr);
            }
            __syncthreads();
            for (int i = threadIdx.x; i < cl; i += C_THREADS) {
                const uint32_t cv = s_cnt[i];
                if (cv) {
                    atomicAdd(&t[cb + c0 + i], cv);
                    s_cnt[i] = 0u;
                }
                const int32_t w = pv2[cb + c0 + i];
                if (w >= 0) bm[w >> 6] = 0ull;
            }
            __syncthreads();
        }
    }
}

}  // namespace

int64_t support_task_capacity(int64_t n, int64_t nnz) {
    // per vertex at most ceil((d+ + deg) / 256) <= 1 + (d+ + deg) / 256 visits
    return n + (nnz + nnz / 2) / 256 + 64;
}

cudaError_t launch_core_labels(const int32_t *deg, int64_t n, const int32_t *ocol, int64_t m,
                               unsigned long long *hist, long long *meta, int64_t *tcnt, int64_t *tbase,
                               int64_t *bsum, int32_t *core_of, int32_t *pv2, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(hist, 0, 33 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        const int64_t g = ceil_div(n, 256);
        k_degree_log_hist<<<(unsigned)(g < 4096 ? g : 4096), 256, 0, s>>>(deg, n, hist);
    }
    k_core_pick<<<1, 1, 0, s>>>(hist, meta);
    const int64_t ntiles = ceil_div(n > 0 ? n : 1, (int64_t)TILE);
    k_core_count<<<(unsigned)ntiles, TILE_THREADS, 0, s>>>(deg, n, meta, tcnt);
    if ((e = scan_exclusive_i64(tcnt, ntiles, tbase, bsum, s)) != cudaSuccess) return e;
    k_core_fill<<<(unsigned)ntiles, TILE_THREADS, 0, s>>>(deg, n, meta, tbase, core_of);
    if (m > 0) {
        const int64_t g = ceil_div(m, 256);
        k_core_codes<<<(unsigned)(g < 65536 ? g : 65536), 256, 0, s>>>(ocol, m, core_of, pv2);
    }
    count_launches(n > 0 ? 6 : 5);
    return cudaGetLastError();
}

int64_t core_order_classes() { return CORE_ORDER != 0 ? ORDER_CLASSES : 0; }

// Measured on R-MAT scale 26 (1 GB300): 2.57 s untiled against 3.0-18 s for
// every tiled setting tried (8..248 ranges, 1..16 candidates per batch, 8 or
// 64 candidates per range): the per-visit start-up (dependent loads of the
// item, the centre and its first rows, and the block barriers) outweighs
// the L2 reuse.  So the automatic rule leaves tiling off; a range count set
// with tec_set_support_tiling still runs it.
int support_auto_groups(int64_t m) {
    (void)m;
    return 0;
}

int64_t support_heavy_capacity(int64_t n) { return std::max<int64_t>(1, std::min<int64_t>(n, CORE_CAP)); }

int64_t support_item_capacity(int64_t nnz, int groups, int64_t heavy_cap) {
    // a tiled centre has ncand >= HEAVY_CAND * groups candidates and
    // sum(ncand) <= m + nnz, so items <= heavy * groups <= 1.5 nnz / HEAVY_CAND
    if (groups <= 0) return 0;
    const int64_t by_cand = (nnz + nnz / 2) / HEAVY_CAND + 1;
    return std::max<int64_t>(1, std::min<int64_t>(heavy_cap * groups, by_cand));
}

cudaError_t launch_support(const int64_t *off, const int32_t *col, const uint32_t *flags, const int64_t *ooff,
                           const int32_t *ocol, int64_t n, int64_t m, uint32_t *t, uint64_t *tasks,
                           int64_t task_cap, unsigned long long *ctr, int num_sms, cudaStream_t s,
                           const int32_t *pv2, const int32_t *core_of, uint64_t *ctasks,
                           const SupportTiling &tl, const CoreOrder &order) {
    if (m > 0) {
        cudaError_t e = cudaMemsetAsync(t, 0, (size_t)m * sizeof(uint32_t), s);
        if (e != cudaSuccess) return e;
    }
    if (n <= 0 || m <= 0) return cudaSuccess;
    const int bsmem = B_WORDS * (int)sizeof(int32_t);
    cudaError_t e = cudaFuncSetAttribute(k_support, cudaFuncAttributeMaxDynamicSharedMemorySize, bsmem);
    if (e != cudaSuccess) return e;
    const bool core = pv2 && core_of && ctasks;
    const int groups = (core && tl.groups > 0 && tl.items) ? tl.groups : 0;
    if (core) {
        e = cudaFuncSetAttribute(k_support_core, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C_SMEM);
        if (e != cudaSuccess) return e;
    }
    if (groups) {
        e = cudaFuncSetAttribute(k_support_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C_SMEM);
        if (e != cudaSuccess) return e;
    }
    k_reset_support_counters<<<1, 1, 0, s>>>(ctr);
    {
        const int64_t g = ceil_div(n, 256);
        k_make_visits<<<(unsigned)(g < 65536 ? g : 65536), 256, 0, s>>>(
            off, ooff, n, tasks, task_cap, core ? core_of : nullptr, ctasks, groups, tl.heavy, tl.heavy_cap, ctr);
    }
    int launched = 2;
    if (groups) {
        k_tile_groups<<<(unsigned)ceil_div(groups + 1, 256), 256, 0, s>>>(ooff, n, m, groups, tl.gb);
        const int64_t hw = ceil_div(tl.heavy_cap, 8);    // 8 warps of 256-thread blocks
        k_tile_bounds<<<(unsigned)std::min<int64_t>(std::max<int64_t>(hw, 1), 8192), 256, 0, s>>>(
            off, col, ooff, ocol, tl.heavy, tl.heavy_cap, groups, tl.gb, tl.bu, tl.bv, ctr);
        if ((e = cudaMemsetAsync(tl.icnt, 0, (size_t)(groups + 1) * sizeof(int64_t), s)) != cudaSuccess) return e;
        const unsigned hx = (unsigned)std::min<int64_t>(std::max<int64_t>(ceil_div(tl.heavy_cap, 256), 1), 64);
        const dim3 grid(hx, (unsigned)std::min(groups, 1024));
        k_tile_count<<<grid, 256, 0, s>>>(tl.bu, tl.bv, tl.heavy_cap, groups, tl.icnt, ctr);
        if ((e = scan_exclusive_i64(tl.icnt, groups, tl.ioff, tl.bsum, s)) != cudaSuccess) return e;
        // the counts are reused as the fill cursors
        if ((e = cudaMemsetAsync(tl.icnt, 0, (size_t)(groups + 1) * sizeof(int64_t), s)) != cudaSuccess) return e;
        k_tile_fill<<<grid, 256, 0, s>>>(tl.bu, tl.bv, tl.heavy_cap, groups, tl.ioff, tl.icnt, tl.items, tl.item_cap,
                                         ctr);
        k_support_tiled<<<(unsigned)num_sms, C_THREADS, C_SMEM, s>>>(off, col, flags, ooff, ocol, pv2, core_of, t,
                                                                     tl.heavy, tl.heavy_cap, tl.bu, tl.bv, tl.items,
                                                                     tl.ioff, groups, ctr);
        launched += 5;
    }
    if (core) {
        const uint64_t *cl = ctasks;
        if (CORE_ORDER != 0 && order.sorted) {
            const size_t hb = (size_t)(ORDER_CLASSES + 1) * sizeof(int64_t);
            if ((e = cudaMemsetAsync(order.hist, 0, hb, s)) != cudaSuccess) return e;
            const unsigned og = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(task_cap, 256), 4096));
            k_order_count<<<og, 256, 0, s>>>(ctasks, ooff, (unsigned long long *)order.hist, ctr);
            if ((e = scan_exclusive_i64(order.hist, ORDER_CLASSES, order.base, order.bsum, s)) != cudaSuccess)
                return e;
            if ((e = cudaMemsetAsync(order.hist, 0, hb, s)) != cudaSuccess) return e;
            k_order_fill<<<og, 256, 0, s>>>(ctasks, ooff, order.base, (unsigned long long *)order.hist, order.sorted,
                                            task_cap, ctr);
            cl = order.sorted;
            launched += 2;
        }
        k_support_core<<<(unsigned)num_sms, C_THREADS, C_SMEM, s>>>(off, col, flags, ooff, ocol, pv2, core_of, t,
                                                                    cl, ctr);
        ++launched;
    }
    k_support<<<(unsigned)(num_sms * 2), B_THREADS, bsmem, s>>>(off, col, flags, ooff, ocol, t, tasks, task_cap, ctr);
    count_launches(launched + 1);
    return cudaGetLastError();
}

}  // namespace tec
