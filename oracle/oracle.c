/*
 * Reference oracle for motif-based community detection -- TEST INFRASTRUCTURE.
 *
 * Plain, slow, obviously correct CPU code that the CUDA path is checked
 * against.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the product path never does.  It shares no code with
 * the CUDA library.
 *
 * Every function follows a definition of the paper (Chen & Tsourakakis,
 * "Parallel Motif-Based Community Detection", arXiv 2412.12382):
 *   - Sec. I "Notations": t(u,v) = |N(u) n N(v)|,
 *     wedge(u,v) = |N(u) u N(v)| - |N(u) n N(v)| - 2.
 *   - Sec. III-C: intersections of sorted adjacency lists by merging, one
 *     independent task per edge.
 *   - Algorithm 1: remove every edge with sim(e) < delta, return the connected
 *     components of what is left.
 *
 * Graph format: symmetric CSR, vertices 0..n-1, rows sorted ascending,
 * off[n+1] int64, col[2m] int32.  Canonical edge e in [0, m) is the e-th pair
 * (u, v), u < v, in lexicographic order (the upper-triangle entries, row by
 * row).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* 0 when the CSR is a valid simple undirected graph with sorted rows:
 * 1 bad offsets, 2 column out of range, 3 row not strictly increasing
 * (unsorted or duplicate), 4 self-loop, 5 not symmetric. */
int orc_check_csr(int64_t n, const int64_t *off, const int32_t *col)
{
    if (n < 0 || off[0] != 0) return 1;
    for (int64_t u = 0; u < n; ++u)
        if (off[u + 1] < off[u]) return 1;
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t k = off[u]; k < off[u + 1]; ++k) {
            int64_t v = col[k];
            if (v < 0 || v >= n) return 2;
            if (k > off[u] && col[k - 1] >= col[k]) return 3;
            if (v == u) return 4;
        }
    }
    /* symmetry: v in N(u) implies u in N(v), by binary search in row v */
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t k = off[u]; k < off[u + 1]; ++k) {
            int64_t v = col[k];
            int64_t lo = off[v], hi = off[v + 1];
            while (lo < hi) {
                int64_t mid = lo + (hi - lo) / 2;
                if (col[mid] < u) lo = mid + 1; else hi = mid;
            }
            if (lo >= off[v + 1] || col[lo] != u) return 5;
        }
    }
    return 0;
}

/* Canonical edge list (u < v, lexicographic).  Returns m. */
int64_t orc_edge_list(int64_t n, const int64_t *off, const int32_t *col,
                      int32_t *eu, int32_t *ev)
{
    int64_t e = 0;
    for (int64_t u = 0; u < n; ++u)
        for (int64_t k = off[u]; k < off[u + 1]; ++k)
            if (col[k] > u) { eu[e] = (int32_t)u; ev[e] = col[k]; ++e; }
    return e;
}

/* For each listed edge (eu[e], ev[e]): inter[e] = |N(u) n N(v)| and
 * uni[e] = |N(u) u N(v)|, each by one merge of the two sorted rows
 * (Sec. III-C).  `nthreads` > 1 splits the independent edges over OpenMP
 * threads; the result does not depend on it. */
void orc_edge_counts(const int64_t *off, const int32_t *col, int64_t m,
                     const int32_t *eu, const int32_t *ev,
                     uint32_t *inter, uint32_t *uni, int nthreads)
{
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads)
#endif
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = off[eu[e]], iend = off[eu[e] + 1];
        int64_t j = off[ev[e]], jend = off[ev[e] + 1];
        uint64_t common = 0, all = 0;
        while (i < iend && j < jend) {
            if (col[i] < col[j]) { ++i; }
            else if (col[i] > col[j]) { ++j; }
            else { ++common; ++i; ++j; }
            ++all;
        }
        all += (uint64_t)(iend - i) + (uint64_t)(jend - j);
        inter[e] = (uint32_t)common;
        if (uni) uni[e] = (uint32_t)all;
    }
}

/* Per-edge triangle counts t(u,v) = |N(u) n N(v)| (Sec. I) by oriented
 * triangle listing -- the textbook "forward" algorithm (Chiba & Nishizeki
 * 1985; Schank & Wagner 2005) -- for graphs on which the per-edge merges of
 * Sec. III-C cost too much (their work is the sum over edges of
 * deg u + deg v, quadratic in the hub degrees).
 *
 *   1. Rank the vertices by (degree, id) ascending (a stable counting sort by
 *      degree); rank_of[v] is v's position and order[i] the vertex of rank i.
 *   2. Orient every edge from its lower-ranked to its higher-ranked end:
 *      out-row i holds the ranks of the higher-ranked neighbours of order[i].
 *   3. For every rank a: mark the heads of out-row a; for every head b of
 *      out-row a and every head c of out-row b, a marked c closes the
 *      triangle a < b < c, which is found only here (c is not in out-row a
 *      of any other pair, and b is not in out-row c).  The triangle adds one
 *      to each of its three oriented edges a->b, a->c, b->c.
 *   4. Every oriented edge is one undirected edge {U, V}; its count goes to
 *      the canonical id of (min, max): the upper-triangle entries before row
 *      min plus the position of max among row min's entries above min,
 *      found by binary search in the sorted row.
 * Additions commute, so the counts do not depend on the thread count.
 * t_out: m uint32 in canonical order.  Returns 0, or -1 if out of memory. */
int orc_forward_counts(int64_t n, const int64_t *off, const int32_t *col, uint32_t *t_out, int nthreads)
{
    if (n <= 0) return 0;
    if (nthreads < 1) nthreads = 1;
    const int64_t nnz = off[n], m = nnz / 2;
    int64_t maxdeg = 0;
    for (int64_t v = 0; v < n; ++v)
        if (off[v + 1] - off[v] > maxdeg) maxdeg = off[v + 1] - off[v];
    int64_t *start = (int64_t *)calloc((size_t)maxdeg + 2, sizeof(int64_t));
    int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *rank_of = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int64_t *roff = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    int64_t *uoff = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    int32_t *rcol = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    uint32_t *rt = (uint32_t *)calloc((size_t)(m > 0 ? m : 1), sizeof(uint32_t));
    int fail = !start || !order || !rank_of || !roff || !uoff || !rcol || !rt;
    if (fail) goto done;
    /* 1. stable counting sort by degree */
    for (int64_t v = 0; v < n; ++v) start[off[v + 1] - off[v] + 1]++;
    for (int64_t d = 0; d <= maxdeg; ++d) start[d + 1] += start[d];
    for (int64_t v = 0; v < n; ++v) {
        const int64_t i = start[off[v + 1] - off[v]]++;
        order[i] = (int32_t)v;
        rank_of[v] = (int32_t)i;
    }
    /* 2. out-rows in rank space: lengths, their prefix sums, then the heads */
    roff[0] = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4096) num_threads(nthreads)
#endif
    for (int64_t i = 0; i < n; ++i) {
        const int32_t u = order[i];
        int64_t c = 0;
        for (int64_t k = off[u]; k < off[u + 1]; ++k) c += rank_of[col[k]] > i;
        roff[i + 1] = c;
    }
    for (int64_t i = 0; i < n; ++i) roff[i + 1] += roff[i];
    if (roff[n] != m) { fail = 1; goto done; }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4096) num_threads(nthreads)
#endif
    for (int64_t i = 0; i < n; ++i) {
        const int32_t u = order[i];
        int64_t j = roff[i];
        for (int64_t k = off[u]; k < off[u + 1]; ++k)
            if (rank_of[col[k]] > i) rcol[j++] = rank_of[col[k]];
    }
    /* 3. list every triangle once, from its lowest-ranked vertex */
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
    {
        /* mark[c] = 1 + position of c in the current out-row a, 0 = unmarked;
         * acc[x] = triangles found so far on the edge a -> (x-th head of a).
         * Other threads add to the same edges (as their b -> c), so every
         * addition to rt is atomic; the edges of row a are added once per
         * row from acc. */
        uint32_t *mark = (uint32_t *)calloc((size_t)n, sizeof(uint32_t));
        uint64_t *bits = (uint64_t *)calloc((size_t)(n + 63) / 64, sizeof(uint64_t));   /* mark[c] != 0 */
        uint32_t *acc = (uint32_t *)calloc((size_t)maxdeg + 1, sizeof(uint32_t));
        if (!mark || !bits || !acc) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            fail = 1;
        }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (int64_t a = 0; a < n; ++a) {
            if (!mark || !bits || !acc) continue;
            const int64_t ab = roff[a], ae = roff[a + 1];
            for (int64_t j = ab; j < ae; ++j) {
                mark[rcol[j]] = (uint32_t)(j - ab + 1);
                bits[rcol[j] >> 6] |= (uint64_t)1 << (rcol[j] & 63);
                acc[j - ab] = 0u;
            }
            for (int64_t j = ab; j < ae; ++j) {
                const int32_t b = rcol[j];
                uint32_t hits = 0;
                for (int64_t k = roff[b]; k < roff[b + 1]; ++k) {
                    const int32_t c = rcol[k];
                    if ((bits[c >> 6] >> (c & 63)) & 1u) {
                        const uint32_t x = mark[c];
                        ++hits;                                               /* a -> b */
                        ++acc[x - 1];                                         /* a -> c */
                        __atomic_fetch_add(&rt[k], 1u, __ATOMIC_RELAXED);     /* b -> c */
                    }
                }
                acc[j - ab] += hits;
            }
            for (int64_t j = ab; j < ae; ++j) {
                mark[rcol[j]] = 0u;
                bits[rcol[j] >> 6] = 0u;
                if (acc[j - ab]) __atomic_fetch_add(&rt[j], acc[j - ab], __ATOMIC_RELAXED);
            }
        }
        free(mark);
        free(bits);
        free(acc);
    }
    if (fail) goto done;
    /* 4. canonical ids: uoff[u] = upper-triangle entries in rows before u */
    uoff[0] = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4096) num_threads(nthreads)
#endif
    for (int64_t u = 0; u < n; ++u) {
        int64_t lo = off[u], hi = off[u + 1];
        while (lo < hi) {                        /* first entry above u */
            const int64_t mid = lo + (hi - lo) / 2;
            if (col[mid] < u) lo = mid + 1; else hi = mid;
        }
        uoff[u + 1] = off[u + 1] - lo;
    }
    for (int64_t u = 0; u < n; ++u) uoff[u + 1] += uoff[u];
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4096) num_threads(nthreads)
#endif
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = roff[i]; j < roff[i + 1]; ++j) {
            const int64_t x = order[i], y = order[rcol[j]];
            const int64_t a = x < y ? x : y, b = x < y ? y : x;
            int64_t lo = off[a], hi = off[a + 1];
            while (lo < hi) {                    /* position of b in row a */
                const int64_t mid = lo + (hi - lo) / 2;
                if (col[mid] < b) lo = mid + 1; else hi = mid;
            }
            const int64_t above = off[a + 1] - (uoff[a + 1] - uoff[a]);   /* first entry above a */
            t_out[uoff[a] + (lo - above)] = rt[j];
        }
    }
done:
    free(start); free(order); free(rank_of); free(roff); free(uoff); free(rcol); free(rt);
    return fail ? -1 : 0;
}

/* K4 participation (Table 1, kappa = 4): for each edge e = (u, v) the number
 * of 4-cliques containing it, i.e. the number of edges {c, d} with both ends
 * in the common neighbourhood C = N(u) n N(v).  C is built by merging the two
 * sorted rows; each c in C is merged with C once more, counting the d > c of
 * N(c) that lie in C. */
void orc_edge_k4(const int64_t *off, const int32_t *col, int64_t m, const int32_t *eu, const int32_t *ev,
                 uint64_t *k4, int nthreads)
{
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads)
#endif
    {
        int64_t cap = 64;
        int32_t *cs = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (int64_t e = 0; e < m; ++e) {
            int64_t i = off[eu[e]], iend = off[eu[e] + 1];
            int64_t j = off[ev[e]], jend = off[ev[e] + 1];
            int64_t nc = 0;
            while (i < iend && j < jend) {
                if (col[i] < col[j]) ++i;
                else if (col[i] > col[j]) ++j;
                else {
                    if (nc == cap) {
                        cap *= 2;
                        cs = (int32_t *)realloc(cs, (size_t)cap * sizeof(int32_t));
                    }
                    cs[nc++] = col[i];
                    ++i;
                    ++j;
                }
            }
            uint64_t count = 0;
            for (int64_t a = 0; a < nc; ++a) {
                const int32_t c = cs[a];
                int64_t x = off[c], xend = off[c + 1], y = a + 1;
                while (x < xend && y < nc) {             /* N(c) merged with the d > c of C */
                    if (col[x] < cs[y]) ++x;
                    else if (col[x] > cs[y]) ++y;
                    else { ++count; ++x; ++y; }
                }
            }
            k4[e] = count;
        }
        free(cs);
    }
}

/* Connected components of (V, {e : keep[e]}) over the canonical edge list
 * (Algorithm 1, second step).  Breadth-first search started from every
 * unvisited vertex in increasing id order, so the start vertex is the smallest
 * id of its component and becomes the label of every vertex reached.
 * Returns the number of components (isolated vertices count).  -1 if out of
 * memory. */
int64_t orc_components(int64_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                       const uint8_t *keep, int32_t *label)
{
    int64_t *koff = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!koff) return -1;
    for (int64_t e = 0; e < m; ++e)
        if (keep[e]) { koff[eu[e] + 1]++; koff[ev[e] + 1]++; }
    for (int64_t u = 0; u < n; ++u) koff[u + 1] += koff[u];
    int32_t *kadj = (int32_t *)malloc((size_t)(koff[n] > 0 ? koff[n] : 1) * sizeof(int32_t));
    int64_t *fill = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int32_t *queue = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!kadj || !fill || !queue) { free(koff); free(kadj); free(fill); free(queue); return -1; }
    memcpy(fill, koff, (size_t)n * sizeof(int64_t));
    for (int64_t e = 0; e < m; ++e)
        if (keep[e]) { kadj[fill[eu[e]]++] = ev[e]; kadj[fill[ev[e]]++] = eu[e]; }
    for (int64_t v = 0; v < n; ++v) label[v] = -1;
    int64_t ncomp = 0;
    for (int64_t s = 0; s < n; ++s) {
        if (label[s] >= 0) continue;
        ++ncomp;
        int64_t head = 0, tail = 0;
        queue[tail++] = (int32_t)s;
        label[s] = (int32_t)s;
        while (head < tail) {
            int64_t x = queue[head++];
            for (int64_t k = koff[x]; k < koff[x + 1]; ++k) {
                int32_t y = kadj[k];
                if (label[y] < 0) { label[y] = (int32_t)s; queue[tail++] = y; }
            }
        }
    }
    free(koff); free(kadj); free(fill); free(queue);
    return ncomp;
}

/* Algorithm 1, first step: keep[e] = 1 iff sim(e) >= p/q, i.e. the edge
 * survives unless sim(e) < delta.  Both measures are compared exactly by
 * cross-multiplying in 128-bit integers (q > 0 is required):
 *   measure 0, Tectonic (Table 1): sim = t / (deg u + deg v),
 *       keep iff t*q >= p*(deg u + deg v);
 *   measure 1, TW (Eq. 1): sim = t - wedge with
 *       wedge = |N(u) u N(v)| - t - 2 (Sec. I), keep iff (t - wedge)*q >= p;
 *   measure 2, Jaccard (Table 1): sim = t / |N(u) u N(v)|, the union
 *       being deg u + deg v - t > 0, keep iff t*q >= p*|N(u) u N(v)|;
 *   measure 3, K3 (Table 1): sim = t, keep iff t*q >= p.
 * Returns the number of kept edges, or -1 on a bad argument. */
int64_t orc_prune(int measure, const int64_t *off, int64_t m,
                  const int32_t *eu, const int32_t *ev,
                  const uint32_t *inter, const uint32_t *uni,
                  int64_t p, int64_t q, uint8_t *keep)
{
    if (q <= 0 || measure < 0 || measure > 3) return -1;
    int64_t kept = 0;
    for (int64_t e = 0; e < m; ++e) {
        __int128 t = inter[e];
        int k;
        if (measure == 0) {
            __int128 du = off[eu[e] + 1] - off[eu[e]];
            __int128 dv = off[ev[e] + 1] - off[ev[e]];
            k = t * q >= (__int128)p * (du + dv);
        } else if (measure == 1) {
            __int128 wedge = (__int128)uni[e] - t - 2;
            k = (t - wedge) * q >= (__int128)p;
        } else if (measure == 2) {
            k = t * q >= (__int128)p * (__int128)uni[e];
        } else {
            k = t * q >= (__int128)p;
        }
        keep[e] = (uint8_t)k;
        kept += k;
    }
    return kept;
}

int orc_num_threads_available(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
