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
