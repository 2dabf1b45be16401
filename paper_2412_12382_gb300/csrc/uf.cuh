// Lock-free union-find on int32 vertex ids (ECL-CC style: hooking of the larger
// root under the smaller with compare-and-swap, intermediate pointer jumping).
//
// Invariant: parent[x] <= x.  Only roots are ever re-pointed, always to a
// smaller root, so the root of every tree is the smallest id in it and the
// final labels are the component minima.  Reads bypass L1 (__ldcg) so a thread
// sees other SMs' hooks; a stale read only costs another retry.
#pragma once

#include "tec_internal.cuh"

namespace tec {

// Root of x given cur = parent[x] already loaded (lets callers batch the first loads).
__device__ __forceinline__ int32_t uf_find_from(int32_t *parent, int32_t x, int32_t cur) {
    if (cur != x) {
        int32_t prev = x, next;
        while (cur > (next = __ldcg(&parent[cur]))) {
            parent[prev] = next;   // any ancestor is a valid parent
            prev = cur;
            cur = next;
        }
    }
    return cur;
}

__device__ __forceinline__ int32_t uf_find(int32_t *parent, int32_t x) {
    return uf_find_from(parent, x, __ldcg(&parent[x]));
}

// The roots of a and b, walked side by side: each step issues the loads of
// both walks before using either, so a link waits for the longer of the two
// pointer chains rather than their sum.  Each walk is uf_find's (same path
// halving writes, same result).
__device__ __forceinline__ void uf_find2(int32_t *parent, int32_t a, int32_t b, int32_t &ra, int32_t &rb) {
    int32_t pa = a, ca = __ldcg(&parent[a]);
    int32_t pb = b, cb = __ldcg(&parent[b]);
    bool wa = ca != a, wb = cb != b;             // still walking
    while (wa || wb) {
        const int32_t na = wa ? __ldcg(&parent[ca]) : ca;
        const int32_t nb = wb ? __ldcg(&parent[cb]) : cb;
        if (wa) {
            if (ca > na) {
                parent[pa] = na;
                pa = ca;
                ca = na;
            } else {
                wa = false;
            }
        }
        if (wb) {
            if (cb > nb) {
                parent[pb] = nb;
                pb = cb;
                cb = nb;
            } else {
                wb = false;
            }
        }
    }
    ra = ca;
    rb = cb;
}

// Retry cap of one link.  Debug builds read a lowered cap from the counter
// block (set from TEC_DEBUG_LINK_CAP by the host), so a test can make the cap
// run out on purpose; 0 there means the normal cap.
__device__ __forceinline__ int link_cap(const unsigned long long *ctr) {
#ifdef TEC_DEBUG
    const unsigned long long c = ctr[C_DEBUG_LINK_CAP];
    return c ? (int)(c - 1) : LINK_RETRY_CAP;
#else
    (void)ctr;
    return LINK_RETRY_CAP;
#endif
}

// Each failed compare-and-swap means a root was hooked by another thread, so
// the retry loop makes global progress; the cap only guards against a broken
// forest and reports TEC_ETIMEOUT.
__device__ __forceinline__ void uf_link(int32_t *parent, int32_t a, int32_t b, unsigned long long *ctr) {
    int32_t ra, rb;
    uf_find2(parent, a, b, ra, rb);
    const int cap = link_cap(ctr);
    for (int it = 0; it < cap; ++it) {
        if (ra == rb) return;
        const int32_t hi = ra > rb ? ra : rb;
        const int32_t lo = ra > rb ? rb : ra;
        const int32_t old = atomicCAS(&parent[hi], hi, lo);
        if (old == hi) return;
        uf_find2(parent, old, lo, ra, rb);
    }
    flag_status(ctr, ST_TIMEOUT);
}

}  // namespace tec

namespace tec {

// uf_link that also reports whether this call joined two different trees
// (exactly one caller succeeds for each merge).
__device__ __forceinline__ bool uf_link_merged(int32_t *parent, int32_t a, int32_t b, unsigned long long *ctr) {
    int32_t ra, rb;
    uf_find2(parent, a, b, ra, rb);
    const int cap = link_cap(ctr);
    for (int it = 0; it < cap; ++it) {
        if (ra == rb) return false;
        const int32_t hi = ra > rb ? ra : rb;
        const int32_t lo = ra > rb ? rb : ra;
        const int32_t old = atomicCAS(&parent[hi], hi, lo);
        if (old == hi) return true;
        uf_find2(parent, old, lo, ra, rb);
    }
    flag_status(ctr, ST_TIMEOUT);
    return false;
}

}  // namespace tec
