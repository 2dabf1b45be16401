"""Oracle for motif-based community detection -- TEST INFRASTRUCTURE ONLY.

A plain, slow CPU statement of what the CUDA library computes, written from
the paper (Chen & Tsourakakis, arXiv 2412.12382).  Only `tests/`,
`__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import
it; the library never does, and the two share no code.  Per-edge merges,
pruning and breadth-first components run in plain C (``oracle.c``, built by
``oracle/build.py``); everything else is numpy in int64 / float64.

Vocabulary (Sec. I, "Notations"): N(u) neighbours of u, deg(u) = |N(u)|,
t(u,v) = |N(u) n N(v)| triangles on edge (u,v),
wedge(u,v) = |N(u) u N(v)| - |N(u) n N(v)| - 2.

Parity unpinned: `features` / MLP training targets depend on project-chosen
definitions (histogram binning, target encoding) that the paper does not fix;
their pins are closed forms and finite differences, not paper values.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

from .build import library_path, build_oracle

TECTONIC = 0
TW = 1
JACCARD = 2
K3 = 3
K4 = 4

_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        build_oracle()
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    lib.orc_check_csr.argtypes = [i64, P, P]
    lib.orc_check_csr.restype = ctypes.c_int
    lib.orc_edge_list.argtypes = [i64, P, P, P, P]
    lib.orc_edge_list.restype = i64
    lib.orc_edge_counts.argtypes = [P, P, i64, P, P, P, P, ctypes.c_int]
    lib.orc_edge_counts.restype = None
    lib.orc_components.argtypes = [i64, i64, P, P, P, P]
    lib.orc_components.restype = i64
    lib.orc_prune.argtypes = [ctypes.c_int, P, i64, P, P, P, P, i64, i64, P]
    lib.orc_prune.restype = i64
    lib.orc_edge_k4.argtypes = [P, P, i64, P, P, P, ctypes.c_int]
    lib.orc_edge_k4.restype = None
    lib.orc_forward_counts.argtypes = [i64, P, P, P, ctypes.c_int]
    lib.orc_forward_counts.restype = ctypes.c_int
    lib.orc_num_threads_available.argtypes = []
    lib.orc_num_threads_available.restype = ctypes.c_int
    _lib = lib
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(off, col):
    off = np.ascontiguousarray(off, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    return off, col


def threads_available() -> int:
    return int(_load().orc_num_threads_available())


# ---------------------------------------------------------------- basics


def check_csr(off, col) -> int:
    """0 if (off, col) is a simple undirected graph with sorted rows, else an error code."""
    off, col = _csr(off, col)
    return int(_load().orc_check_csr(len(off) - 1, _p(off), _p(col)))


def degrees(off):
    """deg(u) = |N(u)| = row length (Sec. I)."""
    return np.diff(np.asarray(off, dtype=np.int64))


def edge_list(off, col):
    """Canonical edges (u < v, lexicographic) as int32 arrays."""
    off, col = _csr(off, col)
    m = int(off[-1]) // 2
    eu = np.empty(m, dtype=np.int32)
    ev = np.empty(m, dtype=np.int32)
    got = _load().orc_edge_list(len(off) - 1, _p(off), _p(col), _p(eu), _p(ev))
    assert got == m, "asymmetric CSR"
    return eu, ev


def edge_counts(off, col, eu=None, ev=None, nthreads: int = 1):
    """(t, union) per edge: |N(u) n N(v)| and |N(u) u N(v)| by merging sorted rows (Sec. III-C)."""
    off, col = _csr(off, col)
    if eu is None:
        eu, ev = edge_list(off, col)
    eu = np.ascontiguousarray(eu, dtype=np.int32)
    ev = np.ascontiguousarray(ev, dtype=np.int32)
    m = eu.size
    t = np.empty(m, dtype=np.uint32)
    uni = np.empty(m, dtype=np.uint32)
    _load().orc_edge_counts(_p(off), _p(col), m, _p(eu), _p(ev), _p(t), _p(uni), int(nthreads))
    return t, uni


def forward_counts(off, col, nthreads: int = 1):
    """t(u,v) = |N(u) n N(v)| for every canonical edge by oriented ("forward")
    triangle listing (Chiba & Nishizeki; Schank & Wagner): each triangle is
    found once from its lowest (degree, id)-ranked vertex and added to its
    three edges.  Same result as edge_counts, with work sum_v d-(v) d+(v)
    instead of the per-edge merges of Sec. III-C, so it reaches R-MAT scale 26.
    The union size follows as deg u + deg v - t (inclusion-exclusion)."""
    off, col = _csr(off, col)
    n = len(off) - 1
    t = np.empty(int(off[-1]) // 2, dtype=np.uint32)
    if _load().orc_forward_counts(n, _p(off), _p(col), _p(t), int(nthreads)) != 0:
        raise MemoryError("oracle forward counts: out of memory or asymmetric CSR")
    return t


def unions_from_counts(off, eu, ev, t):
    """|N(u) u N(v)| = deg u + deg v - |N(u) n N(v)| (inclusion-exclusion), uint32."""
    d = degrees(off)
    return (d[np.asarray(eu)] + d[np.asarray(ev)] - np.asarray(t, dtype=np.int64)).astype(np.uint32)


def wedges(t, uni):
    """wedge(u,v) = |N(u) u N(v)| - |N(u) n N(v)| - 2 (Sec. I)."""
    return np.asarray(uni, dtype=np.int64) - np.asarray(t, dtype=np.int64) - 2


def tectonic_weights(off, eu, ev, t):
    """Tectonic similarity t(u,v) / (deg u + deg v) (Table 1), one IEEE binary64 division."""
    d = degrees(off)
    s = (d[np.asarray(eu)] + d[np.asarray(ev)]).astype(np.float64)
    return np.asarray(t, dtype=np.float64) / s


def jaccard_weights(t, uni):
    """Jaccard similarity |N(u) n N(v)| / |N(u) u N(v)| (Table 1, Sec. II), one IEEE binary64 division."""
    return np.asarray(t, dtype=np.float64) / np.asarray(uni, dtype=np.float64)


def k3_scores(t):
    """K3 similarity: the triangle count t(u,v) itself (Table 1), exact."""
    return np.asarray(t, dtype=np.int64)


def edge_k4(off, col, eu=None, ev=None, nthreads: int = 1):
    """K4 participation (Table 1, kappa = 4): 4-cliques containing each edge, in
    canonical edge order (uint64)."""
    off, col = _csr(off, col)
    if eu is None:
        eu, ev = edge_list(off, col)
    eu = np.ascontiguousarray(eu, dtype=np.int32)
    ev = np.ascontiguousarray(ev, dtype=np.int32)
    k4 = np.empty(eu.size, dtype=np.uint64)
    _load().orc_edge_k4(_p(off), _p(col), eu.size, _p(eu), _p(ev), _p(k4), int(nthreads))
    return k4


def tw_scores(t, wedge):
    """TW(e) = t(e) - wedge(e) (Eq. 1), exact int64."""
    return np.asarray(t, dtype=np.int64) - np.asarray(wedge, dtype=np.int64)


def prune(measure: int, off, eu, ev, t, uni, p: int, q: int, k4=None):
    """keep[e] = 1 iff sim(e) >= p/q (Algorithm 1 removes exactly the edges with sim < delta).
    For K4 the 4-clique counts k4 (edge_k4) are the similarity: keep iff k4*q >= p."""
    if q <= 0:
        raise ValueError("q must be positive")
    if measure == K4:
        if k4 is None:
            raise ValueError("K4 needs the 4-clique counts")
        keep = np.array([1 if int(x) * q >= p else 0 for x in k4], dtype=np.uint8)
        return keep, int(keep.sum())
    if not (-(1 << 63) <= p < (1 << 63) and q < (1 << 63)):
        raise ValueError("p and q must fit in int64")
    off = np.ascontiguousarray(off, dtype=np.int64)
    eu = np.ascontiguousarray(eu, dtype=np.int32)
    ev = np.ascontiguousarray(ev, dtype=np.int32)
    t = np.ascontiguousarray(t, dtype=np.uint32)
    uni = np.ascontiguousarray(uni, dtype=np.uint32)
    keep = np.empty(eu.size, dtype=np.uint8)
    kept = _load().orc_prune(int(measure), _p(off), eu.size, _p(eu), _p(ev), _p(t), _p(uni),
                             int(p), int(q), _p(keep))
    if kept < 0:
        raise ValueError("bad prune arguments")
    return keep, int(kept)


def components(n: int, eu, ev, keep):
    """Components of the kept subgraph (Algorithm 1); label = smallest vertex id of the component."""
    eu = np.ascontiguousarray(eu, dtype=np.int32)
    ev = np.ascontiguousarray(ev, dtype=np.int32)
    keep = np.ascontiguousarray(keep, dtype=np.uint8)
    label = np.empty(n, dtype=np.int32)
    nc = _load().orc_components(int(n), eu.size, _p(eu), _p(ev), _p(keep), _p(label))
    if nc < 0:
        raise MemoryError("oracle components: out of memory")
    return label, int(nc)


@dataclass
class PassResult:
    eu: np.ndarray
    ev: np.ndarray
    t: np.ndarray
    wedge: np.ndarray
    keep: np.ndarray
    kept: int
    labels: np.ndarray
    ncomp: int


def full_pass(off, col, measure: int, p: int, q: int, nthreads: int = 1) -> PassResult:
    """Algorithm 1 end to end: counts, similarity, prune at p/q, components."""
    off, col = _csr(off, col)
    n = len(off) - 1
    eu, ev = edge_list(off, col)
    t, uni = edge_counts(off, col, eu, ev, nthreads)
    k4 = edge_k4(off, col, eu, ev, nthreads) if measure == K4 else None
    keep, kept = prune(measure, off, eu, ev, t, uni, p, q, k4)
    labels, nc = components(n, eu, ev, keep)
    return PassResult(eu, ev, t, wedges(t, uni), keep, kept, labels, nc)


def sweep(off, col, measure: int, ps, qs, nthreads: int = 1):
    """Components at each threshold p_i/q_i: literally one independent prune + components per threshold."""
    off, col = _csr(off, col)
    n = len(off) - 1
    eu, ev = edge_list(off, col)
    t, uni = edge_counts(off, col, eu, ev, nthreads)
    k4 = edge_k4(off, col, eu, ev, nthreads) if measure == K4 else None
    labels = np.empty((len(ps), n), dtype=np.int32)
    ncomp = np.empty(len(ps), dtype=np.int64)
    for i, (p, q) in enumerate(zip(ps, qs)):
        keep, _ = prune(measure, off, eu, ev, t, uni, p, q, k4)
        labels[i], ncomp[i] = components(n, eu, ev, keep)
    return labels, ncomp


# ------------------------------------------------------ evaluation helpers


def ari(a, b) -> float:
    """Adjusted Rand index (Hubert & Arabie 1985) of two labelings, from exact pair counts.

    ARI = (sum_ij C(n_ij,2) - S_a S_b / C(n,2)) / ((S_a + S_b)/2 - S_a S_b / C(n,2)),
    S_a = sum_i C(a_i,2), S_b = sum_j C(b_j,2).  When the denominator is 0 (both
    partitions trivial) the value is 1 if the partitions are equal, else 0.
    """
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    n = a.size
    if n < 2:
        return 1.0
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    pair = ai * (int(bi.max()) + 1) + bi
    _, nij = np.unique(pair, return_counts=True)
    _, na = np.unique(ai, return_counts=True)
    _, nb = np.unique(bi, return_counts=True)

    def c2(x):
        return sum(int(v) * (int(v) - 1) // 2 for v in x)

    sij, sa, sb, total = c2(nij), c2(na), c2(nb), n * (n - 1) // 2
    from fractions import Fraction
    expected = Fraction(sa * sb, total)
    denom = Fraction(sa + sb, 2) - expected
    if denom == 0:
        same = len(nij) == len(na) == len(nb)
        return 1.0 if same else 0.0
    return float((Fraction(sij) - expected) / denom)


def modularity(off, col, labels) -> float:
    """Q = 1/(2m) sum_{u,v} (A_uv - deg u deg v / 2m) delta(c_u, c_v) (Sec. II), via
    its per-community form sum_c [ 2 L_c / 2m - (D_c / 2m)^2 ] (L_c intra edges,
    D_c total degree of c)."""
    off = np.asarray(off, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    labels = np.asarray(labels, dtype=np.int64)
    n = len(off) - 1
    two_m = int(off[-1])
    if two_m == 0:
        return 0.0
    row = np.repeat(np.arange(n), np.diff(off))
    same = labels[row] == labels[col]
    _, li = np.unique(labels, return_inverse=True)
    intra = np.bincount(li[row[same]], minlength=li.max() + 1).astype(np.float64)  # 2 L_c
    D = np.bincount(li, weights=np.diff(off).astype(np.float64), minlength=li.max() + 1)
    return float(np.sum(intra / two_m - (D / two_m) ** 2))


def precision_recall_f1(truth, found):
    """Size-weighted precision / recall / F1 of Sec. IV-A, for a non-overlapping
    ground truth: each found community S_i is matched to the truth community C
    maximising |C n S_i| / |C u S_i|; p_i = |C n S_i|/|S_i|, r_i = |C n S_i|/|C|."""
    truth = np.asarray(truth, dtype=np.int64)
    found = np.asarray(found, dtype=np.int64)
    tsize = {c: int(s) for c, s in zip(*np.unique(truth, return_counts=True))}
    num_p = num_r = num_f = 0.0
    total = 0
    for s in np.unique(found):
        members = truth[found == s]
        size = members.size
        best = None
        for c, inter in zip(*np.unique(members, return_counts=True)):
            j = inter / (tsize[c] + size - inter)
            if best is None or j > best[0]:
                best = (j, int(inter), tsize[c])
        _, inter, csize = best
        p, r = inter / size, inter / csize
        num_p += p * size
        num_r += r * size
        num_f += (2 * p * r / (p + r)) * size
        total += size
    return num_p / total, num_r / total, num_f / total


def histogram64(off, eu, ev, t):
    """Bin counts of b(e) = floor(128 t / (deg u + deg v)), clamped to 63: the
    64-bin histogram of Tectonic weights on the grid i/128 (project definition)."""
    d = degrees(off)
    s = d[np.asarray(eu)] + d[np.asarray(ev)]
    b = np.minimum((128 * np.asarray(t, dtype=np.int64)) // s, 63)
    return np.bincount(b, minlength=64).astype(np.int64)


def features(off, eu, ev, t):
    """66 picker features: the 64 histogram bins divided by m, then ln(2m/n), ln(m)."""
    n = len(off) - 1
    m = len(eu)
    h = histogram64(off, eu, ev, t).astype(np.float64)
    if m == 0:
        return np.concatenate([h, [0.0, 0.0]])
    return np.concatenate([h / m, [math.log(2.0 * m / n), math.log(m)]])


# ------------------------------------------------------ sweep diagnostics, rules of thumb


def sweep_stats(off, col, measure: int, ps, qs, labels, nthreads: int = 1):
    """Per threshold p_i/q_i, the statistics Sec. IV-D plots against the
    threshold (Fig. 6), for the labeling labels[i] of that threshold:
    ncomp (components), kept (edges with sim >= p_i/q_i), largest (size of the
    largest component), intra (edges of the input graph inside one component)
    and the modularity of Sec. II with the components as communities,
    Q = intra/m - sum_c vol(c)^2 / (2m)^2, vol(c) the degree sum of c,
    formed from exact integers and rounded once (0 for a graph without edges)."""
    from fractions import Fraction
    off, col = _csr(off, col)
    n = len(off) - 1
    eu, ev = edge_list(off, col)
    t, uni = edge_counts(off, col, eu, ev, nthreads)
    deg = degrees(off)
    m = len(eu)
    k4 = edge_k4(off, col, eu, ev, nthreads) if measure == K4 else None
    out = []
    for i, (p, q) in enumerate(zip(ps, qs)):
        _, kept = prune(measure, off, eu, ev, t, uni, p, q, k4)
        lab = np.asarray(labels[i], dtype=np.int64)
        _, li = np.unique(lab, return_inverse=True)
        size = np.bincount(li)
        vol = np.zeros(len(size), dtype=np.int64)
        np.add.at(vol, li, deg)
        intra = int(np.count_nonzero(lab[eu] == lab[ev]))
        sum_vol2 = sum(int(v) * int(v) for v in vol)
        qmod = float(Fraction(4 * m * intra - sum_vol2, 4 * m * m)) if m else 0.0
        out.append({"ncomp": int(len(size)), "kept": int(kept), "largest": int(size.max()) if n else 0,
                    "intra": intra, "sum_vol2": sum_vol2, "modularity": qmod})
    return out


def _ascending(ps, qs):
    from fractions import Fraction
    return sorted(range(len(ps)), key=lambda i: (Fraction(int(ps[i]), int(qs[i])), i))


def rule_largest_jump(ps, qs, largest):
    """Rule of thumb R1 (Sec. IV-D): visit the thresholds in decreasing order
    and stop at the sudden increase of the largest component: the index of the
    threshold just above the largest increase (the highest such threshold on
    ties), or None when the largest component never grows."""
    order = _ascending(ps, qs)
    best, best_jump = None, 0
    for j in range(len(order) - 2, -1, -1):          # from theta_(j+1) down to theta_j
        jump = largest[order[j]] - largest[order[j + 1]]
        if jump > best_jump:
            best, best_jump = order[j + 1], jump
    return best


def rule_modularity(ps, qs, modularity):
    """Rule of thumb R2 (Sec. IV-D): the threshold of largest modularity (the
    lowest such threshold on ties)."""
    order = _ascending(ps, qs)
    best = order[0]
    for i in order[1:]:
        if modularity[i] > modularity[best]:
            best = i
    return best


def rule_of_thumb(ps, qs, stats):
    """R1, falling back to R2 where the largest component never grows (the
    paper recommends modularity where no shift shows)."""
    r1 = rule_largest_jump(ps, qs, [s["largest"] for s in stats])
    return r1 if r1 is not None else rule_modularity(ps, qs, [s["modularity"] for s in stats])
