"""Edge lists to cleaned, symmetric CSR (host side, numpy).

The CSR convention used everywhere in this project: vertices 0..n-1, an
undirected simple graph (no self-loops, no duplicate edges) stored with both
directions, rows sorted by neighbour id.  `off` has n+1 int64 entries and
`col` has 2m int32 entries.
"""
from __future__ import annotations

import numpy as np


def csr_from_pairs(n: int, a, b):
    """Symmetric, deduplicated, loop-free CSR from (possibly repeated) pairs (a[i], b[i])."""
    a = np.asarray(a, dtype=np.int64).ravel()
    b = np.asarray(b, dtype=np.int64).ravel()
    if a.shape != b.shape:
        raise ValueError("endpoint arrays differ in length")
    if a.size and (min(a.min(), b.min()) < 0 or max(a.max(), b.max()) >= n):
        raise ValueError("endpoint out of range")
    keep = a != b
    lo = np.minimum(a, b)[keep]
    hi = np.maximum(a, b)[keep]
    key = np.unique(lo * np.int64(n) + hi)
    lo = key // n
    hi = key % n
    src = np.concatenate([lo, hi])
    dst = np.concatenate([hi, lo])
    key2 = np.sort(src * np.int64(n) + dst)
    src = key2 // n
    dst = key2 % n
    off = np.zeros(n + 1, dtype=np.int64)
    if n:
        np.cumsum(np.bincount(src, minlength=n), out=off[1:])
    return off, dst.astype(np.int32)


def num_edges(off) -> int:
    return int(off[-1]) // 2


def upper_pairs(off, col):
    """Canonical undirected edge list: (u, v) with u < v, lexicographic order."""
    n = len(off) - 1
    row = np.repeat(np.arange(n, dtype=np.int64), np.diff(off))
    c = np.asarray(col, dtype=np.int64)
    sel = c > row
    return row[sel], c[sel]


def dense_adjacency(off, col):
    """0/1 adjacency matrix (int64) of a small CSR graph."""
    n = len(off) - 1
    A = np.zeros((n, n), dtype=np.int64)
    row = np.repeat(np.arange(n), np.diff(off))
    A[row, np.asarray(col, dtype=np.int64)] = 1
    return A
