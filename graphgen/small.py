"""Small graphs with closed-form motif counts, used to pin the oracle.

Each function returns a symmetric CSR (off int64, col int32).
"""
from __future__ import annotations

import numpy as np

from .csr import csr_from_pairs


def complete(k: int):
    """K_k: every edge lies in k-2 triangles and 0 wedges."""
    u, v = np.triu_indices(k, 1)
    return csr_from_pairs(k, u, v)


def two_cliques_bridge(a: int, b: int):
    """K_a on 0..a-1, K_b on a..a+b-1, plus the bridge (a-1, a)."""
    u1, v1 = np.triu_indices(a, 1)
    u2, v2 = np.triu_indices(b, 1)
    u = np.concatenate([u1, u2 + a, [a - 1]])
    v = np.concatenate([v1, v2 + a, [a]])
    return csr_from_pairs(a + b, u, v)


def star(k: int):
    """Centre 0 with k leaves 1..k: every edge has t=0 and k-1 wedges."""
    return csr_from_pairs(k + 1, np.zeros(k, dtype=np.int64), np.arange(1, k + 1))


def cycle(k: int):
    """C_k (k >= 4): every edge has t=0 and 2 wedges."""
    u = np.arange(k)
    return csr_from_pairs(k, u, (u + 1) % k)


def empty(n: int):
    """n isolated vertices, no edges."""
    return np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32)


def gnp(n: int, p: float, rng: np.random.Generator):
    """Erdos-Renyi G(n,p) from a numpy Generator (test inputs only)."""
    u, v = np.triu_indices(n, 1)
    hit = rng.random(u.size) < p
    return csr_from_pairs(n, u[hit], v[hit])
