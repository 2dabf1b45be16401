"""Stochastic block model graphs (host side).

Each unordered pair u < v is an edge independently with probability P[b(u), b(v)]
(the i.i.d.-pair model of the paper's Sec. III-B SBM).  Blocks are contiguous
id ranges in the order of `sizes`.  The pair (u, v) uses counter u*n + v of the
(seed, SBM) stream and is an edge iff the top 53 bits of its word are below
floor(p * 2^53), an exact integer test.
"""
from __future__ import annotations

import numpy as np

from .csr import csr_from_pairs
from .prng import STREAM_SBM, draw, stream_key


def block_of(sizes):
    return np.repeat(np.arange(len(sizes), dtype=np.int64), sizes)


def sbm_csr(sizes, P, seed: int, row_chunk: int = 256):
    sizes = [int(s) for s in sizes]
    P = np.asarray(P, dtype=np.float64)
    n = int(sum(sizes))
    blk = block_of(sizes)
    # threshold per block pair: edge iff (word >> 11) < floor(p * 2^53)
    T = np.floor(P * 9007199254740992.0).astype(np.uint64)
    key = stream_key(seed, STREAM_SBM)
    us, vs = [], []
    for r0 in range(0, n, row_chunk):
        rows = np.arange(r0, min(n, r0 + row_chunk), dtype=np.int64)
        cnt = n - 1 - rows
        uu = np.repeat(rows, cnt)
        first = np.concatenate([[0], np.cumsum(cnt)[:-1]]).astype(np.int64)
        vv = np.arange(uu.size, dtype=np.int64) - np.repeat(first, cnt) + uu + 1
        w = draw(key, (uu * n + vv).astype(np.uint64))
        hit = (w >> np.uint64(11)) < T[blk[uu], blk[vv]]
        us.append(uu[hit])
        vs.append(vv[hit])
    off, col = csr_from_pairs(n, np.concatenate(us), np.concatenate(vs))
    return off, col, blk


def planted_partition(n_blocks: int, block_size: int, p_in: float, p_out: float, seed: int):
    P = np.full((n_blocks, n_blocks), p_out)
    np.fill_diagonal(P, p_in)
    return sbm_csr([block_size] * n_blocks, P, seed)
