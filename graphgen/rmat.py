"""R-MAT graphs (Chakrabarti, Zhan & Faloutsos, SDM 2004), host side.

The paper's scalability experiments (Sec. IV-B, Table 5) use R-MAT graphs but
give only the 2x2 seed matrix; everything else here is this project's
definition, shared bit-for-bit by the host generator below and the device
generator in ``gen_kernels.cu``:

* ``edge_factor * 2**scale`` samples, sample ``i`` in [0, samples).
* Sample i draws one 64-bit key k_i = mix64(K ^ mix64(i)) with K the
  (seed, RMAT) stream key; level pair j uses w = mix64(k_i ^ j), the high 32
  bits for level 2j and the low 32 bits for level 2j+1.
* At level l the 32-bit word r picks a quadrant against the integer cut
  points A = floor(a 2^32), AB = floor((a+b) 2^32), ABC = floor((a+b+c) 2^32):
  r < A -> (0,0), r < AB -> (0,1), r < ABC -> (1,0), else (1,1); the pair
  gives bit l of the source and of the destination.  No per-level noise.
* Vertex ids are then relabelled by a keyed 4-round Feistel permutation of the
  ``scale``-bit id space (``feistel``), a bijection that needs no shuffle.
* The pairs are symmetrised, self-loops dropped and duplicates merged.
"""
from __future__ import annotations

import numpy as np

from .csr import csr_from_pairs
from .prng import STREAM_PERM, STREAM_RMAT, draw, mix64, stream_key

FEISTEL_ROUNDS = 4


def cut_points(a: float, b: float, c: float):
    """Integer quadrant cut points for 32-bit words."""
    A = int(a * 4294967296.0)
    AB = int((a + b) * 4294967296.0)
    ABC = int((a + b + c) * 4294967296.0)
    if not (0 <= A <= AB <= ABC <= 4294967296):
        raise ValueError("bad R-MAT probabilities")
    return A, AB, ABC


def feistel_keys(seed: int):
    return [stream_key(seed, STREAM_PERM + r) for r in range(FEISTEL_ROUNDS)]


def feistel(x, scale: int, seed: int):
    """Keyed bijection of [0, 2**scale); hi half gets ceil(scale/2) bits."""
    if scale < 2:
        raise ValueError("scale must be >= 2")
    x = np.asarray(x, dtype=np.uint64)
    lo_bits = scale // 2
    hi_bits = scale - lo_bits
    mask_lo = np.uint64((1 << lo_bits) - 1)
    mask_hi = np.uint64((1 << hi_bits) - 1)
    L = x >> np.uint64(lo_bits)
    R = x & mask_lo
    for r, k in enumerate(feistel_keys(seed)):
        if r % 2 == 0:
            L = L ^ (mix64(np.uint64(k) ^ R) & mask_hi)
        else:
            R = R ^ (mix64(np.uint64(k) ^ L) & mask_lo)
    return (L << np.uint64(lo_bits)) | R


def rmat_samples(scale: int, edge_factor: int, abc, seed: int, start: int = 0, count: int | None = None):
    """Raw (source, destination) samples [start, start+count), before permutation."""
    total = edge_factor << scale
    if count is None:
        count = total - start
    A, AB, ABC = (np.uint64(t) for t in cut_points(*abc))
    key = stream_key(seed, STREAM_RMAT)
    i = np.arange(start, start + count, dtype=np.uint64)
    ki = draw(key, i)
    u = np.zeros(count, dtype=np.uint64)
    v = np.zeros(count, dtype=np.uint64)
    for j in range((scale + 1) // 2):
        w = mix64(ki ^ np.uint64(j))
        for half in (0, 1):
            lvl = 2 * j + half
            if lvl >= scale:
                break
            r = (w >> np.uint64(32)) if half == 0 else (w & np.uint64(0xFFFFFFFF))
            ubit = (r >= AB).astype(np.uint64)
            vbit = (((r >= A) & (r < AB)) | (r >= ABC)).astype(np.uint64)
            u |= ubit << np.uint64(lvl)
            v |= vbit << np.uint64(lvl)
    return u, v


def rmat_csr(scale: int, edge_factor: int, abc=(0.57, 0.19, 0.19), seed: int = 2, chunk: int = 1 << 22):
    """Cleaned symmetric CSR of the permuted R-MAT graph (host; practical to scale ~20)."""
    n = 1 << scale
    total = edge_factor << scale
    us, vs = [], []
    for s in range(0, total, chunk):
        u, v = rmat_samples(scale, edge_factor, abc, seed, s, min(chunk, total - s))
        us.append(feistel(u, scale, seed).astype(np.int64))
        vs.append(feistel(v, scale, seed).astype(np.int64))
    return csr_from_pairs(n, np.concatenate(us), np.concatenate(vs))
