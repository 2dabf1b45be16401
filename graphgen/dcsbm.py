"""Degree-corrected stochastic block model graphs (host side).

Project definition (the paper does not use this model; it is the source of
labelled graphs for the threshold picker).  For seed s:

* n = floor(exp(ln n_lo + u (ln n_hi - ln n_lo))), k = 2 + (w mod 63) blocks,
  mixing fraction mu = 0.05 + 0.45 u'  (u, u' uniform in [0,1) from the
  (s, DCSBM) stream).
* Vertex v: block b(v) = word mod k; propensity phi(v) = (1 - U)^(-1/1.5)
  (Pareto, density proportional to x^-2.5, x >= 1) truncated at sqrt(20 n);
  integer weight w(v) = floor(65536 phi(v)).
* 10 n edge samples (mean degree about 20).  Sample e uses words 4e .. 4e+3
  of the edge stream.  With probability mu (top 53 bits of word 4e below
  floor(mu 2^53)) the sample crosses blocks: u is drawn with probability
  w(u)/W over all vertices, v with probability w(v)/(W - vol b(u)) over the
  vertices outside b(u) (dropped as a self-loop if no other block has
  weight); otherwise a block b is drawn with probability
  vol(b)/W and u, v with probability w/vol(b) inside b.  A draw from [0, X) is
  mulhi(word, X) = floor(word X / 2^64), exact in integers, over vertices
  ordered by (block, id).
* Self-loops are dropped and duplicate pairs merged.

Everything after the vertex weights is integer arithmetic, so the device
sampler in gen_kernels.cu reproduces the host graphs bit for bit.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .csr import csr_from_pairs
from .prng import STREAM_DCSBM, draw, stream_key, uniform53

M32 = np.uint64(0xFFFFFFFF)


@dataclass
class DCSBMSpec:
    seed: int
    n: int
    k: int
    mu: float
    mu_cut: int            # floor(mu * 2^53)
    block: np.ndarray      # int32 [n]
    weight: np.ndarray     # int64 [n]
    order: np.ndarray      # int32 [n]: vertices sorted by (block, id)
    cum: np.ndarray        # int64 [n+1]: cumulative weights in `order`
    bstart: np.ndarray     # int64 [k+1]: cumulative block volumes

    @property
    def samples(self) -> int:
        return 10 * self.n


def dcsbm_spec(seed: int, n_lo: int = 1000, n_hi: int = 100000) -> DCSBMSpec:
    key = stream_key(seed, STREAM_DCSBM)
    u0 = float(uniform53(draw(key, 0)))
    n = int(math.floor(math.exp(math.log(n_lo) + u0 * (math.log(n_hi) - math.log(n_lo)))))
    n = max(2, min(n, n_hi))
    k = 2 + int(draw(key, 1)) % 63
    mu = 0.05 + 0.45 * float(uniform53(draw(key, 2)))
    mu_cut = int(math.floor(mu * 9007199254740992.0))
    v = np.arange(n, dtype=np.uint64)
    block = (draw(stream_key(seed, STREAM_DCSBM + 1), v) % np.uint64(k)).astype(np.int32)
    U = uniform53(draw(stream_key(seed, STREAM_DCSBM + 2), v))
    phi = np.minimum((1.0 - U) ** (-1.0 / 1.5), math.sqrt(20.0 * n))
    weight = np.floor(phi * 65536.0).astype(np.int64)
    order = np.lexsort((np.arange(n), block)).astype(np.int32)
    cum = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(weight[order], out=cum[1:])
    vol = np.bincount(block, weights=None, minlength=k)
    bsz = np.bincount(block, minlength=k)
    bstart_idx = np.concatenate([[0], np.cumsum(bsz)])
    bstart = cum[bstart_idx]
    del vol
    return DCSBMSpec(seed, n, k, mu, mu_cut, block, weight, order, cum, bstart.astype(np.int64))


def mulhi(a, b):
    """floor(a * b / 2^64) for uint64 arrays (exact, 32-bit limbs)."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    a0, a1 = a & M32, a >> np.uint64(32)
    b0, b1 = b & M32, b >> np.uint64(32)
    with np.errstate(over="ignore"):
        ll = a0 * b0
        hl = a1 * b0
        lh = a0 * b1
        hh = a1 * b1
        cross = (ll >> np.uint64(32)) + (hl & M32) + (lh & M32)
        return hh + (hl >> np.uint64(32)) + (lh >> np.uint64(32)) + (cross >> np.uint64(32))


def _pick(cum, pos):
    """Index i in `order` with cum[i] <= pos < cum[i+1]."""
    return np.searchsorted(cum, pos, side="right") - 1


def dcsbm_pairs(spec: DCSBMSpec, start: int = 0, count: int | None = None):
    """Endpoints (u, v) of samples [start, start+count)."""
    if count is None:
        count = spec.samples - start
    key = stream_key(spec.seed, STREAM_DCSBM + 3)
    e = np.arange(start, start + count, dtype=np.uint64)
    w0 = draw(key, np.uint64(4) * e)
    w1 = draw(key, np.uint64(4) * e + np.uint64(1))
    w2 = draw(key, np.uint64(4) * e + np.uint64(2))
    w3 = draw(key, np.uint64(4) * e + np.uint64(3))
    W = np.uint64(spec.cum[-1])
    across = (w0 >> np.uint64(11)) < np.uint64(spec.mu_cut)
    vol = np.diff(spec.bstart).astype(np.uint64)
    # across: u over everything, v outside b(u)
    pu = mulhi(w1, W).astype(np.int64)
    iu = _pick(spec.cum, pu)
    bu = spec.block[spec.order[iu]]
    pv = mulhi(w2, W - vol[bu]).astype(np.int64)
    pv = np.where(pv >= spec.bstart[bu], pv + vol[bu].astype(np.int64), pv)
    iv = np.where(W - vol[bu] == 0, iu, _pick(spec.cum, np.minimum(pv, spec.cum[-1] - 1)))
    # inside: a block by volume, then both ends inside it
    pb = mulhi(w1, W).astype(np.int64)
    b = np.searchsorted(spec.bstart, pb, side="right") - 1
    qu = spec.bstart[b] + mulhi(w2, vol[b]).astype(np.int64)
    qv = spec.bstart[b] + mulhi(w3, vol[b]).astype(np.int64)
    ju, jv = _pick(spec.cum, qu), _pick(spec.cum, qv)
    u = np.where(across, spec.order[iu], spec.order[ju])
    v = np.where(across, spec.order[iv], spec.order[jv])
    return u.astype(np.int64), v.astype(np.int64)


def dcsbm_csr(seed: int, n_lo: int = 1000, n_hi: int = 100000):
    """(off, col, block, spec) of the DC-SBM graph of `seed` (host)."""
    spec = dcsbm_spec(seed, n_lo, n_hi)
    u, v = dcsbm_pairs(spec)
    off, col = csr_from_pairs(spec.n, u, v)
    return off, col, spec.block, spec
