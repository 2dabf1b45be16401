"""Counter-based random numbers shared by every graph generator.

The mixing function is the SplitMix64 output finaliser (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): add the golden
gamma, then two xor-shift-multiply rounds and a final xor-shift.  Every random
draw in this package is ``mix64`` of a counter derived from (seed, stream,
index), so a draw can be recomputed independently on the host (numpy, here) or
on the device (``gen_kernels.cu`` implements the same published definition) and
both give the same 64-bit word.

Nothing here belongs to the community-detection method; it only produces inputs.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

# Stream tags keep the draws of different generators apart.
STREAM_RMAT = 0x524D4154          # "RMAT"
STREAM_PERM = 0x5045524D          # "PERM"
STREAM_SBM = 0x53424D00           # "SBM\0"
STREAM_DCSBM = 0x44435342         # "DCSB"

MASK64 = (1 << 64) - 1


def mix64(x):
    """SplitMix64 finaliser on uint64 (numpy array or scalar), wrapping mod 2^64."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + GAMMA
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        return z ^ (z >> np.uint64(31))


def mix64_int(x: int) -> int:
    """Same finaliser on a Python int (used for scalar keys)."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def stream_key(seed: int, stream: int) -> int:
    """64-bit key of one (seed, stream) pair."""
    return mix64_int(mix64_int(seed & MASK64) ^ (stream & MASK64))


def draw(key: int, counter):
    """The random word for `counter` (uint64 array) under `key`: mix64(key ^ mix64(counter))."""
    c = np.asarray(counter, dtype=np.uint64)
    return mix64(np.uint64(key) ^ mix64(c))


def uniform53(words):
    """Map 64-bit words to doubles in [0,1) using their top 53 bits (exact)."""
    w = np.asarray(words, dtype=np.uint64)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
