"""A batch of graphs as one disjoint union (block-diagonal symmetric CSR)."""
from __future__ import annotations

import numpy as np


def disjoint_union(graphs):
    """graphs: list of (off, col).  Returns (off, col, seg_off) where graph g
    owns vertices seg_off[g] .. seg_off[g+1]-1 of the union."""
    seg = [0]
    offs, cols = [], []
    base_e = 0
    for off, col in graphs:
        off = np.asarray(off, dtype=np.int64)
        n = len(off) - 1
        offs.append(off[:-1] + base_e)
        cols.append(np.asarray(col, dtype=np.int64) + seg[-1])
        base_e += int(off[-1])
        seg.append(seg[-1] + n)
    off = np.concatenate(offs + [np.array([base_e], dtype=np.int64)])
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    return off, col, np.asarray(seg, dtype=np.int64)
