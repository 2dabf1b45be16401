"""Failure paths of the library, driven from the host in a debug build
(-DTEC_DEBUG, loaded through TEC_LIBRARY by test_gpu_failure.py).

Nothing here faults or hangs a GPU: a lowered iteration cap makes a bounded
device loop stop early and report TEC_ETIMEOUT through the status word, and
an injected allocation failure is a host-side refusal of one named buffer.
Each case then checks that the graph is still usable and that the fallback
path gives the oracle's results.  Prints one JSON object of case -> outcome.
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from graphgen import planted_partition, rmat_csr  # noqa: E402


def _graph(T, off, col):
    import torch
    return T.Graph(torch.from_numpy(np.asarray(off, dtype=np.int64)).cuda(),
                   torch.from_numpy(np.asarray(col, dtype=np.int32)).cuda())


def _status(T, fn):
    try:
        fn()
    except T.TectonicError as e:
        return e.status
    return 0


def main():
    import torch
    import paper_2412_12382_gb300 as T
    out = {}
    off, col, _ = planted_partition(4, 500, 0.05, 0.002, seed=1)
    ref = O.full_pass(off, col, O.TECTONIC, 3, 50)
    g = _graph(T, off, col)

    # 1. union-find retry cap 0: every link of two distinct roots gives up
    os.environ["TEC_DEBUG_LINK_CAP"] = "0"
    out["link_cap_status"] = _status(T, lambda: g.full_pass(T.TECTONIC, 3, 50))
    del os.environ["TEC_DEBUG_LINK_CAP"]
    lab, nc = g.full_pass(T.TECTONIC, 3, 50)
    out["link_cap_recall_ok"] = bool(nc == ref.ncomp and np.array_equal(lab.cpu().numpy(), ref.labels))

    # 2. Boruvka rounds capped at 1 on a graph whose forest needs more
    ps, qs = [1, 2, 4, 8], [128] * 4
    ol, onc = O.sweep(off, col, O.TECTONIC, ps, qs)
    os.environ["TEC_DEBUG_MSF_ROUNDS"] = "1"
    out["msf_rounds_status"] = _status(T, lambda: g.sweep(T.TECTONIC, ps, qs))
    del os.environ["TEC_DEBUG_MSF_ROUNDS"]
    sl, snc = g.sweep(T.TECTONIC, ps, qs)
    out["msf_rounds_recall_ok"] = bool(np.array_equal(sl.cpu().numpy(), ol) and np.array_equal(snc, onc))
    g.free()

    # 3. allocation failures of optional buffers: the fallbacks give the same results
    roff, rcol = rmat_csr(13, 16, seed=2)
    rt, _ = O.edge_counts(roff, rcol)
    rol, ronc = O.sweep(roff, rcol, O.TECTONIC, ps, qs)
    for name in ("live edge", "core", "tiling"):
        os.environ["TEC_DEBUG_FAIL_ALLOC"] = name
        g = _graph(T, roff, rcol)
        g.set_support_tiling(3)
        t, _ = g.edge_support(wedges=False)
        sl, snc = g.sweep(T.TECTONIC, ps, qs)
        out[f"fail_alloc_{name}_ok"] = bool(np.array_equal(t.cpu().numpy().view(np.uint32), rt)
                                            and np.array_equal(sl.cpu().numpy(), rol) and np.array_equal(snc, ronc))
        del os.environ["TEC_DEBUG_FAIL_ALLOC"]
        g.free()

    # 4. a lazily allocated buffer that fails, then the same call again
    g = T.Graph(n_cap=len(off) - 1, nnz_cap=len(col))
    os.environ["TEC_DEBUG_FAIL_ALLOC"] = "label buffer"
    out["lazy_alloc_status"] = _status(T, lambda: g.full_pass_host(off, col, T.TECTONIC, 3, 50))
    del os.environ["TEC_DEBUG_FAIL_ALLOC"]
    hl, hnc = g.full_pass_host(off, col, T.TECTONIC, 3, 50)
    out["lazy_alloc_retry_ok"] = bool(hnc == ref.ncomp and np.array_equal(hl, ref.labels))

    # 5. no buffer was written past its end in any of the above
    out["canaries_status"] = _status(T, g.sync)
    g.free()
    torch.cuda.synchronize()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
