"""R-MAT scale 26, edge factor 32, seed 3 -- the benchmark workload -- in the
launch configuration bench.py times (fused full pass, Tectonic at 1/10).

The oracle cannot merge every row of this graph, so triangle counts, wedges,
weights and the keep mask are checked on a sample of edges that it computes
one by one (uniform edges plus the edges of the highest-degree vertex), and
the component labels against the oracle's breadth-first search over the kept
edges of the whole graph.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tec(cuda_device):
    import paper_2412_12382_gb300 as pkg
    from paper_2412_12382_gb300 import build
    build.build()
    pkg.load_library()
    return pkg


def test_rmat26_full_pass(tec):
    import torch
    from graphgen.gpu import rmat_csr_gpu
    off, col = rmat_csr_gpu(26, 32, seed=3)
    n, nnz = off.numel() - 1, col.numel()
    g = tec.Graph(off, col)
    labels, ncomp = g.full_pass(tec.TECTONIC, 1, 10)
    lab = labels.cpu().numpy()
    t, w = g.edge_support()
    wt = g.edge_weights(tec.TECTONIC)
    keep, kept = g.prune(tec.TECTONIC, 1, 10, mask=True)
    eu, ev = g.edge_list()
    m = eu.numel()
    off_h = off.cpu().numpy().astype(np.int64)
    col_h = col.cpu().numpy().astype(np.int32)
    del off, col
    # sampled per-edge quantities: uniform edges and every edge of the top hub
    rng = np.random.default_rng(26)
    hub = int(np.argmax(np.diff(off_h)))
    idx = np.unique(np.concatenate([rng.integers(0, m, 20000),
                                    np.nonzero((eu == hub).cpu().numpy() | (ev == hub).cpu().numpy())[0][:2000]]))
    it = torch.from_numpy(idx).cuda()
    su, sv = eu[it].cpu().numpy(), ev[it].cpu().numpy()
    ot, ouni = O.edge_counts(off_h, col_h, su, sv, nthreads=O.threads_available())
    assert np.array_equal(t[it].cpu().numpy().view(np.uint32), ot)
    assert np.array_equal(w[it].cpu().numpy().view(np.uint32).astype(np.int64), O.wedges(ot, ouni))
    assert np.array_equal(wt[it].cpu().numpy(), O.tectonic_weights(off_h, su, sv, ot))
    okeep, _ = O.prune(O.TECTONIC, off_h, su, sv, ot, ouni, 1, 10)
    assert np.array_equal(keep[it].cpu().numpy(), okeep)
    # labels: the oracle's BFS over the kept edges of the whole graph
    kmask = keep.bool()
    ku = eu[kmask].cpu().numpy()
    kv = ev[kmask].cpu().numpy()
    assert len(ku) == kept
    del eu, ev, keep, t, w, wt, kmask
    olab, onc = O.components(n, ku, kv, np.ones(len(ku), dtype=np.uint8))
    assert ncomp == onc
    assert np.array_equal(lab, olab)
    g.free()
