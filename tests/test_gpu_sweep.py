"""Multi-threshold sweep (maximum spanning forest + offline union-find) against
the oracle's definition: one independent prune + components per threshold."""
import numpy as np
import pytest

import oracle as O
from graphgen import planted_partition, rmat_csr, sbm_csr, small
from graphgen.batch import disjoint_union

pytestmark = pytest.mark.gpu

GRID = [(i, 128) for i in range(1, 65)]          # theta_i = i/128


@pytest.fixture(scope="module")
def tec(cuda_device):
    import paper_2412_12382_gb300 as pkg
    from paper_2412_12382_gb300 import build
    build.build()
    pkg.load_library()
    return pkg


def _graph(tec, off, col, n_cap=None, nnz_cap=None):
    import torch
    return tec.Graph(torch.from_numpy(np.asarray(off, dtype=np.int64)).cuda(),
                     torch.from_numpy(np.asarray(col, dtype=np.int32)).cuda(), n_cap=n_cap, nnz_cap=nnz_cap)


def check_sweep(tec, off, col, measure, thresholds):
    ps = [p for p, _ in thresholds]
    qs = [q for _, q in thresholds]
    ref_lab, ref_nc = O.sweep(off, col, measure, ps, qs)
    g = _graph(tec, off, col)
    lab, nc = g.sweep(measure, ps, qs)
    assert np.array_equal(nc, ref_nc)
    assert np.array_equal(lab.cpu().numpy(), ref_lab)
    g.free()


def test_sweep_sbm_tectonic_grid(tec):
    off, col, _ = planted_partition(4, 500, 0.05, 0.002, seed=1)
    check_sweep(tec, off, col, O.TECTONIC, GRID)


def test_sweep_tw_unsorted_with_repeats(tec):
    off, col, _ = sbm_csr([50, 50], [[0.1, 0.05], [0.05, 0.8]], seed=3)
    th = [(d, 1) for d in (-10, -30, 0, -2, 4, -30, 12, -40, 2)] + [(3, 50), (-7, 3)]
    check_sweep(tec, off, col, O.TW, th)


def test_sweep_rmat_and_random(tec):
    off, col = rmat_csr(13, 16, seed=2)
    check_sweep(tec, off, col, O.TECTONIC, GRID)
    off, col = small.gnp(400, 0.3, np.random.default_rng(7))
    check_sweep(tec, off, col, O.TECTONIC, GRID[::3] + [(0, 1), (1, 2)])


def test_sweep_127_thresholds_wide_and_equal_values(tec):
    """The largest k (127) in shuffled order, with 63 grid values b/128 also
    given as (b 2^33)/(128 2^33): equal values in another representation, and
    numerators and denominators past 2^28, so every edge level comes from
    128-bit comparisons."""
    rng = np.random.default_rng(12)
    th = GRID + [(b << 33, 128 << 33) for b in range(1, 64)]
    assert len(th) == 127
    th = [th[i] for i in rng.permutation(len(th))]
    off, col, _ = planted_partition(4, 200, 0.25, 0.01, seed=4)      # levels from 1 to 800 components
    check_sweep(tec, off, col, O.TECTONIC, th)
    tw = [(d << 35, 1 << 35) for d in range(-40, 10)] + [(d, 1) for d in range(-40, 10)]
    off, col, _ = sbm_csr([50, 50], [[0.1, 0.05], [0.05, 0.8]], seed=5)
    check_sweep(tec, off, col, O.TW, [tw[i] for i in rng.permutation(len(tw))])


def test_sweep_degenerate(tec):
    for off, col in (small.complete(12), small.star(9), small.empty(4), small.two_cliques_bridge(5, 6)):
        check_sweep(tec, off, col, O.TECTONIC, [(0, 1), (1, 1000), (5, 12), (1, 2), (1, 1)])


def test_sweep_batch_of_uneven_graphs(tec):
    import torch
    graphs = [planted_partition(3, 40, 0.3, 0.02, seed=s)[:2] for s in (1, 2)]
    graphs += [rmat_csr(10, 8, seed=5), small.empty(3), small.complete(7), small.gnp(150, 0.1, np.random.default_rng(3))]
    off, col, seg = disjoint_union(graphs)
    g = _graph(tec, off, col)
    lab, nc = g.sweep(O.TECTONIC, [p for p, _ in GRID], [q for _, q in GRID],
                      seg_off=torch.from_numpy(seg).cuda())
    lab = lab.cpu().numpy()
    for gi, (go, gc) in enumerate(graphs):
        ref_lab, ref_nc = O.sweep(go, gc, O.TECTONIC, [p for p, _ in GRID], [q for _, q in GRID])
        assert np.array_equal(nc[:, gi], ref_nc)
        assert np.array_equal(lab[:, seg[gi]:seg[gi + 1]], ref_lab)
    g.free()


def test_sweep_then_prune_components_still_agree(tec):
    off, col, _ = planted_partition(4, 500, 0.05, 0.002, seed=1)
    g = _graph(tec, off, col)
    lab, nc = g.sweep(O.TECTONIC, [1, 3, 9], [40, 50, 128])
    for i, (p, q) in enumerate(((1, 40), (3, 50), (9, 128))):
        g.prune(O.TECTONIC, p, q)
        cl, cn = g.components()
        assert cn == nc[i] and np.array_equal(cl.cpu().numpy(), lab[i].cpu().numpy())
    g.free()


def test_sweep_captured_in_a_cuda_graph(tec):
    """With its buffers allocated and no host read-back, tec_sweep issues only
    kernels and memsets on the graph's stream: captured once into a CUDA
    graph, every replay recomputes the same labels."""
    import torch
    from graphgen.batch import disjoint_union
    from graphgen.dcsbm import dcsbm_csr
    graphs = [dcsbm_csr(s, 500, 4000)[:2] for s in range(41000, 41006)]
    off, col, seg = disjoint_union(graphs)
    ps, qs = list(range(1, 65)), [128] * 64
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = tec.Graph(torch.from_numpy(off).cuda(), torch.from_numpy(col).cuda())
        segd = torch.from_numpy(seg).cuda()
        ref, _ = g.sweep(O.TECTONIC, ps, qs, seg_off=segd, count=False)   # allocates the sweep buffers
    s.synchronize()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=s):
        lab, _ = g.sweep(O.TECTONIC, ps, qs, seg_off=segd, count=False)
    for _ in range(2):
        lab.fill_(-1)
        cg.replay()
        torch.cuda.synchronize()
        assert torch.equal(lab, ref)
    labh = lab.cpu().numpy()
    for i, (go, gc) in enumerate(graphs[:2]):
        ol, _ = O.sweep(go, gc, O.TECTONIC, ps, qs)
        assert np.array_equal(labh[:, seg[i]:seg[i + 1]], ol)
    g.sync()
    g.free()
