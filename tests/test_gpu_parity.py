"""Parity of the CUDA path (through the C ABI) with the oracle, element by element.

Counts, wedges, masks, labels and component counts must be bit-identical;
Tectonic weights must equal the oracle's single IEEE division exactly (0 ULP)
and TW weights the oracle's exact integers.
"""
import numpy as np
import pytest

import oracle as O
from graphgen import planted_partition, rmat_csr, sbm_csr, small

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tec(cuda_device):
    import paper_2412_12382_gb300 as pkg
    from paper_2412_12382_gb300 import build
    build.build()
    pkg.load_library()
    return pkg


def _u32(x):
    return x.cpu().numpy().view(np.uint32)


def _gpu_graph(tec, off, col, validate=True):
    import torch
    return tec.Graph(torch.from_numpy(np.asarray(off, dtype=np.int64)).cuda(),
                     torch.from_numpy(np.asarray(col, dtype=np.int32)).cuda(), validate=validate)


def check_all(tec, off, col, thresholds):
    """Every exported quantity against the oracle, for each (measure, p, q)."""
    n = len(off) - 1
    g = _gpu_graph(tec, off, col)
    eu, ev = O.edge_list(off, col)
    t, uni = O.edge_counts(off, col, eu, ev, nthreads=O.threads_available())
    wedge = O.wedges(t, uni)
    gu, gv = g.edge_list()
    assert np.array_equal(gu.cpu().numpy(), eu) and np.array_equal(gv.cpu().numpy(), ev)
    gt, gw = g.edge_support()
    assert np.array_equal(_u32(gt), t)
    assert np.array_equal(_u32(gw).astype(np.int64), wedge)
    w_tec = g.edge_weights(tec.TECTONIC).cpu().numpy()
    assert np.array_equal(w_tec.view(np.uint64), O.tectonic_weights(off, eu, ev, t).view(np.uint64))
    w_tw = g.edge_weights(tec.TW).cpu().numpy()
    assert np.array_equal(w_tw, O.tw_scores(t, wedge).astype(np.float64))
    w_jac = g.edge_weights(tec.JACCARD).cpu().numpy()
    assert np.array_equal(w_jac.view(np.uint64), O.jaccard_weights(t, uni).view(np.uint64))
    assert np.array_equal(g.edge_weights(tec.K3).cpu().numpy(), O.k3_scores(t).astype(np.float64))
    # K4 (a costly oracle on large hub-heavy graphs): when asked for, or on graphs up to 2M edges
    k4 = None
    if any(th[0] == O.K4 for th in thresholds) or len(eu) <= 2_000_000:
        k4 = O.edge_k4(off, col, eu, ev, nthreads=O.threads_available())
        assert np.array_equal(_u32(g.edge_k4()).astype(np.uint64), np.minimum(k4, 0xFFFFFFFF))
        assert np.array_equal(g.edge_weights(tec.K4).cpu().numpy(), k4.astype(np.float64))
    for measure, p, q in thresholds:
        keep, kept = O.prune(measure, off, eu, ev, t, uni, p, q, k4)
        labels, nc = O.components(n, eu, ev, keep)
        gkeep, gkept = g.prune(measure, p, q, mask=True)
        assert gkept == kept
        assert np.array_equal(gkeep.cpu().numpy(), keep)
        glab, gnc = g.components()
        assert gnc == nc
        assert np.array_equal(glab.cpu().numpy(), labels)
        flab, fnc = g.full_pass(measure, p, q)
        assert fnc == nc
        assert np.array_equal(flab.cpu().numpy(), labels)
    # the other staging of the triangle counts (hashed for every centre) gives the same counts
    g.set_core_staging(False)
    gt2, _ = g.edge_support()
    assert np.array_equal(_u32(gt2), t)
    g.set_core_staging(True)
    # and so does the probe-row tiling, with any number of vertex-id ranges
    for groups in (1, 3, 16, -1):
        g.set_support_tiling(groups)
        gt3, _ = g.edge_support()
        assert np.array_equal(_u32(gt3), t), f"tiling with {groups} ranges"
    g.set_support_tiling(0)
    g.free()


STD = [(O.TECTONIC, 1, 10), (O.TECTONIC, 3, 50), (O.TW, -30, 1), (O.TW, 0, 1), (O.TW, 3, 50),
       (O.JACCARD, 1, 5), (O.JACCARD, 1, 2), (O.K3, 3, 1), (O.K3, 7, 2), (O.K4, 1, 1), (O.K4, 5, 2)]


@pytest.mark.parametrize("name,graph", [
    ("K3", small.complete(3)),
    ("K20", small.complete(20)),
    ("star40", small.star(40)),
    ("cycle9", small.cycle(9)),
    ("cliques6+9", small.two_cliques_bridge(6, 9)),
    ("empty5", small.empty(5)),
    ("single_vertex", small.empty(1)),
])
def test_closed_form_graphs(tec, name, graph):
    off, col = graph
    check_all(tec, off, col, STD)


def test_single_edge_and_isolated_vertices(tec):
    from graphgen import csr_from_pairs
    off, col = csr_from_pairs(10, [3], [7])
    check_all(tec, off, col, STD + [(O.TECTONIC, 0, 1)])


@pytest.mark.parametrize("seed,n,p", [(1, 60, 0.3), (2, 300, 0.5), (3, 500, 0.05), (4, 1200, 0.2)])
def test_random_graphs_span_both_bins(tec, seed, n, p):
    # dense rows give oriented rows longer than 32 (block path), sparse ones the warp path
    off, col = small.gnp(n, p, np.random.default_rng(seed))
    check_all(tec, off, col, STD)


def test_sbm_config(tec):
    # planted partition: n=2000 in 4 blocks of 500, p_in=0.05, p_out=0.002, seed 1;
    # Tectonic and TW at 3/50, plus TW over the grid -30..0 step 2 of Table 4
    off, col, _ = planted_partition(4, 500, 0.05, 0.002, seed=1)
    th = [(O.TECTONIC, 3, 50), (O.TW, 3, 50)] + [(O.TW, d, 1) for d in range(-30, 1, 2)]
    check_all(tec, off, col, th)


def test_rmat_small_with_hubs(tec):
    off, col = rmat_csr(13, 16, seed=2)
    check_all(tec, off, col, [(O.TECTONIC, 1, 10), (O.TW, -20, 1), (O.TECTONIC, (1 << 40) + 1, 10 << 40)])


def test_imbalanced_sbm_theorem1(tec):
    off, col, _ = sbm_csr([50, 50], [[0.1, 0.05], [0.05, 0.8]], seed=3)
    check_all(tec, off, col, [(O.TW, d, 1) for d in range(-40, 12, 4)] + [(O.TECTONIC, 1, 25)])


def test_complete_graph_chunked_rows(tec):
    # K_9000: every degree ties, so ranks follow ids and vertex 0 has 8999
    # oriented neighbours, more than one shared-memory chunk.  Closed
    # form: t = n - 2 on every edge, wedge = 0.
    import torch
    k = 9000
    col = np.empty(k * (k - 1), dtype=np.int32)
    ids = np.arange(k, dtype=np.int32)
    for u in range(k):
        col[u * (k - 1):(u + 1) * (k - 1)] = np.delete(ids, u)
    off = np.arange(0, k * (k - 1) + 1, k - 1, dtype=np.int64)
    g = _gpu_graph(tec, off, col, validate=False)
    for core, groups in ((True, 0), (False, 0), (True, 2), (True, 7)):   # bitmap chunks of 8192 ids,
        g.set_core_staging(core)                                         # hashed chunks of 4096, tiled
        g.set_support_tiling(groups)
        t, w = g.edge_support()
        assert int(t.min()) == k - 2 and int(t.max()) == k - 2
        assert int(w.min()) == 0 and int(w.max()) == 0
    g.set_support_tiling(0)
    lab, nc = g.full_pass(tec.TECTONIC, k - 2, 2 * (k - 1))       # exactly the common weight: keep all
    assert nc == 1 and int(lab.max()) == 0
    lab, nc = g.full_pass(tec.TECTONIC, k - 2 + 1, 2 * (k - 1))   # just above: drop all
    assert nc == k and torch.equal(lab.cpu(), torch.arange(k, dtype=torch.int32))
    g.free()


def test_reload_and_capacity(tec):
    import torch
    off1, col1 = small.two_cliques_bridge(5, 7)
    off2, col2 = small.complete(6)
    g = tec.Graph(n_cap=100, nnz_cap=1000)
    for off, col in ((off1, col1), (off2, col2), (off1, col1)):
        g.load(torch.from_numpy(off).cuda(), torch.from_numpy(col).cuda())
        ref = O.full_pass(off, col, O.TECTONIC, 1, 4)
        lab, nc = g.full_pass(tec.TECTONIC, 1, 4)
        assert nc == ref.ncomp and np.array_equal(lab.cpu().numpy(), ref.labels)
    # host-pointer load and int32 offsets
    g.load(off1.astype(np.int32), col1)
    lab, nc = g.full_pass(tec.TECTONIC, 1, 4)
    ref = O.full_pass(off1, col1, O.TECTONIC, 1, 4)
    assert nc == ref.ncomp and np.array_equal(lab.cpu().numpy(), ref.labels)
    with pytest.raises(tec.TectonicError) as e:
        big = small.complete(40)            # 1560 entries > nnz_cap = 1000
        g.load(torch.from_numpy(big[0]).cuda(), torch.from_numpy(big[1]).cuda())
    assert e.value.status == 1
    g.free()


def test_full_pass_host_buffers(tec):
    off, col, _ = planted_partition(4, 500, 0.05, 0.002, seed=1)
    g = tec.Graph(n_cap=len(off) - 1, nnz_cap=len(col))
    lab, nc = g.full_pass_host(off, col, tec.TECTONIC, 3, 50)
    ref = O.full_pass(off, col, O.TECTONIC, 3, 50)
    assert nc == ref.ncomp and np.array_equal(lab, ref.labels)
    g.free()


def test_errors(tec):
    import torch
    off, col = small.complete(5)
    g = _gpu_graph(tec, off, col)
    with pytest.raises(tec.TectonicError) as e:
        g.components()
    assert e.value.status == 7                     # TEC_ESTATE: no prune yet
    with pytest.raises(tec.TectonicError) as e:
        g.prune(tec.TECTONIC, 1, 0)
    assert e.value.status == 1                     # q <= 0
    with pytest.raises(tec.TectonicError) as e:
        g.prune(tec.TECTONIC, 1 << 62, 1)
    assert e.value.status == 5                     # overflow guard
    # an unsorted row, a self-loop and an asymmetric graph are rejected by validation
    bad = col.copy(); bad[0], bad[1] = bad[1], bad[0]
    for c, o in ((bad, off),
                 (np.array([0, 1], dtype=np.int32), np.array([0, 1, 2], dtype=np.int64)),
                 (np.array([1, 0], dtype=np.int32), np.array([0, 1, 1, 2], dtype=np.int64))):
        with pytest.raises(tec.TectonicError) as e:
            g.load(torch.from_numpy(o).cuda(), torch.from_numpy(c).cuda(), validate=True)
        assert e.value.status == 6
    # the graph stays usable after a rejected load
    g.load(torch.from_numpy(off).cuda(), torch.from_numpy(col).cuda(), validate=True)
    lab, nc = g.full_pass(tec.TECTONIC, 1, 10)
    assert nc == 1
    g.free()


def test_gpu_generator_matches_host(cuda_device):
    # the device R-MAT sampler must reproduce the host generator bit for bit,
    # including when it splits the sources into several bucket groups
    from graphgen.gpu import rmat_csr_gpu
    for scale, ef, seed, group in ((6, 4, 9, 1 << 20), (10, 8, 5, 1 << 12), (13, 16, 2, 1 << 16)):
        off, col = rmat_csr(scale, ef, seed=seed)
        goff, gcol = rmat_csr_gpu(scale, ef, seed=seed, max_group=group)
        assert np.array_equal(goff.cpu().numpy(), off)
        assert np.array_equal(gcol.cpu().numpy(), col)


def test_rmat20_config_full_parity(tec):
    # R-MAT scale 20, edge factor 16, seed 2: every edge's t and wedge, both
    # weights, masks and labels at theta = 1/10 for Tectonic and TW
    from graphgen.gpu import rmat_csr_gpu
    goff, gcol = rmat_csr_gpu(20, 16, seed=2)
    off, col = goff.cpu().numpy(), gcol.cpu().numpy()
    del goff, gcol
    check_all(tec, off, col, [(O.TECTONIC, 1, 10), (O.TW, 1, 10)])


def test_repeated_runs_are_identical(tec):
    # atomics and lock-free union-find run in a different order every time; the
    # exact results must not: 40 runs of every path against the oracle
    import torch
    off, col, _ = planted_partition(4, 500, 0.05, 0.002, seed=1)
    ref = O.full_pass(off, col, O.TECTONIC, 3, 50)
    g = _gpu_graph(tec, off, col)
    g2 = tec.Graph(n_cap=len(off) - 1, nnz_cap=len(col))
    for _ in range(40):
        g.support()
        t, _ = g.edge_support(wedges=False)
        assert np.array_equal(_u32(t), ref.t)
        lab, nc = g.full_pass(tec.TECTONIC, 3, 50)
        assert nc == ref.ncomp and np.array_equal(lab.cpu().numpy(), ref.labels)
        hl, hnc = g2.full_pass_host(off, col, tec.TECTONIC, 3, 50)
        assert hnc == ref.ncomp and np.array_equal(hl, ref.labels)
    g.free()
    g2.free()


def test_dcsbm_gpu_batch_matches_host(cuda_device):
    from graphgen.batch import disjoint_union
    from graphgen.dcsbm import dcsbm_csr
    from graphgen.gpu import dcsbm_batch_gpu
    seeds = [1000, 1001, 1002, 20000]
    host = [dcsbm_csr(s, 1000, 6000) for s in seeds]
    off, col, seg = disjoint_union([(h[0], h[1]) for h in host])
    goff, gcol, gseg, gtruth, _ = dcsbm_batch_gpu(seeds, 1000, 6000)
    assert np.array_equal(gseg.cpu().numpy(), seg)
    assert np.array_equal(goff.cpu().numpy(), off)
    assert np.array_equal(gcol.cpu().numpy(), col)
    assert np.array_equal(gtruth.cpu().numpy(), np.concatenate([h[2] for h in host]))


def test_jaccard_sweep_and_prop1_on_device(tec):
    """Jaccard at p/q and Tectonic at p/(p+q) give the same components on the
    device (Proposition 1), and a Jaccard sweep equals the oracle's passes."""
    import torch
    off, col, _ = planted_partition(4, 500, 0.05, 0.002, seed=1)
    g = _gpu_graph(tec, off, col)
    ps, qs = [1, 1, 1, 2, 3], [20, 10, 5, 5, 5]
    lab, nc = g.sweep(tec.JACCARD, ps, qs)
    ol, onc = O.sweep(off, col, O.JACCARD, ps, qs)
    assert np.array_equal(lab.cpu().numpy(), ol) and np.array_equal(nc, onc)
    for i, (p, q) in enumerate(zip(ps, qs)):
        tl, _ = g.full_pass(tec.TECTONIC, p, p + q)
        assert torch.equal(tl, lab[i])
    g.free()


def test_k4_large_common_neighbourhoods_and_sweep(tec):
    """K4 on a book graph: spine edge (0, 1), pages 2..1101 adjacent to both
    ends and joined in a path, so C(0, 1) holds 1100 ids (more than a warp's
    shared slice: the unstored path) and K4(0, 1) = 1099 path edges; then a
    K4 sweep against the oracle."""
    from graphgen import csr_from_pairs
    pages = np.arange(2, 1102)
    u = np.concatenate([[0], np.zeros(1100, int), np.ones(1100, int), pages[:-1]])
    v = np.concatenate([[1], pages, pages, pages[1:]])
    off, col = csr_from_pairs(1102, u, v)
    check_all(tec, off, col, [(O.K4, 1, 1), (O.K4, 2, 1), (O.K4, 1099, 1), (O.TECTONIC, 1, 10)])
    g = _gpu_graph(tec, off, col)
    eu, ev = O.edge_list(off, col)
    assert _u32(g.edge_k4())[(eu == 0) & (ev == 1)][0] == 1099
    g.free()
    off, col, _ = planted_partition(4, 300, 0.08, 0.004, seed=5)
    g = _gpu_graph(tec, off, col)
    ps, qs = [0, 1, 2, 3, 5, 8], [1] * 6
    lab, nc = g.sweep(tec.K4, ps, qs)
    ol, onc = O.sweep(off, col, O.K4, ps, qs)
    assert np.array_equal(lab.cpu().numpy(), ol) and np.array_equal(nc, onc)
    g.free()
