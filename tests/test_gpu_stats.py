"""Sweep statistics and the threshold rules of thumb (Sec. IV-D) on the GPU
against the oracle.  Integer statistics are compared exactly; modularity is
a ratio of exact integers rounded on both sides, compared to 2e-16 absolute
plus one part in 10^15."""
import itertools

import numpy as np
import pytest

import oracle as O
from graphgen import csr_from_pairs, small
from graphgen.batch import disjoint_union
from graphgen.dcsbm import dcsbm_csr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tec(cuda_device):
    import paper_2412_12382_gb300 as pkg
    from paper_2412_12382_gb300 import build
    build.build()
    pkg.load_library()
    return pkg


def _two_cliques_with_connector():
    pairs = [(a, b) for a, b in itertools.combinations(range(8), 2)]
    pairs += [(a + 8, b + 8) for a, b in itertools.combinations(range(8), 2)]
    pairs += [(16, v) for v in (0, 1, 2, 8, 9, 10)]
    u, v = np.array(pairs).T
    return csr_from_pairs(17, u, v)


def _batch():
    rng = np.random.default_rng(21)
    graphs = [_two_cliques_with_connector(), small.empty(3), small.complete(7), small.gnp(60, 0.12, rng),
              small.gnp(1, 0.5, rng), small.two_cliques_bridge(9, 6)]
    graphs += [dcsbm_csr(s, 200, 1500)[:2] for s in (40100, 40101, 40102)]
    return graphs


def _check(tec, graphs, measure, ps, qs):
    import torch
    from paper_2412_12382_gb300 import tectonic as T
    off, col, seg = disjoint_union(graphs)
    g = tec.Graph(torch.from_numpy(off).cuda(), torch.from_numpy(col).cuda())
    segd = torch.from_numpy(seg).cuda()
    lab, _ = g.sweep(measure, ps, qs, seg_off=segd)
    raw = g.sweep_stats(measure, ps, qs, lab, segd)
    st = T.stats_numpy(raw, len(ps), len(graphs))
    labh = lab.cpu().numpy()
    r1 = T.rule_of_thumb(raw, ps, qs, len(graphs), T.RULE_LARGEST_JUMP).cpu().numpy()
    r2 = T.rule_of_thumb(raw, ps, qs, len(graphs), T.RULE_MODULARITY).cpu().numpy()
    for i, (go, gc) in enumerate(graphs):
        ref = O.sweep_stats(go, gc, measure, ps, qs, labh[:, seg[i]:seg[i + 1]])
        for r, rs in enumerate(ref):
            got = st[r, i]
            assert (got["ncomp"], got["kept"], got["largest"], got["intra"]) == \
                (rs["ncomp"], rs["kept"], rs["largest"], rs["intra"]), (i, r)
            assert abs(got["modularity"] - rs["modularity"]) <= 2e-16 + 1e-15 * abs(rs["modularity"]), (i, r)
        assert r1[i] == O.rule_of_thumb(ps, qs, ref), i
        assert r2[i] == O.rule_modularity(ps, qs, [x["modularity"] for x in ref]), i
    g.free()
    return r1, r2


def test_stats_and_rules_match_oracle_tectonic_grid_shuffled(tec):
    rng = np.random.default_rng(5)
    perm = rng.permutation(64)
    ps = [int(b) for b in (np.arange(1, 65)[perm])]
    qs = [128] * 64
    r1, r2 = _check(tec, _batch(), O.TECTONIC, ps, qs)
    assert ps[r1[0]] == 19 and ps[r2[0]] == 19       # the two-clique fixture


def test_stats_match_oracle_tw_grid(tec):
    ps = list(range(-30, 1, 2))
    _check(tec, _batch(), O.TW, ps, [1] * len(ps))


def test_stats_without_segments_and_from_independent_passes(tec):
    import torch
    from paper_2412_12382_gb300 import tectonic as T
    off, col = dcsbm_csr(40200, 3000, 6000)[:2]
    g = tec.Graph(torch.from_numpy(off).cuda(), torch.from_numpy(col).cuda())
    ps, qs = list(range(1, 65)), [128] * 64
    lab, _ = g.sweep(O.TECTONIC, ps, qs)
    st = T.stats_numpy(g.sweep_stats(O.TECTONIC, ps, qs, lab), 64)
    ref = O.sweep_stats(off, col, O.TECTONIC, ps, qs, lab.cpu().numpy())
    for r in range(64):
        assert st[r, 0]["intra"] == ref[r]["intra"] and st[r, 0]["largest"] == ref[r]["largest"]
        assert abs(st[r, 0]["modularity"] - ref[r]["modularity"]) <= 2e-16 + 1e-15 * abs(ref[r]["modularity"])
    # labels of independent passes at the same thresholds give the same statistics
    seg = torch.tensor([0, g.n], dtype=torch.int64, device="cuda")
    ind = torch.empty_like(lab)
    for r, p in enumerate(ps):
        g.prune_components_batch(O.TECTONIC, torch.tensor([p], device="cuda"), torch.tensor([128], device="cuda"),
                                 seg, labels=ind[r], count=False)
    assert torch.equal(ind, lab)
    st2 = T.stats_numpy(g.sweep_stats(O.TECTONIC, ps, qs, ind, seg), 64)
    assert np.array_equal(st2, st)
    g.free()
