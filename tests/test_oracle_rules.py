"""Pins of the oracle's sweep statistics and rules of thumb (Sec. IV-D, Fig. 6)."""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from graphgen import csr_from_pairs, small

GRID_P = list(range(1, 65))
GRID_Q = [128] * 64


def _two_cliques_with_connector():
    """K8 on 0..7 and K8 on 8..15; vertex 16 adjacent to 0, 1, 2 and 8, 9, 10."""
    pairs = [(a, b) for a, b in itertools.combinations(range(8), 2)]
    pairs += [(a + 8, b + 8) for a, b in itertools.combinations(range(8), 2)]
    pairs += [(16, v) for v in (0, 1, 2, 8, 9, 10)]
    u, v = np.array(pairs).T
    return csr_from_pairs(17, u, v)


def test_stats_against_brute_force():
    rng = np.random.default_rng(3)
    off, col = small.gnp(40, 0.15, rng)
    n = len(off) - 1
    labels, _ = O.sweep(off, col, O.TECTONIC, GRID_P, GRID_Q)
    stats = O.sweep_stats(off, col, O.TECTONIC, GRID_P, GRID_Q, labels)
    eu, ev = O.edge_list(off, col)
    deg = np.diff(off)
    m = len(eu)
    for i, st in enumerate(stats):
        lab = labels[i]
        comps = {}
        for x in range(n):
            comps.setdefault(int(lab[x]), []).append(x)
        assert st["ncomp"] == len(comps)
        assert st["largest"] == max(len(c) for c in comps.values())
        assert st["intra"] == sum(1 for a, b in zip(eu, ev) if lab[a] == lab[b])
        vol2 = sum(sum(int(deg[x]) for x in c) ** 2 for c in comps.values())
        assert st["sum_vol2"] == vol2
        assert st["modularity"] == float(Fraction(4 * m * st["intra"] - vol2, 4 * m * m))
        assert abs(st["modularity"] - O.modularity(off, col, lab)) <= 1e-12
    # arbitrary (not nested) labelings: modularity still agrees with the double sum
    for k in (1, 3, 40):
        lab = rng.integers(0, k, n)
        st = O.sweep_stats(off, col, O.TECTONIC, [1], [128], [lab])[0]
        assert abs(st["modularity"] - O.modularity(off, col, lab)) <= 1e-12
    # one community: Q = 0 exactly
    st = O.sweep_stats(off, col, O.TECTONIC, [1], [128], [np.zeros(n, dtype=np.int64)])[0]
    assert st["modularity"] == 0.0 and st["intra"] == m


def test_rules_pick_the_two_cliques():
    off, col = _two_cliques_with_connector()
    labels, _ = O.sweep(off, col, O.TECTONIC, GRID_P, GRID_Q)
    stats = O.sweep_stats(off, col, O.TECTONIC, GRID_P, GRID_Q, labels)
    largest = [s["largest"] for s in stats]
    # hand-computed levels: connector edges b = 18, connector-adjacent pairs 56,
    # plain pairs 54, mixed pairs 51 (b = floor(128 t / (deg u + deg v)))
    expect = {b: (17 if b <= 18 else 8 if b <= 51 else 5 if b <= 54 else 3 if b <= 56 else 1) for b in GRID_P}
    assert largest == [expect[b] for b in GRID_P]
    r1 = O.rule_largest_jump(GRID_P, GRID_Q, largest)
    r2 = O.rule_modularity(GRID_P, GRID_Q, [s["modularity"] for s in stats])
    assert GRID_P[r1] == 19 and GRID_P[r2] == 19
    assert O.rule_of_thumb(GRID_P, GRID_Q, stats) == r1
    two = labels[r1]
    assert len(set(two[:8])) == 1 and len(set(two[8:16])) == 1 and two[0] != two[8] and two[16] == 16


def test_no_jump_falls_back_to_modularity():
    # a perfect matching: every edge has t = 0, so no grid threshold keeps any
    off, col = csr_from_pairs(8, np.array([0, 2, 4, 6]), np.array([1, 3, 5, 7]))
    labels, _ = O.sweep(off, col, O.TECTONIC, GRID_P, GRID_Q)
    stats = O.sweep_stats(off, col, O.TECTONIC, GRID_P, GRID_Q, labels)
    assert all(s["largest"] == 1 and s["kept"] == 0 for s in stats)
    assert O.rule_largest_jump(GRID_P, GRID_Q, [s["largest"] for s in stats]) is None
    assert O.rule_of_thumb(GRID_P, GRID_Q, stats) == 0      # all modularities equal: the lowest threshold


def test_modularity_against_networkx():
    """Newman-Girvan modularity of the sweep's levels and of arbitrary
    labelings, against networkx's implementation of the same definition."""
    nx = pytest.importorskip("networkx")
    nxc = pytest.importorskip("networkx.algorithms.community")
    rng = np.random.default_rng(11)
    off, col = small.gnp(60, 0.12, rng)
    n = len(off) - 1
    eu, ev = O.edge_list(off, col)
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_edges_from(zip(eu.tolist(), ev.tolist()))
    labels, _ = O.sweep(off, col, O.TECTONIC, GRID_P, GRID_Q)
    cases = [labels[i] for i in (0, 8, 20, 63)] + [rng.integers(0, k, n) for k in (2, 5)]
    stats = O.sweep_stats(off, col, O.TECTONIC, [1] * len(cases), [128] * len(cases), cases)
    for lab, st in zip(cases, stats):
        parts = {}
        for x in range(n):
            parts.setdefault(int(lab[x]), set()).add(x)
        assert abs(st["modularity"] - nxc.modularity(G, list(parts.values()))) <= 1e-12
