"""Pins of the oracle against the paper and against mathematics (CPU only).

Each test checks the oracle against something other than itself: hand-worked
fixtures, closed forms of special graphs, brute force on tiny graphs, dense
matrix identities, exact rational arithmetic, a library routine, or the
expectations of the paper's Table 2.
"""
from fractions import Fraction
import itertools
import math
import os

import numpy as np
import pytest

import oracle as O
from graphgen import csr_from_pairs, dense_adjacency, sbm_csr, small, upper_pairs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_graphs(count=12, seed=7):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(2, 40))
        p = float(rng.uniform(0.05, 0.7))
        out.append(small.gnp(n, p, rng))
    return out


def _nbrs(off, col):
    return [set(col[off[u]:off[u + 1]].tolist()) for u in range(len(off) - 1)]


# ----------------------------------------------------------- counts


def test_bowtie_hand_counts():
    rows = np.loadtxt(os.path.join(GOLDEN, "bowtie_counts.txt"), dtype=np.int64)
    off, col = csr_from_pairs(5, rows[:, 0], rows[:, 1])
    eu, ev = O.edge_list(off, col)
    assert (eu == rows[:, 0]).all() and (ev == rows[:, 1]).all()
    t, uni = O.edge_counts(off, col, eu, ev)
    wedge = O.wedges(t, uni)
    assert (t == rows[:, 2]).all()
    assert (wedge == rows[:, 3]).all()
    assert (O.tw_scores(t, wedge) == rows[:, 4]).all()
    w = O.tectonic_weights(off, eu, ev, t)
    assert (w == rows[:, 5] / rows[:, 6]).all()


def test_counts_brute_force_sets():
    for off, col in _rand_graphs():
        nb = _nbrs(off, col)
        eu, ev = O.edge_list(off, col)
        t, uni = O.edge_counts(off, col, eu, ev)
        for e, (u, v) in enumerate(zip(eu, ev)):
            assert t[e] == len(nb[u] & nb[v])
            assert uni[e] == len(nb[u] | nb[v])


def test_counts_triple_loop_brute_force():
    # t(u,v) counted as the number of w with all three edges present, O(n^3)
    for off, col in _rand_graphs(6, seed=11):
        n = len(off) - 1
        A = dense_adjacency(off, col)
        eu, ev = O.edge_list(off, col)
        t, _ = O.edge_counts(off, col, eu, ev)
        tri = {}
        for a, b, c in itertools.combinations(range(n), 3):
            if A[a, b] and A[b, c] and A[a, c]:
                for x, y in ((a, b), (b, c), (a, c)):
                    tri[(x, y)] = tri.get((x, y), 0) + 1
        for e, (u, v) in enumerate(zip(eu, ev)):
            assert t[e] == tri.get((int(u), int(v)), 0)


def test_counts_dense_matrix_identities():
    for off, col in _rand_graphs(8, seed=3):
        A = dense_adjacency(off, col)
        A2 = A @ A
        eu, ev = O.edge_list(off, col)
        t, _ = O.edge_counts(off, col, eu, ev)
        assert (t.astype(np.int64) == A2[eu, ev]).all()
        # sum_e t(e) = 3 T and trace(A^3) = 6 T
        assert 2 * int(t.sum()) == int(np.trace(A2 @ A))


def test_union_inclusion_exclusion_and_wedge_identity():
    for off, col in _rand_graphs(10, seed=5):
        d = O.degrees(off)
        eu, ev = O.edge_list(off, col)
        t, uni = O.edge_counts(off, col, eu, ev)
        assert (uni.astype(np.int64) == d[eu] + d[ev] - t).all()
        wedge = O.wedges(t, uni)
        assert (wedge >= 0).all()
        T = int(t.sum()) // 3
        # sum_e wedge(e) = 2 (sum_v C(d_v, 2) - 3T): every open 2-path is seen from its 2 edges
        assert int(wedge.sum()) == 2 * (int((d * (d - 1) // 2).sum()) - 3 * T)


def test_threads_do_not_change_counts():
    off, col = _rand_graphs(1, seed=99)[0]
    eu, ev = O.edge_list(off, col)
    a = O.edge_counts(off, col, eu, ev, nthreads=1)
    b = O.edge_counts(off, col, eu, ev, nthreads=4)
    assert (a[0] == b[0]).all() and (a[1] == b[1]).all()


@pytest.mark.parametrize("k", [3, 4, 7, 20])
def test_complete_graph_closed_forms(k):
    off, col = small.complete(k)
    eu, ev = O.edge_list(off, col)
    t, uni = O.edge_counts(off, col, eu, ev)
    wedge = O.wedges(t, uni)
    assert (t == k - 2).all()
    assert (wedge == 0).all()
    assert (O.tw_scores(t, wedge) == k - 2).all()
    w = O.tectonic_weights(off, eu, ev, t)
    assert (w == float(Fraction(k - 2, 2 * (k - 1)))).all()
    # histogram: every edge in bin floor(128 (k-2) / (2(k-1)))
    h = O.histogram64(off, eu, ev, t)
    assert h[(128 * (k - 2)) // (2 * (k - 1))] == k * (k - 1) // 2


@pytest.mark.parametrize("k", [1, 2, 5, 30])
def test_star_closed_forms(k):
    off, col = small.star(k)
    eu, ev = O.edge_list(off, col)
    t, uni = O.edge_counts(off, col, eu, ev)
    wedge = O.wedges(t, uni)
    assert (t == 0).all()
    assert (wedge == k - 1).all()
    assert (O.tw_scores(t, wedge) == 1 - k).all()


@pytest.mark.parametrize("k", [4, 5, 9])
def test_cycle_closed_forms(k):
    off, col = small.cycle(k)
    eu, ev = O.edge_list(off, col)
    t, uni = O.edge_counts(off, col, eu, ev)
    assert (t == 0).all()
    assert (O.wedges(t, uni) == 2).all()


@pytest.mark.parametrize("a,b", [(4, 4), (5, 8), (10, 3)])
def test_two_cliques_bridge(a, b):
    off, col = small.two_cliques_bridge(a, b)
    eu, ev = O.edge_list(off, col)
    t, uni = O.edge_counts(off, col, eu, ev)
    w = O.tectonic_weights(off, eu, ev, t)
    x, y = a - 1, a
    for e, (u, v) in enumerate(zip(eu.tolist(), ev.tolist())):
        if (u, v) == (x, y):
            assert t[e] == 0 and w[e] == 0.0
        elif u < a and v < a:
            k = a
            exp = Fraction(k - 2, 2 * k - 1) if x in (u, v) else Fraction(k - 2, 2 * (k - 1))
            assert w[e] == float(exp)
        else:
            k = b
            exp = Fraction(k - 2, 2 * k - 1) if y in (u, v) else Fraction(k - 2, 2 * (k - 1))
            assert w[e] == float(exp)
    # any 0 < theta <= smallest interior weight cuts exactly the bridge
    lo = min(Fraction(a - 2, 2 * a - 1), Fraction(b - 2, 2 * b - 1))
    if lo > 0:
        keep, kept = O.prune(O.TECTONIC, off, eu, ev, t, uni, lo.numerator, lo.denominator)
        assert kept == len(eu) - 1
        labels, nc = O.components(a + b, eu, ev, keep)
        assert nc == 2
        assert (labels[:a] == 0).all() and (labels[a:] == a).all()


# ----------------------------------------------------------- pruning


def _fraction_keep(measure, off, eu, ev, t, uni, theta):
    d = O.degrees(off)
    out = []
    for e in range(len(eu)):
        if measure == O.TECTONIC:
            sim = Fraction(int(t[e]), int(d[eu[e]] + d[ev[e]]))
        else:
            wedge = int(uni[e]) - int(t[e]) - 2
            sim = Fraction(int(t[e]) - wedge)
        out.append(1 if not (sim < theta) else 0)   # Algorithm 1 removes sim < delta
    return np.array(out, dtype=np.uint8)


def test_prune_matches_exact_rationals():
    rng = np.random.default_rng(1)
    for off, col in _rand_graphs(8, seed=21):
        eu, ev = O.edge_list(off, col)
        if len(eu) == 0:
            continue
        t, uni = O.edge_counts(off, col, eu, ev)
        d = O.degrees(off)
        for measure in (O.TECTONIC, O.TW):
            thetas = [Fraction(int(rng.integers(-40, 40)), int(rng.integers(1, 50))) for _ in range(4)]
            # thresholds exactly equal to an edge's similarity: that edge must survive
            e0 = int(rng.integers(0, len(eu)))
            if measure == O.TECTONIC:
                thetas.append(Fraction(int(t[e0]), int(d[eu[e0]] + d[ev[e0]])))
            else:
                thetas.append(Fraction(2 * int(t[e0]) + 2 - int(uni[e0])))
            for th in thetas:
                keep, kept = O.prune(measure, off, eu, ev, t, uni, th.numerator, th.denominator)
                ref = _fraction_keep(measure, off, eu, ev, t, uni, th)
                assert (keep == ref).all() and kept == int(ref.sum())
            assert keep[e0] == 1


def test_prune_large_numerators_exact():
    off, col = small.complete(6)
    eu, ev = O.edge_list(off, col)
    t, uni = O.edge_counts(off, col, eu, ev)
    # theta = 4/10 exactly scaled by a huge factor: equality must still keep every edge
    big = (1 << 59) - 1
    keep, kept = O.prune(O.TECTONIC, off, eu, ev, t, uni, 4 * big, 10 * big)
    assert kept == len(eu)
    keep, kept = O.prune(O.TECTONIC, off, eu, ev, t, uni, 4 * big + 1, 10 * big)
    assert kept == 0


def test_prop1_jaccard_is_reparametrised_tectonic():
    # Proposition 1: removing J(e) < dJ equals removing Tectonic(e) < dJ / (1 + dJ)
    for off, col in _rand_graphs(8, seed=31):
        eu, ev = O.edge_list(off, col)
        if len(eu) == 0:
            continue
        t, uni = O.edge_counts(off, col, eu, ev)
        d = O.degrees(off)
        for dj in (Fraction(0), Fraction(1, 10), Fraction(1, 3), Fraction(7, 9), Fraction(1)):
            jac_keep = np.array([
                0 if Fraction(int(t[e]), int(d[eu[e]] + d[ev[e]] - t[e])) < dj else 1
                for e in range(len(eu))], dtype=np.uint8)
            th = dj / (1 + dj)
            keep, _ = O.prune(O.TECTONIC, off, eu, ev, t, uni, th.numerator, th.denominator)
            assert (keep == jac_keep).all()


def test_jaccard_and_k3_prune_by_definition():
    # Jaccard from the neighbourhood sets (Sec. II) and K3 = t (Table 1), against Fraction
    for off, col in _rand_graphs(6, seed=41):
        eu, ev = O.edge_list(off, col)
        if len(eu) == 0:
            continue
        t, uni = O.edge_counts(off, col, eu, ev)
        nb = [set(col[off[v]:off[v + 1]].tolist()) for v in range(len(off) - 1)]
        jac = [Fraction(len(nb[a] & nb[b]), len(nb[a] | nb[b])) for a, b in zip(eu, ev)]
        w = O.jaccard_weights(t, uni)
        assert all(w[e] == float(jac[e]) for e in range(len(eu)))
        for p, q in ((0, 1), (1, 10), (1, 3), (2, 3), (1, 1), (-1, 2)):
            keep, kept = O.prune(O.JACCARD, off, eu, ev, t, uni, p, q)
            assert list(keep) == [1 if j >= Fraction(p, q) else 0 for j in jac] and kept == int(keep.sum())
        for p, q in ((0, 1), (1, 1), (3, 2), (2, 1), (7, 3), (100, 1)):
            keep, _ = O.prune(O.K3, off, eu, ev, t, uni, p, q)
            assert list(keep) == [1 if Fraction(int(x)) >= Fraction(p, q) else 0 for x in t]
        assert np.array_equal(O.k3_scores(t), t.astype(np.int64))


def test_prop1_as_two_oracle_prunes():
    # Proposition 1 exactly: Jaccard at p/q keeps what Tectonic at p/(p+q) keeps (p >= 0)
    for off, col in _rand_graphs(6, seed=43):
        eu, ev = O.edge_list(off, col)
        if len(eu) == 0:
            continue
        t, uni = O.edge_counts(off, col, eu, ev)
        for p, q in ((0, 1), (1, 10), (1, 3), (7, 9), (1, 1), (5, 2)):
            kj, _ = O.prune(O.JACCARD, off, eu, ev, t, uni, p, q)
            kt, _ = O.prune(O.TECTONIC, off, eu, ev, t, uni, p, p + q)
            assert np.array_equal(kj, kt)


def test_prune_rejects_nonpositive_q():
    off, col = small.complete(4)
    eu, ev = O.edge_list(off, col)
    t, uni = O.edge_counts(off, col, eu, ev)
    with pytest.raises(ValueError):
        O.prune(O.TECTONIC, off, eu, ev, t, uni, 1, 0)


# ----------------------------------------------------------- components


def test_components_against_scipy():
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    rng = np.random.default_rng(4)
    for off, col in _rand_graphs(10, seed=41):
        n = len(off) - 1
        eu, ev = O.edge_list(off, col)
        keep = (rng.random(len(eu)) < 0.4).astype(np.uint8)
        labels, nc = O.components(n, eu, ev, keep)
        s = keep.astype(bool)
        M = sp.coo_matrix((np.ones(int(s.sum())), (eu[s], ev[s])), shape=(n, n))
        nc_ref, lab = csgraph.connected_components(M, directed=False)
        assert nc == nc_ref
        # library labels are arbitrary ids: map each to its component's smallest vertex
        mins = np.full(nc_ref, n, dtype=np.int64)
        np.minimum.at(mins, lab, np.arange(n))
        assert (labels == mins[lab]).all()


def test_components_degenerate():
    labels, nc = O.components(5, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint8))
    assert nc == 5 and (labels == np.arange(5)).all()
    labels, nc = O.components(0, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint8))
    assert nc == 0 and labels.size == 0


def test_sweep_is_independent_passes_and_monotone():
    off, col, _ = sbm_csr([30, 30, 40], [[0.3, 0.05, 0.02], [0.05, 0.4, 0.03], [0.02, 0.03, 0.25]], seed=8)
    ps = list(range(1, 65))
    qs = [128] * 64
    labels, nc = O.sweep(off, col, O.TECTONIC, ps, qs)
    for i in (0, 17, 63):
        r = O.full_pass(off, col, O.TECTONIC, ps[i], qs[i])
        assert (labels[i] == r.labels).all() and nc[i] == r.ncomp
    # raising the threshold only removes edges: components can only split
    assert all(nc[i] <= nc[i + 1] for i in range(63))


# ----------------------------------------------------------- evaluation


def test_ari_worked_example():
    rows = {}
    for line in open(os.path.join(GOLDEN, "ari_worked_example.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, *vals = line.split()
        rows[k] = [int(v) for v in vals]
    assert O.ari(rows["a"], rows["b"]) == float(Fraction(rows["ari_num"][0], rows["ari_den"][0]))


def test_ari_properties_and_sklearn():
    rng = np.random.default_rng(0)
    a = rng.integers(0, 5, 200)
    assert O.ari(a, a) == 1.0
    assert O.ari(a, (a + 3) * 7) == 1.0          # relabelling does not matter
    assert O.ari(np.zeros(10), np.zeros(10)) == 1.0
    assert O.ari(np.arange(10), np.arange(10)) == 1.0
    assert O.ari(np.zeros(10), np.arange(10)) == 0.0
    skm = pytest.importorskip("sklearn.metrics")
    for _ in range(5):
        x = rng.integers(0, 6, 300)
        y = rng.integers(0, 4, 300)
        assert abs(O.ari(x, y) - skm.adjusted_rand_score(x, y)) < 1e-12


def test_modularity_double_sum():
    for off, col in _rand_graphs(5, seed=51):
        n = len(off) - 1
        if off[-1] == 0:
            continue
        A = dense_adjacency(off, col)
        d = A.sum(1)
        two_m = d.sum()
        lab = np.random.default_rng(n).integers(0, 3, n)
        q = 0.0
        for u in range(n):
            for v in range(n):
                if lab[u] == lab[v]:
                    q += A[u, v] - d[u] * d[v] / two_m
        assert abs(O.modularity(off, col, lab) - q / two_m) < 1e-12


def test_precision_recall_f1():
    truth = np.array([0, 0, 0, 1, 1, 1])
    assert O.precision_recall_f1(truth, truth) == (1.0, 1.0, 1.0)
    # one found community of everything: matched to a size-3 truth block, p=1/2, r=1
    p, r, f = O.precision_recall_f1(truth, np.zeros(6))
    assert (p, r) == (0.5, 1.0) and abs(f - 2 / 3) < 1e-15


def test_precision_recall_f1_hand_worked():
    """Sec. IV-A on a hand-worked case.  Truth blocks {0..3}, {4,5}, {6,7};
    found {0,1,2}, {3,4,5,6}, {7}.  Matches by Jaccard: {0,1,2} -> block 0
    (3/4; p 1, r 3/4), {3,4,5,6} -> block 1 (2/4 beats 1/7 and 1/5; p 1/2,
    r 1), {7} -> block 2 (1/2; p 1, r 1/2).  Size-weighted over 8 vertices:
    P = 6/8, R = 27/32, F1 = (3 * 6/7 + 4 * 2/3 + 1 * 2/3) / 8 = 31/42."""
    truth = np.array([0, 0, 0, 0, 1, 1, 2, 2])
    found = np.array([5, 5, 5, 1, 1, 1, 1, 9])
    p, r, f = O.precision_recall_f1(truth, found)
    assert p == 0.75 and r == 27 / 32 and abs(f - 31 / 42) < 1e-15
    # labels are names only: renaming either side changes nothing
    assert O.precision_recall_f1(truth + 7, 100 - found) == (p, r, f)


def test_precision_recall_f1_jaccard_tie():
    """A Jaccard tie between truth blocks of different sizes: found {0,1,2}
    meets block 0 = {0} in 1 (Jaccard 1/3) and block 1 = {1..5} in 2 (2/6 =
    1/3).  The lower block id wins (p 1/3, r 1); block 1 would give p 2/3,
    r 2/5.  Vertices 3, 4, 5 form a found community matched to block 1 (3/5;
    p 1, r 3/5)."""
    truth = np.array([0, 1, 1, 1, 1, 1])
    found = np.array([0, 0, 0, 1, 1, 1])
    p, r, f = O.precision_recall_f1(truth, found)
    assert abs(p - (3 * (1 / 3) + 3 * 1) / 6) < 1e-15
    assert abs(r - (3 * 1 + 3 * (3 / 5)) / 6) < 1e-15
    f_tie = 2 * (1 / 3) / (4 / 3)
    f_rest = 2 * (3 / 5) / (8 / 5)
    assert abs(f - (3 * f_tie + 3 * f_rest) / 6) < 1e-15


def test_features_shape_and_normalisation():
    off, col = small.two_cliques_bridge(6, 9)
    eu, ev = O.edge_list(off, col)
    t, _ = O.edge_counts(off, col, eu, ev)
    f = O.features(off, eu, ev, t)
    m, n = len(eu), len(off) - 1
    assert f.shape == (66,)
    assert abs(f[:64].sum() - 1.0) < 1e-15
    assert f[64] == math.log(2 * m / n) and f[65] == math.log(m)
    assert f[0] == 1 / m                       # the bridge has t = 0
    # by hand: K6 edges have t = 4, K9 edges t = 7; an edge at a bridge end
    # has one more degree.  K6: 10 edges at 4/10 -> bin 51, 5 at 4/11 -> 46;
    # K9: 28 edges at 7/16 -> bin 56, 8 at 7/17 -> 52; bridge: bin 0.
    expect = {0: 1, 46: 5, 51: 10, 52: 8, 56: 28}
    assert m == 52 and n == 15
    for b in range(64):
        assert f[b] == expect.get(b, 0) / m, b


# ----------------------------------------------------------- paper statistics


def test_table2_expectations_sbm():
    # Table 2: per-edge expectations in a two-block SBM, normalised by n.  At finite
    # n the exact means are (n-2)p1^2 + n q^2 (inside B1) and (n-1) q (p1 + p2)
    # (across); Table 2 is their n -> infinity limit.  Check sample means of the
    # oracle's counts against the exact values within 5 standard errors.
    n, p1, p2, q = 300, 0.12, 0.3, 0.06
    off, col, blk = sbm_csr([n, n], [[p1, q], [q, p2]], seed=12)
    eu, ev = O.edge_list(off, col)
    t, uni = O.edge_counts(off, col, eu, ev)
    d = O.degrees(off)
    s = d[eu] + d[ev]
    b1 = (blk[eu] == 0) & (blk[ev] == 0)
    ac = blk[eu] != blk[ev]
    cases = [
        (t[b1], (n - 2) * p1 ** 2 + n * q ** 2),
        (t[ac], (n - 1) * q * (p1 + p2)),
        (s[b1], 2 + 2 * (n - 2) * p1 + 2 * n * q),
        (s[ac], 2 + (n - 1) * (p1 + p2 + 2 * q)),
    ]
    for x, mu in cases:
        x = x.astype(np.float64)
        se = x.std(ddof=1) / math.sqrt(x.size)
        assert abs(x.mean() - mu) < 5 * se + 1e-9, (x.mean(), mu, se)


def test_theorem1_setting_tw_separates_tectonic_inverts():
    # The imbalanced SBM of Fig. 2 (n=50 per block, p1=0.1, p2=0.8, q=0.05): on
    # average, across-block edges score below both inside kinds under TW, while
    # under Tectonic they score above the sparse block B1 (the failure of Theorem 1).
    tw_in1, tw_ac, tec_in1, tec_ac = [], [], [], []
    for seed in range(20):
        off, col, blk = sbm_csr([50, 50], [[0.1, 0.05], [0.05, 0.8]], seed=100 + seed)
        eu, ev = O.edge_list(off, col)
        t, uni = O.edge_counts(off, col, eu, ev)
        tw = O.tw_scores(t, O.wedges(t, uni))
        tec = O.tectonic_weights(off, eu, ev, t)
        b1 = (blk[eu] == 0) & (blk[ev] == 0)
        ac = blk[eu] != blk[ev]
        tw_in1 += tw[b1].tolist(); tw_ac += tw[ac].tolist()
        tec_in1 += tec[b1].tolist(); tec_ac += tec[ac].tolist()
    assert np.mean(tw_in1) > np.mean(tw_ac)
    assert np.mean(tec_ac) > np.mean(tec_in1)


def test_check_csr_flags_bad_graphs():
    off, col = small.complete(4)
    assert O.check_csr(off, col) == 0
    bad = col.copy(); bad[0], bad[1] = bad[1], bad[0]
    assert O.check_csr(off, bad) == 3
    off2 = np.array([0, 1, 1], dtype=np.int64)
    assert O.check_csr(off2, np.array([0], dtype=np.int32)) == 4
    assert O.check_csr(off2, np.array([1], dtype=np.int32)) == 5
    assert O.check_csr(off2, np.array([7], dtype=np.int32)) == 2


def test_upper_pairs_matches_edge_list():
    off, col = small.two_cliques_bridge(5, 6)
    eu, ev = O.edge_list(off, col)
    u, v = upper_pairs(off, col)
    assert (eu == u).all() and (ev == v).all()


def test_k4_participation_closed_forms_and_brute_force():
    from itertools import combinations
    # K_n: every edge lies in C(n-2, 2) 4-cliques; a triangle-free graph has none
    for k in (4, 5, 9):
        off, col = small.complete(k)
        assert set(O.edge_k4(off, col).tolist()) == {(k - 2) * (k - 3) // 2}
    off, col = small.cycle(8)
    assert not O.edge_k4(off, col).any()
    off, col = small.two_cliques_bridge(5, 6)
    eu, ev = O.edge_list(off, col)
    k4 = O.edge_k4(off, col)
    assert k4[(eu == 0) & (ev == 1)][0] == 3 and k4[(eu == 5) & (ev == 6)][0] == 6
    # brute force over 4-subsets; sum of K4(e) = 6 * #4-cliques
    for off, col in _rand_graphs(5, seed=47):
        n = len(off) - 1
        adj = [set(col[off[v]:off[v + 1]].tolist()) for v in range(n)]
        eu, ev = O.edge_list(off, col)
        k4 = O.edge_k4(off, col)
        cliques = [c for c in combinations(range(n), 4)
                   if all(b in adj[a] for a, b in combinations(c, 2))]
        ref = {(a, b): 0 for a, b in zip(eu.tolist(), ev.tolist())}
        for c in cliques:
            for a, b in combinations(c, 2):
                ref[(a, b)] += 1
        assert [int(x) for x in k4] == [ref[(a, b)] for a, b in zip(eu.tolist(), ev.tolist())]
        assert int(k4.sum()) == 6 * len(cliques)
        keep, kept = O.prune(O.K4, off, eu, ev, None, None, 3, 2, k4)
        assert list(keep) == [1 if 2 * int(x) >= 3 else 0 for x in k4]


# ----------------------------------------------------------- forward (oriented) counts


def test_forward_counts_brute_force_and_dense_identities():
    # the oriented listing against set intersections, (A^2)_uv and trace(A^3) = 6T
    for off, col in _rand_graphs(12, seed=21):
        nb = _nbrs(off, col)
        eu, ev = O.edge_list(off, col)
        t = O.forward_counts(off, col, nthreads=2)
        for e, (u, v) in enumerate(zip(eu, ev)):
            assert t[e] == len(nb[u] & nb[v])
        A = dense_adjacency(off, col)
        A2 = A @ A
        assert (t.astype(np.int64) == A2[eu, ev]).all()
        assert 2 * int(t.sum()) == int(np.trace(A2 @ A))
        # with the merge's union: deg u + deg v - t (inclusion-exclusion)
        _, uni = O.edge_counts(off, col, eu, ev)
        assert np.array_equal(O.unions_from_counts(off, eu, ev, t), uni)


@pytest.mark.parametrize("graph,expect", [
    (small.complete(12), 10), (small.star(25), 0), (small.cycle(7), 0), (small.empty(6), None),
    (small.empty(1), None),
])
def test_forward_counts_closed_forms(graph, expect):
    off, col = graph
    t = O.forward_counts(off, col)
    if expect is None:
        assert t.size == 0
    else:
        assert (t == expect).all()


def test_forward_counts_two_cliques_bridge():
    # interior edges of K_a carry a - 2 triangles, the bridge none
    a, b = 7, 5
    off, col = small.two_cliques_bridge(a, b)
    eu, ev = O.edge_list(off, col)
    t = O.forward_counts(off, col)
    inside_a = (eu < a) & (ev < a)
    inside_b = (eu >= a) & (ev >= a)
    assert (t[inside_a] == a - 2).all() and (t[inside_b] == b - 2).all()
    assert (t[~inside_a & ~inside_b] == 0).all()


@pytest.mark.parametrize("which", ["gnp", "sbm", "rmat13", "rmat16", "rmat18"])
def test_forward_counts_equal_the_merges(which):
    # bit for bit against the per-edge merges of Sec. III-C, on graphs with
    # hubs, many degree ties and isolated vertices, and for any thread count
    from graphgen import planted_partition, rmat_csr
    if which == "gnp":
        off, col = small.gnp(1500, 0.03, np.random.default_rng(4))
    elif which == "sbm":
        off, col, _ = planted_partition(4, 500, 0.05, 0.002, seed=1)
    else:
        off, col = rmat_csr(int(which[4:]), 16, seed=2)
    t, _ = O.edge_counts(off, col, nthreads=O.threads_available())
    for th in (1, O.threads_available()):
        assert np.array_equal(O.forward_counts(off, col, nthreads=th), t)
