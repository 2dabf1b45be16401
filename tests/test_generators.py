"""Input generators (CPU): they produce simple graphs, deterministically."""
import numpy as np

import oracle as O
from graphgen import feistel, planted_partition, rmat_csr
from graphgen.batch import disjoint_union
from graphgen.dcsbm import dcsbm_csr, dcsbm_spec, mulhi
from graphgen.prng import mix64, mix64_int


def test_mix64_matches_scalar_and_reference_value():
    xs = [0, 1, 12345, (1 << 64) - 1]
    assert [int(v) for v in mix64(np.array(xs, dtype=np.uint64))] == [mix64_int(x) for x in xs]
    # SplitMix64 seeded with 0: the first output (Vigna's reference generator)
    assert mix64_int(0) == 0xE220A8397B1DCDAF


def test_feistel_is_a_bijection():
    for scale in (2, 5, 10, 13):
        x = np.arange(1 << scale, dtype=np.uint64)
        y = feistel(x, scale, seed=9)
        assert np.array_equal(np.sort(y), x)


def test_generated_graphs_are_simple_and_deterministic():
    for off, col in (rmat_csr(10, 8, seed=1), planted_partition(3, 60, 0.2, 0.01, seed=2)[:2],
                     dcsbm_csr(1000, 1000, 3000)[:2]):
        assert O.check_csr(off, col) == 0
    a = dcsbm_csr(1234, 1000, 3000)
    b = dcsbm_csr(1234, 1000, 3000)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_dcsbm_spec_ranges():
    for s in range(10000, 10040):
        sp = dcsbm_spec(s, 1000, 100000)
        assert 1000 <= sp.n <= 100000 and 2 <= sp.k <= 64 and 0.05 <= sp.mu < 0.5
        assert sp.block.min() >= 0 and sp.block.max() < sp.k
        assert sp.cum[-1] == sp.weight.sum() and sp.bstart[-1] == sp.cum[-1]


def test_mulhi_exact():
    rng = np.random.default_rng(1)
    a = rng.integers(0, 1 << 62, 2000, dtype=np.uint64) * np.uint64(4) + np.uint64(3)
    b = rng.integers(0, 1 << 45, 2000, dtype=np.uint64)
    got = mulhi(a, b)
    assert all(int(got[i]) == (int(a[i]) * int(b[i])) >> 64 for i in range(2000))


def test_disjoint_union_offsets():
    g1 = planted_partition(2, 10, 0.5, 0.1, seed=1)[:2]
    g2 = rmat_csr(4, 4, seed=3)
    off, col, seg = disjoint_union([g1, g2])
    assert O.check_csr(off, col) == 0
    assert seg.tolist() == [0, 20, 36]
    assert np.array_equal(off[20:] - off[20], g2[0]) and np.array_equal(col[off[20]:] - 20, g2[1])
