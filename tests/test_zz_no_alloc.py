"""The allocation-free components entry point against the graph-owned one.

tec_components_noalloc serves callers that cannot allocate device memory;
its labels and component counts must equal those of tec_prune +
tec_components exactly, on two calls in a row (the shared scratch array keeps
the previous call's contents and must be re-initialised every time).  This
file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from graphgen import planted_partition, rmat_csr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tec(cuda_device):
    import paper_2412_12382_gb300 as pkg
    from paper_2412_12382_gb300 import build
    build.build()
    pkg.load_library()
    return pkg


def _graph(tec, off, col):
    import torch
    return tec.Graph(torch.from_numpy(np.asarray(off, dtype=np.int64)).cuda(),
                     torch.from_numpy(np.asarray(col, dtype=np.int32)).cuda())


@pytest.mark.parametrize("which", ["sbm", "rmat"])
def test_noalloc_components_match_graph_components(tec, which):
    from paper_2412_12382_gb300.tectonic import components_noalloc
    if which == "sbm":
        off, col, _ = planted_partition(4, 500, 0.05, 0.002, seed=1)
        thresholds = [(tec.TECTONIC, 3, 50), (tec.TW, -30, 1)]
    else:
        off, col = rmat_csr(13, 16, seed=2)
        thresholds = [(tec.TECTONIC, 1, 10), (tec.TECTONIC, 1, 40)]
    n = len(off) - 1
    g = _graph(tec, off, col)
    u, v = g.edge_list()
    for measure, p, q in thresholds:
        keep, _ = g.prune(measure, p, q, mask=True)
        ref, ref_nc = g.components()
        ref = ref.cpu().numpy()
        for _ in range(2):                       # two calls in a row share the scratch array
            lab, nc = components_noalloc(n, u, v, keep)
            assert nc == ref_nc
            assert np.array_equal(lab.cpu().numpy(), ref)
    # without a mask every edge counts: the whole graph's components
    keep0, _ = g.prune(tec.TECTONIC, 0, 1, mask=True)
    ref0, nc0 = g.components()
    lab, nc = components_noalloc(n, u, v, None)
    assert nc == nc0 and np.array_equal(lab.cpu().numpy(), ref0.cpu().numpy())
    g.free()


def test_noalloc_rejects_oversized_input(tec):
    import torch
    from paper_2412_12382_gb300.tectonic import NOALLOC_MAX_VERTICES, components_noalloc
    e = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(tec.TectonicError) as err:
        components_noalloc(NOALLOC_MAX_VERTICES + 1, e, e, labels=torch.empty(1, dtype=torch.int32, device="cuda"))
    assert err.value.status == 1


def test_noalloc_rejects_endpoints_outside_the_vertex_range(tec):
    """An endpoint equal to n or negative is reported as TEC_EINVAL (the hook
    checks both ends before it touches the scratch), and the next valid call
    still returns the right labels."""
    import torch
    from paper_2412_12382_gb300.tectonic import components_noalloc
    n = 6
    for bad_u, bad_v in (([0, 1], [n, 2]), ([-1, 3], [0, 4])):
        u = torch.tensor(bad_u, dtype=torch.int32, device="cuda")
        v = torch.tensor(bad_v, dtype=torch.int32, device="cuda")
        with pytest.raises(tec.TectonicError) as err:
            components_noalloc(n, u, v)
        assert err.value.status == 1
    u = torch.tensor([0, 1, 4], dtype=torch.int32, device="cuda")
    v = torch.tensor([2, 2, 5], dtype=torch.int32, device="cuda")
    lab, nc = components_noalloc(n, u, v)
    assert nc == 3
    assert lab.cpu().tolist() == [0, 0, 0, 3, 4, 4]
