"""Learned threshold picker: kernels against the float64 oracle, per-graph
thresholds against the oracle's passes, and what training gains."""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tec(cuda_device):
    import paper_2412_12382_gb300 as pkg
    from paper_2412_12382_gb300 import build
    build.build()
    pkg.load_library()
    return pkg


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 66)).astype(np.float32)
    X[:, 64:] = rng.uniform(2, 12, size=(n, 2))
    return X, rng.uniform(0, 1, n).astype(np.float32)


def test_forward_and_gradient_against_oracle(tec):
    import torch
    from paper_2412_12382_gb300.tectonic import Picker
    X, t = _data(200, 1)
    theta = M.init(4).astype(np.float32)
    theta[-1] = 0.3
    pk = Picker(theta)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    y = pk.forward(Xd).cpu().numpy()
    yo, _ = M.forward(theta.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(y, yo, rtol=1e-4, atol=1e-5)
    loss, g = pk.loss_grad(Xd, td)
    lo, go = M.loss_and_grad(theta.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    g = g.cpu().numpy()
    assert abs(loss - lo) <= 1e-4 * abs(lo)
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
    big = np.abs(go) > 1e-3 * np.abs(go).max()
    np.testing.assert_allclose(g[big], go[big], rtol=1e-3)
    # bf16 inference: bf16 weights and activations, each input as two bf16
    # terms; the output stays within a few bf16 roundings of float32
    yb = pk.forward(Xd, bf16=True).cpu().numpy()
    assert np.max(np.abs(yb - y)) <= 2e-2 * (np.abs(y).max() + 1)
    pk.free()


def test_bf16_picks_the_float32_level_on_held_out_graphs(tec):
    """The shipped picker's bfloat16 inference picks the same grid level as
    its float32 inference on at least 99% of the 500 held-out DC-SBM graphs
    (seeds 20000-20499, n in [1e3, 1e5])."""
    from paper_2412_12382_gb300 import picker as P
    held = P.build_dataset(list(range(20000, 20500)), 1000, 100000)
    pk, _ = P.load(P.CHECKPOINT)
    l32 = P.predict_levels(pk, held["feats"], bf16=False)
    l16 = P.predict_levels(pk, held["feats"], bf16=True)
    same = float((l32 == l16).float().mean().item())
    print("bf16 same level on held-out graphs:", same)
    assert same >= 0.99
    pk.free()


def test_soft_level_loss_and_gradient_against_oracle(tec):
    import torch
    from paper_2412_12382_gb300.tectonic import Picker
    X, t = _data(150, 9)
    L = np.random.default_rng(10).uniform(0, 0.3, (150, 64)).astype(np.float32)
    theta = M.init(11).astype(np.float32)
    theta[-1 - 128:-1] *= 0.02           # small w3: outputs near b3, levels inside the grid
    theta[-1] = 0.35
    pk = Picker(theta)
    y0, _ = M.forward(theta.astype(np.float64), X.astype(np.float64))
    assert ((64 * y0 > 3) & (64 * y0 < 62)).mean() > 0.9
    Xd, td, Ld = (torch.from_numpy(a).cuda() for a in (X, t, L))
    for sigma, mix in ((1.5, 0.3), (0.8, 0.0), (3.0, 1.0)):
        loss, g = pk.soft_loss_grad(Xd, td, Ld, sigma, mix)
        lo, go = M.mixed_loss_and_grad(theta.astype(np.float64), X.astype(np.float64), t.astype(np.float64),
                                       L.astype(np.float64), sigma, mix)
        g = g.cpu().numpy()
        assert abs(loss - lo) <= 1e-4 * abs(lo) + 1e-7
        assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
    pk.free()


def test_adam_step_against_oracle(tec):
    import torch
    from paper_2412_12382_gb300.tectonic import Picker
    X, t = _data(64, 2)
    theta = M.init(5).astype(np.float32)
    pk = Picker(theta)
    m = np.zeros(M.NPARAM)
    v = np.zeros(M.NPARAM)
    th = theta.astype(np.float64)
    for step in range(1, 4):
        _, g = pk.loss_grad(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda())
        gh = g.cpu().numpy().astype(np.float64)
        pk.adam_step(g, lr=1e-2)
        th, m, v = M.adam(th, gh, m, v, step, lr=1e-2)
        np.testing.assert_allclose(pk.get_params(), th, rtol=1e-5, atol=1e-6)
    pk.free()


def test_training_fits_and_checkpoint_round_trip(tec, tmp_path):
    import torch
    from paper_2412_12382_gb300 import picker as P
    from paper_2412_12382_gb300.tectonic import Picker
    rng = np.random.default_rng(3)
    X = rng.uniform(0, 1, (1000, 66)).astype(np.float32)
    t = (0.3 * X[:, 0] + 0.5 * X[:, 1] * X[:, 2]).astype(np.float32)
    pk = Picker(P.init_params(1))
    losses = pk.train(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda(), epochs=60, batch=128, lr=2e-3, seed=7)
    assert losses[-1] < 0.05 * losses[0]
    path = str(tmp_path / "pk.tecp")
    P.save(pk, path, {"note": "test"})
    pk2, meta = P.load(path)
    Xd = torch.from_numpy(X[:50]).cuda()
    assert torch.equal(pk.forward(Xd), pk2.forward(Xd)) and meta["note"] == "test"
    # the library's own save of the loaded picker reproduces the file byte for byte
    pk2.save(str(tmp_path / "again.tecp"), open(path, "rb").read()[36:36 + len('{"note": "test"}')].decode())
    assert open(path, "rb").read() == open(str(tmp_path / "again.tecp"), "rb").read()
    # training resumes from the loaded Adam state exactly as from the original
    pk.train(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda(), epochs=2, batch=128, lr=2e-3, seed=9)
    pk2.train(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda(), epochs=2, batch=128, lr=2e-3, seed=9)
    assert np.array_equal(pk.get_params(), pk2.get_params())
    pk.free()
    pk2.free()


def test_per_graph_thresholds_match_oracle(tec):
    import torch
    from graphgen.batch import disjoint_union
    from graphgen.dcsbm import dcsbm_csr
    graphs = [dcsbm_csr(s, 1000, 3000)[:2] for s in (20000, 20001, 20002)]
    off, col, seg = disjoint_union(graphs)
    g = tec.Graph(torch.from_numpy(off).cuda(), torch.from_numpy(col).cuda())
    ps, qs = [3, 9, 20], [128, 128, 128]
    lab, nc = g.prune_components_batch(tec.TECTONIC, torch.tensor(ps).cuda(), torch.tensor(qs).cuda(),
                                       torch.from_numpy(seg).cuda())
    lab = lab.cpu().numpy()
    for i, (go, gc) in enumerate(graphs):
        r = O.full_pass(go, gc, O.TECTONIC, ps[i], qs[i])
        assert nc[i] == r.ncomp and np.array_equal(lab[seg[i]:seg[i + 1]], r.labels)
    g.free()


def test_picker_gains_over_one_fixed_threshold(tec):
    # trained on 768 DC-SBM graphs (seeds 10000+), judged on 128 held-out
    # graphs (seeds 20000+) by the ARI lost against each graph's best grid
    # threshold; the method without a picker uses one global threshold (the
    # grid level of best mean training ARI)
    from paper_2412_12382_gb300 import picker as P
    train = P.build_dataset(list(range(10000, 10768)), 1000, 4000)
    held = P.build_dataset(list(range(20000, 20128)), 1000, 4000)
    pk, losses = P.train(train, epochs=300, batch=128, lr=1e-3, seed=0)
    res = P.evaluate(pk, held, baseline_level=P.fixed_level(train))
    print("picker evaluation:", res)
    assert losses[-1] < losses[0]
    assert res["mean_dARI"] < res["fixed_mean_dARI"]
    pk.free()


def test_pick_threshold_equals_features_forward_thresholds(tec):
    """The one-call picker entry point gives exactly the grid thresholds of
    features -> network -> thresholds, per graph of a batch, in float32 and
    bfloat16 inference, and for a single graph without a segment table."""
    import torch
    from graphgen.dcsbm import dcsbm_csr
    from graphgen.batch import disjoint_union
    from paper_2412_12382_gb300 import tectonic as T
    from paper_2412_12382_gb300.tectonic import Picker
    graphs = [dcsbm_csr(s, 300, 3000)[:2] for s in range(30500, 30512)]
    off, col, seg = disjoint_union(graphs)
    g = tec.Graph(torch.from_numpy(off).cuda(), torch.from_numpy(col).cuda())
    segd = torch.from_numpy(seg).cuda()
    theta = M.init(7).astype(np.float32)
    theta[-1] = 0.2
    pk = Picker(theta)
    for bf16 in (False, True):
        p, q = g.pick_threshold(pk, segd, bf16=bf16)
        pr, qr = T.picker_thresholds(pk.forward(g.features(segd), bf16=bf16))
        assert torch.equal(p, pr) and torch.equal(q, qr)
        assert int(p.min()) >= 1 and int(p.max()) <= 64 and bool((q == 128).all())
    g.free()
    g1 = tec.Graph(torch.from_numpy(np.asarray(graphs[0][0])).cuda(), torch.from_numpy(np.asarray(graphs[0][1])).cuda())
    p1, q1 = g1.pick_threshold(pk)
    pr1, qr1 = T.picker_thresholds(pk.forward(g1.features()))
    assert p1.shape == (1,) and torch.equal(p1, pr1) and torch.equal(q1, qr1)
    g1.free()
    pk.free()


def test_c_client_loads_the_shipped_picker_and_picks(tec, tmp_path):
    """A C program linked only against the library (and the CUDA runtime for
    its two output buffers) loads the shipped checkpoint, picks the threshold
    of a graph in float32 and bfloat16, prunes and labels at it, and writes
    the picker back byte for byte; its thresholds equal the Python binding's."""
    import os
    import shutil
    import subprocess
    import torch
    from graphgen.dcsbm import dcsbm_csr
    from paper_2412_12382_gb300 import build as libbuild
    from paper_2412_12382_gb300 import picker as P
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    libdir = os.path.dirname(libbuild.library_path())
    exe = str(tmp_path / "picker_client")
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(root, "include"),
                        "-I", os.path.join(cuda, "include"), os.path.join(root, "tests", "abi_c", "picker_client.c"),
                        "-o", exe, "-L", libdir, "-ltectonic", "-L", os.path.join(cuda, "lib64"), "-lcudart",
                        f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    off, col = dcsbm_csr(20007, 1000, 100000)[:2]
    gpath = str(tmp_path / "graph.bin")
    with open(gpath, "wb") as f:
        f.write(np.array([len(off) - 1, len(col)], dtype=np.int64).tobytes())
        f.write(np.asarray(off, dtype=np.int64).tobytes())
        f.write(np.asarray(col, dtype=np.int32).tobytes())
    out = str(tmp_path / "copy.tecp")
    r = subprocess.run([exe, P.CHECKPOINT, gpath, out], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    p32, q32, p16, q16, kept, ncomp = (int(x) for x in r.stdout.split())
    assert open(out, "rb").read() == open(P.CHECKPOINT, "rb").read()
    pk, _ = P.load(P.CHECKPOINT)
    g = tec.Graph(torch.from_numpy(np.asarray(off, dtype=np.int64)).cuda(), torch.from_numpy(np.asarray(col)).cuda())
    for bf16, (pc, qc) in ((False, (p32, q32)), (True, (p16, q16))):
        p, q = g.pick_threshold(pk, bf16=bf16)
        assert (int(p[0]), int(q[0])) == (pc, qc)
    ref = O.full_pass(off, col, O.TECTONIC, p32, q32)
    assert ncomp == ref.ncomp and kept == int(ref.keep.sum())
    g.free()
    pk.free()
