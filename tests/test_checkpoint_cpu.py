"""Picker checkpoints and cached training sets on the host: the shipped
weights pass their checksum and carry the training record; a file whose
parameters, moments or size were changed after saving is refused before
anything reaches a device; a cached dataset round-trips, is keyed by its
seeds and size range, and fails loudly when altered."""
import json
import os

import numpy as np
import pytest

from paper_2412_12382_gb300 import picker as P
from paper_2412_12382_gb300 import tectonic as T

SHIPPED = os.path.join(os.path.dirname(P.__file__), "picker_weights.npz")


def test_shipped_weights_verify():
    params, m, v, step, meta = P.read_checkpoint(SHIPPED)
    assert params.dtype == np.float32 and params.shape == (T.PICKER_PARAMS,)
    assert np.isfinite(params).all() and step > 0
    assert isinstance(meta, dict)


def _rewrite(src, dst, **changes):
    d = dict(np.load(src, allow_pickle=False))
    d.update(changes)
    np.savez(dst, **d)


@pytest.mark.parametrize("field", ["params", "adam_m", "adam_v"])
def test_tampered_arrays_are_refused(tmp_path, field):
    d = np.load(SHIPPED, allow_pickle=False)
    bad = d[field].copy()
    bad[12345] = np.nextafter(bad[12345], np.float32(np.inf))    # one ulp in one entry
    path = str(tmp_path / "bad.npz")
    _rewrite(SHIPPED, path, **{field: bad})
    with pytest.raises(ValueError, match="checksum"):
        P.read_checkpoint(path)


def test_wrong_size_is_refused(tmp_path):
    d = np.load(SHIPPED, allow_pickle=False)
    path = str(tmp_path / "short.npz")
    _rewrite(SHIPPED, path, params=d["params"][:-1])
    with pytest.raises(ValueError, match="parameters"):
        P.read_checkpoint(path)


def test_round_trip_of_a_new_checkpoint(tmp_path):
    rng = np.random.default_rng(0)
    params = rng.standard_normal(T.PICKER_PARAMS).astype(np.float32)
    m = rng.standard_normal(T.PICKER_PARAMS).astype(np.float32)
    v = rng.uniform(0, 1, T.PICKER_PARAMS).astype(np.float32)

    class FakePicker:            # the host side of save() only reads get_params
        def get_params(self, with_adam=False):
            return params, m, v, 17

    path = str(tmp_path / "new.npz")
    P.save(FakePicker(), path, {"epochs": 3})
    p2, m2, v2, step, meta = P.read_checkpoint(path)
    assert np.array_equal(p2, params) and np.array_equal(m2, m) and np.array_equal(v2, v)
    assert step == 17 and meta == {"epochs": 3}
    assert json.loads(str(np.load(path)["meta"])) == {"epochs": 3}


def _fake_dataset(torch, seed=0, graphs=7):
    g = torch.Generator().manual_seed(seed)
    best = torch.randint(0, 64, (graphs,), generator=g)
    return {"feats": torch.rand((graphs, 66), generator=g), "best": best,
            "best_ari": torch.rand((graphs,), generator=g, dtype=torch.float64),
            "ari": torch.rand((64, graphs), generator=g, dtype=torch.float64),
            "target": (best.to(torch.float32) + 1.0) / 64}


def test_dataset_cache_round_trip_key_and_checksum(tmp_path):
    torch = pytest.importorskip("torch")
    ds = _fake_dataset(torch)
    key = P.dataset_key(range(10000, 10007), 1000, 100000)
    assert key != P.dataset_key(range(10000, 10008), 1000, 100000)       # other seeds, other key
    assert key != P.dataset_key(range(10000, 10007), 1000, 200000)
    path = str(tmp_path / "ds.npz")
    P.save_dataset(ds, path, key)
    back = P.load_dataset(path, key, device="cpu")
    for name in P.DATASET_FIELDS:
        assert torch.equal(back[name], ds[name]), name
    assert P.load_dataset(path, "another key", device="cpu") is None
    assert P.load_dataset(str(tmp_path / "missing.npz"), key, device="cpu") is None
    d = dict(np.load(path, allow_pickle=False))
    d["best_ari"] = d["best_ari"].copy()
    d["best_ari"][3] += 1e-12
    np.savez(path, **d)
    with pytest.raises(ValueError, match="checksum"):
        P.load_dataset(path, key, device="cpu")


def test_cached_dataset_builds_once(tmp_path, monkeypatch):
    torch = pytest.importorskip("torch")
    calls = []

    def fake_build(seeds, n_lo, n_hi, batch, measure):
        calls.append(list(seeds))
        return _fake_dataset(torch, seed=len(calls))

    monkeypatch.setattr(P, "build_dataset", fake_build)
    a = P.cached_dataset([1, 2, 3], cache_dir=str(tmp_path), device="cpu")
    b = P.cached_dataset([1, 2, 3], cache_dir=str(tmp_path), device="cpu")
    assert len(calls) == 1 and torch.equal(a["feats"], b["feats"])
    P.cached_dataset([1, 2, 4], cache_dir=str(tmp_path), device="cpu")
    assert len(calls) == 2
