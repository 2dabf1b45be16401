"""Picker checkpoints and cached training sets on the host: the shipped
weights pass their checksum and carry the training record; a file whose
parameters, moments or size were changed after saving is refused before
anything reaches a device; a cached dataset round-trips, is keyed by its
seeds and size range, and fails loudly when altered."""
import os

import numpy as np
import pytest

from paper_2412_12382_gb300 import picker as P
from paper_2412_12382_gb300 import tectonic as T

SHIPPED = os.path.join(os.path.dirname(P.__file__), "picker_weights.tecp")
HEADER = 36


def test_shipped_weights_verify():
    params, m, v, step, meta = P.read_checkpoint(SHIPPED)
    assert params.dtype == np.float32 and params.shape == (T.PICKER_PARAMS,)
    assert np.isfinite(params).all() and step > 0
    assert isinstance(meta, dict) and "eval" in meta


def _meta_len(raw):
    return int.from_bytes(raw[32:36], "little")


def _refused(path, what):
    with pytest.raises(T.TectonicError) as e:
        P.read_checkpoint(path)
    assert e.value.status == 8 and what in str(e.value)


@pytest.mark.parametrize("field", [0, 1, 2])
def test_tampered_arrays_are_refused(tmp_path, field):
    # one bit of one entry of the parameters, the first or the second moments
    raw = bytearray(open(SHIPPED, "rb").read())
    at = HEADER + _meta_len(raw) + 4 * (field * T.PICKER_PARAMS + 12345)
    raw[at] ^= 1
    path = str(tmp_path / "bad.tecp")
    open(path, "wb").write(raw)
    _refused(path, "checksum")


def test_wrong_size_shape_and_magic_are_refused(tmp_path):
    raw = open(SHIPPED, "rb").read()
    cases = {"short": raw[:-4], "magic": b"XECPICK1" + raw[8:],
             "shape": raw[:20] + (T.PICKER_PARAMS - 1).to_bytes(4, "little") + raw[24:],
             "version": raw[:8] + (2).to_bytes(4, "little") + raw[12:]}
    expect = {"short": "size", "magic": "not a picker checkpoint", "shape": "shape", "version": "version"}
    for name, data in cases.items():
        path = str(tmp_path / f"{name}.tecp")
        open(path, "wb").write(data)
        _refused(path, expect[name])
    _refused(str(tmp_path / "missing.tecp"), "cannot open")


def test_round_trip_of_a_new_checkpoint(tmp_path):
    rng = np.random.default_rng(0)
    params = rng.standard_normal(T.PICKER_PARAMS).astype(np.float32)
    m = rng.standard_normal(T.PICKER_PARAMS).astype(np.float32)
    v = rng.uniform(0, 1, T.PICKER_PARAMS).astype(np.float32)

    class FakePicker:            # the host side of save() only reads get_params
        def get_params(self, with_adam=False):
            return params, m, v, 17

    path = str(tmp_path / "new.tecp")
    P.save(FakePicker(), path, {"epochs": 3})
    p2, m2, v2, step, meta = P.read_checkpoint(path)
    assert np.array_equal(p2, params) and np.array_equal(m2, m) and np.array_equal(v2, v)
    assert step == 17 and meta == {"epochs": 3}


def test_file_layout_is_the_documented_one(tmp_path):
    """The bytes follow the layout of the header: magic, version, shape,
    step, meta, three little-endian float32 arrays, FNV-1a 64 of the rest
    (computed here from its published definition)."""
    params = np.arange(T.PICKER_PARAMS, dtype=np.float32) / 7
    path = str(tmp_path / "layout.tecp")
    T.picker_file_write(path, params, None, None, -5, "ab")
    raw = open(path, "rb").read()
    assert raw[:8] == b"TECPICK1"
    assert [int.from_bytes(raw[i:i + 4], "little") for i in (8, 12, 16, 20)] == [1, 66, 128, T.PICKER_PARAMS]
    assert int.from_bytes(raw[24:32], "little", signed=True) == -5
    assert _meta_len(raw) == 2 and raw[36:38] == b"ab"
    body = np.frombuffer(raw[38:38 + 12 * T.PICKER_PARAMS], dtype="<f4")
    assert np.array_equal(body[:T.PICKER_PARAMS], params) and not body[T.PICKER_PARAMS:].any()
    h = 0xCBF29CE484222325
    for b in raw[:-8]:
        h = ((h ^ b) * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    assert int.from_bytes(raw[-8:], "little") == h and len(raw) == 38 + 12 * T.PICKER_PARAMS + 8


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
