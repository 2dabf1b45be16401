"""Learned threshold picker: labelled data, training and inference.

Orchestration of library calls only (every computation is a kernel of
libtectonic.so): a batch of degree-corrected SBM graphs is built on the GPU,
`tec_features` gives the 66 inputs per graph, `tec_sweep` the components at
the 64 grid thresholds b/128, `tec_ari` their adjusted Rand index against the
planted blocks, `tec_ari_best` the best level b*; the network regresses b*/64
(`tec_picker_train`).  Inference: features -> `tec_picker_forward` ->
`tec_picker_thresholds` -> `tec_prune_components_batch`.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import tectonic as T

K = 64
DEN = 128
GRID_P = list(range(1, K + 1))
GRID_Q = [DEN] * K


def label_batch(seeds, n_lo=1000, n_hi=100000, measure=T.TECTONIC):
    """Features, best level (0-based), best ARI and the full ARI table (K x G)
    for the DC-SBM graphs of `seeds` (CUDA tensors)."""
    from graphgen.gpu import dcsbm_batch_gpu
    off, col, seg, truth, specs = dcsbm_batch_gpu(seeds, n_lo, n_hi)
    g = T.Graph(off, col)
    feats = g.features(seg)
    labels, _ = g.sweep(measure, GRID_P, GRID_Q, seg_off=seg, count=False)
    ari = g.ari(labels, truth, seg)
    best, best_ari = T.ari_best(ari)
    g.free()
    return {"feats": feats, "best": best, "best_ari": best_ari, "ari": ari, "n": [s.n for s in specs]}


def build_dataset(seeds, n_lo=1000, n_hi=100000, batch=256, measure=T.TECTONIC):
    import torch
    parts = [label_batch(list(seeds[i:i + batch]), n_lo, n_hi, measure) for i in range(0, len(seeds), batch)]
    out = {k: torch.cat([p[k] for p in parts], dim=1 if k == "ari" else 0) for k in ("feats", "best", "best_ari", "ari")}
    out["target"] = (out["best"].to(torch.float32) + 1.0) / K
    return out


DATASET_FIELDS = ("feats", "best", "best_ari", "ari", "target")


def dataset_key(seeds, n_lo, n_hi, measure=T.TECTONIC) -> str:
    """Identity of a labelled dataset: its seeds, size range, measure and grid
    (the labels are exact, so the kernels' version does not enter)."""
    desc = json.dumps({"seeds": [int(x) for x in seeds], "n": [int(n_lo), int(n_hi)], "measure": int(measure),
                       "grid": [K, DEN]})
    return hashlib.sha256(desc.encode()).hexdigest()[:16]


def _dataset_digest(arrays) -> str:
    h = hashlib.sha256()
    for name in DATASET_FIELDS:
        h.update(name.encode())
        h.update(np.ascontiguousarray(arrays[name]).tobytes())
    return h.hexdigest()


def save_dataset(dataset, path, key: str):
    """Writes a dataset (tensors on any device) with its key and a checksum."""
    arrays = {name: dataset[name].detach().cpu().numpy() for name in DATASET_FIELDS}
    np.savez(path, key=key, sha256=_dataset_digest(arrays), **arrays)


def load_dataset(path, key: str, device="cuda"):
    """The dataset saved at `path` as torch tensors on `device`, or None when
    the file is missing or was saved under another key.  ValueError when the
    arrays fail their checksum."""
    import torch
    if not os.path.exists(path):
        return None
    d = np.load(path, allow_pickle=False)
    if str(d["key"]) != key:
        return None
    arrays = {name: d[name] for name in DATASET_FIELDS}
    if _dataset_digest(arrays) != str(d["sha256"]):
        raise ValueError(f"dataset {path} fails its checksum")
    return {name: torch.from_numpy(arrays[name]).to(device) for name in DATASET_FIELDS}


def cached_dataset(seeds, n_lo=1000, n_hi=100000, cache_dir=None, batch=256, measure=T.TECTONIC,
                   device="cuda"):
    """build_dataset, kept under cache_dir (when given) as dataset_<key>.npz
    and reused by later runs with the same seeds, size range and measure."""
    if not cache_dir:
        return build_dataset(seeds, n_lo, n_hi, batch, measure)
    key = dataset_key(seeds, n_lo, n_hi, measure)
    path = os.path.join(cache_dir, f"dataset_{key}.npz")
    ds = load_dataset(path, key, device)
    if ds is None:
        ds = build_dataset(seeds, n_lo, n_hi, batch, measure)
        os.makedirs(cache_dir, exist_ok=True)
        save_dataset(ds, path, key)
    return ds


def fixed_level(dataset) -> int:
    """The single grid level of highest mean ARI over a dataset (0-based):
    the method with one global threshold, as in the paper."""
    return int(dataset["ari"].mean(dim=1).argmax().item())


def init_params(seed: int = 0):
    """Kaiming-uniform weights (bound sqrt(6 / fan_in)), zero biases, float32."""
    rng = np.random.default_rng(seed)
    IN, H = 66, 128
    parts = [rng.uniform(-np.sqrt(6 / IN), np.sqrt(6 / IN), H * IN), np.zeros(H),
             rng.uniform(-np.sqrt(6 / H), np.sqrt(6 / H), H * H), np.zeros(H),
             rng.uniform(-np.sqrt(6 / H), np.sqrt(6 / H), H), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def ari_loss_rows(dataset):
    """N x 64 float32: the ARI each graph loses at each grid level against its
    best level (the table the soft-level loss weighs)."""
    return (dataset["best_ari"][None, :] - dataset["ari"]).T.contiguous().float()


def train(dataset, epochs=300, batch=256, lr=1e-3, seed=0):
    picker = T.Picker(init_params(seed))
    losses = picker.train(dataset["feats"], dataset["target"], epochs, batch, lr, seed)
    return picker, losses


def predict_levels(picker, feats, bf16=False):
    """0-based grid level per graph."""
    p, _ = T.picker_thresholds(picker.forward(feats, bf16))
    return p - 1


def evaluate(picker, dataset, bf16=False, baseline_level=None):
    """ARI lost against the best grid threshold, per graph, for the picker and
    (optionally) one fixed level."""
    import torch
    lv = predict_levels(picker, dataset["feats"], bf16).long()
    cols = torch.arange(lv.numel(), device=lv.device)
    got = dataset["ari"][lv, cols]
    loss = (dataset["best_ari"] - got).cpu().numpy()
    out = {"mean_dARI": float(loss.mean()), "p95_dARI": float(np.percentile(loss, 95)), "max_dARI": float(loss.max()),
           "mean_ARI": float(got.mean().item()), "mean_best_ARI": float(dataset["best_ari"].mean().item())}
    if baseline_level is not None:
        fixed = dataset["ari"][baseline_level]
        out["fixed_level"] = int(baseline_level) + 1
        out["fixed_mean_ARI"] = float(fixed.mean().item())
        out["fixed_mean_dARI"] = float((dataset["best_ari"] - fixed).mean().item())
    return out


CHECKPOINT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "picker_weights.tecp")


def save(picker, path, meta=None):
    """Writes a checkpoint file in the library's format (tec_picker_file_write):
    parameters, Adam moments, step and the training record as JSON text."""
    params, m, v, step = picker.get_params(with_adam=True)
    T.picker_file_write(path, params, m, v, step, json.dumps(meta or {}))


def read_checkpoint(path):
    """The arrays of a checkpoint file, checked by the library (host only;
    TectonicError TEC_EIO when the file is damaged or not a checkpoint)."""
    params, m, v, step, meta = T.picker_file_read(path)
    return params, m, v, step, json.loads(meta or "{}")


def load(path):
    """A device picker holding the file's state (tec_picker_load) and its record."""
    meta = read_checkpoint(path)[4]
    return T.Picker.load(path), meta
