"""The setting of Theorem 1 (Sec. III-B, Fig. 2), reproduced on the GPU.

An imbalanced two-block SBM: a sparse block B1 (p1 = 0.1), a dense block B2
(p2 = 0.8), cross-block probability q = p1 / 2 = 0.05, 50 vertices per
block.  Theorem 1: in expectation TW recovers the two blocks and Tectonic
does not.  For `seeds` graphs (one batch), this sweeps TW, Tectonic, K3 and
K4 over their threshold grids with tec_sweep and scores every threshold
against the planted blocks with tec_ari and tec_prf (Sec. IV-A).

    python -m paper_2412_12382_gb300.demo_theorem1 [--seeds 20]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SIZES = [50, 50]
PROBS = [[0.1, 0.05], [0.05, 0.8]]


def grids():
    """Threshold grid (p, q) of each measure: TW over -30..10 (Table 4 sweeps
    -30..0), Tectonic over b/128, K3 over 0..30 triangles, K4 over 0..60."""
    from paper_2412_12382_gb300 import K3, K4, TECTONIC, TW
    return {"TW": (TW, list(range(-30, 11)), [1] * 41),
            "Tectonic": (TECTONIC, list(range(1, 65)), [128] * 64),
            "K3": (K3, list(range(0, 31)), [1] * 31),
            "K4": (K4, list(range(0, 61, 2)), [1] * 31)}


def run(seeds: int = 20, first_seed: int = 100):
    """Per measure: mean ARI, precision, recall and F1 over the seeds at every
    threshold, and the threshold of best mean F1 with its exact-recovery rate."""
    import torch
    from graphgen import sbm_csr
    from graphgen.batch import disjoint_union
    from paper_2412_12382_gb300 import Graph
    graphs, truths = [], []
    for s in range(seeds):
        off, col, blk = sbm_csr(SIZES, PROBS, seed=first_seed + s)
        graphs.append((off, col))
        truths.append(blk)
    off, col, seg = disjoint_union(graphs)
    g = Graph(torch.from_numpy(off).cuda(), torch.from_numpy(col).cuda())
    segd = torch.from_numpy(seg).cuda()
    truth = torch.from_numpy(np.concatenate(truths).astype(np.int32)).cuda()
    out = {}
    for name, (measure, ps, qs) in grids().items():
        lab, _ = g.sweep(measure, ps, qs, seg_off=segd)
        ari = g.ari(lab, truth, segd).cpu().numpy()              # thresholds x seeds
        prf = g.prf(lab, truth, segd).cpu().numpy()              # thresholds x seeds x 3
        mean_f1 = prf[:, :, 2].mean(axis=1)
        best = int(mean_f1.argmax())
        out[name] = {"thresholds": [f"{p}/{q}" for p, q in zip(ps, qs)],
                     "mean_ari": ari.mean(axis=1).tolist(),
                     "mean_precision": prf[:, :, 0].mean(axis=1).tolist(),
                     "mean_recall": prf[:, :, 1].mean(axis=1).tolist(),
                     "mean_f1": mean_f1.tolist(),
                     "best_threshold": f"{ps[best]}/{qs[best]}", "best_mean_f1": float(mean_f1[best]),
                     "best_mean_ari": float(ari[best].mean()),
                     "exact_recovery_rate": float((ari[best] == 1.0).mean())}
    g.free()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--seeds", type=int, default=20)
    ap.add_argument("--json", action="store_true", help="print every threshold's scores as JSON")
    args = ap.parse_args(argv)
    from paper_2412_12382_gb300 import build
    build.build()
    res = run(args.seeds)
    if args.json:
        print(json.dumps(res))
        return
    print(f"imbalanced SBM {SIZES}, p1 = {PROBS[0][0]}, p2 = {PROBS[1][1]}, q = {PROBS[0][1]}, {args.seeds} seeds")
    for name, r in res.items():
        print(f"{name:9s} best threshold {r['best_threshold']:>7s}: mean F1 {r['best_mean_f1']:.3f}, "
              f"mean ARI {r['best_mean_ari']:.3f}, blocks recovered exactly in {100 * r['exact_recovery_rate']:.0f}%")


if __name__ == "__main__":
    main()
