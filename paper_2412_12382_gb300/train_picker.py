"""Trains the threshold picker and writes its checkpoint.

    python -m paper_2412_12382_gb300.train_picker [--out PATH] [--epochs E]

Training graphs: degree-corrected SBM graphs of seeds 10000-19999 with
n in [1000, 100000]; 10% of them (every tenth seed) are a validation split
that picks the epoch count kept.  With --refit the network is then trained
again from the same initialisation on all 10,000 graphs for that epoch
count.  Held-out evaluation: seeds 20000-20499.
Labels: the grid threshold b/128 (b = 1..64) of highest ARI against the
planted blocks, from the full sweep.  Everything runs in the library's
kernels; this script only orders the calls.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DEFAULT_OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "picker_weights.tecp")


def main(argv=None):
    import torch

    from paper_2412_12382_gb300 import build
    from paper_2412_12382_gb300 import picker as P
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--chunk", type=int, default=50, help="epochs between validation checks")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--batch", type=int, default=128)
    ap.add_argument("--train-seeds", type=int, nargs=2, default=(10000, 20000))
    ap.add_argument("--eval-seeds", type=int, nargs=2, default=(20000, 20500))
    ap.add_argument("--n-range", type=int, nargs=2, default=(1000, 100000))
    ap.add_argument("--refit", action="store_true",
                    help="after choosing the epoch count on the validation split, train again from the same "
                         "initialisation on all training graphs (validation split included) for that many "
                         "epochs, and keep that network")
    ap.add_argument("--dataset-cache", default=None,
                    help="directory for the labelled datasets (features + best levels), reused by later runs")
    args = ap.parse_args(argv)
    build.build()
    t0 = time.time()
    seeds = list(range(*args.train_seeds))
    val_seeds = seeds[::10]
    tr_seeds = [s for s in seeds if s % 10 != seeds[0] % 10]
    train = P.cached_dataset(tr_seeds, *args.n_range, cache_dir=args.dataset_cache)
    val = P.cached_dataset(val_seeds, *args.n_range, cache_dir=args.dataset_cache)
    held = P.cached_dataset(list(range(*args.eval_seeds)), *args.n_range, cache_dir=args.dataset_cache)
    t_data = time.time() - t0
    pk = P.T.Picker(P.init_params(0))
    best = (float("inf"), None, 0)
    losses = []
    done = 0
    t1 = time.time()
    while done < args.epochs:
        e = min(args.chunk, args.epochs - done)
        losses += pk.train(train["feats"], train["target"], e, args.batch, args.lr, seed=done + 1).tolist()
        done += e
        v = P.evaluate(pk, val)["mean_dARI"]
        if v < best[0]:
            best = (v, pk.get_params(with_adam=True), done)
    t_train = time.time() - t1
    params, m, v, step = best[1]
    pk.set_params(params, m, v, step)
    epochs_run = done
    refit = None
    if args.refit:
        import torch
        full = {k: torch.cat([train[k], val[k]], dim=1 if k == "ari" else 0) for k in P.DATASET_FIELDS}
        pk.free()
        pk = P.T.Picker(P.init_params(0))
        done = 0
        while done < best[2]:
            e = min(args.chunk, best[2] - done)
            losses += pk.train(full["feats"], full["target"], e, args.batch, args.lr, seed=done + 1).tolist()
            done += e
        refit = {"graphs": int(full["feats"].shape[0]), "epochs": best[2]}
    fixed = P.fixed_level(train)
    res = P.evaluate(pk, held, baseline_level=fixed)
    res_bf16 = P.evaluate(pk, held, bf16=True)
    agree = float((P.predict_levels(pk, held["feats"], False) == P.predict_levels(pk, held["feats"], True))
                  .float().mean().item())
    meta = {"train_seeds": [tr_seeds[0], tr_seeds[-1], len(tr_seeds)], "val_seeds": len(val_seeds),
            "eval_seeds": list(args.eval_seeds), "n_range": list(args.n_range), "epochs_run": epochs_run,
            "epochs_kept": best[2], "val_mean_dARI": best[0], "lr": args.lr, "batch": args.batch,
            "final_train_loss": losses[-1], "first_train_loss": losses[0], "eval": res,
            "eval_bf16": res_bf16, "bf16_same_level_fraction": agree, "refit": refit,
            "seconds": {"data": t_data, "train": t_train}}
    P.save(pk, args.out, meta)
    print(json.dumps(meta))
    pk.free()
    torch.cuda.synchronize()


if __name__ == "__main__":
    main()
