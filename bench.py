"""Benchmark of the full Tectonic pass (Algorithm 1 on one GPU).

One step = one full pass over a graph already resident in HBM: degree
orientation, per-edge triangle counts, Tectonic similarity, pruning at
theta = 1/10 with fused union-find hooking, component labels.  Default
workload: R-MAT scale 26, edge factor 32, (a,b,c,d) = (0.57,0.19,0.19,0.05),
seed 3, generated on the GPU (untimed input preparation).

Prints one JSON line (rank 0): the pass's edges/s, the triangle stage
against the measured HBM bandwidth (`roofline`), the same pass from host
buffers (`e2e`), the oracle on a bounded sample (`cpu_baseline`), and two
further blocks: the batched 64-threshold sweep over 256 DC-SBM graphs and
the learned picker against the full sweep on 500 held-out DC-SBM graphs.
`--impl reference` times the CPU oracle on a bounded edge sample instead.
Under torchrun every rank runs its own replica (the path does not shard:
replicas only) and rank 0 reports the total.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Tectonic pass edges/s (1 GB300, % HBM roofline)"
UNIT = "edges/s"

WORKLOADS = {
    "rmat26": dict(kind="rmat", scale=26, edge_factor=32, seed=3, p=1, q=10,
                   name="R-MAT scale 26, edge factor 32, (0.57,0.19,0.19,0.05), seed 3; Tectonic full pass at 1/10"),
    "rmat20": dict(kind="rmat", scale=20, edge_factor=16, seed=2, p=1, q=10,
                   name="R-MAT scale 20, edge factor 16, (0.57,0.19,0.19,0.05), seed 2; Tectonic full pass at 1/10"),
    "rmat22": dict(kind="rmat", scale=22, edge_factor=16, seed=2, p=1, q=10,
                   name="R-MAT scale 22, edge factor 16, (0.57,0.19,0.19,0.05), seed 2; Tectonic full pass at 1/10"),
    "sbm": dict(kind="sbm", p=3, q=50,
                name="planted-partition SBM n=2000, 4x500, p_in=0.05, p_out=0.002, seed 1; Tectonic at 3/50"),
}

# DRAM bytes per launch of the triangle-count stage from an ncu capture, per
# unit of algorithmic bytes, valid only for the support.cu it was taken on
# (see profiles/).  None until a capture exists for the current source.
TRAFFIC_CAPTURE = {"support_sha": "9f53b7b10502a1dc", "dram_per_alg_byte": 86.613 / 49.162954,
                   "source": "ncu DRAM bytes of the triangle-count stage's kernels at R-MAT scale 22, "
                             "scaled by algorithmic bytes",
                   # the same counters taken directly on the R-MAT scale-26 launch (one-pass capture)
                   "rmat26_bytes": 10731397195520 + 3483785178112 + 177139897856 + 3276615168,
                   "rmat26_source": "ncu DRAM bytes (read + write) of k_support_core and k_support, one launch "
                                    "each, on the R-MAT scale-26 workload itself"}

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def support_sha() -> str:
    """Hash of the triangle-count source with comments and whitespace removed:
    a comment edit leaves a recorded capture valid, a code edit does not."""
    import re
    with open(os.path.join(ROOT, "paper_2412_12382_gb300", "csrc", "support.cu")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = re.sub(r"\s+", " ", src)
    return hashlib.sha256(src.encode()).hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks sampled every 200 ms while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={CLOCK_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_workload(spec, device):
    import numpy as np
    import torch
    if spec["kind"] == "rmat":
        from graphgen.gpu import rmat_csr_gpu
        off, col = rmat_csr_gpu(spec["scale"], spec["edge_factor"], seed=spec["seed"])
        return off, col
    from graphgen import planted_partition
    off, col, _ = planted_partition(4, 500, 0.05, 0.002, seed=1)
    return torch.from_numpy(off).to(device), torch.from_numpy(np.asarray(col)).to(device)


def algorithmic_bytes(off, ooff, ocol, m):
    """Algorithmic bytes of one pass.

    W = sum_v d-(v) d+(v) + m: neighbour reads when every oriented edge u->v
    reads N+(v) and every N+(u) is staged once.  B_alg = 4W + 36m + 16n.
    W_min = sum over oriented edges x->y of min(d+(x), d+(y)): the probes the
    implemented kernels make (each edge is intersected from its shorter side).
    B_sup = 4 W_min + 28m for the triangle-count stage: probe reads, each
    out-row staged once (4m), row bounds of each probe row (16m), one
    read-modify-write of every counter (8m).  B_alg_min = 4 W_min + 40m + 16n
    replaces 4W by 4(W_min + m) in B_alg."""
    import torch
    n = off.numel() - 1
    deg = off[1:] - off[:-1]
    dplus = ooff[1:] - ooff[:-1]
    W = int(((deg - dplus) * dplus).sum().item()) + m
    W_min = 0
    r0 = 0
    step = 1 << 22
    while r0 < n:
        r1 = min(n, r0 + step)
        a, b = int(ooff[r0].item()), int(ooff[r1].item())
        if b > a:
            rows = torch.repeat_interleave(torch.arange(r0, r1, device=off.device), dplus[r0:r1])
            W_min += int(torch.minimum(dplus[rows], dplus[ocol[a:b].long()]).sum().item())
            del rows
        r0 = r1
    return {"W": W, "W_min": W_min, "B_alg": 4 * W + 36 * m + 16 * n,
            "B_alg_min": 4 * W_min + 40 * m + 16 * n, "B_sup": 4 * W_min + 28 * m}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline line."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_sample_rate(off_h, col_h, p, q, target_s=12.0, seed=0):
    """The oracle as it stands on a uniform sample of canonical edges: merge
    counts (all host threads) + exact prune.  Returns (edges/s, sample, threads)."""
    import numpy as np
    import oracle as O
    threads = O.threads_available()
    n = len(off_h) - 1
    rng = np.random.default_rng(seed)
    deg = np.diff(off_h)
    m = int(off_h[-1]) // 2

    def sample(k):
        # uniform over symmetric entries, keep the u < v copy -> uniform over edges
        ks = rng.integers(0, len(col_h), size=2 * k)
        rows = np.searchsorted(off_h, ks, side="right") - 1
        cols = col_h[ks].astype(np.int64)
        sel = rows < cols
        return rows[sel][:k].astype(np.int32), cols[sel][:k].astype(np.int32)

    k = 2000
    total_e, total_t = 0, 0.0
    while total_t < target_s:
        eu, ev = sample(k)
        t0 = time.perf_counter()
        t, uni = O.edge_counts(off_h, col_h, eu, ev, nthreads=threads)
        O.prune(O.TECTONIC, off_h, eu, ev, t, uni, p, q)
        dt = time.perf_counter() - t0
        total_e += len(eu)
        total_t += dt
        rate = len(eu) / max(dt, 1e-9)
        k = int(min(max(k * 2, rate * 2.0), 50_000_000))
    return total_e / total_t, total_e, threads, total_t


def _timed(fn, stream, reps):
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    out = None
    for a, b in ev:
        a.record(stream)
        out = fn()
        b.record(stream)
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in ev), out


def bench_batched_sweep(reps=3):
    """256 degree-corrected SBM graphs (seeds 1000-1255, n log-uniform in
    [1000, 200000]) as one batch: components at the 64 thresholds b/128 by the
    spanning-forest sweep, against 64 independent prune + components passes."""
    import torch
    side = torch.cuda.Stream()          # CUDA-graph capture needs a non-default stream
    with torch.cuda.stream(side):
        return _bench_batched_sweep(reps)


def _bench_batched_sweep(reps):
    import torch
    from graphgen.gpu import dcsbm_batch_gpu
    from paper_2412_12382_gb300 import TECTONIC, Graph
    from paper_2412_12382_gb300 import picker as PK
    t0 = time.time()
    off, col, seg, truth, specs = dcsbm_batch_gpu(list(range(1000, 1256)), 1000, 200000)
    gen_s = time.time() - t0
    g = Graph(off, col)
    stream = g.stream
    sup_ms, _ = _timed(lambda: g.support(), stream, 2)
    nseg = seg.numel() - 1
    sweep_ms, _ = _timed(lambda: g.sweep(TECTONIC, PK.GRID_P, PK.GRID_Q, seg_off=seg, count=False), stream,
                         reps + 1)
    thr = [(torch.full((nseg,), b, dtype=torch.int64, device="cuda"),
            torch.full((nseg,), 128, dtype=torch.int64, device="cuda")) for b in PK.GRID_P]
    lab = torch.empty(g.n, dtype=torch.int32, device="cuda")

    def independent():
        for p, q in thr:
            g.prune_components_batch(TECTONIC, p, q, seg, labels=lab, count=False)

    ind_ms, _ = _timed(independent, stream, reps)
    # the same sweep captured once in a CUDA graph and replayed
    lab_g = None
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=stream):
        lab_g, _ = g.sweep(TECTONIC, PK.GRID_P, PK.GRID_Q, seg_off=seg, count=False)
    graph_ms, _ = _timed(cg.replay, stream, reps + 1)
    ref, _ = g.sweep(TECTONIC, PK.GRID_P, PK.GRID_Q, seg_off=seg, count=False)
    same = bool(torch.equal(lab_g, ref))
    del cg
    m = g.m
    g.free()
    return {"workload": "256 DC-SBM graphs, seeds 1000-1255, n log-uniform in [1e3, 2e5], 64 thresholds b/128",
            "graphs": nseg, "n": int(off.numel() - 1), "m": int(m), "support_ms": sup_ms,
            "sweep_ms": sweep_ms, "sweep_cuda_graph_ms": graph_ms, "cuda_graph_labels_match": same,
            "independent_passes_ms": ind_ms, "speedup_vs_independent": ind_ms / sweep_ms,
            "graphs_per_s": nseg / (sweep_ms / 1e3), "edges_per_s": m / (sweep_ms / 1e3),
            "input_generation_s": gen_s}


def bench_picker(reps=3):
    """Held-out DC-SBM graphs (seeds 20000-20499, n log-uniform in [1000,
    100000]) as one batch, with the shipped picker checkpoint.
    Picker path: tec_pick_threshold (features, bf16 network, grid threshold)
    and one batched prune + components.  Sweep path: components at the 64
    thresholds b/128 (64 independent batched passes; the spanning-forest sweep
    is reported beside it), 64 ARI evaluations and the best level per graph.
    The triangle counts, shared by both, are timed apart."""
    import numpy as np
    import torch
    from graphgen.gpu import dcsbm_batch_gpu
    from paper_2412_12382_gb300 import TECTONIC, Graph
    from paper_2412_12382_gb300 import picker as PK
    from paper_2412_12382_gb300 import tectonic as T
    ckpt = os.path.join(ROOT, "paper_2412_12382_gb300", "picker_weights.tecp")
    pk, meta = PK.load(ckpt)
    off, col, seg, truth, specs = dcsbm_batch_gpu(list(range(20000, 20500)), 1000, 100000)
    g = Graph(off, col)
    stream = g.stream
    nseg = seg.numel() - 1
    sup_ms, _ = _timed(lambda: g.support(), stream, 2)
    lab_all = torch.empty((PK.K, g.n), dtype=torch.int32, device="cuda")
    thr = [(torch.full((nseg,), b, dtype=torch.int64, device="cuda"),
            torch.full((nseg,), PK.DEN, dtype=torch.int64, device="cuda")) for b in PK.GRID_P]

    def picker_path():
        p, q = g.pick_threshold(pk, seg, bf16=True)
        return g.prune_components_batch(TECTONIC, p, q, seg, count=False)[0]

    def sweep_independent():
        for L, (p, q) in enumerate(thr):
            g.prune_components_batch(TECTONIC, p, q, seg, labels=lab_all[L], count=False)
        return T.ari_best(g.ari(lab_all, truth, seg))

    def sweep_msf():
        labels, _ = g.sweep(TECTONIC, PK.GRID_P, PK.GRID_Q, seg_off=seg, count=False)
        return T.ari_best(g.ari(labels, truth, seg))

    picker_ms, plab = _timed(picker_path, stream, reps + 1)
    ind_ms, (best_i, best_ari_i) = _timed(sweep_independent, stream, reps)
    msf_ms, (best, best_ari) = _timed(sweep_msf, stream, reps + 1)
    got = g.ari(plab[None, :], truth, seg)[0]
    ari_all = g.ari(lab_all, truth, seg)
    # the same picker with float32 inference, for the bf16 / fp32 comparison
    p32, _ = g.pick_threshold(pk, seg, bf16=False)
    p16, _ = g.pick_threshold(pk, seg, bf16=True)
    cols32 = torch.arange(nseg, device="cuda")
    got32 = ari_all[(p32 - 1).long(), cols32]
    same_level = float((p32 == p16).float().mean().item())
    fixed_level = int(meta.get("eval", {}).get("fixed_level", 8)) - 1
    # the paper's rules of thumb (Sec. IV-D) on the same sweep, as baselines
    stats = g.sweep_stats(TECTONIC, PK.GRID_P, PK.GRID_Q, lab_all, seg)
    cols = torch.arange(nseg, device="cuda")
    rule_ari = {}
    for name, rule in (("R1", T.RULE_LARGEST_JUMP), ("R2", T.RULE_MODULARITY)):
        rows = T.rule_of_thumb(stats, PK.GRID_P, PK.GRID_Q, nseg, rule).long()
        rule_ari[name] = float(ari_all[rows, cols].mean())
    stats_ms, _ = _timed(lambda: g.sweep_stats(TECTONIC, PK.GRID_P, PK.GRID_Q, lab_all, seg), stream, 2)
    d = (best_ari - got).cpu().numpy()
    out = {"workload": "500 held-out DC-SBM graphs, seeds 20000-20499, n log-uniform in [1e3, 1e5]",
           "graphs": int(nseg), "n": int(g.n), "m": int(g.m), "picker_ms": picker_ms,
           "sweep_independent_ms": ind_ms, "sweep_msf_ms": msf_ms,
           "ratio_sweep_over_picker": ind_ms / picker_ms, "ratio_msf_sweep_over_picker": msf_ms / picker_ms,
           "support_ms": sup_ms, "ratio_including_support": (ind_ms + sup_ms) / (picker_ms + sup_ms),
           "ratio_msf_including_support": (msf_ms + sup_ms) / (picker_ms + sup_ms),
           "same_best_both_sweeps": bool(torch.equal(best, best_i)),
           "mean_dARI": float(d.mean()), "p95_dARI": float(np.percentile(d, 95)), "max_dARI": float(d.max()),
           "mean_dARI_fp32": float((best_ari - got32).mean().item()), "bf16_same_level_fraction": same_level,
           "mean_ARI_picker": float(got.mean()), "mean_ARI_best": float(best_ari.mean()),
           "mean_ARI_fixed": float(ari_all[fixed_level].mean()), "fixed_threshold": f"{fixed_level + 1}/128",
           "mean_ARI_R1_largest_jump": rule_ari["R1"], "mean_ARI_R2_modularity": rule_ari["R2"],
           "sweep_stats_ms": stats_ms,
           "inference": "bf16", "trained_on": meta.get("train_seeds"), "epochs_kept": meta.get("epochs_kept")}
    g.free()
    pk.free()
    return out


def slowest(seconds: float, dist=None, device=None) -> float:
    """The largest of every rank's `seconds` (the local value without a process group)."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, seconds: float, world: int, dist=None, device=None):
    """Whole-job throughput of `world` replicas that each processed
    units_per_rank: all units over the slowest rank's time.  Returns
    (units per second, that time)."""
    s = slowest(seconds, dist, device)
    return world * units_per_rank / s, s


def run_reference(args, spec, rank, world):
    import numpy as np
    import torch
    if rank != 0:
        return 0
    dev = torch.device("cuda", 0) if torch.cuda.is_available() else None
    if dev is None and spec["kind"] == "rmat" and spec["scale"] > 18:
        print(json.dumps({"impl": "reference", "unavailable": "workload generator needs a GPU"}))
        return 0
    off, col = make_workload(spec, dev)
    off_h = off.cpu().numpy().astype(np.int64)
    col_h = col.cpu().numpy().astype(np.int32)
    del off, col
    m = int(off_h[-1]) // 2
    import oracle as O
    threads = O.threads_available()
    for _ in range(args.warmup):
        oracle_sample_rate(off_h, col_h, spec["p"], spec["q"], target_s=0.5)
    times, edges, walls = [], 0, []
    for s in range(args.steps):
        w0 = time.perf_counter()
        rate, k, thr, tt = oracle_sample_rate(off_h, col_h, spec["p"], spec["q"], target_s=6.0, seed=s)
        walls.append(time.perf_counter() - w0)
        times.append(tt)
        edges += k
    value = edges / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(walls),
            "ms_per_step_kind": "measured: one step = one bounded edge sample of the workload",
            "projected_ms_per_full_graph": 1e3 * m / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": spec["name"], "m": m, "n": len(off_h) - 1},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "cpu_model": cpu_model(),
                             "kind": "oracle",
                             "sample": f"{edges} uniformly sampled edges over {args.steps} steps: merge "
                                       "intersections + exact prune (components not included)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat26", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the batched sweep measurement")
    ap.add_argument("--no-picker", action="store_true", help="skip the picker-vs-sweep measurement")
    ap.add_argument("--only", choices=["sweep", "picker"], default=None,
                    help="profiling aid: run only the batched sweep or only the picker-vs-sweep block "
                         "and print its result (not a bench line)")
    args = ap.parse_args()
    if args.warmup < 3:
        log("warning: fewer than 3 warm-up steps")
    spec = WORKLOADS[args.workload]

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))

    import numpy as np
    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if args.impl == "reference":
        rc = run_reference(args, spec, rank, world)
        if dist is not None:
            dist.destroy_process_group()
        return rc

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a GPU for --impl ours")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2412_12382_gb300 import TECTONIC, Graph
    from paper_2412_12382_gb300 import build as libbuild
    from paper_2412_12382_gb300 import tectonic as T
    libbuild.build()
    if args.only:
        res = bench_batched_sweep() if args.only == "sweep" else bench_picker()
        print(json.dumps({"only": args.only, "result": res}), flush=True)
        return 0

    t0 = time.time()
    off, col = make_workload(spec, dev)
    torch.cuda.synchronize()
    n = off.numel() - 1
    nnz = col.numel()
    m = nnz // 2
    log(f"workload {args.workload}: n={n} m={m} nnz={nnz} built in {time.time() - t0:.1f}s")

    g = Graph(off, col)
    stream = g.stream
    p, q = spec["p"], spec["q"]
    labels = torch.empty(n, dtype=torch.int32, device=dev)

    for _ in range(args.warmup):
        g.full_pass(TECTONIC, p, q, labels=labels, count=False)
    g.sync()
    ooff, ocol = g.oriented_csr()
    ab = algorithmic_bytes(off, ooff, ocol, m)
    del ooff, ocol
    torch.cuda.empty_cache()
    B_sup = ab["B_sup"]
    # one set of stage events per timed step, recorded on the graph's stream
    step_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = T.launch_count()
    with ClockSampler(torch.cuda.current_device()) as clk:
        start.record(stream)
        for k in range(args.steps):
            g.set_stage_events(step_ev[k])
            g.full_pass(TECTONIC, p, q, labels=labels, count=False)
        end.record(stream)
        torch.cuda.synchronize()
    launches = T.launch_count() - l0
    g.sync()
    stage_ms = [[e[i].elapsed_time(e[i + 1]) for e in step_ev] for i in range(4)]
    value, step_s = job_throughput(m, start.elapsed_time(end) / 1e3 / args.steps, world, dist, dev)
    if dist is not None:
        dist.barrier()
    ms_per_step = step_s * 1e3
    _, ncomp = g.full_pass(TECTONIC, p, q, labels=labels, count=True)
    g.set_stage_events([])

    peak, peak_kind = load_peaks()
    sup_ms = statistics.mean(stage_ms[1])
    achieved = B_sup / (sup_ms / 1e3) / 1e9
    traffic = None
    traffic_source = None
    if TRAFFIC_CAPTURE["support_sha"] == support_sha():
        if args.workload == "rmat26" and TRAFFIC_CAPTURE["rmat26_bytes"]:
            traffic, traffic_source = TRAFFIC_CAPTURE["rmat26_bytes"], TRAFFIC_CAPTURE["rmat26_source"]
        elif TRAFFIC_CAPTURE["dram_per_alg_byte"]:
            traffic = TRAFFIC_CAPTURE["dram_per_alg_byte"] * B_sup
            traffic_source = TRAFFIC_CAPTURE["source"]
    pass_gbs = ab["B_alg_min"] / (ms_per_step / 1e3) / 1e9

    e2e = None
    if not args.no_e2e:
        off_h = torch.empty(n + 1, dtype=torch.int64, pin_memory=True)
        col_h = torch.empty(nnz, dtype=torch.int32, pin_memory=True)
        off_h.copy_(off)
        col_h.copy_(col)
        lab_h = torch.empty(n, dtype=torch.int32, pin_memory=True)
        on, cn, ln = off_h.numpy(), col_h.numpy(), lab_h.numpy()
        g.full_pass_host(on, cn, TECTONIC, p, q, ln)
        k_e2e = max(1, min(args.steps, 3))
        if dist is not None:
            dist.barrier()
        t1 = time.perf_counter()
        for _ in range(k_e2e):
            g.full_pass_host(on, cn, TECTONIC, p, q, ln)
        e2e_value, _ = job_throughput(m, (time.perf_counter() - t1) / k_e2e, world, dist, dev)
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": (n + 1) * 8 + nnz * 4,
               "d2h_bytes_per_step": n * 4 + 8 * 16}
        ok = np.array_equal(ln, labels.cpu().numpy())
        if not ok:
            raise SystemExit("host-buffer pass disagrees with the device pass")

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        off_np = off.cpu().numpy().astype(np.int64)
        col_np = col.cpu().numpy().astype(np.int32)
        rate, k, thr, tt = oracle_sample_rate(off_np, col_np, p, q, target_s=12.0)
        cpu = {"value": rate, "unit": UNIT, "cores": thr, "cpu_model": cpu_model(), "kind": "oracle",
               "sample": f"{k} uniformly sampled edges of the same graph: merge intersections (Sec. III-C) "
                         f"+ exact prune, {tt:.1f} s on {thr} host threads; components not included"}
        del off_np, col_np

    g.free()
    del off, col, labels
    torch.cuda.empty_cache()
    sweep = picker = None
    if rank == 0 and not args.no_sweep:
        sweep = bench_batched_sweep()
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_picker:
        picker = bench_picker()
        torch.cuda.empty_cache()

    if rank == 0:
        clocks = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": spec["name"], "n": n, "m": m, "theta": f"{p}/{q}",
                       "components": ncomp, "W": ab["W"], "W_min": ab["W_min"],
                       "l2": f"inputs larger than L2: CSR {nnz * 4 / 1e9:.2f} GB vs 0.129 GB",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "pass_alg_bytes": ab["B_alg_min"], "pass_alg_GBps": pass_gbs,
                       "pass_alg_bytes_W": ab["B_alg"],
                       "pass_frac_of_peak": pass_gbs / peak,
                       "stage_ms": {"orient": statistics.mean(stage_ms[0]), "support": sup_ms,
                                    "prune_hook": statistics.mean(stage_ms[2]),
                                    "finish": statistics.mean(stage_ms[3])}},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "frac_survey": ab["B_alg"] / (ms_per_step / 1e3) / 1e9 / peak,
                         "frac_survey_def": "whole pass: B_alg = 4W + 36m + 16n, W = sum_v d-(v) d+(v) + m, "
                                            "over the pass time, of the peak",
                         "kernel": "triangle-count stage (support kernels)",
                         "alg_bytes_per_launch": B_sup, "peak_kind": peak_kind,
                         "traffic_source": traffic_source,
                         "traffic_GBps": traffic / (sup_ms / 1e3) / 1e9 if traffic else None,
                         "traffic_frac": traffic / (sup_ms / 1e3) / 1e9 / peak if traffic else None},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "gpu_launches_per_step": launches / args.steps, "clocks": clocks,
            "batched_sweep": sweep, "picker_vs_sweep": picker,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
