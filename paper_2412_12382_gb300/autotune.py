"""Autotuner for the compile-time tile, batch and visit sizes of the CUDA library.

Every tunable is one ``constexpr int NAME = value;`` (or ``int64_t``) line of a
file under ``csrc/``.  A variant is the library built from copies of the
sources with some of those values replaced (`build_variant`).  A variant
whose kernels spill more than the current sources do (from ``-Xptxas -v``;
the current values are built first as that baseline) is rejected, and so is
one that fails to build.  Each kept variant is timed by running a command,
normally a short ``bench.py`` run, with ``TEC_LIBRARY`` pointing the binding
at the variant's library.  A metric is read from the command's last JSON
line, and the median of ``reps`` runs is the variant's cost.  A check
command (``--check-cmd``, e.g. the GPU parity tests) can be required to pass
against each variant before it is timed.

The search is coordinate descent from the current values: each parameter in
turn takes its best candidate with the others fixed, until a full round
changes nothing.  Every timed point goes into a JSON cache.  The cache key
covers the device, the workload's size class, the hash of the sources, the
command and the metric, so a later run resumes, each size class keeps its own
optimum, and a source change starts afresh.

    python -m paper_2412_12382_gb300.autotune --params C_BATCH,B_BATCH \\
        --metric config.stage_ms.support \\
        --cmd "python bench.py --steps 2 --warmup 3 --no-cpu-baseline --no-e2e --no-sweep --no-picker"
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import shlex
import shutil
import statistics
import subprocess
import sys
import tempfile

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

# name -> (file under csrc/, candidate values).  The candidates respect each
# constant's limits: batches and per-lane loads fit a warp's registers and
# lanes (at most 32 candidates per batch), visit sizes are powers of two.
TUNABLES = {
    "C_BATCH": ("support.cu", [8, 12, 16, 24, 32]),
    "B_BATCH": ("support.cu", [4, 8, 16, 32]),
    "C_ROW_LOADS": ("support.cu", [8, 12, 16, 20, 24]),
    "C_SHORT_LOADS": ("support.cu", [2, 4, 6, 8]),
    "UNROLL": ("support.cu", [2, 4, 6, 8]),
    "VISIT_PROBES_B": ("support.cu", [1 << 23, 1 << 24, 1 << 25, 1 << 26]),
    "W_GRAB": ("support.cu", [4, 8, 16, 32]),
    "K4_GRAB": ("k4.cu", [1, 2, 4, 8]),
    "VCHUNK_V": ("tec_internal.cuh", [4, 8, 16]),      # vertices per lane in the sweep's vertex passes
    "BS_CHUNK": ("eval.cu", [2048, 4096, 8192, 16384]),
    "T_BATCH": ("support.cu", [1, 2, 4, 8, 16]),          # candidates per batch of a tiled visit
    "HEAVY_CAND": ("support.cu", [4, 8, 16, 32, 64]),     # candidates per range for a centre to be tiled
    "CORE_ORDER": ("support.cu", [0, 1, 2]),                  # core visits: id order, d+ down, d+ up
    "ORIENT_FLAGS_PERSISTENT": ("orient.cu", [0, 1]),       # orientation passes: one block per tile or
    "ORIENT_FILL_PERSISTENT": ("orient.cu", [0, 1]),        # persistent with bulk-copied tiles
    "ORIENT_FLAGS_MIN_BLOCKS": ("orient.cu", [1, 6, 7, 8]),  # register budget of the flag pass
    "ORIENT_GATHER_CG": ("orient.cu", [0, 1]),              # degree gathers bypass L1
    "PRUNE_SEG_ITEMS": ("prune.cu", [1, 2, 4, 8]),          # batched prune: items whose loads fly together
    "PRUNE_SEG_PERSISTENT": ("prune.cu", [0, 1]),           # batched prune: tiles per block or persistent warps
    "FEAT_PERSISTENT": ("eval.cu", [0, 1]),                 # feature histogram: tiles per block or persistent warps
}


def _pattern(name: str):
    return re.compile(r"(constexpr\s+(?:int|int64_t|unsigned)\s+" + re.escape(name) + r"\s*=\s*)([^;]+)(;)")


def current_value(text: str, name: str) -> str:
    """The right-hand side of NAME's constexpr line (exactly one must exist)."""
    found = _pattern(name).findall(text)
    if len(found) != 1:
        raise ValueError(f"{name}: expected one constexpr definition, found {len(found)}")
    return found[0][1].strip()


def int_value(expr: str) -> int:
    """An integer constant as written in the sources: `123` or `1 << 25`."""
    m = re.fullmatch(r"\s*(\d+)\s*(?:<<\s*(\d+)\s*)?", expr)
    if not m:
        raise ValueError(f"not a plain integer constant: {expr!r}")
    return int(m.group(1)) << int(m.group(2) or 0)


def substitute(text: str, name: str, value: int) -> str:
    """`text` with NAME's constexpr value replaced by `value`."""
    current_value(text, name)
    return _pattern(name).sub(lambda m: m.group(1) + str(int(value)) + m.group(3), text, count=1)


def source_hash() -> str:
    h = hashlib.sha256()
    for path in sorted(os.listdir(_build.CSRC)):
        if path.endswith((".cu", ".cuh", ".h")):
            h.update(path.encode())
            h.update(open(os.path.join(_build.CSRC, path), "rb").read())
    h.update(open(os.path.join(INCLUDE, "tectonic.h"), "rb").read())
    return h.hexdigest()[:16]


def spill_bytes(diagnostics: dict) -> dict:
    """Per source file, the spill store + load bytes of all its kernels in the
    ptxas report."""
    out = {}
    for name, text in diagnostics.items():
        out[name] = sum(int(a) + int(b) for a, b in
                        re.findall(r"(\d+) bytes spill stores, (\d+) bytes spill loads", text))
    return out


def spills_worse(variant: dict, baseline: dict) -> list:
    """Files whose kernels spill more in the variant than in the baseline."""
    return sorted(f for f, v in variant.items() if v > baseline.get(f, 0))


def write_variant_sources(overrides: dict, root: str) -> str:
    """Copies csrc/ and the public header under `root` with the overrides
    applied; returns the variant's csrc directory."""
    csrc = os.path.join(root, "pkg", "csrc")
    os.makedirs(csrc, exist_ok=True)
    os.makedirs(os.path.join(root, "include"), exist_ok=True)
    shutil.copy(os.path.join(INCLUDE, "tectonic.h"), os.path.join(root, "include", "tectonic.h"))
    by_file = {}
    for name, value in overrides.items():
        if name not in TUNABLES:
            raise ValueError(f"{name} is not a tunable")
        by_file.setdefault(TUNABLES[name][0], []).append((name, value))
    for fname in os.listdir(_build.CSRC):
        if not fname.endswith((".cu", ".cuh", ".h")):
            continue
        text = open(os.path.join(_build.CSRC, fname)).read()
        for name, value in by_file.get(fname, []):
            text = substitute(text, name, value)
        with open(os.path.join(csrc, fname), "w") as f:
            f.write(text)
    return csrc


def build_variant(overrides: dict, root: str):
    """Builds the variant under `root`: (library path, spill bytes per file)."""
    csrc = write_variant_sources(overrides, root)
    lib, diags = _build.compile_library(csrc, os.path.join(root, "build"), ptxas_info=True)
    return lib, spill_bytes(diags)


def read_metric(stdout: str, path: str) -> float:
    """Value at a dotted path of the last JSON object line of `stdout`."""
    for line in reversed(stdout.strip().splitlines()):
        line = line.strip()
        if line.startswith("{"):
            node = json.loads(line)
            for key in path.split("."):
                node = node[key]
            return float(node)
    raise ValueError("the command printed no JSON line")


def time_variant(lib: str, cmd: str, metric: str, reps: int, cwd: str) -> float:
    values = []
    env = dict(os.environ, TEC_LIBRARY=lib)
    for _ in range(reps):
        r = subprocess.run(shlex.split(cmd), capture_output=True, text=True, env=env, cwd=cwd)
        if r.returncode != 0:
            raise RuntimeError(f"timing command failed ({r.returncode}):\n{r.stderr[-2000:]}")
        values.append(read_metric(r.stdout, metric))
    return statistics.median(values)


def coordinate_descent(space: dict, start: dict, evaluate, lower_is_better: bool = True, max_rounds: int = 4,
                       min_gain: float = 0.0):
    """Coordinate descent over `space` (name -> candidates) from `start`.
    evaluate(point) returns a cost, or None for a point that cannot run.  A
    move is taken only when it improves the cost by more than the fraction
    `min_gain` (differences within one run's noise do not change constants).
    Returns (best point, best cost, {point key: cost})."""
    seen = {}

    def cost(point):
        key = json.dumps(point, sort_keys=True)
        if key not in seen:
            seen[key] = evaluate(dict(point))
        return seen[key]

    def better(a, b):
        if a is None:
            return False
        if b is None:
            return True
        return a < b * (1.0 - min_gain) if lower_is_better else a > b * (1.0 + min_gain)

    best = dict(start)
    best_cost = cost(best)
    for _ in range(max_rounds):
        changed = False
        for name, candidates in space.items():
            for v in candidates:
                if v == best[name]:
                    continue
                trial = dict(best, **{name: v})
                c = cost(trial)
                if better(c, best_cost):
                    best, best_cost, changed = trial, c, True
        if not changed:
            break
    return best, best_cost, seen


def check_variant(lib: str, check_cmd: str, cwd: str) -> bool:
    """Runs a correctness command (e.g. the GPU parity tests) against the variant."""
    env = dict(os.environ, TEC_LIBRARY=lib)
    return subprocess.run(shlex.split(check_cmd), capture_output=True, text=True, env=env, cwd=cwd).returncode == 0


def tune(params, cmd, metric, reps=3, lower_is_better=True, cache_path=None, device="", cwd=None, log=print,
         check_cmd=None, size_class="", min_gain=0.005):
    cwd = cwd or os.path.dirname(HERE)
    texts = {f: open(os.path.join(_build.CSRC, f)).read() for f in {TUNABLES[p][0] for p in params}}
    start = {p: int_value(current_value(texts[TUNABLES[p][0]], p)) for p in params}
    space = {p: sorted(set(TUNABLES[p][1]) | {start[p]}) for p in params}
    key = json.dumps({"device": device, "size_class": size_class, "sources": source_hash(), "cmd": cmd,
                      "metric": metric, "reps": reps, "check": check_cmd})
    cache = {}
    if cache_path and os.path.exists(cache_path):
        cache = json.load(open(cache_path))
    entries = cache.setdefault(key, {})

    with tempfile.TemporaryDirectory(prefix="tec_variant_") as root:
        _, baseline = build_variant(start, root)     # the current sources' own spills are accepted

    def evaluate(point):
        pk = json.dumps(point, sort_keys=True)
        if pk in entries:
            return entries[pk]
        with tempfile.TemporaryDirectory(prefix="tec_variant_") as root:
            try:
                lib, spilled = build_variant(point, root)
            except RuntimeError as e:
                log(f"{point}: build failed: {str(e).splitlines()[0]}")
                entries[pk] = None
                return None
            bad = spills_worse(spilled, baseline)
            if bad:
                log(f"{point}: spills more than the current sources in {', '.join(bad)}, skipped")
                entries[pk] = None
            elif check_cmd and not check_variant(lib, check_cmd, cwd):
                log(f"{point}: fails the check command, skipped")
                entries[pk] = None
            else:
                entries[pk] = time_variant(lib, cmd, metric, reps, cwd)
                log(f"{point}: {entries[pk]:.4g}")
        if cache_path:
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
        return entries[pk]

    best, best_cost, _ = coordinate_descent(space, start, evaluate, lower_is_better, min_gain=min_gain)
    return start, best, best_cost, entries


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--params", required=True, help="comma-separated tunables: " + ", ".join(TUNABLES))
    ap.add_argument("--cmd", required=True, help="timing command, run from the repository root")
    ap.add_argument("--metric", required=True, help="dotted path of the value in the command's JSON line")
    ap.add_argument("--higher-is-better", action="store_true")
    ap.add_argument("--check-cmd", default=None,
                    help="correctness command each variant must pass before it is timed, e.g. "
                         "'python -m pytest tests/test_gpu_parity.py -m gpu -x -q'")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--cache", default="autotune_cache.json")
    ap.add_argument("--min-gain", type=float, default=0.005,
                    help="smallest relative improvement that changes a constant (default 0.5%%, about one run's "
                         "noise on the scale-26 triangle stage)")
    ap.add_argument("--size-class", default="",
                    help="label of the workload's size class (e.g. rmat26, rmat22, dcsbm256): the best "
                         "constants differ between classes, so each has its own cache entries")
    args = ap.parse_args(argv)
    params = [p.strip() for p in args.params.split(",") if p.strip()]
    device = ""
    try:
        import torch
        if torch.cuda.is_available():
            device = torch.cuda.get_device_name(0)
    except ImportError:
        pass
    start, best, cost, _ = tune(params, args.cmd, args.metric, args.reps, not args.higher_is_better,
                                args.cache, device, check_cmd=args.check_cmd, size_class=args.size_class,
                                min_gain=args.min_gain)
    print(json.dumps({"start": start, "best": best, "cost": cost, "metric": args.metric,
                      "size_class": args.size_class}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
