"""The reference arm of bench.py (the oracle timed on host cores) keeps the
JSON-line contract on a machine without a GPU: one line, the same metric and
unit as the CUDA arm, `impl` = reference, a cpu_baseline describing the run,
and an e2e block without host-device bytes.  Workloads whose input needs the
device generator say so in an `unavailable` line and exit 0."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args, timeout=300):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       cwd=ROOT, env=env, timeout=timeout)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def test_reference_arm_line_on_the_sbm_workload():
    pytest.importorskip("torch")
    import bench
    d = _run("--impl", "reference", "--workload", "sbm", "--steps", "1", "--warmup", "0")
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["m"] == 28039 and d["config"]["n"] == 2000
    # the step time is the one measured (a bounded sample), the full-graph projection a key of its own
    assert 0 < d["ms_per_step"] < 60_000 and d["ms_per_step_kind"].startswith("measured")
    assert d["projected_ms_per_full_graph"] > 0 and cb["cpu_model"]


def test_reference_arm_without_the_device_generator_is_unavailable():
    pytest.importorskip("torch")
    d = _run("--impl", "reference", "--workload", "rmat26", "--steps", "1", "--warmup", "0")
    assert d["impl"] == "reference" and "unavailable" in d
