"""Failure detection on the GPU without a GPU fault (debug build).

A debug build of the library (-DTEC_DEBUG) lets the host lower the
union-find retry cap and the number of Boruvka rounds, and refuse named
allocations.  failure_driver.py runs in a fresh process with that build and
checks, for each case, the reported status (TEC_ETIMEOUT = 4 for a cap that
ran out, TEC_ENOMEM = 2 for a refused buffer), that the same graph answers
the next call with the oracle's results, that the fallbacks (sweep without
its live-edge list, triangle counts without core staging or tiling) match
the oracle, and that no buffer was written past its end (canaries).
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_capped_loops_and_refused_allocations_recover(cuda_device, tmp_path):
    from paper_2412_12382_gb300 import build as libbuild
    lib, _ = libbuild.compile_library(libbuild.CSRC, str(tmp_path / "debug"), defines=("TEC_DEBUG",))
    env = dict(os.environ, TEC_LIBRARY=lib)
    for k in ("TEC_DEBUG_LINK_CAP", "TEC_DEBUG_MSF_ROUNDS", "TEC_DEBUG_FAIL_ALLOC"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "failure_driver.py")], capture_output=True,
                       text=True, env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    print(out)
    assert out["link_cap_status"] == 4 and out["link_cap_recall_ok"]
    assert out["msf_rounds_status"] == 4 and out["msf_rounds_recall_ok"]
    for name in ("live edge", "core", "tiling"):
        assert out[f"fail_alloc_{name}_ok"], name
    assert out["lazy_alloc_status"] == 2 and out["lazy_alloc_retry_ok"]
    assert out["canaries_status"] == 0
