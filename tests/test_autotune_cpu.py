"""Host side of the autotuner: constant substitution, the current values of
every tunable, the spill filter, metric reading, the search and its cache,
and one variant built with nvcc.  No GPU: the timing step is replaced."""
import json
import os
import shutil

import pytest

from paper_2412_12382_gb300 import autotune as A
from paper_2412_12382_gb300 import build as B


def test_every_tunable_has_one_definition_and_safe_candidates():
    for name, (fname, cands) in A.TUNABLES.items():
        text = open(os.path.join(B.CSRC, fname)).read()
        v = A.int_value(A.current_value(text, name))
        if name == "CORE_ORDER":                       # a choice of order, 0..2
            assert v in (0, 1, 2) and set(cands) <= {0, 1, 2}
            continue
        if name == "ORIENT_GATHER_CG" or name.endswith("_PERSISTENT"):  # a switch
            assert v in (0, 1) and set(cands) == {0, 1}
            continue
        assert v > 0 and all(c > 0 for c in cands)
        if name in ("C_BATCH", "B_BATCH", "T_BATCH"):  # one candidate per lane of a warp
            assert max(cands) <= 32 and v <= 32


def test_substitute_changes_only_its_constant():
    text = "constexpr int A = 4;   // a\nconstexpr int64_t B = 1 << 25;\nconstexpr int AB = 7;\n"
    out = A.substitute(text, "A", 12)
    assert "constexpr int A = 12;   // a" in out and "constexpr int AB = 7;" in out
    out = A.substitute(text, "B", 1 << 23)
    assert A.int_value(A.current_value(out, "B")) == 1 << 23
    with pytest.raises(ValueError):
        A.substitute(text, "C", 1)
    with pytest.raises(ValueError):
        A.substitute(text + "constexpr int A = 5;\n", "A", 1)      # two definitions
    assert A.int_value(" 1 << 20 ") == 1 << 20 and A.int_value("64") == 64
    with pytest.raises(ValueError):
        A.int_value("W_MAX * 2")


def test_spill_filter_compares_with_the_baseline():
    clean = "ptxas info    : Function properties for k\n    0 bytes stack frame, 0 bytes spill stores, 0 bytes spill loads"
    dirty = clean + "\n    8 bytes stack frame, 8 bytes spill stores, 8 bytes spill loads"
    worse = dirty + "\n    16 bytes stack frame, 16 bytes spill stores, 8 bytes spill loads"
    base = A.spill_bytes({"a.cu": clean, "b.cu": dirty})
    assert base == {"a.cu": 0, "b.cu": 16}
    assert A.spills_worse(base, base) == []                      # existing spills are accepted
    assert A.spills_worse(A.spill_bytes({"a.cu": dirty, "b.cu": worse}), base) == ["a.cu", "b.cu"]


def test_read_metric_takes_the_last_json_line():
    out = 'log line\n{"x": {"y": 1.5}}\nmore\n{"x": {"y": 2.5}, "z": 3}\n'
    assert A.read_metric(out, "x.y") == 2.5 and A.read_metric(out, "z") == 3.0
    with pytest.raises(ValueError):
        A.read_metric("no json here", "x")


def test_coordinate_descent_finds_a_separable_optimum_and_skips_invalid_points():
    space = {"a": [1, 2, 4, 8, 16], "b": [4, 8, 12, 16], "c": [0, 1]}
    calls = []

    def cost(p):
        calls.append(dict(p))
        if p["c"] == 1 and p["a"] == 16:
            return None                               # a point that cannot run
        return (p["a"] - 4) ** 2 + (p["b"] - 12) ** 2 + 0.5 * p["c"]

    best, c, seen = A.coordinate_descent(space, {"a": 16, "b": 4, "c": 1}, cost)
    assert best == {"a": 4, "b": 12, "c": 0} and c == 0
    assert len(calls) == len(seen)                    # every point evaluated once
    best, c, _ = A.coordinate_descent(space, {"a": 4, "b": 12, "c": 0}, lambda p: -cost(p) if cost(p) is not None else None,
                                      lower_is_better=False)
    assert c == 0 and best == {"a": 4, "b": 12, "c": 0}


def test_tune_uses_and_fills_its_cache(tmp_path, monkeypatch):
    built = []

    def fake_build(point, root):
        built.append(dict(point))
        return "lib.so", {"support.cu": 0}

    monkeypatch.setattr(A, "build_variant", fake_build)
    monkeypatch.setattr(A, "time_variant", lambda lib, cmd, metric, reps, cwd: float(abs(built[-1]["C_BATCH"] - 12)))
    cache = str(tmp_path / "cache.json")
    start, best, cost, entries = A.tune(["C_BATCH"], "cmd", "m", reps=1, cache_path=cache, log=lambda *a: None)
    assert start == {"C_BATCH": A.int_value(A.current_value(open(os.path.join(B.CSRC, "support.cu")).read(), "C_BATCH"))}
    assert best == {"C_BATCH": 12} and cost == 0.0
    n_built = len(built)
    assert n_built == len(entries) + 1 and json.load(open(cache))    # + the baseline build
    A.tune(["C_BATCH"], "cmd", "m", reps=1, cache_path=cache, log=lambda *a: None)
    assert len(built) == n_built + 1                  # only the baseline is rebuilt; points come from the cache


def test_a_variant_builds_with_nvcc(tmp_path):
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no nvcc")
    _, base = A.build_variant({}, str(tmp_path / "base"))
    lib, spilled = A.build_variant({"C_BATCH": 12, "K4_GRAB": 2}, str(tmp_path))
    assert os.path.exists(lib) and A.spills_worse(spilled, base) == []
    src = open(os.path.join(str(tmp_path), "pkg", "csrc", "support.cu")).read()
    assert A.int_value(A.current_value(src, "C_BATCH")) == 12
    assert A.int_value(A.current_value(open(os.path.join(B.CSRC, "support.cu")).read(), "C_BATCH")) != 12


def test_a_variant_failing_its_check_is_not_timed(tmp_path, monkeypatch):
    monkeypatch.setattr(A, "build_variant", lambda point, root: ("lib.so", {}))
    monkeypatch.setattr(A, "check_variant", lambda lib, cmd, cwd: False)
    timed = []
    monkeypatch.setattr(A, "time_variant", lambda *a: timed.append(a) or 1.0)
    start, best, cost, entries = A.tune(["K4_GRAB"], "cmd", "m", reps=1, log=lambda *a: None, check_cmd="check")
    assert timed == [] and cost is None and all(v is None for v in entries.values())


def test_library_override_is_only_for_loading(monkeypatch):
    monkeypatch.setenv("TEC_LIBRARY", "/nonexistent/variant.so")
    assert B.library_path() == "/nonexistent/variant.so"
    assert B.default_library_path().endswith(os.path.join("_build", "libtectonic.so"))


def test_descent_ignores_gains_within_noise():
    # a 0.1% better neighbour does not move the constants at min_gain = 0.5%, a 2% better one does
    costs = {(16, 16): 100.0, (12, 16): 99.9, (16, 12): 100.05, (12, 12): 99.9}
    space = {"A": [12, 16], "B": [12, 16]}
    ev = lambda p: costs[(p["A"], p["B"])]
    best, cost, _ = A.coordinate_descent(space, {"A": 16, "B": 16}, ev, min_gain=0.005)
    assert best == {"A": 16, "B": 16} and cost == 100.0
    costs[(12, 16)] = 98.0
    best, cost, _ = A.coordinate_descent(space, {"A": 16, "B": 16}, ev, min_gain=0.005)
    assert best["A"] == 12 and cost == 98.0


def test_shipped_cache_records_the_gpu_run():
    """The committed cache holds the scale-26 run on a GB300: every point of
    the descent with its triangle-stage time, keyed by device and size class."""
    path = os.path.join(os.path.dirname(A.__file__), "autotune_cache.json")
    cache = json.load(open(path))
    keys = [json.loads(k) for k in cache]
    k26 = [k for k in keys if k.get("size_class") == "rmat26"]
    assert k26 and k26[0]["device"] == "NVIDIA GB300" and k26[0]["metric"] == "config.stage_ms.support"
    entries = cache[json.dumps(k26[0])] if json.dumps(k26[0]) in cache else next(iter(cache.values()))
    times = [v for v in entries.values() if v is not None]
    assert len(times) >= 9 and min(times) > 0
