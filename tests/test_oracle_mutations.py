"""Planted mistakes in the oracle, each caught by the oracle's pins.

Every case changes one place of the oracle's source: a dropped term, a
flipped comparison, a wrong sign, index or operand.  The changed copy is
built (C: a temporary shared library; Python: a fresh module), swapped in for
the real oracle, and the pin tests of test_oracle_pins.py,
test_oracle_rules.py and test_oracle_mlp.py run against it.  Each mutant must
fail at least one pin.  The real oracle passes the same pins, unmodified,
elsewhere in the suite.  Nothing here touches a GPU.
"""
import importlib.util
import os
import shutil
import subprocess
import sys
import types

import pytest

import oracle
from oracle import mlp as oracle_mlp
from oracle import reference

wedges_real, forward_real = reference.wedges, oracle_mlp.forward

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE_DIR = os.path.dirname(os.path.abspath(reference.__file__))
PIN_FILES = ["test_oracle_pins.py", "test_oracle_rules.py", "test_oracle_mlp.py"]

# (where, text in the oracle, planted mistake, what the mistake is)
C_MUTANTS = [
    ("else { ++common; ++i; ++j; }", "else { ++common; ++i; }",
     "merge forgets to advance the second row on a common neighbour"),
    ("all += (uint64_t)(iend - i) + (uint64_t)(jend - j);", "all += (uint64_t)(iend - i);",
     "union drops the tail of the second row"),
    ("k = t * q >= (__int128)p * (du + dv);", "k = t * q > (__int128)p * (du + dv);",
     "Tectonic prune removes edges exactly at the threshold"),
    ("__int128 wedge = (__int128)uni[e] - t - 2;", "__int128 wedge = (__int128)uni[e] - t;",
     "TW wedge keeps u and v in the union"),
    ("k = (t - wedge) * q >= (__int128)p;", "k = (wedge - t) * q >= (__int128)p;",
     "TW with the sign of t - wedge flipped"),
    ("k = t * q >= (__int128)p * (__int128)uni[e];", "k = t * q >= (__int128)p * (__int128)(uni[e] - t);",
     "Jaccard denominator without the common neighbours"),
    ("k = t * q >= (__int128)p;", "k = t >= (__int128)p;",
     "K3 prune ignores the denominator q"),
    ("for (int64_t s = 0; s < n; ++s) {", "for (int64_t s = n - 1; s >= 0; --s) {",
     "components labelled by their largest vertex id"),
    ("int64_t x = off[c], xend = off[c + 1], y = a + 1;", "int64_t x = off[c], xend = off[c + 1], y = 0;",
     "K4 counts every inner edge of C twice"),
    ("++hits;                                               /* a -> b */", "/* a -> b dropped */",
     "forward listing never credits the edge a -> b"),
    ("__atomic_fetch_add(&rt[k], 1u, __ATOMIC_RELAXED);     /* b -> c */",
     "__atomic_fetch_add(&rt[j], 1u, __ATOMIC_RELAXED);     /* b -> c */",
     "forward listing credits b -> c to a -> b"),
    ("acc[j - ab] += hits;", "acc[j - ab] = hits;",
     "forward listing overwrites the a -> c credits of an edge with its a -> b hits"),
]

PY_MUTANTS = [
    ("return np.asarray(uni, dtype=np.int64) - np.asarray(t, dtype=np.int64) - 2",
     "return np.asarray(uni, dtype=np.int64) - np.asarray(t, dtype=np.int64)",
     "wedge keeps u and v in the union"),
    ("return np.asarray(t, dtype=np.int64) - np.asarray(wedge, dtype=np.int64)",
     "return np.asarray(t, dtype=np.int64) + np.asarray(wedge, dtype=np.int64)",
     "TW adds the wedges"),
    ("s = (d[np.asarray(eu)] + d[np.asarray(ev)]).astype(np.float64)",
     "s = (d[np.asarray(eu)] + d[np.asarray(ev)] - np.asarray(t)).astype(np.float64)",
     "Tectonic weight with the Jaccard denominator"),
    ("return np.asarray(t, dtype=np.float64) / np.asarray(uni, dtype=np.float64)",
     "return np.asarray(t, dtype=np.float64) / (np.asarray(uni, dtype=np.float64) - np.asarray(t))",
     "Jaccard weight without the common neighbours in the denominator"),
    ("return float((Fraction(sij) - expected) / denom)", "return float(Fraction(sij) / denom)",
     "ARI numerator without the expected index"),
    ("denom = Fraction(sa + sb, 2) - expected", "denom = Fraction(sa + sb, 2)",
     "ARI denominator without the expected index"),
    ("return float(np.sum(intra / two_m - (D / two_m) ** 2))",
     "return float(np.sum(intra / two_m - (D / (2 * two_m)) ** 2))",
     "modularity with 4m in the degree term"),
    ("p, r = inter / size, inter / csize", "p, r = inter / size, inter / size",
     "recall divided by the found community's size"),
    ("if best is None or j > best[0]:", "if best is None or j >= best[0]:",
     "Jaccard ties go to the highest block id"),
    ("num_p += p * size", "num_p += p",
     "precision not weighted by community size"),
    ("b = np.minimum((128 * np.asarray(t, dtype=np.int64)) // s, 63)",
     "b = np.minimum((64 * np.asarray(t, dtype=np.int64)) // s, 63)",
     "histogram on the grid i/64"),
    ("return np.concatenate([h / m, [math.log(2.0 * m / n), math.log(m)]])",
     "return np.concatenate([h / m, [math.log(m / n), math.log(m)]])",
     "mean-degree feature without the factor 2"),
    ("qmod = float(Fraction(4 * m * intra - sum_vol2, 4 * m * m)) if m else 0.0",
     "qmod = float(Fraction(2 * m * intra - sum_vol2, 4 * m * m)) if m else 0.0",
     "sweep modularity with 2m in the intra term"),
    ("intra = int(np.count_nonzero(lab[eu] == lab[ev]))", "intra = int(np.count_nonzero(lab[eu] != lab[ev]))",
     "intra counts the edges between components"),
    ("best, best_jump = order[j + 1], jump", "best, best_jump = order[j], jump",
     "R1 picks the threshold just below the jump"),
    ("if modularity[i] > modularity[best]:", "if modularity[i] >= modularity[best]:",
     "R2 ties go to the highest threshold"),
    ("for i, (p, q) in enumerate(zip(ps, qs)):\n        keep, _ = prune(measure, off, eu, ev, t, uni, p, q, k4)",
     "for i, (p, q) in enumerate(zip(list(ps[1:]) + list(ps[:1]), qs)):\n"
     "        keep, _ = prune(measure, off, eu, ev, t, uni, p, q, k4)",
     "sweep level i uses threshold i + 1"),
]

MLP_MUTANTS = [
    ('dz1 = (dz2 @ p["W2"]) * (z1 > 0)', 'dz1 = (dz2 @ p["W2"].T) * (z1 > 0)',
     "backpropagation through W2 with the operand transposed"),
    ('g["W2"] = dz2.T @ h1', 'g["W2"] = h1.T @ dz2',
     "W2 gradient transposed"),
    ("dy = 2.0 * (y - np.asarray(target, dtype=np.float64)) / n",
     "dy = (y - np.asarray(target, dtype=np.float64)) / n",
     "loss gradient without the factor 2"),
    ("mhat = m / (1 - beta1 ** step)", "mhat = m",
     "Adam without the first-moment bias correction"),
    ("dval = 64.0 / (sigma * sigma) * ((w * L * d).sum(axis=1) - val * (w * d).sum(axis=1))",
     "dval = 64.0 / (sigma * sigma) * (w * L * d).sum(axis=1)",
     "soft-level loss derivative without the normalisation term"),
    ("d = i[None, :] - 64.0 * y[:, None]", "d = i[None, :] - 63.0 * y[:, None]",
     "soft-level loss centred on 63 y instead of 64 y"),
]


def _mutate(path, old, new):
    src = open(path).read()
    assert src.count(old) == 1, f"{os.path.basename(path)} no longer holds exactly one {old!r}"
    return src.replace(old, new)


def _pin_cases():
    """(name, callable) for every pin test; parametrized ones once per value."""
    cases = []
    for fname in PIN_FILES:
        spec = importlib.util.spec_from_file_location("_pins_" + fname[:-3], os.path.join(HERE, fname))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        for name, fn in vars(mod).items():
            if not name.startswith("test_") or not callable(fn):
                continue
            marks = [mk for mk in getattr(fn, "pytestmark", []) if mk.name == "parametrize"]
            if not marks:
                if fn.__code__.co_argcount == 0:
                    cases.append((f"{fname}::{name}", fn))
                continue
            argnames = [a.strip() for a in marks[0].args[0].split(",")]
            for values in marks[0].args[1]:
                values = values if len(argnames) > 1 else (values,)
                cases.append((f"{fname}::{name}{list(values)}",
                              (lambda f=fn, kw=dict(zip(argnames, values)): f(**kw))))
    return cases


def _first_failing_pin():
    for name, call in _pin_cases():
        try:
            call()
        except pytest.skip.Exception:
            continue
        except Exception:                        # an assertion, or the mutant broke outright
            return name
    return None


def _install_module(monkeypatch, target, path, source):
    """Executes `source` as a fresh copy of the module at `path` and swaps its
    functions and constants into `target` (and into the oracle package)."""
    mod = types.ModuleType(target.__name__ + "_mutant")
    mod.__file__ = path
    mod.__package__ = "oracle"
    monkeypatch.setitem(sys.modules, mod.__name__, mod)     # dataclasses look their module up
    exec(compile(source, path, "exec"), mod.__dict__)
    for name, value in vars(mod).items():
        if name.startswith("__") or isinstance(value, types.ModuleType):
            continue
        if hasattr(target, name):
            monkeypatch.setattr(target, name, value)
        if target is reference and hasattr(oracle, name):
            monkeypatch.setattr(oracle, name, value)


def test_pins_pass_on_the_real_oracle():
    assert _first_failing_pin() is None


def _use_c_library(monkeypatch, tmp_path, source):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "oracle_variant.c"
    src.write_text(source)
    so = str(tmp_path / "liboracle_variant.so")
    subprocess.run([gcc, "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", str(src), "-o", so], check=True)
    monkeypatch.setattr(reference, "library_path", lambda: so)
    monkeypatch.setattr(reference, "_lib", None)
    return so


def test_control_unchanged_c_copy_passes(monkeypatch, tmp_path):
    """Control: the C part rebuilt from an unchanged copy and swapped in the
    way the C mutants are passes every pin, and is the library the pins used."""
    so = _use_c_library(monkeypatch, tmp_path, open(os.path.join(ORACLE_DIR, "oracle.c")).read())
    assert _first_failing_pin() is None
    assert reference._lib is not None and reference._lib._name == so


def test_control_unchanged_python_copies_pass(monkeypatch):
    """Control: unchanged copies of both Python modules, swapped in the way
    the Python mutants are, pass every pin."""
    for target in (reference, oracle_mlp):
        _install_module(monkeypatch, target, target.__file__, open(target.__file__).read())
    assert oracle.wedges is not wedges_real and oracle_mlp.forward is not forward_real
    assert _first_failing_pin() is None


@pytest.mark.parametrize("old,new,what", C_MUTANTS, ids=[w for _, _, w in C_MUTANTS])
def test_c_mutant_is_caught(monkeypatch, tmp_path, old, new, what):
    _use_c_library(monkeypatch, tmp_path, _mutate(os.path.join(ORACLE_DIR, "oracle.c"), old, new))
    assert _first_failing_pin() is not None, f"no pin catches: {what}"


@pytest.mark.parametrize("old,new,what", PY_MUTANTS, ids=[w for _, _, w in PY_MUTANTS])
def test_python_mutant_is_caught(monkeypatch, old, new, what):
    path = reference.__file__
    _install_module(monkeypatch, reference, path, _mutate(path, old, new))
    assert _first_failing_pin() is not None, f"no pin catches: {what}"


@pytest.mark.parametrize("old,new,what", MLP_MUTANTS, ids=[w for _, _, w in MLP_MUTANTS])
def test_mlp_mutant_is_caught(monkeypatch, old, new, what):
    path = oracle_mlp.__file__
    _install_module(monkeypatch, oracle_mlp, path, _mutate(path, old, new))
    assert _first_failing_pin() is not None, f"no pin catches: {what}"
