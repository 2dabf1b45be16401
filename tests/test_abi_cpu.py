"""C-ABI library checks that need no GPU: it loads, exports every symbol the
public header declares, and the binding refuses to run without a GPU."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2412_12382_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tectonic.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tec_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    path = libbuild.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("tec_graph_upload", "tec_edge_support", "tec_edge_weights", "tec_prune",
              "tec_components", "tec_full_pass", "tec_full_pass_host"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_version_and_error_buffer(lib):
    lib.tec_version.restype = ctypes.c_int
    assert lib.tec_version() == 100
    lib.tec_last_error.restype = ctypes.c_size_t
    lib.tec_last_error.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    assert lib.tec_last_error(None, 0) >= 0


def test_null_arguments_rejected_without_touching_a_device(lib):
    from paper_2412_12382_gb300 import tectonic as T
    L = T.load_library()
    assert L.tec_graph_free(None) == 0
    assert L.tec_graph_info(None, None, None) == 1          # TEC_EINVAL
    assert L.tec_prune(None, 0, 1, 10, None, None) == 1
    assert L.tec_graph_create(-1, 0, None, None) == 1
    # the later entry points check their arguments before any device call
    assert L.tec_sweep(None, 0, None, None, 64, None, 0, None, None) == 1
    assert L.tec_sweep_stats(None, 0, None, None, 64, None, None, 0, None) == 1
    assert L.tec_rule_of_thumb(None, None, None, 0, 1, 0, None, None) == 1       # k < 1
    assert L.tec_rule_of_thumb(None, None, None, 200, 1, 0, None, None) == 1     # k > 127
    assert L.tec_edge_k4(None, None) == 1
    assert L.tec_prf(None, 1, None, None, None, 0, None) == 1
    assert L.tec_ari(None, 1, None, None, None, 0, None) == 1
    assert L.tec_features(None, None, 0, None) == 1
    assert L.tec_pick_threshold(None, None, None, 0, 1, None, None) == 1
    assert L.tec_set_core_staging(None, 1) == 1
    assert L.tec_prune_components_batch(None, 0, None, None, None, 0, None, None) == 1
    assert L.tec_picker_thresholds(None, -1, None, None, None) == 1
    assert L.tec_set_support_tiling(None, 0) == 1
    assert L.tec_picker_file_write(None, None, None, None, 0, None) == 1
    assert L.tec_picker_file_read(None, None, None, None, None, None, 0, None) == 1
    assert L.tec_picker_save(None, b"x", None) == 1
    assert L.tec_picker_load(None, None, None) == 1
    assert L.tec_picker_train_soft(None, None, None, None, 0, 1, 1, 1e-3, 0, 1.0, 0.5, None) == 1
    assert L.tec_picker_soft_loss_grad(None, None, None, None, 0, 1.0, 0.5, None, None) == 1


def test_binding_fails_loudly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2412_12382_gb300 import Graph
    with pytest.raises(RuntimeError):
        Graph(n_cap=4, nnz_cap=8)


def test_c_client_compiles_links_and_runs(lib, tmp_path):
    """The header is plain C11 (-pedantic -Werror) and a C program linked
    against the library gets the documented statuses without a device."""
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(libbuild.library_path())
    exe = str(tmp_path / "abi_smoke")
    src = os.path.join(ROOT, "tests", "abi_c", "abi_smoke.c")
    cmd = [gcc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
           src, "-o", exe, "-L", libdir, "-ltectonic", f"-Wl,-rpath,{libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_debug_build_compiles_and_answers_from_c(tmp_path):
    """The -DTEC_DEBUG library (canaries after every graph-owned buffer)
    builds, exports the same symbols, and a C client linked to it gets the
    same statuses without a device."""
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib_path, _ = libbuild.compile_library(libbuild.CSRC, str(tmp_path / "dbg"), defines=("TEC_DEBUG",))
    dbg = ctypes.CDLL(lib_path)
    missing = [s for s in declared_symbols() if not hasattr(dbg, s)]
    assert not missing, missing
    exe = str(tmp_path / "abi_smoke_dbg")
    src = os.path.join(ROOT, "tests", "abi_c", "abi_smoke.c")
    libdir = os.path.dirname(lib_path)
    r = subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe, "-L", libdir,
                        "-ltectonic", f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_sweep_offer_key_round_trip(tmp_path):
    """The sweep's packed offer key keeps every edge index a graph can hold
    (m < 2^40, beyond 2^32) and orders offers by (level, -edge index)."""
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "key.cc"
    src.write_text(r'''
#include <stdio.h>
#include "msf_key.h"
using namespace tec;
int main() {
    const int64_t js[] = {0, 1, 12345, (1ll << 32) - 1, 1ll << 32, (1ll << 32) + 1, (1ll << 39) - 1, (1ll << 40) - 1};
    for (int L = 1; L <= 127; ++L)
        for (int64_t j : js) {
            const uint64_t k = msf_key_pack((uint8_t)L, j);
            if (k == 0 || msf_key_edge(k) != j || msf_key_level(k) != L) { printf("bad %d %lld\n", L, (long long)j); return 1; }
            if (msf_key_pack((uint8_t)L, j + 1) >= k) { printf("order j %lld\n", (long long)j); return 1; }
            if (L < 127 && msf_key_pack((uint8_t)(L + 1), (1ll << 40) - 1) <= k) { printf("order L\n"); return 1; }
        }
    /* two edges 2^32 apart get distinct keys (a 32-bit field would merge them) */
    if (msf_key_pack(5, 7) == msf_key_pack(5, 7 + (1ll << 32))) { printf("collision\n"); return 1; }
    printf("ok\n");
    return 0;
}
''')
    exe = str(tmp_path / "key")
    r = subprocess.run([gxx, "-std=c++17", "-Wall", "-Werror", "-I", os.path.join(ROOT, "paper_2412_12382_gb300", "csrc"),
                        str(src), "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=30)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
