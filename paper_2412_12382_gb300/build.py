"""Builds libtectonic.so (the C-ABI library) from csrc/*.cu for sm_103a.

Each translation unit is compiled in parallel with nvcc, then linked into one
shared library (CUDA runtime linked statically) under ``_build/``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr"] + ARCH


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def default_library_path() -> str:
    """The in-tree build that build() writes."""
    return os.path.join(BUILD, "libtectonic.so")


def library_path() -> str:
    """The library the binding loads: $TEC_LIBRARY when set (a variant built
    by the autotuner), else the in-tree build."""
    return os.environ.get("TEC_LIBRARY") or default_library_path()


def _sources(csrc: str = CSRC):
    return sorted(glob.glob(os.path.join(csrc, "*.cu")))


def _deps():
    return _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))) + [
        os.path.join(os.path.dirname(HERE), "include", "tectonic.h")]


def up_to_date() -> bool:
    lib = default_library_path()
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def compile_library(csrc: str, build_dir: str, ptxas_info: bool = False, defines=()):
    """Compiles every .cu of `csrc` in parallel and links build_dir/libtectonic.so.
    `defines`: extra preprocessor names (e.g. TEC_DEBUG).  Returns (library
    path, {source name: compiler diagnostics})."""
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + [f"-D{d}" for d in defines]

    def compile_one(src):
        obj = os.path.join(build_dir, os.path.basename(src).replace(".cu", ".o"))
        cmd = [cc] + NVCC_FLAGS + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(compile_one, _sources(csrc)))
    lib = os.path.join(build_dir, "libtectonic.so")
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, "-shared", "-o", tmp] + [o for o, _ in results] + ARCH
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib, {os.path.basename(o).replace(".o", ".cu"): err for o, err in results}


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and up_to_date():
        return default_library_path()
    lib, diags = compile_library(CSRC, BUILD, ptxas_info)
    if verbose or ptxas_info:
        for name, err in diags.items():
            if err.strip():
                print(f"--- {name}\n{err}")
    return lib


DEBUG_BUILD = os.path.join(HERE, "_build_debug")


def build_debug() -> str:
    """The debug library (-DTEC_DEBUG: canary bytes after every graph-owned
    device buffer, checked by tec_sync) in _build_debug/; load it by setting
    TEC_LIBRARY to the returned path."""
    lib, _ = compile_library(CSRC, DEBUG_BUILD, defines=("TEC_DEBUG",))
    return lib


if __name__ == "__main__":
    import sys
    if "--debug" in sys.argv:
        print(build_debug())
    else:
        print(build(force=True, verbose=True, ptxas_info="-v" in sys.argv))
