"""Device-side R-MAT generator: the same graphs as ``rmat.rmat_csr``, built on
the GPU for sizes the host generator cannot reach in reasonable time
(scale 20+).  Sampling runs in ``gen_kernels.cu``; deduplication and sorting
use torch.unique, one bucket range of source ids at a time.  This is input
preparation only."""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

from .prng import STREAM_RMAT, stream_key
from .rmat import cut_points, feistel_keys

HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def library_path() -> str:
    return os.path.join(HERE, "_build", "libgraphgen.so")


def build(force: bool = False) -> str:
    out = library_path()
    src = os.path.join(HERE, "gen_kernels.cu")
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    nvcc = next((c for c in ("/usr/local/cuda/bin/nvcc", shutil.which("nvcc")) if c and os.path.exists(c)), None)
    if nvcc is None:
        raise RuntimeError("nvcc not found")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run([nvcc, "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-gencode",
                    "arch=compute_103a,code=sm_103a", src, "-o", tmp], check=True)
    os.replace(tmp, out)
    return out


def _load():
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            build()
        lib = ctypes.CDLL(path)
        u32, u64, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        P = ctypes.c_void_p
        lib.gg_rmat_count.argtypes = [i32, u64, u32, u32, u32, u64, P, i32, P, P]
        lib.gg_rmat_emit.argtypes = [i32, u64, u32, u32, u32, u64, P, i32, i32, i32, P, P, ctypes.c_longlong, P]
        lib.gg_rmat_count.restype = i32
        lib.gg_rmat_emit.restype = i32
        _lib = lib
    return _lib


def rmat_csr_gpu(scale: int, edge_factor: int, abc=(0.57, 0.19, 0.19), seed: int = 2,
                 max_group: int = 1 << 30, bucket_bits: int | None = None):
    """Cleaned symmetric CSR (off int64 [n+1], col int32 [2m]) as CUDA tensors."""
    import torch
    lib = _load()
    dev = torch.device("cuda")
    n = 1 << scale
    nsamples = edge_factor << scale
    A, AB, ABC = cut_points(*abc)
    key = stream_key(seed, STREAM_RMAT)
    fk = (ctypes.c_uint64 * 4)(*feistel_keys(seed))
    bb = min(scale, 10) if bucket_bits is None else bucket_bits
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    counts = torch.zeros(1 << bb, dtype=torch.int64, device=dev)
    rc = lib.gg_rmat_count(scale, nsamples, A, AB, ABC, key, fk, bb, ctypes.c_void_p(counts.data_ptr()), stream)
    if rc:
        raise RuntimeError(f"gg_rmat_count failed ({rc})")
    counts = counts.cpu().tolist()
    groups, b0, acc = [], 0, 0
    for b, c in enumerate(counts):
        if acc and acc + c > max_group:
            groups.append((b0, b, acc))
            b0, acc = b, 0
        acc += c
    groups.append((b0, len(counts), acc))
    cap = max(g[2] for g in groups)
    buf = torch.empty(max(cap, 1), dtype=torch.int64, device=dev)
    cursor = torch.zeros(1, dtype=torch.int64, device=dev)
    shift = scale - bb
    deg = torch.zeros(n, dtype=torch.int64, device=dev)
    parts = []
    mask = (1 << 32) - 1
    for g0, g1, cnt in groups:
        if cnt == 0:
            continue
        cursor.zero_()
        rc = lib.gg_rmat_emit(scale, nsamples, A, AB, ABC, key, fk, bb, g0, g1, ctypes.c_void_p(buf.data_ptr()),
                              ctypes.c_void_p(cursor.data_ptr()), cap, stream)
        if rc:
            raise RuntimeError(f"gg_rmat_emit failed ({rc})")
        keys = torch.unique(buf[:cnt])
        src = keys >> 32
        v0, v1 = g0 << shift, g1 << shift
        deg[v0:v1] = torch.bincount(src - v0, minlength=v1 - v0)
        parts.append((keys & mask).to(torch.int32))
        del keys, src
    del buf
    col = torch.cat(parts) if parts else torch.zeros(0, dtype=torch.int32, device=dev)
    del parts
    off = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    torch.cumsum(deg, 0, out=off[1:])
    return off, col
