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

import numpy as np

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
        i64 = ctypes.c_int64
        lib.gg_dcsbm.argtypes = [u64, i64, i32, i32, u64, P, P, P, P, ctypes.c_longlong, P, P]
        lib.gg_dcsbm.restype = i32
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


def dcsbm_batch_gpu(seeds, n_lo: int = 1000, n_hi: int = 100000):
    """A batch of DC-SBM graphs (graphgen.dcsbm definition) as one disjoint
    union, built on the GPU.  Returns CUDA tensors (off int64, col int32,
    seg_off int64, truth int32 block ids) and the host specs."""
    import torch
    from .dcsbm import dcsbm_spec
    from .prng import STREAM_DCSBM, stream_key
    lib = _load()
    dev = torch.device("cuda")
    specs = [dcsbm_spec(s, n_lo, n_hi) for s in seeds]
    seg = [0]
    for sp in specs:
        seg.append(seg[-1] + sp.n)
    N = seg[-1]
    total = sum(sp.samples for sp in specs)
    keys = torch.empty(2 * total, dtype=torch.int64, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    at = 0
    keep = []
    for sp, voff in zip(specs, seg[:-1]):
        arrs = [torch.from_numpy(a).to(dev) for a in (sp.block, sp.order, sp.cum, sp.bstart)]
        keep.append(arrs)
        rc = lib.gg_dcsbm(stream_key(sp.seed, STREAM_DCSBM + 3), sp.samples, sp.n, sp.k, sp.mu_cut,
                          ctypes.c_void_p(arrs[0].data_ptr()), ctypes.c_void_p(arrs[1].data_ptr()),
                          ctypes.c_void_p(arrs[2].data_ptr()), ctypes.c_void_p(arrs[3].data_ptr()), voff,
                          ctypes.c_void_p(keys[2 * at].data_ptr()), stream)
        if rc:
            raise RuntimeError(f"gg_dcsbm failed ({rc})")
        at += sp.samples
    keys = torch.unique(keys[keys >= 0])
    src = keys >> 32
    col = (keys & ((1 << 32) - 1)).to(torch.int32)
    off = torch.zeros(N + 1, dtype=torch.int64, device=dev)
    torch.cumsum(torch.bincount(src, minlength=N), 0, out=off[1:])
    truth = torch.from_numpy(np.concatenate([sp.block for sp in specs]).astype(np.int32)).to(dev)
    seg_off = torch.tensor(seg, dtype=torch.int64, device=dev)
    torch.cuda.synchronize()
    del keep
    return off, col, seg_off, truth, specs
