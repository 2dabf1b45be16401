"""Python binding of the C ABI in include/tectonic.h (argument marshalling only).

Every computation runs in the CUDA kernels of ``libtectonic.so``; this module
only allocates output tensors with PyTorch, passes raw pointers and raises on
a non-zero status.  There is no fallback: if the library is missing or no GPU
is present, calls fail loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

TECTONIC = 0
TW = 1
JACCARD = 2
K3 = 3
K4 = 4
HOST_PTR = 0x1
VALIDATE = 0x2

STATUS_NAMES = {0: "TEC_OK", 1: "TEC_EINVAL", 2: "TEC_ENOMEM", 3: "TEC_ECUDA", 4: "TEC_ETIMEOUT",
                5: "TEC_EOVERFLOW", 6: "TEC_EBADGRAPH", 7: "TEC_ESTATE"}


class TectonicError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_PI64 = ctypes.POINTER(ctypes.c_int64)

SIGNATURES = {
    "tec_version": ([], ctypes.c_int),
    "tec_last_error": ([ctypes.c_char_p, ctypes.c_size_t], ctypes.c_size_t),
    "tec_graph_create": ([_I64, _I64, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "tec_graph_load": ([_P, _P, ctypes.c_int, _P, _I64, _I64, ctypes.c_uint32], ctypes.c_int),
    "tec_graph_upload": ([_P, ctypes.c_int, _P, _I64, _I64, ctypes.c_uint32, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "tec_graph_free": ([_P], ctypes.c_int),
    "tec_graph_info": ([_P, _PI64, _PI64], ctypes.c_int),
    "tec_sync": ([_P], ctypes.c_int),
    "tec_orient": ([_P], ctypes.c_int),
    "tec_support": ([_P], ctypes.c_int),
    "tec_edge_list": ([_P, _P, _P], ctypes.c_int),
    "tec_edge_support": ([_P, _P, _P], ctypes.c_int),
    "tec_edge_weights": ([_P, ctypes.c_int, _P], ctypes.c_int),
    "tec_prune": ([_P, ctypes.c_int, _I64, _I64, _P, _PI64], ctypes.c_int),
    "tec_components": ([_P, _P, _PI64], ctypes.c_int),
    "tec_full_pass": ([_P, ctypes.c_int, _I64, _I64, _P, _PI64], ctypes.c_int),
    "tec_full_pass_host": ([_P, _P, _P, _I64, _I64, ctypes.c_int, _I64, _I64, _P, _PI64], ctypes.c_int),
    "tec_oriented_csr": ([_P, _P, _P], ctypes.c_int),
    "tec_launch_count": ([], ctypes.c_longlong),
    "tec_set_stage_events": ([_P, ctypes.POINTER(_P), ctypes.c_int], ctypes.c_int),
    "tec_sweep": ([_P, ctypes.c_int, _P, _P, ctypes.c_int, _P, ctypes.c_int, _P, _P], ctypes.c_int),
    "tec_features": ([_P, _P, ctypes.c_int, _P], ctypes.c_int),
    "tec_ari": ([_P, ctypes.c_int, _P, _P, _P, ctypes.c_int, _P], ctypes.c_int),
    "tec_ari_best": ([_P, ctypes.c_int, ctypes.c_int, _P, _P, _P], ctypes.c_int),
    "tec_prune_components_batch": ([_P, ctypes.c_int, _P, _P, _P, ctypes.c_int, _P, _P], ctypes.c_int),
    "tec_picker_create": ([_P, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "tec_picker_free": ([_P], ctypes.c_int),
    "tec_picker_get_params": ([_P, _P, _P, _P, _PI64], ctypes.c_int),
    "tec_picker_set_params": ([_P, _P, _P, _P, _I64], ctypes.c_int),
    "tec_picker_file_write": ([ctypes.c_char_p, _P, _P, _P, _I64, ctypes.c_char_p], ctypes.c_int),
    "tec_picker_file_read": ([ctypes.c_char_p, _P, _P, _P, _PI64, ctypes.c_char_p, ctypes.c_size_t,
                              ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "tec_picker_save": ([_P, ctypes.c_char_p, ctypes.c_char_p], ctypes.c_int),
    "tec_picker_load": ([ctypes.c_char_p, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "tec_picker_forward": ([_P, _P, _I64, ctypes.c_int, _P], ctypes.c_int),
    "tec_picker_loss_grad": ([_P, _P, _P, _I64, _P, _P], ctypes.c_int),
    "tec_picker_adam_step": ([_P, _P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float], ctypes.c_int),
    "tec_picker_train": ([_P, _P, _P, _I64, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_uint64, _P],
                         ctypes.c_int),
    "tec_picker_soft_loss_grad": ([_P, _P, _P, _P, _I64, ctypes.c_float, ctypes.c_float, _P, _P], ctypes.c_int),
    "tec_picker_train_soft": ([_P, _P, _P, _P, _I64, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_uint64,
                               ctypes.c_float, ctypes.c_float, _P], ctypes.c_int),
    "tec_picker_thresholds": ([_P, _I64, _P, _P, _P], ctypes.c_int),
    "tec_pick_threshold": ([_P, _P, _P, ctypes.c_int, ctypes.c_int, _P, _P], ctypes.c_int),
    "tec_sweep_stats": ([_P, ctypes.c_int, _P, _P, ctypes.c_int, _P, _P, ctypes.c_int, _P], ctypes.c_int),
    "tec_rule_of_thumb": ([_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P], ctypes.c_int),
    "tec_set_core_staging": ([_P, ctypes.c_int], ctypes.c_int),
    "tec_set_support_tiling": ([_P, ctypes.c_int], ctypes.c_int),
    "tec_edge_k4": ([_P, _P], ctypes.c_int),
    "tec_prf": ([_P, ctypes.c_int, _P, _P, _P, ctypes.c_int, _P], ctypes.c_int),
    "tec_components_noalloc": ([_I64, _I64, _P, _P, _P, _P, _PI64, _P], ctypes.c_int),
}

NOALLOC_MAX_VERTICES = 4194304

# tec_sweep_stat, field for field
STAT_DTYPE = np.dtype([("ncomp", "<i8"), ("kept", "<i8"), ("largest", "<i8"), ("intra", "<i8"),
                       ("modularity", "<f8")])
RULE_LARGEST_JUMP = 0
RULE_MODULARITY = 1


def components_noalloc(n: int, eu, ev, keep=None, labels=None, stream=None):
    """Components of the edge list (eu, ev) (CUDA int32 tensors; keep: optional
    uint8 mask) through the entry point that allocates no device memory.
    Returns (labels, number of components)."""
    torch = _require_cuda()
    lib = load_library()
    if labels is None:
        labels = torch.empty(max(n, 0), dtype=torch.int32, device="cuda")
    if stream is None:
        stream = torch.cuda.current_stream()
    nc = ctypes.c_int64(-1)
    check(lib.tec_components_noalloc(int(n), int(eu.numel()), _ptr(eu), _ptr(ev), _ptr(keep), _ptr(labels),
                                     ctypes.byref(nc), _P(stream.cuda_stream)))
    return labels, nc.value


def library_path() -> str:
    return _build.library_path()


def load_library(build_if_missing: bool = False):
    """Loads libtectonic.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"CUDA library not built ({path}); run paper_2412_12382_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    return int(load_library().tec_launch_count())


def last_error() -> str:
    lib = load_library()
    buf = ctypes.create_string_buffer(1024)
    lib.tec_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def check(status: int):
    if status != 0:
        raise TectonicError(status, last_error())


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _torch():
    import torch
    return torch


def _require_cuda():
    torch = _torch()
    if not torch.cuda.is_available():
        raise RuntimeError("the tectonic library needs a CUDA GPU; none is available")
    return torch


class Graph:
    """A graph resident on the GPU (a ``tec_graph``).

    ``off`` / ``col``: symmetric CSR, either CUDA tensors (int64 or int32
    offsets, int32 ids) or numpy arrays (copied from host memory).

    Every call runs on the graph's stream (``stream``, by default torch's
    current stream when the graph is made), and output tensors are allocated
    by torch on the current stream.  Use the graph from that stream, or
    synchronise before touching its results (or, for CUDA input tensors,
    before freeing them) from another one."""

    def __init__(self, off=None, col=None, *, n_cap: int | None = None, nnz_cap: int | None = None,
                 validate: bool = False, stream=None):
        torch = _require_cuda()
        self._lib = load_library()
        self._h = _P()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        if off is not None:
            n = len(off) - 1
            nnz = len(col)
            n_cap = max(n, n_cap or 0)
            nnz_cap = max(nnz, nnz_cap or 0)
        check(self._lib.tec_graph_create(int(n_cap or 0), int(nnz_cap or 0), _P(stream.cuda_stream),
                                         ctypes.byref(self._h)))
        self.n = 0
        self.m = 0
        if off is not None:
            self.load(off, col, validate=validate)

    # ------------------------------------------------------------ lifetime
    def load(self, off, col, validate: bool = False):
        host = isinstance(off, np.ndarray)
        flags = (HOST_PTR if host else 0) | (VALIDATE if validate else 0)
        if host:
            off = np.ascontiguousarray(off)
            col = np.ascontiguousarray(col, dtype=np.int32)
            i64 = off.dtype == np.int64
            if not i64:
                off = off.astype(np.int32)
        else:
            i64 = off.dtype == _torch().int64
            off = off.contiguous()
            col = col.contiguous()
        self._keep = (off, col)
        check(self._lib.tec_graph_load(self._h, _ptr(off), int(i64), _ptr(col), len(off) - 1, len(col), flags))
        self._keep = None
        n, m = ctypes.c_int64(), ctypes.c_int64()
        check(self._lib.tec_graph_info(self._h, ctypes.byref(n), ctypes.byref(m)))
        self.n, self.m = n.value, m.value
        return self

    def free(self):
        if getattr(self, "_h", None) and self._h.value:
            check(self._lib.tec_graph_free(self._h))
            self._h = _P()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def sync(self):
        check(self._lib.tec_sync(self._h))

    def set_stage_events(self, events):
        """torch.cuda.Event objects (timing enabled) recorded between the fused pass's stages."""
        self._events = list(events)
        for e in self._events:
            if not e.cuda_event:          # torch creates its events lazily on first record
                e.record(self.stream)
        arr = (_P * 5)(*[_P(e.cuda_event) for e in self._events])
        check(self._lib.tec_set_stage_events(self._h, arr, len(self._events)))

    # ------------------------------------------------------------ steps
    def _empty(self, count, dtype):
        torch = _torch()
        return torch.empty(max(count, 0), dtype=dtype, device="cuda")

    def orient(self):
        check(self._lib.tec_orient(self._h))

    def support(self):
        check(self._lib.tec_support(self._h))

    def oriented_csr(self):
        torch = _torch()
        ooff = self._empty(self.n + 1, torch.int64)
        ocol = self._empty(self.m, torch.int32)
        check(self._lib.tec_oriented_csr(self._h, _ptr(ooff), _ptr(ocol)))
        return ooff, ocol

    def edge_list(self):
        torch = _torch()
        u = self._empty(self.m, torch.int32)
        v = self._empty(self.m, torch.int32)
        check(self._lib.tec_edge_list(self._h, _ptr(u), _ptr(v)))
        return u, v

    def edge_support(self, wedges: bool = True):
        """(t, wedge) in canonical order, uint32 values in int32 tensors."""
        torch = _torch()
        t = self._empty(self.m, torch.int32)
        w = self._empty(self.m, torch.int32) if wedges else None
        check(self._lib.tec_edge_support(self._h, _ptr(t), _ptr(w)))
        return t, w

    def edge_k4(self):
        """4-cliques containing each edge (canonical order, CUDA uint32 as int32 storage)."""
        torch = _torch()
        out = self._empty(self.m, torch.int32)
        check(self._lib.tec_edge_k4(self._h, _ptr(out)))
        return out

    def edge_weights(self, measure: int = TECTONIC):
        torch = _torch()
        w = self._empty(self.m, torch.float64)
        check(self._lib.tec_edge_weights(self._h, int(measure), _ptr(w)))
        return w

    def prune(self, measure: int, p: int, q: int, mask: bool = False, count: bool = True):
        torch = _torch()
        keep = self._empty(self.m, torch.uint8) if mask else None
        kept = ctypes.c_int64(-1)
        check(self._lib.tec_prune(self._h, int(measure), int(p), int(q), _ptr(keep),
                                  ctypes.byref(kept) if count else None))
        return keep, (kept.value if count else None)

    def components(self, labels=None, count: bool = True):
        torch = _torch()
        if labels is None:
            labels = self._empty(self.n, torch.int32)
        nc = ctypes.c_int64(-1)
        check(self._lib.tec_components(self._h, _ptr(labels), ctypes.byref(nc) if count else None))
        return labels, (nc.value if count else None)

    def sweep(self, measure: int, ps, qs, seg_off=None, count: bool = True):
        """Labels (k x n CUDA int32) and component counts (k, or k x nseg with a
        segment table of the graphs in a batch) at thresholds ps[i]/qs[i]."""
        torch = _torch()
        k = len(ps)
        hp = np.ascontiguousarray(ps, dtype=np.int64)
        hq = np.ascontiguousarray(qs, dtype=np.int64)
        labels = self._empty(k * self.n, torch.int32)
        nseg = 0 if seg_off is None else seg_off.numel() - 1
        nc = np.empty(k * max(nseg, 1), dtype=np.int64)
        check(self._lib.tec_sweep(self._h, int(measure), _ptr(hp), _ptr(hq), k,
                                  _ptr(seg_off) if seg_off is not None else None, nseg, _ptr(labels),
                                  _ptr(nc) if count else None))
        nc = nc.reshape(k, max(nseg, 1)) if nseg else nc
        return labels.view(k, self.n), (nc if count else None)

    def features(self, seg_off=None):
        """Picker features: (nseg, 66) float32 CUDA tensor (one row without segments)."""
        torch = _torch()
        nseg = 0 if seg_off is None else seg_off.numel() - 1
        f = torch.empty((max(nseg, 1), 66), dtype=torch.float32, device="cuda")
        check(self._lib.tec_features(self._h, _ptr(seg_off) if seg_off is not None else None, nseg, _ptr(f)))
        return f

    def ari(self, labels, truth, seg_off=None):
        """ARI of each row of `labels` (k x n) against `truth` (n): (k, nseg) float64 tensor."""
        torch = _torch()
        k = labels.shape[0] if labels.dim() == 2 else 1
        nseg = 0 if seg_off is None else seg_off.numel() - 1
        out = torch.empty((k, max(nseg, 1)), dtype=torch.float64, device="cuda")
        check(self._lib.tec_ari(self._h, k, _ptr(labels.contiguous()), _ptr(truth.contiguous()),
                                _ptr(seg_off) if seg_off is not None else None, nseg, _ptr(out)))
        return out

    def set_support_tiling(self, groups: int):
        """Probe-row tiling of the triangle counts: -1 off, 0 automatic, k > 0 that many ranges."""
        check(self._lib.tec_set_support_tiling(self._h, int(groups)))

    def set_core_staging(self, enable: bool):
        """Exact bitmap staging of high-degree centres in the triangle counts (default on)."""
        check(self._lib.tec_set_core_staging(self._h, int(bool(enable))))

    def sweep_stats(self, measure: int, ps, qs, labels, seg_off=None):
        """Statistics of k nested labelings (k x n CUDA int32, rows at ps[i]/qs[i]):
        raw device buffer of k x nseg tec_sweep_stat (see stats_numpy)."""
        torch = _torch()
        k = len(ps)
        hp = np.ascontiguousarray(ps, dtype=np.int64)
        hq = np.ascontiguousarray(qs, dtype=np.int64)
        nseg = 0 if seg_off is None else seg_off.numel() - 1
        buf = torch.empty(k * max(nseg, 1) * STAT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        check(self._lib.tec_sweep_stats(self._h, int(measure), _ptr(hp), _ptr(hq), k, _ptr(labels.contiguous()),
                                        _ptr(seg_off) if seg_off is not None else None, nseg, _ptr(buf)))
        return buf

    def pick_threshold(self, picker, seg_off=None, bf16: bool = True):
        """Learned grid threshold per graph: (p, q) CUDA int64 tensors (nseg, or 1 without segments)."""
        torch = _torch()
        nseg = 0 if seg_off is None else seg_off.numel() - 1
        p = torch.empty(max(nseg, 1), dtype=torch.int64, device="cuda")
        q = torch.empty(max(nseg, 1), dtype=torch.int64, device="cuda")
        check(self._lib.tec_pick_threshold(self._h, picker._h, _ptr(seg_off) if seg_off is not None else None, nseg,
                                           int(bf16), _ptr(p), _ptr(q)))
        return p, q

    def prf(self, labels, truth, seg_off=None):
        """Precision, recall, F1 (Sec. IV-A) of each row of `labels` (k x n) against `truth`:
        (k, nseg, 3) float64 tensor."""
        torch = _torch()
        k = labels.shape[0] if labels.dim() == 2 else 1
        nseg = 0 if seg_off is None else seg_off.numel() - 1
        out = torch.empty((k, max(nseg, 1), 3), dtype=torch.float64, device="cuda")
        check(self._lib.tec_prf(self._h, k, _ptr(labels.contiguous()), _ptr(truth.contiguous()),
                                _ptr(seg_off) if seg_off is not None else None, nseg, _ptr(out)))
        return out

    def prune_components_batch(self, measure: int, p, q, seg_off, labels=None, count: bool = True):
        """Per-graph thresholds p[s]/q[s] (CUDA int64): local labels (n) and components per graph."""
        torch = _torch()
        nseg = seg_off.numel() - 1
        if labels is None:
            labels = self._empty(self.n, torch.int32)
        nc = np.empty(nseg, dtype=np.int64)
        check(self._lib.tec_prune_components_batch(self._h, int(measure), _ptr(p), _ptr(q), _ptr(seg_off), nseg,
                                                   _ptr(labels), _ptr(nc) if count else None))
        return labels, (nc if count else None)

    def full_pass(self, measure: int, p: int, q: int, labels=None, count: bool = True):
        torch = _torch()
        if labels is None:
            labels = self._empty(self.n, torch.int32)
        nc = ctypes.c_int64(-1)
        check(self._lib.tec_full_pass(self._h, int(measure), int(p), int(q), _ptr(labels),
                                      ctypes.byref(nc) if count else None))
        return labels, (nc.value if count else None)

    def full_pass_host(self, off: np.ndarray, col: np.ndarray, measure: int, p: int, q: int,
                       labels: np.ndarray | None = None):
        off = np.ascontiguousarray(off, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        n = len(off) - 1
        if labels is None:
            labels = np.empty(n, dtype=np.int32)
        nc = ctypes.c_int64(-1)
        check(self._lib.tec_full_pass_host(self._h, _ptr(off), _ptr(col), n, len(col), int(measure), int(p),
                                           int(q), _ptr(labels), ctypes.byref(nc)))
        n_, m_ = ctypes.c_int64(), ctypes.c_int64()
        check(self._lib.tec_graph_info(self._h, ctypes.byref(n_), ctypes.byref(m_)))
        self.n, self.m = n_.value, m_.value
        return labels, nc.value


PICKER_PARAMS = 25217


def ari_best(ari, stream=None):
    """Row of highest ARI per graph (first on ties) and its value: (int32, float64) CUDA tensors."""
    torch = _require_cuda()
    k, nseg = ari.shape
    best = torch.empty(nseg, dtype=torch.int32, device="cuda")
    val = torch.empty(nseg, dtype=torch.float64, device="cuda")
    stream = stream or torch.cuda.current_stream()
    check(load_library().tec_ari_best(_ptr(ari.contiguous()), k, nseg, _ptr(best), _ptr(val), _P(stream.cuda_stream)))
    return best, val


def stats_numpy(buf, k: int, nseg: int = 1):
    """Host copy of a tec_sweep_stats buffer as a (k, nseg) structured array."""
    return np.frombuffer(buf.cpu().numpy().tobytes(), dtype=STAT_DTYPE).reshape(k, max(nseg, 1))


def rule_of_thumb(stats_buf, ps, qs, nseg: int = 1, rule: int = RULE_LARGEST_JUMP, stream=None):
    """Row picked per graph by a threshold rule of thumb (Sec. IV-D): CUDA int32 tensor."""
    torch = _require_cuda()
    k = len(ps)
    hp = np.ascontiguousarray(ps, dtype=np.int64)
    hq = np.ascontiguousarray(qs, dtype=np.int64)
    best = torch.empty(max(nseg, 1), dtype=torch.int32, device="cuda")
    stream = stream or torch.cuda.current_stream()
    check(load_library().tec_rule_of_thumb(_ptr(stats_buf), _ptr(hp), _ptr(hq), k, max(nseg, 1), int(rule),
                                           _ptr(best), _P(stream.cuda_stream)))
    return best


def picker_thresholds(y, stream=None):
    """Grid thresholds (p, q) as CUDA int64 tensors from picker outputs y."""
    torch = _require_cuda()
    n = y.numel()
    p = torch.empty(n, dtype=torch.int64, device="cuda")
    q = torch.empty(n, dtype=torch.int64, device="cuda")
    stream = stream or torch.cuda.current_stream()
    check(load_library().tec_picker_thresholds(_ptr(y.contiguous()), n, _ptr(p), _ptr(q), _P(stream.cuda_stream)))
    return p, q


def picker_file_write(path: str, params, adam_m=None, adam_v=None, step: int = 0, meta: str = ""):
    """Writes a picker checkpoint file from host arrays (tec_picker_file_write; no device needed)."""
    arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float32) for a in (params, adam_m, adam_v)]
    for a in arrs:
        if a is not None and a.shape != (PICKER_PARAMS,):
            raise ValueError(f"a checkpoint holds {PICKER_PARAMS} parameters and moments")
    check(load_library().tec_picker_file_write(os.fsencode(path), *[_ptr(a) for a in arrs], int(step),
                                               meta.encode()))


def picker_file_read(path: str):
    """(params, adam_m, adam_v, step, meta text) of a checkpoint file, checked
    by the library (tec_picker_file_read; no device needed)."""
    lib = load_library()
    L = ctypes.c_size_t(0)
    check(lib.tec_picker_file_read(os.fsencode(path), None, None, None, None, None, 0, ctypes.byref(L)))
    p, m, v = (np.empty(PICKER_PARAMS, dtype=np.float32) for _ in range(3))
    step = ctypes.c_int64(0)
    buf = ctypes.create_string_buffer(L.value + 1)
    check(lib.tec_picker_file_read(os.fsencode(path), _ptr(p), _ptr(m), _ptr(v), ctypes.byref(step), buf,
                                   L.value + 1, ctypes.byref(L)))
    return p, m, v, step.value, buf.raw[:L.value].decode()


class Picker:
    """The learned threshold picker (a ``tec_picker``)."""

    def __init__(self, init_params=None, stream=None, _handle=None):
        torch = _require_cuda()
        self._lib = load_library()
        self.stream = stream or torch.cuda.current_stream()
        self._h = _P()
        if _handle is not None:
            self._h = _handle
            return
        init = None if init_params is None else np.ascontiguousarray(init_params, dtype=np.float32)
        check(self._lib.tec_picker_create(_ptr(init), _P(self.stream.cuda_stream), ctypes.byref(self._h)))

    @classmethod
    def load(cls, path: str, stream=None):
        """A picker holding the state of a checkpoint file (tec_picker_load)."""
        torch = _require_cuda()
        stream = stream or torch.cuda.current_stream()
        h = _P()
        check(load_library().tec_picker_load(os.fsencode(path), _P(stream.cuda_stream), ctypes.byref(h)))
        return cls(stream=stream, _handle=h)

    def save(self, path: str, meta: str = ""):
        """Writes the current parameters, Adam moments and step (tec_picker_save)."""
        check(self._lib.tec_picker_save(self._h, os.fsencode(path), meta.encode()))

    def free(self):
        if getattr(self, "_h", None) and self._h.value:
            check(self._lib.tec_picker_free(self._h))
            self._h = _P()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def get_params(self, with_adam: bool = False):
        p = np.empty(PICKER_PARAMS, dtype=np.float32)
        m = np.empty_like(p) if with_adam else None
        v = np.empty_like(p) if with_adam else None
        step = ctypes.c_int64(0)
        check(self._lib.tec_picker_get_params(self._h, _ptr(p), _ptr(m), _ptr(v), ctypes.byref(step)))
        return (p, m, v, step.value) if with_adam else p

    def set_params(self, params, m=None, v=None, step: int = 0):
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float32) for a in (params, m, v)]
        check(self._lib.tec_picker_set_params(self._h, *[_ptr(a) for a in arrs], int(step)))

    def forward(self, feats, bf16: bool = False):
        torch = _torch()
        out = torch.empty(feats.shape[0], dtype=torch.float32, device="cuda")
        check(self._lib.tec_picker_forward(self._h, _ptr(feats.contiguous()), feats.shape[0], int(bf16), _ptr(out)))
        return out

    def loss_grad(self, feats, target):
        torch = _torch()
        g = torch.empty(PICKER_PARAMS, dtype=torch.float32, device="cuda")
        loss = ctypes.c_float(0.0)
        check(self._lib.tec_picker_loss_grad(self._h, _ptr(feats.contiguous()), _ptr(target.contiguous()),
                                             feats.shape[0], ctypes.byref(loss), _ptr(g)))
        return loss.value, g

    def adam_step(self, grad=None, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        check(self._lib.tec_picker_adam_step(self._h, _ptr(grad), lr, beta1, beta2, eps))

    def soft_loss_grad(self, feats, target, ari_loss, sigma: float, mix: float):
        """Soft-level loss (mean) and its gradient (tec_picker_soft_loss_grad)."""
        torch = _torch()
        g = torch.empty(PICKER_PARAMS, dtype=torch.float32, device="cuda")
        loss = ctypes.c_float(0.0)
        check(self._lib.tec_picker_soft_loss_grad(self._h, _ptr(feats.contiguous()), _ptr(target.contiguous()),
                                                  _ptr(ari_loss.contiguous()), feats.shape[0], float(sigma),
                                                  float(mix), ctypes.byref(loss), _ptr(g)))
        return loss.value, g

    def train_soft(self, feats, target, ari_loss, epochs: int, batch: int = 256, lr: float = 1e-3, seed: int = 0,
                   sigma: float = 1.5, mix: float = 0.5):
        """tec_picker_train with the soft-level loss; returns the mean loss per epoch."""
        losses = np.empty(max(epochs, 1), dtype=np.float32)
        check(self._lib.tec_picker_train_soft(self._h, _ptr(feats.contiguous()), _ptr(target.contiguous()),
                                              _ptr(ari_loss.contiguous()), feats.shape[0], int(epochs), int(batch),
                                              float(lr), int(seed), float(sigma), float(mix), _ptr(losses)))
        return losses[:epochs]

    def train(self, feats, target, epochs: int, batch: int = 256, lr: float = 1e-3, seed: int = 0):
        losses = np.empty(max(epochs, 1), dtype=np.float32)
        check(self._lib.tec_picker_train(self._h, _ptr(feats.contiguous()), _ptr(target.contiguous()),
                                         feats.shape[0], int(epochs), int(batch), float(lr), int(seed),
                                         _ptr(losses)))
        return losses[:epochs]
