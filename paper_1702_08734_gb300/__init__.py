"""gbknn: exact and IVFADC k-NN search on one GB300 (sm_103a), arXiv 1702.08734.

Thin ctypes binding over the C ABI in ``include/gbknn.h``: it only checks tensor
shapes, allocates outputs with PyTorch and passes raw device pointers and the current
CUDA stream.  Every step of the computation runs in the library's own CUDA kernels.
There is no CPU fallback: without the compiled library every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import datagen  # noqa: F401  (seeded synthetic inputs)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbknn.so")
_lib = None
_lock = threading.Lock()

METRIC_L2 = 0
METRIC_IP = 1

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


class GbkError(RuntimeError):
    """A library call returned a non-zero gbk_status."""

    def __init__(self, status, msg):
        super().__init__("gbknn status %d: %s" % (status, msg))
        self.status = status


# (name, argtypes); every entry point returns gbk_status (int32)
_SIGNATURES = {
    "gbk_kselect": [_vp, _i64, _i64, _i32, _i32, _vp, _vp, _vp],
    "gbk_kselect_ex": [_vp, _i64, _i64, _i32, _i32, _vp, _vp, _vp, _vp],
    "gbk_row_norms": [_vp, _i64, _i32, _vp, _vp],
    "gbk_device_status": [_vp],
    "gbk_selftest_wait_timeout": [_i64, _vp],
    "gbk_knn_brute": [_vp, _i64, _vp, _i64, _i32, _i32, _i32, _vp, _vp, _vp, _vp],
    "gbk_knn_brute_host": [_vp, _i64, _vp, _i64, _i32, _i32, _i32, _vp, _vp, _vp, _vp],
    "gbk_knn_db_create": [_vp, _i64, _i32, _i32, _vp, _vp],
    "gbk_knn_db_search": [_vp, _vp, _i64, _i32, _i32, _vp, _vp, _vp, _vp],
    "gbk_pairwise_distances": [_vp, _i64, _vp, _i64, _i32, _i32, _i32, _vp, _i64, _vp],
}


def build(force: bool = False) -> str:
    """Compile the CUDA library in-tree (nvcc, sm_103a)."""
    from . import buildlib as _b
    return _b.build(force=force)


def load(path: str | None = None):
    """Load libgbknn.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError("libgbknn.so not built (run paper_1702_08734_gb300.build())")
            lib = ctypes.CDLL(p)
            for name, args in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int32
            lib.gbk_last_error.restype = ctypes.c_char_p
            lib.gbk_profile_enable.argtypes = [ctypes.c_int32]
            lib.gbk_profile_enable.restype = None
            lib.gbk_profile_read.argtypes = [ctypes.c_char_p, ctypes.c_void_p, ctypes.c_int32]
            lib.gbk_profile_read.restype = ctypes.c_int32
            lib.gbk_version.restype = ctypes.c_int32
            lib.gbk_ivfpq_destroy.argtypes = [ctypes.c_void_p]
            lib.gbk_ivfpq_destroy.restype = None
            _lib = lib
    return _lib


def _call(name, *args):
    lib = load()
    st = getattr(lib, name)(*args)
    if st != 0:
        raise GbkError(st, lib.gbk_last_error().decode())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _dev(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t


class KselectOpts(ctypes.Structure):
    _fields_ = [("segments", ctypes.c_int32), ("unroll", ctypes.c_int32)]


def device_status():
    """Synchronise the current stream and raise if a kernel flagged an error."""
    _call("gbk_device_status", _stream())


def selftest_wait_timeout(limit_ns: int = 1000000):
    """Launch the bounded-wait self-test: the next device_status() raises GBK_ETIMEOUT."""
    _call("gbk_selftest_wait_timeout", int(limit_ns), _stream())


_ALLOC_CB = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_CB = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class _Allocator(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("alloc", _ALLOC_CB), ("free", _FREE_CB)]


_installed_allocator = None


def set_allocator(alloc=None, free=None):
    """Install alloc(nbytes, stream) -> device pointer (int; 0 = failure) and
    free(ptr, stream) as the library's scratch allocator; alloc=None restores the default
    (cudaMallocAsync on the call's stream)."""
    global _installed_allocator
    lib = load()
    lib.gbk_set_allocator.argtypes = [ctypes.c_void_p]
    if alloc is None:
        _call("gbk_set_allocator", None)
        _installed_allocator = None
        return

    def a(ctx, n, st):
        try:
            return int(alloc(int(n), st) or 0) or None
        except Exception:
            return None

    def f(ctx, p, st):
        if free is not None and p:
            free(int(p), st)

    cb = _Allocator(None, _ALLOC_CB(a), _FREE_CB(f))
    _call("gbk_set_allocator", ctypes.cast(ctypes.pointer(cb), ctypes.c_void_p))
    _installed_allocator = cb  # keeps the callbacks alive


def use_torch_allocator():
    """Scratch memory from PyTorch's caching allocator (on the current stream)."""
    set_allocator(lambda n, st: torch.cuda.caching_allocator_alloc(n),
                  lambda p, st: torch.cuda.caching_allocator_delete(p))


def kselect(vals: torch.Tensor, k: int, largest: bool = False, out=None, segments: int = 0,
            unroll: int = 0):
    """Row-wise k smallest (largest) values and their int64 indices, sorted best first.

    segments / unroll are launch parameters (0 = library default); results never depend
    on them."""
    _dev(vals, torch.float32, "vals")
    if vals.dim() != 2:
        raise ValueError("vals must be 2-D")
    rows, length = vals.shape
    if out is None:
        D = torch.empty((rows, k), dtype=torch.float32, device=vals.device)
        I = torch.empty((rows, k), dtype=torch.int64, device=vals.device)
    else:
        D, I = out
    if segments or unroll:
        opts = KselectOpts(int(segments), int(unroll))
        _call("gbk_kselect_ex", _ptr(vals), rows, length, int(k), int(bool(largest)), _ptr(D),
              _ptr(I), ctypes.byref(opts), _stream())
    else:
        _call("gbk_kselect", _ptr(vals), rows, length, int(k), int(bool(largest)), _ptr(D),
              _ptr(I), _stream())
    return D, I


def row_norms(x: torch.Tensor, out=None):
    """Squared L2 norm of every row of x (float32)."""
    _dev(x, torch.float32, "x")
    n, d = x.shape
    o = torch.empty(n, dtype=torch.float32, device=x.device) if out is None else out
    _call("gbk_row_norms", _ptr(x), n, int(d), _ptr(o), _stream())
    return o


PRECISIONS = {"fp32": 0, "bf16": 1, "fp8": 2, "tf32x3": 3}


class KnnOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("kprime", ctypes.c_int32),
                ("chunks", ctypes.c_int32), ("certified", ctypes.c_void_p),
                ("error_bound", ctypes.c_void_p), ("exact", ctypes.c_int32),
                ("prefilter", ctypes.c_int32)]


def _metric(m):
    return {"l2": METRIC_L2, "ip": METRIC_IP}[m] if isinstance(m, str) else int(m)


def knn_brute(xq: torch.Tensor, xb: torch.Tensor, k: int, metric="l2", precision="fp32",
              kprime: int = 0, chunks: int = 0, out=None, certify: bool = False,
              exact: bool = False, prefilter: int = 0):
    """Exact k-NN (squared L2 ascending, or inner product descending) with int64 ids.

    precision "bf16"/"fp8": over-fetch kprime candidates, exact float32 re-rank; with
    certify=True also returns (certified [nq] int32, error_bound [nq] float32); with
    exact=True the queries the certificate does not cover are re-run in float32
    (certified = 2 for them).  prefilter: threshold pre-pass of the fused selection (1 on,
    -1 off, 0 automatic); the results are the same either way."""
    _dev(xq, torch.float32, "xq")
    _dev(xb, torch.float32, "xb")
    nq, d = xq.shape
    nb = xb.shape[0]
    if xb.shape[1] != d:
        raise ValueError("dimension mismatch")
    if out is None:
        D = torch.empty((nq, k), dtype=torch.float32, device=xq.device)
        I = torch.empty((nq, k), dtype=torch.int64, device=xq.device)
    else:
        D, I = out
    cert = eb = None
    if certify:
        cert = torch.empty(nq, dtype=torch.int32, device=xq.device)
        eb = torch.empty(nq, dtype=torch.float32, device=xq.device)
    opts = KnnOpts(PRECISIONS[precision], int(kprime), int(chunks),
                   cert.data_ptr() if cert is not None else None,
                   eb.data_ptr() if eb is not None else None, int(bool(exact)),
                   int(prefilter))
    _call("gbk_knn_brute", _ptr(xq), nq, _ptr(xb), nb, int(d), int(k), _metric(metric), _ptr(D),
          _ptr(I), ctypes.byref(opts), _stream())
    return (D, I, cert, eb) if certify else (D, I)


class KnnDatabase:
    """A database prepared once for repeated exact k-NN searches (gbk_knn_db_*): the operand
    pieces of `precision` and the norms stay on the device; `xb` (CUDA float32) is kept
    referenced, unchanged, for the re-rank and repair.  search() takes knn_brute's arguments
    and returns the same results."""

    def __init__(self, xb: torch.Tensor, precision="fp32"):
        _dev(xb, torch.float32, "xb")
        lib = load()
        lib.gbk_knn_db_destroy.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        lib.gbk_knn_db_destroy.restype = None
        self._xb = xb.contiguous()
        self.precision = precision
        self._h = ctypes.c_void_p()
        _call("gbk_knn_db_create", _ptr(self._xb), self._xb.shape[0], int(self._xb.shape[1]),
              PRECISIONS[precision], ctypes.byref(self._h), _stream())

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            load().gbk_knn_db_destroy(self._h, _stream())
            self._h = ctypes.c_void_p()

    def search(self, xq: torch.Tensor, k: int, metric="l2", kprime: int = 0, chunks: int = 0,
               out=None, certify: bool = False, exact: bool = False, prefilter: int = 0):
        _dev(xq, torch.float32, "xq")
        nq, d = xq.shape
        if d != self._xb.shape[1]:
            raise ValueError("dimension mismatch")
        if out is None:
            D = torch.empty((nq, k), dtype=torch.float32, device=xq.device)
            I = torch.empty((nq, k), dtype=torch.int64, device=xq.device)
        else:
            D, I = out
        cert = eb = None
        if certify:
            cert = torch.empty(nq, dtype=torch.int32, device=xq.device)
            eb = torch.empty(nq, dtype=torch.float32, device=xq.device)
        opts = KnnOpts(PRECISIONS[self.precision], int(kprime), int(chunks),
                       cert.data_ptr() if cert is not None else None,
                       eb.data_ptr() if eb is not None else None, int(bool(exact)),
                       int(prefilter))
        _call("gbk_knn_db_search", self._h, _ptr(xq), nq, int(k), _metric(metric), _ptr(D),
              _ptr(I), ctypes.byref(opts), _stream())
        return (D, I, cert, eb) if certify else (D, I)


def knn_brute_host(xq: torch.Tensor, xb: torch.Tensor, k: int, metric="l2", precision="fp32",
                   kprime: int = 0, chunks: int = 0, out=None, exact: bool = False,
                   prefilter: int = 0, sync: bool = True):
    """knn_brute on host (CPU) float32 tensors, pinned for the copies to overlap the search:
    the library copies the inputs in, searches and copies D, I (CPU tensors) back, all on the
    current stream; with sync=False the caller synchronises the stream before reading them."""
    for t, nm in ((xq, "xq"), (xb, "xb")):
        if t.device.type != "cpu" or t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError("%s must be a contiguous float32 CPU tensor" % nm)
    nq, d = xq.shape
    nb = xb.shape[0]
    if xb.shape[1] != d:
        raise ValueError("dimension mismatch")
    if out is None:
        D = torch.empty((nq, k), dtype=torch.float32).pin_memory()
        I = torch.empty((nq, k), dtype=torch.int64).pin_memory()
    else:
        D, I = out
    opts = KnnOpts(PRECISIONS[precision], int(kprime), int(chunks), None, None,
                   int(bool(exact)), int(prefilter))
    _call("gbk_knn_brute_host", ctypes.c_void_p(xq.data_ptr()), nq,
          ctypes.c_void_p(xb.data_ptr()), nb, int(d), int(k), _metric(metric),
          ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(I.data_ptr()), ctypes.byref(opts),
          _stream())
    if sync:
        torch.cuda.current_stream().synchronize()
    return D, I


def pairwise_distances(xq: torch.Tensor, xb: torch.Tensor, metric="l2", precision="fp32"):
    """Full [nq][nb] squared L2 distance (or inner product) matrix on the tensor cores."""
    _dev(xq, torch.float32, "xq")
    _dev(xb, torch.float32, "xb")
    nq, d = xq.shape
    nb = xb.shape[0]
    out = torch.empty((nq, nb), dtype=torch.float32, device=xq.device)
    _call("gbk_pairwise_distances", _ptr(xq), nq, _ptr(xb), nb, int(d), _metric(metric),
          PRECISIONS[precision], _ptr(out), nb, _stream())
    return out


def profile_enable(on: bool = True):
    """Record a CUDA event pair around every library kernel launch (see profile_read)."""
    load().gbk_profile_enable(int(bool(on)))


def profile_read(max_records: int = 4096):
    """[(kernel name, ms)] recorded since the last read, in launch order."""
    names = ctypes.create_string_buffer(32 * max_records)
    ms = (ctypes.c_float * max_records)()
    n = load().gbk_profile_read(names, ctypes.cast(ms, ctypes.c_void_p), max_records)
    raw = names.raw
    return [(raw[32 * i:32 * i + 32].split(b"\0", 1)[0].decode(), float(ms[i])) for i in range(n)]


# ---------------------------------------------------------------------------- k-means / IVFPQ

_SIGNATURES.update({
    "gbk_kmeans": [_vp, _i64, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _i32, _vp],
    "gbk_ivfpq_create": [_i32, _i32, _i32, _i32, _i32, _vp],
    "gbk_ivfpq_train": [_vp, _vp, _i64, _vp, _vp],
    "gbk_ivfpq_set_quantizers": [_vp, _vp, _vp, _i32, _vp],
    "gbk_ivfpq_add": [_vp, _vp, _i64, _vp, _vp],
    "gbk_ivfpq_search": [_vp, _vp, _i64, _i32, _i32, _vp, _vp, _vp],
    "gbk_ivfpq_info": [_vp, _vp, _vp, _vp, _vp, _vp],
    "gbk_ivfpq_export": [_vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "gbk_ivfpq_keep_vectors": [_vp, _i32],
    "gbk_ivfpq_set_coarse_precision": [_vp, _i32],
    "gbk_ivfpq_set_rotation": [_vp, _vp, _vp],
    "gbk_ivfpq_rotate": [_vp, _vp, _i64, _vp, _vp],
    "gbk_ivfpq_search_refine": [_vp, _vp, _i64, _i32, _i32, _i32, _vp, _vp, _vp],
    "gbk_ivfflat_create": [_i32, _i32, _i32, _vp],
    "gbk_ivfflat_train": [_vp, _vp, _i64, _vp, _vp],
    "gbk_ivfflat_set_centroids": [_vp, _vp, _vp],
    "gbk_ivfflat_add": [_vp, _vp, _i64, _vp, _vp],
    "gbk_ivfflat_search": [_vp, _vp, _i64, _i32, _i32, _vp, _vp, _vp],
    "gbk_ivfflat_info": [_vp, _vp, _vp, _vp, _vp],
    "gbk_ivfflat_export": [_vp, _vp, _vp, _vp, _vp],
})


def _host_i64(a):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def kmeans(x: torch.Tensor, init_idx, niter: int, direct: bool = False):
    """Lloyd's k-means on the GPU.  init_idx: row numbers of x used as initial centroids.
    Returns (centroids [nc][d] CUDA tensor, objective per iteration (host float64 array),
    number of empty-cluster re-seeds)."""
    import numpy as np
    _dev(x, torch.float32, "x")
    n, d = x.shape
    ii, iip = _host_i64(init_idx)
    nc = ii.size
    cent = torch.empty((nc, d), dtype=torch.float32, device=x.device)
    obj = torch.zeros(max(niter, 1), dtype=torch.float64, device=x.device)
    ns = torch.zeros(1, dtype=torch.int64, device=x.device)
    _call("gbk_kmeans", _ptr(x), n, int(d), int(nc), int(niter), iip, _ptr(cent), _ptr(obj),
          _ptr(ns), int(bool(direct)), _stream())
    return cent, obj[:niter].cpu().numpy(), int(ns.item())


class TrainOpts(ctypes.Structure):
    _fields_ = [("niter", ctypes.c_int32), ("pq_niter", ctypes.c_int32),
                ("coarse_init", ctypes.c_void_p), ("pq_init", ctypes.c_void_p),
                ("use_precomputed", ctypes.c_int32)]


class OpqOpts(ctypes.Structure):
    _fields_ = [("niter", ctypes.c_int32), ("pq_niter", ctypes.c_int32),
                ("polar_iters", ctypes.c_int32), ("pq_init", ctypes.c_void_p)]


class IVFPQIndex:
    """IVFADC index on the GPU (coarse quantizer + 8-bit product quantizer, inverted lists)."""

    def __init__(self, d: int, nlist: int, M: int, nbits: int = 8, metric="l2"):
        self.d, self.nlist, self.M = int(d), int(nlist), int(M)
        h = ctypes.c_void_p()
        _call("gbk_ivfpq_create", self.d, self.nlist, self.M, int(nbits), _metric(metric),
              ctypes.byref(h))
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.gbk_ivfpq_destroy(self._h)
            self._h = None

    def train(self, x: torch.Tensor, niter: int = 20, pq_niter: int = 0, coarse_init=None,
              pq_init=None, use_precomputed: bool = True):
        _dev(x, torch.float32, "x")
        ci = pi = None
        cip = pip = None
        if coarse_init is not None:
            ci, cip = _host_i64(coarse_init)
        if pq_init is not None:
            pi, pip = _host_i64(pq_init)
        o = TrainOpts(int(niter), int(pq_niter), cip, pip, int(bool(use_precomputed)))
        _call("gbk_ivfpq_train", self._h, _ptr(x), x.shape[0], ctypes.byref(o), _stream())
        torch.cuda.current_stream().synchronize()
        return self

    def set_quantizers(self, coarse: torch.Tensor, pq: torch.Tensor, use_precomputed=True):
        _dev(coarse, torch.float32, "coarse")
        _dev(pq, torch.float32, "pq")
        _call("gbk_ivfpq_set_quantizers", self._h, _ptr(coarse), _ptr(pq),
              int(bool(use_precomputed)), _stream())
        return self

    def add(self, x: torch.Tensor, ids: torch.Tensor = None):
        _dev(x, torch.float32, "x")
        if ids is not None:
            _dev(ids, torch.int64, "ids")
        _call("gbk_ivfpq_add", self._h, _ptr(x), x.shape[0], _ptr(ids), _stream())
        return self

    def search(self, xq: torch.Tensor, k: int, nprobe: int, out=None):
        _dev(xq, torch.float32, "xq")
        nq = xq.shape[0]
        if out is None:
            D = torch.empty((nq, k), dtype=torch.float32, device=xq.device)
            I = torch.empty((nq, k), dtype=torch.int64, device=xq.device)
        else:
            D, I = out
        _call("gbk_ivfpq_search", self._h, _ptr(xq), nq, int(k), int(nprobe), _ptr(D), _ptr(I),
              _stream())
        return D, I

    def set_rotation(self, R: torch.Tensor = None):
        """OPQ pre-rotation R [d][d]: every input vector y becomes R y (before training)."""
        if R is not None:
            _dev(R, torch.float32, "R")
        _call("gbk_ivfpq_set_rotation", self._h, _ptr(R), _stream())
        return self

    def train_rotation(self, x: torch.Tensor, niter: int = 10, pq_niter: int = 4, pq_init=None,
                       polar_iters: int = 12):
        """Train the OPQ rotation on x (before train/add) and install it; returns R [d][d]."""
        _dev(x, torch.float32, "x")
        pi = pip = None
        if pq_init is not None:
            pi, pip = _host_i64(pq_init)
        o = OpqOpts(int(niter), int(pq_niter), int(polar_iters), pip)
        R = torch.empty((self.d, self.d), dtype=torch.float32, device=x.device)
        _call("gbk_ivfpq_train_rotation", self._h, _ptr(x), x.shape[0], ctypes.byref(o), _ptr(R),
              _stream())
        return R

    def rotate(self, x: torch.Tensor):
        """x rotated by the index's R (the space of its quantizers)."""
        _dev(x, torch.float32, "x")
        out = torch.empty_like(x)
        _call("gbk_ivfpq_rotate", self._h, _ptr(x), x.shape[0], _ptr(out), _stream())
        return out

    def set_coarse_precision(self, precision="fp32"):
        """Coarse-search GEMM precision ("fp32", "bf16", "fp8"; low precision re-ranks the
        over-fetched lists in float32)."""
        _call("gbk_ivfpq_set_coarse_precision", self._h, PRECISIONS[precision])
        return self

    def keep_vectors(self, keep: bool = True):
        """Keep float32 copies of the vectors added from now on (for search_refine)."""
        _call("gbk_ivfpq_keep_vectors", self._h, int(bool(keep)))
        return self

    def search_refine(self, xq: torch.Tensor, k: int, nprobe: int, kprime: int, out=None):
        """kprime ADC candidates per query, re-ranked by exact float32 distances to k."""
        _dev(xq, torch.float32, "xq")
        nq = xq.shape[0]
        if out is None:
            D = torch.empty((nq, k), dtype=torch.float32, device=xq.device)
            I = torch.empty((nq, k), dtype=torch.int64, device=xq.device)
        else:
            D, I = out
        _call("gbk_ivfpq_search_refine", self._h, _ptr(xq), nq, int(k), int(nprobe), int(kprime),
              _ptr(D), _ptr(I), _stream())
        return D, I

    @property
    def ntotal(self):
        n = ctypes.c_int64()
        _call("gbk_ivfpq_info", self._h, ctypes.byref(n), None, None, None, _stream())
        return n.value

    def save(self, path: str):
        """Write the index to a file (gbk_ivfpq_save)."""
        _call("gbk_ivfpq_save", self._h, os.fsencode(path), _stream())
        return self

    @classmethod
    def load(cls, path: str):
        """A new index read from a file written by save()."""
        h = ctypes.c_void_p()
        _call("gbk_ivfpq_load", os.fsencode(path), ctypes.byref(h), _stream())
        ix = cls.__new__(cls)
        ix._h = h
        n = ctypes.c_int64()
        nl, d, M = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _call("gbk_ivfpq_info", h, ctypes.byref(n), ctypes.byref(nl), ctypes.byref(d),
              ctypes.byref(M), _stream())
        ix.d, ix.nlist, ix.M = d.value, nl.value, M.value
        return ix

    def export(self):
        """Host copies: coarse [nlist][d], pq [M][256][d/M], list_off, codes, ids."""
        import numpy as np
        n = self.ntotal
        coarse = np.empty((self.nlist, self.d), np.float32)
        pq = np.empty((self.M, 256, self.d // self.M), np.float32)
        off = np.empty(self.nlist + 1, np.int64)
        codes = np.empty((max(n, 1), self.M), np.uint8)
        ids = np.empty(max(n, 1), np.int64)
        _call("gbk_ivfpq_export", self._h, coarse.ctypes.data_as(_vp), pq.ctypes.data_as(_vp),
              off.ctypes.data_as(_vp), codes.ctypes.data_as(_vp), ids.ctypes.data_as(_vp),
              _stream())
        torch.cuda.current_stream().synchronize()
        return {"coarse": coarse, "pq": pq, "list_off": off, "codes": codes[:n], "ids": ids[:n]}


class IVFFlatIndex:
    """Inverted file with float32 lists: coarse quantizer + exact list scan on the GPU."""

    def __init__(self, d: int, nlist: int, metric="l2"):
        self.d, self.nlist = int(d), int(nlist)
        h = ctypes.c_void_p()
        _call("gbk_ivfflat_create", self.d, self.nlist, _metric(metric), ctypes.byref(h))
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.gbk_ivfflat_destroy(self._h)
            self._h = None

    def train(self, x: torch.Tensor, niter: int = 20, coarse_init=None):
        _dev(x, torch.float32, "x")
        ci = cip = None
        if coarse_init is not None:
            ci, cip = _host_i64(coarse_init)
        o = TrainOpts(int(niter), 0, cip, None, 0)
        _call("gbk_ivfflat_train", self._h, _ptr(x), x.shape[0], ctypes.byref(o), _stream())
        torch.cuda.current_stream().synchronize()
        return self

    def set_centroids(self, coarse: torch.Tensor):
        _dev(coarse, torch.float32, "coarse")
        _call("gbk_ivfflat_set_centroids", self._h, _ptr(coarse), _stream())
        return self

    def add(self, x: torch.Tensor, ids: torch.Tensor = None):
        _dev(x, torch.float32, "x")
        if ids is not None:
            _dev(ids, torch.int64, "ids")
        _call("gbk_ivfflat_add", self._h, _ptr(x), x.shape[0], _ptr(ids), _stream())
        return self

    def search(self, xq: torch.Tensor, k: int, nprobe: int, out=None):
        _dev(xq, torch.float32, "xq")
        nq = xq.shape[0]
        if out is None:
            D = torch.empty((nq, k), dtype=torch.float32, device=xq.device)
            I = torch.empty((nq, k), dtype=torch.int64, device=xq.device)
        else:
            D, I = out
        _call("gbk_ivfflat_search", self._h, _ptr(xq), nq, int(k), int(nprobe), _ptr(D), _ptr(I),
              _stream())
        return D, I

    @property
    def ntotal(self):
        n = ctypes.c_int64()
        _call("gbk_ivfflat_info", self._h, ctypes.byref(n), None, None, _stream())
        return n.value

    def export(self):
        """Host copies: coarse [nlist][d], list_off [nlist+1], ids [ntotal] in list order."""
        import numpy as np
        n = self.ntotal
        coarse = np.empty((self.nlist, self.d), np.float32)
        off = np.empty(self.nlist + 1, np.int64)
        ids = np.empty(max(n, 1), np.int64)
        _call("gbk_ivfflat_export", self._h, coarse.ctypes.data_as(_vp), off.ctypes.data_as(_vp),
              ids.ctypes.data_as(_vp), _stream())
        torch.cuda.current_stream().synchronize()
        return {"coarse": coarse, "list_off": off, "ids": ids[:n]}


# ---------------------------------------------------------------------------- learned nprobe MLP

_SIGNATURES.update({
    "gbk_mlp_create": [_i32, _i32, _i32, _i32, _vp, _vp],
    "gbk_mlp_params": [_vp, _vp, _vp, _vp],
    "gbk_mlp_forward": [_vp, _vp, _i64, _vp, _vp, _vp],
    "gbk_mlp_train_step": [_vp, _vp, _vp, _i64, ctypes.c_float, _i32, _vp, _vp],
})


class MLP:
    """f -> relu(W1 f + b1) -> relu(W2 . + b2) -> W3 . + b3, trained on the GPU (BF16 weights
    in the passes, float32 master copy and accumulation, Adam)."""

    def __init__(self, n_in, h1, h2, n_out, params=None, seed=None):
        lib = load()
        lib.gbk_mlp_num_params.argtypes = [_vp]
        lib.gbk_mlp_num_params.restype = ctypes.c_int64
        lib.gbk_mlp_destroy.argtypes = [_vp]
        lib.gbk_mlp_destroy.restype = None
        self.sizes = (int(n_in), int(h1), int(h2), int(n_out))
        p = None
        if params is not None:
            p = torch.as_tensor(params, dtype=torch.float32).contiguous()
        h = ctypes.c_void_p()
        _call("gbk_mlp_create", *self.sizes, _ptr(p) if p is not None else None, ctypes.byref(h))
        self._h = h
        self.nparam = int(lib.gbk_mlp_num_params(h))
        if seed is not None:
            if params is not None:
                raise ValueError("give params or seed, not both")
            self.init_uniform(seed)

    def init_uniform(self, seed: int):
        """U(-1/sqrt(fan_in), 1/sqrt(fan_in)) parameters from a seeded hash (library kernel)."""
        _call("gbk_mlp_init_uniform", self._h, ctypes.c_uint64(int(seed)), _stream())
        return self

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.gbk_mlp_destroy(self._h)
            self._h = None

    def params(self):
        out = torch.empty(self.nparam, dtype=torch.float32, device="cuda")
        _call("gbk_mlp_params", self._h, _ptr(out), None, _stream())
        return out

    def grads(self):
        out = torch.empty(self.nparam, dtype=torch.float32, device="cuda")
        _call("gbk_mlp_params", self._h, None, _ptr(out), _stream())
        return out

    def forward(self, X: torch.Tensor):
        _dev(X, torch.float32, "X")
        B = X.shape[0]
        z = torch.empty((B, self.sizes[3]), dtype=torch.float32, device=X.device)
        cls = torch.empty(B, dtype=torch.int32, device=X.device)
        _call("gbk_mlp_forward", self._h, _ptr(X), B, _ptr(z), _ptr(cls), _stream())
        return z, cls

    def train_step(self, X: torch.Tensor, labels: torch.Tensor, lr: float = 1e-3,
                   update: bool = True):
        _dev(X, torch.float32, "X")
        _dev(labels, torch.int32, "labels")
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        _call("gbk_mlp_train_step", self._h, _ptr(X), _ptr(labels), X.shape[0], float(lr),
              int(bool(update)), _ptr(loss), _stream())
        return loss


class NprobeTrainOpts(ctypes.Structure):
    _fields_ = [("n_classes", ctypes.c_int32), ("k", ctypes.c_int32), ("target", ctypes.c_float),
                ("kprime", ctypes.c_int32), ("epochs", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("lr", ctypes.c_float), ("seed", ctypes.c_uint64), ("chunk", ctypes.c_int64)]


def _nprobe_opts(n_classes=9, k=10, target=0.95, kprime=0, epochs=15, batch=4096, lr=1e-3,
                 seed=0, chunk=20000):
    return NprobeTrainOpts(int(n_classes), int(k), float(target), int(kprime), int(epochs),
                           int(batch), float(lr), int(seed), int(chunk))


def nprobe_labels(index, xq, gt=None, counts=False, **opts):
    """Labels of training queries for the nprobe network (smallest class reaching the recall
    target), from exact neighbours gt [n][>=k] or the index's kept vectors.  Returns labels
    [n] int32 (and the recall counts [n_classes][n] with counts=True)."""
    _dev(xq, torch.float32, "xq")
    o = _nprobe_opts(**opts)
    n = xq.shape[0]
    lab = torch.empty(n, dtype=torch.int32, device=xq.device)
    cnt = torch.empty((o.n_classes, n), dtype=torch.int32, device=xq.device) if counts else None
    kgt = 0
    if gt is not None:
        _dev(gt, torch.int64, "gt")
        kgt = gt.shape[1]
    _call("gbk_nprobe_labels", index._h, _ptr(xq), n, _ptr(gt), int(kgt), ctypes.byref(o),
          _ptr(lab), _ptr(cnt), _stream())
    return (lab, cnt) if counts else lab


def nprobe_mlp_train(index, net, xq, labels=None, gt=None, **opts):
    """Trains net on the training queries xq inside the library (features, labels if not
    given, seeded epochs of Adam).  Returns the mean batch loss of each epoch."""
    import numpy as np
    _dev(xq, torch.float32, "xq")
    if labels is not None:
        _dev(labels, torch.int32, "labels")
    kgt = 0
    if gt is not None:
        _dev(gt, torch.int64, "gt")
        kgt = gt.shape[1]
    o = _nprobe_opts(n_classes=net.sizes[3], **opts)
    loss = np.zeros(o.epochs, np.float32)
    _call("gbk_nprobe_mlp_train", index._h, net._h, _ptr(xq), xq.shape[0], _ptr(labels),
          _ptr(gt), int(kgt), ctypes.byref(o), loss.ctypes.data_as(_vp), _stream())
    return loss


_SIGNATURES.update({
    "gbk_mlp_init_uniform": [_vp, ctypes.c_uint64, _vp],
    "gbk_ivfpq_save": [_vp, ctypes.c_char_p, _vp],
    "gbk_ivfpq_train_rotation": [_vp, _vp, _i64, _vp, _vp, _vp],
    "gbk_ivfpq_load": [ctypes.c_char_p, _vp, _vp],
    "gbk_nprobe_labels": [_vp, _vp, _i64, _vp, _i32, _vp, _vp, _vp, _vp],
    "gbk_nprobe_mlp_train": [_vp, _vp, _vp, _i64, _vp, _vp, _i32, _vp, _vp, _vp],
    "gbk_recall_counts": [_vp, _vp, _i64, _i32, _i32, _vp, _vp],
    "gbk_nprobe_features": [_vp, _i64, _i32, _vp, _i32, _i32, _vp, _vp],
    "gbk_ivfpq_search_batched": [_vp, _vp, _i64, _vp, _i32, _vp, _i32, _vp, _vp, _vp, _vp, _vp,
                                 _vp],
    "gbk_ivfpq_search_batched_refine": [_vp, _vp, _i64, _i32, _i32, _vp, _i32, _vp, _vp, _vp,
                                        _vp, _vp],
    "gbk_ivfpq_batched_graph": [_vp, _vp, _i64, _vp, _i32, _vp, _i32, _vp, _vp, _vp, _vp, _vp,
                                _vp, _vp],
    "gbk_graph_launch": [_vp, _vp],
    "gbk_ivfpq_knn_graph": [_vp, _vp, _i64, _vp, _i32, _i32, _vp, _i64, _vp, _vp, _vp],
    "gbk_ivfpq_knn_graph_refine": [_vp, _vp, _i64, _vp, _i32, _i32, _i32, _vp, _i64, _vp,
                                   _vp, _vp],
    "gbk_merge_topk": [_vp, _vp, _i32, _i64, _i32, _i32, _i32, _vp, _vp, _vp],
    "gbk_ivfpq_set_tuning": [_vp, _i32, _i32],
    "gbk_ivfpq_get_tuning": [_vp, _vp, _vp],
    "gbk_ivfpq_set_scan_options": [_vp, _i32, _i32],
    "gbk_ivfpq_set_learned_route": [_vp, ctypes.c_float, _i32],
    "gbk_ivfpq_autotune": [_vp, _vp, _i64, _vp, _i32, _vp, _i32, _vp, _vp, _vp, _vp, _i32, _vp,
                           _vp],
})


def merge_topk(D_parts: torch.Tensor, I_parts: torch.Tensor, k: int, largest: bool = False):
    """k best per query of stacked partial results [nparts][nq][k_in] (value, then id)."""
    _dev(D_parts, torch.float32, "D_parts")
    _dev(I_parts, torch.int64, "I_parts")
    nparts, nq, kin = D_parts.shape
    D = torch.empty((nq, k), dtype=torch.float32, device=D_parts.device)
    I = torch.empty((nq, k), dtype=torch.int64, device=D_parts.device)
    _call("gbk_merge_topk", _ptr(D_parts), _ptr(I_parts), int(nparts), nq, int(kin), int(k),
          int(bool(largest)), _ptr(D), _ptr(I), _stream())
    return D, I


def ivfpq_set_tuning(index, codes_per_thread: int, blocks_per_sm: int):
    _call("gbk_ivfpq_set_tuning", index._h, int(codes_per_thread), int(blocks_per_sm))


def ivfpq_set_learned_route(index, alpha: float = 0.0, shift: int = 0):
    """Learned nprobe operating point: class = argmax (alpha 0) or the smallest class of
    cumulative probability >= alpha; class c probes 2^max(c + shift, 0) lists."""
    _call("gbk_ivfpq_set_learned_route", index._h, float(alpha), int(shift))


def ivfpq_set_scan_options(index, threads: int = 384, by_list: bool = False):
    """Table-mode scan block size (256 or 512) and whether a plain search scans its queries
    in the order of their nearest list (True) or as given."""
    _call("gbk_ivfpq_set_scan_options", index._h, int(threads), int(bool(by_list)))


def ivfpq_get_tuning(index):
    u, b = ctypes.c_int32(), ctypes.c_int32()
    _call("gbk_ivfpq_get_tuning", index._h, ctypes.byref(u), ctypes.byref(b))
    return u.value, b.value


def ivfpq_autotune(index, xq, k_per_q, max_k, nprobe_per_q=None, max_nprobe=256, mlp=None,
                   reps=3):
    """Time the mixed-batch search over the scan's launch shapes and keep the fastest in the
    index.  Returns ((codes_per_thread, blocks_per_sm), ms per batch)."""
    nq, kq, off, D, I, used, npq = _batched_args(index, xq, k_per_q, max_k, nprobe_per_q,
                                                 max_nprobe, mlp)
    ms = ctypes.c_float()
    _call("gbk_ivfpq_autotune", index._h, _ptr(xq), nq, _ptr(kq), int(max_k), _ptr(npq),
          int(max_nprobe), mlp._h if mlp is not None else None, _ptr(off), _ptr(D), _ptr(I),
          int(reps), ctypes.byref(ms), _stream())
    return ivfpq_get_tuning(index), ms.value


def recall_counts(I: torch.Tensor, G: torch.Tensor, out: torch.Tensor):
    """out[q] = |{I[q][i]} intersect {G[q][j]}| (ids; -1 entries ignored)."""
    _dev(I, torch.int64, "I")
    _dev(G, torch.int64, "G")
    _call("gbk_recall_counts", _ptr(I), _ptr(G), I.shape[0], I.shape[1], G.shape[1], _ptr(out),
          _stream())
    return out


def nprobe_features(xq: torch.Tensor, coarse_dist: torch.Tensor, nfeat: int = 64):
    """[x, d_i / d_0 - 1 for the nfeat nearest coarse distances] per query."""
    nq, d = xq.shape
    F = torch.empty((nq, d + nfeat), dtype=torch.float32, device=xq.device)
    _call("gbk_nprobe_features", _ptr(xq), nq, int(d), _ptr(coarse_dist),
          coarse_dist.shape[1], int(nfeat), _ptr(F), _stream())
    return F


def _batched_args(index, xq, k_per_q, max_k, nprobe_per_q, max_nprobe, mlp):
    nq = xq.shape[0]
    k_per_q = k_per_q.to(torch.int32).contiguous()
    off = torch.zeros(nq + 1, dtype=torch.int64, device=xq.device)
    off[1:] = torch.cumsum(k_per_q.to(torch.int64), 0)
    total = int(off[-1].item())
    D = torch.empty(total, dtype=torch.float32, device=xq.device)
    I = torch.empty(total, dtype=torch.int64, device=xq.device)
    used = torch.empty(nq, dtype=torch.int32, device=xq.device)
    npq = nprobe_per_q.to(torch.int32).contiguous() if nprobe_per_q is not None else None
    return nq, k_per_q, off, D, I, used, npq


def ivfpq_search_batched(index, xq, k_per_q, max_k, nprobe_per_q=None, max_nprobe=256, mlp=None):
    """Mixed batch: per-query k (and nprobe, or nprobe chosen by a trained MLP).  Returns
    (D, I, offsets, nprobe_used): results of query q are D/I[offsets[q]:offsets[q+1]]."""
    nq, kq, off, D, I, used, npq = _batched_args(index, xq, k_per_q, max_k, nprobe_per_q,
                                                 max_nprobe, mlp)
    _call("gbk_ivfpq_search_batched", index._h, _ptr(xq), nq, _ptr(kq), int(max_k), _ptr(npq),
          int(max_nprobe), mlp._h if mlp is not None else None, _ptr(off), _ptr(D), _ptr(I),
          _ptr(used), _stream())
    return D, I, off, used


def ivfpq_search_batched_refine(index, xq, k, kprime, nprobe_per_q=None, max_nprobe=256,
                                mlp=None):
    """Batched search (per-query nprobe, or chosen by a trained MLP) of kprime ADC candidates
    re-ranked by exact float32 distances to the kept vectors.  Returns (D, I, nprobe_used)."""
    _dev(xq, torch.float32, "xq")
    nq = xq.shape[0]
    D = torch.empty((nq, k), dtype=torch.float32, device=xq.device)
    I = torch.empty((nq, k), dtype=torch.int64, device=xq.device)
    used = torch.empty(nq, dtype=torch.int32, device=xq.device)
    npq = nprobe_per_q.to(torch.int32).contiguous() if nprobe_per_q is not None else None
    _call("gbk_ivfpq_search_batched_refine", index._h, _ptr(xq), nq, int(k), int(kprime),
          _ptr(npq), int(max_nprobe), mlp._h if mlp is not None else None, _ptr(D), _ptr(I),
          _ptr(used), _stream())
    return D, I, used


def knn_graph(index, x, k, nprobe, mlp=None, self_ids=None, batch=0, distances=True, kprime=0):
    """k-NN graph (section 6.5): each row of x searched for k+1 neighbours, its own id
    (self_ids[i], default i) removed; kprime > k re-ranks that many ADC candidates by exact
    distances to the kept vectors.  Returns (GD, G) [n][k] (GD None if not requested)."""
    _dev(x, torch.float32, "x")
    n = x.shape[0]
    G = torch.empty((n, k), dtype=torch.int64, device=x.device)
    GD = torch.empty((n, k), dtype=torch.float32, device=x.device) if distances else None
    sid = self_ids.to(torch.int64).contiguous() if self_ids is not None else None
    h = mlp._h if mlp is not None else None
    if kprime:
        _call("gbk_ivfpq_knn_graph_refine", index._h, _ptr(x), n, _ptr(sid), int(k), int(nprobe),
              int(kprime), h, int(batch), _ptr(GD), _ptr(G), _stream())
    else:
        _call("gbk_ivfpq_knn_graph", index._h, _ptr(x), n, _ptr(sid), int(k), int(nprobe), h,
              int(batch), _ptr(GD), _ptr(G), _stream())
    return GD, G


class BatchedGraph:
    """A captured CUDA graph of one mixed-batch search over fixed buffers; launch() replays
    it (new query contents may be written into `xq` between launches)."""

    def __init__(self, index, xq, k_per_q, max_k, nprobe_per_q=None, max_nprobe=256, mlp=None):
        lib = load()
        lib.gbk_graph_destroy.argtypes = [_vp]
        lib.gbk_graph_destroy.restype = None
        nq, kq, off, D, I, used, npq = _batched_args(index, xq, k_per_q, max_k, nprobe_per_q,
                                                     max_nprobe, mlp)
        self._keep = (index, xq, kq, off, npq, mlp)
        self.D, self.I, self.offsets, self.nprobe_used = D, I, off, used
        h = ctypes.c_void_p()
        _call("gbk_ivfpq_batched_graph", index._h, _ptr(xq), nq, _ptr(kq), int(max_k), _ptr(npq),
              int(max_nprobe), mlp._h if mlp is not None else None, _ptr(off), _ptr(D), _ptr(I),
              _ptr(used), ctypes.byref(h), _stream())
        self._h = h

    def launch(self):
        _call("gbk_graph_launch", self._h, _stream())

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.gbk_graph_destroy(self._h)
            self._h = None
