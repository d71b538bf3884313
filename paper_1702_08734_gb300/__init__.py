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
    "gbk_row_norms": [_vp, _i64, _i32, _vp, _vp],
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
            lib.gbk_version.restype = ctypes.c_int32
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


def kselect(vals: torch.Tensor, k: int, largest: bool = False, out=None):
    """Row-wise k smallest (largest) values and their int64 indices, sorted best first."""
    _dev(vals, torch.float32, "vals")
    if vals.dim() != 2:
        raise ValueError("vals must be 2-D")
    rows, length = vals.shape
    if out is None:
        D = torch.empty((rows, k), dtype=torch.float32, device=vals.device)
        I = torch.empty((rows, k), dtype=torch.int64, device=vals.device)
    else:
        D, I = out
    _call("gbk_kselect", _ptr(vals), rows, length, int(k), int(bool(largest)), _ptr(D), _ptr(I),
          _stream())
    return D, I


def row_norms(x: torch.Tensor, out=None):
    """Squared L2 norm of every row of x (float32)."""
    _dev(x, torch.float32, "x")
    n, d = x.shape
    o = torch.empty(n, dtype=torch.float32, device=x.device) if out is None else out
    _call("gbk_row_norms", _ptr(x), n, int(d), _ptr(o), _stream())
    return o
