"""The C-ABI library loads (no GPU needed) and exports every entry point its header declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gbk_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1702_08734_gb300 import buildlib as b
    path = b.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    d = _declared()
    assert "gbk_kselect" in d and "gbk_last_error" in d


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_argument_errors_need_no_gpu(lib):
    lib.gbk_kselect.restype = ctypes.c_int32
    lib.gbk_kselect.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.gbk_last_error.restype = ctypes.c_char_p
    assert lib.gbk_kselect(None, 4, 10, 0, 0, None, None, None) == 1
    assert b"k=0" in lib.gbk_last_error()
    assert lib.gbk_kselect(None, 4, 10, 11, 0, None, None, None) == 1
    assert lib.gbk_kselect(None, 4, 5000, 1025, 0, None, None, None) == 1
    assert lib.gbk_kselect(None, 0, 10, 3, 0, None, None, None) == 0
    lib.gbk_version.restype = ctypes.c_int32
    assert lib.gbk_version() >= 100


def test_index_argument_errors_need_no_gpu(lib):
    # index creation and option setters are host-side: their argument checks run anywhere
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    for name, args in (("gbk_ivfpq_create", [i32, i32, i32, i32, i32, vp]),
                       ("gbk_ivfflat_create", [i32, i32, i32, vp]),
                       ("gbk_ivfpq_set_coarse_precision", [vp, i32]),
                       ("gbk_ivfpq_keep_vectors", [vp, i32])):
        getattr(lib, name).restype = i32
        getattr(lib, name).argtypes = args
    lib.gbk_ivfpq_destroy.argtypes = [vp]
    lib.gbk_ivfflat_destroy.argtypes = [vp]
    h = ctypes.c_void_p()
    assert lib.gbk_ivfpq_create(30, 16, 8, 8, 0, ctypes.byref(h)) == 1   # M does not divide d
    assert lib.gbk_ivfpq_create(30, 16, 10, 8, 0, ctypes.byref(h)) == 5  # M not a multiple of 4
    assert lib.gbk_ivfpq_create(136, 16, 68, 8, 0, ctypes.byref(h)) == 5  # M above 64
    assert lib.gbk_ivfpq_create(36, 16, 12, 8, 0, ctypes.byref(h)) == 0  # 12-byte codes
    lib.gbk_ivfpq_destroy(h)
    assert lib.gbk_ivfpq_create(32, 16, 8, 8, 1, ctypes.byref(h)) == 5   # inner product
    assert lib.gbk_ivfpq_create(32, 16, 4, 8, 0, ctypes.byref(h)) == 0   # 4-byte codes
    assert lib.gbk_ivfpq_set_coarse_precision(h, 7) == 1
    assert lib.gbk_ivfpq_set_coarse_precision(h, 2) == 0
    assert lib.gbk_ivfpq_keep_vectors(h, 1) == 0
    lib.gbk_ivfpq_destroy(h)
    f = ctypes.c_void_p()
    assert lib.gbk_ivfflat_create(16, 4, 1, ctypes.byref(f)) == 5        # L2 only
    assert lib.gbk_ivfflat_create(0, 4, 0, ctypes.byref(f)) == 1
    assert lib.gbk_ivfflat_create(16, 4, 0, ctypes.byref(f)) == 0
    lib.gbk_ivfflat_destroy(f)
