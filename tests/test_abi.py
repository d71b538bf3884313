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
