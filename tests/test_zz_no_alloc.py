"""gbk_kselect_static: the k-selection entry point that makes no allocation.

It serves callers that cannot allocate device memory during a call (graph capture on a
pool they do not own, allocation-free latency paths, hosts with their own allocator): the
row-split selection keeps its partial results in a fixed device array instead of scratch.
Checked through the C ABI against gbk_kselect_ex with the same segment count, bit for bit
(the selection tests' tolerance), on two calls in a row with different inputs - the second
call must not see anything of the first one's partials - and for the capacity check.
Collected last (file name) so that a failure here does not hide other tests."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1702_08734_gb300 import datagen

pytestmark = pytest.mark.gpu


def _lib(gbk):
    lib = gbk.load()
    vp = ctypes.c_void_p
    lib.gbk_kselect_static.argtypes = [vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32, vp, vp, vp]
    lib.gbk_kselect_static.restype = ctypes.c_int32
    return lib


def _static(gbk, lib, v, k, largest, segments):
    rows, length = v.shape
    D = torch.empty((rows, k), dtype=torch.float32, device="cuda")
    I = torch.empty((rows, k), dtype=torch.int64, device="cuda")
    st = lib.gbk_kselect_static(ctypes.c_void_p(v.data_ptr()), rows, length, k, int(largest),
                                segments, ctypes.c_void_p(D.data_ptr()),
                                ctypes.c_void_p(I.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.gbk_last_error()
    return D, I


@pytest.mark.parametrize("rows,length,k,segments,largest", [
    (3, 1 << 20, 256, 0, False),   # library plan: rows split across many segments
    (50, 30011, 77, 7, True),      # explicit split, ragged segment tail
    (8, 200003, 1, 16, False),     # k = 1 partials
])
def test_static_matches_existing_entry_point_on_consecutive_calls(gbk, rows, length, k,
                                                                  segments, largest):
    lib = _lib(gbk)
    for call in range(2):
        v = torch.from_numpy(datagen.uniform_matrix(900 + 7 * call + k, rows, length)).cuda()
        Ds, Is = _static(gbk, lib, v, k, largest, segments)
        De, Ie = gbk.kselect(v, k, largest=largest, segments=segments)
        torch.cuda.synchronize()
        assert torch.equal(Is, Ie)
        np.testing.assert_array_equal(Ds.cpu().numpy().view(np.uint32),
                                      De.cpu().numpy().view(np.uint32))


def test_static_rejects_requests_beyond_its_capacity(gbk):
    lib = _lib(gbk)
    v = torch.zeros((64, 1 << 16), device="cuda")
    D = torch.empty((64, 1024), device="cuda")
    I = torch.empty((64, 1024), dtype=torch.int64, device="cuda")
    # 64 rows x 64 segments x 1024 = 2^22 partial results > 2^21
    st = lib.gbk_kselect_static(ctypes.c_void_p(v.data_ptr()), 64, 1 << 16, 1024, 0, 64,
                                ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(I.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 1
    assert b"capacity" in lib.gbk_last_error()
