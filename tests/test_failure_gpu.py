"""Failure detection without a GPU fault.

* A bounded device-side wait that nothing satisfies gives up after its limit, sets the
  status word and returns: gbk_device_status reports GBK_ETIMEOUT (4) once, the context
  stays usable and later calls are exact.
* The scratch-allocator hook: an allocator that fails makes every entry point that needs
  scratch memory return GBK_ENOMEM (2) before or between launches, with nothing leaked or
  left behind that changes later results; failing the n-th allocation of an IVFADC search
  for every n up to its count exercises each allocation site."""
import numpy as np
import pytest
import torch

from paper_1702_08734_gb300 import datagen

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(gbk):
    v = torch.from_numpy(datagen.uniform_matrix(5, 64, 3000)).cuda()
    D0, I0 = gbk.kselect(v, 16)
    gbk.selftest_wait_timeout(2000000)  # 2 ms
    with pytest.raises(gbk.GbkError) as e:
        gbk.device_status()
    assert e.value.status == 4
    gbk.device_status()  # reported once, then cleared
    D1, I1 = gbk.kselect(v, 16)
    assert torch.equal(D0, D1) and torch.equal(I0, I1)
    with pytest.raises(gbk.GbkError):
        gbk.selftest_wait_timeout(10)  # limit outside [1 us, 2 s]


class _Counting:
    """torch-backed allocator that fails the n-th request (n = None: never)."""

    def __init__(self, fail_at=None):
        self.fail_at, self.calls, self.live = fail_at, 0, set()

    def alloc(self, n, st):
        self.calls += 1
        if self.fail_at is not None and self.calls == self.fail_at:
            return 0
        p = torch.cuda.caching_allocator_alloc(n)
        self.live.add(p)
        return p

    def free(self, p, st):
        self.live.discard(p)
        torch.cuda.caching_allocator_delete(p)


def test_failing_allocator_gives_enomem(gbk):
    v = torch.from_numpy(datagen.uniform_matrix(6, 32, 200000)).cuda()
    ref = gbk.kselect(v, 64, segments=8)
    try:
        gbk.set_allocator(lambda n, st: 0)
        with pytest.raises(gbk.GbkError) as e:
            gbk.kselect(v, 64, segments=8)  # the segment partials need scratch
        assert e.value.status == 2
    finally:
        gbk.set_allocator(None)
    out = gbk.kselect(v, 64, segments=8)
    assert torch.equal(out[0], ref[0]) and torch.equal(out[1], ref[1])


def test_every_allocation_site_of_a_search_fails_cleanly(gbk):
    cen = datagen.mixture_centres(7, 64, 32)
    x = torch.from_numpy(datagen.mixture_points(cen, 8, 20000)).cuda()
    xq = torch.from_numpy(datagen.mixture_points(cen, 9, 300)).cuda()
    ix = gbk.IVFPQIndex(32, 64, 8)
    ix.train(x, niter=4, coarse_init=datagen.permutation_prefix(10, 20000, 64),
             pq_init=datagen.permutation_prefix(11, 20000, 256))
    ix.add(x)
    D0, I0 = ix.search(xq, 20, 8)
    torch.cuda.synchronize()
    counter = _Counting()
    try:
        gbk.set_allocator(counter.alloc, counter.free)
        D1, I1 = ix.search(xq, 20, 8)
        torch.cuda.synchronize()
        n = counter.calls
        assert n >= 3 and not counter.live  # everything freed again
        assert torch.equal(D1, D0) and torch.equal(I1, I0)
        for fail in range(1, n + 1):
            c = _Counting(fail)
            gbk.set_allocator(c.alloc, c.free)
            with pytest.raises(gbk.GbkError) as e:
                ix.search(xq, 20, 8)
            assert e.value.status == 2
            torch.cuda.synchronize()
            assert not c.live, fail
    finally:
        gbk.set_allocator(None)
    D2, I2 = ix.search(xq, 20, 8)
    assert torch.equal(D2, D0) and torch.equal(I2, I0)
    gbk.device_status()
