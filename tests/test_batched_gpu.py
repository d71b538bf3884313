"""Mixed-batch IVFADC search (per-query k and nprobe in one persistent launch), its CUDA
graph replay, and nprobe chosen by the learned network.

A mixed batch must return, for every query, exactly what a plain search with that query's
own k and nprobe returns (same arithmetic; the coarse list for the largest nprobe starts
with the lists of any smaller nprobe)."""
import numpy as np
import pytest
import torch

from paper_1702_08734_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def index(gbk):
    cen = datagen.mixture_centres(70, 256, 64)
    x = torch.from_numpy(datagen.mixture_points(cen, 71, 60000)).cuda()
    ix = gbk.IVFPQIndex(64, 128, 16)
    ix.train(x[:20000], niter=8, coarse_init=datagen.permutation_prefix(72, 20000, 128),
             pq_init=datagen.permutation_prefix(73, 20000, 256))
    ix.add(x)
    xq = torch.from_numpy(datagen.mixture_points(cen, 74, 700)).cuda()
    return ix, xq


def _mixed(nq, seed):
    k = torch.from_numpy(np.array([1, 10, 100])[datagen.randint(seed, 0, nq, 3)]).cuda()
    npb = torch.from_numpy(np.array([8, 32, 128])[datagen.randint(seed, 0, nq, 3, stream=1)]).cuda()
    return k.to(torch.int32), npb.to(torch.int32)


def _check_against_plain(ix, xq, kq, npq, D, I, off):
    kq_h, np_h, off_h = kq.cpu().numpy(), npq.cpu().numpy(), off.cpu().numpy()
    Dh, Ih = D.cpu().numpy(), I.cpu().numpy()
    for kk in (1, 10, 100):
        for nn in (8, 32, 128):
            sel = np.nonzero((kq_h == kk) & (np_h == nn))[0]
            if sel.size == 0:
                continue
            Dp, Ip = ix.search(xq[torch.from_numpy(sel).cuda()], kk, nn)
            Dp, Ip = Dp.cpu().numpy(), Ip.cpu().numpy()
            for r, q in enumerate(sel):
                np.testing.assert_array_equal(Ih[off_h[q]:off_h[q + 1]], Ip[r])
                np.testing.assert_array_equal(Dh[off_h[q]:off_h[q + 1]], Dp[r])


def test_mixed_batch_equals_per_query_searches(gbk, index):
    ix, xq = index
    kq, npq = _mixed(xq.shape[0], 75)
    D, I, off, used = gbk.ivfpq_search_batched(ix, xq, kq, 100, npq, 128)
    assert torch.equal(used, npq)
    _check_against_plain(ix, xq, kq, npq, D, I, off)


def test_graph_replay_matches_and_follows_new_queries(gbk, index):
    ix, xq = index
    kq, npq = _mixed(xq.shape[0], 76)
    buf = xq.clone()
    gr = gbk.BatchedGraph(ix, buf, kq, 100, npq, 128)
    for it in range(2):
        if it == 1:  # new query contents in the captured buffer
            buf.copy_(xq.flip(0))
        gr.launch()
        torch.cuda.synchronize()
        _check_against_plain(ix, buf, kq, npq, gr.D, gr.I, gr.offsets)


def test_learned_nprobe_routing(gbk, index):
    ix, xq = index
    from oracle import mlp as omlp  # initial weights only (seeded uniforms)
    n = 256 * 128 + 256 + 256 * 256 + 256 + 9 * 256 + 9
    p = omlp.init_params((128, 256, 256, 9), datagen.uniform24(77, 0, n).astype(np.float64))
    flat = np.concatenate([p[k].ravel() for k in omlp.PARAM_NAMES]).astype(np.float32)
    net = gbk.MLP(128, 256, 256, 9, params=flat)
    kq = torch.full((xq.shape[0],), 10, dtype=torch.int32, device="cuda")
    D, I, off, used = gbk.ivfpq_search_batched(ix, xq, kq, 10, None, 128, mlp=net)
    u = used.cpu().numpy()
    assert np.all((u >= 1) & (u <= 128) & ((u & (u - 1)) == 0))
    # the same routing given explicitly reproduces the results
    D2, I2, _, _ = gbk.ivfpq_search_batched(ix, xq, kq, 10, used, 128)
    assert torch.equal(I, I2) and torch.equal(D, D2)


def test_launch_shapes_do_not_change_results(gbk, index):
    ix, xq = index
    kq, npq = _mixed(xq.shape[0], 78)
    ref = None
    for u, b in ((4, 2), (2, 1), (8, 4), (8, 1), (2, 3)):
        gbk.ivfpq_set_tuning(ix, u, b)
        assert gbk.ivfpq_get_tuning(ix) == (u, b)
        D, I, off, _ = gbk.ivfpq_search_batched(ix, xq, kq, 100, npq, 128)
        Dp, Ip = ix.search(xq, 10, 32)
        if ref is None:
            ref = (D, I, Dp, Ip)
        else:
            assert torch.equal(ref[1], I) and torch.equal(ref[0], D)
            assert torch.equal(ref[3], Ip) and torch.equal(ref[2], Dp)
    gbk.ivfpq_set_tuning(ix, 4, 2)
    for u, b in ((3, 2), (4, 0), (4, 9)):
        with pytest.raises(gbk.GbkError):
            gbk.ivfpq_set_tuning(ix, u, b)


def test_autotune_keeps_a_valid_shape(gbk, index):
    ix, xq = index
    kq, npq = _mixed(xq.shape[0], 79)
    (u, b), ms = gbk.ivfpq_autotune(ix, xq, kq, 100, npq, 128, reps=2)
    assert u in (2, 4, 8) and 1 <= b <= 4 and ms > 0
    D, I, off, used = gbk.ivfpq_search_batched(ix, xq, kq, 100, npq, 128)
    _check_against_plain(ix, xq, kq, npq, D, I, off)
    gbk.ivfpq_set_tuning(ix, 4, 2)
