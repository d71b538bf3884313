"""IVFADC on the GPU vs the oracle.

* k-means: same initial rows -> same centroids (member sums in the same order and
  precision; well-separated data so that no assignment is a near-tie).
* encoding: given the same quantizers, lists are bit-exact and codes bit-exact except
  argmin near-ties (checked to be ties within 1e-5 relative in float64).
* search: given the same index, ADC distances within 1e-4 relative (float32 tables through
  the term decomposition of Eq. 11) and the same ids except near-ties; padding when the
  probed lists hold fewer than k vectors; every list probed = exhaustive ADC."""
import numpy as np
import pytest
import torch

import oracle
from paper_1702_08734_gb300 import datagen

pytestmark = pytest.mark.gpu


def _mixture(seed, n, d, ncent=64, std=2.0):
    cen = datagen.mixture_centres(seed, ncent, d, std)
    return datagen.mixture_points(cen, seed + 1, n), cen


@pytest.mark.parametrize("d,nc,direct", [(16, 20, True), (8, 256, True), (128, 64, False),
                                         (96, 50, False)])
def test_kmeans_matches_oracle(gbk, d, nc, direct):
    x, _ = _mixture(10 + d, 6000, d, ncent=nc, std=6.0)
    init = datagen.permutation_prefix(11 + d, x.shape[0], nc)
    c, obj, _ = gbk.kmeans(torch.from_numpy(x).cuda(), init, 8, direct=direct)
    co, objo, _ = oracle.kmeans(x, init, 8)
    np.testing.assert_allclose(c.cpu().numpy(), co, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(obj, objo, rtol=1e-4)


@pytest.mark.parametrize("d,direct", [(32, False), (16, True)])
def test_kmeans_segmented_update_matches_oracle(gbk, d, direct):
    # few large clusters: each cluster's member sum is split into segments added in order;
    # the double sums then differ from the oracle's sequential ones far below float32
    # one initial row per mixture component: every assignment is far from a tie
    x, _ = _mixture(30 + d, 200000, d, ncent=8, std=8.0)
    u = datagen.randint(31 + d, 0, x.shape[0], 8, stream=0)
    init = np.array([int(np.argmax(u == c)) for c in range(8)])
    c, obj, _ = gbk.kmeans(torch.from_numpy(x).cuda(), init, 3, direct=direct)
    co, objo, _ = oracle.kmeans(x, init, 3)
    np.testing.assert_allclose(c.cpu().numpy(), co, rtol=1e-6, atol=1e-6)
    # the objective sums the assignment's float32 distances, formed as ||x||^2 + ||c||^2 -
    # 2<x,c> (Eq. 2): cancellation against norms ~60x the distances costs ~1e-5 relative
    np.testing.assert_allclose(obj, objo, rtol=1e-4)


@pytest.mark.parametrize("direct", [True, False])
def test_kmeans_empty_cluster_rule_matches_oracle(gbk, direct):
    # Duplicate initial rows tie exactly, so the lowest centroid takes every point and the
    # others are re-seeded by the split rule.  One iteration: the split is exact float64
    # arithmetic on both sides (later iterations would meet genuine near-ties, since a
    # split leaves two centroids 2/1024 apart).
    d = 16 if direct else 64
    x, _ = _mixture(20, 3000, d, ncent=10, std=8.0)
    init = np.array([0, 0, 0, 5, 9, 9, 100, 101, 102, 103])
    c, _, ns = gbk.kmeans(torch.from_numpy(x).cuda(), init, 1, direct=direct)
    co, _, nso = oracle.kmeans(x, init, 1)
    assert ns == nso == 3
    np.testing.assert_allclose(c.cpu().numpy(), co, rtol=1e-6, atol=1e-6)


def _index_with_oracle_quantizers(gbk, seed, n=20000, d=32, nlist=16, M=8, precomputed=True):
    x, cen = _mixture(seed, n, d)
    nt = min(4000, n)
    coarse, _, _ = oracle.kmeans(x[:nt], datagen.permutation_prefix(seed + 2, nt, nlist), 6)
    res = oracle.residual_training_set(x[:nt], coarse)
    books = oracle.train_pq(res, M, datagen.permutation_prefix(seed + 3, nt, 256), 6)
    ix = gbk.IVFPQIndex(d, nlist, M)
    ix.set_quantizers(torch.from_numpy(coarse).cuda(), torch.from_numpy(books).cuda(),
                      use_precomputed=precomputed)
    ix.add(torch.from_numpy(x).cuda())
    return ix, x, coarse, books


@pytest.mark.parametrize("d,M", [(64, 4), (64, 8), (64, 16), (64, 32), (64, 64), (96, 12),
                                 (96, 24), (96, 48), (120, 20), (120, 60)])
def test_encode_and_lists_match_oracle(gbk, d, M):
    ix, x, coarse, books = _index_with_oracle_quantizers(gbk, 30 + M, d=d, M=M)
    ex = ix.export()
    lists, codes = oracle.ivfpq_encode(x, coarse, books)
    off, order = oracle.ivf_bucket(lists, coarse.shape[0])
    np.testing.assert_array_equal(ex["list_off"], off)
    np.testing.assert_array_equal(ex["ids"], order)
    mism = np.argwhere(ex["codes"] != codes[order])
    assert len(mism) <= max(2, codes.size // 100000), len(mism)
    dsub = d // M
    for j, m in mism:  # each mismatch must be an argmin near-tie
        v = order[j]
        r = x[v].astype(np.float64) - coarse[lists[v]].astype(np.float64)
        sub = r[m * dsub:(m + 1) * dsub]
        eg = books[m, ex["codes"][j, m]].astype(np.float64) - sub
        eo = books[m, codes[v, m]].astype(np.float64) - sub
        dg, do = (eg ** 2).sum(), (eo ** 2).sum()
        # the encoder rounds the residual and each difference to float32 (u = 2^-24) before
        # squaring: each distance is within 2 |e| u (|r| + |e|) per coordinate (2u: margin),
        # which dominates for one-coordinate sub-vectors with tiny distances
        u = 2.0 ** -23
        tol = sum((2 * np.abs(e) * u * (np.abs(sub) + np.abs(e))).sum() for e in (eg, eo))
        assert abs(dg - do) <= 1e-5 * max(do, 1e-12) + tol, (dg, do, tol)


def _check_search(D, I, Do, Io, rtol=1e-4, Do_next=None):
    """Do_next: the oracle's (k+1)-th distances, so that a near-tie across the k-th place
    (the list's last entry against the first one left out) is recognised as one."""
    D = D.cpu().numpy().astype(np.float64)
    I = I.cpu().numpy()
    fin = np.isfinite(Do)
    assert np.array_equal(np.isfinite(D), fin)
    assert np.all(I[~fin] == -1)
    scale = np.maximum(np.abs(Do[fin]), 1e-2)
    assert np.all(np.abs(D[fin] - Do[fin]) <= rtol * scale + 1e-4), np.abs(D[fin] - Do[fin]).max()
    gap = np.full(Do.shape, np.inf)
    dd = np.abs(np.diff(np.where(fin, Do, 1e30), axis=1))
    gap[:, 1:] = np.minimum(gap[:, 1:], dd)
    gap[:, :-1] = np.minimum(gap[:, :-1], dd)
    if Do_next is not None:
        gap[:, -1] = np.minimum(gap[:, -1], np.abs(np.where(np.isfinite(Do_next), Do_next, 1e30)
                                                   - np.where(fin[:, -1], Do[:, -1], 1e30)))
    sep = fin & (gap > 4 * rtol * np.maximum(np.abs(np.where(fin, Do, 0)), 1e-2))
    assert (I[sep] == Io[sep]).mean() > 0.999


@pytest.mark.parametrize("precomputed", [True, False])
@pytest.mark.parametrize("nprobe,k", [(1, 10), (4, 100), (16, 33), (16, 1024)])
def test_search_matches_oracle(gbk, precomputed, nprobe, k):
    ix, x, coarse, books = _index_with_oracle_quantizers(gbk, 40, precomputed=precomputed)
    ex = ix.export()
    xq, _ = _mixture(40, 300, 32)  # same mixture as the database
    xq = xq + datagen.gaussian_matrix(44, 300, 32) * 0.1
    D, I = ix.search(torch.from_numpy(xq).cuda(), k, nprobe)
    Do, Io = oracle.ivfadc_search(xq, coarse, books, ex["list_off"], ex["codes"], ex["ids"], k,
                                  nprobe)
    _check_search(D, I, Do, Io)


@pytest.mark.parametrize("M", [4, 32])
@pytest.mark.parametrize("nprobe,k", [(2, 10), (8, 100)])
def test_search_other_code_sizes_match_oracle(gbk, M, nprobe, k):
    # 4-byte codes (8 LUT copies per warp row) and 32-byte codes against the oracle
    ix, x, coarse, books = _index_with_oracle_quantizers(gbk, 45 + M, M=M)
    ex = ix.export()
    xq, _ = _mixture(45 + M, 300, 32)
    xq = xq + datagen.gaussian_matrix(46, 300, 32) * 0.1
    D, I = ix.search(torch.from_numpy(xq).cuda(), k, nprobe)
    Do, Io = oracle.ivfadc_search(xq, coarse, books, ex["list_off"], ex["codes"], ex["ids"],
                                  k + 1, nprobe)
    _check_search(D, I, Do[:, :k], Io[:, :k], Do_next=Do[:, k])


def test_full_probe_is_exhaustive_adc_and_padding(gbk):
    ix, x, coarse, books = _index_with_oracle_quantizers(gbk, 50, n=3000, nlist=16)
    ex = ix.export()
    xq = x[:50]
    D, I = ix.search(torch.from_numpy(xq).cuda(), 40, 16)
    Do, Io = oracle.ivfadc_search(xq, coarse, books, ex["list_off"], ex["codes"], ex["ids"], 40, 16)
    _check_search(D, I, Do, Io)
    # one probed list with fewer than k members pads with (+inf, -1)
    D1, I1 = ix.search(torch.from_numpy(xq).cuda(), 1000, 1)
    Do1, Io1 = oracle.ivfadc_search(xq, coarse, books, ex["list_off"], ex["codes"], ex["ids"],
                                    1000, 1)
    _check_search(D1, I1, Do1, Io1)
    assert (I1.cpu().numpy() == -1).any()


def test_train_add_search_end_to_end(gbk):
    x, cen = _mixture(60, 30000, 64, ncent=128)
    xt = torch.from_numpy(x).cuda()
    ix = gbk.IVFPQIndex(64, 64, 16)
    ix.train(xt, niter=10, coarse_init=datagen.permutation_prefix(61, 30000, 64),
             pq_init=datagen.permutation_prefix(62, 30000, 256))
    ix.add(xt)
    assert ix.ntotal == 30000
    ex = ix.export()
    # the oracle, given the GPU-trained quantizers, assigns the same lists
    lists, _ = oracle.ivfpq_encode(x[:2000], ex["coarse"], ex["pq"])
    pos = np.argsort(ex["ids"])
    glist = np.searchsorted(ex["list_off"], pos, side="right") - 1
    assert (glist[:2000] == lists).mean() > 0.999
    # recall of the true nearest neighbour grows with nprobe
    xq = x[:200] + datagen.gaussian_matrix(63, 200, 64) * 0.05
    _, Ie = oracle.knn(xq, x, 1)
    r = []
    for nprobe in (1, 8, 64):
        _, I = ix.search(torch.from_numpy(xq).cuda(), 10, nprobe)
        r.append((I.cpu().numpy() == Ie).any(1).mean())
    assert r[0] <= r[1] <= r[2] and r[2] > 0.9, r


def test_errors(gbk):
    with pytest.raises(gbk.GbkError):
        gbk.IVFPQIndex(30, 8, 16)  # M does not divide d
    ix = gbk.IVFPQIndex(32, 8, 8)
    with pytest.raises(gbk.GbkError):
        ix.search(torch.zeros((2, 32), device="cuda"), 5, 2)  # not trained


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_low_precision_coarse_search(gbk, prec):
    # pattern 1 on the coarse quantizer: low-precision GEMM, over-fetched lists re-ranked in
    # float32 - the probed lists and term 2 equal the float32 search's for nearly every
    # query, so the results do too; batched and plain searches agree with each other
    ix, x, coarse, books = _index_with_oracle_quantizers(gbk, 70, nlist=64)
    xq, _ = _mixture(70, 400, 32)
    xqt = torch.from_numpy(xq + datagen.gaussian_matrix(71, 400, 32) * 0.1).cuda()
    D32, I32 = ix.search(xqt, 20, 8)
    ix.set_coarse_precision(prec)
    D, I = ix.search(xqt, 20, 8)
    same = (I == I32).all(dim=1).float().mean().item()
    assert same > 0.97, same
    # term 2 comes from the exact re-rank (sum of squared differences) instead of Eq. 2's
    # norm expansion: the distances differ by float32 rounding of the latter
    agree = torch.isclose(D, D32, rtol=1e-4, atol=1e-3).all(dim=1)
    assert agree.float().mean().item() > 0.97
    kq = torch.full((400,), 20, dtype=torch.int32, device="cuda")
    npq = torch.full((400,), 8, dtype=torch.int32, device="cuda")
    Db, Ib, _, _ = gbk.ivfpq_search_batched(ix, xqt, kq, 20, npq, 8)
    assert torch.equal(Ib.view(400, 20), I) and torch.equal(Db.view(400, 20), D)
    ix.set_coarse_precision("fp32")
    D2, I2 = ix.search(xqt, 20, 8)
    assert torch.equal(I2, I32) and torch.equal(D2, D32)
