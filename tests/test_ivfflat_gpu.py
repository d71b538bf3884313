"""IVF-Flat (inverted lists of float32 vectors, exact list scan) and IVFADC with exact
re-ranking from kept vectors, against the oracle.

The oracle takes the GPU's inverted file (its list offsets and list-order ids) as input, so
both sides scan the same lists; the GPU's list assignment is checked separately against the
oracle's exact nearest centroid (differences only at distance near-ties).  Distances are
float32 sums of d squared differences on the GPU and double sums in the oracle: relative
error below d * 2^-24 per term order, bounded here by 1e-5 relative + 1e-5 absolute.  Ids
agree exactly except where two candidates' distances are within that tolerance."""
import numpy as np
import pytest
import torch

import oracle
from paper_1702_08734_gb300 import datagen

pytestmark = pytest.mark.gpu


def _tol(D):
    return 1e-5 * np.abs(D) + 1e-5


def _same_up_to_near_ties(D, I, Do, Io):
    """Equal ids wherever a distance is separated from its neighbours by more than the
    tolerance; equal distances (within it) everywhere."""
    fin = np.isfinite(Do)
    assert np.array_equal(np.isfinite(D), fin)
    assert np.all(I[~fin] == -1)
    diff = np.zeros_like(Do)
    diff[fin] = D[fin] - Do[fin]
    assert np.all(np.abs(diff) <= _tol(np.where(fin, Do, 0)))
    gap = np.full(Do.shape, np.inf)
    dd = np.abs(np.diff(np.where(fin, Do, 1e30), axis=1))
    gap[:, 1:] = np.minimum(gap[:, 1:], dd)
    gap[:, :-1] = np.minimum(gap[:, :-1], dd)
    sep = fin & (gap > 2 * _tol(np.where(fin, Do, 0)))
    np.testing.assert_array_equal(I[sep], Io[sep])


def _data(seed, n, d, nc=48):
    cen = datagen.mixture_centres(seed, nc, d)
    x = datagen.mixture_points(cen, seed + 1, n)
    xq = datagen.mixture_points(cen, seed + 2, 300)
    return x, xq


def _flat(gbk, x, nlist, seed):
    coarse, _, _ = oracle.kmeans(x[:6000], datagen.permutation_prefix(seed, 6000, nlist), 5)
    ix = gbk.IVFFlatIndex(x.shape[1], nlist).set_centroids(torch.from_numpy(coarse).cuda())
    xt = torch.from_numpy(x).cuda()
    h = x.shape[0] // 3
    ix.add(xt[:h])          # two adds: the lists keep insertion order across calls
    ix.add(xt[h:])
    ex = ix.export()
    return ix, coarse, ex


@pytest.mark.parametrize("d", [32, 20])
@pytest.mark.parametrize("k,nprobe", [(1, 1), (10, 4), (100, 8), (700, 2)])
def test_ivfflat_matches_oracle(gbk, d, k, nprobe):
    x, xq = _data(200 + d, 20000, d)
    x[15000:15300] = x[:300]  # duplicates: equal distances broken by list position
    ix, coarse, ex = _flat(gbk, x, 64, 210 + d)
    assert ix.ntotal == x.shape[0]
    off, ids = ex["list_off"], ex["ids"]
    # list assignment = the oracle's nearest centroid, except at near-ties
    lists = np.repeat(np.arange(64), np.diff(off))
    a, _ = oracle.assign(x[ids], coarse)
    bad = np.nonzero(a != lists)[0]
    if bad.size:
        y = x[ids[bad]].astype(np.float64)
        d_gpu = ((y - coarse[lists[bad]]) ** 2).sum(1)
        d_or = ((y - coarse[a[bad]]) ** 2).sum(1)
        assert np.all(d_gpu - d_or <= 1e-5 * d_or + 1e-5)
    # ids within a list ascend (insertion order)
    for L in range(64):
        assert np.all(np.diff(ids[off[L]:off[L + 1]]) > 0)
    D, I = ix.search(torch.from_numpy(xq).cuda(), k, nprobe)
    D, I = D.cpu().numpy(), I.cpu().numpy()
    Do, Io = oracle.ivfflat_search(xq, coarse, off, x[ids], ids, k, nprobe)
    _same_up_to_near_ties(D, I, Do, Io)
    if k == 700 and nprobe == 2:
        assert (I == -1).any()  # some probed pairs of lists hold fewer than 700 vectors


def test_ivfflat_full_probe_equals_brute_force(gbk):
    x, xq = _data(230, 12000, 32)
    ix, coarse, ex = _flat(gbk, x, 16, 231)
    D, I = ix.search(torch.from_numpy(xq).cuda(), 50, 16)
    Do, Io = oracle.knn(xq, x, 50)
    _same_up_to_near_ties(D.cpu().numpy(), I.cpu().numpy(), Do, Io)


def test_ivfflat_empty_lists_and_small_index(gbk):
    d = 8
    coarse = np.zeros((5, d), np.float32)
    coarse[:, 0] = np.arange(5) * 100.0   # lists 3 and 4 stay empty
    x = (datagen.gaussian_matrix(240, 50, d) + coarse[datagen.randint(241, 0, 50, 3)]).astype(
        np.float32)
    ix = gbk.IVFFlatIndex(d, 5).set_centroids(torch.from_numpy(coarse).cuda())
    ix.add(torch.from_numpy(x).cuda(), ids=torch.arange(1000, 1050, device="cuda"))
    # x[:4]; a query nearest the empty list 3 whose second list (2) is full; one nearest
    # the empty lists 4 and 3 (nothing to return)
    far = np.zeros((2, d), np.float32)
    far[0, 0], far[1, 0] = 260.0, 401.0
    xq = np.concatenate([x[:4], far]).astype(np.float32)
    D, I = ix.search(torch.from_numpy(xq).cuda(), 20, 2)
    ex = ix.export()
    Do, Io = oracle.ivfflat_search(xq, coarse, ex["list_off"], x[ex["ids"] - 1000], ex["ids"], 20, 2)
    D, I = D.cpu().numpy(), I.cpu().numpy()
    _same_up_to_near_ties(D, I, Do, Io)
    assert (I[4] >= 1000).sum() >= 10 and (I[5] == -1).all() and np.isinf(D[5]).all()


def test_ivfflat_arguments(gbk):
    with pytest.raises(gbk.GbkError):
        gbk.IVFFlatIndex(16, 4, metric="ip")
    ix = gbk.IVFFlatIndex(16, 4)
    xq = torch.zeros((2, 16), device="cuda")
    with pytest.raises(gbk.GbkError):
        ix.search(xq, 1, 1)  # not trained
    ix.set_centroids(torch.zeros((4, 16), device="cuda"))
    for k, nprobe in ((0, 1), (1025, 1), (1, 0), (1, 5)):
        with pytest.raises(gbk.GbkError):
            ix.search(xq, k, nprobe)


# ------------------------------------------------------------------ IVFADC + exact re-rank

def _ivfpq(gbk, seed, n=15000, d=32, nlist=32, M=8, keep=True):
    x, xq = _data(seed, n, d)
    nt = min(5000, n)
    coarse, _, _ = oracle.kmeans(x[:nt], datagen.permutation_prefix(seed + 3, nt, nlist), 5)
    books = oracle.train_pq(oracle.residual_training_set(x[:nt], coarse), M,
                            datagen.permutation_prefix(seed + 4, nt, 256), 5)
    ix = gbk.IVFPQIndex(d, nlist, M).set_quantizers(torch.from_numpy(coarse).cuda(),
                                                   torch.from_numpy(books).cuda())
    if keep:
        ix.keep_vectors()
    ix.add(torch.from_numpy(x).cuda())
    return ix, x, xq, coarse, books


@pytest.mark.parametrize("k,nprobe,kprime", [(1, 2, 16), (10, 4, 40), (100, 8, 400),
                                             (10, 1, 1024)])
def test_refine_matches_oracle(gbk, k, nprobe, kprime):
    ix, x, xq, coarse, books = _ivfpq(gbk, 250)
    xqt = torch.from_numpy(xq).cuda()
    D, I = ix.search_refine(xqt, k, nprobe, kprime)
    D, I = D.cpu().numpy(), I.cpu().numpy()
    Dc, Ic = ix.search(xqt, kprime, nprobe)  # the same k' candidates, as ids
    Ic = Ic.cpu().numpy()
    for q in range(xq.shape[0]):
        cand = Ic[q][Ic[q] >= 0]
        ex = oracle.pair_dist(xq, x, np.full(cand.size, q), cand)
        o = np.lexsort((cand, ex))[:k]
        got = o.size
        # D = exact distance of the returned ids; I = exact top-k of the candidates
        np.testing.assert_allclose(D[q, :got], ex[o], rtol=1e-5, atol=1e-5)
        assert np.all(I[q, got:] == -1)
        _same_up_to_near_ties(D[q:q + 1, :got], I[q:q + 1, :got], ex[o][None], cand[o][None])
    # and the whole pipeline against the oracle's (its own ADC candidates): the candidate
    # sets can differ only at ADC near-ties at the k'-th place, which almost never reach the
    # exact top k
    ex_ = ix.export()
    Do, Io, _, _ = oracle.ivfadc_refine(xq, x, coarse, books, ex_["list_off"], ex_["codes"],
                                        ex_["ids"], k, nprobe, kprime)
    agree = np.mean([len(set(I[q]) & set(Io[q])) / k for q in range(xq.shape[0])])
    assert agree >= 0.995, agree


def test_refine_raises_recall(gbk):
    ix, x, xq, _, _ = _ivfpq(gbk, 260, d=64, M=8)
    xqt = torch.from_numpy(xq).cuda()
    _, Igt = gbk.knn_brute(xqt, torch.from_numpy(x).cuda(), 10)
    Igt = Igt.cpu().numpy()

    def r10(I):
        I = I.cpu().numpy()
        return np.mean([len(set(I[q]) & set(Igt[q])) / 10 for q in range(I.shape[0])])

    plain = r10(ix.search(xqt, 10, 8)[1])
    refined = r10(ix.search_refine(xqt, 10, 8, 200)[1])
    print("10-R@10 plain %.4f, re-ranked %.4f" % (plain, refined))
    assert refined >= plain + 0.1 and refined >= 0.9, (plain, refined)


def test_refine_arguments(gbk):
    ix, x, xq, _, _ = _ivfpq(gbk, 270, n=3000, keep=False)
    xqt = torch.from_numpy(xq).cuda()
    with pytest.raises(gbk.GbkError):
        ix.search_refine(xqt, 10, 2, 40)  # no kept vectors
    with pytest.raises(gbk.GbkError):
        ix.keep_vectors()                 # after the first add
    ix2, _, _, _, _ = _ivfpq(gbk, 271, n=3000)
    for k, kprime in ((10, 5), (0, 5), (10, 1025)):
        with pytest.raises(gbk.GbkError):
            ix2.search_refine(xqt, k, 2, kprime)


def test_batched_refine_equals_per_query_refine(gbk):
    # mixed nprobe in one persistent scan + re-rank: each query's results are those of the
    # single-nprobe refine search (same candidates, same re-rank arithmetic)
    ix, x, xq, _, _ = _ivfpq(gbk, 280)
    xqt = torch.from_numpy(xq).cuda()
    npq = torch.from_numpy(np.array([1, 2, 4, 8])[datagen.randint(281, 0, xq.shape[0], 4)]).cuda()
    D, I, used = gbk.ivfpq_search_batched_refine(ix, xqt, 10, 60, npq, 8)
    assert torch.equal(used, npq.to(torch.int32))
    for t in (1, 2, 4, 8):
        sel = (npq == t).nonzero().flatten()
        Dr, Ir = ix.search_refine(xqt[sel].contiguous(), 10, t, 60)
        assert torch.equal(I[sel], Ir) and torch.equal(D[sel], Dr)
