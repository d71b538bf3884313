"""Virtual shards on one GPU (section 5.4): the database split into S shards, each searched
on its own with global ids, and the partial results joined by one more k-selection
(gbk_merge_topk) must equal the unsharded search bit for bit.

Exact search uses integer lattices (every distance exact, so the unsharded ranking and the
merge's (value, id) order agree on ties): bit-exact.  IVFADC shards share the unsharded
index's quantizers, so every vector's ADC distance is the same sum of the same table
entries; the scan adds a code's M entries in an order rotated by the code's position in its
list (the bank-conflict-free table layout), and positions differ between a shard and the
full index, so distances agree to float rounding of that sum and the ids exactly."""
import numpy as np
import pytest
import torch

import oracle
from paper_1702_08734_gb300 import datagen

pytestmark = pytest.mark.gpu


def _split(n, S):
    b = np.linspace(0, n, S + 1).astype(int)
    return list(zip(b[:-1], b[1:]))


@pytest.mark.parametrize("metric", ["l2", "ip"])
@pytest.mark.parametrize("S,k", [(2, 1), (3, 10), (5, 64)])
def test_exact_shards_equal_unsharded(gbk, metric, S, k):
    rng = np.random.default_rng(7 + S)
    xb = rng.integers(-3, 4, size=(6000, 24)).astype(np.float32)
    xb[5000:5200] = xb[10:210]  # duplicates across shards: ties resolved by the lower id
    xq = torch.from_numpy(rng.integers(-3, 4, size=(300, 24)).astype(np.float32)).cuda()
    xbt = torch.from_numpy(xb).cuda()
    D, I = gbk.knn_brute(xq, xbt, k, metric=metric)
    Dp, Ip = [], []
    for r0, r1 in _split(xb.shape[0], S):
        d, i = gbk.knn_brute(xq, xbt[r0:r1].contiguous(), k, metric=metric)
        Dp.append(d)
        Ip.append(i + r0)
    Dm, Im = gbk.merge_topk(torch.stack(Dp), torch.stack(Ip), k, largest=(metric == "ip"))
    assert torch.equal(Im, I) and torch.equal(Dm, D)
    Do, Io = oracle.knn(xq.cpu().numpy(), xb, k, metric=metric)
    np.testing.assert_array_equal(Im.cpu().numpy(), Io)


def _ivf(gbk, seed=120, n=9000, d=32, nlist=16, M=8):
    cen = datagen.mixture_centres(seed, 64, d)
    x = datagen.mixture_points(cen, seed + 1, n)
    nt = 4000
    coarse, _, _ = oracle.kmeans(x[:nt], datagen.permutation_prefix(seed + 2, nt, nlist), 6)
    books = oracle.train_pq(oracle.residual_training_set(x[:nt], coarse), M,
                            datagen.permutation_prefix(seed + 3, nt, 256), 6)
    return x, torch.from_numpy(coarse).cuda(), torch.from_numpy(books).cuda(), cen


@pytest.mark.parametrize("S,k,nprobe", [(2, 10, 4), (3, 100, 8), (4, 700, 1)])
def test_ivfadc_shards_equal_unsharded(gbk, S, k, nprobe):
    x, coarse, books, cen = _ivf(gbk)
    xt = torch.from_numpy(x).cuda()
    full = gbk.IVFPQIndex(32, 16, 8).set_quantizers(coarse, books)
    full.add(xt)
    xq = torch.from_numpy(datagen.mixture_points(cen, 125, 400)).cuda()
    D, I = full.search(xq, k, nprobe)
    Dp, Ip = [], []
    for r0, r1 in _split(x.shape[0], S):
        sh = gbk.IVFPQIndex(32, 16, 8).set_quantizers(coarse, books)
        sh.add(xt[r0:r1].contiguous(), ids=torch.arange(r0, r1, device="cuda"))
        d, i = sh.search(xq, k, nprobe)
        Dp.append(d)
        Ip.append(i)
    Dm, Im = gbk.merge_topk(torch.stack(Dp), torch.stack(Ip), k)
    D, I, Dm, Im = D.cpu().numpy(), I.cpu().numpy(), Dm.cpu().numpy(), Im.cpu().numpy()
    fin = np.isfinite(D)
    assert np.array_equal(fin, np.isfinite(Dm)) and np.all(Im[~fin] == -1)
    # M = 8 float additions in another order: a few ulps of the sum
    tol = 8 * 1.2e-7 * np.abs(np.where(fin, D, 0)) + 1e-6
    diff = np.zeros_like(D)
    diff[fin] = Dm[fin] - D[fin]
    assert np.all(np.abs(diff) <= tol)
    # same ids wherever the distance is not within that tolerance of a neighbour's
    gap = np.full(D.shape, np.inf)
    dd = np.abs(np.diff(np.where(fin, D, 1e30), axis=1))
    gap[:, 1:] = np.minimum(gap[:, 1:], dd)
    gap[:, :-1] = np.minimum(gap[:, :-1], dd)
    sep = fin & (gap > 2 * tol)
    np.testing.assert_array_equal(Im[sep], I[sep])
    for r in range(I.shape[0]):  # and the same set of ids per query
        assert set(Im[r][fin[r]].tolist()) == set(I[r][fin[r]].tolist())
    if k == 700:  # one probed list holds fewer than k: the padding survives the merge
        assert (I == -1).any()


def test_merge_topk_arguments(gbk):
    Dp = torch.zeros((2, 3, 4), device="cuda")
    Ip = torch.zeros((2, 3, 4), dtype=torch.int64, device="cuda")
    for k in (0, 1025):
        with pytest.raises(gbk.GbkError):
            gbk.merge_topk(Dp, Ip, k)
