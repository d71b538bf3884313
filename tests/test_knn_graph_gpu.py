"""k-NN graph over the indexed vectors (section 6.5): every vector searched in the index for
k + 1 neighbours with its own id removed.

* Lossless codes on an integer lattice (codebooks holding every sub-vector value, coarse
  centroid at the origin) make every ADC distance exact, so the graph must equal the
  oracle's exact k-NN graph bit for bit, ties (lattice distances tie often) by lower id.
* With trained quantizers the graph matches the oracle's IVFADC search of the same index
  with the query's own id removed (distances to 1e-4 relative, ids except near-ties).
* Custom self ids, batching with a ragged tail and the learned-nprobe route are checked
  against the plain search of the same rows."""
import numpy as np
import pytest
import torch

import oracle
from paper_1702_08734_gb300 import datagen

pytestmark = pytest.mark.gpu


def _drop_self(D, I, self_ids, k):
    """The graph's rule: remove the first occurrence of the row's own id, else keep k."""
    Dg = np.empty((I.shape[0], k), D.dtype)
    Ig = np.empty((I.shape[0], k), np.int64)
    for r in range(I.shape[0]):
        keep = list(range(I.shape[1]))
        hit = np.nonzero(I[r] == self_ids[r])[0]
        if hit.size:
            keep.remove(int(hit[0]))
        keep = keep[:k]
        Dg[r], Ig[r] = D[r, keep], I[r, keep]
    return Dg, Ig


def _lattice_index(gbk, n=3000, d=16, M=8, seed=81):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 4, size=(n, d)).astype(np.float32)
    x[2000:2050] = x[100:150]  # exact duplicates under other ids
    dsub = d // M
    vals = np.stack(np.meshgrid(*[np.arange(4)] * dsub, indexing="ij"), -1).reshape(-1, dsub)
    books = np.full((M, 256, dsub), 1000.0, np.float32)
    books[:, :vals.shape[0]] = vals
    books[:, vals.shape[0]:] += np.arange(256 - vals.shape[0])[None, :, None]
    ix = gbk.IVFPQIndex(d, 1, M)
    ix.set_quantizers(torch.zeros((1, d), device="cuda"), torch.from_numpy(books).cuda())
    ix.add(torch.from_numpy(x).cuda())
    return ix, x


@pytest.mark.parametrize("k", [1, 6, 40])
def test_lossless_graph_equals_exact_graph(gbk, k):
    ix, x = _lattice_index(gbk)
    GD, G = gbk.knn_graph(ix, torch.from_numpy(x).cuda(), k, 1, batch=700)
    Do, Io = oracle.knn(x, x, k + 1)
    Dg, Ig = _drop_self(Do, Io, np.arange(x.shape[0]), k)
    np.testing.assert_array_equal(G.cpu().numpy(), Ig)
    np.testing.assert_array_equal(GD.cpu().numpy(), Dg.astype(np.float32))
    # the duplicates are each other's nearest neighbour at distance 0
    g = G.cpu().numpy()
    assert np.all(g[2000:2050, 0] == np.arange(100, 150))
    assert np.all(g[100:150, 0] == np.arange(2000, 2050))


def _trained_index(gbk, seed=90, n=6000, d=32, nlist=16, M=8):
    cen = datagen.mixture_centres(seed, 64, d)
    x = datagen.mixture_points(cen, seed + 1, n)
    nt = 4000
    coarse, _, _ = oracle.kmeans(x[:nt], datagen.permutation_prefix(seed + 2, nt, nlist), 6)
    books = oracle.train_pq(oracle.residual_training_set(x[:nt], coarse), M,
                            datagen.permutation_prefix(seed + 3, nt, 256), 6)
    ix = gbk.IVFPQIndex(d, nlist, M)
    ix.set_quantizers(torch.from_numpy(coarse).cuda(), torch.from_numpy(books).cuda())
    ix.add(torch.from_numpy(x).cuda())
    return ix, x, coarse, books


def test_graph_matches_oracle_ivfadc(gbk):
    ix, x, coarse, books = _trained_index(gbk)
    ex = ix.export()
    k, nprobe = 7, 4
    GD, G = gbk.knn_graph(ix, torch.from_numpy(x).cuda(), k, nprobe, batch=2500)
    Do, Io = oracle.ivfadc_search(x, coarse, books, ex["list_off"], ex["codes"], ex["ids"],
                                  k + 1, nprobe)
    Dg, Ig = _drop_self(Do, Io, np.arange(x.shape[0]), k)
    Dgpu = GD.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(Dgpu - Dg) <= 1e-4 * np.maximum(np.abs(Dg), 1e-2) + 1e-4)
    gap = np.full(Dg.shape, np.inf)
    dd = np.abs(np.diff(Dg, axis=1))
    gap[:, 1:] = np.minimum(gap[:, 1:], dd)
    gap[:, :-1] = np.minimum(gap[:, :-1], dd)
    sep = gap > 4e-4 * np.maximum(np.abs(Dg), 1e-2)
    assert (G.cpu().numpy()[sep] == Ig[sep]).mean() > 0.999


def test_self_ids_batches_and_plain_search(gbk):
    ix, x, _, _ = _trained_index(gbk, seed=95)
    xt = torch.from_numpy(x).cuda()
    k, nprobe = 5, 3
    GD, G = gbk.knn_graph(ix, xt, k, nprobe, batch=1777)
    D1, I1 = ix.search(xt, k + 1, nprobe)
    Dg, Ig = _drop_self(D1.cpu().numpy(), I1.cpu().numpy(), np.arange(x.shape[0]), k)
    np.testing.assert_array_equal(G.cpu().numpy(), Ig)
    np.testing.assert_array_equal(GD.cpu().numpy(), Dg)
    # rows given in another order, with their ids
    perm = torch.from_numpy(datagen.permutation_prefix(96, x.shape[0], x.shape[0])).cuda()
    GDp, Gp = gbk.knn_graph(ix, xt[perm].contiguous(), k, nprobe, self_ids=perm)
    assert torch.equal(Gp, G[perm]) and torch.equal(GDp, GD[perm])


def test_learned_route_graph(gbk):
    cen = datagen.mixture_centres(97, 70, 64)
    x = torch.from_numpy(datagen.mixture_points(cen, 98, 12000)).cuda()
    ix = gbk.IVFPQIndex(64, 128, 16)
    ix.train(x[:8000], niter=6, coarse_init=datagen.permutation_prefix(99, 8000, 128),
             pq_init=datagen.permutation_prefix(100, 8000, 256))
    ix.add(x)
    from oracle import mlp as omlp  # initial weights only (seeded uniforms)
    n = 128 * 128 + 128 + 128 * 128 + 128 + 5 * 128 + 5
    p = omlp.init_params((128, 128, 128, 5), datagen.uniform24(101, 0, n).astype(np.float64))
    net = gbk.MLP(128, 128, 128, 5,
                  params=np.concatenate([p[kk].ravel() for kk in omlp.PARAM_NAMES]).astype(np.float32))
    k = 10
    GD, G = gbk.knn_graph(ix, x, k, 16, mlp=net, batch=5000)
    kq = torch.full((x.shape[0],), k + 1, dtype=torch.int32, device="cuda")
    D1, I1, _, used = gbk.ivfpq_search_batched(ix, x, kq, k + 1, None, 16, mlp=net)
    Dg, Ig = _drop_self(D1.view(-1, k + 1).cpu().numpy(), I1.view(-1, k + 1).cpu().numpy(),
                        np.arange(x.shape[0]), k)
    np.testing.assert_array_equal(G.cpu().numpy(), Ig)
    np.testing.assert_array_equal(GD.cpu().numpy(), Dg)


def test_refined_graph_equals_per_row_refine(gbk):
    # the re-ranked graph: each row's k' ADC candidates re-scored exactly from the kept
    # vectors, then its own id dropped - the rows of search_refine(k + 1) minus self
    d, nlist, M, seed = 32, 16, 8, 97
    cen = datagen.mixture_centres(seed, 64, d)
    x = datagen.mixture_points(cen, seed + 1, 5000)
    nt = 3000
    coarse, _, _ = oracle.kmeans(x[:nt], datagen.permutation_prefix(seed + 2, nt, nlist), 6)
    books = oracle.train_pq(oracle.residual_training_set(x[:nt], coarse), M,
                            datagen.permutation_prefix(seed + 3, nt, 256), 6)
    ix = gbk.IVFPQIndex(d, nlist, M).set_quantizers(torch.from_numpy(coarse).cuda(),
                                                   torch.from_numpy(books).cuda())
    ix.keep_vectors()
    xt = torch.from_numpy(x).cuda()
    ix.add(xt)
    k, nprobe, kp = 10, 2, 64
    GD, G = gbk.knn_graph(ix, xt, k, nprobe, batch=1300, kprime=kp)
    Dr, Ir = ix.search_refine(xt, k + 1, nprobe, kp)
    Dg, Ig = _drop_self(Dr.cpu().numpy(), Ir.cpu().numpy(), np.arange(x.shape[0]), k)
    np.testing.assert_array_equal(G.cpu().numpy(), Ig)
    np.testing.assert_array_equal(GD.cpu().numpy(), Dg)
    # exact distances of the listed neighbours
    qi = np.repeat(np.arange(x.shape[0]), k)
    ex = oracle.pair_dist(x, x, qi, G.cpu().numpy().ravel()).reshape(G.shape)
    np.testing.assert_allclose(GD.cpu().numpy(), ex, rtol=1e-5, atol=1e-5)
    with pytest.raises(gbk.GbkError):
        gbk.knn_graph(ix, xt, k, nprobe, kprime=k)  # kprime must exceed k
