"""OPQ pre-rotation (the rotation the paper's DEEP1B / YFCC100M experiments apply before
product quantization): the index replaces every input vector y by R y with a float32-
accurate GEMM, so its results must equal the oracle's IVFADC on the oracle's rotated
vectors, up to the rounding of that product (codes and ids identical except at near-ties,
distances within 1e-4 relative)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1702_08734_gb300 import datagen

pytestmark = pytest.mark.gpu


def _orth(seed, d):
    Q, _ = np.linalg.qr(datagen.gaussian_matrix(seed, d, d).astype(np.float64))
    return Q.astype(np.float32)


def test_rotate_matches_oracle(gbk):
    d = 64
    R = _orth(300, d)
    x = datagen.gaussian_matrix(301, 3000, d) * 3
    ix = gbk.IVFPQIndex(d, 8, 8).set_rotation(torch.from_numpy(R).cuda())
    y = ix.rotate(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.rotate(x, R)
    scale = np.linalg.norm(x, axis=1, keepdims=True)
    assert np.all(np.abs(y - ref) <= 4e-6 * scale)  # TF32x3 split + float32 accumulation


def test_rotated_ivfadc_matches_oracle(gbk):
    d, nlist, M = 32, 16, 8
    R = _orth(310, d)
    cen = datagen.mixture_centres(311, 64, d)
    x = datagen.mixture_points(cen, 312, 12000)
    xq = datagen.mixture_points(cen, 313, 300)
    xr, xqr = oracle.rotate(x, R), oracle.rotate(xq, R)
    nt = 4000
    coarse, _, _ = oracle.kmeans(xr[:nt], datagen.permutation_prefix(314, nt, nlist), 6)
    books = oracle.train_pq(oracle.residual_training_set(xr[:nt], coarse), M,
                            datagen.permutation_prefix(315, nt, 256), 6)
    ix = gbk.IVFPQIndex(d, nlist, M).set_rotation(torch.from_numpy(R).cuda())
    ix.set_quantizers(torch.from_numpy(coarse).cuda(), torch.from_numpy(books).cuda())
    ix.keep_vectors()
    ix.add(torch.from_numpy(x).cuda())  # rotated inside the index
    ex = ix.export()
    # lists and codes: the oracle's encoding of its rotated vectors, except near-ties
    lists_o, codes_o = oracle.ivfpq_encode(xr[ex["ids"]], coarse, books)
    lists = np.repeat(np.arange(nlist), np.diff(ex["list_off"]))
    assert (lists_o == lists).mean() > 0.999
    assert (codes_o == ex["codes"]).all(axis=1).mean() > 0.99
    xqt = torch.from_numpy(xq).cuda()
    D, I = ix.search(xqt, 20, 4)
    D, I = D.cpu().numpy(), I.cpu().numpy()
    Do, Io = oracle.ivfadc_search(xqr, coarse, books, ex["list_off"], ex["codes"], ex["ids"], 20, 4)
    fin = np.isfinite(Do)
    assert np.array_equal(fin, np.isfinite(D))
    assert np.all(np.abs(D[fin] - Do[fin]) <= 1e-4 * np.abs(Do[fin]) + 1e-4)
    assert (I == Io).mean() > 0.99
    # exact re-rank through the rotation: distances of the ORIGINAL vectors (R orthogonal)
    Dr, Ir = ix.search_refine(xqt, 10, 4, 100)
    Dr, Ir = Dr.cpu().numpy(), Ir.cpu().numpy()
    qi = np.repeat(np.arange(Ir.shape[0]), 10)
    exd = oracle.pair_dist(xq, x, qi, Ir.ravel()).reshape(Ir.shape)
    np.testing.assert_allclose(Dr, exd, rtol=1e-4, atol=1e-3)


def test_rotation_must_precede_training(gbk):
    ix = gbk.IVFPQIndex(16, 4, 8)
    ix.set_quantizers(torch.zeros((4, 16), device="cuda"), torch.zeros((8, 256, 2), device="cuda"))
    with pytest.raises(gbk.GbkError):
        ix.set_rotation(torch.eye(16, device="cuda"))


def _block_tagged(M, dsub, n, seed, noise=0.0):
    """Rows whose block m holds one of 256 well-separated sub-vectors (tagged by +100 m),
    rows 0..255 carrying every one of them; optional small Gaussian noise."""
    rng = np.random.default_rng(seed)
    V = (rng.normal(size=(M, 256, dsub)) * 3 + 100.0 * np.arange(M)[:, None, None]).astype(np.float32)
    r = np.empty((n, M * dsub), np.float32)
    for m in range(M):
        j = np.concatenate([np.arange(256), rng.integers(0, 256, n - 256)])
        r[:, m * dsub:(m + 1) * dsub] = V[m][j]
    if noise:
        r = (r + rng.normal(size=r.shape) * noise).astype(np.float32)
    return r


@pytest.mark.parametrize("d,M", [(32, 8), (64, 16)])
def test_trained_rotation_matches_oracle(gbk, d, M):
    # the library's alternation (PQ k-means on x R^T, reconstruction, A = Y^T x in double,
    # Newton-Schulz polar factor) against the oracle's (same k-means, numpy SVD)
    x = _block_tagged(M, d // M, 6000, 60 + d, noise=0.05)
    ix = gbk.IVFPQIndex(d, 16, M)
    R = ix.train_rotation(torch.from_numpy(x).cuda(), niter=3, pq_niter=3,
                          pq_init=np.arange(256)).cpu().numpy()
    Ro, _ = oracle.opq_train(x, M, np.arange(256), 3, 3)
    np.testing.assert_allclose(R @ R.T, np.eye(d), atol=2e-6)
    np.testing.assert_allclose(R, Ro, atol=2e-5)


def test_trained_rotation_is_identity_when_pq_is_lossless(gbk):
    x = _block_tagged(8, 4, 4000, 70)
    ix = gbk.IVFPQIndex(32, 16, 8)
    R = ix.train_rotation(torch.from_numpy(x).cuda(), niter=2, pq_niter=2).cpu().numpy()
    np.testing.assert_allclose(R, np.eye(32), atol=1e-5)


def test_trained_rotation_helps_rotated_data(gbk):
    # block structure hidden by a rotation: with the trained rotation the index quantises
    # the data better and finds more true neighbours than without it
    d, M = 32, 8
    z = _block_tagged(M, d // M, 30000, 80, noise=0.3)
    Q = _orth(81, d)
    x = (z.astype(np.float64) @ Q.T).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    xq = torch.from_numpy(x[:300] + datagen.gaussian_matrix(82, 300, d) * 0.05).cuda()
    _, Ie = oracle.knn(xq.cpu().numpy(), x, 10)
    recalls = []
    for trained in (False, True):
        ix = gbk.IVFPQIndex(d, 16, M)
        if trained:
            R = ix.train_rotation(xt, niter=8, pq_niter=4)
            np.testing.assert_allclose((R @ R.T).cpu().numpy(), np.eye(d), atol=2e-6)
        ix.train(xt, niter=6, coarse_init=datagen.permutation_prefix(83, 30000, 16),
                 pq_init=datagen.permutation_prefix(84, 30000, 256))
        ix.add(xt)
        _, I = ix.search(xq, 10, 16)
        I = I.cpu().numpy()
        recalls.append(np.mean([len(set(I[q]) & set(Ie[q])) / 10 for q in range(300)]))
    assert recalls[1] > recalls[0], recalls
