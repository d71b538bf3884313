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
