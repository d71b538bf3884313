"""Pins for the oracle's k-means, product quantizer, inverted file and IVFADC search."""
import numpy as np
import pytest

import oracle
from paper_1702_08734_gb300 import datagen


def test_kmeans_single_centroid_is_global_mean():
    x = datagen.gaussian_matrix(31, 999, 12)
    c, obj, _ = oracle.kmeans(x, [17], 3)
    np.testing.assert_array_equal(c[0], x.astype(np.float64).mean(0).astype(np.float32))
    # objective before the 2nd update is the total scatter around the mean
    mu = x.astype(np.float64).mean(0)
    np.testing.assert_allclose(obj[1], ((x - mu) ** 2).sum(), rtol=1e-6)


def test_kmeans_n_equals_k_reaches_zero():
    x = datagen.gaussian_matrix(32, 64, 6)
    c, obj, _ = oracle.kmeans(x, np.arange(64)[::-1], 2)
    assert obj[0] == 0.0 and obj[1] == 0.0
    assert sorted(map(tuple, c.tolist())) == sorted(map(tuple, x.tolist()))


def test_kmeans_objective_non_increasing_and_sklearn():
    x = datagen.mixture_points(datagen.mixture_centres(33, 20, 8), 34, 4000)
    init = datagen.permutation_prefix(35, x.shape[0], 20)
    c, obj, splits = oracle.kmeans(x, init, 12)
    assert splits == 0
    assert np.all(np.diff(obj) <= 1e-9 * obj[0])
    sk = pytest.importorskip("sklearn.cluster")
    km = sk.KMeans(n_clusters=20, init=x[init].astype(np.float64), n_init=1, max_iter=12,
                   tol=0.0, algorithm="lloyd").fit(x.astype(np.float64))
    if km.n_iter_ == 12:  # same number of updates (sklearn stops early at a fixed point)
        np.testing.assert_allclose(c, km.cluster_centers_, rtol=1e-5, atol=1e-5)


def test_kmeans_well_separated_clusters_recovered():
    centres = np.eye(5, 16, dtype=np.float32) * 100
    x = np.repeat(centres, 50, axis=0) + datagen.gaussian_matrix(36, 250, 16) * 0.01
    init = np.arange(0, 250, 50)
    c, _, _ = oracle.kmeans(x, init, 5)
    for j in range(5):
        np.testing.assert_allclose(c[j], x[j * 50:(j + 1) * 50].astype(np.float64).mean(0),
                                   rtol=1e-6, atol=1e-6)


def test_kmeans_empty_cluster_split_rule():
    # Two identical initial rows: ties go to the lower centroid, so centroid 1 is empty
    # after the first assignment and is re-seeded by splitting the largest cluster.
    x = np.array([[1.0, 2.0], [1.0, 2.0], [1.5, 2.5], [10.0, 10.0]], np.float32)
    c, _, splits = oracle.kmeans(x, [0, 1, 3], 1)
    assert splits == 1
    mean0 = np.array([(1 + 1 + 1.5) / 3, (2 + 2 + 2.5) / 3])
    g = np.array([1.0, -1.0])
    np.testing.assert_array_equal(c[1], (mean0.astype(np.float32).astype(np.float64)
                                         * (1 + g / 1024)).astype(np.float32))
    np.testing.assert_array_equal(c[0], (mean0.astype(np.float32).astype(np.float64)
                                         * (1 - g / 1024)).astype(np.float32))
    np.testing.assert_array_equal(c[2], [10.0, 10.0])


def test_ivf_bucket_is_stable_argsort():
    lists = datagen.randint(41, 0, 5000, 37)
    off, order = oracle.ivf_bucket(lists, 37)
    np.testing.assert_array_equal(order, np.argsort(lists, kind="stable"))
    np.testing.assert_array_equal(np.diff(off), np.bincount(lists, minlength=37))


def test_encode_ties_to_lowest_centroid():
    coarse = np.zeros((2, 4), np.float32)
    coarse[1] = 5.0
    pq = np.zeros((2, 256, 2), np.float32)
    pq[:, :, 0] = np.arange(256)[None, :] * 0.0 + 7.0
    pq[0, 9] = [0.5, 0.0]
    pq[0, 3] = [0.5, 0.0]          # duplicate of 9: lower index 3 wins
    pq[1, 200] = [0.0, 0.25]
    x = np.array([[0.5, 0.0, 0.0, 0.25]], np.float32)
    lists, codes = oracle.ivfpq_encode(x, coarse, pq)
    assert lists.tolist() == [0] and codes.tolist() == [[3, 200]]


def _tiny_index(seed, n=3000, d=16, nlist=8, M=4, niter=6):
    cen = datagen.mixture_centres(seed, 12, d)
    x = datagen.mixture_points(cen, seed + 1, n)
    coarse, _, _ = oracle.kmeans(x, datagen.permutation_prefix(seed + 2, n, nlist), niter)
    res = oracle.residual_training_set(x, coarse)
    books = oracle.train_pq(res, M, datagen.permutation_prefix(seed + 3, n, 256), niter)
    lists, codes = oracle.ivfpq_encode(x, coarse, books)
    off, order = oracle.ivf_bucket(lists, nlist)
    return x, coarse, books, off, codes[order], order.astype(np.int64)


def test_adc_two_forms_agree_eq10():
    x, coarse, books, off, codes, ids = _tiny_index(50)
    xq = datagen.mixture_points(datagen.mixture_centres(50, 12, 16), 60, 20)
    Dr, Ir = oracle.ivfadc_search(xq, coarse, books, off, codes, ids, 30, 3, form="recon")
    Dl, Il = oracle.ivfadc_search(xq, coarse, books, off, codes, ids, 30, 3, form="lut")
    np.testing.assert_allclose(Dr, Dl, rtol=1e-12)
    np.testing.assert_array_equal(Ir, Il)


def test_ivfadc_full_probe_equals_brute_force_over_reconstructions():
    x, coarse, books, off, codes, ids = _tiny_index(70)
    lists = np.repeat(np.arange(coarse.shape[0]), np.diff(off))
    M, _, dsub = books.shape
    recon = coarse[lists].astype(np.float64) + np.concatenate(
        [books[m][codes[:, m]].astype(np.float64) for m in range(M)], axis=1)
    xq = datagen.gaussian_matrix(71, 15, 16) * 2
    D, I = oracle.ivfadc_search(xq, coarse, books, off, codes, ids, 25, coarse.shape[0])
    for q in range(xq.shape[0]):
        dist = ((recon - xq[q].astype(np.float64)) ** 2).sum(1)
        order = np.lexsort((ids, dist))[:25]
        np.testing.assert_array_equal(I[q], ids[order])
        np.testing.assert_allclose(D[q], dist[order], rtol=1e-12)


def test_lossless_pq_makes_ivfadc_exact():
    # Residual sub-vectors take <= 256 distinct values, so the product quantizer can be
    # lossless; with every list probed, IVFADC then equals exact search (Eq. 6 = Eq. 1).
    d, M, n, nlist = 8, 4, 600, 4
    coarse = (np.arange(nlist, dtype=np.float32)[:, None] * 50.0).repeat(d, 1)
    L = datagen.randint(80, 0, n, nlist)
    sub = (datagen.randint(81, 0, n * M, 16).reshape(n, M) - 8).astype(np.float32)
    resid = np.repeat(sub, d // M, axis=1) * np.float32(0.5)
    x = (coarse[L] + resid).astype(np.float32)
    lists_chk, _ = oracle.assign(x, coarse)
    assert np.array_equal(lists_chk, L)
    books = np.zeros((M, 256, d // M), np.float32)
    books[:, :16, :] = ((np.arange(16) - 8) * 0.5)[None, :, None]
    books[:, 16:, :] = 1e6
    lists, codes = oracle.ivfpq_encode(x, coarse, books)
    off, order = oracle.ivf_bucket(lists, nlist)
    xq = datagen.gaussian_matrix(82, 12, d) * 40
    D, I = oracle.ivfadc_search(xq, coarse, books, off, codes[order], order, 10, nlist)
    De, Ie = oracle.knn(xq, x, 10)
    np.testing.assert_array_equal(I, Ie)
    np.testing.assert_allclose(D, De, rtol=1e-12)


def test_ivfadc_pads_when_fewer_than_k():
    x, coarse, books, off, codes, ids = _tiny_index(90, n=400, nlist=8)
    xq = x[:3]
    D, I = oracle.ivfadc_search(xq, coarse, books, off, codes, ids, 150, 1)
    for q in range(3):
        got = int((I[q] >= 0).sum())
        assert np.all(I[q, got:] == -1) and np.all(np.isinf(D[q, got:]))
        assert np.all(np.diff(D[q, :got]) >= 0)


# ------------------------------------------------------------------ IVF-Flat and re-ranking

def _flat_lists(x, coarse):
    lists, _ = oracle.assign(x, coarse)
    off, order = oracle.ivf_bucket(lists, coarse.shape[0])
    return off, x[order], order.astype(np.int64)


def test_ivfflat_full_probe_equals_exact_search():
    # every list probed: the inverted file changes only the visiting order, so the result is
    # exact search (Eq. 1), ties included (duplicated rows land in the same list)
    x, coarse, _, _, _, _ = _tiny_index(140, n=2000)
    x[1500:1600] = x[100:200]
    off, vecs, ids = _flat_lists(x, coarse)
    xq = datagen.gaussian_matrix(141, 25, 16) * 3
    D, I = oracle.ivfflat_search(xq, coarse, off, vecs, ids, 40, coarse.shape[0])
    De, Ie = oracle.knn(xq, x, 40)
    np.testing.assert_array_equal(I, Ie)
    np.testing.assert_array_equal(D, De)


def test_ivfflat_partial_probe_is_brute_force_over_probed_lists():
    x, coarse, _, _, _, _ = _tiny_index(150, n=1500)
    off, vecs, ids = _flat_lists(x, coarse)
    xq = datagen.mixture_points(datagen.mixture_centres(150, 12, 16), 151, 12)
    lists = np.repeat(np.arange(coarse.shape[0]), np.diff(off))
    for nprobe in (1, 3):
        D, I = oracle.ivfflat_search(xq, coarse, off, vecs, ids, 15, nprobe)
        for q in range(xq.shape[0]):
            cd = ((coarse.astype(np.float64) - xq[q].astype(np.float64)) ** 2).sum(1)
            probed = np.lexsort((np.arange(coarse.shape[0]), cd))[:nprobe]
            sel = np.isin(lists, probed)
            dist = ((vecs[sel].astype(np.float64) - xq[q].astype(np.float64)) ** 2).sum(1)
            o = np.lexsort((ids[sel], dist))[:15]
            got = min(15, int(sel.sum()))
            np.testing.assert_array_equal(I[q, :got], ids[sel][o])
            np.testing.assert_allclose(D[q, :got], dist[o], rtol=1e-12)
            assert np.all(I[q, got:] == -1) and np.all(np.isinf(D[q, got:]))


def test_refine_with_every_candidate_is_exact_search():
    # k' >= the database and every list probed: the re-rank sees every vector
    x, coarse, books, off, codes, ids = _tiny_index(160, n=700)
    xq = datagen.gaussian_matrix(161, 10, 16) * 2
    D, I, _, _ = oracle.ivfadc_refine(xq, x, coarse, books, off, codes, ids, 20, coarse.shape[0],
                                      700)
    De, Ie = oracle.knn(xq, x, 20)
    np.testing.assert_array_equal(I, Ie)
    np.testing.assert_allclose(D, De, rtol=1e-12)


def test_refine_is_exact_top_k_of_the_adc_candidates():
    x, coarse, books, off, codes, ids = _tiny_index(170)
    xq = datagen.mixture_points(datagen.mixture_centres(170, 12, 16), 171, 15)
    D, I, Dc, Ic = oracle.ivfadc_refine(xq, x, coarse, books, off, codes, ids, 10, 2, 40)
    Da, Ia = oracle.ivfadc_search(xq, coarse, books, off, codes, ids, 40, 2)
    np.testing.assert_array_equal(Ic, Ia)
    for q in range(xq.shape[0]):
        cand = Ia[q][Ia[q] >= 0]
        ex = ((x[cand].astype(np.float64) - xq[q].astype(np.float64)) ** 2).sum(1)
        o = np.lexsort((cand, ex))[:10]
        np.testing.assert_array_equal(I[q], cand[o])
        np.testing.assert_allclose(D[q], ex[o], rtol=1e-12)
        # re-ranking never loses ground: the k-th exact distance is at most ADC's choice's
        ex_adc = ((x[Ia[q, :10]].astype(np.float64) - xq[q].astype(np.float64)) ** 2).sum(1)
        assert D[q, -1] <= np.sort(ex_adc)[-1] + 1e-12


# ------------------------------------------------------------------ OPQ pre-rotation

def test_rotate_by_permutation_and_identity():
    x = datagen.gaussian_matrix(180, 50, 6)
    P = np.zeros((6, 6), np.float32)
    perm = [1, 2, 0, 4, 5, 3]           # R y picks y[perm[i]] for output i (not an involution)
    P[np.arange(6), perm] = 1.0
    np.testing.assert_array_equal(oracle.rotate(x, P), x[:, perm])
    np.testing.assert_array_equal(oracle.rotate(x, np.eye(6, dtype=np.float32)), x)


def test_orthogonal_rotation_preserves_distances():
    d = 24
    Q, _ = np.linalg.qr(datagen.gaussian_matrix(181, d, d).astype(np.float64))
    x = datagen.gaussian_matrix(182, 40, d)
    y = oracle.rotate(x, Q.astype(np.float32))
    D0 = ((x[:, None].astype(np.float64) - x[None]) ** 2).sum(-1)
    D1 = ((y[:, None].astype(np.float64) - y[None]) ** 2).sum(-1)
    np.testing.assert_allclose(D1, D0, rtol=1e-5, atol=1e-5)


def _block_tagged_residuals(M, dsub, n, seed):
    """Residuals whose sub-block m holds exactly 256 distinct sub-vectors V[m] (tagged by
    an offset of 100 m, so that a sub-vector read from the wrong block is far from every
    codeword); rows 0..255 carry V[m][j] in every block m, later rows a seeded choice."""
    rng = np.random.default_rng(seed)
    V = (rng.normal(size=(M, 256, dsub)) + 100.0 * np.arange(M)[:, None, None]).astype(np.float32)
    r = np.empty((n, M * dsub), np.float32)
    for m in range(M):
        j = np.concatenate([np.arange(256), rng.integers(0, 256, n - 256)])
        r[:, m * dsub:(m + 1) * dsub] = V[m][j]
    return r, V


@pytest.mark.parametrize("M,dsub", [(4, 3), (8, 2), (16, 8)])
def test_train_pq_lossless_books_in_dimension_order(M, dsub):
    # section 2 "Product quantizer": one 256-centroid codebook per block of d/M consecutive
    # dimensions.  With exactly 256 distinct sub-vectors per block and every one of them
    # among the initial rows, Lloyd's iterations keep them: codebook m, row j = V[m][j]
    # exactly (a strided or shifted slice, or blocks mixed up, lands elsewhere).
    r, V = _block_tagged_residuals(M, dsub, 3000, 11 + M)
    books = oracle.train_pq(r, M, np.arange(256), 4)
    np.testing.assert_array_equal(books, V)
    # and the codes are lossless: every residual is reconstructed exactly
    coarse = np.zeros((1, M * dsub), np.float32)
    _, codes = oracle.ivfpq_encode(r, coarse, books)
    rec = np.concatenate([books[m][codes[:, m]] for m in range(M)], axis=1)
    np.testing.assert_array_equal(rec, r)


def test_train_pq_follows_a_block_permutation():
    # permuting whole blocks of dimensions permutes the codebooks the same way
    M, dsub = 4, 3
    r, V = _block_tagged_residuals(M, dsub, 2000, 21)
    perm = [2, 0, 3, 1]
    rp = np.concatenate([r[:, p * dsub:(p + 1) * dsub] for p in perm], axis=1)
    books = oracle.train_pq(r, M, np.arange(256), 3)
    books_p = oracle.train_pq(rp, M, np.arange(256), 3)
    np.testing.assert_array_equal(books_p, books[perm])


def test_residual_training_set_is_offset_from_nearest_centroid():
    # Eq. 3's residual r = y - q1(y): rows built as centroid j + a small known offset give
    # that offset (in double) and centroid rows give zero
    rng = np.random.default_rng(3)
    cen = (rng.normal(size=(5, 6)) * 50).astype(np.float32)
    off = (rng.normal(size=(40, 6)) * 0.1).astype(np.float32)
    j = rng.integers(0, 5, 40)
    x = (cen[j] + off).astype(np.float32)
    res = oracle.residual_training_set(x, cen)
    np.testing.assert_allclose(res, x.astype(np.float64) - cen[j].astype(np.float64), rtol=0,
                               atol=0)
    np.testing.assert_array_equal(oracle.residual_training_set(cen, cen), np.zeros((5, 6)))


def test_procrustes_recovers_a_known_rotation():
    # y = x Q^T with Q orthogonal: the minimiser is Q itself (the SVD formula's orientation
    # - R, not R^T - is what this pins)
    rng = np.random.default_rng(8)
    x = rng.normal(size=(500, 12))
    Q, _ = np.linalg.qr(rng.normal(size=(12, 12)))
    np.testing.assert_allclose(oracle.procrustes(x, x @ Q.T), Q, atol=1e-10)
    # a reflection-free case and a case with noise: still orthogonal, and optimal against
    # random orthogonal alternatives
    y = x @ Q.T + 0.05 * rng.normal(size=x.shape)
    R = oracle.procrustes(x, y)
    np.testing.assert_allclose(R @ R.T, np.eye(12), atol=1e-10)
    err = np.linalg.norm(x @ R.T - y)
    for s in range(20):
        W, _ = np.linalg.qr(np.random.default_rng(100 + s).normal(size=(12, 12)))
        assert err <= np.linalg.norm(x @ W.T - y)


def test_opq_keeps_identity_when_pq_is_lossless():
    # every row exactly representable by the product quantizer: the reconstruction is x,
    # A = x^T x is symmetric positive definite and its polar factor is the identity
    r, V = _block_tagged_residuals(4, 3, 2000, 31)
    R, books = oracle.opq_train(r, 4, np.arange(256), 2, 3)
    np.testing.assert_allclose(R, np.eye(12), atol=1e-5)
    np.testing.assert_array_equal(books, V)


def test_opq_lowers_quantization_error_of_rotated_data():
    # block-structured data mixed by a hidden rotation: the trained rotation reconstructs
    # better than the plain product quantizer of the unrotated data
    r, V = _block_tagged_residuals(4, 3, 3000, 41)
    r = r + np.random.default_rng(42).normal(size=r.shape).astype(np.float32) * 0.05
    Q, _ = np.linalg.qr(np.random.default_rng(43).normal(size=(12, 12)))
    x = (r.astype(np.float64) @ Q.T).astype(np.float32)

    def mse(xr, books):
        _, codes = oracle.ivfpq_encode(xr, np.zeros((1, 12), np.float32), books)
        y = np.concatenate([books[m][codes[:, m]] for m in range(4)], axis=1)
        return float(((xr.astype(np.float64) - y) ** 2).sum(1).mean())

    plain = oracle.train_pq(x, 4, np.arange(256), 4)
    R, books = oracle.opq_train(x, 4, np.arange(256), 6, 4)
    np.testing.assert_allclose(R @ R.T, np.eye(12), atol=1e-5)
    assert mse(oracle.rotate(x, R), books) < mse(x, plain)
