"""Exact k-NN on the tensor cores vs the oracle (Eq. 1 evaluated directly in float64).

Distances: within 1e-5 relative of float64 (float32-accurate TF32 hi/lo path).  Ids: the
oracle's id at every rank whose distance is not tied (within tolerance) with a neighbour;
and every returned id's exact distance is no worse than the oracle's k-th (within
tolerance).  Integer lattices give exact distances, where ids must match bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_1702_08734_gb300 import datagen

pytestmark = pytest.mark.gpu
RTOL = 1e-5


def _check_knn(xq, xb, D, I, k, metric="l2", rtol=RTOL):
    D = D.cpu().numpy().astype(np.float64)
    I = I.cpu().numpy()
    Do, Io = oracle.knn(xq, xb, k, metric=metric)
    scale = np.maximum(np.abs(Do), 1e-3 * (np.abs(Do).max() + 1))
    assert np.all(np.abs(D - Do) <= rtol * scale + 1e-6), np.abs(D - Do).max()
    # ids where the oracle's distance is well separated from its neighbours
    gap = np.full(Do.shape, np.inf)
    gap[:, 1:] = np.minimum(gap[:, 1:], np.abs(np.diff(Do, axis=1)))
    gap[:, :-1] = np.minimum(gap[:, :-1], np.abs(np.diff(Do, axis=1)))
    sep = gap > 4 * rtol * scale
    assert np.array_equal(I[sep], Io[sep])
    # every returned id is valid, distinct, and as good as the oracle's k-th
    assert I.min() >= 0 and I.max() < xb.shape[0]
    for q in range(I.shape[0]):
        assert len(set(I[q].tolist())) == k
    qi = np.repeat(np.arange(I.shape[0]), k)
    ex = oracle.pair_dist(xq, xb, qi, I.ravel(), metric=metric).reshape(I.shape)
    kth = Do[:, -1:]
    tol = 4 * rtol * np.maximum(np.abs(kth), 1e-3)
    if metric == "l2":
        assert np.all(ex <= kth + tol)
    else:
        assert np.all(ex >= kth - tol)


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
@pytest.mark.parametrize("d", [8, 32, 100, 128])
@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_pairwise_fp32_matches_float64(gbk, d, metric, prec):
    # both float32-accurate kinds: FP16 hi/lo of power-of-two scaled rows (the default) and
    # TF32 hi/lo
    xq = datagen.gaussian_matrix(500 + d, 300, d)
    xb = datagen.gaussian_matrix(600 + d, 1000, d)
    out = gbk.pairwise_distances(torch.from_numpy(xq).cuda(), torch.from_numpy(xb).cuda(),
                                 metric=metric, precision=prec).cpu().numpy().astype(np.float64)
    x = xq.astype(np.float64)
    y = xb.astype(np.float64)
    ref = x @ y.T if metric == "ip" else ((x[:, None, :] - y[None]) ** 2).sum(-1)
    mag = (np.abs(x)[:, None, :] * np.abs(y)[None]).sum(-1) + 1
    assert np.abs(out - ref).max() / 1 <= np.max(1e-5 * (mag + np.abs(ref))), \
        np.abs(out - ref).max()


@pytest.mark.parametrize("prec,tol", [("bf16", 2 ** -7), ("fp8", 2 ** -3)])
def test_pairwise_low_precision_error_bounds(gbk, prec, tol):
    xq = datagen.gaussian_matrix(701, 200, 128)
    xb = datagen.gaussian_matrix(702, 700, 128)
    out = gbk.pairwise_distances(torch.from_numpy(xq).cuda(), torch.from_numpy(xb).cuda(),
                                 metric="ip", precision=prec).cpu().numpy().astype(np.float64)
    x = xq.astype(np.float64)
    y = xb.astype(np.float64)
    ref = x @ y.T
    bound = tol * np.linalg.norm(x, axis=1)[:, None] * np.linalg.norm(y, axis=1)[None]
    assert np.all(np.abs(out - ref) <= bound)


@pytest.mark.parametrize("nq,nb,d,k", [(1, 100, 8, 1), (40, 3000, 128, 10), (130, 2000, 96, 1),
                                       (300, 20000, 128, 100), (257, 5000, 32, 256),
                                       (77, 4099, 100, 33)])
@pytest.mark.parametrize("metric", ["l2", "ip"])
@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_knn_fp32_vs_oracle(gbk, nq, nb, d, k, metric, prec):
    xq = datagen.gaussian_matrix(800 + nq, nq, d)
    xb = datagen.gaussian_matrix(900 + nb, nb, d)
    D, I = gbk.knn_brute(torch.from_numpy(xq).cuda(), torch.from_numpy(xb).cuda(), k,
                         metric=metric, precision=prec)
    _check_knn(xq, xb, D, I, k, metric)


def test_knn_chunking_does_not_change_results(gbk):
    xq = datagen.gaussian_matrix(31, 200, 128)
    xb = datagen.gaussian_matrix(32, 30000, 128)
    ref = None
    for ch in (1, 3, 17, 200):
        D, I = gbk.knn_brute(torch.from_numpy(xq).cuda(), torch.from_numpy(xb).cuda(), 50,
                             chunks=ch)
        if ref is None:
            ref = (D.cpu(), I.cpu())
        else:
            assert torch.equal(ref[1], I.cpu()) and torch.equal(ref[0], D.cpu())


def test_knn_integer_lattice_bit_exact(gbk):
    # integer coordinates: every distance is exact in float32, so ties (duplicate rows and
    # equidistant points) must resolve to the lower id exactly as in the oracle
    rng = np.random.default_rng(5)
    xb = rng.integers(-3, 4, size=(5000, 16)).astype(np.float32)
    xb[4000:4100] = xb[100:200]
    xq = rng.integers(-3, 4, size=(150, 16)).astype(np.float32)
    for k in (1, 7, 64, 300):
        D, I = gbk.knn_brute(torch.from_numpy(xq).cuda(), torch.from_numpy(xb).cuda(), k)
        Do, Io = oracle.knn(xq, xb, k)
        np.testing.assert_array_equal(I.cpu().numpy(), Io)
        np.testing.assert_array_equal(D.cpu().numpy(), Do.astype(np.float32))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("metric", ["l2", "ip"])
@pytest.mark.parametrize("k", [1, 10])
def test_knn_nan_rows_rank_last(gbk, prec, metric, k):
    # NaN database rows give NaN distances, which rank after every number (the oracle's
    # order): they never displace a finite neighbour, whatever batch they fall in
    xq = datagen.gaussian_matrix(61, 100, 64)
    xb = datagen.gaussian_matrix(62, 6000, 64)
    bad = np.unique(datagen.randint(63, 0, 300, 6000))
    xb[bad, 5] = np.nan
    D, I = gbk.knn_brute(torch.from_numpy(xq).cuda(), torch.from_numpy(xb).cuda(), k,
                         metric=metric, precision=prec)
    I = I.cpu().numpy()
    assert not np.isin(I, bad).any()
    good = np.setdiff1d(np.arange(6000), bad)
    Do, Io = oracle.knn(xq, xb[good], k, metric=metric)
    if prec == "fp32":
        _check_knn(xq, xb[good], D, torch.from_numpy(np.searchsorted(good, I)), k, metric)
    else:
        assert (np.searchsorted(good, I) == Io).mean() > 0.95


@pytest.mark.parametrize("k", [300, 1024])
def test_knn_large_k_path(gbk, k):
    xq = datagen.gaussian_matrix(41, 50, 64)
    xb = datagen.gaussian_matrix(42, 9000, 64)
    D, I = gbk.knn_brute(torch.from_numpy(xq).cuda(), torch.from_numpy(xb).cuda(), k)
    _check_knn(xq, xb, D, I, k)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_low_precision_rerank_certified_queries_are_exact(gbk, prec, metric):
    xq = datagen.gaussian_matrix(51, 200, 128)
    xb = datagen.gaussian_matrix(52, 20000, 128)
    k = 10
    D, I, cert, eb = gbk.knn_brute(torch.from_numpy(xq).cuda(), torch.from_numpy(xb).cuda(), k,
                                   metric=metric, precision=prec, kprime=40, certify=True)
    D = D.cpu().numpy().astype(np.float64)
    I = I.cpu().numpy()
    cert = cert.cpu().numpy().astype(bool)
    Do, Io = oracle.knn(xq, xb, k, metric=metric)
    # re-ranked distances are exact float32 evaluations of the returned ids
    qi = np.repeat(np.arange(I.shape[0]), k)
    ex = oracle.pair_dist(xq, xb, qi, I.ravel(), metric=metric).reshape(I.shape)
    np.testing.assert_allclose(D, ex, rtol=1e-5, atol=1e-4)
    # certified queries carry the exact top-k.  The bound is a rigorous worst case; with
    # FP8's 4-bit significand it is rarely tight enough to certify, BF16 usually is.
    if prec == "bf16":
        assert cert.mean() > 0.5, cert.mean()
    np.testing.assert_allclose(D[cert], Do[cert], rtol=1e-5, atol=1e-4)
    if cert.any():
        assert (I[cert] == Io[cert]).mean() > 0.999
    assert np.all(eb.cpu().numpy() > 0)


def test_invalid_arguments(gbk):
    x = torch.zeros((4, 8), device="cuda")
    for k in (0, 5, 2000):
        with pytest.raises(gbk.GbkError):
            gbk.knn_brute(x, x, k)


@pytest.fixture(scope="module")
def sift_like():
    xb = torch.from_numpy(datagen.gaussian_matrix(211, 1000000, 128)).cuda()
    xq = torch.from_numpy(datagen.gaussian_matrix(212, 10000, 128)).cuda()
    return xq, xb


@pytest.mark.parametrize("k", [10, 100])
@pytest.mark.parametrize("prefilter", [-1, 1])
def test_benchmark_workload_sampled(gbk, sift_like, k, prefilter):
    xq, xb = sift_like
    D, I = gbk.knn_brute(xq, xb, k, prefilter=prefilter)
    torch.cuda.synchronize()
    sample = np.unique(datagen.randint(213, 0, 12, xq.shape[0]))
    xs = xq[torch.from_numpy(sample).cuda()].cpu().numpy()
    _check_knn(xs, xb.cpu().numpy(), D[torch.from_numpy(sample).cuda()],
               I[torch.from_numpy(sample).cuda()], k)
    Dc = D.cpu()
    assert bool((Dc[:, 1:] >= Dc[:, :-1]).all())


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_fused_large_k(gbk, prec, metric):
    # nb > 65,536 and k >= 32: the fused selection with candidate lists of 128
    xq = datagen.gaussian_matrix(71, 300, 64)
    xb = datagen.gaussian_matrix(72, 100000, 64)
    k = 100
    if prec == "fp32":
        D, I = gbk.knn_brute(torch.from_numpy(xq).cuda(), torch.from_numpy(xb).cuda(), k,
                             metric=metric)
        _check_knn(xq, xb, D, I, k, metric)
    else:
        # low precision with the exact repair: every row is the float32 top-k, so the same
        # element-wise check as the float32 path holds
        D, I = gbk.knn_brute(torch.from_numpy(xq).cuda(), torch.from_numpy(xb).cuda(), k,
                             metric=metric, precision=prec, exact=True)
        _check_knn(xq, xb, D, I, k, metric)


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16"])
@pytest.mark.parametrize("metric", ["l2", "ip"])
@pytest.mark.parametrize("k", [2, 33, 100, 256])
def test_prefilter_does_not_change_results(gbk, prec, metric, k):
    # the threshold pre-pass only removes rows that cannot be among the k best: the
    # output is bit-identical with and without it (the TF32 split at k = 256 has too few
    # 128-row blocks for it and runs without, as the documented rule says)
    xq = torch.from_numpy(datagen.gaussian_matrix(75, 300, 64)).cuda()
    xb = torch.from_numpy(datagen.gaussian_matrix(76, 100000, 64)).cuda()
    D0, I0 = gbk.knn_brute(xq, xb, k, metric=metric, precision=prec, prefilter=-1)
    D1, I1 = gbk.knn_brute(xq, xb, k, metric=metric, precision=prec, prefilter=1)
    assert torch.equal(I0, I1) and torch.equal(D0, D1)


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_prefilter_one_pass_bound(gbk, prec, metric):
    # The split kinds' pre-pass runs one MMA pass over the high pieces and widens its k-th
    # value by a bound on the two cross terms it leaves out.  Rows here are 40 far-apart
    # base rows (entries ~50, row scales 2^7..2^8) plus perturbations well below the high
    # pieces' resolution, so the left-out terms decide the order among thousands of
    # near-equal rows: a bound that is too tight (a dropped term, a missing row scale)
    # prunes rows the plain search keeps and the outputs differ.
    rng = np.random.default_rng(11)
    d = 64
    base = 50.0 * rng.standard_normal((40, d))
    xb = (base[rng.integers(0, 40, 100000)] + 0.05 * rng.standard_normal((100000, d)))
    xq = base[rng.integers(0, 40, 200)] + 0.05 * rng.standard_normal((200, d))
    xq = torch.from_numpy(xq.astype(np.float32)).cuda()
    xb = torch.from_numpy(xb.astype(np.float32)).cuda()
    for k in (64, 100):
        D0, I0 = gbk.knn_brute(xq, xb, k, metric=metric, precision=prec, prefilter=-1)
        D1, I1 = gbk.knn_brute(xq, xb, k, metric=metric, precision=prec, prefilter=1)
        assert torch.equal(I0, I1) and torch.equal(D0, D1)


def test_prefilter_integer_lattice_ties(gbk):
    # exact distances with many ties (duplicated rows, equidistant lattice points): the
    # pre-pass bound equals some rows' distances, which must still be kept, so the lower-id
    # tie order of the oracle holds bit for bit
    rng = np.random.default_rng(6)
    xb = rng.integers(-2, 3, size=(80000, 12)).astype(np.float32)  # > 65,536: fused path
    xb[70000:71000] = xb[:1000]
    xq = rng.integers(-2, 3, size=(150, 12)).astype(np.float32)
    for k in (7, 64, 100):
        D, I = gbk.knn_brute(torch.from_numpy(xq).cuda(), torch.from_numpy(xb).cuda(), k,
                             prefilter=1)
        Do, Io = oracle.knn(xq, xb, k)
        np.testing.assert_array_equal(I.cpu().numpy(), Io)
        np.testing.assert_array_equal(D.cpu().numpy(), Do.astype(np.float32))


def test_clustered_near_duplicates_in_one_tile(gbk):
    # the only close points sit in the first 128-row tile, far points elsewhere: one chunk
    # holds every neighbour of queries 0 and 1, the others none (thresholds published by
    # the first chunk must still leave the rest of the search exact)
    rng = np.random.default_rng(3)
    nq, d, k = 64, 32, 64
    xq = rng.standard_normal((nq, d)).astype(np.float32)
    xb = (rng.standard_normal((70000, d)) * 10).astype(np.float32)
    xb[:40] = xq[0] + 0.01 * rng.standard_normal((40, d)).astype(np.float32)  # tile 0
    xb[40:128] = xq[1] + 0.01 * rng.standard_normal((88, d)).astype(np.float32)
    D, I = gbk.knn_brute(torch.from_numpy(xq).cuda(), torch.from_numpy(xb).cuda(), k)
    # absolute tolerance: distances ~2e-3 between near-duplicates come out of
    # ||x||^2 + ||y||^2 - 2<x, y> with norms ~32 (Eq. 2 cancels; the oracle sums (x - y)^2)
    D, I = D.cpu().numpy().astype(np.float64), I.cpu().numpy()
    Do, Io = oracle.knn(xq, xb, k)
    assert np.all(np.abs(D - Do) <= 1e-5 * np.abs(Do) + 2e-4)
    qi = np.repeat(np.arange(nq), k)
    ex = oracle.pair_dist(xq, xb, qi, I.ravel()).reshape(I.shape)
    assert np.all(ex <= Do[:, -1:] + 2e-4)
    assert all(len(set(r.tolist())) == k for r in I)
    assert np.array_equal(np.sort(I[2:], axis=1), np.sort(Io[2:], axis=1))


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_small_exact_configuration(gbk, prec):
    # the small exact configuration: database 65,536 x 128 and 1,024 queries, N(0,1), k = 10
    xb = datagen.gaussian_matrix(101, 65536, 128)
    xq = datagen.gaussian_matrix(102, 1024, 128)
    D, I = gbk.knn_brute(torch.from_numpy(xq).cuda(), torch.from_numpy(xb).cuda(), 10,
                         precision=prec)
    _check_knn(xq, xb, D, I, 10)


def test_fp32_wide_dynamic_range(gbk):
    # rows spanning many octaves (each row scaled by its own power of two, elements down to
    # 2^-20 of the row's largest) and rows of very different norms: the FP16 pieces of the
    # scaled rows still give float32-accurate distances
    rng = np.random.default_rng(12)
    xb = (rng.standard_normal((20000, 64)) * np.exp2(rng.integers(-20, 1, (20000, 64)))
          * np.exp2(rng.integers(-30, 30, (20000, 1)))).astype(np.float32)
    xq = xb[rng.integers(0, 20000, 150)] * np.float32(1.0001)
    for metric in ("l2", "ip"):
        D, I = gbk.knn_brute(torch.from_numpy(xq).cuda(), torch.from_numpy(xb).cuda(), 10,
                             metric=metric)
        D32, I32 = gbk.knn_brute(torch.from_numpy(xq).cuda(), torch.from_numpy(xb).cuda(), 10,
                                 metric=metric, precision="tf32x3")
        Do, Io = oracle.knn(xq, xb, 10, metric=metric)
        for Dg in (D, D32):
            Dg = Dg.cpu().numpy().astype(np.float64)
            scale = np.abs(Do).max(1, keepdims=True) + 1e-30
            assert np.all(np.abs(Dg - Do) <= 1e-5 * scale)


@pytest.mark.parametrize("d,offset", [(32, 1), (30, 0)])
def test_low_precision_rerank_unaligned_rows(gbk, d, offset):
    # database rows that are not 16-byte aligned (a view one float into its storage) or of a
    # length that is not a multiple of 4: the re-rank reads them with scalar loads
    xq = datagen.gaussian_matrix(81, 150, d)
    xb = datagen.gaussian_matrix(82, 8000, d)
    store = torch.zeros(xb.size + 4, device="cuda")
    store[offset:offset + xb.size] = torch.from_numpy(xb.ravel()).cuda()
    xbt = store[offset:offset + xb.size].view(8000, d)
    assert (xbt.data_ptr() % 16 == 0) == (offset == 0)
    D, I = gbk.knn_brute(torch.from_numpy(xq).cuda(), xbt, 10, precision="bf16", kprime=40,
                         exact=True)
    Dn, In = D.cpu().numpy().astype(np.float64), I.cpu().numpy()
    qi = np.repeat(np.arange(In.shape[0]), 10)
    ex = oracle.pair_dist(xq, xb, qi, In.ravel()).reshape(In.shape)
    np.testing.assert_allclose(Dn, ex, rtol=1e-5, atol=1e-4)
    _check_knn(xq, xb, D, I, 10)


@pytest.mark.parametrize("d", [160, 784, 1000])
@pytest.mark.parametrize("k", [1, 10, 100])
@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_knn_long_rows_stream_query_tile(gbk, d, k, prec):
    # rows too long to keep a 128-query tile resident beside the ring (float32-accurate
    # pieces beyond d = 128): the query k-blocks travel with the database's through the ring
    xq = datagen.gaussian_matrix(91, 200, d)
    xb = datagen.gaussian_matrix(92, 3000, d)
    D, I = gbk.knn_brute(torch.from_numpy(xq).cuda(), torch.from_numpy(xb).cuda(), k,
                         precision=prec)
    _check_knn(xq, xb, D, I, k)


@pytest.mark.parametrize("prec,d", [("bf16", 784), ("fp8", 1200)])
def test_low_precision_long_rows(gbk, prec, d):
    xq = datagen.gaussian_matrix(93, 150, d)
    xb = datagen.gaussian_matrix(94, 4000, d)
    D, I = gbk.knn_brute(torch.from_numpy(xq).cuda(), torch.from_numpy(xb).cuda(), 10,
                         precision=prec, kprime=80, exact=True)
    Dn, In = D.cpu().numpy().astype(np.float64), I.cpu().numpy()
    qi = np.repeat(np.arange(In.shape[0]), 10)
    ex = oracle.pair_dist(xq, xb, qi, In.ravel()).reshape(In.shape)
    np.testing.assert_allclose(Dn, ex, rtol=1e-5, atol=1e-3)
    _check_knn(xq, xb, D, I, 10)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("k", [10, 100])
@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_low_precision_exact_equals_fp32_path(gbk, prec, k, metric):
    # pattern 1 contract: BF16 / FP8 distances, k' = 4k over-fetch, float32 re-rank, and the
    # queries the certificate cannot prove re-run in float32 -> the float32 path's top-k,
    # element by element (ids at every rank not tied within rounding; distances to 1e-5)
    xq = datagen.gaussian_matrix(97, 700, 128)
    xb = datagen.gaussian_matrix(98, 60000, 128)
    xqt, xbt = torch.from_numpy(xq).cuda(), torch.from_numpy(xb).cuda()
    D32, I32 = gbk.knn_brute(xqt, xbt, k, metric=metric)
    D, I, cert, eb = gbk.knn_brute(xqt, xbt, k, metric=metric, precision=prec, certify=True,
                                   exact=True)
    c = cert.cpu().numpy()
    assert np.all((c == 1) | (c == 2))
    D32, I32 = D32.cpu().numpy().astype(np.float64), I32.cpu().numpy()
    D, I = D.cpu().numpy().astype(np.float64), I.cpu().numpy()
    scale = np.maximum(np.abs(D32), 1e-3 * (np.abs(D32).max() + 1))
    assert np.all(np.abs(D - D32) <= 1e-5 * scale)
    gap = np.full(D32.shape, np.inf)
    gap[:, 1:] = np.minimum(gap[:, 1:], np.abs(np.diff(D32, axis=1)))
    gap[:, :-1] = np.minimum(gap[:, :-1], np.abs(np.diff(D32, axis=1)))
    sep = gap > 4e-5 * scale
    assert sep.mean() > 0.8  # most ranks are decided by their distance
    assert np.array_equal(I[sep], I32[sep])
    for q in range(I.shape[0]):  # and the same set of neighbours
        if not np.array_equal(np.sort(I[q]), np.sort(I32[q])):
            # only possible through a tie at the k-th place: the swapped ids are equidistant
            miss = np.setdiff1d(I[q], I32[q])
            ex = oracle.pair_dist(xq, xb, np.full(miss.size, q), miss, metric=metric)
            assert np.all(np.abs(ex - D32[q, -1]) <= 4e-5 * scale[q, -1])


def test_pairwise_long_rows(gbk):
    d = 784
    xq = datagen.gaussian_matrix(95, 130, d)
    xb = datagen.gaussian_matrix(96, 700, d)
    P = gbk.pairwise_distances(torch.from_numpy(xq).cuda(), torch.from_numpy(xb).cuda())
    ex = ((xq.astype(np.float64)[:, None, :] - xb.astype(np.float64)[None]) ** 2).sum(-1)
    np.testing.assert_allclose(P.cpu().numpy(), ex, rtol=2e-5, atol=1e-3)


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
@pytest.mark.parametrize("metric", ["l2", "ip"])
@pytest.mark.parametrize("k", [1, 10, 100])
def test_host_buffers_match_device_search(gbk, prec, metric, k):
    # host inputs and outputs: the database crosses in growing pieces while the
    # search runs over the pieces already copied; the result is the device search's, bit
    # for bit (same per-pair arithmetic, one shared threshold, one final merge)
    xq = torch.from_numpy(datagen.gaussian_matrix(91, 700, 64)).pin_memory()
    xb = torch.from_numpy(datagen.gaussian_matrix(92, 600000, 64)).pin_memory()
    Dd, Id = gbk.knn_brute(xq.cuda(), xb.cuda(), k, metric=metric, precision=prec)
    Dh, Ih = gbk.knn_brute_host(xq, xb, k, metric=metric, precision=prec)
    assert Dh.device.type == "cpu"
    assert torch.equal(Id.cpu(), Ih) and torch.equal(Dd.cpu(), Dh)


def test_host_buffers_ties_and_other_paths(gbk):
    # integer lattice (exact distances, many ties) across pieces; the paths that copy
    # everything first (low precision, k > 512, short databases) give the device result too
    rng = np.random.default_rng(9)
    xb = torch.from_numpy(rng.integers(-2, 3, size=(300000, 12)).astype(np.float32))
    xb[290000:291000] = xb[:1000]
    xq = torch.from_numpy(rng.integers(-2, 3, size=(100, 12)).astype(np.float32))
    Dh, Ih = gbk.knn_brute_host(xq.pin_memory(), xb.pin_memory(), 50)
    Do, Io = oracle.knn(xq.numpy(), xb.numpy(), 50)
    np.testing.assert_array_equal(Ih.numpy(), Io)
    np.testing.assert_array_equal(Dh.numpy(), Do.astype(np.float32))
    xq2 = torch.from_numpy(datagen.gaussian_matrix(93, 200, 32))
    xb2 = torch.from_numpy(datagen.gaussian_matrix(94, 70000, 32))
    for kw in ({"k": 600}, {"k": 10, "precision": "bf16", "exact": True}):
        Dd, Id = gbk.knn_brute(xq2.cuda(), xb2.cuda(), **kw)
        Dh, Ih = gbk.knn_brute_host(xq2, xb2, **kw)  # pageable host memory
        assert torch.equal(Id.cpu(), Ih) and torch.equal(Dd.cpu(), Dh)
    xb3 = torch.from_numpy(datagen.gaussian_matrix(95, 5000, 32))
    Dd, Id = gbk.knn_brute(xq2.cuda(), xb3.cuda(), 20)
    Dh, Ih = gbk.knn_brute_host(xq2, xb3, 20)
    assert torch.equal(Id.cpu(), Ih) and torch.equal(Dd.cpu(), Dh)
    with pytest.raises(gbk.GbkError):
        gbk.knn_brute_host(xq2, xb3, 6000)


@pytest.mark.parametrize("prec", ["fp32", "tf32x3", "bf16", "fp8"])
@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_prepared_database_matches_brute(gbk, prec, metric):
    # a database prepared once and searched repeatedly gives knn_brute's results bit for bit
    xb = torch.from_numpy(datagen.gaussian_matrix(96, 90000, 64)).cuda()
    db = gbk.KnnDatabase(xb, precision=prec)
    for seed, k in ((97, 10), (98, 100), (99, 1)):
        xq = torch.from_numpy(datagen.gaussian_matrix(seed, 300, 64)).cuda()
        D0, I0 = gbk.knn_brute(xq, xb, k, metric=metric, precision=prec, exact=prec in ("bf16", "fp8"))
        D1, I1 = db.search(xq, k, metric=metric, exact=prec in ("bf16", "fp8"))
        assert torch.equal(I0, I1) and torch.equal(D0, D1)
    with pytest.raises(gbk.GbkError):  # another precision than the prepared one
        gbk.load()
        opts = gbk.KnnOpts(gbk.PRECISIONS["fp32" if prec != "fp32" else "bf16"], 0, 0, None, None, 0, 0)
        D = torch.empty((300, 10), device="cuda")
        I = torch.empty((300, 10), dtype=torch.int64, device="cuda")
        gbk._call("gbk_knn_db_search", db._h, gbk._ptr(xq), 300, 10, 0, gbk._ptr(D), gbk._ptr(I),
                  gbk.ctypes.byref(opts), gbk._stream())
    del db
