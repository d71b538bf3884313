"""IVFADC at the configured code size (PQ16, 8-bit codes, d = 128 and d = 96) against the
oracle, element by element.

Tolerances, per result:
* direct tables (LUT[m][c] = ||(x - c_L)^m - C_m[c]||^2 summed over M = 16 sub-quantizers,
  every term positive): 1e-5 relative to the oracle's double-precision distance;
* precomputed tables (Eq. 11: term 2 + term 1 + term 3, which cancel against each other):
  32 u A with u = 2^-24 and A = ||x||^2 + ||c_L||^2 + sum_m (|T[L][m][c_m]| + 2 |<x^m, C_m[c_m]>|),
  the magnitudes the float32 terms are rounded at (term 2 from the norm expansion of Eq. 2,
  the 16 term-1 entries and the 16 term-3 entries of the code; 32 bounds the operations
  each passes through).
Ids must equal the oracle's at every rank whose distance is separated from its neighbours'
(and, at the k-th rank, from the oracle's (k+1)-th) by more than both tolerances; at the
other ranks the GPU's id must be a distinct stored vector whose exact ADC distance equals
the oracle's at that rank within the tolerance.  Queries whose probed set is ambiguous (the
nprobe-th and (nprobe+1)-th coarse distances within 1e-4 relative) are left out; the tests
check that they are rare."""
import numpy as np
import pytest
import torch

import oracle
from paper_1702_08734_gb300 import datagen

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _mixture(seed, n, d, ncent=64, std=2.0):
    cen = datagen.mixture_centres(seed, ncent, d, std)
    return datagen.mixture_points(cen, seed + 1, n), cen


_CACHE = {}


def _quantizers(d, seed, n=20000, nlist=32, M=16):
    """Database, oracle-trained coarse centroids and PQ16 codebooks (cached per shape)."""
    key = (d, seed, n, nlist, M)
    if key not in _CACHE:
        x, cen = _mixture(seed, n, d)
        nt = 4000
        coarse, _, _ = oracle.kmeans(x[:nt], datagen.permutation_prefix(seed + 2, nt, nlist), 6)
        res = oracle.residual_training_set(x[:nt], coarse)
        books = oracle.train_pq(res, M, datagen.permutation_prefix(seed + 3, nt, 256), 6)
        _CACHE[key] = (x, cen, coarse, books)
    return _CACHE[key]


def _index(gbk, d, precomputed, seed=400, nlist=32, M=16):
    x, cen, coarse, books = _quantizers(d, seed, nlist=nlist, M=M)
    ix = gbk.IVFPQIndex(d, coarse.shape[0], books.shape[0])
    ix.set_quantizers(torch.from_numpy(coarse).cuda(), torch.from_numpy(books).cuda(),
                      use_precomputed=precomputed)
    ix.add(torch.from_numpy(x).cuda())
    return ix, x, cen, coarse, books


def _queries(cen, seed, nq, d):
    xq = datagen.mixture_points(cen, seed, nq)
    return (xq + datagen.gaussian_matrix(seed + 1, nq, d) * 0.1).astype(np.float32)


class Adc:
    """Exact (double) ADC distances and rounding magnitudes of stored vectors, from the
    exported index: used to validate the GPU's ids at non-separated ranks."""

    def __init__(self, ex, coarse, books):
        self.off, self.codes, self.ids = ex["list_off"], ex["codes"], ex["ids"]
        self.pos = np.empty(self.ids.size, np.int64)
        self.pos[self.ids] = np.arange(self.ids.size)
        self.coarse = coarse.astype(np.float64)
        self.books = books.astype(np.float64)
        self.M, self.dsub = books.shape[0], books.shape[2]

    def dist_and_mag(self, x, ids):
        """x [d], ids [n] >= 0 -> (ADC distance, magnitude A) per id."""
        j = self.pos[ids]
        L = np.searchsorted(self.off, j, side="right") - 1
        c = self.codes[j].astype(np.int64)                               # [n][M]
        sub = self.books[np.arange(self.M)[None, :], c]                  # [n][M][dsub]
        rec = self.coarse[L] + sub.reshape(len(ids), -1)
        x64 = x.astype(np.float64)
        d = ((x64[None, :] - rec) ** 2).sum(1)
        cl = self.coarse[L].reshape(len(ids), self.M, self.dsub)
        xm = x64.reshape(self.M, self.dsub)[None]
        T = (sub ** 2).sum(2) + 2 * (cl * sub).sum(2)
        t3 = (xm * sub).sum(2)
        A = (x64 ** 2).sum() + (self.coarse[L] ** 2).sum(1) + np.abs(T).sum(1) + 2 * np.abs(t3).sum(1)
        return d, A


def _ambiguous_probes(xq, coarse, nprobe, rel=1e-4):
    """Queries whose nprobe-th and (nprobe+1)-th coarse distances nearly tie."""
    if nprobe >= coarse.shape[0]:
        return np.zeros(xq.shape[0], bool)
    dc = ((xq.astype(np.float64)[:, None, :] - coarse.astype(np.float64)[None]) ** 2).sum(2)
    dc.sort(1)
    return (dc[:, nprobe] - dc[:, nprobe - 1]) <= rel * dc[:, nprobe]


def check_strict(D, I, Do, Io, xq, adc, direct, skip=None):
    """Element-wise comparison of one batch of GPU results with the oracle's (k+1) results."""
    k = D.shape[1]
    D = np.asarray(D, np.float64)
    I = np.asarray(I)
    Dk, Ik, Dn = Do[:, :k], Io[:, :k], Do[:, k]
    nq = D.shape[0]
    rows = np.nonzero(~skip)[0] if skip is not None else np.arange(nq)
    nsep = 0
    for q in rows:
        fin = np.isfinite(Dk[q])
        assert np.array_equal(np.isfinite(D[q]), fin), q
        assert np.all(I[q][~fin] == -1)
        nf = int(fin.sum())
        if nf == 0:
            continue
        ids = I[q][:nf]
        assert np.all(ids >= 0) and np.unique(ids).size == nf, q
        de, A = adc.dist_and_mag(xq[q], ids)
        _, Ao = adc.dist_and_mag(xq[q], Ik[q][:nf])
        # table mode: max(32, 2M) u A (the per-vector term-1 sum alone rounds M - 1 times)
        cm = max(32, 2 * adc.M)
        tol_g = 1e-5 * np.abs(de) if direct else cm * U32 * A
        tol_o = 1e-5 * np.abs(Dk[q][:nf]) if direct else cm * U32 * Ao
        # the GPU's distance is its id's ADC distance, and that is the oracle's at the rank
        assert np.all(np.abs(D[q][:nf] - de) <= tol_g), (q, np.abs(D[q][:nf] - de).max())
        assert np.all(np.abs(de - Dk[q][:nf]) <= tol_g + tol_o), q
        # same id wherever the oracle's distance is separated from its neighbours'
        dq = Dk[q][:nf]
        gap = np.full(nf, np.inf)
        if nf > 1:
            dd = np.diff(dq)
            gap[1:] = np.minimum(gap[1:], dd - tol_o[1:] - tol_o[:-1])
            gap[:-1] = np.minimum(gap[:-1], dd - tol_o[1:] - tol_o[:-1])
        if nf == k and np.isfinite(Dn[q]):
            gap[-1] = min(gap[-1], Dn[q] - dq[-1] - 2 * tol_o[-1])
        sep = gap > tol_o + tol_g
        assert np.array_equal(ids[sep], Ik[q][:nf][sep]), (q, np.nonzero(ids[sep] != Ik[q][:nf][sep]))
        nsep += int(sep.sum())
    return nsep


@pytest.mark.parametrize("d", [128, 96])
@pytest.mark.parametrize("precomputed", [True, False])
@pytest.mark.parametrize("nprobe", [3, 32])
@pytest.mark.parametrize("k", [1, 10, 100])
def test_pq16_search_matches_oracle(gbk, d, precomputed, nprobe, k):
    ix, x, cen, coarse, books = _index(gbk, d, precomputed)
    ex = ix.export()
    xq = _queries(cen, 410 + d, 200, d)
    D, I = ix.search(torch.from_numpy(xq).cuda(), k, nprobe)
    Do, Io = oracle.ivfadc_search(xq, coarse, books, ex["list_off"], ex["codes"], ex["ids"],
                                  k + 1, nprobe)
    skip = _ambiguous_probes(xq, coarse, nprobe)
    assert skip.mean() <= 0.02
    nsep = check_strict(D.cpu().numpy(), I.cpu().numpy(), Do, Io, xq, Adc(ex, coarse, books),
                        not precomputed, skip)
    assert nsep >= 0.9 * (~skip).sum() * k  # nearly every rank is decided by its distance


@pytest.mark.parametrize("precomputed", [True, False])
@pytest.mark.parametrize("nprobe,k", [(1, 10), (8, 100)])
def test_search_64_byte_codes_match_oracle(gbk, precomputed, nprobe, k):
    # 64-byte codes at d = 128 (sub-vectors of 2): the term-3 table in 128-word rows, the
    # look-ups summed in groups of 16, codes rotated by list position mod 32; both table
    # modes against the oracle's ADC search under the same strict check as PQ16
    ix, x, cen, coarse, books = _index(gbk, 128, precomputed, seed=470, M=64)
    ex = ix.export()
    xq = _queries(cen, 480, 200, 128)
    D, I = ix.search(torch.from_numpy(xq).cuda(), k, nprobe)
    Do, Io = oracle.ivfadc_search(xq, coarse, books, ex["list_off"], ex["codes"], ex["ids"],
                                  k + 1, nprobe)
    skip = _ambiguous_probes(xq, coarse, nprobe)
    assert skip.mean() <= 0.02
    nsep = check_strict(D.cpu().numpy(), I.cpu().numpy(), Do, Io, xq, Adc(ex, coarse, books),
                        not precomputed, skip)
    # the table-mode bound is 2M u A, four times PQ16's, so more neighbouring ranks fall
    # within it (74% of them decided by distance at nprobe 8, k = 100; 90% in direct mode)
    assert nsep >= (0.9 if not precomputed else 0.7) * (~skip).sum() * k


@pytest.mark.parametrize("precomputed", [True, False])
@pytest.mark.parametrize("d,M", [(96, 12), (120, 20), (96, 24), (112, 28), (108, 36), (120, 40),
                                 (132, 44), (96, 48), (104, 52), (112, 56), (120, 60)])
def test_search_other_multiples_of_4_match_oracle(gbk, precomputed, d, M):
    # code sizes between the powers of two (the light launch shape: 4-, 8- or 16-byte code
    # loads, pairwise sums over lengths that are not powers of two, a direct LUT of
    # M ceil(32 / M) words per row) against the oracle's ADC search, strict check
    x, cen, coarse, books = _quantizers(d, 500 + M, n=12000, M=M)
    ix = gbk.IVFPQIndex(d, coarse.shape[0], M)
    ix.set_quantizers(torch.from_numpy(coarse).cuda(), torch.from_numpy(books).cuda(),
                      use_precomputed=precomputed)
    ix.add(torch.from_numpy(x).cuda())
    ex = ix.export()
    xq = _queries(cen, 510 + M, 100, d)
    k, nprobe = 50, 8
    D, I = ix.search(torch.from_numpy(xq).cuda(), k, nprobe)
    Do, Io = oracle.ivfadc_search(xq, coarse, books, ex["list_off"], ex["codes"], ex["ids"],
                                  k + 1, nprobe)
    skip = _ambiguous_probes(xq, coarse, nprobe)
    assert skip.mean() <= 0.03
    nsep = check_strict(D.cpu().numpy(), I.cpu().numpy(), Do, Io, xq, Adc(ex, coarse, books),
                        not precomputed, skip)
    assert nsep >= (0.85 if not precomputed else 0.6) * (~skip).sum() * k


def test_scan_shape_does_not_change_results(gbk):
    # block size, codes per thread and query order change the schedule, not the arithmetic
    ix, x, cen, coarse, books = _index(gbk, 128, True)
    xq = torch.from_numpy(_queries(cen, 430, 300, 128)).cuda()
    ref = None
    for threads in (256, 384, 512):
        for u in (2, 4, 8):
            for by_list in (True, False):
                gbk.ivfpq_set_scan_options(ix, threads, by_list)
                gbk.ivfpq_set_tuning(ix, u, 2)
                D, I = ix.search(xq, 50, 8)
                if ref is None:
                    ref = (D, I)
                assert torch.equal(D, ref[0]) and torch.equal(I, ref[1])
    gbk.ivfpq_set_scan_options(ix, 256, True)
    gbk.ivfpq_set_tuning(ix, 4, 2)


def _groups(kq, npq):
    for kk in np.unique(kq):
        for nn in np.unique(npq):
            sel = np.nonzero((kq == kk) & (npq == nn))[0]
            if sel.size:
                yield int(kk), int(nn), sel


def _check_batched(D, I, off, kq, npq, xq, ix, coarse, books, direct):
    ex = ix.export()
    adc = Adc(ex, coarse, books)
    D, I, off = D.cpu().numpy(), I.cpu().numpy(), off.cpu().numpy()
    for kk, nn, sel in _groups(kq, npq):
        Do, Io = oracle.ivfadc_search(xq[sel], coarse, books, ex["list_off"], ex["codes"],
                                      ex["ids"], kk + 1, nn)
        Dg = np.stack([D[off[q]:off[q + 1]] for q in sel])
        Ig = np.stack([I[off[q]:off[q + 1]] for q in sel])
        check_strict(Dg, Ig, Do, Io, xq[sel], adc, direct, _ambiguous_probes(xq[sel], coarse, nn))


@pytest.mark.parametrize("precomputed", [True, False])
def test_batched_mixed_matches_oracle(gbk, precomputed):
    # one persistent launch over mixed k in {1, 10, 100} and nprobe in {1, 4, 8}; every
    # query's results are checked against the oracle's search with its own k and nprobe,
    # and the graph-captured replay returns the same bits
    ix, x, cen, coarse, books = _index(gbk, 128, precomputed)
    nq = 240
    xq = _queries(cen, 440, nq, 128)
    kq = np.array([1, 10, 100])[datagen.randint(441, 0, nq, 3)].astype(np.int32)
    npq = np.array([1, 4, 8])[datagen.randint(441, 0, nq, 3, stream=1)].astype(np.int32)
    xqt = torch.from_numpy(xq).cuda()
    kqt, npqt = torch.from_numpy(kq).cuda(), torch.from_numpy(npq).cuda()
    D, I, off, used = gbk.ivfpq_search_batched(ix, xqt, kqt, 100, npqt, 8)
    assert torch.equal(used, npqt)
    _check_batched(D, I, off, kq, npq, xq, ix, coarse, books, not precomputed)
    gr = gbk.BatchedGraph(ix, xqt, kqt, 100, npqt, 8)
    gr.launch()
    torch.cuda.synchronize()
    assert torch.equal(gr.D, D) and torch.equal(gr.I, I)


@pytest.mark.parametrize("alpha,shift", [(0.0, 0), (0.9, 1)])
def test_learned_routing_matches_oracle(gbk, alpha, shift):
    # nprobe chosen per query by a (seeded, untrained) network at an operating point: each
    # query's results equal the oracle's search at the nprobe the network chose
    ix, x, cen, coarse, books = _index(gbk, 128, True, nlist=64)  # 64 coarse features
    nq = 200
    xq = _queries(cen, 450, nq, 128)
    xqt = torch.from_numpy(xq).cuda()
    net = gbk.MLP(128 + 64, 256, 256, 9, seed=451)
    kq = np.full(nq, 10, np.int32)
    gbk.ivfpq_set_learned_route(ix, 0.0, 0)
    _, _, _, used0 = gbk.ivfpq_search_batched(ix, xqt, torch.from_numpy(kq).cuda(), 10, None, 32,
                                              mlp=net)
    gbk.ivfpq_set_learned_route(ix, alpha, shift)
    D, I, off, used = gbk.ivfpq_search_batched(ix, xqt, torch.from_numpy(kq).cuda(), 10, None, 32,
                                               mlp=net)
    u = used.cpu().numpy()
    assert np.all((u >= 1) & (u <= 32) & ((u & (u - 1)) == 0))
    assert np.all(u >= used0.cpu().numpy())  # a higher confidence or shift never probes fewer
    _check_batched(D, I, off, kq, u, xq, ix, coarse, books, False)
    gr = gbk.BatchedGraph(ix, xqt, torch.from_numpy(kq).cuda(), 10, None, 32, mlp=net)
    gr.launch()
    torch.cuda.synchronize()
    assert torch.equal(gr.I, I) and torch.equal(gr.nprobe_used, used)
    gbk.ivfpq_set_learned_route(ix, 0.0, 0)


def _pq_structured(seed, n, d, M, ncoarse):
    """Rows x = C[u] + R with well-separated coarse centres C and, in every sub-block m, the
    residual R^m one of 256 well-separated points P_m[j] plus small noise.  Rows 0..ncoarse-1
    take u = 0..ncoarse-1 and rows 0..255 take, in block m, point pi_m(row) for a seeded
    permutation pi_m, so that those rows seed one centroid per cluster on both levels."""
    dsub = d // M
    C = datagen.gaussian_matrix(seed, ncoarse, d) * 40.0
    P = datagen.gaussian_matrix(seed + 1, M * 256, dsub).reshape(M, 256, dsub) * 3.0
    u = datagen.randint(seed + 2, 0, n, ncoarse)
    u[:ncoarse] = np.arange(ncoarse)
    R = np.empty((n, d), np.float32)
    for m in range(M):
        j = datagen.randint(seed + 3, 0, n, 256, stream=m)
        j[:256] = np.argsort(datagen.hash_u64(seed + 4, 0, 256, stream=m))
        R[:, m * dsub:(m + 1) * dsub] = P[m][j]
    noise = datagen.gaussian_matrix(seed + 5, n, d) * 0.02
    return (C[u] + R + noise).astype(np.float32)


@pytest.mark.parametrize("d,M", [(128, 16), (96, 16), (64, 8)])
def test_gpu_pq_training_matches_oracle(gbk, d, M):
    # IVFPQIndex.train (coarse k-means, residuals, one 256-centroid k-means per sub-vector
    # block, read with the row stride d) against oracle.kmeans + oracle.train_pq given the
    # same rows and initial centroids: the same codebooks
    n, ncoarse = 12000, 16
    x = _pq_structured(460 + d, n, d, M, ncoarse)
    ix = gbk.IVFPQIndex(d, ncoarse, M)
    ix.train(torch.from_numpy(x).cuda(), niter=4, coarse_init=np.arange(ncoarse),
             pq_init=np.arange(256))
    ex = ix.export()
    co, _, _ = oracle.kmeans(x, np.arange(ncoarse), 4)
    np.testing.assert_allclose(ex["coarse"], co, rtol=1e-5, atol=1e-4)
    books = oracle.train_pq(oracle.residual_training_set(x, co), M, np.arange(256), 4)
    np.testing.assert_allclose(ex["pq"], books, rtol=1e-5, atol=2e-4)
