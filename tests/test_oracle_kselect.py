"""Pins for the oracle's k-selection and exact k-NN (CPU only).

Each check ties the oracle to something other than itself: Python's and numpy's own
sorts, scipy's distance routine, hand-computed cases, and the Appendix's closed form for
the expected number of successive min-k events of a sequential scan.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1702_08734_gb300 import datagen


def _py_sorted_first_k(row, k, largest):
    # Library sort with an explicit key: NaN last, then value (negated for largest), then index.
    def key(i):
        v = float(row[i])
        if math.isnan(v):
            return (1, 0.0, i)
        return (0, -v if largest else v, i)
    return sorted(range(len(row)), key=key)[:k]


@pytest.mark.parametrize("largest", [False, True])
@pytest.mark.parametrize("method", ["heap", "sort"])
def test_kselect_matches_library_sort_with_specials(largest, method):
    rng = np.random.default_rng(5)
    rows, length = 40, 37
    v = rng.integers(-4, 5, size=(rows, length)).astype(np.float32)  # heavy ties
    v[0, :5] = np.nan
    v[1, 3] = np.inf
    v[1, 4] = -np.inf
    v[2, :] = -0.0
    v[2, ::2] = 0.0
    v[3, :] = np.nan
    for k in (1, 5, 37):
        D, I = oracle.kselect(v, k, largest=largest, method=method)
        for r in range(rows):
            ref = _py_sorted_first_k(v[r], k, largest)
            assert list(I[r]) == ref, (r, k)
            np.testing.assert_array_equal(D[r].view(np.uint32), v[r, ref].view(np.uint32))


def test_kselect_numpy_lexsort_and_invariants():
    v = datagen.uniform_matrix(201, 64, 4096)  # 24-bit uniforms: ties occur
    k = 100
    D, I = oracle.kselect(v, k)
    for r in range(v.shape[0]):
        order = np.lexsort((np.arange(v.shape[1]), v[r]))[:k]
        np.testing.assert_array_equal(I[r], order)
        assert np.all(np.diff(D[r]) >= 0)
        assert len(set(I[r].tolist())) == k
        assert np.sum(v[r] < D[r, -1]) <= k - 1


def test_kselect_len_shorter_than_k_pads():
    v = np.array([[3.0, 1.0, 2.0]], np.float32)
    D, I = oracle.kselect(v, 5)
    assert I[0].tolist() == [1, 2, 0, -1, -1]
    assert np.isnan(D[0, 3]) and np.isnan(D[0, 4])


def test_successive_min_events_k1_are_records():
    # k=1 on a sequential scan: a new running minimum enters exactly at each strict record.
    rng = np.random.default_rng(11)
    v = rng.permutation(5000).astype(np.float32)[None, :]
    _, _, ev = oracle.kselect(v, 1, return_events=True)
    prefix_min = np.minimum.accumulate(v[0])
    records = 1 + int(np.sum(v[0, 1:] < prefix_min[:-1]))
    assert ev[0] == records


def test_successive_min_events_match_appendix_closed_form():
    # Appendix: pi(l, k, 1, 1) = k + k (H_l - H_k) for a random permutation of distinct keys.
    l, k, rows = 2000, 16, 600
    rng = np.random.default_rng(3)
    v = np.stack([rng.permutation(l) for _ in range(rows)]).astype(np.float32)
    _, _, ev = oracle.kselect(v, k, return_events=True)
    H = lambda n: sum(1.0 / i for i in range(1, n + 1))
    expect = k + k * (H(l) - H(k))
    assert abs(ev.mean() - expect) / expect < 0.03, (ev.mean(), expect)
    _, _, ev1 = oracle.kselect(v, 1, return_events=True)
    assert abs(ev1.mean() - H(l)) / H(l) < 0.08


def test_knn_hand_case_1d_ties_to_lower_id():
    xb = np.array([[0.0], [1.0], [3.0], [6.0], [10.0]], np.float32)
    xq = np.array([[2.0]], np.float32)
    D, I = oracle.knn(xq, xb, 3)
    assert I[0].tolist() == [1, 2, 0]
    assert D[0].tolist() == [1.0, 1.0, 4.0]
    D, I = oracle.knn(xq, xb, 2, metric="ip")
    assert I[0].tolist() == [4, 3] and D[0].tolist() == [20.0, 12.0]


def test_knn_lattice_2d():
    g = np.array([(i, j) for i in range(4) for j in range(4)], np.float32)  # id = 4i + j
    q = np.array([[1.5, 1.5]], np.float32)
    D, I = oracle.knn(q, g, 6)
    assert I[0, :4].tolist() == [5, 6, 9, 10] and np.all(D[0, :4] == 0.5)
    assert np.all(D[0, 4:] == 2.5) and I[0, 4:].tolist() == [1, 2]


def test_knn_matches_scipy_cdist():
    scipy_distance = pytest.importorskip("scipy.spatial.distance")
    xb = datagen.gaussian_matrix(7, 3000, 24)
    xq = datagen.gaussian_matrix(8, 50, 24)
    D, I = oracle.knn(xq, xb, 20)
    ref = scipy_distance.cdist(xq.astype(np.float64), xb.astype(np.float64), "sqeuclidean")
    for q in range(xq.shape[0]):
        order = np.lexsort((np.arange(xb.shape[0]), ref[q]))[:20]
        np.testing.assert_array_equal(I[q], order)
        np.testing.assert_allclose(D[q], ref[q, order], rtol=1e-12)
    Dp, Ip = oracle.knn(xq, xb, 20, metric="ip")
    ip = xq.astype(np.float64) @ xb.astype(np.float64).T
    for q in range(xq.shape[0]):
        order = np.lexsort((np.arange(xb.shape[0]), -ip[q]))[:20]
        np.testing.assert_array_equal(Ip[q], order)


def test_knn_duplicate_rows_and_eq2_identity():
    xb = datagen.gaussian_matrix(9, 200, 16)
    xb[150] = xb[20]
    xb[199] = xb[20]
    D, I = oracle.knn(xb[20:21], xb, 3)
    assert I[0].tolist() == [20, 150, 199] and np.all(D[0] == 0.0)
    # Eq. (2): ||x||^2 + ||y||^2 - 2<x,y> equals the direct squared distance.
    x = xb[3].astype(np.float64)
    Dd, Id = oracle.knn(xb[3:4], xb, 200)
    y = xb[Id[0]].astype(np.float64)
    eq2 = (x @ x) + (y * y).sum(1) - 2 * (y @ x)
    np.testing.assert_allclose(Dd[0], eq2, atol=1e-9)


def test_pair_dist_matches_knn():
    xb = datagen.gaussian_matrix(21, 500, 8)
    xq = datagen.gaussian_matrix(22, 5, 8)
    D, I = oracle.knn(xq, xb, 4)
    qi = np.repeat(np.arange(5), 4)
    pd = oracle.pair_dist(xq, xb, qi, I.ravel())
    np.testing.assert_array_equal(pd, D.ravel())


def test_event_distribution_matches_appendix_recurrence():
    # Brute force over every permutation of l distinct keys: the distribution of the number
    # of successive min-k elements the oracle's single scan meets equals gamma(l, m, k) of
    # the Appendix recurrence (tests/golden/appendix_min_k_distribution.txt, exact fractions)
    import itertools
    import math
    import os
    from fractions import Fraction
    path = os.path.join(os.path.dirname(__file__), "golden", "appendix_min_k_distribution.txt")
    want = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        l, k, m, num, den = map(int, line.split())
        want.setdefault((l, k), {})[m] = Fraction(num, den)
    assert len(want) == sum(min(3, l) for l in range(1, 8))
    for (l, k), dist in want.items():
        perms = np.array(list(itertools.permutations(range(l))), dtype=np.float32)
        _, _, ev = oracle.kselect(perms, k, return_events=True)
        vals, cnt = np.unique(ev, return_counts=True)
        got = {int(m): Fraction(int(c), math.factorial(l)) for m, c in zip(vals, cnt)}
        assert got == dist, (l, k, got, dist)
