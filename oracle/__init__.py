"""CPU oracle for the similarity-search hot path (arXiv 1702.08734).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline / reference leg call it; the library (``paper_1702_08734_gb300``) never
imports it and has no CPU fallback.

The arithmetic lives in ``oracle.c`` (plain C, double precision, POSIX threads) and in
``mlp.py`` (numpy, double precision).  This file only compiles the C part with gcc and
marshals numpy arrays.  Functions and the passages they follow:

* ``kselect``      - section 2 "k-selection" (sorted k smallest / largest with indices)
* ``knn``          - Eq. (1), evaluated directly (not through Eq. (2))
* ``assign``       - nearest centroid, the coarse quantizer q1 of Eq. (3)
* ``kmeans``       - Lloyd's algorithm (sections 2 and 6.2)
* ``train_pq``     - product quantizer of section 2 trained on residuals of Eq. (3)
* ``ivfpq_encode`` - q1 + product-quantizer codes (section 2)
* ``ivf_bucket``   - the inverted file, lists in insertion order (section 2)
* ``ivfadc_search``- Algorithm 4 / Eq. (5), (6) and (10)
* ``ivfflat_search``- the inverted file of section 2 with uncompressed lists: Eq. (5) for
  the probed lists, then Eq. (1) directly for their vectors
* ``ivfadc_refine`` - Algorithm 4 for k' candidates, then Eq. (1) for those and the k best
* ``rotate``        - the OPQ pre-rotation y -> R y (sections 1 and 6.4), in double
* ``procrustes``    - the orthogonal R minimising ||x R^T - y||_F (numpy SVD)
* ``opq_train``     - non-parametric OPQ: alternating ``train_pq`` and ``procrustes``
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (plain gcc, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_POSIX_C_SOURCE=200809L", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.or_kselect.argtypes = [_f32p, _i64, _i64, _i32, _i32, _i32, _f32p, _i64p, _i64p,
                                       ctypes.c_int]
            lib.or_knn.argtypes = [_f32p, _i64, _f32p, _i64, _i32, _i32, _i32, _f64p, _i64p,
                                   ctypes.c_int]
            lib.or_pair_dist.argtypes = [_f32p, _f32p, _i32, _i64p, _i64p, _i64, _i32, _f64p]
            lib.or_assign.argtypes = [_f32p, _i64, _i32, _f32p, _i32, _i64p, _f64p, ctypes.c_int]
            lib.or_kmeans.argtypes = [_f32p, _i64, _i32, _i32, _i32, _i64p, _f32p, _f64p, _i64p,
                                      ctypes.c_int]
            lib.or_ivfpq_encode.argtypes = [_f32p, _i64, _i32, _f32p, _i32, _f32p, _i32, _i64p,
                                            _u8p, ctypes.c_int]
            lib.or_ivf_bucket.argtypes = [_i64p, _i64, _i32, _i64p, _i64p]
            lib.or_ivfadc_search.argtypes = [_f32p, _i64, _i32, _f32p, _i32, _f32p, _i32, _i64p,
                                             _u8p, _i64p, _i32, _i32, _i32, _f64p, _i64p, _i64p,
                                             ctypes.c_int]
            lib.or_ivfflat_search.argtypes = [_f32p, _i64, _i32, _f32p, _i32, _i64p, _f32p,
                                              _i64p, _i32, _i32, _f64p, _i64p, ctypes.c_int]
            lib.or_default_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _check(rc):
    if rc != 0:
        raise ValueError("oracle: invalid arguments (code %d)" % rc)


def default_threads() -> int:
    return int(_load().or_default_threads())


def kselect(vals, k: int, largest: bool = False, method: str = "heap", threads: int = 0,
            return_events: bool = False):
    """Row-wise k smallest (largest) values with their indices, sorted best first.

    Ties go to the lower index, NaN ranks last in both directions, -0 == +0; the
    returned values are the input's own float32 bits.  ``method`` is "heap" (one pass
    with a size-k heap) or "sort" (full sort of (value, index) pairs, first k)."""
    v = _c(vals, np.float32)
    if v.ndim == 1:
        v = v[None, :]
    rows, length = v.shape
    D = np.empty((rows, k), np.float32)
    I = np.empty((rows, k), np.int64)
    ev = np.empty(rows, np.int64) if return_events else None
    _check(_load().or_kselect(_p(v, _f32p), rows, length, k, int(largest),
                              0 if method == "heap" else 1, _p(D, _f32p), _p(I, _i64p),
                              _p(ev, _i64p) if ev is not None else None, threads))
    return (D, I, ev) if return_events else (D, I)


def knn(xq, xb, k: int, metric: str = "l2", threads: int = 0):
    """Exact k nearest neighbours (Eq. 1): squared L2 ascending, or inner product
    descending; double-precision distances; ties to the lower database id."""
    xq = _c(xq, np.float32)
    xb = _c(xb, np.float32)
    nq, d = xq.shape
    nb = xb.shape[0]
    D = np.empty((nq, k), np.float64)
    I = np.empty((nq, k), np.int64)
    _check(_load().or_knn(_p(xq, _f32p), nq, _p(xb, _f32p), nb, d, k,
                          0 if metric == "l2" else 1, _p(D, _f64p), _p(I, _i64p), threads))
    return D, I


def pair_dist(xq, xb, qi, bi, metric: str = "l2"):
    """Exact double-precision distance of each (query qi[p], database bi[p]) pair."""
    xq = _c(xq, np.float32)
    xb = _c(xb, np.float32)
    qi = _c(qi, np.int64).ravel()
    bi = _c(bi, np.int64).ravel()
    out = np.empty(qi.size, np.float64)
    _check(_load().or_pair_dist(_p(xq, _f32p), _p(xb, _f32p), xq.shape[1], _p(qi, _i64p),
                                _p(bi, _i64p), qi.size, 0 if metric == "l2" else 1,
                                _p(out, _f64p)))
    return out


def assign(x, centroids, threads: int = 0):
    """Nearest centroid per row (ties to the lowest index) and its squared distance."""
    x = _c(x, np.float32)
    c = _c(centroids, np.float32)
    a = np.empty(x.shape[0], np.int64)
    dist = np.empty(x.shape[0], np.float64)
    _check(_load().or_assign(_p(x, _f32p), x.shape[0], x.shape[1], _p(c, _f32p), c.shape[0],
                             _p(a, _i64p), _p(dist, _f64p), threads))
    return a, dist


def kmeans(x, init_idx, niter: int, threads: int = 0):
    """Lloyd's k-means from the given initial rows.  Returns (float32 centroids,
    objective before each update, number of empty-cluster splits)."""
    x = _c(x, np.float32)
    init_idx = _c(init_idx, np.int64)
    nc = init_idx.size
    n, d = x.shape
    cent = np.empty((nc, d), np.float32)
    obj = np.empty(max(niter, 1), np.float64)
    ns = np.zeros(1, np.int64)
    _check(_load().or_kmeans(_p(x, _f32p), n, d, nc, niter, _p(init_idx, _i64p),
                             _p(cent, _f32p), _p(obj, _f64p), _p(ns, _i64p), threads))
    return cent, obj[:niter], int(ns[0])


def ivfpq_encode(x, coarse, pq, threads: int = 0):
    """Coarse list and M-byte PQ code of each row; pq has shape (M, 256, d/M)."""
    x = _c(x, np.float32)
    coarse = _c(coarse, np.float32)
    pq = _c(pq, np.float32)
    M = pq.shape[0]
    n, d = x.shape
    lists = np.empty(n, np.int64)
    codes = np.empty((n, M), np.uint8)
    _check(_load().or_ivfpq_encode(_p(x, _f32p), n, d, _p(coarse, _f32p), coarse.shape[0],
                                   _p(pq, _f32p), M, _p(lists, _i64p), _p(codes, _u8p), threads))
    return lists, codes


def ivf_bucket(list_of, nlist: int):
    """Inverted-list offsets (nlist+1) and the batch positions in list order."""
    list_of = _c(list_of, np.int64)
    offsets = np.empty(nlist + 1, np.int64)
    order = np.empty(list_of.size, np.int64)
    _check(_load().or_ivf_bucket(_p(list_of, _i64p), list_of.size, nlist, _p(offsets, _i64p),
                                 _p(order, _i64p)))
    return offsets, order


def residual_training_set(x, coarse, threads: int = 0):
    """Residuals y - q1(y) of Eq. (3), in double, for training the fine quantizer."""
    a, _ = assign(x, coarse, threads)
    return x.astype(np.float64) - coarse[a].astype(np.float64)


def train_pq(residuals, M: int, init_idx, niter: int, threads: int = 0):
    """Product-quantizer codebooks (M, 256, d/M): k-means with 256 centroids on each
    sub-vector block of the residuals (section 2 "Product quantizer")."""
    r = np.asarray(residuals)
    n, d = r.shape
    dsub = d // M
    books = np.empty((M, 256, dsub), np.float32)
    for m in range(M):
        sub = np.ascontiguousarray(r[:, m * dsub:(m + 1) * dsub], dtype=np.float32)
        books[m], _, _ = kmeans(sub, init_idx, niter, threads)
    return books


def ivfadc_search(xq, coarse, pq, offsets, codes, ids, k: int, nprobe: int, form: str = "recon",
                  threads: int = 0, return_probes: bool = False):
    """IVFADC search (Algorithm 4): double-precision ADC distances, (+inf, -1) padding."""
    xq = _c(xq, np.float32)
    coarse = _c(coarse, np.float32)
    pq = _c(pq, np.float32)
    offsets = _c(offsets, np.int64)
    codes = _c(codes, np.uint8)
    ids = _c(ids, np.int64)
    nq, d = xq.shape
    D = np.empty((nq, k), np.float64)
    I = np.empty((nq, k), np.int64)
    probes = np.empty((nq, nprobe), np.int64)
    _check(_load().or_ivfadc_search(_p(xq, _f32p), nq, d, _p(coarse, _f32p), coarse.shape[0],
                                    _p(pq, _f32p), pq.shape[0], _p(offsets, _i64p),
                                    _p(codes, _u8p), _p(ids, _i64p), k, nprobe,
                                    0 if form == "recon" else 1, _p(D, _f64p), _p(I, _i64p),
                                    _p(probes, _i64p), threads))
    return (D, I, probes) if return_probes else (D, I)


def ivfflat_search(xq, coarse, offsets, vecs, ids, k: int, nprobe: int, threads: int = 0):
    """IVF-Flat search: the nprobe nearest centroids (exact, ties to the lower list), exact
    double-precision distances to every vector of those lists (``vecs`` and ``ids`` in list
    order), k smallest by (distance, id), (+inf, -1) padding."""
    xq = _c(xq, np.float32)
    coarse = _c(coarse, np.float32)
    offsets = _c(offsets, np.int64)
    vecs = _c(vecs, np.float32)
    ids = _c(ids, np.int64)
    nq, d = xq.shape
    D = np.empty((nq, k), np.float64)
    I = np.empty((nq, k), np.int64)
    _check(_load().or_ivfflat_search(_p(xq, _f32p), nq, d, _p(coarse, _f32p), coarse.shape[0],
                                     _p(offsets, _i64p), _p(vecs, _f32p), _p(ids, _i64p), k,
                                     nprobe, _p(D, _f64p), _p(I, _i64p), threads))
    return D, I


def ivfadc_refine(xq, xb, coarse, pq, offsets, codes, ids, k: int, nprobe: int, kprime: int,
                  threads: int = 0):
    """IVFADC followed by exact re-ranking: the kprime best ADC candidates (Algorithm 4),
    their exact distances (Eq. 1, double) to the vectors xb[id], and the k best by
    (distance, id); (+inf, -1) padding.  Also returns the candidates' ADC distances and ids."""
    Dc, Ic = ivfadc_search(xq, coarse, pq, offsets, codes, ids, kprime, nprobe, threads=threads)
    nq = Dc.shape[0]
    D = np.full((nq, k), np.inf)
    I = np.full((nq, k), -1, np.int64)
    for q in range(nq):
        cand = Ic[q][Ic[q] >= 0]
        if cand.size == 0:
            continue
        ex = pair_dist(xq, xb, np.full(cand.size, q), cand)
        o = np.lexsort((cand, ex))[:k]
        D[q, :o.size] = ex[o]
        I[q, :o.size] = cand[o]
    return D, I, Dc, Ic


def rotate(x, R):
    """Rows y of x replaced by R y, computed in double and rounded to float32 once."""
    x = np.asarray(x, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    return (x @ R.T).astype(np.float32)


def procrustes(x, y):
    """The orthogonal R minimising ||x R^T - y||_F over the rows: U V^T for the SVD
    y^T x = U S V^T, in double (the library routine numpy.linalg.svd as the step)."""
    A = np.asarray(y, np.float64).T @ np.asarray(x, np.float64)
    U, _, Vt = np.linalg.svd(A)
    return U @ Vt


def opq_train(x, M: int, init_idx, niter: int, pq_niter: int, threads: int = 0):
    """OPQ, non-parametric form (cited, not specified, by the paper): from R = I, niter
    times train the product quantizer of x R^T (train_pq from the rows init_idx), encode
    and reconstruct every row, and replace R by procrustes(x, reconstruction).  Returns
    (R float32 [d][d], the last codebooks)."""
    x = _c(x, np.float32)
    n, d = x.shape
    R = np.eye(d)
    books = None
    for _ in range(niter):
        xr = rotate(x, R)
        books = train_pq(xr, M, init_idx, pq_niter, threads)
        _, codes = ivfpq_encode(xr, np.zeros((1, d), np.float32), books, threads)
        y = np.concatenate([books[m][codes[:, m]] for m in range(M)], axis=1)
        R = procrustes(x, y)
    return R.astype(np.float32), books
