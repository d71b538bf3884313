"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and the oracle.

This module holds no arithmetic of the similarity-search method itself: it only turns
(seed, stream, counter) triples into numbers.  Every value is a pure function of its
counter, so any row of any matrix can be regenerated on its own (random access), which
is what lets the oracle check sampled rows of workloads too large to hold twice.

Generator (counter-based, after SplitMix64 by Steele, Lea and Flood, OOPSLA 2014):
    key(seed, stream) = mix64(seed ^ (stream << 48) ^ 0x5851F42D4C957F2D)
    h(key, i)         = mix64(key + (i + 1) * 0x9E3779B97F4A7C15)   (mod 2**64)
    mix64(z):  z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
               z *= 0x94D049BB133111EB; z ^= z >> 31
Derived draws:
    uniform24(i) = (h(i) >> 40) * 2**-24                  -> float32 in [0, 1), 2**24 levels
    normal(i)    = Box-Muller in float64 on u1 = ((h(2i) >> 11) + 1) * 2**-53 (in (0, 1])
                   and u2 = (h(2i+1) >> 11) * 2**-53, rounded once to float32
    randint(i,n) = h(i) mod n

The 24-bit uniform deliberately has repeated values (about 4 ties per 65,536-long row
near the low end), so k-selection's tie rule is exercised by the benchmark inputs.
"""
from __future__ import annotations

import numpy as np

_M64 = (1 << 64) - 1
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def _mix64_int(z: int) -> int:
    z &= _M64
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) & _M64
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) & _M64
    z ^= z >> 31
    return z


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> np.uint64(30))
    z = z * _C1
    z = z ^ (z >> np.uint64(27))
    z = z * _C2
    z = z ^ (z >> np.uint64(31))
    return z


def stream_key(seed: int, stream: int = 0) -> int:
    return _mix64_int((seed ^ (stream << 48) ^ 0x5851F42D4C957F2D) & _M64)


def hash_u64(seed: int, start: int, count: int, stream: int = 0) -> np.ndarray:
    """h(key(seed, stream), i) for i in [start, start + count)."""
    key = np.uint64(stream_key(seed, stream))
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix64(key + i * _GAMMA)


def uniform24(seed: int, start: int, count: int, stream: int = 0) -> np.ndarray:
    h = hash_u64(seed, start, count, stream)
    return ((h >> np.uint64(40)).astype(np.float64) * 2.0 ** -24).astype(np.float32)


def normal(seed: int, start: int, count: int, stream: int = 0) -> np.ndarray:
    h = hash_u64(seed, 2 * start, 2 * count, stream)
    u1 = ((h[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (h[1::2] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return z.astype(np.float32)


def randint(seed: int, start: int, count: int, n: int, stream: int = 0) -> np.ndarray:
    return (hash_u64(seed, start, count, stream) % np.uint64(n)).astype(np.int64)


def _chunked(fn, seed, total, stream, chunk=1 << 24, **kw):
    out = np.empty(total, dtype=np.float32)
    for s in range(0, total, chunk):
        c = min(chunk, total - s)
        out[s:s + c] = fn(seed, s, c, stream=stream, **kw)
    return out


# ---------------------------------------------------------------------------
# Workload recipes (shapes and distributions of the paper's workloads)
# ---------------------------------------------------------------------------

def gaussian_matrix(seed: int, n: int, d: int, row0: int = 0) -> np.ndarray:
    """Rows row0..row0+n-1 of an i.i.d. N(0,1) float32 matrix with d columns."""
    if n * d <= (1 << 24):
        return normal(seed, row0 * d, n * d).reshape(n, d)
    out = np.empty((n, d), dtype=np.float32)
    step = max(1, (1 << 24) // d)
    for r in range(0, n, step):
        c = min(step, n - r)
        out[r:r + c] = normal(seed, (row0 + r) * d, c * d).reshape(c, d)
    return out


def uniform_matrix(seed: int, rows: int, cols: int, row0: int = 0) -> np.ndarray:
    """Rows of an i.i.d. U[0,1) float32 matrix (24-bit levels, so ties occur)."""
    out = np.empty((rows, cols), dtype=np.float32)
    step = max(1, (1 << 24) // cols)
    for r in range(0, rows, step):
        c = min(step, rows - r)
        out[r:r + c] = uniform24(seed, (row0 + r) * cols, c * cols).reshape(c, cols)
    return out


def mixture_centres(seed: int, ncentres: int, d: int, std: float = 2.0) -> np.ndarray:
    """Centres ~ N(0, std^2 I); std=2 gives the N(0, 4I) centres of the IVFADC workload."""
    return (gaussian_matrix(seed, ncentres, d) * np.float32(std)).astype(np.float32)


def mixture_points(centres: np.ndarray, seed: int, n: int, row0: int = 0) -> np.ndarray:
    """Points = centre[u] + N(0, I), u uniform over centres (stream 0), noise stream 1."""
    nc, d = centres.shape
    u = randint(seed, row0, n, nc, stream=0)
    out = np.empty((n, d), dtype=np.float32)
    step = max(1, (1 << 24) // d)
    for r in range(0, n, step):
        c = min(step, n - r)
        noise = normal(seed, (row0 + r) * d, c * d, stream=1).reshape(c, d)
        out[r:r + c] = centres[u[r:r + c]] + noise
    return out


def anisotropic_sigmas(d: int, lo: float = 0.05) -> np.ndarray:
    """Per-dimension std decaying geometrically from 1 to `lo` (PCA-like spectrum)."""
    j = np.arange(d, dtype=np.float64)
    return (lo ** (j / max(1, d - 1))).astype(np.float32)


def anisotropic_points(seed: int, n: int, d: int, row0: int = 0) -> np.ndarray:
    return (gaussian_matrix(seed, n, d, row0) * anisotropic_sigmas(d)[None, :]).astype(np.float32)


def permutation_prefix(seed: int, n: int, m: int) -> np.ndarray:
    """First m entries of a seeded random permutation of range(n): the k-means init draw.

    Sort-by-hash of the counters; ties of the 64-bit hash are broken by position."""
    h = hash_u64(seed, 0, n, stream=7)
    order = np.lexsort((np.arange(n), h))
    return order[:m].astype(np.int64)


# ---------------------------------------------------------------------------
# The same generator evaluated on a CUDA device (torch), for workloads too large to
# generate on the host.  Integer hashing is bit-identical to the numpy version (int64
# arithmetic wraps mod 2**64; right shifts are masked to be logical); Box-Muller runs in
# float64 on the device, whose log/cos may differ from the host's in the last double ulp,
# so an N(0,1) value can differ by one float32 ulp in rare (~1e-8) cases.
# ---------------------------------------------------------------------------

def _t_signed(v: int) -> int:
    v &= _M64
    return v - (1 << 64) if v >= (1 << 63) else v


def _t_shr(z, s):
    import torch
    return (z >> s) & torch.tensor(_t_signed((1 << (64 - s)) - 1), dtype=torch.int64,
                                   device=z.device)


def _t_mix64(z):
    z = z ^ _t_shr(z, 30)
    z = z * _t_signed(0xBF58476D1CE4E5B9)
    z = z ^ _t_shr(z, 27)
    z = z * _t_signed(0x94D049BB133111EB)
    z = z ^ _t_shr(z, 31)
    return z


def hash_u64_cuda(seed: int, start: int, count: int, stream: int = 0, device="cuda"):
    """h(key(seed, stream), i) as int64 bit patterns on the device."""
    import torch
    key = _t_signed(stream_key(seed, stream))
    i = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    return _t_mix64(key + i * _t_signed(0x9E3779B97F4A7C15))


def normal_cuda(seed: int, start: int, count: int, stream: int = 0, device="cuda"):
    import torch
    h = hash_u64_cuda(seed, 2 * start, 2 * count, stream, device)
    u1 = (_t_shr(h[0::2], 11).to(torch.float64) + 1.0) * 2.0 ** -53
    u2 = _t_shr(h[1::2], 11).to(torch.float64) * 2.0 ** -53
    return (torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * np.pi * u2)).to(torch.float32)


def randint_cuda(seed: int, start: int, count: int, n: int, stream: int = 0, device="cuda"):
    """h mod n for n a power of two (the only case the workloads use)."""
    assert n & (n - 1) == 0
    return hash_u64_cuda(seed, start, count, stream, device) & (n - 1)


def gaussian_matrix_cuda(seed: int, n: int, d: int, row0: int = 0, device="cuda"):
    import torch
    out = torch.empty((n, d), dtype=torch.float32, device=device)
    step = max(1, (1 << 24) // d)
    for r in range(0, n, step):
        c = min(step, n - r)
        out[r:r + c] = normal_cuda(seed, (row0 + r) * d, c * d, device=device).view(c, d)
    return out


def mixture_points_cuda(centres, seed: int, n: int, row0: int = 0, device="cuda"):
    """Device version of mixture_points (centres: host or device float32 [nc][d])."""
    import torch
    cen = torch.as_tensor(centres, device=device)
    nc, d = cen.shape
    out = torch.empty((n, d), dtype=torch.float32, device=device)
    step = max(1, (1 << 24) // d)
    for r in range(0, n, step):
        c = min(step, n - r)
        u = randint_cuda(seed, row0 + r, c, nc, stream=0, device=device)
        noise = normal_cuda(seed, (row0 + r) * d, c * d, stream=1, device=device).view(c, d)
        out[r:r + c] = cen[u] + noise
    return out
