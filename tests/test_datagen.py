"""The seeded input generator: published SplitMix64 outputs and distribution sanity."""
import numpy as np

from paper_1702_08734_gb300 import datagen


def test_splitmix64_published_first_outputs():
    # SplitMix64 seeded with state 0 emits mix64(gamma), mix64(2 gamma), ...
    g = 0x9E3779B97F4A7C15
    assert datagen._mix64_int(g) == 0xE220A8397B1DCDAF
    assert datagen._mix64_int(2 * g) == 0x6E789E6AA1B965F4
    z = datagen._mix64(np.array([g, (2 * g) % (1 << 64)], dtype=np.uint64))
    assert z.tolist() == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]


def test_random_access_and_distributions():
    a = datagen.normal(5, 0, 20000)
    b = datagen.normal(5, 1000, 500)
    np.testing.assert_array_equal(a[1000:1500], b)
    assert abs(a.mean()) < 0.03 and abs(a.var() - 1) < 0.03
    u = datagen.uniform24(6, 0, 100000)
    assert u.min() >= 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.01
    assert np.all(u * (1 << 24) == np.floor(u * (1 << 24)))
    m = datagen.gaussian_matrix(7, 300, 128)
    np.testing.assert_array_equal(m[100:110], datagen.gaussian_matrix(7, 10, 128, row0=100))
    s = datagen.anisotropic_sigmas(96)
    assert s[0] == 1.0 and abs(s[-1] - 0.05) < 1e-7
    p = datagen.permutation_prefix(9, 1000, 1000)
    assert sorted(p.tolist()) == list(range(1000))
