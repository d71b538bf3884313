"""The device generator reproduces the host generator (integer hashing bit for bit)."""
import numpy as np
import pytest
import torch

from paper_1702_08734_gb300 import datagen

pytestmark = pytest.mark.gpu


def test_hash_and_values_match_host():
    h = datagen.hash_u64_cuda(17, 1000, 5000, stream=1).cpu().numpy().view(np.uint64)
    np.testing.assert_array_equal(h, datagen.hash_u64(17, 1000, 5000, stream=1))
    g = datagen.gaussian_matrix_cuda(18, 300, 128, row0=77).cpu().numpy()
    ref = datagen.gaussian_matrix(18, 300, 128, row0=77)
    assert (g != ref).mean() < 1e-4
    np.testing.assert_allclose(g, ref, rtol=1e-6, atol=1e-6)
    cen = datagen.mixture_centres(19, 64, 32)
    m = datagen.mixture_points_cuda(cen, 20, 1000, row0=5).cpu().numpy()
    np.testing.assert_allclose(m, datagen.mixture_points(cen, 20, 1000, row0=5), rtol=1e-6,
                               atol=1e-5)
