"""Pins for the learned-nprobe network's oracle: central finite differences, torch autograd
in float64 (a library routine), and torch's own Adam."""
import numpy as np
import pytest

from oracle import mlp
from paper_1702_08734_gb300 import datagen

SIZES = (7, 6, 5, 4)


def _setup(seed=3, n=11):
    nparam = 7 * 6 + 6 + 6 * 5 + 5 + 5 * 4 + 4
    p = mlp.init_params(SIZES, datagen.uniform24(seed, 0, nparam).astype(np.float64))
    F = datagen.gaussian_matrix(seed + 1, n, 7).astype(np.float64)
    y = datagen.randint(seed + 2, 0, n, 4)
    return p, F, y


def test_init_bounds_and_shapes():
    p, _, _ = _setup()
    assert p["W1"].shape == (6, 7) and p["b3"].shape == (4,)
    assert np.abs(p["W1"]).max() <= 1 / np.sqrt(7) and np.abs(p["W3"]).max() <= 1 / np.sqrt(5)


def test_gradients_match_central_differences():
    p, F, y = _setup()
    _, g = mlp.loss_and_grads(p, F, y)
    h = 1e-6
    for name in mlp.PARAM_NAMES:
        flat = p[name].reshape(-1)
        for j in range(0, flat.size, max(1, flat.size // 9)):
            old = flat[j]
            flat[j] = old + h
            lp, _ = mlp.loss_and_grads(p, F, y)
            flat[j] = old - h
            lm, _ = mlp.loss_and_grads(p, F, y)
            flat[j] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name].reshape(-1)[j]) < 1e-7 + 1e-5 * abs(fd), (name, j)


def test_gradients_match_torch_autograd():
    torch = pytest.importorskip("torch")
    p, F, y = _setup(seed=9, n=17)
    loss, g = mlp.loss_and_grads(p, F, y)
    tp = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in p.items()}
    h1 = torch.relu(torch.tensor(F) @ tp["W1"].T + tp["b1"])
    h2 = torch.relu(h1 @ tp["W2"].T + tp["b2"])
    z = h2 @ tp["W3"].T + tp["b3"]
    tl = torch.nn.functional.cross_entropy(z, torch.tensor(y))
    tl.backward()
    assert abs(tl.item() - loss) < 1e-12
    for k in mlp.PARAM_NAMES:
        np.testing.assert_allclose(g[k], tp[k].grad.numpy(), rtol=1e-10, atol=1e-14)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    p, F, y = _setup(seed=12, n=9)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(x) for k, x in p.items()}
    tp = [torch.tensor(p[k], dtype=torch.float64, requires_grad=True) for k in mlp.PARAM_NAMES]
    opt = torch.optim.Adam(tp, lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    cur = p
    for t in range(1, 4):
        _, g = mlp.loss_and_grads(cur, F, y)
        cur, m, v = mlp.adam_step(cur, g, m, v, t, 3e-3)
        for tt, k in zip(tp, mlp.PARAM_NAMES):
            tt.grad = torch.tensor(g[k])
        opt.step()
    for tt, k in zip(tp, mlp.PARAM_NAMES):
        np.testing.assert_allclose(cur[k], tt.detach().numpy(), rtol=1e-12, atol=1e-15)


def test_features_definition():
    xq = np.ones((2, 3))
    d = np.array([[2.0, 3.0, 4.0], [0.0, 1.0, 1.0]])
    f = mlp.coarse_features(xq, d, nfeat=3)
    np.testing.assert_allclose(f[0], [1, 1, 1, 0.0, 0.5, 1.0])
    assert f[1, 3] == -1.0 and f[1, 4] == 1e12 - 1.0
