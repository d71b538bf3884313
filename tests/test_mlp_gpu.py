"""Learned-nprobe network: GPU forward / backward / Adam vs the float64 oracle.

The oracle is given the same BF16-rounded weights the kernels read, so forward and
gradients agree to float32-accumulation accuracy; Adam is checked on the master copy."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_1702_08734_gb300 import datagen

pytestmark = pytest.mark.gpu
SIZES = (192, 256, 256, 9)


def _init(seed=1):
    n = sum(a * b + a for a, b in [(256, 192), (256, 256), (9, 256)])
    p = omlp.init_params(SIZES, datagen.uniform24(seed, 0, n).astype(np.float64))
    flat = np.concatenate([p[k].ravel() for k in omlp.PARAM_NAMES]).astype(np.float32)
    return flat


def _unflat(flat, rnd=True):
    out, pos = {}, 0
    shapes = [(256, 192), (256,), (256, 256), (256,), (9, 256), (9,)]
    for name, shp in zip(omlp.PARAM_NAMES, shapes):
        cnt = int(np.prod(shp))
        v = torch.from_numpy(np.ascontiguousarray(flat[pos:pos + cnt]))
        if rnd and name.startswith("W"):  # the kernels read weight matrices as BF16
            v = v.to(torch.bfloat16).to(torch.float32)
        out[name] = v.numpy().astype(np.float64).reshape(shp)
        pos += cnt
    return out


def _batch(seed, B=512):
    X = datagen.gaussian_matrix(seed, B, 192)
    y = datagen.randint(seed + 1, 0, B, 9).astype(np.int32)
    return X, y


def test_forward_matches_oracle(gbk):
    flat = _init()
    net = gbk.MLP(*SIZES, params=flat)
    X, _ = _batch(3)
    z, cls = net.forward(torch.from_numpy(X).cuda())
    zo, _ = omlp.forward(_unflat(flat), X)
    np.testing.assert_allclose(z.cpu().numpy(), zo, rtol=1e-4, atol=1e-4)
    assert (cls.cpu().numpy() == zo.argmax(1)).mean() > 0.99


def test_gradients_match_oracle(gbk):
    flat = _init(2)
    net = gbk.MLP(*SIZES, params=flat)
    X, y = _batch(5)
    loss = net.train_step(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), update=False)
    g = net.grads().cpu().numpy()
    lo, go = omlp.loss_and_grads(_unflat(flat), X, y)
    assert abs(loss.item() - lo) < 1e-4 * max(1, abs(lo))
    pos = 0
    for name in omlp.PARAM_NAMES:
        ref = go[name].ravel()
        got = g[pos:pos + ref.size]
        pos += ref.size
        scale = np.abs(ref).max() + 1e-12
        assert np.abs(got - ref).max() <= 2e-3 * scale, name


def test_adam_step_matches_oracle(gbk):
    flat = _init(4)
    net = gbk.MLP(*SIZES, params=flat)
    X, y = _batch(7)
    Xt, yt = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    master = _unflat(flat, rnd=False)
    m = {k: np.zeros_like(v) for k, v in master.items()}
    v = {k: np.zeros_like(x) for k, x in master.items()}
    for t in range(1, 4):
        net.train_step(Xt, yt, lr=1e-3, update=False)
        g = net.grads().cpu().numpy().astype(np.float64)
        gd, pos = {}, 0
        for name in omlp.PARAM_NAMES:
            gd[name] = g[pos:pos + master[name].size].reshape(master[name].shape)
            pos += master[name].size
        master, m, v = omlp.adam_step(master, gd, m, v, t, 1e-3)
        net.train_step(Xt, yt, lr=1e-3, update=True)
    got = net.params().cpu().numpy()
    ref = np.concatenate([master[k].ravel() for k in omlp.PARAM_NAMES])
    np.testing.assert_allclose(got, ref, rtol=1e-4, atol=1e-6)


def test_training_reduces_loss_and_is_deterministic(gbk):
    flat = _init(9)
    X, y = _batch(11, B=2048)
    # learnable labels: the class is a function of the features
    y = (np.argmax(X[:, :9], axis=1)).astype(np.int32)
    runs = []
    for _ in range(2):
        net = gbk.MLP(*SIZES, params=flat)
        Xt, yt = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
        l0 = net.train_step(Xt, yt, update=False).item()
        for _ in range(60):
            net.train_step(Xt, yt, lr=3e-3)
        l1 = net.train_step(Xt, yt, update=False).item()
        runs.append((l0, l1, net.params().cpu().numpy()))
    assert runs[0][1] < 0.5 * runs[0][0], runs[0][:2]
    np.testing.assert_array_equal(runs[0][2], runs[1][2])


@pytest.mark.parametrize("sizes", [(100, 70, 50, 5), (64, 256, 33, 40), (300, 64, 64, 9)])
def test_forward_other_sizes_match_oracle(gbk, sizes):
    # shapes other than the learned-nprobe network's: ragged tiles in every layer
    n_in, h1, h2, n_out = sizes
    shapes = [(h1, n_in), (h1,), (h2, h1), (h2,), (n_out, h2), (n_out,)]
    n = sum(int(np.prod(s)) for s in shapes)
    p = omlp.init_params(sizes, datagen.uniform24(7, 0, n).astype(np.float64))
    flat = np.concatenate([p[k].ravel() for k in omlp.PARAM_NAMES]).astype(np.float32)
    net = gbk.MLP(*sizes, params=flat)
    X = datagen.gaussian_matrix(8, 77, n_in)  # a ragged last block of rows
    z, cls = net.forward(torch.from_numpy(X).cuda())
    ref, pos = {}, 0
    for name, shp in zip(omlp.PARAM_NAMES, shapes):
        cnt = int(np.prod(shp))
        v = torch.from_numpy(np.ascontiguousarray(flat[pos:pos + cnt]))
        if name.startswith("W"):
            v = v.to(torch.bfloat16).to(torch.float32)
        ref[name] = v.numpy().astype(np.float64).reshape(shp)
        pos += cnt
    zo, _ = omlp.forward(ref, X)
    np.testing.assert_allclose(z.cpu().numpy(), zo, rtol=1e-4, atol=1e-4)
    assert (cls.cpu().numpy() == zo.argmax(1)).mean() > 0.97
