"""Double-precision CPU oracle for the learned-nprobe network.  TEST INFRASTRUCTURE ONLY.

The network maps a per-query feature vector f (the query followed by features of its
nearest coarse-centroid distances) to logits over nprobe classes:
    h1 = relu(W1 f + b1),  h2 = relu(W2 h1 + b2),  z = W3 h2 + b3
trained with the mean softmax cross-entropy of integer labels and Adam
(Kingma & Ba, 2015: beta1, beta2, eps, bias-corrected moments).  Weights are stored
out x in, row-major, as in the CUDA kernels' parameter buffer.  Everything here is
plain numpy in float64; there is no blocking or fusion.
"""
from __future__ import annotations

import numpy as np

PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def init_params(sizes, seed_uniforms):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) initialisation from given U[0,1) draws.

    sizes = (n_in, h1, h2, n_out); seed_uniforms holds at least as many U[0,1) numbers as
    there are parameters, consumed in PARAM_NAMES order."""
    n_in, h1, h2, n_out = sizes
    shapes = [(h1, n_in), (h1,), (h2, h1), (h2,), (n_out, h2), (n_out,)]
    fan = [n_in, n_in, h1, h1, h2, h2]
    u = np.asarray(seed_uniforms, np.float64)
    out, pos = {}, 0
    for name, shp, fi in zip(PARAM_NAMES, shapes, fan):
        cnt = int(np.prod(shp))
        bound = 1.0 / np.sqrt(fi)
        out[name] = ((u[pos:pos + cnt] * 2.0 - 1.0) * bound).reshape(shp)
        pos += cnt
    return out


def forward(p, F):
    F = np.asarray(F, np.float64)
    a1 = F @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    z = h2 @ p["W3"].T + p["b3"]
    return z, (F, a1, h1, a2, h2)


def loss_and_grads(p, F, labels):
    """Mean cross-entropy of softmax(z) against labels, and its analytic gradient."""
    z, (F, a1, h1, a2, h2) = forward(p, F)
    n = z.shape[0]
    labels = np.asarray(labels, np.int64)
    zmax = z.max(axis=1, keepdims=True)
    e = np.exp(z - zmax)
    s = e.sum(axis=1, keepdims=True)
    logp = z - zmax - np.log(s)
    loss = -logp[np.arange(n), labels].mean()
    dz = e / s
    dz[np.arange(n), labels] -= 1.0
    dz /= n
    g = {}
    g["W3"] = dz.T @ h2
    g["b3"] = dz.sum(0)
    dh2 = dz @ p["W3"]
    da2 = dh2 * (a2 > 0)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(0)
    dh1 = da2 @ p["W2"]
    da1 = dh1 * (a1 > 0)
    g["W1"] = da1.T @ F
    g["b1"] = da1.sum(0)
    return loss, g


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns new (params, m, v)."""
    newp, newm, newv = {}, {}, {}
    for k in PARAM_NAMES:
        newm[k] = beta1 * m[k] + (1 - beta1) * g[k]
        newv[k] = beta2 * v[k] + (1 - beta2) * g[k] * g[k]
        mhat = newm[k] / (1 - beta1 ** t)
        vhat = newv[k] / (1 - beta2 ** t)
        newp[k] = p[k] - lr * mhat / (np.sqrt(vhat) + eps)
    return newp, newm, newv


def coarse_features(xq, coarse_dist, nfeat=64):
    """Feature vector of each query: the query itself, then d_i / d_0 - 1 for its nfeat
    smallest coarse distances d_0 <= d_1 <= ... (d_0 clamped below at 1e-12)."""
    xq = np.asarray(xq, np.float64)
    d = np.asarray(coarse_dist, np.float64)[:, :nfeat]
    d0 = np.maximum(d[:, :1], 1e-12)
    return np.concatenate([xq, d / d0 - 1.0], axis=1)
