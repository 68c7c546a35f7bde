"""FP64 oracle of the learned score surrogate: an MLP s_theta (SiLU hidden
layers) trained by denoising score matching, with Adam.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The surrogate is not in
the paper; its definitions follow the standard ones:
  forward   z_l = h_{l-1} W_l^T + b_l,  h_l = silu(z_l) = z_l / (1 + exp(-z_l))
            (no activation on the last layer), h_0 = input;
  DSM loss  L = (1/B) sum_b || s_theta(x_b + sigma eps_b) + eps_b / sigma ||^2,
            whose minimiser is the score of the data density smoothed by
            N(0, sigma^2 I);
  Adam      m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
            p -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def as64(layers):
    return [(np.asarray(W, dtype=np.float64), np.asarray(b, dtype=np.float64)) for W, b in layers]


def forward(layers, x):
    """Returns (output, cache) with cache = [(h_in, z)] per layer."""
    h = np.asarray(x, dtype=np.float64)
    cache = []
    L = len(layers)
    for l, (W, b) in enumerate(layers):
        z = h @ W.T + b
        cache.append((h, z))
        h = silu(z) if l < L - 1 else z
    return h, cache


def dsm_loss(layers, x, eps, sigma):
    xt = np.asarray(x, dtype=np.float64) + sigma * np.asarray(eps, dtype=np.float64)
    s, _ = forward(layers, xt)
    r = s + np.asarray(eps, dtype=np.float64) / sigma
    return np.mean(np.sum(r * r, axis=1))


def dsm_loss_of_score(score, x, eps, sigma):
    """DSM loss of an arbitrary score function (used to pin the loss)."""
    xt = np.asarray(x, dtype=np.float64) + sigma * np.asarray(eps, dtype=np.float64)
    r = score(xt) + np.asarray(eps, dtype=np.float64) / sigma
    return np.mean(np.sum(r * r, axis=1))


def dsm_grad(layers, x, eps, sigma):
    """(loss, [(dW, db)]) by backpropagation."""
    eps = np.asarray(eps, dtype=np.float64)
    xt = np.asarray(x, dtype=np.float64) + sigma * eps
    s, cache = forward(layers, xt)
    B = xt.shape[0]
    r = s + eps / sigma
    loss = np.mean(np.sum(r * r, axis=1))
    d = 2.0 * r / B                      # dL/ds
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        h_in, z = cache[l]
        if l < len(layers) - 1:
            d = d * silu_grad(z)         # through the activation of this layer
        grads[l] = (d.T @ h_in, d.sum(axis=0))
        d = d @ layers[l][0]             # to the previous layer's output
    return loss, grads


def adam_init(layers):
    return [(np.zeros_like(W), np.zeros_like(b)) for W, b in layers], \
           [(np.zeros_like(W), np.zeros_like(b)) for W, b in layers]


def adam_step(layers, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new (layers, m, v)."""
    out, mo, vo = [], [], []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(layers, grads, m, v):
        res = []
        for p, g, mm, vv in ((W, gW, mW, vW), (b, gb, mb, vb)):
            mm = b1 * mm + (1 - b1) * g
            vv = b2 * vv + (1 - b2) * g * g
            mh = mm / (1 - b1 ** t)
            vh = vv / (1 - b2 ** t)
            res.append((p - lr * mh / (np.sqrt(vh) + eps), mm, vv))
        out.append((res[0][0], res[1][0]))
        mo.append((res[0][1], res[1][1]))
        vo.append((res[0][2], res[1][2]))
    return out, mo, vo


def fit_grad(layers, x, target):
    """(loss, grads) of the supervised fit L = (1/B) sum_b |s_theta(x_b) - t_b|^2."""
    x = np.asarray(x, dtype=np.float64)
    s, cache = forward(layers, x)
    B = x.shape[0]
    r = s - np.asarray(target, dtype=np.float64)
    loss = np.mean(np.sum(r * r, axis=1))
    d = 2.0 * r / B
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        h_in, z = cache[l]
        if l < len(layers) - 1:
            d = d * silu_grad(z)
        grads[l] = (d.T @ h_in, d.sum(axis=0))
        d = d @ layers[l][0]
    return loss, grads
