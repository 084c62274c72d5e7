"""FP64 oracle of the population surrogate network (forward, backward, Adam).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The network (not in the paper; it warm-starts the rate solves): input x,
hidden layers h_k = GELU(h_{k-1} W_k + b_k) for k = 1..n_hidden, output
y = h_n W_out + b_out.  GELU in its tanh form (Hendrycks & Gimpel 2016):
GELU(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))).  Loss: masked mean
squared error sum(mask (y - t)^2) / sum(mask).  Adam (Kingma & Ba 2015) with
bias correction.  Weights W_k are [fan_in, fan_out] row-major.
"""
from __future__ import annotations

import numpy as np

SQRT_2_OVER_PI = np.sqrt(2.0 / np.pi)


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(SQRT_2_OVER_PI * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    u = SQRT_2_OVER_PI * (z + 0.044715 * z ** 3)
    th = np.tanh(u)
    du = SQRT_2_OVER_PI * (1.0 + 3 * 0.044715 * z ** 2)
    return 0.5 * (1.0 + th) + 0.5 * z * (1.0 - th * th) * du


def forward(params, x):
    """params: list of (W, b); the last pair is the linear output layer.
    Returns y and the per-layer (input, pre-activation) cache."""
    h = x
    cache = []
    for k, (W, b) in enumerate(params):
        z = h @ W + b
        cache.append((h, z))
        h = z if k == len(params) - 1 else gelu(z)
    return h, cache


def loss_and_grads(params, x, t, mask):
    y, cache = forward(params, x)
    msum = mask.sum()
    r = mask * (y - t)
    loss = float((r * (y - t)).sum() / msum)
    dy = 2.0 * r / msum
    grads = [None] * len(params)
    g = dy
    for k in range(len(params) - 1, -1, -1):
        h_in, z = cache[k]
        if k < len(params) - 1:
            g = g * gelu_grad(z)
        W, _ = params[k]
        grads[k] = (h_in.T @ g, g.sum(axis=0))
        g = g @ W.T
    return loss, grads


def adam_step(params, grads, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    state["t"] += 1
    t = state["t"]
    out = []
    for k, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        new = []
        for j, (p, gp) in enumerate(((W, gW), (b, gb))):
            key = (k, j)
            m = state.setdefault(("m",) + key, np.zeros_like(p))
            v = state.setdefault(("v",) + key, np.zeros_like(p))
            m[...] = b1 * m + (1 - b1) * gp
            v[...] = b2 * v + (1 - b2) * gp * gp
            mh = m / (1 - b1 ** t)
            vh = v / (1 - b2 ** t)
            new.append(p - lr * mh / (np.sqrt(vh) + eps))
        out.append((new[0], new[1]))
    return out


def flatten(params):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def unflatten(flat, sizes):
    """sizes: [n_in, h, ..., n_out]; returns [(W, b), ...]."""
    out, o = [], 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = flat[o:o + a * b].reshape(a, b); o += a * b
        bb = flat[o:o + b]; o += b
        out.append((W, bb))
    return out
