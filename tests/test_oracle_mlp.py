"""Pins of the FP64 surrogate-network oracle (no GPU): gradients vs central
finite differences of the loss; GELU and its derivative vs the erf form
(they agree to ~1e-3, the tanh approximation's known accuracy) and vs finite
differences; one Adam step vs its closed form on a quadratic."""
import math

import numpy as np

from oracle import mlp


def _net(rng, sizes):
    return [(rng.standard_normal((a, b)) / np.sqrt(a), rng.standard_normal(b) * 0.1)
            for a, b in zip(sizes[:-1], sizes[1:])]


def test_gradients_vs_finite_differences():
    rng = np.random.default_rng(0)
    sizes = [7, 9, 9, 5]
    params = _net(rng, sizes)
    x = rng.standard_normal((11, 7))
    t = rng.standard_normal((11, 5))
    mask = (rng.random((11, 5)) > 0.3).astype(float)
    loss, grads = mlp.loss_and_grads(params, x, t, mask)
    flat = mlp.flatten(params)
    gflat = np.concatenate([np.concatenate([gW.ravel(), gb.ravel()]) for gW, gb in grads])
    h = 1e-6
    for i in rng.choice(flat.size, 60, replace=False):
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        lp, _ = mlp.loss_and_grads(mlp.unflatten(fp, sizes), x, t, mask)
        lm, _ = mlp.loss_and_grads(mlp.unflatten(fm, sizes), x, t, mask)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, gflat[i])


def test_gelu_forms():
    z = np.linspace(-6, 6, 1001)
    exact = np.array([0.5 * v * (1 + math.erf(v / math.sqrt(2))) for v in z])
    assert np.max(np.abs(mlp.gelu(z) - exact)) < 1e-3
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, rtol=1e-6, atol=1e-8)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0


def test_adam_first_step_closed_form():
    # first Adam step moves every parameter by lr * sign(g) (bias-corrected m/sqrt(v) = g/|g|)
    W = np.array([[1.0, -2.0]]); b = np.array([0.5, 0.0])
    g = [(np.array([[3.0, -0.1]]), np.array([-4.0, 2.0]))]
    st = {"t": 0}
    (W2, b2), = mlp.adam_step([(W, b)], g, st, lr=0.01, eps=0.0)
    np.testing.assert_allclose(W2, W - 0.01 * np.sign(g[0][0]), rtol=1e-12)
    np.testing.assert_allclose(b2, b - 0.01 * np.sign(g[0][1]), rtol=1e-12)
