"""Pins of the float64 perceptron oracle: its analytic gradients against
central finite differences, and its loss against the closed form of a uniform
prediction (log C when all logits are equal)."""
import math

import numpy as np

from oracle import mlp


def _net(rng, B=7, F=9, H=6, C=5):
    X = rng.standard_normal((B, F))
    y = rng.integers(0, C, B)
    W1 = rng.standard_normal((H, F)) * 0.5
    b1 = rng.standard_normal(H) * 0.1
    W2 = rng.standard_normal((C, H)) * 0.5
    b2 = rng.standard_normal(C) * 0.1
    return X, y, W1, b1, W2, b2


def test_uniform_logits_loss_is_log_c():
    rng = np.random.default_rng(0)
    X, y, W1, b1, W2, b2 = _net(rng)
    loss, *_ = mlp.loss_and_grads(X, y, W1, b1, np.zeros_like(W2), np.zeros_like(b2))
    assert abs(loss - math.log(5)) < 1e-12


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    X, y, W1, b1, W2, b2 = _net(rng)
    params = [W1, b1, W2, b2]
    _, *grads = mlp.loss_and_grads(X, y, *params)
    eps = 1e-6
    for pi, (P, G) in enumerate(zip(params, grads)):
        flat = P.reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 11)):
            old = flat[idx]
            flat[idx] = old + eps
            lp = mlp.forward(X, y, *params)[0]
            flat[idx] = old - eps
            lm = mlp.forward(X, y, *params)[0]
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - G.reshape(-1)[idx]) <= 1e-7 + 1e-6 * abs(fd), (pi, idx, fd, G.reshape(-1)[idx])
