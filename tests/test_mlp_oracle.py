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


def test_start_depth_rule_hand_values():
    """A model whose logits put (almost) all mass on stop depth c predicts
    q = c, so the start is min(C - 1, c + margin); mass split 0.9 / 0.1 between
    depths 3 and 7 puts q at 7 for a tail of 0.05 and at 3 for a tail of 0.2."""
    from oracle import mlp

    C, H, F = 12, 4, 3
    X = np.ones((1, F))
    W1 = np.zeros((H, F))
    b1 = np.ones(H)  # h = 1 for every unit
    W2 = np.zeros((C, H))
    for c in (0, 4, 11):
        b2 = np.full(C, -50.0)
        b2[c] = 50.0
        s, A = mlp.start_depths(X, W1, b1, W2, b2, 0.05, 6)
        assert s[0] == min(C - 1, c + 6)
        assert np.all(A[0, c:] < 1e-12) and np.all(A[0, :c] > 1 - 1e-12)
    b2 = np.full(C, -np.inf)
    b2[3], b2[7] = np.log(0.9), np.log(0.1)
    assert mlp.start_depths(X, W1, b1, W2, b2, 0.05, 0)[0][0] == 7
    assert mlp.start_depths(X, W1, b1, W2, b2, 0.2, 0)[0][0] == 3
