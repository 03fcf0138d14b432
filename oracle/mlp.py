"""Float64 CPU statement of the start-depth perceptron's loss and gradients.

TEST INFRASTRUCTURE ONLY (used by the tests to check the library's training
kernels).  Plain definitions:
    h = relu(X W1^T + b1),  z = h W2^T + b2,
    loss = mean_i [ -z[i, y_i] + log sum_c exp(z[i, c]) ]
and their gradients by the chain rule, written out term by term.
"""
from __future__ import annotations

import numpy as np


def forward(X, y, W1, b1, W2, b2):
    X, W1, b1, W2, b2 = (np.asarray(a, np.float64) for a in (X, W1, b1, W2, b2))
    pre = X @ W1.T + b1
    h = np.maximum(pre, 0.0)
    z = h @ W2.T + b2
    zmax = z.max(axis=1, keepdims=True)
    lse = zmax[:, 0] + np.log(np.exp(z - zmax).sum(axis=1))
    loss = float(np.mean(lse - z[np.arange(z.shape[0]), y]))
    return loss, pre, h, z


def loss_and_grads(X, y, W1, b1, W2, b2):
    X = np.asarray(X, np.float64)
    loss, pre, h, z = forward(X, y, W1, b1, W2, b2)
    B = X.shape[0]
    p = np.exp(z - z.max(axis=1, keepdims=True))
    p /= p.sum(axis=1, keepdims=True)
    dz = p.copy()
    dz[np.arange(B), y] -= 1.0
    dz /= B
    dW2 = dz.T @ h
    db2 = dz.sum(axis=0)
    dh = dz @ np.asarray(W2, np.float64)
    dpre = dh * (pre > 0)
    dW1 = dpre.T @ X
    db1 = dpre.sum(axis=0)
    return loss, dW1, db1, dW2, db2
