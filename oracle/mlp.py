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


def start_depths(X, W1, b1, W2, b2, tail, margin):
    """The start depth the perceptron predicts for each row of features X:
    with p = softmax(z) over the stop depths 0..C-1 and A[d] = sum_{c > d} p_c
    (the predicted chance that the query stops deeper than d), q is the smallest
    d with A[d] <= tail, and the start is min(C - 1, q + margin).  Returns the
    starts and A (float64 throughout)."""
    _, _, _, z = forward(X, np.zeros(np.asarray(X).shape[0], np.int64), W1, b1, W2, b2)
    p = np.exp(z - z.max(axis=1, keepdims=True))
    p /= p.sum(axis=1, keepdims=True)
    C = p.shape[1]
    A = np.zeros_like(p)
    for d in range(C - 2, -1, -1):
        A[:, d] = A[:, d + 1] + p[:, d + 1]
    q = np.array([int(np.nonzero(A[i] <= tail)[0].min()) for i in range(p.shape[0])])
    return np.minimum(C - 1, q + margin), A
