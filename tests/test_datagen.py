"""The synthetic inputs follow their stated constructions (they hold none of
the method's arithmetic; these checks pin the generators themselves)."""
import numpy as np

import datagen


def test_paper_synthetic_construction():
    d, n, m = 100, 4000, 60
    X = datagen.paper_synthetic_points(n, d, seed=3)
    Q = datagen.paper_synthetic_queries(m, d, seed=3)
    assert X.shape == (n, 3 * d) and Q.shape == (m, 3 * d)
    # x_i = (0, y_i, z_i) for i < n; x_n = (v, w, 0); q = (v, 0, r) with |r| = sqrt(1/2)
    assert not X[: n - 1, :d].any() and not X[n - 1, 2 * d:].any()
    assert not Q[:, d:2 * d].any()
    assert np.all(Q[:, :d] == X[n - 1, :d])
    assert np.allclose(np.linalg.norm(Q[:, 2 * d:], axis=1), np.sqrt(0.5), rtol=1e-6)
    # coordinates N(0, 1/(2d)): squared lengths of y and z average 1/2
    for blk in (X[: n - 1, d:2 * d], X[: n - 1, 2 * d:]):
        assert abs(float(np.mean(np.sum(blk.astype(np.float64) ** 2, axis=1))) - 0.5) < 0.01
        assert abs(float(np.std(blk)) - np.sqrt(1 / (2 * d))) < 0.002
    # the last point is every query's nearest neighbour (cosine), well ahead of the rest
    Xn = X / np.linalg.norm(X, axis=1, keepdims=True)
    Qn = Q / np.linalg.norm(Q, axis=1, keepdims=True)
    S = Qn @ Xn.T
    assert np.all(S.argmax(axis=1) == n - 1)
    assert float(np.min(S[:, -1] - np.sort(S, axis=1)[:, -2])) > 0.1
    # other query streams: new r, the same v
    Q2 = datagen.paper_synthetic_queries(m, d, seed=3, stream=1)
    assert np.all(Q2[:, :d] == Q[:, :d]) and not np.array_equal(Q2, Q)


def test_query_streams_share_the_mixture():
    a = datagen.vmf_mixture(500, 16, 5, 200.0, seed=0, purpose="queries")
    b = datagen.vmf_mixture(500, 16, 5, 200.0, seed=0, purpose="queries", stream=1)
    pts = datagen.vmf_mixture(2000, 16, 5, 200.0, seed=0, purpose="points")
    assert not np.array_equal(a, b)
    # the same five centres: every query of either stream is close to some point
    for q in (a, b):
        assert float(np.min(np.max(q @ pts.T, axis=1))) > 0.8
    # stream 0 is the default stream
    assert np.array_equal(a, datagen.vmf_mixture(500, 16, 5, 200.0, seed=0, purpose="queries", stream=0))
