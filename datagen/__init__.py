"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws raw points and queries (and per-query k / recall mixes).
It holds none of the method's arithmetic: normalisation, hashing and search
happen on each side (CUDA library, CPU oracle) separately.  Both sides consume
the same arrays, so a run is reproducible from (workload, seed).

Streams are separated by a purpose word passed to numpy's SeedSequence, so the
points, the queries and each auxiliary draw come from independent streams.
"""
from __future__ import annotations

import numpy as np

_PURPOSE = {"points": 11, "queries": 12, "centres": 13, "kappa": 14, "mix": 15,
            "planted": 16, "train": 17, "params": 18, "tune": 19, "queries2": 20}


def _rng(seed: int, purpose: str, stream: int = 0) -> np.random.Generator:
    """Stream 0 is the default stream of (seed, purpose); other streams give
    independent draws of the same distribution (e.g. one query batch per rank)."""
    words = [int(seed), _PURPOSE[purpose]] + ([int(stream)] if stream else [])
    return np.random.Generator(np.random.Philox(np.random.SeedSequence(words)))


def gaussian(n: int, d: int, seed: int = 0, purpose: str = "points") -> np.ndarray:
    """i.i.d. N(0,1) coordinates, float32 [n][d] (not normalised)."""
    return _rng(seed, purpose).standard_normal((n, d), dtype=np.float32)


def uniform_sphere(n: int, d: int, seed: int = 0, purpose: str = "points") -> np.ndarray:
    g = _rng(seed, purpose).standard_normal((n, d))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return g.astype(np.float32)


def _vmf_w(rng: np.random.Generator, kappa: np.ndarray, d: int) -> np.ndarray:
    """Wood (1994) rejection sampler for the cosine W = <x, mu> of a
    von Mises-Fisher draw on S^(d-1) with concentration kappa (vector)."""
    kappa = np.asarray(kappa, np.float64)
    m = d - 1
    b = (-2.0 * kappa + np.sqrt(4.0 * kappa ** 2 + m ** 2)) / m
    x0 = (1.0 - b) / (1.0 + b)
    c = kappa * x0 + m * np.log(1.0 - x0 ** 2)
    out = np.empty(kappa.shape[0])
    todo = np.arange(kappa.shape[0])
    while todo.size:
        z = rng.beta(m / 2.0, m / 2.0, size=todo.size)
        w = (1.0 - (1.0 + b[todo]) * z) / (1.0 - (1.0 - b[todo]) * z)
        u = rng.random(todo.size)
        ok = kappa[todo] * w + m * np.log(1.0 - x0[todo] * w) - c[todo] >= np.log(u)
        out[todo[ok]] = w[ok]
        todo = todo[~ok]
    return out


def vmf_mixture(n: int, d: int, components: int, kappa, seed: int = 0, purpose: str = "points",
                chunk: int = 1 << 18, stream: int = 0) -> np.ndarray:
    """Unit vectors from an equal-weight mixture of von Mises-Fisher
    distributions; centres are normalised N(0, I) draws (shared by all
    purposes and streams of one seed).  kappa: a scalar, or a (lo, hi) pair for
    a per-component concentration drawn uniformly from [lo, hi]."""
    crng = _rng(seed, "centres")
    centres = crng.standard_normal((components, d))
    centres /= np.linalg.norm(centres, axis=1, keepdims=True)
    if np.ndim(kappa) == 0:
        kap = np.full(components, float(kappa))
    else:
        lo, hi = kappa
        kap = _rng(seed, "kappa").uniform(lo, hi, size=components)
    rng = _rng(seed, purpose, stream)
    out = np.empty((n, d), np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        comp = rng.integers(0, components, size=e - s)
        mu = centres[comp]
        w = _vmf_w(rng, kap[comp], d)
        v = rng.standard_normal((e - s, d))
        v -= np.sum(v * mu, axis=1, keepdims=True) * mu
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        x = w[:, None] * mu + np.sqrt(np.maximum(0.0, 1.0 - w ** 2))[:, None] * v
        out[s:e] = x.astype(np.float32)
    return out


def planted(n_background: int, d: int, n_queries: int, c_nn: float = 0.8, n_decoys: int = 2000,
            decoy_range=(0.55, 0.65), seed: int = 0):
    """Hard planted instance: uniform background on the sphere, and for every
    query one planted neighbour at cosine c_nn and n_decoys decoys at cosines
    drawn uniformly from decoy_range.  Planted point = c q + sqrt(1-c^2) u with
    u uniform on the sphere orthogonal to q.  Returns (points, queries,
    neighbour_index[n_queries])."""
    q = uniform_sphere(n_queries, d, seed, "queries").astype(np.float64)
    bg = uniform_sphere(n_background, d, seed, "points")
    rng = _rng(seed, "planted")
    per = 1 + n_decoys
    pts = np.empty((n_background + n_queries * per, d), np.float32)
    pts[:n_background] = bg
    nn = np.empty(n_queries, np.int64)
    for i in range(n_queries):
        c = np.concatenate([[c_nn], rng.uniform(decoy_range[0], decoy_range[1], size=n_decoys)])
        u = rng.standard_normal((per, d))
        u -= (u @ q[i])[:, None] * q[i][None, :]
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        x = c[:, None] * q[i][None, :] + np.sqrt(1.0 - c ** 2)[:, None] * u
        base = n_background + i * per
        pts[base:base + per] = x.astype(np.float32)
        nn[i] = base
    return pts, q.astype(np.float32), nn


def _synthetic_vw(d: int, seed: int):
    s = np.sqrt(1.0 / (2 * d))
    rng = _rng(seed, "centres")
    return rng.normal(0, s, d), rng.normal(0, s, d)


def paper_synthetic_points(n: int, d: int, seed: int = 0, chunk: int = 1 << 18) -> np.ndarray:
    """Points of the SYNTHETIC construction of Sec. 5 (dimension 3d): n - 1
    points (0, y_i, z_i) whose coordinates are N(0, 1/(2d)) draws, and as the
    last point (v, w, 0) with v, w of the same law (expected squared length 1/2
    each): the nearest neighbour, in expectation, of every query."""
    rng = _rng(seed, "points")
    s = np.sqrt(1.0 / (2 * d))
    pts = np.zeros((n, 3 * d), np.float32)
    for a in range(0, n - 1, chunk):
        e = min(n - 1, a + chunk)
        pts[a:e, d:] = rng.normal(0, s, (e - a, 2 * d))
    v, w = _synthetic_vw(d, seed)
    pts[n - 1, :d] = v
    pts[n - 1, d:2 * d] = w
    return pts


def paper_synthetic_queries(m: int, d: int, seed: int = 0, purpose: str = "queries", stream: int = 0) -> np.ndarray:
    """Queries of the SYNTHETIC construction of Sec. 5: (v, 0, r_i) with the v of
    the last point and r_i uniform of length sqrt(1/2)."""
    v, _ = _synthetic_vw(d, seed)
    r = _rng(seed, purpose, stream).standard_normal((m, d))
    r *= np.sqrt(0.5) / np.linalg.norm(r, axis=1, keepdims=True)
    qs = np.zeros((m, 3 * d), np.float32)
    qs[:, :d] = v
    qs[:, 2 * d:] = r
    return qs


def mixed_k_recall(Q: int, ks=(1, 10, 100), deltas=(0.5, 0.1, 0.01), seed: int = 0):
    """Per-query k and recall target drawn uniformly and independently."""
    rng = _rng(seed, "mix")
    k = rng.choice(np.asarray(ks, np.int32), size=Q)
    delta = rng.choice(np.asarray(deltas, np.float64), size=Q)
    return k.astype(np.int32), (1.0 - delta)


# ---------------------------------------------------------------- workloads
WORKLOADS = {
    "gauss-n10k-d64": dict(n=10_000, d=64, Q=100, family="simhash", budget=32 << 20, k=10, recall=0.9),
    "vmf1k-n1m-d100": dict(n=1_000_000, d=100, Q=10_000, family="crosspolytope", budget=4 << 30, k=10,
                           recall=0.9, components=1000, kappa=50.0),
    "planted-n3m-d256": dict(n=3_001_000, d=256, Q=1000, family="crosspolytope", budget=8 << 30, k=1,
                             recall=0.95),
    "vmf4k-n2m-d128-mixed": dict(n=2_000_000, d=128, Q=100_000, family="crosspolytope", budget=8 << 30,
                                 components=4000, kappa=(20.0, 200.0), recall=None, k=100),
    "vmf10k-n10m-d96-f16": dict(n=10_000_000, d=96, Q=100_000, family="crosspolytope", budget=40 << 30, k=10,
                                recall=0.9, components=10_000, kappa=100.0, rows="f16"),
    # Sec. 5 SYNTHETIC: n = 10^6, 3 x 100 dimensions, 1,000 queries
    "paper-synthetic-n1m-d300": dict(n=1_000_000, d=300, Q=1000, family="crosspolytope", budget=8 << 30, k=10,
                                     recall=0.99, block=100),
}


def make(name: str, seed: int = 0, n: int | None = None, Q: int | None = None):
    """Points and queries of a named workload (optionally truncated)."""
    w = WORKLOADS[name]
    n = w["n"] if n is None else n
    Q = w["Q"] if Q is None else Q
    if name == "gauss-n10k-d64":
        return gaussian(n, w["d"], seed, "points"), gaussian(Q, w["d"], seed, "queries")
    if name.startswith("vmf"):
        return (vmf_mixture(n, w["d"], w["components"], w["kappa"], seed, "points"),
                vmf_mixture(Q, w["d"], w["components"], w["kappa"], seed, "queries"))
    if name == "paper-synthetic-n1m-d300":
        return (paper_synthetic_points(n, w["block"], seed),
                paper_synthetic_queries(Q, w["block"], seed))
    if name == "planted-n3m-d256":
        nb = max(0, n - Q * 2001)
        pts, qs, _ = planted(nb, w["d"], Q, seed=seed)
        return pts, qs
    raise KeyError(name)
