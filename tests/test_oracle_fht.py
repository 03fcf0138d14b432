"""Pins of the oracle's pseudo-random cross-polytope family (oracle/fht.py):
the butterfly against the Walsh-Hadamard matrix, the three-round rotation
against explicit matrices, the hash values and code layout against a scalar
restatement, the collision table's invariants and its closeness to the exact
family's, and the query guarantee on a small index."""
import numpy as np
import pytest

import datagen
import oracle
from oracle import fht

scipy_linalg = pytest.importorskip("scipy.linalg")


def test_dimension_and_layout():
    assert [fht.dim(d) for d in (1, 2, 3, 64, 65, 100, 128, 300)] == [1, 2, 4, 64, 128, 128, 128, 512]
    assert fht.layout(100) == {"dp": 128, "ell": 8, "F": 4, "Kb": 32}
    assert fht.layout(300) == {"dp": 512, "ell": 10, "F": 3, "Kb": 30}
    assert fht.layout(20) == {"dp": 32, "ell": 6, "F": 5, "Kb": 30}


@pytest.mark.parametrize("dp", [1, 2, 8, 64, 128])
def test_butterfly_is_the_walsh_hadamard_matrix(dp):
    rng = np.random.default_rng(dp)
    H = scipy_linalg.hadamard(dp).astype(np.float64)
    v = rng.integers(-1000, 1000, size=(5, dp)).astype(np.float64)  # integers: every sum is exact
    assert np.array_equal(fht.fwht(v), v @ H.T)
    w = rng.standard_normal((3, dp))
    assert np.allclose(fht.fwht(w), w @ H.T, rtol=1e-12, atol=1e-12)


def test_rotation_equals_explicit_matrices_and_scales_norms():
    rng = np.random.default_rng(1)
    dp = 64
    H = scipy_linalg.hadamard(dp).astype(np.float64)
    D = rng.choice([-1.0, 1.0], size=(3, dp))
    x = rng.integers(-50, 50, size=(4, 50)).astype(np.float64)  # d = 50 < d' = 64: zero padding
    xp = np.zeros((4, dp))
    xp[:, :50] = x
    Mx = H @ np.diag(D[2]) @ H @ np.diag(D[1]) @ H @ np.diag(D[0])
    y = fht.rotate(x, D)
    assert np.array_equal(y, xp @ Mx.T)
    assert np.array_equal(np.sum(y * y, axis=1), dp ** 3 * np.sum(x * x, axis=1))


def test_signs_are_deterministic_balanced_and_distinct():
    a = fht.signs(7, fht.PURPOSE_FHT, 3, 5, 512)
    assert np.array_equal(a, fht.signs(7, fht.PURPOSE_FHT, 3, 5, 512))
    assert set(np.unique(a)) <= {-1.0, 1.0}
    assert not np.array_equal(a, fht.signs(7, fht.PURPOSE_FHT, 3, 6, 512))
    assert not np.array_equal(a, fht.signs(8, fht.PURPOSE_FHT, 3, 5, 512))
    many = np.concatenate([fht.signs(0, fht.PURPOSE_FHT, j, 0, 512) for j in range(40)])
    assert abs(float(many.mean())) < 4.0 / np.sqrt(many.size)


def test_values_and_code_layout_match_a_scalar_restatement():
    d = 100
    lay = fht.layout(d)
    D = fht.gen_params(3, 2, d)
    x = oracle.normalize(datagen.gaussian(20, d, seed=9))
    codes = fht.hash_codes(D, x, d)
    for j in range(2):
        for p in range(20):
            code = 0
            for f in range(lay["F"]):
                y = fht.rotate(x[p].astype(np.float64), D[j, f])
                best, best_abs = 0, -1.0
                for c in range(lay["dp"]):
                    if abs(y[c]) > best_abs:
                        best, best_abs = c, abs(y[c])
                value = ((1 if y[best] < 0 else 0) << (lay["ell"] - 1)) | best
                code |= value << (32 - lay["ell"] * (f + 1))
            assert codes[j, p] == code
    # ties go to the smaller coordinate; the sign is that of the chosen coordinate
    y = np.zeros((1, 8))
    y[0, 3], y[0, 6] = -2.0, 2.0
    assert fht.values(y, 4)[0] == (1 << 3) | 3


def test_collision_table_invariants_and_closeness_to_the_exact_family():
    d = 128
    P = fht.cp_table(0, d, draws=1000)
    ell = fht.layout(d)["ell"]
    assert P.shape == (oracle.ALPHA_STEPS, ell + 1)
    assert np.all(P[:, 0] == 1.0)
    assert np.all(P[-1] == 1.0)        # alpha = 1: the same vector
    assert np.all(P[0, 1:] == 0.0)     # alpha = -1: opposite signs
    assert np.all(np.diff(P, axis=0) >= 0.0)
    assert np.all(np.diff(P, axis=1) <= 0.0)
    E = oracle.cp_table(0, d, draws=1000)  # exact family, d = 128: the same l = 8
    assert E.shape == P.shape
    diff = np.abs(P - E)
    assert float(diff.mean()) < 0.02 and float(diff.max()) < 0.1, (diff.mean(), diff.max())


def test_small_index_meets_the_recall_target_with_the_filter_off():
    X = datagen.vmf_mixture(3000, 100, 30, 40.0, seed=4)
    Q = datagen.vmf_mixture(60, 100, 30, 40.0, seed=4, purpose="queries")
    ix = oracle.OracleIndex(X, oracle.CROSSPOLYTOPE_FHT, L=30, seed=2)
    assert (ix.ell, ix.F, ix.Kb) == (8, 4, 32)
    out = ix.search(Q, 10, 0.9, filter=False)
    bf_ids, bf_sims = oracle.brute_force(ix.x, oracle.normalize(Q), 10)
    kth = bf_sims[:, 9:10]
    hit = float(np.mean(out["sims"] >= kth))
    assert hit >= 0.9 - 3 * np.sqrt(0.9 * 0.1 / out["sims"].size), hit
    # returned similarities are canonical similarities of the returned points
    qn = oracle.normalize(Q)
    for t in range(0, 60, 7):
        for u in range(10):
            assert out["sims"][t, u] == oracle.sim(qn[t], ix.x[out["ids"][t, u]])
    # a budget gives the L of the budget rule (three sign vectors per function)
    small = oracle.OracleIndex(X, oracle.CROSSPOLYTOPE_FHT, budget_bytes=4 << 20)
    assert small.L == oracle.budget_L(oracle.CROSSPOLYTOPE_FHT, 3000, 100, 32, 4 << 20) >= 1
