"""Pins of the oracle's pooled hash functions (Sec. 3.2 "Pooling", App. B.2):
the random subsets, the codes against a numpy restatement, the stop rule
(Cantelli's inequality, the reading for general delta) against its limits, the
paper's delta = 1/2 rule and a simulation of the pooled collisions, and the
recall guarantee of a small pooled index."""
import math

import numpy as np
import pytest

import datagen


def test_subsets_are_distinct_uniform_and_deterministic(orc):
    m, F, L = 64, 4, 6000
    sel = orc.pool_select(11, L, F, m)
    assert np.array_equal(sel, orc.pool_select(11, L, F, m))
    assert not np.array_equal(sel, orc.pool_select(12, L, F, m))
    assert sel.min() >= 0 and sel.max() < m
    assert all(len(set(r)) == F for r in sel.tolist())
    # every function is chosen with probability F/m; every pair with F(F-1)/(m(m-1))
    counts = np.bincount(sel.ravel(), minlength=m)
    exp = L * F / m
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < m + 6 * math.sqrt(2 * m), chi2
    pair = np.mean([(0 in r) and (1 in r) for r in sel.tolist()])
    assert abs(pair - F * (F - 1) / (m * (m - 1))) < 4 * math.sqrt(F * (F - 1) / (m * (m - 1)) / L)
    # the order inside a subset is random too: position 0 holds each function equally often
    first = np.bincount(sel[:, 0], minlength=m)
    assert float(((first - L / m) ** 2 / (L / m)).sum()) < m + 6 * math.sqrt(2 * m)


@pytest.mark.parametrize("family,d", [(0, 24), (1, 12)])
def test_codes_match_a_numpy_restatement(orc, family, d):
    lay = orc.layout(family, d)
    ell, F = lay["ell"], lay["F"]
    m, L = 3072 // ell, 7
    x = orc.normalize(datagen.gaussian(150, d, seed=3))
    A = orc.gen_pool_params(5, family, m, d)
    sel = orc.pool_select(5, L, F, m)
    codes = orc.pool_codes(family, A, sel, x)
    v = np.einsum("fri,pi->pfr", A.astype(np.float64), x.astype(np.float64))  # [n][m][R]
    if family == 0:
        val = (v[:, :, 0] >= 0).astype(np.uint32)
        safe = np.all(np.abs(v[:, :, 0]) > 1e-9, axis=1)
    else:
        c = np.argmax(np.abs(v), axis=2)
        top = np.take_along_axis(v, c[..., None], axis=2)[..., 0]
        val = ((top < 0).astype(np.uint32) << np.uint32(ell - 1)) | c.astype(np.uint32)
        srt = np.sort(np.abs(v), axis=2)
        safe = np.all(srt[..., -1] - srt[..., -2] > 1e-9, axis=1)
    want = np.zeros((L, x.shape[0]), np.uint32)
    for s in range(F):
        want |= val[:, sel[:, s]].T << np.uint32(32 - ell * (s + 1))
    assert np.array_equal(codes[:, safe], want[:, safe]) and safe.mean() > 0.9
    # the hyperplanes are the generator's N(0,1) draws at (i, c, f, purpose 6)
    assert A[3, 0, 2] == np.float32(orc.gauss(5, 6, 3, 0, 2))


def _bound(mu, f, m, P):
    c = f * f / ((m - f) * P)
    if not c < 1:
        return 1.0
    var = mu + mu * mu * (c / (1 - c))
    return var / (mu * mu + var)


def test_stop_rule_limits_and_the_papers_half_rule(orc):
    # HP at s_k = 0: every bit collides with probability 1/2, p_i = 2^-i
    m_inf = 10 ** 9
    for i in (3, 6, 9):
        for j in (1, 10, 100, 1000):
            mu = j * 2.0 ** -i
            # m -> infinity: the bound is 1/(1 + mu) (Cantelli for a sum of independent indicators)
            for delta in (0.5, 0.1, 0.01):
                if abs(1 / (1 + mu) - delta) > 1e-6:
                    assert orc.pool_stop(0, 1, None, m_inf, 0.0, i, j, delta) == (1 / (1 + mu) <= delta)
    # the paper's rule for delta = 1/2 (mu >= 2 and m >= 5 i^2 / P) stops whenever it holds with
    # a little room; and a small pool never stops
    for i in (2, 4, 8):
        for m in (int(6 * i * i / 0.5) + i, 2000, 20000):
            j = int(math.ceil(2.2 * 2 ** i))
            assert orc.pool_stop(0, 1, None, m, 0.0, i, j, 0.5)
        assert not orc.pool_stop(0, 1, None, i + 1, 0.0, i, 10 ** 6, 0.5)
    # cross-polytope: f counts the functions behind the first i bits (l = 8 here)
    P = orc.cp_table(0, 100)
    s = 0.9
    for i, f in ((8, 1), (9, 2), (16, 2), (17, 3)):
        p_i = orc.collision_prob(1, 8, P, s, i)
        P1 = orc.collision_prob(1, 8, P, s, 8)
        for j in (5, 50, 500):
            b = _bound(j * p_i, f, 384, P1)
            if abs(b - 0.1) > 1e-9:
                assert orc.pool_stop(1, 8, P, 384, s, i, j, 0.1) == (b <= 0.1)


def test_bound_holds_for_simulated_pools():
    """Simulate the scheme: m pooled one-bit functions, each colliding with
    probability P independently; j tables, each the first f of F random
    distinct functions; X = tables in which all f collide.  The empirical
    Pr[X = 0] stays below the bound the stop rule uses."""
    rng = np.random.default_rng(1)
    for m, f, P, j in ((64, 3, 0.7, 20), (200, 4, 0.6, 40), (40, 2, 0.5, 12), (500, 6, 0.8, 30)):
        trials = 4000
        zero = 0
        for _ in range(trials):
            hit = rng.random(m) < P
            sel = np.argsort(rng.random((j, m)), axis=1)[:, :f]
            zero += not np.any(np.all(hit[sel], axis=1))
        emp = zero / trials
        b = _bound(j * P ** f, f, m, P)
        assert emp <= b + 3 * math.sqrt(max(b, 1e-3) / trials), (m, f, P, j, emp, b)


def test_pooled_index_meets_the_recall_target_with_the_filter_off(orc):
    X = datagen.vmf_mixture(5000, 24, 30, 20.0, seed=4)
    Qs = datagen.vmf_mixture(150, 24, 30, 20.0, seed=4, purpose="queries")
    ix = orc.OracleIndex(X, 1, L=40, seed=5, pool_bits=3072)
    assert ix.pool_fns == 3072 // ix.ell
    _, bs = orc.brute_force(ix.x, orc.normalize(Qs), 10)
    for recall in (0.5, 0.9):
        res = ix.search(Qs, 10, recall, filter=False)
        got = float(np.mean(res["sims"] >= bs[:, -1:]))
        N = Qs.shape[0] * 10
        assert got >= recall - 3 * math.sqrt(recall * (1 - recall) / N), (recall, got)
    # Lemma 1's rule on the pooled index stops at least as early (no guarantee)
    cant = ix.search(Qs, 10, 0.9, filter=False)["stats"]["stop_depth"]
    ind = ix.search(Qs, 10, 0.9, filter=False, pool_rule="independent")["stats"]["stop_depth"]
    assert np.all(ind >= cant)


def test_pooled_budget(orc):
    n, d, M = 1_000_000, 100, 32
    dp, F, m = 112, 4, 384
    fixed = n * dp * 6 + 64 * M * dp * 6 + (m // F) * F * dp * dp * 6
    per = n * 16 + 8193 * 4 + F * 4
    assert orc.budget_L(1, n, d, M, 4 << 30, 0, 0, 0, m) == ((4 << 30) - fixed) // per
