"""Pins of the oracle's stop test after groups of repetitions (Algorithm 1 tests
after every repetition; `stop_every` = G tests after every G repetitions and
after the last one of a round).

After j repetitions of the round at prefix length i, repetitions 0..j-1 have
been searched to length i and the others to length i + 1 (to nothing yet in
the first round), so the chance that a point at similarity s_k was missed is
(1 - p_i)^j (1 - p_{i+1})^(L - j), which is the stop test (Lemma 1).  A replay
of the oracle's trace in numpy rebuilds the top-k at every test point and checks
that the oracle stops at the first test point where the top-k is full and this
bound is <= delta, and not before."""
import math

import numpy as np
import pytest

import datagen


def _setup(orc, family):
    X = datagen.vmf_mixture(5000, 32, 25, 25.0, seed=31)
    Q = datagen.vmf_mixture(40, 32, 25, 25.0, seed=31, purpose="queries")
    ix = orc.OracleIndex(X, family, L=24, M=32, seed=3)
    qn = orc.normalize(Q)
    sims = np.array([[orc.sim(qn[t], ix.x[p]) for p in range(ix.n)] for t in range(qn.shape[0])], np.float32)
    return ix, Q, sims


@pytest.fixture(scope="module")
def cases(orc):
    return {fam: _setup(orc, fam) for fam in (orc.SIMHASH, orc.CROSSPOLYTOPE)}


def _fail(orc, ix, s_k, depth, j, first_round):
    f = (1.0 - orc.collision_prob(ix.family, ix.ell, ix.P, s_k, depth)) ** j
    if not first_round:
        f *= (1.0 - orc.collision_prob(ix.family, ix.ell, ix.P, s_k, depth + 1)) ** (ix.L - j)
    return f


def _first_stop(orc, ix, res, t, k, delta, G, sims_t):
    """(depth, j) of the first test point where the replayed top-k is full and
    the bound is <= delta; None if the schedule reaches depth 0."""
    tr = res["trace"][t, : res["trace_len"][t]]
    key = tr[:, 0].astype(np.int64)
    flag = (key >> 31) & 1
    depth = (key >> 24) & 0x3F
    j = key & 0xFFFFFF
    ids = tr[:, 1].astype(np.int64)
    start = int(res["stats"]["start_depth"][t])
    top = {}
    e = 0
    for d in range(start, 0, -1):
        ends = sorted({min(ix.L, g + G) for g in range(0, ix.L, G)})
        for jend in ends:
            while e < len(tr) and (depth[e] > d or (depth[e] == d and j[e] < jend)):
                if flag[e]:
                    top[int(ids[e])] = float(sims_t[ids[e]])
                e += 1
            if len(top) >= k:
                s_k = sorted(top.items(), key=lambda v: (-v[1], v[0]))[k - 1][1]
                # the bound uses float32 s_k; compare away from exact ties
                fl = _fail(orc, ix, s_k, d, jend, d == start)
                if fl <= delta:
                    return d, jend, fl
    return None


@pytest.mark.parametrize("G", [1, 5, 8])
@pytest.mark.parametrize("fam", [0, 1])
@pytest.mark.parametrize("filt", [True, False])
def test_stops_at_the_first_group_that_meets_the_bound(orc, cases, fam, G, filt):
    ix, Q, sims = cases[fam]
    k, recall = 10, 0.9
    res = ix.search(Q, k, recall, trace_cap=ix.n * ix.L, stop_every=G, filter=filt)
    plain = ix.search(Q, k, recall, filter=filt)["stats"]
    stopped_mid = 0
    for t in range(Q.shape[0]):
        st = res["stats"][t]
        want = _first_stop(orc, ix, res, t, k, 1 - recall, G, sims[t])
        tr = res["trace"][t, : res["trace_len"][t]]
        if want is None:
            assert st["stop_depth"] == 0
            continue
        d, jend, _ = want
        assert st["stop_depth"] == d
        assert st["last_reps"] == jend  # and not a group earlier or later
        # nothing of the stopping round was visited past the stopping group
        key = tr[:, 0].astype(np.int64)
        last = key[((key >> 24) & 0x3F) == d] & 0xFFFFFF
        assert last.size == 0 or last.max() < jend
        stopped_mid += jend < ix.L
    if not filt:  # same candidates per round: the test after the last group is the per-round test
        assert np.all(res["stats"]["stop_depth"] >= plain["stop_depth"])
    assert stopped_mid > 0


def test_recall_guarantee_with_per_repetition_tests(orc):
    # Lemma 1 with the bound (1 - p_i)^j (1 - p_{i+1})^(L - j) <= delta: each
    # true neighbour is still reported with probability >= 1 - delta (filter off)
    X = datagen.vmf_mixture(6000, 24, 30, 20.0, seed=4)
    Qs = datagen.vmf_mixture(200, 24, 30, 20.0, seed=4, purpose="queries")
    ix = orc.OracleIndex(X, 1, L=12, seed=5)
    qn = orc.normalize(Qs)
    _, bs = orc.brute_force(ix.x, qn, 10)
    for recall in (0.5, 0.8):
        res = ix.search(Qs, 10, recall, filter=False, stop_every=1)
        got = np.mean(res["sims"] >= bs[:, -1:])
        N = Qs.shape[0] * 10
        assert got >= recall - 3 * math.sqrt(recall * (1 - recall) / N), (recall, got)
        per_round = ix.search(Qs, 10, recall, filter=False)
        # testing after every repetition never looks at more candidates
        assert res["stats"]["retrieved"].sum() <= per_round["stats"]["retrieved"].sum()


_MUTANTS = {
    "exponent_L_not_j": ("(double)ps[k - 1], depth), j + 1);", "(double)ps[k - 1], depth), L);"),
    "no_second_factor": ("          if (s.rounds > 0)\n            fail = fail *",
                         "          if (0)\n            fail = fail *"),
    "second_factor_at_depth": ("(double)ps[k - 1], depth + 1),", "(double)ps[k - 1], depth),"),
}


@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_planted_stop_rule_mistakes_are_caught(orc, cases, tmp_path, name):
    import os

    src = open(os.path.join(os.path.dirname(orc.__file__), "puffinn_oracle.c")).read()
    old, new = _MUTANTS[name]
    assert src.count(old) == 1, name
    variant = orc.compile_variant(src.replace(old, new), str(tmp_path / f"lib_{name}.so"))
    caught = False
    for fam in (0, 1):
        ix, Q, sims = cases[fam]
        for G in (1, 5):
            res = ix.search(Q, 10, 0.9, trace_cap=ix.n * ix.L, stop_every=G, filter=False, variant=variant)
            for t in range(Q.shape[0]):
                want = _first_stop(orc, ix, res, t, 10, 0.1, G, sims[t])
                st = res["stats"][t]
                got = (int(st["stop_depth"]), int(st["last_reps"]))
                caught |= (want[:2] if want is not None else (0, ix.L)) != got
    assert caught, name
