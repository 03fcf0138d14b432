"""Pins of the oracle's query (Algorithm 1 as implemented in Sec. 4) against
brute force and the invariants the paper states."""
import math

import numpy as np
import pytest

import datagen


def _small_index(orc, family=0, n=3000, d=32, L=30, B=12, seed=0, kind="gauss"):
    if kind == "gauss":
        X = datagen.gaussian(n, d, seed=seed)
        Q = datagen.gaussian(60, d, seed=seed, purpose="queries")
    else:
        X = datagen.vmf_mixture(n, d, 20, 30.0, seed=seed)
        Q = datagen.vmf_mixture(60, d, 20, 30.0, seed=seed, purpose="queries")
    return orc.OracleIndex(X, family, L=L, B=B, seed=seed + 1, cp_draws=1000), Q


@pytest.fixture(scope="module")
def hp_index(orc):
    return _small_index(orc, family=0)


@pytest.fixture(scope="module")
def cp_index(orc):
    return _small_index(orc, family=1, n=2500, d=16, L=24, kind="vmf")


def _check_result_wellformed(orc, ix, qn, res, k):
    for t in range(qn.shape[0]):
        ids, sims = res["ids"][t], res["sims"][t]
        valid = ids != 0xFFFFFFFF
        assert len(set(ids[valid].tolist())) == valid.sum()  # unique
        for u in np.nonzero(valid)[0]:
            assert sims[u] == orc.sim(qn[t], ix.x[ids[u]])
        for u in range(1, valid.sum()):  # (sim desc, id asc)
            assert sims[u - 1] > sims[u] or (sims[u - 1] == sims[u] and ids[u - 1] < ids[u])


@pytest.mark.parametrize("which", ["hp", "cp"])
def test_depth_zero_is_exact(orc, hp_index, cp_index, which):
    # Lemma 1, case i = 0: the query degrades to a linear scan.
    ix, Q = hp_index if which == "hp" else cp_index
    qn = orc.normalize(Q)
    bi, bs = orc.brute_force(ix.x, qn, 10)
    res = ix.search(Q, 10, 0.9, start_depth=0)
    assert np.all(res["stats"]["stop_depth"] == 0)
    assert np.array_equal(res["ids"], bi) and np.array_equal(res["sims"], bs)
    # recall target so close to 1 that no depth > 0 can stop: same result
    res2 = ix.search(Q[:10], 10, 1.0 - 2.0 ** -52)
    assert np.all(res2["stats"]["stop_depth"] == 0)
    assert np.array_equal(res2["ids"], bi[:10]) and np.array_equal(res2["sims"], bs[:10])


def test_fewer_points_than_k(orc):
    X = datagen.gaussian(7, 16, seed=2)
    ix = orc.OracleIndex(X, 0, L=5, seed=3)
    res = ix.search(X[:3], 10, 0.9)
    assert np.all(res["stats"]["stop_depth"] == 0)
    assert np.all(res["ids"][:, :7] != 0xFFFFFFFF)
    assert np.all(res["ids"][:, 7:] == 0xFFFFFFFF) and np.all(np.isneginf(res["sims"][:, 7:]))


@pytest.mark.parametrize("which", ["hp", "cp"])
def test_results_wellformed_and_stop_rule_holds(orc, hp_index, cp_index, which):
    ix, Q = hp_index if which == "hp" else cp_index
    qn = orc.normalize(Q)
    res = ix.search(Q, 10, 0.8)
    _check_result_wellformed(orc, ix, qn, res, 10)
    delta = 1 - 0.8
    for t in range(Q.shape[0]):
        dstop = int(res["stats"]["stop_depth"][t])
        if dstop > 0:
            s_k = float(res["sims"][t, 9])
            p = orc.collision_prob(ix.family, ix.ell, ix.P, s_k, dstop)
            assert (1 - p) ** ix.L <= delta * (1 + 1e-12)


def test_prefix_blocks_with_unit_segments(orc):
    # Fact 1 / Sec. 4.2: with B = 1 the round at depth i of repetition j visits
    # exactly S_{i,j} minus S_{i+1,j} (and S_{K,j} in the first round).
    ix, Q = _small_index(orc, family=0, n=1500, d=24, L=8, B=1)
    qn, qcodes, _ = ix.hash_queries(Q)
    res = ix.search(Q, 5, 0.9, trace_cap=1500 * 8 * 2)
    code_of = np.zeros((ix.L, ix.n), np.uint32)
    for j in range(ix.L):
        code_of[j, ix.ids[j]] = ix.codes[j]
    for t in range(Q.shape[0]):
        tr = res["trace"][t, : res["trace_len"][t]]
        seen = {}
        for key, pid in tr:
            seen.setdefault(((int(key) >> 24) & 0x3F, int(key) & 0xFFFFFF), []).append(int(pid))
        depths = sorted({k[0] for k in seen}, reverse=True)
        stop = int(res["stats"]["stop_depth"][t])
        for j in range(ix.L):
            for i in range(ix.Kb, stop - 1, -1):
                lcp_ge = lambda dd: (np.ones(ix.n, bool) if dd == 0 else
                                     (code_of[j] >> (32 - dd)) == (qcodes[t, j] >> (32 - dd)))
                want = lcp_ge(i) & (~lcp_ge(i + 1) if i < ix.Kb else True)
                got = sorted(seen.get((i, j), []))
                assert got == sorted(np.nonzero(want)[0].tolist()), (t, j, i)
        assert depths == [] or depths[-1] >= stop


def test_segments_extend_one_side_in_whole_segments(orc):
    # Sec. 4.2: dropping one bit extends the range on one side only; every
    # extension is a whole number of segments of B entries (clamped at the ends).
    B = 12
    ix, Q = _small_index(orc, family=0, n=4000, d=24, L=6, B=B)
    qn, qcodes, _ = ix.hash_queries(Q)
    res = ix.search(Q, 5, 0.95, trace_cap=4000 * 6 * 2)
    pos_of = np.zeros((ix.L, ix.n), np.int64)
    for j in range(ix.L):
        pos_of[j, ix.ids[j]] = np.arange(ix.n)
    for t in range(Q.shape[0]):
        tr = res["trace"][t, : res["trace_len"][t]]
        by = {}
        for key, pid in tr:
            by.setdefault(((int(key) >> 24) & 0x3F, int(key) & 0xFFFFFF), []).append(int(pid))
        for (i, j), pids in by.items():
            pos = np.sort(pos_of[j, pids])
            runs = np.split(pos, np.nonzero(np.diff(pos) != 1)[0] + 1)
            if i < ix.Kb:
                assert len(runs) == 1  # one side per dropped bit
            for run in runs:
                assert len(run) % B == 0 or run[0] == 0 or run[-1] == ix.n - 1


def test_recall_guarantee_without_filter(orc):
    # Definition 1 + Lemma 1: each true neighbour is reported w.p. >= 1 - delta,
    # so the mean recall over Q*k trials is >= 1 - delta up to sampling noise.
    X = datagen.vmf_mixture(6000, 24, 30, 20.0, seed=4)
    Qs = datagen.vmf_mixture(200, 24, 30, 20.0, seed=4, purpose="queries")
    ix = orc.OracleIndex(X, 1, L=12, seed=5)
    qn = orc.normalize(Qs)
    bi, bs = orc.brute_force(ix.x, qn, 10)
    for recall in (0.5, 0.8):
        res = ix.search(Qs, 10, recall, filter=False)
        got = np.mean(res["sims"] >= bs[:, -1:])
        N = Qs.shape[0] * 10
        assert got >= recall - 3 * math.sqrt(recall * (1 - recall) / N), (recall, got)


def test_filter_reduces_scoring(orc, hp_index):
    ix, Q = hp_index
    on = ix.search(Q, 10, 0.9, filter=True)["stats"]
    off = ix.search(Q, 10, 0.9, filter=False)["stats"]
    assert on["passed_filter"].sum() < on["retrieved"].sum()
    assert np.all(off["passed_filter"] == off["retrieved"])


def test_start_depth_schedule(orc, cp_index):
    # A start depth i0 runs rounds i0, i0-1, ...: the first round takes the
    # whole block at i0, later rounds one bit each; the result still obeys the
    # stop rule and is exact when the schedule reaches depth 0.
    ix, Q = cp_index
    qn = orc.normalize(Q)
    i0 = ix.Kb - 10
    res = ix.search(Q, 10, 0.9, start_depth=i0)
    st = res["stats"]
    assert np.all(st["start_depth"] == i0)
    assert np.all(st["stop_depth"] <= i0)
    assert np.all(st["rounds"] == i0 - st["stop_depth"] + 1)
    _check_result_wellformed(orc, ix, qn, res, 10)
    plain = ix.search(Q, 10, 0.9)["stats"]
    assert np.all(plain["rounds"] == ix.Kb - plain["stop_depth"] + 1)
    # full_depth: first depth after which k points were held (plain schedule)
    assert np.all((plain["full_depth"] >= plain["stop_depth"]) & (plain["full_depth"] <= ix.Kb))


def test_start_at_full_depth_keeps_the_filtered_work(orc, cp_index):
    # Starting at the depth where the plain schedule first holds k points skips
    # only rounds that ran unfiltered anyway: the retrieved positions can only
    # shrink (segments are rounded once instead of per round) and the stop
    # depth is unchanged for most queries.
    ix, Q = cp_index
    plain = ix.search(Q, 10, 0.9)
    fd = plain["stats"]["full_depth"]
    jump = ix.search(Q, 10, 0.9, start_depth=fd)
    assert np.all(jump["stats"]["rounds"] <= plain["stats"]["rounds"])
    same = np.mean(jump["stats"]["stop_depth"] == plain["stats"]["stop_depth"])
    assert same >= 0.8


def test_one_thread_gives_the_same_answers():
    import datagen
    import oracle as O

    X = datagen.vmf_mixture(3000, 48, 20, 40.0, seed=6)
    Q = datagen.vmf_mixture(24, 48, 20, 40.0, seed=6, purpose="queries")
    ix = O.OracleIndex(X, O.CROSSPOLYTOPE, L=12, seed=1)
    a = ix.search(Q, 10, 0.9)
    O.set_threads(1)
    try:
        b = ix.search(Q, 10, 0.9)
    finally:
        O.set_threads(0)
    assert np.array_equal(a["ids"], b["ids"]) and np.array_equal(a["sims"], b["sims"])
    assert np.array_equal(a["stats"], b["stats"])
