"""Pins of the sketch filter inside the oracle's query loop (Sec. 4.2
"Filtering candidate points" and "Computing distances", the footnote of
Fig. 2, Sec. 3.3 for the law of the sketch distance).

The oracle's trace lists every retrieved entry in visiting order with a flag
telling whether it passed the filter and was scored.  `_replay` recomputes that
decision for every entry with nothing from the oracle's query code: the Hamming
distance of sketch (j mod M) of the query and of the point (popcount in
numpy), and the threshold from the top-k of the entries scored before the
entry's snapshot (the largest t with cos(t*pi/64) >= s_k, numpy float64).
Snapshots: at the start of every round and, in the first round, before
repetitions 1, 2, 4, 8, 16 and every 32 after that.  A plausible slip in the oracle ('>=' for
'>', the wrong sketch, a threshold that is not refreshed) changes some flags;
`test_planted_mistakes_are_caught` plants each one in a copy of the oracle and
checks that the replay sees it.

The statistical pin: for points at a fixed angle theta from the query, the
Hamming distance of two 64-bit sketches is Binomial(64, theta/pi) (Sec. 3.3),
so the share of such entries that pass at threshold tau is that law's CDF at
tau."""
import math
import os

import numpy as np
import pytest

import datagen

GROUP = 32  # repetitions per threshold snapshot in a query's first round, after 1, 2, 4, 8, 16


def _first_round_group(j: int) -> int:
    """Snapshot group of repetition j in a first round: boundaries 1, 2, 4, 8,
    16, then every 32."""
    return 0 if j == 0 else (j.bit_length() if j < GROUP else 5 + j // GROUP)
_COS = np.cos(np.arange(65) * np.pi / 64.0)


def _tau(s_k: float) -> int:
    ok = np.nonzero(_COS >= s_k)[0]
    return int(ok.max()) if ok.size else 0


def _popcount64(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, np.uint64)
    return np.unpackbits(a.view(np.uint8).reshape(-1, 8), axis=1).sum(axis=1)


def _replay(orc, ix, res, t: int, k: int, sims_t: np.ndarray):
    """Replay query t's trace.  Returns (mismatching entries, final ids, final
    sims, per-entry threshold, per-entry flag)."""
    tr = res["trace"][t, : res["trace_len"][t]]
    key = tr[:, 0].astype(np.int64)
    ids = tr[:, 1].astype(np.int64)
    flag = (key >> 31) & 1
    depth = (key >> 24) & 0x3F
    j = key & 0xFFFFFF
    m = j % ix.M
    ham = _popcount64(res["qsk"][t, m] ^ ix.sk[m, ids])
    start = int(res["stats"]["start_depth"][t])
    top = []  # (sim, id), sorted by sim desc then id asc, unique ids
    taus = np.zeros(len(tr), np.int64)
    bad = 0
    tau = 64
    prev = None
    for e in range(len(tr)):
        d_e, j_e = int(depth[e]), int(j[e])
        snap = (d_e, _first_round_group(j_e) if d_e == start else -1)
        if snap != prev:
            tau = 64 if len(top) < k else _tau(float(top[-1][0]))
            prev = snap
        taus[e] = tau
        expect = d_e == 0 or int(ham[e]) <= tau
        if expect != bool(flag[e]):
            bad += 1
        if expect:
            pid = int(ids[e])
            if all(p != pid for _, p in top):
                top.append((float(sims_t[pid]), pid))
                top.sort(key=lambda v: (-v[0], v[1]))
                del top[k:]
    return bad, [p for _, p in top], [s for s, _ in top], taus, flag


def _all_sims(orc, ix, qn):
    return np.array([[orc.sim(qn[t], ix.x[p]) for p in range(ix.n)] for t in range(qn.shape[0])], np.float32)


def _index(orc, family, L=40):
    X = datagen.vmf_mixture(4000, 32, 25, 25.0, seed=17)
    Q = datagen.vmf_mixture(30, 32, 25, 25.0, seed=17, purpose="queries")
    return orc.OracleIndex(X, family, L=L, M=32, seed=9), Q


@pytest.fixture(scope="module")
def cases(orc):
    out = {}
    for fam in (orc.SIMHASH, orc.CROSSPOLYTOPE):
        ix, Q = _index(orc, fam)
        qn = orc.normalize(Q)
        out[fam] = (ix, Q, _all_sims(orc, ix, qn))
    return out


def _check_all(orc, ix, Q, sims, k, recall, variant=None, start=None):
    cap = ix.n * ix.L
    res = ix.search(Q, k, recall, trace_cap=cap, variant=variant, start_depth=start)
    assert np.all(res["trace_len"] <= cap)
    total_bad, same_result = 0, True
    for t in range(Q.shape[0]):
        bad, ids, ss, _, flag = _replay(orc, ix, res, t, k, sims[t])
        total_bad += bad
        assert int(flag.sum()) == int(res["stats"]["passed_filter"][t])
        got = [int(v) for v in res["ids"][t] if v != 0xFFFFFFFF]
        same_result &= got == ids and np.array_equal(res["sims"][t, : len(ss)], np.float32(ss))
    return total_bad, same_result, res


@pytest.mark.parametrize("start", [None, 6])
@pytest.mark.parametrize("k,recall", [(10, 0.9), (1, 0.9), (5, 0.99)])
@pytest.mark.parametrize("fam", [0, 1])
def test_filter_decisions_match_independent_replay(orc, cases, fam, k, recall, start):
    """start 6: a first round that takes a large block, so that the first
    round's group snapshots tighten the threshold within the round."""
    ix, Q, sims = cases[fam]
    assert ix.L > ix.M  # repetitions j >= M reuse sketch j mod M
    bad, same, res = _check_all(orc, ix, Q, sims, k, recall, start=start)
    assert bad == 0
    assert same
    st = res["stats"]
    # the filter did act
    assert st["passed_filter"].sum() < st["retrieved"].sum()


def test_ties_at_the_threshold_pass(orc, cases):
    """Sec. 4.2: a point passes when its distance is *at most* tau.  Entries
    with distance exactly tau occur and were all scored."""
    ix, Q, sims = cases[1]
    res = ix.search(Q, 10, 0.9, trace_cap=ix.n * ix.L)
    at_tau = 0
    for t in range(Q.shape[0]):
        _, _, _, taus, flag = _replay(orc, ix, res, t, 10, sims[t])
        tr = res["trace"][t, : res["trace_len"][t]]
        key = tr[:, 0].astype(np.int64)
        m = (key & 0xFFFFFF) % ix.M
        ham = _popcount64(res["qsk"][t, m] ^ ix.sk[m, tr[:, 1].astype(np.int64)])
        sel = (ham == taus) & (((key >> 24) & 0x3F) > 0)
        at_tau += int(sel.sum())
        assert np.all(flag[sel] == 1)
    assert at_tau > 20


_MUTANTS = {
    "ge_instead_of_gt": ("if (ham > tau) continue;", "if (ham >= tau) continue;"),
    "query_sketch_index": ("popcount64(qsk[j % M] ^", "popcount64(qsk[(j + 1) % M] ^"),
    "no_first_round_groups": ("(s.rounds == 0 && first_round_snapshot(j))", "(0)"),
    "first_round_groups_of_32": ("(s.rounds == 0 && first_round_snapshot(j))",
                                 "(s.rounds == 0 && j % ORC_SNAPSHOT_GROUP == 0)"),
    "no_refresh_per_round": ("if (j == 0 || (stop_every", "if ((j == 0 && s.rounds == 0) || (stop_every"),
    "kth_from_wrong_slot": ("orc_filter_tau_eps((double)ps[k - 1]", "orc_filter_tau_eps((double)ps[0]"),
}


@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_planted_mistakes_are_caught(orc, cases, tmp_path, name):
    src = open(os.path.join(os.path.dirname(orc.__file__), "puffinn_oracle.c")).read()
    old, new = _MUTANTS[name]
    assert src.count(old) == 1
    variant = orc.compile_variant(src.replace(old, new), str(tmp_path / f"lib_{name}.so"))
    caught = False
    for fam in (0, 1):
        ix, Q, sims = cases[fam]
        for k, recall, start in ((10, 0.9, None), (5, 0.99, None), (10, 0.9, 6)):
            bad, same, _ = _check_all(orc, ix, Q, sims, k, recall, variant=variant, start=start)
            caught |= bad > 0 or not same
    assert caught, name


def _fixed_angle_data(n_q=40, per_q=300, d=64, c_bg=0.9, c_top=0.95, seed=23):
    """Per query q: one point at cosine c_top and per_q points at cosine c_bg
    (x = c q + sqrt(1 - c^2) u with u a random unit vector orthogonal to q)."""
    g = datagen.gaussian(n_q * (per_q + 2), d, seed=seed).astype(np.float64)
    q = g[:n_q] / np.linalg.norm(g[:n_q], axis=1, keepdims=True)
    pts, owner = [], []
    r = n_q
    for t in range(n_q):
        for c in [c_top] + [c_bg] * per_q:
            u = g[r] - (g[r] @ q[t]) * q[t]
            u /= np.linalg.norm(u)
            pts.append(c * q[t] + math.sqrt(1 - c * c) * u)
            owner.append(t)
            r += 1
    return np.asarray(pts, np.float32), q.astype(np.float32), np.asarray(owner)


def test_pass_rate_at_a_fixed_angle_is_binomial(orc):
    from scipy.stats import binom

    c_bg = 0.9
    X, Q, owner = _fixed_angle_data(c_bg=c_bg)
    ix = orc.OracleIndex(X, orc.SIMHASH, L=64, M=32, seed=4)
    qn = orc.normalize(Q)
    sims = _all_sims(orc, ix, qn)
    res = ix.search(Q, 1, 1.0 - 1e-6, trace_cap=ix.n * ix.L)
    theta = math.acos(c_bg)
    by_tau = {}
    for t in range(Q.shape[0]):
        bad, _, _, taus, flag = _replay(orc, ix, res, t, 1, sims[t])
        assert bad == 0
        tr = res["trace"][t, : res["trace_len"][t]]
        ids = tr[:, 1].astype(np.int64)
        depth = (tr[:, 0].astype(np.int64) >> 24) & 0x3F
        bg = (owner[ids] == t) & (np.abs(sims[t][ids] - c_bg) < 1e-5) & (depth > 0) & (taus < 64)
        for tau in np.unique(taus[bg]):
            sel = bg & (taus == tau)
            n_, p_ = by_tau.get(int(tau), (0, 0))
            by_tau[int(tau)] = (n_ + int(sel.sum()), p_ + int(flag[sel].sum()))
    n_tot = sum(v[0] for v in by_tau.values())
    assert n_tot > 20_000
    exp = sum(v[0] * binom.cdf(tau, 64, theta / math.pi) for tau, v in by_tau.items())
    obs = sum(v[1] for v in by_tau.values())
    assert abs(obs - exp) <= 0.05 * exp, (obs, exp, by_tau)
    for tau, (n_, p_) in by_tau.items():
        if n_ >= 5000:  # each well-populated threshold on its own
            assert abs(p_ / n_ - binom.cdf(tau, 64, theta / math.pi)) < 0.04, (tau, n_, p_)
