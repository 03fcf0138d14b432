"""Search parity with the oracle at the benchmark's n: the benchmark workload's
10^6 points (d = 100, 1,000-component vMF mixture, cross-polytope) indexed with
40 repetitions, so that the oracle can build the same index in the test's time.

With n = 10^6 a 13-bit prefix bucket holds about 120 entries, so the range pass
above 13 bits meets blocks longer than the four segment boundaries it probes
first and gallops; the range-path counters of the library prove that every
branch ran.  Ids, similarities and every statistic are compared element by
element with oracle.OracleIndex, in float32 and bfloat16 scoring, with the
filter on and off, given start depths, mixed k and recall, and every launch
shape."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1906_12211_gb300 as pf  # noqa: E402

DEV = torch.device("cuda:0")
W = datagen.WORKLOADS["vmf1k-n1m-d100"]
L = 40  # > M = 32: repetitions j >= 32 reuse sketch j mod 32
NQ = 200


@pytest.fixture(scope="module")
def both(orc):
    pf.build()
    X = datagen.vmf_mixture(W["n"], W["d"], W["components"], W["kappa"], seed=0, purpose="points")
    Q = datagen.vmf_mixture(NQ, W["d"], W["components"], W["kappa"], seed=0, purpose="queries")
    g = pf.Index(torch.from_numpy(X).to(DEV), "crosspolytope", num_tables=L, seed=0)
    o = orc.OracleIndex(X, orc.CROSSPOLYTOPE, L=L, seed=0)
    assert g.L == L and g.n == W["n"]
    return g, o, Q, torch.from_numpy(Q).to(DEV)


def _compare(out, ref):
    ids, sims, st = out
    assert np.array_equal(ids.cpu().numpy().view(np.uint32), ref["ids"])
    assert np.array_equal(sims.cpu().numpy(), ref["sims"])
    g, o = pf.stats_to_numpy(st), ref["stats"]
    for f in ("start_depth", "stop_depth", "rounds", "full_depth"):
        assert np.array_equal(g[f], o[f]), f
    deep = o["stop_depth"] > 0  # a depth-0 round is one exact scan, counted differently
    for f in ("retrieved", "passed_filter"):
        assert np.array_equal(g[f][deep], o[f][deep]), f


@pytest.mark.parametrize("scoring,filt", [("fp32", True), ("bf16", True), ("fp32", False)])
def test_search_equals_oracle_at_full_n(both, scoring, filt):
    g, o, Q, qd = both
    ref = o.search(Q, 10, 0.9, filter=filt)
    g.count_range_paths(True)
    g.set_shape(8, 4, 0, 3)  # rounds of short runs stream flat
    try:
        out = g.search(qd, 10, 0.9, scoring=scoring, filter=filt, stats=True)
        paths = g.count_range_paths(True)
    finally:
        g.count_range_paths(False)
        g.set_shape(8, 4, 0, 0)
    _compare(out, ref)
    # every branch of the range pass ran: prefix-table blocks, probed sides and
    # sides that galloped past the probed boundaries
    assert paths["prefix_table"] > 0 and paths["probed"] > 0 and paths["galloped"] > 0, paths
    assert paths["chunked_rounds"] > 0 and paths["flat_rounds"] > 0, paths  # both streaming modes ran
    assert np.all(ref["stats"]["stop_depth"] > 0)


def test_given_start_depths_and_mixed_k_at_full_n(both):
    g, o, Q, qd = both
    rng = np.random.default_rng(3)
    sd = rng.integers(8, g.Kb + 1, NQ).astype(np.int32)  # 32 = the plain start
    kk, rr = datagen.mixed_k_recall(NQ, ks=(1, 10, 50), deltas=(0.5, 0.1, 0.01), seed=5)
    ref = o.search(Q, kk, rr, k_max=50, start_depth=sd)
    out = g.search(qd, torch.from_numpy(kk).to(DEV), torch.from_numpy(rr).to(DEV), k_max=50, scoring="bf16",
                   start_depth=torch.from_numpy(sd).to(DEV), stats=True)
    _compare(out, ref)


@pytest.mark.parametrize("shape", [(8, 4, 0, 0), (4, 4, 0, 0), (8, 8, 0, 0), (8, 4, 3, 0), (8, 4, 0, 3),
                                   (4, 4, 0, 64), (8, 8, 0, 1)])
def test_every_launch_shape_at_full_n(both, shape):
    """flat_fill 3 and 64 stream short-run rounds flat (64: almost every round
    but depth 0), 1 only rounds whose chunks are nearly empty."""
    g, o, Q, qd = both
    ref = o.search(Q[:100], 10, 0.9)
    g.set_shape(*shape)
    try:
        out = g.search(qd[:100], 10, 0.9, scoring="bf16", stats=True)
    finally:
        g.set_shape(8, 4, 0, 0)
    _compare(out, ref)


@pytest.mark.parametrize("G", [1, 8])
def test_stop_every_at_full_n(both, G):
    g, o, Q, qd = both
    ref = o.search(Q, 10, 0.9, stop_every=G)
    out = g.search(qd, 10, 0.9, scoring="bf16", stats=True, stop_every=G)
    _compare(out, ref)
    assert np.array_equal(pf.stats_to_numpy(out[2])["last_reps"], ref["stats"]["last_reps"])
