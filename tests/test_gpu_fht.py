"""The pseudo-random cross-polytope family (Sec. 4.3: three fast Hadamard
transforms with random sign diagonals, after Andoni et al. 2015) in the library
against the oracle's statement of it (oracle/fht.py): the sign vectors, the
Monte-Carlo collision table, every point's and query's code, and the whole
search, bit for bit.  Transform lengths 8 to 512 cover every register layout
of the kernel (fewer coordinates than lanes, one per lane, 2 to 16 per lane);
the data include rows whose top two |y| tie exactly (the zero vector, unit
vectors, sums of two unit vectors), which exercise the float64 recomputation
and the first-index rule."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1906_12211_gb300 as pf  # noqa: E402

DEV = torch.device("cuda:0")
DIMS = [5, 12, 20, 37, 100, 200, 300]  # transform lengths 8, 16, 32, 64, 128, 256, 512
L = 12


def _special_rows(d):
    e = np.eye(d, dtype=np.float32)
    rows = [np.zeros(d, np.float32), e[0], e[d - 1], e[0] + e[1], e[0] - e[1], np.ones(d, np.float32)]
    return np.stack(rows)


@pytest.fixture(scope="module", params=DIMS)
def case(request, orc):
    pf.build()
    d = request.param
    X = np.concatenate([datagen.vmf_mixture(3000, d, 20, 30.0, seed=d), _special_rows(d)])
    Q = np.concatenate([datagen.vmf_mixture(60, d, 20, 30.0, seed=d, purpose="queries"), _special_rows(d)[1:]])
    g = pf.Index(torch.from_numpy(X).to(DEV), "fht", num_tables=L, seed=5)
    o = orc.OracleIndex(X, orc.CROSSPOLYTOPE_FHT, L=L, seed=5)
    return g, o, X, Q


def test_layout_and_signs_equal_oracle(case):
    from oracle import fht

    g, o, X, _ = case
    lay = fht.layout(X.shape[1])
    assert (g.ell, g.fns, g.Kb, g.L) == (lay["ell"], lay["F"], lay["Kb"], L)
    dp = lay["dp"]
    words = max(1, dp // 32)
    w = g.array("fht_signs", device="cpu").numpy().view(np.uint32).reshape(L, g.fns, 3, words)
    bits = (w[..., None] >> np.arange(32, dtype=np.uint32)) & 1  # [L][F][3][words][32]
    bits = bits.reshape(L, g.fns, 3, words * 32)[..., :dp]
    assert np.array_equal(np.where(bits == 1, -1.0, 1.0), o.A)


def test_collision_table_equals_oracle(case):
    g, o, _, _ = case
    P = g.array("cp_table", device="cpu").numpy().view(np.float64).reshape(o.P.shape)
    assert np.array_equal(P, o.P)


def test_point_codes_and_tables_equal_oracle(case):
    g, o, X, _ = case
    n = X.shape[0]
    codes = g.array("codes").view(torch.int32).reshape(L, n).cpu().numpy().view(np.uint32)
    ids = g.array("ids").view(torch.int32).reshape(L, n).cpu().numpy().view(np.uint32)
    assert np.array_equal(codes, o.codes)
    assert np.array_equal(ids, o.ids)


def test_query_codes_equal_oracle(case):
    g, o, _, Q = case
    qc, qs = g.hash_queries(torch.from_numpy(Q).to(DEV))
    _, oqc, oqs = o.hash_queries(Q)
    assert np.array_equal(qc.cpu().numpy().view(np.uint32), oqc)
    assert np.array_equal(qs.cpu().numpy().view(np.uint64), oqs)


@pytest.mark.parametrize("scoring,filt", [("fp32", True), ("bf16", True), ("fp32", False)])
def test_search_equals_oracle(case, scoring, filt):
    g, o, _, Q = case
    ref = o.search(Q, 10, 0.9, filter=filt)
    ids, sims, st = g.search(torch.from_numpy(Q).to(DEV), 10, 0.9, scoring=scoring, filter=filt, stats=True)
    assert np.array_equal(ids.cpu().numpy().view(np.uint32), ref["ids"])
    assert np.array_equal(sims.cpu().numpy(), ref["sims"])
    gs, os_ = pf.stats_to_numpy(st), ref["stats"]
    for f in ("start_depth", "stop_depth", "rounds", "full_depth"):
        assert np.array_equal(gs[f], os_[f]), f
    deep = os_["stop_depth"] > 0
    assert np.array_equal(gs["retrieved"][deep], os_["retrieved"][deep])
    assert np.array_equal(gs["passed_filter"][deep], os_["passed_filter"][deep])


def test_budget_rule_matches_oracle(orc):
    pf.build()
    X = datagen.vmf_mixture(20_000, 100, 30, 40.0, seed=3)
    g = pf.Index(torch.from_numpy(X).to(DEV), "fht", budget_bytes=64 << 20, seed=1)
    assert g.L == orc.budget_L(orc.CROSSPOLYTOPE_FHT, 20_000, 100, 32, 64 << 20, 0)
    assert g.info["bytes_used"] <= 64 << 20
