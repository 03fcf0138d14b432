"""Pooled hash functions (Sec. 3.2 "Pooling", App. B.2) in the library against
the oracle: each table's subset of the pool, the codes of points and queries,
and the search under both stop rules (Cantelli's bound, and Lemma 1's test as
if the functions were independent), bit for bit.  The cases cover SimHash
(3,072 one-bit functions), cross-polytope on the tensor-core path (d' <= 128,
including a last pool group that is only partly used) and with d' = 160 (one
point tile per hashing unit, two N tiles per function)."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1906_12211_gb300 as pf  # noqa: E402

DEV = torch.device("cuda:0")
L = 30


@pytest.fixture(scope="module", params=[("simhash", 64), ("crosspolytope", 100), ("crosspolytope", 37),
                                        ("crosspolytope", 150)])
def case(request, orc):
    pf.build()
    fam, d = request.param
    X = datagen.vmf_mixture(12_000, d, 40, 40.0, seed=d + 1)
    Q = datagen.vmf_mixture(120, d, 40, 40.0, seed=d + 1, purpose="queries")
    g = pf.Index(torch.from_numpy(X).to(DEV), fam, num_tables=L, seed=9, pool_bits=3072)
    o = orc.OracleIndex(X, orc.SIMHASH if fam == "simhash" else orc.CROSSPOLYTOPE, L=L, seed=9, pool_bits=3072)
    return g, o, X, Q


def test_subsets_equal_oracle(case):
    g, o, _, _ = case
    sel = g.array("pool_select", device="cpu").numpy().view(np.int32).reshape(L, g.fns)
    assert np.array_equal(sel, o.sel)


def test_point_and_query_codes_equal_oracle(case):
    g, o, X, Q = case
    n = X.shape[0]
    codes = g.array("codes").view(torch.int32).reshape(L, n).cpu().numpy().view(np.uint32)
    ids = g.array("ids").view(torch.int32).reshape(L, n).cpu().numpy().view(np.uint32)
    assert np.array_equal(codes, o.codes) and np.array_equal(ids, o.ids)
    qc, qs = g.hash_queries(torch.from_numpy(Q).to(DEV))
    _, oqc, oqs = o.hash_queries(Q)
    assert np.array_equal(qc.cpu().numpy().view(np.uint32), oqc)
    assert np.array_equal(qs.cpu().numpy().view(np.uint64), oqs)


@pytest.mark.parametrize("rule", ["cantelli", "independent"])
@pytest.mark.parametrize("scoring,stop_every", [("fp32", 0), ("bf16", 0), ("bf16", 4)])
def test_search_equals_oracle(case, rule, scoring, stop_every):
    g, o, _, Q = case
    ref = o.search(Q, 10, 0.9, pool_rule=rule, stop_every=stop_every)
    ids, sims, st = g.search(torch.from_numpy(Q).to(DEV), 10, 0.9, scoring=scoring, stats=True, pool_rule=rule,
                             stop_every=stop_every)
    assert np.array_equal(ids.cpu().numpy().view(np.uint32), ref["ids"])
    assert np.array_equal(sims.cpu().numpy(), ref["sims"])
    gs, os_ = pf.stats_to_numpy(st), ref["stats"]
    for f in ("start_depth", "stop_depth", "rounds", "full_depth", "last_reps"):
        assert np.array_equal(gs[f], os_[f]), f
    deep = os_["stop_depth"] > 0
    assert np.array_equal(gs["retrieved"][deep], os_["retrieved"][deep])


def test_budget_and_rejections(orc):
    pf.build()
    X = datagen.vmf_mixture(20_000, 100, 30, 40.0, seed=3)
    Xd = torch.from_numpy(X).to(DEV)
    g = pf.Index(Xd, "crosspolytope", budget_bytes=128 << 20, seed=1, pool_bits=3072)
    assert g.L == orc.budget_L(orc.CROSSPOLYTOPE, 20_000, 100, 32, 128 << 20, 0, 0, 0, 3072 // 8)
    assert g.info["bytes_used"] <= 128 << 20
    with pytest.raises(pf.PuffinnError):  # fewer pool functions than a table needs
        pf.Index(Xd, "crosspolytope", num_tables=4, pool_bits=24)
    with pytest.raises(pf.PuffinnError):  # the pseudo-random family is not pooled
        pf.Index(Xd, "fht", num_tables=4, pool_bits=3072)
