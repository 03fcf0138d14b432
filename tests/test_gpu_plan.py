"""Captured searches (CUDA graphs of one batch shape) and launch-shape tuning:
both must leave every result and statistic exactly as pf_index_search gives it."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1906_12211_gb300 as pf  # noqa: E402

DEV = torch.device("cuda:0")
KMAX = 32


@pytest.fixture(scope="module")
def idx():
    pf.build()
    X = datagen.vmf_mixture(20_000, 100, 50, 50.0, seed=21)
    Qs = datagen.vmf_mixture(600, 100, 50, 50.0, seed=21, purpose="queries")
    Qt = datagen.vmf_mixture(4000, 100, 50, 50.0, seed=21, purpose="train")
    ix = pf.Index(torch.from_numpy(X).to(DEV), "crosspolytope", num_tables=40, seed=8)
    ix.learned_train(torch.from_numpy(Qt).to(DEV), 10, 0.9, epochs=10, seed=3)
    kk, rr = datagen.mixed_k_recall(300, ks=(1, 10, 32), deltas=(0.5, 0.1), seed=4)
    return {"ix": ix, "Q": torch.from_numpy(Qs).to(DEV), "k": torch.from_numpy(kk).to(DEV),
            "r": torch.from_numpy(rr).to(DEV)}


def _bufs(Qn):
    return (torch.empty((Qn, KMAX), dtype=torch.int32, device=DEV),
            torch.empty((Qn, KMAX), dtype=torch.float32, device=DEV),
            torch.empty((Qn, pf.STATS_DTYPE.itemsize), dtype=torch.uint8, device=DEV))


@pytest.mark.parametrize("scoring,learned", [("fp32", False), ("bf16", False), ("bf16", True)])
def test_plan_equals_search_and_follows_its_buffers(idx, scoring, learned):
    ix, k, r = idx["ix"], idx["k"], idx["r"]
    qbuf = idx["Q"][:300].clone()
    ids, sims, st = _bufs(300)
    plan = ix.plan(qbuf, k, r, ids, sims, k_max=KMAX, stats=st, scoring=scoring, learned=learned)
    try:
        for batch in (idx["Q"][:300], idx["Q"][300:], idx["Q"][:300]):
            qbuf.copy_(batch)  # new queries in the bound buffer
            ref = ix.search(batch, k, r, k_max=KMAX, scoring=scoring, learned=learned, stats=True)
            ids.fill_(7)
            plan.run()
            plan.check()
            assert torch.equal(ids, ref[0]) and torch.equal(sims, ref[1]) and torch.equal(st, ref[2])
    finally:
        plan.close()


def test_plan_with_start_depths(idx):
    ix, k, r = idx["ix"], idx["k"], idx["r"]
    q = idx["Q"][:300]
    sd = torch.from_numpy(np.random.default_rng(5).integers(0, ix.Kb + 1, 300).astype(np.int32)).to(DEV)
    ids, sims, st = _bufs(300)
    plan = ix.plan(q, k, r, ids, sims, k_max=KMAX, stats=st, start_depth=sd, scoring="bf16")
    try:
        plan.run()
        plan.check()
        ref = ix.search(q, k, r, k_max=KMAX, scoring="bf16", start_depth=sd, stats=True)
        assert torch.equal(ids, ref[0]) and torch.equal(sims, ref[1]) and torch.equal(st, ref[2])
    finally:
        plan.close()


def test_plan_reports_bad_k_and_keeps_other_rows(idx):
    ix, r = idx["ix"], idx["r"]
    q = idx["Q"][:300]
    k = idx["k"].clone()
    k[17] = 0  # outside [1, k_max]
    ids, sims, _ = _bufs(300)
    plan = ix.plan(q, k, r, ids, sims, k_max=KMAX)
    try:
        plan.run()
        with pytest.raises(pf.PuffinnError) as e:
            plan.check()
        assert e.value.status == -1
        assert bool((ids[17] == -1).all())
        good = torch.ones(300, dtype=torch.bool, device=DEV)
        good[17] = False
        kk = idx["k"].clone()
        ref = ix.search(q, kk, r, k_max=KMAX)
        assert torch.equal(ids[good], ref[0][good]) and torch.equal(sims[good], ref[1][good])
    finally:
        plan.close()


def test_live_plans_block_retraining_and_tuning(idx):
    ix, k, r = idx["ix"], idx["k"], idx["r"]
    q = idx["Q"][:300]
    ids, sims, _ = _bufs(300)
    plan = ix.plan(q, k, r, ids, sims, k_max=KMAX)
    try:
        with pytest.raises(pf.PuffinnError) as e:
            ix.tune(q, 10, 0.9)
        assert e.value.status == -1
        with pytest.raises(pf.PuffinnError) as e:
            ix.learned_train(q, 10, 0.9, epochs=1)
        assert e.value.status == -1
    finally:
        plan.close()
    ix.tune(q, 10, 0.9)  # allowed again


@pytest.mark.parametrize("scoring,learned", [("fp32", False), ("bf16", True)])
def test_tuning_changes_no_result(idx, scoring, learned):
    ix, k, r = idx["ix"], idx["k"], idx["r"]
    q = idx["Q"]
    kk = torch.full((600,), 10, dtype=torch.int32, device=DEV)
    before = ix.search(q, kk, 0.9, k_max=KMAX, scoring=scoring, learned=learned, stats=True)
    rep = ix.tune(q, 10, 0.9, scoring=scoring, learned=learned)
    assert rep["unroll"] in (4, 8) and rep["warps"] in (4, 8) and rep["ctas_per_sm"] >= 1
    assert rep["candidates"] >= 3 and (rep["warps"] == 4 or rep["unroll"] == 8)
    assert 0.0 < rep["best_ms"] <= rep["default_ms"]
    after = ix.search(q, kk, 0.9, k_max=KMAX, scoring=scoring, learned=learned, stats=True)
    assert torch.equal(before[0], after[0]) and torch.equal(before[1], after[1])
    # the method's counts are the same for every shape; how many bf16 estimates
    # needed an exact rerank depends on how the candidates meet the warp lists
    sb, sa = pf.stats_to_numpy(before[2]), pf.stats_to_numpy(after[2])
    for f in sb.dtype.names:
        if f != "reranked":
            assert np.array_equal(sb[f], sa[f]), f


@pytest.mark.parametrize("learned", [False, True])
def test_plan_on_page_locked_host_buffers(idx, learned):
    """A plan bound to page-locked host buffers copies its inputs in and its
    outputs out inside its graph: after check() the host buffers hold what
    pf_index_search returns; a second plan on another stream runs beside it."""
    ix, k, r = idx["ix"], idx["k"], idx["r"]
    hq = [idx["Q"][:300].cpu().pin_memory(), idx["Q"][300:].cpu().pin_memory()]
    hk = [k.cpu().pin_memory() for _ in range(2)]
    hr = [r.cpu().pin_memory() for _ in range(2)]
    hi = [torch.empty((300, KMAX), dtype=torch.int32).pin_memory() for _ in range(2)]
    hs = [torch.empty((300, KMAX), dtype=torch.float32).pin_memory() for _ in range(2)]
    hst = [torch.zeros((300, pf.STATS_DTYPE.itemsize), dtype=torch.uint8).pin_memory() for _ in range(2)]
    plans = [ix.plan(hq[b], hk[b], hr[b], hi[b], hs[b], k_max=KMAX, stats=hst[b], scoring="bf16", learned=learned)
             for b in range(2)]
    streams = [torch.cuda.current_stream(), torch.cuda.Stream(DEV)]
    try:
        for rep in range(2):
            for b in range(2):
                hi[b].fill_(7)
            for b in range(2):
                plans[b].run(streams[b])
            for b in range(2):
                plans[b].check(streams[b])
            for b in range(2):
                ref = ix.search(hq[b].to(DEV), k, r, k_max=KMAX, scoring="bf16", learned=learned, stats=True)
                assert torch.equal(hi[b], ref[0].cpu()) and torch.equal(hs[b], ref[1].cpu())
                assert torch.equal(hst[b], ref[2].cpu())
    finally:
        for p in plans:
            p.close()


def test_plan_rejects_pageable_host_buffers(idx):
    ix, k, r = idx["ix"], idx["k"], idx["r"]
    q = idx["Q"][:10].cpu()  # pageable
    ids, sims, _ = _bufs(10)
    with pytest.raises(pf.PuffinnError) as e:
        ix.plan(q, k[:10], r[:10], ids, sims, k_max=KMAX)
    assert e.value.status == -1
