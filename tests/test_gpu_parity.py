"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle on the
same seeded inputs.  Integer and index results are compared bit-exactly;
similarities too (both sides compute the same canonical float32 sum)."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1906_12211_gb300 as pf  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="session", autouse=True)
def _built():
    pf.build()
    pf.lib()


def u32(t, shape=None):
    a = t.cpu().numpy().view(np.uint32)
    return a.reshape(shape) if shape is not None else a


def gpu_index(X, family, **kw):
    return pf.Index(torch.from_numpy(np.ascontiguousarray(X)).to(DEV), family, **kw)


def oracle_rows_from_lib(ix, W):
    """Re-arrange the library's padded hash rows into the oracle's layout."""
    L, d, dp = ix.L, ix.d, ix.d_pad
    if ix.family == pf.CROSSPOLYTOPE:
        F = ix.fns
        A = W[: L * F * dp].reshape(L, F, dp, dp)[:, :, :d, :d].reshape(L, F * d, d)
    else:
        A = W[: L * 32].reshape(L, 32, dp)[:, :, :d]
    S = W[-64 * ix.M:, :d]
    return A, S


class Case:
    def __init__(self, orc, name, X, Q, family, L=None, budget=None, seed=0, B=12, layout="table", rows="f32"):
        self.name, self.X, self.Q, self.layout, self.rows = name, X, Q, layout, rows
        kw = dict(seed=seed, segment_B=B, sketch_layout=layout, rows=rows)
        if budget is not None:
            kw["budget_bytes"] = budget
        else:
            kw["num_tables"] = L
        self.gpu = gpu_index(X, family, **kw)
        fam = orc.SIMHASH if family == "simhash" else orc.CROSSPOLYTOPE
        self.orc = orc.OracleIndex(X, fam, L=self.gpu.L, seed=seed, B=B, row_storage=1 if rows == "f16" else 0)
        self.qd = torch.from_numpy(Q).to(DEV)


@pytest.fixture(scope="module")
def cfg1(orc):
    # points and queries i.i.d. N(0,1), n = 10,000, d = 64, SimHash, 32 MiB
    X, Q = datagen.make("gauss-n10k-d64", seed=0)
    c = Case(orc, "gauss-n10k-d64", X, Q, "simhash", budget=32 << 20)
    assert c.gpu.L == orc.budget_L(orc.SIMHASH, 10_000, 64, 32, 32 << 20, 0)
    return c


@pytest.fixture(scope="module")
def cfg1pp(orc):
    # the same workload with M sketches per point (the paper's layout), 32 MiB
    X, Q = datagen.make("gauss-n10k-d64", seed=0)
    c = Case(orc, "gauss-n10k-d64-pp", X, Q, "simhash", budget=32 << 20, layout="point")
    assert c.gpu.L == orc.budget_L(orc.SIMHASH, 10_000, 64, 32, 32 << 20, 1)
    return c


@pytest.fixture(scope="module")
def cpmidpp(orc):
    X = datagen.vmf_mixture(20_000, 100, 50, 50.0, seed=3)
    Q = datagen.vmf_mixture(150, 100, 50, 50.0, seed=3, purpose="queries")
    return Case(orc, "vmf-n20k-d100-pp", X, Q, "crosspolytope", L=40, seed=7, layout="point")


@pytest.fixture(scope="module")
def cpmid(orc):
    # vMF mixture, n = 20,000 (several sort tiles + a ragged tail), d = 100, CP
    X = datagen.vmf_mixture(20_000, 100, 50, 50.0, seed=3)
    Q = datagen.vmf_mixture(150, 100, 50, 50.0, seed=3, purpose="queries")
    return Case(orc, "vmf-n20k-d100", X, Q, "crosspolytope", L=40, seed=7)


@pytest.fixture(scope="module")
def cpodd(orc):
    # ragged dimension (d = 37 -> 48 padded), small n, CP with l = 7
    X = datagen.gaussian(1500, 37, seed=4)
    Q = datagen.gaussian(40, 37, seed=4, purpose="queries")
    return Case(orc, "gauss-n1500-d37", X, Q, "crosspolytope", L=16, seed=9)


@pytest.fixture(scope="module")
def cpwide(orc):
    # d = 150 (d_pad 160 > 128: one point tile per hashing unit and CP functions
    # of two N tiles, 128 + 32 rows), CP with l = 9
    X = datagen.vmf_mixture(3000, 150, 20, 40.0, seed=5)
    Q = datagen.vmf_mixture(40, 150, 20, 40.0, seed=5, purpose="queries")
    return Case(orc, "vmf-n3000-d150", X, Q, "crosspolytope", L=12, seed=4)


@pytest.fixture(scope="module")
def hpodd(orc):
    # SimHash with L = 7 (not a multiple of the 4-repetition hashing groups), d = 20
    X = datagen.gaussian(2500, 20, seed=6)
    Q = datagen.gaussian(50, 20, seed=6, purpose="queries")
    return Case(orc, "gauss-n2500-d20", X, Q, "simhash", L=7, seed=2)


@pytest.fixture(scope="module")
def cfg1h(orc):
    # config 1 with binary16 rows (the stored points are the rounded rows), 32 MiB
    X, Q = datagen.make("gauss-n10k-d64", seed=0)
    c = Case(orc, "gauss-n10k-d64-f16", X, Q, "simhash", budget=32 << 20, rows="f16")
    assert c.gpu.L == orc.budget_L(orc.SIMHASH, 10_000, 64, 32, 32 << 20, 0, 1)
    assert c.gpu.L > orc.budget_L(orc.SIMHASH, 10_000, 64, 32, 32 << 20, 0, 0)  # rows take less of the budget
    return c


@pytest.fixture(scope="module")
def cpmidh(orc):
    # the vMF case (d = 96 as in the 10M-point workload) with binary16 rows
    X = datagen.vmf_mixture(20_000, 96, 50, 100.0, seed=8)
    Q = datagen.vmf_mixture(150, 96, 50, 100.0, seed=8, purpose="queries")
    return Case(orc, "vmf-n20k-d96-f16", X, Q, "crosspolytope", L=40, seed=5, rows="f16")


@pytest.fixture(scope="module")
def cpwideh(orc):
    # d = 150 (two N tiles per CP function, hashing the rounded rows) with binary16 rows
    X = datagen.vmf_mixture(3000, 150, 20, 40.0, seed=5)
    Q = datagen.vmf_mixture(40, 150, 20, 40.0, seed=5, purpose="queries")
    return Case(orc, "vmf-n3000-d150-f16", X, Q, "crosspolytope", L=12, seed=4, rows="f16")


@pytest.fixture(scope="module")
def cpsyn(orc):
    # the paper's SYNTHETIC construction (Sec. 5) at n = 3,000: 3 x 100 = 300
    # dimensions (d_pad 304: CP functions of three N tiles, 128 + 128 + 48 rows,
    # five K blocks; l = 10, three functions of 30 bits)
    X = datagen.paper_synthetic_points(3000, 100, seed=2)
    Q = datagen.paper_synthetic_queries(40, 100, seed=2)
    return Case(orc, "paper-synthetic-n3000-d300", X, Q, "crosspolytope", L=8, seed=6)


@pytest.fixture(scope="module")
def cpmaxd(orc):
    # the largest dimension the library takes (d = 320), HP to keep the oracle fast
    X = datagen.gaussian(1200, 320, seed=12)
    Q = datagen.gaussian(30, 320, seed=12, purpose="queries")
    return Case(orc, "gauss-n1200-d320", X, Q, "simhash", L=10, seed=3)


@pytest.fixture(scope="module")
def cp256(orc):
    # d = 256 (the planted workload's dimension): CP functions of exactly two
    # full N tiles, four K blocks, one point tile per hashing unit
    X, Q, _ = datagen.planted(1500, 256, 30, n_decoys=15, seed=13)
    return Case(orc, "planted-n1980-d256", X, Q, "crosspolytope", L=6, seed=8)


CASES = ["cfg1", "cpmid", "cpodd", "cpwide", "hpodd", "cfg1pp", "cpmidpp", "cfg1h", "cpmidh", "cpwideh", "cpsyn",
         "cpmaxd", "cp256"]


@pytest.fixture
def case(request):
    return request.getfixturevalue(request.param)


# ------------------------------------------------------------------ build
@pytest.mark.parametrize("case", CASES, indirect=True)
def test_parameters_bit_equal(case):
    ix = case.gpu
    rows = (ix.L * (ix.fns * ix.d_pad if ix.family == pf.CROSSPOLYTOPE else 32) + 64 * ix.M)
    W = ix.array("hash_rows").cpu().numpy().view(np.float32).reshape(rows, ix.d_pad)
    A, S = oracle_rows_from_lib(ix, W)
    assert np.array_equal(A, case.orc.A)
    assert np.array_equal(S, case.orc.S)
    if ix.family == pf.CROSSPOLYTOPE:
        P = ix.array("cp_table").cpu().numpy().view(np.float64).reshape(41, ix.ell + 1)
        assert np.array_equal(P, case.orc.P)


@pytest.mark.parametrize("case", CASES, indirect=True)
def test_normalised_rows_bit_exact(case):
    ix = case.gpu
    if case.rows == "f16":
        h = ix.array("rows_f16").cpu().numpy().view(np.float16).reshape(ix.n, ix.d_pad)
        assert np.array_equal(h[:, : ix.d].view(np.uint16), case.orc.x.astype(np.float16).view(np.uint16))
        x = h.astype(np.float32)
        with pytest.raises(pf.PuffinnError):
            ix.array("rows_f32")
    else:
        x = ix.array("rows_f32").cpu().numpy().view(np.float32).reshape(ix.n, ix.d_pad)
    assert np.array_equal(x[:, : ix.d], case.orc.x)
    assert np.all(x[:, ix.d:] == 0)
    xb = ix.array("rows_bf16").view(torch.bfloat16).reshape(ix.n, ix.d_pad)
    ref = torch.from_numpy(x).to(torch.bfloat16)  # round to nearest even
    assert torch.equal(xb.cpu(), ref)


@pytest.mark.parametrize("case", CASES, indirect=True)
def test_tables_sketches_prefix_bit_exact(case):
    ix = case.gpu
    codes = u32(ix.array("codes"), (ix.L, ix.n))
    ids = u32(ix.array("ids"), (ix.L, ix.n))
    assert np.array_equal(codes, case.orc.codes)
    assert np.array_equal(ids, case.orc.ids)
    pfx = u32(ix.array("prefix"), (ix.L, 8193))
    assert np.array_equal(pfx, case.orc.pfx)
    if case.layout == "point":
        sk = ix.array("sketches").cpu().numpy().view(np.uint64).reshape(ix.M, ix.n)
        assert np.array_equal(sk, case.orc.sk)
    else:
        skc = ix.array("table_sketches").cpu().numpy().view(np.uint64).reshape(ix.L, ix.n)
        ref = np.stack([case.orc.sk[j % ix.M][case.orc.ids[j]] for j in range(ix.L)])
        assert np.array_equal(skc, ref)


@pytest.mark.parametrize("case", CASES, indirect=True)
def test_query_hashing_bit_exact(case):
    qc, qs = case.gpu.hash_queries(case.qd)
    _, oqc, oqs = case.orc.hash_queries(case.Q)
    assert np.array_equal(u32(qc), oqc)
    assert np.array_equal(qs.cpu().numpy().view(np.uint64), oqs)


# ------------------------------------------------------------------ search
def _compare(gpu_out, ref, check_stats=True):
    ids, sims, st = gpu_out
    assert np.array_equal(u32(ids), ref["ids"])
    assert np.array_equal(sims.cpu().numpy(), ref["sims"])
    if check_stats and st is not None:
        g = pf.stats_to_numpy(st)
        o = ref["stats"]
        assert np.array_equal(g["stop_depth"], o["stop_depth"])
        assert np.array_equal(g["rounds"], o["rounds"])
        assert np.array_equal(g["full_depth"], o["full_depth"])
        assert np.array_equal(g["start_depth"], o["start_depth"])
        deep = o["stop_depth"] > 0
        assert np.array_equal(g["retrieved"][deep], o["retrieved"][deep])
        assert np.array_equal(g["passed_filter"][deep], o["passed_filter"][deep])
        assert np.array_equal(g["last_reps"], o["last_reps"])


@pytest.mark.parametrize("case", CASES, indirect=True)
@pytest.mark.parametrize("filt", [True, False])
def test_search_bit_exact(case, filt):
    ref = case.orc.search(case.Q, 10, 0.9, filter=filt)
    out = case.gpu.search(case.qd, 10, 0.9, filter=filt, stats=True)
    _compare(out, ref)


@pytest.mark.parametrize("case", CASES, indirect=True)
def test_bf16_scoring_equals_fp32(case):
    ref = case.orc.search(case.Q, 10, 0.9)
    out = case.gpu.search(case.qd, 10, 0.9, scoring="bf16", stats=True)
    _compare(out, ref)
    st = pf.stats_to_numpy(out[2])
    assert np.all(st["reranked"] <= st["scored"])


def test_mixed_k_and_recall(cpmid, orc):
    k, rec = datagen.mixed_k_recall(cpmid.Q.shape[0], seed=1)
    ref = cpmid.orc.search(cpmid.Q, k, rec, k_max=128)
    out = cpmid.gpu.search(cpmid.qd, torch.from_numpy(k).to(DEV), torch.from_numpy(rec).to(DEV), k_max=128,
                           stats=True)
    _compare(out, ref)
    out2 = cpmid.gpu.search(cpmid.qd, torch.from_numpy(k).to(DEV), torch.from_numpy(rec).to(DEV), k_max=128,
                            scoring="bf16")
    _compare(out2, ref, check_stats=False)


@pytest.mark.parametrize("start", [0, 5, 20, 29, 31])
def test_start_depth_override(cpmid, start):
    ref = cpmid.orc.search(cpmid.Q[:40], 10, 0.9, start_depth=start)
    sd = torch.full((40,), start, dtype=torch.int32, device=DEV)
    out = cpmid.gpu.search(cpmid.qd[:40], 10, 0.9, start_depth=sd, stats=True)
    _compare(out, ref)


def test_depth_zero_is_brute_force(cfg1, orc):
    qn = orc.normalize(cfg1.Q[:20])
    bi, bs = orc.brute_force(cfg1.orc.x, qn, 10)
    sd = torch.zeros(20, dtype=torch.int32, device=DEV)
    ids, sims, _ = cfg1.gpu.search(cfg1.qd[:20], 10, 0.9, start_depth=sd)
    assert np.array_equal(u32(ids), bi) and np.array_equal(sims.cpu().numpy(), bs)


def test_host_buffers_match_device(cpmid):
    Qh = np.ascontiguousarray(cpmid.Q[:50])
    kh = np.full(50, 10, np.int32)
    rh = np.full(50, 0.9, np.float64)
    ids_h = np.zeros((50, 10), np.uint32)
    sims_h = np.zeros((50, 10), np.float32)
    st_h = np.zeros(50, pf.STATS_DTYPE)
    pf._check(pf.lib().pf_index_search(cpmid.gpu._h, pf._ptr(Qh), 50, pf._ptr(kh), pf._ptr(rh), 10,
                                       pf._ptr(ids_h), pf._ptr(sims_h), pf._ptr(st_h), None, None))
    ids, sims, _ = cpmid.gpu.search(cpmid.qd[:50], 10, 0.9)
    assert np.array_equal(ids_h, u32(ids)) and np.array_equal(sims_h, sims.cpu().numpy())


def test_fewer_points_than_k(orc):
    X = datagen.gaussian(7, 16, seed=2)
    g = gpu_index(X, "simhash", num_tables=5, seed=3)
    o = orc.OracleIndex(X, orc.SIMHASH, L=5, seed=3)
    ref = o.search(X[:3], 10, 0.9)
    out = g.search(torch.from_numpy(X[:3]).to(DEV), 10, 0.9, stats=True)
    _compare(out, ref)
    assert np.all(u32(out[0])[:, 7:] == 0xFFFFFFFF)


def test_single_point_and_k_max_128(orc):
    X = datagen.gaussian(1, 8, seed=5)
    g = gpu_index(X, "crosspolytope", num_tables=3, seed=1)
    ids, sims, _ = g.search(torch.from_numpy(X).to(DEV), 1, 0.5, k_max=128)
    assert u32(ids)[0, 0] == 0 and np.all(u32(ids)[0, 1:] == 0xFFFFFFFF)


def test_errors_are_statuses():
    X = torch.randn(100, 16, device=DEV)
    with pytest.raises(pf.PuffinnError) as e:
        pf.Index(X, "simhash", budget_bytes=1000)
    assert e.value.status == -2
    g = pf.Index(X, "simhash", num_tables=4)
    with pytest.raises(pf.PuffinnError) as e:
        g.search(X[:4], 10, 1.5)
    assert e.value.status == -1
    with pytest.raises(pf.PuffinnError) as e:
        g.search(X[:4], torch.full((4,), 20, dtype=torch.int32, device=DEV), 0.9, k_max=10)
    assert e.value.status == -1
    ids, sims, _ = g.search(X[:0], 10, 0.9)
    assert ids.shape[0] == 0


@pytest.mark.parametrize("shape", [(4, 4, 0), (8, 8, 0), (8, 4, 3), (8, 4, 0, 3), (4, 4, 0, 64), (8, 8, 0, 3)])
def test_every_launch_shape_equals_the_oracle(cpmid, shape):
    # positions per lane, warps per query, CTAs per SM and the streaming rule change no result
    ref = cpmid.orc.search(cpmid.Q, 10, 0.9)
    cpmid.gpu.set_shape(*shape)
    try:
        _compare(cpmid.gpu.search(cpmid.qd, 10, 0.9, stats=True), ref)
        _compare(cpmid.gpu.search(cpmid.qd, 10, 0.9, scoring="bf16", stats=True), ref)
    finally:
        cpmid.gpu.set_shape(8, 4, 0)


def test_invalid_launch_shapes_are_rejected(cpmid):
    for bad in ((4, 8, 0), (6, 4, 0), (8, 5, 0), (8, 4, -1), (8, 4, 0, -1), (8, 4, 0, 65)):
        with pytest.raises(pf.PuffinnError) as e:
            cpmid.gpu.set_shape(*bad)
        assert e.value.status == -1


# ------------------------------------------------------------------ stop test after groups of repetitions
@pytest.mark.parametrize("case", ["cfg1", "cpmid", "cpwide", "cpmidpp"], indirect=True)
@pytest.mark.parametrize("G", [1, 5, 32])
@pytest.mark.parametrize("scoring", ["fp32", "bf16"])
def test_stop_every_bit_exact(case, G, scoring):
    """Alg. 1's stop test after every G repetitions: the same stop depth and the
    same number of repetitions searched in the last round as the oracle."""
    ref = case.orc.search(case.Q, 10, 0.9, stop_every=G)
    out = case.gpu.search(case.qd, 10, 0.9, scoring=scoring, stats=True, stop_every=G)
    _compare(out, ref)
    assert np.any(ref["stats"]["last_reps"] < case.gpu.L) or G >= case.gpu.L


def test_stop_every_with_start_depths_and_mixed_k(cpmid):
    k, rec = datagen.mixed_k_recall(cpmid.Q.shape[0], seed=6)
    sd = np.random.default_rng(2).integers(0, cpmid.gpu.Kb + 1, cpmid.Q.shape[0]).astype(np.int32)
    ref = cpmid.orc.search(cpmid.Q, k, rec, k_max=128, start_depth=sd, stop_every=3)
    out = cpmid.gpu.search(cpmid.qd, torch.from_numpy(k).to(DEV), torch.from_numpy(rec).to(DEV), k_max=128,
                           start_depth=torch.from_numpy(sd).to(DEV), stats=True, scoring="bf16", stop_every=3)
    _compare(out, ref)


# ------------------------------------------------------------------ filter slack (Fig. 2 footnote)
@pytest.mark.parametrize("case", ["cfg1", "cpmid", "cpmidpp"], indirect=True)
@pytest.mark.parametrize("eps", [0.1, 0.3])
def test_filter_slack_bit_exact(case, eps):
    ref = case.orc.search(case.Q, 10, 0.9, filter_eps=eps)
    out = case.gpu.search(case.qd, 10, 0.9, scoring="bf16", stats=True, filter_eps=eps)
    _compare(out, ref)
    # a captured plan and the no-allocation entry point take the same slack
    Q = case.qd.shape[0]
    ids = torch.empty((Q, 10), dtype=torch.int32, device=DEV)
    sims = torch.empty((Q, 10), dtype=torch.float32, device=DEV)
    k = torch.full((Q,), 10, dtype=torch.int32, device=DEV)
    r = torch.full((Q,), 0.9, dtype=torch.float64, device=DEV)
    plan = case.gpu.plan(case.qd, k, r, ids, sims, k_max=10, scoring="bf16", filter_eps=eps)
    try:
        plan.run()
        plan.check()
    finally:
        plan.close()
    assert np.array_equal(u32(ids), ref["ids"]) and np.array_equal(sims.cpu().numpy(), ref["sims"])
    ids2, sims2 = torch.empty_like(ids), torch.empty_like(sims)
    case.gpu.search_noalloc(case.qd, k, r, ids2, sims2, k_max=10, scoring="bf16", filter_eps=eps)
    assert torch.equal(ids2, ids) and torch.equal(sims2, sims)
