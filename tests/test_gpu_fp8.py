"""Scoring with an 8-bit float (e4m3) copy of the rows and a per-row scale:
the estimate only drops candidates whose bound proves they cannot enter the
top-k, and the float32 rerank decides, so the results equal the oracle's
float32 search bit for bit.  The stored codes are checked against an
independent e4m3 rounding in numpy, and the per-row bound against the float64
error of the estimate for sampled query-point pairs."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1906_12211_gb300 as pf  # noqa: E402

DEV = torch.device("cuda:0")


def e4m3_decode(c):
    """float64 value of e4m3 codes (1 sign, 4 exponent bits with bias 7, 3
    mantissa bits; exponent 0 is subnormal)."""
    c = c.astype(np.int64)
    s = np.where(c & 0x80, -1.0, 1.0)
    e = (c >> 3) & 0xF
    m = c & 0x7
    return s * np.where(e == 0, m / 8.0 * 2.0 ** -6, (1 + m / 8.0) * 2.0 ** (e - 7.0))


def e4m3_round(v):
    """Nearest e4m3 value of float64 v, ties to the even code, saturated to
    +-448 (the largest finite value)."""
    codes = np.arange(256)
    keep = ((codes & 0x7F) != 0x7F) & (codes != 0x80)  # no NaN codes, one zero
    vals, cds = e4m3_decode(codes[keep]), codes[keep]
    order = np.argsort(vals)
    vals, cds = vals[order], cds[order]
    v = np.clip(v, -448.0, 448.0)
    idx = np.clip(np.searchsorted(vals, v), 1, len(vals) - 1)
    lo, hi = vals[idx - 1], vals[idx]
    dlo, dhi = v - lo, hi - v
    pick_hi = (dhi < dlo) | ((dhi == dlo) & ((cds[idx] & 1) == 0))
    return np.where(pick_hi, hi, lo)


@pytest.fixture(scope="module", params=[("vmf", 100, "crosspolytope"), ("gauss", 64, "simhash"),
                                        ("vmf", 37, "crosspolytope"), ("vmf", 300, "crosspolytope")])
def case(request, orc):
    pf.build()
    kind, d, fam = request.param
    if kind == "vmf":
        X = datagen.vmf_mixture(20_000, d, 50, 50.0, seed=d)
        Q = datagen.vmf_mixture(150, d, 50, 50.0, seed=d, purpose="queries")
    else:
        X = datagen.gaussian(10_000, d, seed=0)
        Q = datagen.gaussian(100, d, seed=0, purpose="queries")
    L = 30
    g = pf.Index(torch.from_numpy(X).to(DEV), fam, num_tables=L, seed=7, fp8_rows=True)
    o = orc.OracleIndex(X, orc.SIMHASH if fam == "simhash" else orc.CROSSPOLYTOPE, L=L, seed=7)
    return g, o, X, Q


@pytest.mark.parametrize("filt", [True, False])
def test_fp8_scoring_equals_oracle(case, filt):
    g, o, _, Q = case
    ref = o.search(Q, 10, 0.9, filter=filt)
    ids, sims, st = g.search(torch.from_numpy(Q).to(DEV), 10, 0.9, scoring="fp8", filter=filt, stats=True)
    assert np.array_equal(ids.cpu().numpy().view(np.uint32), ref["ids"])
    assert np.array_equal(sims.cpu().numpy(), ref["sims"])
    gs = pf.stats_to_numpy(st)
    assert np.array_equal(gs["stop_depth"], ref["stats"]["stop_depth"])
    deep = ref["stats"]["stop_depth"] > 0
    assert np.array_equal(gs["scored"][deep], ref["stats"]["scored"][deep])
    assert np.all(gs["reranked"] <= gs["scored"]) and gs["reranked"].sum() > 0


def test_mixed_k_and_start_depths_with_fp8(case):
    g, o, _, Q = case
    k, rec = datagen.mixed_k_recall(Q.shape[0], ks=(1, 10, 50), seed=3)
    sd = np.random.default_rng(1).integers(0, g.Kb + 1, Q.shape[0]).astype(np.int32)
    ref = o.search(Q, k, rec, k_max=50, start_depth=sd)
    ids, sims, _ = g.search(torch.from_numpy(Q).to(DEV), torch.from_numpy(k).to(DEV), torch.from_numpy(rec).to(DEV),
                            k_max=50, scoring="fp8", start_depth=torch.from_numpy(sd).to(DEV), stats=True)
    assert np.array_equal(ids.cpu().numpy().view(np.uint32), ref["ids"])
    assert np.array_equal(sims.cpu().numpy(), ref["sims"])


def test_codes_scales_and_bounds(case, orc):
    g, o, X, Q = case
    n, dp, d = X.shape[0], g.d_pad, X.shape[1]
    codes = g.array("rows_fp8", device="cpu").numpy().reshape(n, dp)
    meta = g.array("fp8_meta", device="cpu").numpy().view(np.float32).reshape(n, 2)
    xn = o.x.astype(np.float64)  # the oracle's normalised rows (bit-equal to the library's)
    scale = np.where(np.abs(xn).max(axis=1) > 0, (np.abs(xn).max(axis=1).astype(np.float32) / np.float32(448)), 1.0)
    assert np.array_equal(meta[:, 0], scale.astype(np.float32))
    rng = np.random.default_rng(0)
    rows = rng.choice(n, 2000, replace=False)
    dec = e4m3_decode(codes[rows, :d])
    # the library divides in float32 and rounds that quotient
    q32 = (o.x[rows].astype(np.float32) / meta[rows, 0:1]).astype(np.float64)
    assert np.array_equal(dec, e4m3_round(q32)), np.argwhere(dec != e4m3_round(q32))[:5]
    assert np.all(codes[:, d:] == 0)
    # the bound covers the estimate's error for every sampled (query, point)
    qn = orc.normalize(Q).astype(np.float64)
    approx = meta[rows, 0:1].astype(np.float64) * dec  # [rows][d]
    for t in range(0, Q.shape[0], 10):
        exact = xn[rows] @ qn[t]
        est = approx @ qn[t]
        assert np.all(np.abs(exact - est) <= meta[rows, 1]), (t, np.max(np.abs(exact - est) - meta[rows, 1]))


def test_budget_counts_the_fp8_copy(orc):
    pf.build()
    X = datagen.vmf_mixture(20_000, 100, 30, 40.0, seed=3)
    g = pf.Index(torch.from_numpy(X).to(DEV), "crosspolytope", budget_bytes=256 << 20, seed=1, fp8_rows=True)
    assert g.L == orc.budget_L(orc.CROSSPOLYTOPE, 20_000, 100, 32, 256 << 20, 0, 0, 1)
    assert g.L < orc.budget_L(orc.CROSSPOLYTOPE, 20_000, 100, 32, 256 << 20, 0, 0, 0)
    assert g.info["bytes_used"] <= 256 << 20
    plain = pf.Index(torch.from_numpy(X[:100]).to(DEV), "crosspolytope", num_tables=2, seed=1)
    with pytest.raises(pf.PuffinnError):
        plain.search(torch.from_numpy(X[:4]).to(DEV), 5, 0.9, scoring="fp8")
