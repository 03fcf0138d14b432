"""The benchmark workload at full size (n = 1,000,000, d = 100, 4 GiB index,
10,000 queries, k = 10), in the launch configuration bench.py times.

The oracle cannot build a million-point index in a test's time, so the checks
are of two kinds: values the oracle computes one by one for a sample (hash codes
and sketches of sampled points from the oracle's own parameters, the CP table,
canonical similarities of returned points, the stop test of Lemma 1), and
properties that hold at any size (sorted stable tables, prefix tables, valid
unique ordered results, recall >= 1 - delta, bf16 == fp32, determinism)."""
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


@pytest.fixture(scope="module")
def full(orc):
    pf.build()
    X = datagen.vmf_mixture(W["n"], W["d"], W["components"], W["kappa"], seed=0, purpose="points")
    Q = datagen.vmf_mixture(W["Q"], W["d"], W["components"], W["kappa"], seed=0, purpose="queries")
    Xd = torch.from_numpy(X).to(DEV)
    ix = pf.Index(Xd, "crosspolytope", budget_bytes=W["budget"], seed=0)
    assert ix.L == orc.budget_L(orc.CROSSPOLYTOPE, W["n"], W["d"], 32, W["budget"], 0)
    return {"X": X, "Q": Q, "Xd": Xd, "Qd": torch.from_numpy(Q).to(DEV), "ix": ix}


def _u32(t, shape):
    return t.view(torch.int32).reshape(shape)


@pytest.fixture(scope="module")
def tables(full):
    ix, n = full["ix"], W["n"]
    codes = _u32(full["ix"].array("codes"), (ix.L, n))
    ids = _u32(full["ix"].array("ids"), (ix.L, n))
    return codes, ids


def test_sampled_codes_and_sketches_equal_oracle(full, tables, orc):
    # Sec. 2.2 / 4.3: the code of point p in repetition j, from the oracle's own
    # Gaussian parameters and float64 decisions, for 256 sampled points
    ix, n = full["ix"], W["n"]
    rng = np.random.default_rng(7)
    sample = np.sort(rng.choice(n, 256, replace=False))
    A = orc.gen_hash_params(0, orc.CROSSPOLYTOPE, ix.L, W["d"])
    S = orc.gen_sketch_params(0, ix.M, W["d"])
    xn = orc.normalize(full["X"][sample])
    want_codes = orc.hash_codes(orc.CROSSPOLYTOPE, A, xn)  # [L][256]
    want_sk = orc.sketches(S, xn)  # [M][256]
    codes, ids = tables
    inv = torch.empty_like(ids)
    inv.scatter_(1, ids.long(), torch.arange(n, dtype=torch.int32, device=DEV).expand(ix.L, n).contiguous())
    sd = torch.from_numpy(sample).to(DEV).long()
    pos = inv[:, sd].long()  # [L][256] position of each sampled point
    got_codes = torch.gather(codes, 1, pos).cpu().numpy().view(np.uint32)
    assert np.array_equal(got_codes, want_codes)
    skc = full["ix"].array("table_sketches").view(torch.int64).reshape(ix.L, n)
    got_sk = torch.gather(skc, 1, pos).cpu().numpy().view(np.uint64)
    m = np.arange(ix.L) % ix.M
    assert np.array_equal(got_sk, want_sk[m])


def test_cp_table_equals_oracle(full, orc):
    got = full["ix"].array("cp_table", device="cpu").numpy().view(np.float64)
    assert np.array_equal(got, orc.cp_table(0, W["d"]).reshape(-1))


def test_tables_sorted_stable_and_prefix(full, tables):
    # Sec. 4.2: (code, pos) sorted per repetition, ties by position; every point
    # once per repetition; the 13-bit table gives the first position of a prefix
    ix, n = full["ix"], W["n"]
    codes, ids = tables
    c64 = codes.long() & 0xFFFFFFFF
    dc = c64[:, 1:] - c64[:, :-1]
    assert bool((dc >= 0).all())
    ties = dc == 0
    assert bool(((ids[:, 1:] > ids[:, :-1]) | ~ties).all())
    cnt = torch.zeros((ix.L, n), dtype=torch.int32, device=DEV)
    cnt.scatter_add_(1, ids.long(), torch.ones_like(ids))
    assert bool((cnt == 1).all())
    pfx = _u32(full["ix"].array("prefix"), (ix.L, 8193)).long() & 0xFFFFFFFF
    keys = (torch.arange(8193, device=DEV, dtype=torch.int64) << 19).expand(ix.L, 8193).contiguous()
    want = torch.searchsorted(c64.contiguous(), keys)
    assert torch.equal(pfx, want)


@pytest.fixture(scope="module")
def searched(full):
    ix, Qd, k = full["ix"], full["Qd"], W["k"]
    out = {}
    for mode in ("fp32", "bf16"):
        out[mode] = ix.search(Qd, k, W["recall"], scoring=mode, stats=True)
    Qt = datagen.vmf_mixture(100_000, W["d"], W["components"], W["kappa"], seed=0, purpose="train")
    ix.learned_train(torch.from_numpy(Qt).to(DEV), k, W["recall"], epochs=20, seed=0)
    out["learned"] = ix.search(Qd, k, W["recall"], scoring="bf16", learned=True, stats=True)
    return out


def test_bf16_equals_fp32_at_full_size(searched):
    a, b = searched["fp32"], searched["bf16"]
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    sa, sb = pf.stats_to_numpy(a[2]), pf.stats_to_numpy(b[2])
    for f in ("start_depth", "stop_depth", "rounds", "retrieved", "passed_filter", "scored"):
        assert np.array_equal(sa[f], sb[f]), f


@pytest.mark.parametrize("mode", ["fp32", "learned"])
def test_results_are_canonical_sorted_and_stop_rule_holds(full, searched, orc, mode):
    ix, k, delta = full["ix"], W["k"], 1.0 - W["recall"]
    ids, sims, st = searched[mode]
    ids = ids.cpu().numpy().view(np.uint32)
    sims = sims.cpu().numpy()
    st = pf.stats_to_numpy(st)
    P = orc.cp_table(0, W["d"])
    ell = orc.layout(orc.CROSSPOLYTOPE, W["d"])["ell"]
    rng = np.random.default_rng(3)
    for t in rng.choice(W["Q"], 64, replace=False):
        assert len(set(ids[t].tolist())) == k and ids[t].max() < W["n"]
        qn = orc.normalize(full["Q"][t:t + 1])[0]
        xn = orc.normalize(full["X"][ids[t]])
        for u in range(k):  # canonical float32 similarity (R16), recomputed by the oracle
            assert sims[t, u] == orc.sim(qn, xn[u])
        for u in range(1, k):  # (similarity desc, id asc)
            assert sims[t, u - 1] > sims[t, u] or (sims[t, u - 1] == sims[t, u] and ids[t, u - 1] < ids[t, u])
        dstop = int(st["stop_depth"][t])
        if dstop > 0:  # Lemma 1 at the stop depth, with the final k-th similarity
            p = orc.collision_prob(orc.CROSSPOLYTOPE, ell, P, float(sims[t, k - 1]), dstop)
            assert orc.ipow(1.0 - p, ix.L) <= delta * (1 + 1e-12)
    if mode == "learned":
        sd = st["start_depth"]
        assert np.all((sd >= 0) & (sd <= ix.Kb))
        part = sd < ix.Kb
        assert np.array_equal(st["rounds"][part], sd[part] - st["stop_depth"][part] + 1)


@pytest.mark.parametrize("mode", ["fp32", "learned"])
def test_recall_at_least_one_minus_delta(full, searched, mode):
    # Definition 1: each true neighbour is reported with probability >= 1 - delta;
    # brute force by a float32 matmul (ties within 1e-6 count as found)
    k = W["k"]
    Xn = torch.nn.functional.normalize(full["Xd"], dim=1)
    Qn = torch.nn.functional.normalize(full["Qd"], dim=1)
    kth = torch.cat([(Qn[s:s + 1024] @ Xn.T).topk(k, dim=1).values[:, -1] for s in range(0, W["Q"], 1024)])
    sims = searched[mode][1]
    rec = float((sims >= kth[:, None] - 1e-6).float().mean().item())
    n_trials = W["Q"] * k
    assert rec >= W["recall"] - 3 * np.sqrt(W["recall"] * (1 - W["recall"]) / n_trials), rec


def test_deterministic(full, searched):
    again = full["ix"].search(full["Qd"], W["k"], W["recall"], scoring="bf16", learned=True, stats=True)
    ref = searched["learned"]
    assert torch.equal(again[0], ref[0]) and torch.equal(again[1], ref[1]) and torch.equal(again[2], ref[2])
