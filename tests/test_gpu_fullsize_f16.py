"""The 10M-point workload with binary16 rows at full size (n = 10,000,000,
d = 96, 10,000-component vMF mixture with kappa = 100, 40 GiB index), checked
on samples the oracle computes one by one and on properties that hold at any
size: the budget's L, stored rows, hash codes and sketches of sampled points,
canonical similarities of returned points, Lemma 1 at the stop depth, and
recall >= 1 - delta over a 1,000-query batch."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1906_12211_gb300 as pf  # noqa: E402

DEV = torch.device("cuda:0")
N, D, COMP, KAPPA, BUDGET, Q, K, RECALL = 10_000_000, 96, 10_000, 100.0, 40 << 30, 1000, 10, 0.9


@pytest.fixture(scope="module")
def big(orc):
    pf.build()
    X = datagen.vmf_mixture(N, D, COMP, KAPPA, seed=0, purpose="points")
    Qs = datagen.vmf_mixture(Q, D, COMP, KAPPA, seed=0, purpose="queries")
    Xd = torch.from_numpy(X).to(DEV)
    ix = pf.Index(Xd, "crosspolytope", budget_bytes=BUDGET, seed=0, rows="f16")
    assert ix.L == orc.budget_L(orc.CROSSPOLYTOPE, N, D, 32, BUDGET, 0, 1) == 244
    return {"X": X, "Q": Qs, "Xd": Xd, "Qd": torch.from_numpy(Qs).to(DEV), "ix": ix}


def test_sampled_rows_codes_and_sketches_equal_oracle(big, orc):
    ix = big["ix"]
    rng = np.random.default_rng(11)
    sample = np.sort(rng.choice(N, 200, replace=False))
    xn = orc.round_rows_f16(orc.normalize(big["X"][sample]))
    rows = ix.array("rows_f16").view(torch.float16).reshape(N, ix.d_pad)
    got = rows[torch.from_numpy(sample).to(DEV).long()][:, :D].float().cpu().numpy()
    assert np.array_equal(got, xn)
    A = orc.gen_hash_params(0, orc.CROSSPOLYTOPE, ix.L, D)
    S = orc.gen_sketch_params(0, ix.M, D)
    want_codes = orc.hash_codes(orc.CROSSPOLYTOPE, A, xn)
    want_sk = orc.sketches(S, xn)
    codes = ix.array("codes").view(torch.int32).reshape(ix.L, N)
    ids = ix.array("ids").view(torch.int32).reshape(ix.L, N)
    sd = torch.from_numpy(sample).to(DEV).long()
    # position of each sampled point in every repetition
    pos = torch.empty((ix.L, len(sample)), dtype=torch.int64, device=DEV)
    for j in range(ix.L):
        inv = torch.empty(N, dtype=torch.int64, device=DEV)
        inv[ids[j].long()] = torch.arange(N, device=DEV)
        pos[j] = inv[sd]
    got_codes = torch.gather(codes, 1, pos).cpu().numpy().view(np.uint32)
    assert np.array_equal(got_codes, want_codes)
    skc = ix.array("table_sketches").view(torch.int64).reshape(ix.L, N)
    got_sk = torch.gather(skc, 1, pos).cpu().numpy().view(np.uint64)
    assert np.array_equal(got_sk, want_sk[np.arange(ix.L) % ix.M])


def test_search_canonical_stop_rule_and_recall(big, orc):
    ix = big["ix"]
    ids, sims, st = ix.search(big["Qd"], K, RECALL, scoring="bf16", stats=True)
    ids_n = ids.cpu().numpy().view(np.uint32)
    sims_n = sims.cpu().numpy()
    stn = pf.stats_to_numpy(st)
    P = orc.cp_table(0, D)
    ell = orc.layout(orc.CROSSPOLYTOPE, D)["ell"]
    rng = np.random.default_rng(2)
    for t in rng.choice(Q, 48, replace=False):
        assert len(set(ids_n[t].tolist())) == K and ids_n[t].max() < N
        qn = orc.normalize(big["Q"][t:t + 1])[0]
        xn = orc.round_rows_f16(orc.normalize(big["X"][ids_n[t]]))
        for u in range(K):
            assert sims_n[t, u] == orc.sim(qn, xn[u])
        dstop = int(stn["stop_depth"][t])
        if dstop > 0:
            p = orc.collision_prob(orc.CROSSPOLYTOPE, ell, P, float(sims_n[t, K - 1]), dstop)
            assert orc.ipow(1.0 - p, ix.L) <= (1 - RECALL) * (1 + 1e-12)
    # recall against brute force over the stored (binary16) rows
    rows = ix.array("rows_f16").view(torch.float16).reshape(N, ix.d_pad)[:, :D]
    Qn = torch.nn.functional.normalize(big["Qd"], dim=1)
    kth = []
    for s in range(0, Q, 100):
        best = None
        for c in range(0, N, 2_000_000):
            blk = (Qn[s:s + 100] @ rows[c:c + 2_000_000].float().T).topk(K, dim=1).values
            best = blk if best is None else torch.cat([best, blk], 1).topk(K, dim=1).values
        kth.append(best[:, -1])
    kth = torch.cat(kth)
    rec = float((sims >= kth[:, None] - 1e-6).float().mean().item())
    assert rec >= RECALL - 3 * np.sqrt(RECALL * (1 - RECALL) / (Q * K)), rec
    # bf16 estimates change no result
    ids2, sims2, _ = ix.search(big["Qd"], K, RECALL, scoring="fp32", stats=True)
    assert torch.equal(ids, ids2) and torch.equal(sims, sims2)
