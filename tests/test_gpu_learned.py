"""Learned start depth on the GPU: the perceptron's training kernels against
the float64 CPU oracle, and the trained model's effect on the search (same
results as the oracle at the predicted start depths, fewer rounds than the
plain schedule, recall kept)."""
import numpy as np
import pytest

import datagen
from oracle import mlp as mlp_oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1906_12211_gb300 as pf  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.mark.parametrize("B,F,H,C", [(300, 176, 256, 33), (37, 20, 256, 5), (1024, 128, 256, 29)])
def test_mlp_gradients_match_float64_oracle(B, F, H, C):
    pf.build()
    rng = np.random.default_rng(B + F)
    X = rng.standard_normal((B, F)).astype(np.float32)
    y = rng.integers(0, C, B).astype(np.int32)
    W1 = (rng.standard_normal((H, F)) * np.sqrt(2.0 / F)).astype(np.float32)
    b1 = (rng.standard_normal(H) * 0.1).astype(np.float32)
    W2 = (rng.standard_normal((C, H)) * np.sqrt(1.0 / H)).astype(np.float32)
    b2 = (rng.standard_normal(C) * 0.1).astype(np.float32)
    t = [torch.from_numpy(a).to(DEV) for a in (X, y, W1, b1, W2, b2)]
    loss, dW1, db1, dW2, db2 = pf.mlp_forward_backward(*t)
    ref = mlp_oracle.loss_and_grads(X, y, W1, b1, W2, b2)
    assert abs(loss.item() - ref[0]) <= 1e-5 * max(1.0, abs(ref[0]))
    for got, want in zip((dW1, db1, dW2, db2), ref[1:]):
        g = got.cpu().numpy().astype(np.float64)
        # float32 sums of up to B*F terms: tolerance relative to the gradient's scale
        assert np.max(np.abs(g - want)) <= 2e-5 * max(1e-3, np.max(np.abs(want))), (np.max(np.abs(g - want)),)


@pytest.fixture(scope="module")
def trained(orc):
    pf.build()
    X = datagen.vmf_mixture(20_000, 100, 50, 50.0, seed=21)
    Qtrain = datagen.vmf_mixture(4000, 100, 50, 50.0, seed=21, purpose="train")
    Qtest = datagen.vmf_mixture(300, 100, 50, 50.0, seed=21, purpose="queries")
    ix = pf.Index(torch.from_numpy(X).to(DEV), "crosspolytope", num_tables=40, seed=8)
    rep = ix.learned_train(torch.from_numpy(Qtrain).to(DEV), 10, 0.9, epochs=30, seed=3)
    o = orc.OracleIndex(X, orc.CROSSPOLYTOPE, L=40, seed=8)
    return ix, o, rep, X, Qtest


def test_training_report(trained):
    ix, _, rep, _, _ = trained
    assert rep["samples"] == 4000 and rep["epochs"] == 30
    assert np.isfinite(rep["final_loss"]) and rep["final_loss"] < np.log(ix.Kb + 1)
    assert rep["train_accuracy"] >= 0.8  # predicted quantile at or deeper than the stop depth
    assert rep["mean_start"] >= rep["mean_stop"]


def test_learned_search_equals_oracle_at_predicted_depths(trained):
    ix, o, _, _, Q = trained
    qd = torch.from_numpy(Q).to(DEV)
    sd = ix.learned_predict(qd)
    ids, sims, st = ix.search(qd, 10, 0.9, learned=True, stats=True)
    ref = o.search(Q, 10, 0.9, start_depth=sd.cpu().numpy())
    assert np.array_equal(ids.cpu().numpy().view(np.uint32), ref["ids"])
    assert np.array_equal(sims.cpu().numpy(), ref["sims"])
    g = pf.stats_to_numpy(st)
    assert np.array_equal(g["stop_depth"], ref["stats"]["stop_depth"])
    assert np.array_equal(g["start_depth"], ref["stats"]["start_depth"])


def test_learned_start_saves_rounds_and_keeps_recall(trained, orc):
    ix, o, _, X, Q = trained
    qd = torch.from_numpy(Q).to(DEV)
    _, sp, stp = ix.search(qd, 10, 0.9, stats=True, filter=False)
    _, sl, stl = ix.search(qd, 10, 0.9, stats=True, filter=False, learned=True)
    gp, gl = pf.stats_to_numpy(stp), pf.stats_to_numpy(stl)
    assert gl["rounds"].mean() <= gp["rounds"].mean() - 2.0
    qn = orc.normalize(Q)
    _, bs = orc.brute_force(o.x, qn, 10)
    rec_plain = float(np.mean(sp.cpu().numpy() >= bs[:, -1:]))
    rec_learned = float(np.mean(sl.cpu().numpy() >= bs[:, -1:]))
    # Lemma 1 holds for any start depth: recall >= 1 - delta up to sampling noise
    assert rec_learned >= 0.9 - 3 * np.sqrt(0.09 / 3000)
    assert rec_plain >= 0.9 - 3 * np.sqrt(0.09 / 3000)


def test_not_trained_is_an_error():
    pf.build()
    g = pf.Index(torch.randn(500, 16, device=DEV), "simhash", num_tables=4)
    with pytest.raises(pf.PuffinnError) as e:
        g.search(torch.randn(3, 16, device=DEV), 5, 0.9, learned=True)
    assert e.value.status == -6


def test_predict_forward_equals_float64_oracle(trained, orc):
    """The bfloat16 inference kernel against the float64 forward of oracle/mlp.py
    run with the same rounded weights: features = the normalised query (zero
    padded to d_pad) and the 64 bits of its sketch 0 as +-1.  Start depths agree
    except where the predicted tail mass sits within float32 rounding of the
    0.05 threshold."""
    ix, o, _, _, Q = trained
    qd = torch.from_numpy(Q).to(DEV)
    got = ix.learned_predict(qd).cpu().numpy()
    F, H, C = ix.d_pad + 64, 256, ix.Kb + 1
    w32 = ix.array("mlp_f32", device="cpu").numpy().view(np.float32)
    assert w32.size == H * F + H + C * H + C
    b1 = w32[H * F:H * F + H].astype(np.float64)
    b2 = w32[H * F + H + C * H:].astype(np.float64)
    bf = lambda name, shape: (ix.array(name, device="cpu").view(torch.bfloat16).float().numpy()
                              .astype(np.float64).reshape(shape))
    W1 = bf("mlp_w1_bf16", (F, H)).T  # stored transposed
    W2 = bf("mlp_w2_bf16", (C, H))
    # the rounded weights are the float32 master weights rounded to nearest even
    W1_32 = w32[:H * F].reshape(H, F)
    assert np.array_equal(W1, torch.from_numpy(W1_32).to(torch.bfloat16).float().numpy().astype(np.float64))
    qn, _, qsk = o.hash_queries(Q)
    X = np.zeros((Q.shape[0], F))
    X[:, :ix.d] = qn
    bits = (qsk[:, 0][:, None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1)
    X[:, ix.d_pad:] = np.where(bits == 1, 1.0, -1.0)
    want, A = mlp_oracle.start_depths(X, W1, b1, W2, b2, 0.05, 0)  # the default rule
    near = np.any(np.abs(A - 0.05) < 1e-4, axis=1)
    assert np.all((got == want) | near), np.nonzero((got != want) & ~near)
    assert np.mean(got == want) >= 0.98


def test_start_rule_moves_the_start_and_keeps_the_results_equal_to_the_oracle(trained):
    """A larger margin starts earlier in the schedule's order (a longer prefix,
    capped at K): the search still equals the oracle at the predicted depths."""
    ix, o, _, _, Q = trained
    qd = torch.from_numpy(Q).to(DEV)
    base = ix.learned_predict(qd).cpu().numpy()
    try:
        ix.learned_start_rule(0.05, 3)
        high = ix.learned_predict(qd).cpu().numpy()
        assert np.all(high >= base) and np.any(high > base)
        assert np.all((high == np.minimum(base + 3, ix.Kb)) | (high == ix.Kb))
        ids, sims, st = ix.search(qd, 10, 0.9, learned=True, stats=True)
        ref = o.search(Q, 10, 0.9, start_depth=high)
        assert np.array_equal(ids.cpu().numpy().view(np.uint32), ref["ids"])
        assert np.array_equal(sims.cpu().numpy(), ref["sims"])
        with pytest.raises(pf.PuffinnError):
            ix.learned_start_rule(1.5, 2)
    finally:
        ix.learned_start_rule(0.05, 0)
