"""The per-repetition sort (Sec. 4.2: sorted (code, position) arrays and the
13-bit prefix table) against the oracle, bit for bit, on points whose codes
crowd into few values: 6,000 or 1,500 copies of one point and 1,500 / 700 / 900
of another among 12,000 others, so long runs of equal codes must keep their
position order (the stable order) and the prefix table has very large
buckets."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1906_12211_gb300 as pf  # noqa: E402

DEV = torch.device("cuda:0")


def _points(copies_a, copies_b, n_rand, d, seed):
    X = datagen.gaussian(n_rand + 2, d, seed=seed)
    rows = [np.repeat(X[:1], copies_a, axis=0), np.repeat(X[1:2], copies_b, axis=0), X[2:]]
    P = np.concatenate(rows)
    perm = np.random.default_rng(seed).permutation(P.shape[0])  # the copies spread over the positions
    return np.ascontiguousarray(P[perm])


@pytest.mark.parametrize("copies_a,copies_b,family", [
    (6000, 1500, "crosspolytope"),
    (1500, 700, "crosspolytope"),
    (1500, 900, "simhash"),
])
def test_sorted_tables_equal_the_oracle(orc, copies_a, copies_b, family):
    pf.build()
    X = _points(copies_a, copies_b, 12_000, 48, seed=copies_a + copies_b)
    ix = pf.Index(torch.from_numpy(X).to(DEV), family, num_tables=5, seed=3)
    try:
        o = orc.OracleIndex(X, orc.CROSSPOLYTOPE if family == "crosspolytope" else orc.SIMHASH, L=ix.L, seed=3)
        codes = ix.array("codes").cpu().numpy().view(np.uint32).reshape(ix.L, ix.n)
        ids = ix.array("ids").cpu().numpy().view(np.uint32).reshape(ix.L, ix.n)
        pfx = ix.array("prefix").cpu().numpy().view(np.uint32).reshape(ix.L, 8193)
        assert np.array_equal(codes, o.codes)
        assert np.array_equal(ids, o.ids)
        assert np.array_equal(pfx, o.pfx)
        # the copies share one code in every repetition
        assert np.all(np.diff(pfx, axis=1).max(axis=1) >= copies_a)
    finally:
        ix.close()
