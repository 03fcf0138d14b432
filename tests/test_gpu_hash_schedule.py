"""The tensor-core hashing kernel's work schedule: with more groups of point
tiles than CTAs, the CTAs first take whole groups round robin (all segments of
each, walking the hash rows in step) and split the remaining groups' units
evenly.  Both phases must give the oracle's codes and sketches: 40,000 points
are 157 pairs of point tiles at d' = 112 (one round of 152 pairs, then five
pairs split by segments) and 313 single tiles at d' = 160 (two rounds, then
nine); the parity cases elsewhere are too small for the first phase."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1906_12211_gb300 as pf  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.mark.parametrize("d,family", [(100, "crosspolytope"), (150, "crosspolytope"), (100, "simhash")])
def test_round_robin_and_tail_phases_equal_the_oracle(orc, d, family):
    pf.build()
    X = datagen.vmf_mixture(40_000, d, 200, 30.0, seed=d)
    ix = pf.Index(torch.from_numpy(X).to(DEV), family, num_tables=3, seed=7)
    try:
        o = orc.OracleIndex(X, orc.CROSSPOLYTOPE if family == "crosspolytope" else orc.SIMHASH, L=ix.L, seed=7)
        codes = ix.array("codes").cpu().numpy().view(np.uint32).reshape(ix.L, ix.n)
        ids = ix.array("ids").cpu().numpy().view(np.uint32).reshape(ix.L, ix.n)
        assert np.array_equal(codes, o.codes)
        assert np.array_equal(ids, o.ids)
        skc = ix.array("table_sketches").cpu().numpy().view(np.uint64).reshape(ix.L, ix.n)
        ref = np.stack([o.sk[j % ix.M][o.ids[j]] for j in range(ix.L)])
        assert np.array_equal(skc, ref)
        # a query batch this size goes through both phases as well
        Qs = datagen.vmf_mixture(40_000, d, 200, 30.0, seed=d, purpose="queries")
        qc, qs = ix.hash_queries(torch.from_numpy(Qs).to(DEV))
        _, oqc, oqs = o.hash_queries(Qs)
        assert np.array_equal(qc.cpu().numpy().view(np.uint32), oqc)
        assert np.array_equal(qs.cpu().numpy().view(np.uint64), oqs)
    finally:
        ix.close()
