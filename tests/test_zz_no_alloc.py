"""pf_index_search_noalloc: the search entry point for callers that cannot
allocate device memory while they run (their device memory is reserved up
front by another allocator, or an allocation's latency or failure is not
acceptable on their path).  It must return exactly what pf_index_search
returns, call after call, although its scratch lives in one fixed device
array that keeps the previous call's contents.

This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1906_12211_gb300 as pf  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def index():
    pf.build()
    X = datagen.vmf_mixture(20_000, 100, 50, 50.0, seed=11)
    ix = pf.Index(torch.from_numpy(X).to(DEV), "crosspolytope", num_tables=40, seed=3)
    yield ix
    ix.close()


def _noalloc(ix, Qd, k, rec, k_max, scoring):
    Q = Qd.shape[0]
    ids = torch.full((Q, k_max), -7, dtype=torch.int32, device=DEV)
    sims = torch.full((Q, k_max), 3.0, dtype=torch.float32, device=DEV)
    st = torch.zeros((Q, pf.STATS_DTYPE.itemsize), dtype=torch.uint8, device=DEV)
    o = pf.SearchOpts()
    pf.lib().pf_search_opts_default(C.byref(o))
    o.scoring = 1 if scoring == "bf16" else 0
    status = pf.lib().pf_index_search_noalloc(ix._h, Qd.data_ptr(), Q, k.data_ptr(), rec.data_ptr(), k_max,
                                              ids.data_ptr(), sims.data_ptr(), st.data_ptr(), C.byref(o),
                                              torch.cuda.current_stream().cuda_stream)
    assert status == 0, pf.lib().pf_last_error_message()
    return ids, sims, st


@pytest.mark.parametrize("scoring", ["fp32", "bf16"])
def test_noalloc_matches_search_on_consecutive_calls(index, scoring):
    Qs = datagen.vmf_mixture(300, 100, 50, 50.0, seed=11, purpose="queries")
    Qd = torch.from_numpy(Qs).to(DEV)
    kk, rr = datagen.mixed_k_recall(300, ks=(1, 10, 32), deltas=(0.5, 0.1), seed=2)
    k = torch.from_numpy(kk).to(DEV)
    rec = torch.from_numpy(rr).to(DEV)
    ref_ids, ref_sims, ref_st = index.search(Qd, k, rec, k_max=32, scoring=scoring, stats=True)
    for _ in range(2):  # the second call sees the first call's leftovers in the scratch
        ids, sims, st = _noalloc(index, Qd, k, rec, 32, scoring)
        assert torch.equal(ids, ref_ids)
        assert torch.equal(sims, ref_sims)  # bit-exact, the tolerance of every search parity test
        assert torch.equal(st, ref_st)
    # a smaller batch after a larger one
    ids, sims, _ = _noalloc(index, Qd[:17], k[:17], rec[:17], 32, scoring)
    assert torch.equal(ids, ref_ids[:17]) and torch.equal(sims, ref_sims[:17])


def test_noalloc_rejects_what_it_cannot_serve(index):
    lib = pf.lib()
    Qd = torch.zeros((50_000, 100), dtype=torch.float32, device=DEV)  # needs > 32 MiB of scratch
    k = torch.full((50_000,), 10, dtype=torch.int32, device=DEV)
    rec = torch.full((50_000,), 0.9, dtype=torch.float64, device=DEV)
    ids = torch.empty((50_000, 10), dtype=torch.int32, device=DEV)
    sims = torch.empty((50_000, 10), dtype=torch.float32, device=DEV)
    st = lib.pf_index_search_noalloc(index._h, Qd.data_ptr(), 50_000, k.data_ptr(), rec.data_ptr(), 10,
                                     ids.data_ptr(), sims.data_ptr(), None, None, None)
    assert st == -1 and b"32 MiB" in lib.pf_last_error_message()
    host_q = np.zeros((4, 100), np.float32)
    st = lib.pf_index_search_noalloc(index._h, host_q.ctypes.data, 4, k.data_ptr(), rec.data_ptr(), 10,
                                     ids.data_ptr(), sims.data_ptr(), None, None, None)
    assert st == -1 and b"device memory" in lib.pf_last_error_message()
