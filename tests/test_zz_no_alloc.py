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
    # host stats or a host start_depth are rejected like host queries
    Qd4 = Qd[:4]
    host_stats = np.zeros((4, pf.STATS_DTYPE.itemsize), np.uint8)
    st = lib.pf_index_search_noalloc(index._h, Qd4.data_ptr(), 4, k.data_ptr(), rec.data_ptr(), 10,
                                     ids.data_ptr(), sims.data_ptr(), host_stats.ctypes.data, None, None)
    assert st == -1 and b"stats must be device memory" in lib.pf_last_error_message()
    host_start = np.zeros(4, np.int32)
    o = pf.SearchOpts()
    lib.pf_search_opts_default(C.byref(o))
    o.start_depth = host_start.ctypes.data
    st = lib.pf_index_search_noalloc(index._h, Qd4.data_ptr(), 4, k.data_ptr(), rec.data_ptr(), 10,
                                     ids.data_ptr(), sims.data_ptr(), None, C.byref(o), None)
    assert st == -1 and b"start_depth must be device memory" in lib.pf_last_error_message()
    o.start_depth = None
    o.learned_start = 1
    st = lib.pf_index_search_noalloc(index._h, Qd4.data_ptr(), 4, k.data_ptr(), rec.data_ptr(), 10,
                                     ids.data_ptr(), sims.data_ptr(), None, C.byref(o), None)
    assert st == -1 and b"learned start" in lib.pf_last_error_message()


def test_noalloc_allocates_nothing(index):
    Qs = datagen.vmf_mixture(200, 100, 50, 50.0, seed=12, purpose="queries")
    Qd = torch.from_numpy(Qs).to(DEV)
    k = torch.full((200,), 10, dtype=torch.int32, device=DEV)
    rec = torch.full((200,), 0.9, dtype=torch.float64, device=DEV)
    _noalloc(index, Qd, k, rec, 10, "bf16")  # the first call looks up the array's address
    outs = [torch.empty((200, 10), dtype=torch.int32, device=DEV), torch.empty((200, 10), device=DEV),
            torch.zeros((200, pf.STATS_DTYPE.itemsize), dtype=torch.uint8, device=DEV)]
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    o = pf.SearchOpts()
    pf.lib().pf_search_opts_default(C.byref(o))
    for _ in range(3):
        st = pf.lib().pf_index_search_noalloc(index._h, Qd.data_ptr(), 200, k.data_ptr(), rec.data_ptr(), 10,
                                              outs[0].data_ptr(), outs[1].data_ptr(), outs[2].data_ptr(),
                                              C.byref(o), torch.cuda.current_stream().cuda_stream)
        assert st == 0, pf.lib().pf_last_error_message()
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before


def test_noalloc_with_wide_rows():
    """d = 150 (d' = 160 > 128): the hashing kernel takes one point tile per
    unit and two N tiles per function, with near-boundary decisions rechecked
    inline (the no-alloc call has no recheck queue)."""
    pf.build()
    X = datagen.vmf_mixture(6_000, 150, 30, 50.0, seed=21)
    ix = pf.Index(torch.from_numpy(X).to(DEV), "crosspolytope", num_tables=12, seed=5)
    try:
        Qd = torch.from_numpy(datagen.vmf_mixture(120, 150, 30, 50.0, seed=21, purpose="queries")).to(DEV)
        k = torch.full((120,), 10, dtype=torch.int32, device=DEV)
        rec = torch.full((120,), 0.9, dtype=torch.float64, device=DEV)
        ref_ids, ref_sims, ref_st = ix.search(Qd, k, rec, k_max=10, scoring="bf16", stats=True)
        for _ in range(2):
            ids, sims, st = _noalloc(ix, Qd, k, rec, 10, "bf16")
            assert torch.equal(ids, ref_ids) and torch.equal(sims, ref_sims) and torch.equal(st, ref_st)
    finally:
        ix.close()


def test_noalloc_reports_and_clears_a_device_time_out(index):
    """A no-alloc call whose hashing waits expire returns PF_ERR_DEVICE_TIMEOUT
    and clears the index's error word, so the next call succeeds and again
    equals pf_index_search."""
    Qs = datagen.vmf_mixture(64, 100, 50, 50.0, seed=13, purpose="queries")
    Qd = torch.from_numpy(Qs).to(DEV)
    k = torch.full((64,), 10, dtype=torch.int32, device=DEV)
    rec = torch.full((64,), 0.9, dtype=torch.float64, device=DEV)
    ref_ids, ref_sims, _ = index.search(Qd, k, rec, k_max=10, scoring="bf16", stats=True)
    ids = torch.empty((64, 10), dtype=torch.int32, device=DEV)
    sims = torch.empty((64, 10), dtype=torch.float32, device=DEV)
    o = pf.SearchOpts()
    pf.lib().pf_search_opts_default(C.byref(o))
    o.scoring = 1
    index.selftest_hold(True)
    try:
        st = pf.lib().pf_index_search_noalloc(index._h, Qd.data_ptr(), 64, k.data_ptr(), rec.data_ptr(), 10,
                                              ids.data_ptr(), sims.data_ptr(), None, C.byref(o),
                                              torch.cuda.current_stream().cuda_stream)
    finally:
        index.selftest_hold(False)
    assert st == -5, pf.lib().pf_last_error_message()  # PF_ERR_DEVICE_TIMEOUT
    for _ in range(2):
        ids2, sims2, _ = _noalloc(index, Qd, k, rec, 10, "bf16")
        assert torch.equal(ids2, ref_ids) and torch.equal(sims2, ref_sims)
