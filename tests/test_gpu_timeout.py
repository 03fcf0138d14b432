"""The bounded waits of the tensor-core hashing kernel: with its weight-tile
loads withheld (pf_index_selftest_timeout), every wait on them gives up after
about a second, the call returns PF_ERR_DEVICE_TIMEOUT, and the index and the
CUDA context stay usable: later hashing and searches give the results they gave
before.  Nothing faults or hangs: the waits end by themselves."""
import time

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
def idx():
    pf.build()
    X = datagen.vmf_mixture(20_000, 100, 50, 50.0, seed=31)
    Qs = datagen.vmf_mixture(300, 100, 50, 50.0, seed=31, purpose="queries")
    ix = pf.Index(torch.from_numpy(X).to(DEV), "crosspolytope", num_tables=30, seed=4)
    return ix, torch.from_numpy(Qs).to(DEV), Qs


def test_withheld_loads_time_out_and_the_index_stays_usable(idx):
    ix, qd, qh = idx
    before = ix.search(qd, 10, 0.9, scoring="bf16", stats=True)
    codes_before = ix.hash_queries(qd)
    t = time.perf_counter()
    with pytest.raises(pf.PuffinnError) as e:
        ix.selftest_timeout(qd)
    el = time.perf_counter() - t
    assert e.value.status == -5  # PF_ERR_DEVICE_TIMEOUT
    assert 0.9 <= el < 30.0, el  # the waits gave up after their 1 s bound
    # the error word was cleared: the next calls succeed and agree with the earlier ones
    codes_after = ix.hash_queries(qd)
    for a, b in zip(codes_before, codes_after):
        assert torch.equal(a, b)
    after = ix.search(qd, 10, 0.9, scoring="bf16", stats=True)
    for a, b in zip(before, after):
        assert torch.equal(a, b)
    # host queries take the same path
    with pytest.raises(pf.PuffinnError) as e:
        ix.selftest_timeout(np.ascontiguousarray(qh[:64]))
    assert e.value.status == -5
    torch.cuda.synchronize()


def test_one_point_tile_per_unit_times_out_too():
    """d = 150 (d' = 160 > 128): one point tile per work unit and CP functions
    of two N tiles; the withheld loads time out there as well."""
    pf.build()
    X = datagen.vmf_mixture(3_000, 150, 20, 50.0, seed=2)
    ix = pf.Index(torch.from_numpy(X).to(DEV), "crosspolytope", num_tables=4, seed=1)
    q = torch.from_numpy(X[:10]).to(DEV)
    before = ix.hash_queries(q)
    with pytest.raises(pf.PuffinnError) as e:
        ix.selftest_timeout(q)
    assert e.value.status == -5
    for a, b in zip(before, ix.hash_queries(q)):
        assert torch.equal(a, b)
    torch.cuda.synchronize()
