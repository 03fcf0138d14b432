"""The measurement arithmetic of bench.py on the CPU: the per-query byte count
behind `roofline` (written out term by term here from its definition: prefix
lookup and binary search per repetition, id + code + sketch per retrieved
entry, the row of every candidate that passed the filter, the float32 row of
every reranked one, the query and the output), the narrower count without the
code bytes, and the rule that reports the committed DRAM traffic only for the
workload and kernel source it was measured on."""
import math
import os
import sys
import types

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _stats(retrieved, passed, reranked):
    return {"retrieved": np.array(retrieved, np.int64), "passed_filter": np.array(passed, np.int64),
            "reranked": np.array(reranked, np.int64)}


def test_byte_count_term_by_term():
    L, n, d, k = 221, 1_000_000, 100, 10
    st = _stats([377_000, 1000], [24_000, 10], [400, 0])
    probes = math.ceil(math.log2(n / 8192))  # 7 binary-search steps inside a 13-bit bucket
    assert probes == 7
    per_query = [L * (8 + 4 * probes) + r * 16 + p * 2 * d + rr * 4 * d + 4 * d + 8 * k
                 for r, p, rr in zip(st["retrieved"], st["passed_filter"], st["reranked"])]
    assert bench.algorithmic_bytes(st, L, n, d, k, "bf16") == np.mean(per_query)
    narrow = [b - r * 4 for b, r in zip(per_query, st["retrieved"])]
    assert bench.algorithmic_bytes(st, L, n, d, k, "bf16", code_bytes=0) == np.mean(narrow)
    # float32 rows cost 4d per passed candidate, e4m3 rows d + 8 (codes, scale and bound)
    f32 = [b + p * 2 * d for b, p in zip(per_query, st["passed_filter"])]
    assert bench.algorithmic_bytes(st, L, n, d, k, "fp32") == np.mean(f32)
    fp8 = [b - p * (d - 8) for b, p in zip(per_query, st["passed_filter"])]
    assert bench.algorithmic_bytes(st, L, n, d, k, "fp8") == np.mean(fp8)


def test_traffic_is_reported_only_for_the_measured_configuration(tmp_path):
    base = types.SimpleNamespace(points=None, queries=None, budget=None, mode="learned", train_queries=100_000,
                                 epochs=20, recall=0.9, workload=bench.WORKLOAD, family="crosspolytope",
                                 estimate="bf16", stop_every=0, pool_bits=0, filter_eps=0.0,
                                 learned_margin=None, flat_fill=None, no_filter=False)
    # any option that changes the workload or the kernel's work gives no traffic
    for key, val in [("budget", 1 << 30), ("mode", "bf16"), ("estimate", "fp8"), ("stop_every", 8),
                     ("pool_bits", 3072), ("filter_eps", 0.1), ("no_filter", True), ("flat_fill", 3),
                     ("learned_margin", 2), ("points", 1000), ("family", "fht")]:
        args = types.SimpleNamespace(**{**vars(base), key: val})
        assert bench.search_kernel_traffic(args) is None, key
    # with the default configuration it is the committed figure, or None once
    # the kernel source no longer matches the one profiled
    t = bench.search_kernel_traffic(base)
    assert t is None or t > 0
