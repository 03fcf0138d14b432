"""GB300 (sm_103a) implementation of PUFFINN's LSH-forest k-NN index.

A thin ctypes binding over the C ABI in ``include/puffinn_gb300.h``: it only
marshals arguments (torch CUDA tensors or numpy host arrays) into the library's
``pf_*`` calls.  Every step of index build and search runs in the library's
CUDA kernels; there is no CPU fallback -- if the compiled library is missing,
every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpuffinn_gb300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "puffinn_gb300.h")

SIMHASH, CROSSPOLYTOPE, CROSSPOLYTOPE_FHT = 0, 1, 2
FAMILIES = {"simhash": SIMHASH, "hp": SIMHASH, "crosspolytope": CROSSPOLYTOPE, "cp": CROSSPOLYTOPE,
            "crosspolytope-fht": CROSSPOLYTOPE_FHT, "fht": CROSSPOLYTOPE_FHT}

PF_OK = 0
STATUS = {0: "PF_OK", -1: "PF_ERR_INVALID_ARG", -2: "PF_ERR_BUDGET_TOO_SMALL", -3: "PF_ERR_OOM",
          -4: "PF_ERR_CUDA", -5: "PF_ERR_DEVICE_TIMEOUT", -6: "PF_ERR_NOT_TRAINED"}

ARRAYS = {"rows_f32": 0, "rows_bf16": 1, "codes": 2, "ids": 3, "prefix": 4, "sketches": 5, "hash_rows": 6,
          "cp_table": 7, "table_sketches": 8, "rows_f16": 9, "mlp_f32": 10, "mlp_w1_bf16": 11, "mlp_w2_bf16": 12,
          "fht_signs": 13,
          "rows_fp8": 14, "fp8_meta": 15, "pool_select": 16}
ROW_STORAGE = {"f32": 0, "f16": 1}
SCORING = {"fp32": 0, "bf16": 1, "fp8": 2}
POOL_RULES = {"cantelli": 0, "independent": 1}
SKETCH_LAYOUTS = {"table": 0, "point": 1}


class BuildParams(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("dtype", C.c_int32), ("family", C.c_int32),
                ("num_sketches", C.c_int32), ("memory_budget_bytes", C.c_uint64), ("seed", C.c_uint64),
                ("segment_B", C.c_int32), ("cp_draws", C.c_int32), ("num_tables", C.c_int32),
                ("sketch_layout", C.c_int32), ("row_storage", C.c_int32), ("fp8_rows", C.c_int32),
                ("pool_bits", C.c_int32)]


class SearchOpts(C.Structure):
    _fields_ = [("scoring", C.c_int32), ("filter", C.c_int32), ("learned_start", C.c_int32),
                ("timing", C.c_int32), ("start_depth", C.c_void_p), ("pool_rule", C.c_int32),
                ("filter_eps", C.c_double), ("stop_every", C.c_int32)]


class QueryStats(C.Structure):
    _fields_ = [("start_depth", C.c_int32), ("stop_depth", C.c_int32), ("rounds", C.c_int32),
                ("full_depth", C.c_int32), ("retrieved", C.c_int64), ("passed_filter", C.c_int64),
                ("scored", C.c_int64), ("reranked", C.c_int64), ("last_reps", C.c_int32), ("reserved", C.c_int32)]


STATS_DTYPE = np.dtype([("start_depth", np.int32), ("stop_depth", np.int32), ("rounds", np.int32),
                        ("full_depth", np.int32), ("retrieved", np.int64), ("passed_filter", np.int64),
                        ("scored", np.int64), ("reranked", np.int64), ("last_reps", np.int32),
                        ("reserved", np.int32)])


class IndexInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("d_pad", C.c_int32), ("family", C.c_int32),
                ("L", C.c_int32), ("Kb", C.c_int32), ("ell", C.c_int32), ("fns", C.c_int32), ("M", C.c_int32),
                ("B", C.c_int32), ("trained", C.c_int32), ("sketch_layout", C.c_int32), ("row_storage", C.c_int32),
                ("bytes_used", C.c_uint64), ("budget_bytes", C.c_uint64)]


class LearnedReport(C.Structure):
    _fields_ = [("final_loss", C.c_float), ("train_accuracy", C.c_float), ("mean_stop", C.c_float),
                ("mean_start", C.c_float), ("samples", C.c_int32), ("epochs", C.c_int32)]


class TuneReport(C.Structure):
    _fields_ = [("unroll", C.c_int32), ("warps", C.c_int32), ("ctas_per_sm", C.c_int32), ("flat_fill", C.c_int32),
                ("candidates", C.c_int32), ("best_ms", C.c_float), ("default_ms", C.c_float)]


class PlanIO(C.Structure):
    _fields_ = [("queries", C.c_void_p), ("k", C.c_void_p), ("recall", C.c_void_p), ("start_depth", C.c_void_p),
                ("out_ids", C.c_void_p), ("out_sims", C.c_void_p), ("stats", C.c_void_p)]


class PuffinnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    from . import _build

    return _build.build(force=force)


def lib():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run paper_1906_12211_gb300.build()")
            L = C.CDLL(LIB_PATH)
            vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
            sig = {
                "pf_index_build": (i32, [vp, vp, vp, vp]),
                "pf_index_search": (i32, [vp, vp, i64, vp, vp, i32, vp, vp, vp, vp, vp]),
                "pf_index_search_noalloc": (i32, [vp, vp, i64, vp, vp, i32, vp, vp, vp, vp, vp]),
                "pf_hash_queries": (i32, [vp, vp, i64, vp, vp, vp]),
                "pf_index_info": (i32, [vp, vp]),
                "pf_index_last_timing": (i32, [vp, vp, i32]),
                "pf_learned_train": (i32, [vp, vp, i64, i32, C.c_double, i32, C.c_uint64, vp, vp]),
                "pf_learned_predict": (i32, [vp, vp, i64, vp, vp]),
                "pf_learned_set_start_rule": (i32, [vp, C.c_float, i32]),
                "pf_mlp_forward_backward": (i32, [vp, vp, i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                                  vp]),
                "pf_index_array": (i32, [vp, i32, vp, vp]),
                "pf_index_read_array": (i32, [vp, i32, vp, C.c_uint64, vp]),
                "pf_search_opts_default": (None, [vp]),
                "pf_index_free": (None, [vp]),
                "pf_index_tune": (i32, [vp, vp, i64, i32, C.c_double, vp, vp, vp]),
                "pf_index_selftest_timeout": (i32, [vp, vp, i64, vp]),
                "pf_index_selftest_hold": (i32, [vp, i32]),
                "pf_index_count_range_paths": (i32, [vp, i32, vp]),
                "pf_index_set_shape": (i32, [vp, i32, i32, i32, i32]),
                "pf_search_plan_create": (i32, [vp, i64, i32, vp, vp, vp]),
                "pf_search_plan_run": (i32, [vp, vp]),
                "pf_search_plan_check": (i32, [vp, vp]),
                "pf_search_plan_free": (None, [vp]),
                "pf_status_string": (C.c_char_p, [i32]),
                "pf_last_error_message": (C.c_char_p, []),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def header_functions() -> list[str]:
    """Names of the functions the public header declares."""
    import re

    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:[\w\*]+\s+)+\**(pf_\w+)\s*\(", txt, re.M)))


def _check(status: int):
    if status != PF_OK:
        raise PuffinnError(status, lib().pf_last_error_message().decode())


def _ptr(x):
    """Address of a torch tensor or numpy array (contiguous)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    assert isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"]
    return x.ctypes.data


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    return stream if isinstance(stream, int) else stream.cuda_stream


def _family(f) -> int:
    return FAMILIES[f] if isinstance(f, str) else int(f)


class Index:
    """An LSH forest over n points (Sec. 4 of the paper), resident on the GPU."""

    def __init__(self, points, family="crosspolytope", *, budget_bytes: int = 0, num_tables: int = 0,
                 seed: int = 0, num_sketches: int = 32, segment_B: int = 12, cp_draws: int = 1000,
                 sketch_layout: str = "table", rows: str = "f32", fp8_rows: bool = False, pool_bits: int = 0,
                 stream=None):
        n, d = int(points.shape[0]), int(points.shape[1])
        p = BuildParams(n=n, d=d, dtype=0, family=_family(family), num_sketches=num_sketches,
                        memory_budget_bytes=int(budget_bytes), seed=int(seed), segment_B=segment_B,
                        cp_draws=cp_draws, num_tables=int(num_tables),
                        sketch_layout=SKETCH_LAYOUTS[sketch_layout], row_storage=ROW_STORAGE[rows],
                        fp8_rows=1 if fp8_rows else 0, pool_bits=int(pool_bits))
        self._points_keepalive = points
        h = C.c_void_p()
        _check(lib().pf_index_build(C.byref(p), _ptr(points), C.byref(h), _stream_ptr(stream)))
        self._h = h
        self._points_keepalive = None
        inf = IndexInfo()
        _check(lib().pf_index_info(self._h, C.byref(inf)))
        self.info = {f: getattr(inf, f) for f, _ in IndexInfo._fields_}
        for key in ("n", "d", "d_pad", "L", "Kb", "ell", "fns", "M", "B", "sketch_layout", "row_storage"):
            setattr(self, key, self.info[key])
        self.family = self.info["family"]

    def close(self):
        if getattr(self, "_h", None):
            lib().pf_index_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def array(self, name: str, device: str = "cuda"):
        """A copy of an internal array as a flat uint8 torch tensor (for verification)."""
        import torch

        ptr, nb = C.c_void_p(), C.c_uint64()
        _check(lib().pf_index_array(self._h, ARRAYS[name], C.byref(ptr), C.byref(nb)))
        out = torch.empty(int(nb.value), dtype=torch.uint8, device=device)
        if device != "cpu":
            torch.cuda.synchronize()
        _check(lib().pf_index_read_array(self._h, ARRAYS[name], _ptr(out), int(nb.value), _stream_ptr(None)))
        return out

    def hash_queries(self, queries, qcodes=None, qsk=None, stream=None):
        import torch

        Q = int(queries.shape[0])
        dev = queries.device if hasattr(queries, "device") else torch.device("cpu")
        if qcodes is None:
            qcodes = torch.empty((Q, self.L), dtype=torch.int32, device=dev)
        if qsk is None:
            qsk = torch.empty((Q, self.M), dtype=torch.int64, device=dev)
        _check(lib().pf_hash_queries(self._h, _ptr(queries), Q, _ptr(qcodes), _ptr(qsk), _stream_ptr(stream)))
        return qcodes, qsk

    def learned_train(self, train_queries, k: int, recall: float, *, epochs: int = 20, seed: int = 0, stream=None):
        """Train the start-depth model on traces of the plain search; returns the report."""
        rep = LearnedReport()
        _check(lib().pf_learned_train(self._h, _ptr(train_queries), int(train_queries.shape[0]), int(k),
                                      float(recall), int(epochs), int(seed), C.byref(rep), _stream_ptr(stream)))
        return {f: getattr(rep, f) for f, _ in LearnedReport._fields_}

    def learned_predict(self, queries, out=None, stream=None):
        import torch

        Q = int(queries.shape[0])
        dev = queries.device if hasattr(queries, "device") else torch.device("cpu")
        if out is None:
            out = torch.empty(Q, dtype=torch.int32, device=dev)
        _check(lib().pf_learned_predict(self._h, _ptr(queries), Q, _ptr(out), _stream_ptr(stream)))
        return out

    def search(self, queries, k, recall, *, k_max: int | None = None, scoring: str = "fp32", filter: bool = True,
               start_depth=None, out_ids=None, out_sims=None, stats=None, stream=None, timing: bool = False,
               learned: bool = False, stop_every: int = 0, pool_rule: str = "cantelli", filter_eps: float = 0.0):
        """Answer a batch of queries; k and recall are per-query arrays (same
        device as the queries) or scalars.  Returns (ids, sims, stats)."""
        import torch

        Q = int(queries.shape[0])
        dev = queries.device if hasattr(queries, "device") else torch.device("cpu")
        if not torch.is_tensor(k):
            k = torch.full((Q,), int(k), dtype=torch.int32, device=dev)
        if not torch.is_tensor(recall):
            recall = torch.full((Q,), float(recall), dtype=torch.float64, device=dev)
        if k_max is None:
            k_max = int(k.max().item()) if Q else 1
        if out_ids is None:
            out_ids = torch.empty((Q, k_max), dtype=torch.int32, device=dev)
        if out_sims is None:
            out_sims = torch.empty((Q, k_max), dtype=torch.float32, device=dev)
        if stats is True:
            stats = torch.empty((Q, STATS_DTYPE.itemsize), dtype=torch.uint8, device=dev)
        elif stats is False:
            stats = None
        o = SearchOpts()
        lib().pf_search_opts_default(C.byref(o))
        o.scoring = SCORING[scoring]
        o.filter = 1 if filter else 0
        o.timing = 1 if timing else 0
        o.learned_start = 1 if learned else 0
        o.stop_every = int(stop_every)
        o.pool_rule = POOL_RULES[pool_rule]
        o.filter_eps = float(filter_eps)
        sd = None
        if start_depth is not None:
            sd = start_depth if torch.is_tensor(start_depth) else torch.full((Q,), int(start_depth),
                                                                              dtype=torch.int32, device=dev)
            o.start_depth = _ptr(sd)
        _check(lib().pf_index_search(self._h, _ptr(queries), Q, _ptr(k), _ptr(recall), int(k_max), _ptr(out_ids),
                                     _ptr(out_sims), _ptr(stats), C.byref(o), _stream_ptr(stream)))
        return out_ids, out_sims, stats


    def search_noalloc(self, queries, k, recall, out_ids, out_sims, *, k_max: int, scoring: str = "fp32",
                       filter: bool = True, stats=None, stream=None, stop_every: int = 0, filter_eps: float = 0.0):
        """pf_index_search_noalloc: every buffer already on the device, no
        allocation inside the call (fixed 32 MiB scratch)."""
        o = self._opts(scoring, filter, False, stop_every, filter_eps=filter_eps)
        _check(lib().pf_index_search_noalloc(self._h, _ptr(queries), int(queries.shape[0]), _ptr(k), _ptr(recall),
                                             int(k_max), _ptr(out_ids), _ptr(out_sims), _ptr(stats), C.byref(o),
                                             _stream_ptr(stream)))
        return out_ids, out_sims, stats

    def _opts(self, scoring, filter, learned, stop_every=0, pool_rule="cantelli", filter_eps=0.0):
        o = SearchOpts()
        lib().pf_search_opts_default(C.byref(o))
        o.scoring = SCORING[scoring]
        o.filter = 1 if filter else 0
        o.learned_start = 1 if learned else 0
        o.stop_every = int(stop_every)
        o.pool_rule = POOL_RULES[pool_rule]
        o.filter_eps = float(filter_eps)
        return o

    def tune(self, queries, k: int, recall: float, *, scoring: str = "fp32", filter: bool = True,
             learned: bool = False, stream=None, stop_every: int = 0, pool_rule: str = "cantelli",
             filter_eps: float = 0.0):
        """pf_index_tune: time the search launch shapes on this batch and keep the fastest."""
        rep = TuneReport()
        o = self._opts(scoring, filter, learned, stop_every, pool_rule, filter_eps)
        _check(lib().pf_index_tune(self._h, _ptr(queries), int(queries.shape[0]), int(k), float(recall),
                                   C.byref(o), C.byref(rep), _stream_ptr(stream)))
        return {f: getattr(rep, f) for f, _ in TuneReport._fields_}

    def set_shape(self, unroll: int = 8, warps: int = 4, ctas_per_sm: int = 0, flat_fill: int = 0):
        """pf_index_set_shape: the launch shape of later searches and plans."""
        _check(lib().pf_index_set_shape(self._h, int(unroll), int(warps), int(ctas_per_sm), int(flat_fill)))

    def selftest_timeout(self, queries, stream=None):
        """pf_index_selftest_timeout: hash with the weight loads withheld; raises
        PuffinnError(PF_ERR_DEVICE_TIMEOUT) when the bounded waits work."""
        _check(lib().pf_index_selftest_timeout(self._h, _ptr(queries), int(queries.shape[0]), _stream_ptr(stream)))

    def learned_start_rule(self, tail: float = 0.05, margin: int = 0):
        """pf_learned_set_start_rule: start = the tail-quantile depth + margin."""
        _check(lib().pf_learned_set_start_rule(self._h, float(tail), int(margin)))

    def count_range_paths(self, enable: bool = True):
        """pf_index_count_range_paths: the counts since the last call (range
        steps by branch, rounds by streaming mode); enable=False stops counting."""
        c = (C.c_uint64 * 5)()
        _check(lib().pf_index_count_range_paths(self._h, 1 if enable else 0, c))
        return {"prefix_table": int(c[0]), "probed": int(c[1]), "galloped": int(c[2]), "chunked_rounds": int(c[3]),
                "flat_rounds": int(c[4])}

    def selftest_hold(self, hold: bool):
        """pf_index_selftest_hold: withhold (True) or restore (False) the weight
        loads of every later tensor-core hashing launch of this index."""
        _check(lib().pf_index_selftest_hold(self._h, 1 if hold else 0))

    def plan(self, queries, k, recall, out_ids, out_sims, *, k_max: int, stats=None, start_depth=None,
             scoring: str = "fp32", filter: bool = True, learned: bool = False, stop_every: int = 0,
             pool_rule: str = "cantelli", filter_eps: float = 0.0):
        """pf_search_plan_create: a CUDA graph of this search bound to these device tensors (or
        page-locked host tensors)."""
        return SearchPlan(self, queries, k, recall, out_ids, out_sims, k_max=k_max, stats=stats,
                          start_depth=start_depth, opts=self._opts(scoring, filter, learned, stop_every,
                                                                   pool_rule, filter_eps))

    def last_timing(self):
        """(hash_ms, search_kernel_ms, total_ms) of the last search run with timing=True."""
        t = (C.c_float * 3)()
        _check(lib().pf_index_last_timing(self._h, t, 3))
        return tuple(float(v) for v in t)


class SearchPlan:
    """A captured search (CUDA graph) bound to device tensors or page-locked
    host tensors (copied in and out inside the graph); run() launches it."""

    def __init__(self, index, queries, k, recall, out_ids, out_sims, *, k_max, stats, start_depth, opts):
        self._index = index
        self._keep = (queries, k, recall, out_ids, out_sims, stats, start_depth)
        io = PlanIO(_ptr(queries), _ptr(k), _ptr(recall), _ptr(start_depth), _ptr(out_ids), _ptr(out_sims),
                    _ptr(stats))
        h = C.c_void_p()
        _check(lib().pf_search_plan_create(index._h, int(queries.shape[0]), int(k_max), C.byref(io), C.byref(opts),
                                           C.byref(h)))
        self._h = h

    def run(self, stream=None):
        _check(lib().pf_search_plan_run(self._h, _stream_ptr(stream)))

    def check(self, stream=None):
        _check(lib().pf_search_plan_check(self._h, _stream_ptr(stream)))

    def close(self):
        if getattr(self, "_h", None):
            lib().pf_search_plan_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlp_forward_backward(X, y, W1, b1, W2, b2, stream=None):
    """pf_mlp_forward_backward on torch CUDA tensors; returns (loss, dW1, db1, dW2, db2)."""
    import torch

    B, F = X.shape
    H, C = W1.shape[0], W2.shape[0]
    loss = torch.zeros(1, dtype=torch.float32, device=X.device)
    g = [torch.empty_like(t) for t in (W1, b1, W2, b2)]
    _check(lib().pf_mlp_forward_backward(_ptr(X), _ptr(y), B, F, H, C, _ptr(W1), _ptr(b1), _ptr(W2), _ptr(b2),
                                         _ptr(loss), *[_ptr(t) for t in g], _stream_ptr(stream)))
    return (loss, *g)


def stats_to_numpy(stats) -> np.ndarray:
    """Per-query statistics as a numpy structured array."""
    raw = stats.cpu().numpy() if hasattr(stats, "cpu") else np.asarray(stats)
    return raw.reshape(-1).view(STATS_DTYPE)
