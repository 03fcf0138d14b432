"""Plain CPU oracle for PUFFINN (ESA 2019), wrapped with ctypes.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg use this package; the product library never imports it.  The
arithmetic lives in ``puffinn_oracle.c`` (each function cites its section of the
paper); this module only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "puffinn_oracle.c")
_LIB = os.path.join(_HERE, "libpuffinn_oracle.so")

SIMHASH = 0
CROSSPOLYTOPE = 1
CROSSPOLYTOPE_FHT = 2  # pseudo-random cross-polytope (oracle/fht.py)
PREFIX_BITS = 13
ALPHA_STEPS = 41

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no contraction of a*b+c, OpenMP across items)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "puffinn_oracle.h"))
    ):
        cmd = ["gcc", "-O3", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Stats(C.Structure):
    _fields_ = [("start_depth", C.c_int32), ("stop_depth", C.c_int32), ("rounds", C.c_int32),
                ("full_depth", C.c_int32), ("retrieved", C.c_int64), ("passed_filter", C.c_int64),
                ("scored", C.c_int64), ("last_reps", C.c_int32)]


class _Index(C.Structure):
    _fields_ = [("family", C.c_int), ("d", C.c_int), ("ell", C.c_int), ("Kb", C.c_int),
                ("L", C.c_int), ("M", C.c_int), ("B", C.c_int), ("n", C.c_int64),
                ("x", C.c_void_p), ("codes", C.c_void_p), ("ids", C.c_void_p),
                ("sk", C.c_void_p), ("P", C.c_void_p), ("pool_fns", C.c_int), ("pool_as_independent", C.c_int),
                ("filter_eps", C.c_double)]


STATS_DTYPE = np.dtype([("start_depth", np.int32), ("stop_depth", np.int32), ("rounds", np.int32),
                        ("full_depth", np.int32), ("retrieved", np.int64), ("passed_filter", np.int64),
                        ("scored", np.int64), ("last_reps", np.int32)], align=True)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            vp, i32, i64, u64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
            sig = {
                "orc_set_threads": (None, [C.c_int]),
                "orc_philox4x32_10": (None, [vp, vp, vp]),
                "orc_gauss": (C.c_float, [u64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32]),
                "orc_layout": (None, [C.c_int, C.c_int, vp, vp, vp, vp]),
                "orc_gen_hash_params": (None, [u64, C.c_int, C.c_int, C.c_int, vp]),
                "orc_gen_sketch_params": (None, [u64, C.c_int, C.c_int, vp]),
                "orc_normalize": (None, [vp, i64, C.c_int, vp]),
                "orc_hash_one": (None, [C.c_int, C.c_int, C.c_int, vp, vp, vp]),
                "orc_hash_codes": (None, [C.c_int, C.c_int, C.c_int, vp, vp, i64, vp]),
                "orc_sketches": (None, [C.c_int, C.c_int, vp, vp, i64, vp]),
                "orc_sort_tables": (None, [C.c_int, i64, vp, vp, vp]),
                "orc_prefix_table": (None, [C.c_int, i64, vp, vp]),
                "orc_alpha": (f64, [C.c_int]),
                "orc_alpha_index": (C.c_int, [f64]),
                "orc_cp_table": (None, [u64, C.c_int, C.c_int, vp]),
                "orc_collision_prob": (f64, [C.c_int, C.c_int, vp, f64, C.c_int]),
                "orc_ipow": (f64, [f64, i64]),
                "orc_filter_tau": (C.c_int, [f64]),
                "orc_filter_tau_eps": (C.c_int, [f64, f64]),
                "orc_budget_L": (i64, [C.c_int, i64, C.c_int, C.c_int, u64, C.c_int, C.c_int, C.c_int, C.c_int]),
                "orc_sim": (C.c_float, [vp, vp, C.c_int]),
                "orc_search": (None, [vp, vp, vp, vp, i64, vp, vp, i32, vp, C.c_int, C.c_int, vp, vp, vp, vp, i64, vp]),
                "orc_brute_force": (None, [vp, i64, C.c_int, vp, i64, C.c_int, vp, vp]),
                "orc_pool_select": (None, [u64, C.c_int, C.c_int, C.c_int, vp]),
                "orc_gen_pool_params": (None, [u64, C.c_int, C.c_int, C.c_int, vp]),
                "orc_pool_codes": (None, [C.c_int, C.c_int, C.c_int, vp, C.c_int, vp, vp, i64, vp]),
                "orc_pool_stop": (C.c_int, [C.c_int, C.c_int, vp, C.c_int, f64, C.c_int, i64, f64]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def compile_variant(src_text: str, out_path: str):
    """Compile a modified copy of the oracle's source (tests plant mistakes in
    it to show that a pin catches them) and load it with the query signature."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O3", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                           "-shared", "-I", _HERE, "-o", out_path, src, "-lm"])
    L = C.CDLL(out_path)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    L.orc_search.restype = None
    L.orc_search.argtypes = [vp, vp, vp, vp, i64, vp, vp, i32, vp, C.c_int, C.c_int, vp, vp, vp, vp, i64, vp]
    return L


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------- primitives
def philox4x32_10(ctr, key) -> np.ndarray:
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def set_threads(n: int) -> None:
    """Host threads of the oracle's parallel loops (n <= 0: all processors)."""
    lib().orc_set_threads(int(n))


def gauss(seed: int, purpose: int, a: int, b: int, c: int) -> float:
    return float(lib().orc_gauss(seed, purpose, a, b, c))


def layout(family: int, d: int):
    v = [C.c_int() for _ in range(4)]
    lib().orc_layout(family, d, *[C.byref(x) for x in v])
    ell, F, Kb, rows = (x.value for x in v)
    return {"ell": ell, "F": F, "Kb": Kb, "rows": rows}


def gen_hash_params(seed: int, family: int, L: int, d: int) -> np.ndarray:
    rows = layout(family, d)["rows"]
    A = np.zeros((L, rows, d), np.float32)
    lib().orc_gen_hash_params(seed, family, L, d, _p(A))
    return A


def gen_sketch_params(seed: int, M: int, d: int) -> np.ndarray:
    S = np.zeros((M * 64, d), np.float32)
    lib().orc_gen_sketch_params(seed, M, d, _p(S))
    return S


def normalize(x) -> np.ndarray:
    x = _c(x, np.float32)
    out = np.empty_like(x)
    lib().orc_normalize(_p(x), x.shape[0], x.shape[1], _p(out))
    return out


def hash_codes(family: int, A: np.ndarray, x: np.ndarray) -> np.ndarray:
    """codes[L][n] of normalised points x under parameters A[L][rows][d]."""
    A = _c(A, np.float32)
    x = _c(x, np.float32)
    L, _, d = A.shape
    codes = np.zeros((L, x.shape[0]), np.uint32)
    lib().orc_hash_codes(family, L, d, _p(A), _p(x), x.shape[0], _p(codes))
    return codes


def sketches(S: np.ndarray, x: np.ndarray) -> np.ndarray:
    S = _c(S, np.float32)
    x = _c(x, np.float32)
    M = S.shape[0] // 64
    sk = np.zeros((M, x.shape[0]), np.uint64)
    lib().orc_sketches(M, x.shape[1], _p(S), _p(x), x.shape[0], _p(sk))
    return sk


def sort_tables(codes: np.ndarray):
    codes = _c(codes, np.uint32)
    L, n = codes.shape
    sc = np.zeros_like(codes)
    ids = np.zeros_like(codes)
    lib().orc_sort_tables(L, n, _p(codes), _p(sc), _p(ids))
    return sc, ids


def prefix_table(sorted_codes: np.ndarray) -> np.ndarray:
    sorted_codes = _c(sorted_codes, np.uint32)
    L, n = sorted_codes.shape
    pfx = np.zeros((L, (1 << PREFIX_BITS) + 1), np.uint32)
    lib().orc_prefix_table(L, n, _p(sorted_codes), _p(pfx))
    return pfx


def alpha(t: int) -> float:
    return float(lib().orc_alpha(t))


def alpha_index(s: float) -> int:
    return int(lib().orc_alpha_index(s))


def cp_table(seed: int, d: int, draws: int = 1000) -> np.ndarray:
    ell = layout(CROSSPOLYTOPE, d)["ell"]
    P = np.zeros((ALPHA_STEPS, ell + 1), np.float64)
    lib().orc_cp_table(seed, d, draws, _p(P))
    return P


def collision_prob(family: int, ell: int, P, s: float, depth: int) -> float:
    keep = _c(P, np.float64) if P is not None else None
    return float(lib().orc_collision_prob(family, ell, _p(keep) if keep is not None else None, s, depth))


def ipow(x: float, e: int) -> float:
    return float(lib().orc_ipow(x, e))


def filter_tau(s_k: float, eps: float = 0.0) -> int:
    return int(lib().orc_filter_tau_eps(s_k, eps))


def budget_L(family: int, n: int, d: int, M: int, budget_bytes: int, sketch_layout: int = 0,
             row_storage: int = 0, fp8_rows: int = 0, pool_fns: int = 0) -> int:
    """sketch_layout 0: a sketch per repetition entry; 1: M sketches per point.
    row_storage 0: float32 rows; 1: binary16 rows.  fp8_rows 1: an 8-bit float
    copy of the rows is kept too.  pool_fns > 0: functions drawn from a pool."""
    return int(lib().orc_budget_L(family, n, d, M, budget_bytes, sketch_layout, row_storage, fp8_rows, pool_fns))


def pool_select(seed: int, L: int, F: int, m: int) -> np.ndarray:
    sel = np.zeros((L, F), np.int32)
    lib().orc_pool_select(seed, L, F, m, _p(sel))
    return sel


def gen_pool_params(seed: int, family: int, m: int, d: int) -> np.ndarray:
    R = d if family == CROSSPOLYTOPE else 1
    A = np.zeros((m, R, d), np.float32)
    lib().orc_gen_pool_params(seed, family, m, d, _p(A))
    return A


def pool_codes(family: int, A: np.ndarray, sel: np.ndarray, x: np.ndarray) -> np.ndarray:
    A, sel, x = _c(A, np.float32), _c(sel, np.int32), _c(x, np.float32)
    L = sel.shape[0]
    codes = np.zeros((L, x.shape[0]), np.uint32)
    lib().orc_pool_codes(family, A.shape[0], x.shape[1], _p(A), L, _p(sel), _p(x), x.shape[0], _p(codes))
    return codes


def pool_stop(family: int, ell: int, P, m: int, s_k: float, depth: int, j: int, delta: float) -> bool:
    keep = _c(P, np.float64) if P is not None else None
    return bool(lib().orc_pool_stop(family, ell, _p(keep) if keep is not None else None, m, s_k, depth, j, delta))


def round_rows_f16(x: np.ndarray) -> np.ndarray:
    """Normalised rows as stored in binary16 (round to nearest, ties to even),
    read back exactly as float32."""
    return np.ascontiguousarray(x, np.float32).astype(np.float16).astype(np.float32)


def sim(q, x) -> np.float32:
    q = _c(q, np.float32)
    x = _c(x, np.float32)
    return np.float32(lib().orc_sim(_p(q), _p(x), q.shape[0]))


def brute_force(x_norm: np.ndarray, q_norm: np.ndarray, k: int):
    x_norm = _c(x_norm, np.float32)
    q_norm = _c(q_norm, np.float32)
    Q = q_norm.shape[0]
    ids = np.zeros((Q, k), np.uint32)
    sims = np.zeros((Q, k), np.float32)
    lib().orc_brute_force(_p(x_norm), x_norm.shape[0], x_norm.shape[1], _p(q_norm), Q, k, _p(ids), _p(sims))
    return ids, sims


# ---------------------------------------------------------------- the index
class OracleIndex:
    """The whole index of Sec. 4, built step by step on the CPU."""

    def __init__(self, points, family: int, *, L: int | None = None, budget_bytes: int | None = None,
                 seed: int = 0, M: int = 32, B: int = 12, cp_draws: int = 1000, sketch_layout: int = 0,
                 row_storage: int = 0, fp8_rows: int = 0, pool_bits: int = 0):
        points = _c(points, np.float32)
        self.n, self.d = points.shape
        self.family, self.seed, self.M, self.B = family, seed, M, B
        if family == CROSSPOLYTOPE_FHT:
            from . import fht

            lay = fht.layout(self.d)
        else:
            lay = layout(family, self.d)
        self.ell, self.F, self.Kb = lay["ell"], lay["F"], lay["Kb"]
        # pooling (Sec. 3.2): a pool of pool_bits // l functions shared by the tables
        self.pool_fns = pool_bits // self.ell if pool_bits else 0
        if self.pool_fns and family == CROSSPOLYTOPE_FHT:
            raise ValueError("pooling is stated for the Gaussian families")
        if L is None:
            L = budget_L(family, self.n, self.d, M, int(budget_bytes), sketch_layout, row_storage, fp8_rows,
                         self.pool_fns)
        self.L = int(L)
        if self.L < 1:
            raise ValueError("memory budget too small for one repetition")
        self.x = normalize(points)
        if row_storage == 1:  # the stored point is the binary16 rounding of the normalised row
            self.x = round_rows_f16(self.x)
        self.S = gen_sketch_params(seed, M, self.d)
        if family == CROSSPOLYTOPE_FHT:
            self.A = fht.gen_params(seed, self.L, self.d)
            codes = fht.hash_codes(self.A, self.x, self.d)
            self.P = fht.cp_table(seed, self.d, cp_draws)
        elif self.pool_fns:
            self.A = gen_pool_params(seed, family, self.pool_fns, self.d)
            self.sel = pool_select(seed, self.L, self.F, self.pool_fns)
            codes = pool_codes(family, self.A, self.sel, self.x)
            self.P = cp_table(seed, self.d, cp_draws) if family == CROSSPOLYTOPE else None
        else:
            self.A = gen_hash_params(seed, family, self.L, self.d)
            codes = hash_codes(family, self.A, self.x)
            self.P = cp_table(seed, self.d, cp_draws) if family == CROSSPOLYTOPE else None
        self.sk = sketches(self.S, self.x)
        self.codes, self.ids = sort_tables(codes)
        self.pfx = prefix_table(self.codes)

    def _codes(self, x):
        if self.family == CROSSPOLYTOPE_FHT:
            from . import fht

            return fht.hash_codes(self.A, x, self.d)
        if self.pool_fns:
            return pool_codes(self.family, self.A, self.sel, x)
        return hash_codes(self.family, self.A, x)

    def hash_queries(self, queries):
        qn = normalize(queries)
        qcodes = np.ascontiguousarray(self._codes(qn).T)
        qsk = np.ascontiguousarray(sketches(self.S, qn).T)
        return qn, qcodes, qsk

    def search(self, queries, k, recall, *, k_max: int | None = None, start_depth=None,
               filter: bool = True, trace_cap: int = 0, variant=None, stop_every: int = 0,
               pool_rule: str = "cantelli", filter_eps: float = 0.0):
        qn, qcodes, qsk = self.hash_queries(queries)
        Q = qn.shape[0]
        k = np.broadcast_to(np.asarray(k, np.int32), (Q,)).copy()
        recall = np.broadcast_to(np.asarray(recall, np.float64), (Q,)).copy()
        k_max = int(k.max()) if k_max is None else int(k_max)
        ids = np.zeros((Q, k_max), np.uint32)
        sims = np.zeros((Q, k_max), np.float32)
        stats = np.zeros(Q, STATS_DTYPE)
        sd = None if start_depth is None else np.broadcast_to(np.asarray(start_depth, np.int32), (Q,)).copy()
        # the query procedure sees a cross-polytope family through its table P
        fam = CROSSPOLYTOPE if self.family == CROSSPOLYTOPE_FHT else self.family
        ix = _Index(fam, self.d, self.ell, self.Kb, self.L, self.M, self.B, self.n,
                    self.x.ctypes.data, self.codes.ctypes.data, self.ids.ctypes.data,
                    self.sk.ctypes.data, self.P.ctypes.data if self.P is not None else None, self.pool_fns,
                    1 if pool_rule == "independent" else 0, float(filter_eps))
        trace = np.zeros((Q, trace_cap, 2), np.uint32) if trace_cap else None
        tlen = np.zeros(Q, np.int64) if trace_cap else None
        (variant or lib()).orc_search(C.byref(ix), _p(qn), _p(qcodes), _p(qsk), Q, _p(k), _p(recall), k_max,
                         _p(sd) if sd is not None else None, 1 if filter else 0, int(stop_every), _p(ids), _p(sims),
                         _p(stats), _p(trace) if trace is not None else None, trace_cap,
                         _p(tlen) if tlen is not None else None)
        out = {"ids": ids, "sims": sims, "stats": stats, "qn": qn, "qsk": qsk}
        if trace_cap:
            out["trace"] = trace
            out["trace_len"] = tlen
        return out
