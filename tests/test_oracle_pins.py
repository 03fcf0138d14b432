"""Pins of the CPU oracle against things other than itself: published test
vectors, closed forms, hand-worked examples, independent library routines,
brute force on small inputs and the paper's invariants."""
import math

import numpy as np
import pytest

from conftest import read_golden

import datagen


# ------------------------------------------------------------ random numbers
def test_philox_known_answers(orc):
    for row in read_golden("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        out = orc.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_gaussian_moments(orc):
    # 2048 x 64 = 131072 draws; N(0,1): mean 0, variance 1, P(|z|<1) = 0.682689
    S = orc.gen_sketch_params(123, 32, 64).ravel().astype(np.float64)
    N = S.size
    assert abs(S.mean()) < 5 / math.sqrt(N)
    assert abs(S.var() - 1.0) < 5 * math.sqrt(2.0 / N)
    frac = np.mean(np.abs(S) < 1.0)
    assert abs(frac - 0.682689) < 5 * math.sqrt(0.6827 * 0.3173 / N)
    # every entry is a bfloat16 value (the low 16 bits of its float32 are zero)
    assert np.all(S.astype(np.float32).view(np.uint32) & 0xFFFF == 0)
    # different purposes / seeds give different streams
    assert orc.gauss(1, 1, 0, 0, 0) != orc.gauss(2, 1, 0, 0, 0)
    assert orc.gauss(1, 1, 0, 0, 0) != orc.gauss(1, 2, 0, 0, 0)


# ------------------------------------------------------------ normalisation
def test_normalize_matches_fp64(orc):
    x = datagen.gaussian(500, 37, seed=3)
    x[7] = 0.0
    out = orc.normalize(x)
    x64 = x.astype(np.float64)
    nrm = np.sqrt(np.sum(x64 * x64, axis=1, keepdims=True))
    with np.errstate(invalid="ignore", divide="ignore"):
        ref = np.where(nrm > 0, x64 / nrm, 0.0).astype(np.float32)
    # numpy sums pairwise: the FP64 norms can differ in the last bit, which
    # moves a float32 quotient by at most one ulp.
    ulps = np.abs(out.view(np.int32).astype(np.int64) - ref.view(np.int32).astype(np.int64))
    assert ulps.max() <= 1
    assert np.all(out[7] == 0)
    n2 = np.linalg.norm(out.astype(np.float64), axis=1)
    assert np.all(np.abs(n2[np.arange(500) != 7] - 1.0) < 1e-6)


# ------------------------------------------------------------ hashing
def test_hp_bits_match_independent_projection(orc):
    d, L = 48, 6
    x = orc.normalize(datagen.gaussian(300, d, seed=4))
    A = orc.gen_hash_params(9, orc.SIMHASH, L, d)
    codes = orc.hash_codes(orc.SIMHASH, A, x)
    v = np.einsum("jbi,pi->jpb", A.astype(np.float64), x.astype(np.float64))  # [L][n][32]
    bits = (v >= 0).astype(np.uint64)
    ref = np.zeros((L, 300), np.uint64)
    for b in range(32):
        ref |= bits[:, :, b] << np.uint64(31 - b)
    safe = np.all(np.abs(v) > 1e-9, axis=2)
    assert np.array_equal(codes[safe], ref.astype(np.uint32)[safe])


def test_cp_code_hand_example(orc):
    for row in read_golden("cp_code_example.txt"):
        x = np.array([float(t) for t in row[:4]], np.float32)[None, :]
        lay = orc.layout(orc.CROSSPOLYTOPE, 4)
        assert (lay["ell"], lay["F"], lay["Kb"]) == (3, 10, 30)
        A = np.tile(np.eye(4, dtype=np.float32), (10, 1))[None]  # one table, 10 functions
        code = orc.hash_codes(orc.CROSSPOLYTOPE, A, orc.normalize(x))[0, 0]
        assert int(code) == int(row[4], 16)


def test_cp_codes_brute_force_argmax(orc):
    d, L = 8, 5
    lay = orc.layout(orc.CROSSPOLYTOPE, d)
    ell, F = lay["ell"], lay["F"]
    x = orc.normalize(datagen.gaussian(200, d, seed=5))
    A = orc.gen_hash_params(11, orc.CROSSPOLYTOPE, L, d)
    codes = orc.hash_codes(orc.CROSSPOLYTOPE, A, x)
    for j in range(L):
        for p in range(200):
            code = 0
            for f in range(F):
                v = A[j, f * d:(f + 1) * d].astype(np.float64) @ x[p].astype(np.float64)
                c = int(np.argmax(np.abs(v)))
                val = ((1 if v[c] < 0 else 0) << (ell - 1)) | c
                code |= val << (32 - ell * (f + 1))
            assert code == int(codes[j, p])


def _pair_at(theta, d, seed):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(d)
    u /= np.linalg.norm(u)
    w = rng.standard_normal(d)
    w -= (w @ u) * u
    w /= np.linalg.norm(w)
    y = math.cos(theta) * u + math.sin(theta) * w
    return np.stack([u, y]).astype(np.float32)


@pytest.mark.parametrize("theta", [0.3, 1.0, 2.0])
def test_hp_collision_rate_closed_form(orc, theta):
    # Sec. 2.2 / 4.3: Pr[HP bit agrees] = 1 - theta/pi.  3000 tables x 32 bits.
    d, L = 32, 3000
    xy = orc.normalize(_pair_at(theta, d, 1))
    A = orc.gen_hash_params(21, orc.SIMHASH, L, d)
    codes = orc.hash_codes(orc.SIMHASH, A, xy)
    agree = ~(codes[:, 0] ^ codes[:, 1])
    hits = sum(bin(int(a)).count("1") for a in agree)
    N = L * 32
    p = 1 - theta / math.pi
    assert abs(hits / N - p) < 5 * math.sqrt(p * (1 - p) / N)


def test_sketch_hamming_is_binomial(orc):
    # Fig. 2 footnote: Hamming distance of 64-bit HP sketches ~ Bin(64, theta/pi)
    theta, d, M = 1.2, 40, 512
    xy = orc.normalize(_pair_at(theta, d, 2))
    S = orc.gen_sketch_params(33, M, d)
    sk = orc.sketches(S, xy)
    ham = np.array([bin(int(a) ^ int(b)).count("1") for a, b in zip(sk[:, 0], sk[:, 1])])
    mean, var = 64 * theta / math.pi, 64 * (theta / math.pi) * (1 - theta / math.pi)
    assert abs(ham.mean() - mean) < 5 * math.sqrt(var / M)
    assert abs(ham.var() - var) < 0.25 * var


# ------------------------------------------------------------ tables
def test_sorted_tables_and_prefix(orc):
    rng = np.random.default_rng(7)
    codes = rng.integers(0, 1 << 32, size=(4, 5000), dtype=np.uint64).astype(np.uint32)
    codes[:, ::7] = codes[:, 3:4]  # many equal codes
    sc, ids = orc.sort_tables(codes)
    for j in range(4):
        order = np.lexsort((np.arange(5000), codes[j]))
        assert np.array_equal(ids[j], order.astype(np.uint32))
        assert np.array_equal(sc[j], codes[j][order])
    pfx = orc.prefix_table(sc)
    for j in range(4):
        top = (sc[j] >> 19).astype(np.int64)
        ref = np.searchsorted(top, np.arange(8193), side="left")
        assert np.array_equal(pfx[j], ref.astype(np.uint32))


# ------------------------------------------------------------ collision model
def test_alpha_grid(orc):
    assert orc.alpha(0) == -1.0 and orc.alpha(20) == 0.0 and orc.alpha(40) == 1.0
    assert orc.alpha_index(0.05) == 21
    assert orc.alpha_index(0.0499) == 20
    assert orc.alpha_index(-1.0) == 0 and orc.alpha_index(-1.5) == 0
    assert orc.alpha_index(1.0) == 40 and orc.alpha_index(0.999) == 39


def test_hp_collision_probability_closed_form(orc):
    assert orc.collision_prob(orc.SIMHASH, 1, None, 0.0, 1) == 0.5
    assert orc.collision_prob(orc.SIMHASH, 1, None, 1.0, 17) == 1.0
    assert orc.collision_prob(orc.SIMHASH, 1, None, -1.0, 1) == 0.0
    assert abs(orc.collision_prob(orc.SIMHASH, 1, None, 0.5, 1) - 2.0 / 3.0) < 1e-15
    assert abs(orc.collision_prob(orc.SIMHASH, 1, None, 0.5, 3) - (2.0 / 3.0) ** 3) < 1e-15
    assert orc.collision_prob(orc.SIMHASH, 1, None, 0.3, 0) == 1.0


def test_stop_rule_hand_values(orc):
    for row in read_golden("stop_rule_hp.txt"):
        s, depth, L, fail, stop = float(row[0]), int(row[1]), int(row[2]), float(row[3]), int(row[4])
        p = orc.collision_prob(orc.SIMHASH, 1, None, s, depth)
        f = orc.ipow(1.0 - p, L)
        assert abs(f - fail) < 1e-5 * fail  # six significant digits
        assert (f <= 0.1) == bool(stop)
        assert abs(f - (1 - p) ** L) < 1e-14


def test_ipow(orc):
    for x in (0.5, 0.9, 1.0 - 2 ** -20, 0.123456789):
        for e in (0, 1, 2, 7, 100, 401, 1023):
            assert abs(orc.ipow(x, e) - x ** e) <= 1e-13 * x ** e


def test_filter_tau(orc):
    for row in read_golden("filter_tau.txt"):
        assert orc.filter_tau(float(np.float32(row[0]))) == int(row[1])
    rng = np.random.default_rng(0)
    for s in rng.uniform(-1, 1, 2000):
        v = 64 * math.acos(s) / math.pi
        if abs(v - round(v)) > 1e-9:
            assert orc.filter_tau(s) == math.floor(v)


def test_cp_table_properties(orc):
    for d in (16, 100):
        P = orc.cp_table(5, d, 1000)
        ell = orc.layout(orc.CROSSPOLYTOPE, d)["ell"]
        assert P.shape == (41, ell + 1)
        assert np.all(P[:, 0] == 1.0)
        assert np.all(P[40] == 1.0)  # alpha = 1: y = x
        assert np.all(P[0, 1:] == 0.0)  # alpha = -1: y = -x, sign bit differs
        assert np.all(np.diff(P, axis=0) >= 0)  # monotone in alpha
        assert np.all(np.diff(P, axis=1) <= 0)  # longer prefixes collide less


def _numpy_cp_value(v, ell):
    c = np.argmax(np.abs(v), axis=-1)
    neg = np.take_along_axis(v, c[..., None], -1)[..., 0] < 0
    return (neg.astype(np.int64) << (ell - 1)) | c


def test_cp_table_vs_independent_monte_carlo(orc):
    d, N = 24, 20000
    ell = orc.layout(orc.CROSSPOLYTOPE, d)["ell"]
    P = orc.cp_table(8, d, N)
    rng = np.random.default_rng(99)
    a = rng.standard_normal((N, d, 2))
    for t in (10, 20, 26, 30, 34, 37):
        al = orc.alpha(t)
        hx = _numpy_cp_value(a[:, :, 0], ell)
        hy = _numpy_cp_value(al * a[:, :, 0] + math.sqrt(1 - al * al) * a[:, :, 1], ell)
        for r in range(1, ell + 1):
            est = np.mean((hx >> (ell - r)) == (hy >> (ell - r)))
            sd = math.sqrt(max(est * (1 - est), 1e-4) * 2 / N)
            assert abs(P[t, r] - est) < 5 * sd + 1e-3, (t, r, P[t, r], est)


def test_cp_full_code_collision_matches_table(orc):
    # Independent functions compose: Pr[all Kb bits of a table agree] =
    # P_full(alpha)^F.  Empirical rate over many tables at alpha = 0.8.
    d, L = 16, 4000
    lay = orc.layout(orc.CROSSPOLYTOPE, d)
    F, ell = lay["F"], lay["ell"]
    xy = orc.normalize(_pair_at(math.acos(0.8), d, 3))
    A = orc.gen_hash_params(44, orc.CROSSPOLYTOPE, L, d)
    codes = orc.hash_codes(orc.CROSSPOLYTOPE, A, xy)
    s = float(np.float64(xy[0]) @ np.float64(xy[1]))
    P = orc.cp_table(45, d, 20000)
    t = orc.alpha_index(s)
    for depth in (ell, 2 * ell, 2 * ell + 2):
        shift = 32 - depth
        hits = np.mean((codes[:, 0] >> shift) == (codes[:, 1] >> shift))
        # the table is evaluated at the grid point below s, so it bounds from below
        lo = orc.collision_prob(orc.CROSSPOLYTOPE, ell, P, orc.alpha(t), depth)
        hi = orc.collision_prob(orc.CROSSPOLYTOPE, ell, P, orc.alpha(min(t + 1, 40)), depth)
        sd = math.sqrt(max(hits * (1 - hits), 1e-3) / L)
        assert lo - 5 * sd - 0.01 <= hits <= hi + 5 * sd + 0.01, (depth, lo, hits, hi)
    assert F * ell == lay["Kb"]


# ------------------------------------------------------------ budget
def test_budget_formula_values(orc):
    # hand-evaluated with the layouts stated in orc_budget_L
    n, d, M = 1_000_000, 100, 32
    dp, R = 112, 4 * 112
    # hyperplane entries are bfloat16 values: float32 + one exact bfloat16 copy = 6 bytes each
    fixed_point = n * dp * 6 + n * M * 8 + 64 * M * dp * 6
    per_point = n * 8 + 8193 * 4 + R * dp * 6
    assert orc.budget_L(orc.CROSSPOLYTOPE, n, d, M, 4 << 30, 1) == ((4 << 30) - fixed_point) // per_point == 403
    fixed_table = n * dp * 6 + 64 * M * dp * 6
    per_table = n * 16 + 8193 * 4 + R * dp * 6
    assert orc.budget_L(orc.CROSSPOLYTOPE, n, d, M, 4 << 30, 0) == ((4 << 30) - fixed_table) // per_table == 221
    assert orc.budget_L(orc.SIMHASH, 10_000, 64, 32, 32 << 20, 1) == 210
    assert orc.budget_L(orc.SIMHASH, 10_000, 64, 32, 1 << 20, 0) == 0
    # pseudo-random CP: the hash functions are three sign vectors of d'' = 128
    # bits per function (4 words each) instead of d' x d' rows
    per_fht = n * 16 + 8193 * 4 + 4 * 3 * 4 * 4
    assert orc.budget_L(orc.CROSSPOLYTOPE_FHT, n, d, M, 4 << 30, 0) == ((4 << 30) - fixed_table) // per_fht == 225
    # an 8-bit float copy of the rows: d' bytes + scale + bound per row, fixed
    fixed_fp8 = fixed_table + n * (dp + 8)
    assert orc.budget_L(orc.CROSSPOLYTOPE, n, d, M, 4 << 30, 0, 0, 1) == ((4 << 30) - fixed_fp8) // per_table


def test_budget_with_binary16_rows(orc):
    # the 10M x 96 workload with binary16 rows (2 B) + the bfloat16 copy (2 B), 40 GiB, a sketch per entry
    n, d, M = 10_000_000, 96, 32
    dp, R = 96, 4 * 96  # CP with l = ceil(log2 192) = 8: 4 functions of 96 rows
    fixed = n * dp * 4 + 64 * M * dp * 6
    per_table = n * 16 + 8193 * 4 + R * dp * 6
    want = ((40 << 30) - fixed) // per_table
    assert want == 244
    assert orc.budget_L(orc.CROSSPOLYTOPE, n, d, M, 40 << 30, 0, 1) == want
    # float32 rows leave room for fewer repetitions
    assert orc.budget_L(orc.CROSSPOLYTOPE, n, d, M, 40 << 30, 0, 0) == ((40 << 30) - fixed - n * dp * 2) // per_table


def test_binary16_rows_round_to_nearest_even(orc):
    # binary16 has 10 fraction bits: at 1 the spacing is 2^-10, so 1 + 2^-11 and
    # 1 + 3*2^-11 are ties that go to the even neighbours 1 and 1 + 2^-9
    x = np.array([[1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, 1 + 2.0 ** -12, -0.1, 6.1e-5]], np.float32)
    got = orc.round_rows_f16(x)[0]
    assert got[0] == 1.0 and got[1] == np.float32(1 + 2.0 ** -9) and got[2] == 1.0
    assert got[3] == np.float32(np.float16(-0.1)) and abs(got[3] + 0.1) <= 2.0 ** -14
    assert got[4] == np.float32(np.float16(6.1e-5))  # the subnormal range is kept (no flush to zero)


# ------------------------------------------------------------ similarity
def test_canonical_sim(orc):
    e = np.zeros(100, np.float32)
    e[3] = 1
    assert orc.sim(e, e) == 1.0
    f = np.zeros(100, np.float32)
    f[4] = 1
    assert orc.sim(e, f) == 0.0
    x = orc.normalize(datagen.gaussian(400, 100, seed=6))
    for i in range(0, 400, 2):
        s = orc.sim(x[i], x[i + 1])
        ref = float(x[i].astype(np.float64) @ x[i + 1].astype(np.float64))
        bound = 100 * 2.0 ** -24 * float(np.abs(x[i].astype(np.float64) * x[i + 1]).sum()) * 1.01
        assert abs(float(s) - ref) <= bound
    # the 32-way split: a vector with mass only on coordinates = 5 (mod 32)
    q = np.zeros(100, np.float32)
    q[[5, 37, 69]] = [1, 2, 3]
    assert orc.sim(q, q) == 14.0


@pytest.mark.parametrize("family,d", [(0, 37), (1, 37), (1, 100)])
def test_blocked_hashing_equals_one_point_at_a_time(orc, family, d):
    """orc_hash_codes (blocks of points, rows transposed) returns exactly the
    codes of orc_hash_one (one point, one row at a time): same sums in the same
    order.  300 points span two blocks; 37 dimensions leave ragged row blocks."""
    import ctypes as C

    L, n = 7, 300
    x = orc.normalize(datagen.gaussian(n, d, seed=8))
    A = orc.gen_hash_params(12, family, L, d)
    codes = orc.hash_codes(family, A, x)
    one = np.zeros(L, np.uint32)
    for p in range(n):
        xp = np.ascontiguousarray(x[p])
        orc.lib().orc_hash_one(family, L, d, A.ctypes.data_as(C.c_void_p), xp.ctypes.data_as(C.c_void_p),
                               one.ctypes.data_as(C.c_void_p))
        assert np.array_equal(codes[:, p], one), p


def test_filter_tau_with_slack(orc):
    """Fig. 2 footnote: tau = (1 + eps) times the expected number of differing
    bits, 64 arccos(s_k)/pi, rounded down (at most 64)."""
    rng = np.random.default_rng(1)
    for eps in (0.1, 0.25, 0.5):
        for s in rng.uniform(-1, 1, 1000):
            v = (1 + eps) * 64 * math.acos(s) / math.pi
            if abs(v - round(v)) > 1e-9:
                assert orc.filter_tau(s, eps) == min(64, math.floor(v)), (eps, s)
        assert orc.filter_tau(1.0, eps) == 0 and orc.filter_tau(-1.0, eps) == 64


def test_filter_slack_only_admits_more(orc):
    """A slack eps > 0 lets through a superset at every snapshot with the same
    top-k, so the plain search's recall with eps is at least eps = 0's."""
    X = datagen.vmf_mixture(4000, 32, 25, 25.0, seed=17)
    Q = datagen.vmf_mixture(60, 32, 25, 25.0, seed=17, purpose="queries")
    ix = orc.OracleIndex(X, 1, L=30, seed=9)
    _, bs = orc.brute_force(ix.x, orc.normalize(Q), 10)
    rec = []
    for eps in (0.0, 0.2, 1e9):
        r = ix.search(Q, 10, 0.9, filter_eps=eps)
        rec.append(float(np.mean(r["sims"] >= bs[:, -1:])))
        if eps > 1e6:  # everything passes: the unfiltered search
            off = ix.search(Q, 10, 0.9, filter=False)
            assert np.array_equal(r["ids"], off["ids"]) and np.array_equal(r["stats"], off["stats"])
    assert rec[0] <= rec[1] + 0.02 and rec[1] <= rec[2] + 1e-12
