"""The search kernel decides the sketch threshold and the collision model's grid
point in float32 against tables rounded toward the side that keeps each
comparison exact (Sec. 4.2 threshold, Sec. 4.3 grid).  These host checks run the
float64 rule and the float32 rule side by side on every float32 near a table
entry and on a dense sweep of [-1, 1]."""
import math

import numpy as np


def _round_down_f32(c):
    f = np.float32(c)
    return np.nextafter(f, np.float32(-np.inf)) if float(f) > c else f


def _round_up_f32(c):
    f = np.float32(c)
    return np.nextafter(f, np.float32(np.inf)) if float(f) < c else f


def _probes(table):
    out = [np.linspace(-1.0, 1.0, 200_001, dtype=np.float32)]
    for c in table:
        f = np.float32(c)
        near = [f]
        for _ in range(3):
            near.append(np.nextafter(near[-1], np.float32(np.inf)))
        g = f
        for _ in range(3):
            g = np.nextafter(g, np.float32(-np.inf))
            near.append(g)
        out.append(np.array(near, dtype=np.float32))
    out.append(np.array([1.0000001, -1.0000001, 1.5, -1.5], dtype=np.float32))
    return np.concatenate(out)


def test_threshold_lookup_float32_equals_float64():
    cos_tab = [math.cos(t * math.pi / 64.0) for t in range(65)]
    cosf = np.array([_round_down_f32(c) for c in cos_tab], dtype=np.float32)
    assert np.all(np.diff(cosf) <= 0)
    for s in _probes(cos_tab):
        want = 0
        for t in range(65):
            if cos_tab[t] >= float(s):
                want = t
        lo, hi = 0, 65  # the kernel's binary search for the first t with cosf[t] < s
        while lo < hi:
            mid = (lo + hi) >> 1
            if cosf[mid] >= s:
                lo = mid + 1
            else:
                hi = mid
        assert (lo - 1 if lo > 0 else 0) == want, float(s)


def test_grid_point_float32_equals_float64():
    alpha = [(5 * u - 100) / 100.0 for u in range(41)]
    alpha_up = np.array([_round_up_f32(a) for a in alpha], dtype=np.float32)
    for s in _probes(alpha):
        want = 0
        for u in range(41):
            if alpha[u] <= float(s):
                want = u
        got = 0
        for u in range(41):
            if alpha_up[u] <= s:
                got = u
        assert got == want, float(s)
