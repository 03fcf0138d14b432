"""Pseudo-random cross-polytope LSH with three fast Hadamard transforms (the
"FHT-CP" family of Sec. 4.3, after Andoni et al. 2015), stated plainly in numpy.

TEST INFRASTRUCTURE ONLY, like the rest of this package: the product library
never imports it.  It reuses the oracle's counter-based generator and its
query procedure (the search of Sec. 4 only needs codes and a collision table);
the family's own arithmetic is here.

Readings (the paper names the construction but does not spell it out):
  - dimension: d' = the smallest power of two >= d; a vector is padded with
    zeros to d' coordinates;
  - one function applies  H D3 H D2 H D1  to the padded vector, H the
    unnormalised Walsh-Hadamard matrix (entries +-1; the scale does not change
    the argmax) and D_r diagonal with random +-1 entries, three per function;
  - H v is evaluated in float64 by the in-place butterfly: for h = 1, 2, 4, ...,
    d'/2 and every block of 2h coordinates, (a, b) -> (a + b, a - b) for the
    pairs (i, i + h) of the block;
  - the value is that of the exact family: c = argmax |y_c| over the d'
    coordinates (ties to the smaller c), sign = [y_c < 0], value =
    (sign << (l - 1)) | c with l = log2(2 d'), and a table concatenates
    floor(32 / l) functions, function 0 in the most significant bits;
  - signs: the generator's counter (purpose, table, 3 f + r, i // 128) with
    the seed as key gives 128 bits; bit i % 128 (word (i % 128) // 32, bit
    i % 32) set means D_r[i] = -1;
  - collision table: the Monte-Carlo estimate of Sec. 4.3 with this family
    (x = e_0, y = (alpha, sqrt(1 - alpha^2), 0, ...), 1,000 draws, the same draws
    for every alpha, made non-decreasing in alpha).
"""
from __future__ import annotations

import numpy as np

from . import ALPHA_STEPS, alpha, philox4x32_10

PURPOSE_FHT = 4     # signs of the index's functions
PURPOSE_FHT_MC = 5  # signs of the Monte-Carlo draws


def dim(d: int) -> int:
    """d' = the smallest power of two >= d."""
    p = 1
    while p < d:
        p *= 2
    return p


def layout(d: int):
    dp = dim(d)
    ell = dp.bit_length()  # log2(2 d')
    F = 32 // ell
    return {"dp": dp, "ell": ell, "F": F, "Kb": F * ell}


def signs(seed: int, purpose: int, a: int, b: int, dp: int) -> np.ndarray:
    """+-1 float64 vector of length dp for the counter (purpose, a, b, block)."""
    out = np.empty(dp, np.float64)
    key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
    for blk in range(0, dp, 128):
        w = philox4x32_10([blk // 128, b, a, purpose], key)
        for i in range(blk, min(dp, blk + 128)):
            bit = (int(w[(i % 128) // 32]) >> (i % 32)) & 1
            out[i] = -1.0 if bit else 1.0
    return out


def gen_params(seed: int, L: int, d: int) -> np.ndarray:
    """Signs [L][F][3][d'] of an index's functions."""
    lay = layout(d)
    D = np.empty((L, lay["F"], 3, lay["dp"]), np.float64)
    for j in range(L):
        for f in range(lay["F"]):
            for r in range(3):
                D[j, f, r] = signs(seed, PURPOSE_FHT, j, 3 * f + r, lay["dp"])
    return D


def fwht(v: np.ndarray) -> np.ndarray:
    """Unnormalised Walsh-Hadamard transform of the rows of v (float64), by the
    butterfly order stated in the module docstring."""
    v = np.array(v, dtype=np.float64, copy=True)
    dp = v.shape[-1]
    h = 1
    while h < dp:
        w = v.reshape(v.shape[:-1] + (dp // (2 * h), 2, h))
        a = w[..., 0, :].copy()
        b = w[..., 1, :].copy()
        w[..., 0, :] = a + b
        w[..., 1, :] = a - b
        v = w.reshape(v.shape)
        h *= 2
    return v


def rotate(x: np.ndarray, D3: np.ndarray) -> np.ndarray:
    """H D3 H D2 H D1 x for the rows of x (zero-padded to d'), D3 = [3][d'] signs."""
    dp = D3.shape[-1]
    v = np.zeros(x.shape[:-1] + (dp,), np.float64)
    v[..., : x.shape[-1]] = x
    for r in range(3):
        v = fwht(v * D3[r])
    return v


def values(y: np.ndarray, ell: int) -> np.ndarray:
    """l-bit cross-polytope values of the rows of y."""
    c = np.argmax(np.abs(y), axis=-1)  # first index of the largest |y|
    neg = np.take_along_axis(y, c[..., None], axis=-1)[..., 0] < 0.0
    return (neg.astype(np.uint32) << np.uint32(ell - 1)) | c.astype(np.uint32)


def hash_codes(D: np.ndarray, x: np.ndarray, d: int) -> np.ndarray:
    """codes[L][n] of the normalised rows x [n][d]."""
    lay = layout(d)
    L = D.shape[0]
    codes = np.zeros((L, x.shape[0]), np.uint32)
    for j in range(L):
        code = np.zeros(x.shape[0], np.uint32)
        for f in range(lay["F"]):
            v = values(rotate(x.astype(np.float64), D[j, f]), lay["ell"])
            code |= v << np.uint32(32 - lay["ell"] * (f + 1))
        codes[j] = code
    return codes


def cp_table(seed: int, d: int, draws: int = 1000) -> np.ndarray:
    """P[alpha][r]: Monte-Carlo probability that the first r bits of the values
    of x = e_0 and y = (alpha, sqrt(1 - alpha^2), 0, ...) agree (Sec. 4.3)."""
    lay = layout(d)
    dp, ell = lay["dp"], lay["ell"]
    al = np.array([alpha(t) for t in range(ALPHA_STEPS)])
    X = np.zeros((ALPHA_STEPS + 1, dp))
    X[0, 0] = 1.0
    X[1:, 0] = al
    X[1:, 1] = np.sqrt(1.0 - al * al)
    hits = np.zeros((ALPHA_STEPS, ell + 1), np.int64)
    for t in range(draws):
        D3 = np.stack([signs(seed, PURPOSE_FHT_MC, t, r, dp) for r in range(3)])
        v = values(rotate(X, D3), ell)
        hx, hy = v[0], v[1:]
        for r in range(ell + 1):
            hits[:, r] += (hx >> np.uint32(ell - r)) == (hy >> np.uint32(ell - r))
    P = hits / float(draws)
    for g in range(ALPHA_STEPS - 2, -1, -1):
        P[g] = np.minimum(P[g], P[g + 1])
    return P
