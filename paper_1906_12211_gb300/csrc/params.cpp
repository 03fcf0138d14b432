// Host-side random parameters, collision tables and the budget rule.
//
// Compiled with -ffp-contract=off: every expression below is evaluated as
// written (no fused multiply-add), so the same seed gives the same bits on any
// host, whichever compiler built this file.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "pf_internal.h"

namespace pf {

// The recheck band of a hash row w is |w| * 2^-e: a tensor-core projection of a
// unit point errs by at most 2^-18 |w| (the split of the point into bfloat16
// halves) plus one float32 rounding of the partial sum per add inside each of
// the 2 * 4 * ceil(d_pad / 64) MMAs of 16 products (17 adds, each within 2^-23
// of a partial sum bounded by |w|): 3.6e-5 |w| for d_pad <= 128, under the band
// 2^-14 |w| = 6.1e-5 |w|; 8.5e-5 |w| for d_pad <= 320, under 2^-12 |w|.
int band_exponent(int d_pad) { return d_pad <= 128 ? 14 : 12; }

namespace {

// Philox4x32 with 10 rounds (Salmon et al., SC 2011).  State: four 32-bit
// counter words and two key words; each round multiplies two words by fixed
// odd constants and mixes the halves of the products with the other words
// and the key; the key advances by the golden-ratio Weyl increments.
struct Philox4x32 {
  static constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
  static constexpr uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
  static void block(uint32_t w[4], uint32_t ka, uint32_t kb) {
    for (int r = 0; r < 10; ++r) {
      const uint64_t pa = uint64_t(kMulA) * w[0];
      const uint64_t pb = uint64_t(kMulB) * w[2];
      const uint32_t x0 = uint32_t(pb >> 32) ^ w[1] ^ ka;
      const uint32_t x1 = uint32_t(pb);
      const uint32_t x2 = uint32_t(pa >> 32) ^ w[3] ^ kb;
      const uint32_t x3 = uint32_t(pa);
      w[0] = x0; w[1] = x1; w[2] = x2; w[3] = x3;
      ka += kWeylA;
      kb += kWeylB;
    }
  }
};

template <class F>
void parallel_for(int64_t count, F&& body) {
  unsigned nt = std::thread::hardware_concurrency();
  if (nt == 0) nt = 4;
  if (nt > 64) nt = 64;
  if (count < 2 || nt == 1) {
    for (int64_t i = 0; i < count; ++i) body(i);
    return;
  }
  std::vector<std::thread> pool;
  for (unsigned t = 0; t < nt; ++t)
    pool.emplace_back([&, t] {
      for (int64_t i = t; i < count; i += nt) body(i);
    });
  for (auto& th : pool) th.join();
}

}  // namespace

// One N(0,1) draw per counter: counter words (c, b, a, purpose), key = seed.
// Two 53-bit uniforms u1 in (0,1] (words 0-1) and u2 in [0,1) (words 2-3);
// Box-Muller cosine branch in double, rounded to float, then to bfloat16.
float gaussian(uint64_t seed, uint32_t purpose, uint32_t a, uint32_t b, uint32_t c) {
  uint32_t w[4] = {c, b, a, purpose};
  Philox4x32::block(w, uint32_t(seed), uint32_t(seed >> 32));
  const double scale = 1.0 / 9007199254740992.0;  // 2^-53
  const uint64_t hi = (uint64_t(w[0]) << 32) | w[1];
  const uint64_t lo = (uint64_t(w[2]) << 32) | w[3];
  const double u1 = double((hi >> 11) + 1) * scale;
  const double u2 = double(lo >> 11) * scale;
  const double radius = std::sqrt(-2.0 * std::log(u1));
  const double z = radius * std::cos(2.0 * M_PI * u2);
  // then to bfloat16, nearest even (R2: every hyperplane entry is a bfloat16
  // value, so the tensor-core products with it are exact)
  uint32_t u;
  const float f = float(z);
  std::memcpy(&u, &f, sizeof(u));
  u += 0x7fffu + ((u >> 16) & 1u);
  u &= 0xffff0000u;
  float r;
  std::memcpy(&r, &u, sizeof(r));
  return r;
}

Layout make_layout(int family, int d) {
  Layout L;
  L.d_pad = (d + 15) / 16 * 16;
  if (family == PF_CROSSPOLYTOPE_FHT) {
    // Sec. 4.3, pseudo-random CP: the transform runs over d'' = 2^ceil(log2 d)
    // coordinates, so a value is an index below d'' and a sign:
    // l = log2(2 d'') = ceil(log2 2d) bits, as for the exact family
    int n2 = 1;
    while (n2 < d) n2 *= 2;
    int ell = 0;
    while ((1 << ell) < 2 * n2) ++ell;
    L.ell = ell;
    L.fns = 32 / ell;
    L.Kb = L.fns * ell;
    L.rows_fn = 0;
    L.rows_table = 0;
    L.fht_n = n2;
    L.fht_words = n2 < 32 ? 1 : n2 / 32;
  } else if (family == PF_CROSSPOLYTOPE) {
    int ell = 0;
    while ((int64_t(1) << ell) < 2 * int64_t(d)) ++ell;  // ceil(log2 2d)
    L.ell = ell;
    L.fns = 32 / ell;
    L.Kb = L.fns * ell;
    L.rows_fn = L.d_pad;
    L.rows_table = L.fns * L.d_pad;
  } else {
    L.ell = 1;
    L.fns = 32;
    L.Kb = 32;
    L.rows_fn = 1;
    L.rows_table = 32;
  }
  return L;
}

// Hash rows: CP function f of table j owns rows (j*fns + f)*d_pad + c, row c
// holding hyperplane c (zero for c >= d); HP table j owns rows j*32 + b; the
// 64*M sketch rows follow.  Counter words: (col, row-in-table, table,
// purpose), with row-in-table = f*d + c for CP.  thr[row] is the recheck band
// |a_row|_2 * 2^-band_exponent (for CP the largest band of the function, on every row of
// it): projections closer to a decision boundary than that are recomputed in
// float64 by the kernels.
void gen_hash_rows(uint64_t seed, int family, int L, int M, int d, const Layout& lay, float* W, float* thr) {
  const int dp = lay.d_pad;
  const int64_t rows = int64_t(L) * lay.rows_table + 64LL * M;
  std::memset(W, 0, sizeof(float) * size_t(rows) * dp);
  auto norm_band = [&](const float* row) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) s = s + double(row[i]) * double(row[i]);
    return float(std::ldexp(std::sqrt(s), -band_exponent(lay.d_pad)));
  };
  // the pseudo-random family keeps no rows for its repetitions (sign vectors instead)
  parallel_for(lay.rows_table > 0 ? L : 0, [&](int64_t j) {
    for (int f = 0; f < lay.fns; ++f) {
      const int nrow = family == PF_CROSSPOLYTOPE ? d : 1;
      float band = 0.f;
      for (int c = 0; c < nrow; ++c) {
        const int64_t row = family == PF_CROSSPOLYTOPE ? (j * lay.fns + f) * int64_t(dp) + c : j * 32 + f;
        const uint32_t rin = family == PF_CROSSPOLYTOPE ? uint32_t(f * d + c) : uint32_t(f);
        float* w = W + row * dp;
        for (int i = 0; i < d; ++i) w[i] = gaussian(seed, kPurposeHash, uint32_t(j), rin, uint32_t(i));
        const float b = norm_band(w);
        if (family == PF_CROSSPOLYTOPE) {
          if (b > band) band = b;
        } else {
          thr[row] = b;
        }
      }
      if (family == PF_CROSSPOLYTOPE)
        for (int c = 0; c < dp; ++c) thr[(j * lay.fns + f) * int64_t(dp) + c] = band;
    }
  });
  const int64_t base = int64_t(L) * lay.rows_table;
  parallel_for(64LL * M, [&](int64_t r) {
    float* w = W + (base + r) * dp;
    for (int i = 0; i < d; ++i) w[i] = gaussian(seed, kPurposeSketch, 0u, uint32_t(r), uint32_t(i));
    thr[base + r] = norm_band(w);
  });
}

// Pooling (Sec. 3.2, App. B.2).  Pool function f lives in group f / fns at
// position f % fns, rows laid out exactly as a table's (so the hashing kernels
// treat the groups as tables); its hyperplane c has N(0,1) entries at counter
// (col, c, f, kPurposePool) (HP: c = 0).  Functions past m in the last group
// are zero rows (hashed, never used).
void gen_pool_rows(uint64_t seed, int family, int m, int M, int d, const Layout& lay, float* W, float* thr) {
  const int dp = lay.d_pad;
  const int groups = (m + lay.fns - 1) / lay.fns;
  const int64_t rows = int64_t(groups) * lay.rows_table + 64LL * M;
  std::memset(W, 0, sizeof(float) * size_t(rows) * dp);
  std::memset(thr, 0, sizeof(float) * size_t(rows));
  auto norm_band = [&](const float* row) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) s = s + double(row[i]) * double(row[i]);
    return float(std::ldexp(std::sqrt(s), -band_exponent(lay.d_pad)));
  };
  parallel_for(m, [&](int64_t f) {
    const int64_t g = f / lay.fns, slot = f % lay.fns;
    const int nrow = family == PF_CROSSPOLYTOPE ? d : 1;
    float band = 0.f;
    for (int c = 0; c < nrow; ++c) {
      const int64_t row = family == PF_CROSSPOLYTOPE ? (g * lay.fns + slot) * int64_t(dp) + c : g * 32 + slot;
      float* w = W + row * dp;
      for (int i = 0; i < d; ++i) w[i] = gaussian(seed, kPurposePool, uint32_t(f), uint32_t(c), uint32_t(i));
      const float b = norm_band(w);
      if (family == PF_CROSSPOLYTOPE) band = std::max(band, b);
      else thr[row] = b;
    }
    if (family == PF_CROSSPOLYTOPE)
      for (int c = 0; c < dp; ++c) thr[(g * lay.fns + slot) * int64_t(dp) + c] = band;
  });
  const int64_t base = int64_t(groups) * lay.rows_table;
  parallel_for(64LL * M, [&](int64_t r) {
    float* w = W + (base + r) * dp;
    for (int i = 0; i < d; ++i) w[i] = gaussian(seed, kPurposeSketch, 0u, uint32_t(r), uint32_t(i));
    thr[base + r] = norm_band(w);
  });
}

// Table j's subset: a partial Fisher-Yates shuffle of 0..m-1; at step s the
// swap partner is s + floor(w (m - s) / 2^32), w word 0 of the generator at
// counter (s, j, 0, kPurposePoolSelect); the subset in step order.
void pool_select(uint64_t seed, int L, int F, int m, int32_t* sel) {
  parallel_for(L, [&](int64_t j) {
    std::vector<int32_t> perm(size_t(m > 0 ? m : 1));
    for (int t = 0; t < m; ++t) perm[size_t(t)] = t;
    for (int st = 0; st < F && st < m; ++st) {
      uint32_t w[4] = {uint32_t(st), uint32_t(j), 0u, uint32_t(kPurposePoolSelect)};
      Philox4x32::block(w, uint32_t(seed), uint32_t(seed >> 32));
      const int r = st + int((uint64_t(w[0]) * uint64_t(m - st)) >> 32);
      std::swap(perm[size_t(st)], perm[size_t(r)]);
      sel[j * F + st] = perm[size_t(st)];
    }
  });
}

namespace {
// index and sign bit of the largest |v_c| (first c on ties)
uint32_t cp_code_of(const double* v, int d, int ell) {
  int arg = 0;
  double top = -1.0;
  for (int c = 0; c < d; ++c) {
    const double a = std::fabs(v[c]);
    if (a > top) {
      top = a;
      arg = c;
    }
  }
  const uint32_t neg = v[arg] < 0.0 ? 1u : 0u;
  return (neg << (ell - 1)) | uint32_t(arg);
}
}  // namespace

// Sec. 4.3: Monte-Carlo estimate of Pr[first r bits of two CP values agree]
// for x = e_1 and y = (alpha, sqrt(1 - alpha^2), 0, ...), alpha on the grid
// -1, -0.95, ..., 1, r = 0..l.  Only the first two coordinates of each
// hyperplane matter; the same draws serve every alpha.  Afterwards every entry
// is lowered to the smallest entry at any larger alpha, so the table is a
// non-decreasing function of the similarity.
void cp_collision_table(uint64_t seed, int d, int ell, int draws, double* P) {
  const int W = ell + 1;
  std::vector<int64_t> hits(size_t(kAlphaSteps) * W, 0);
  std::vector<double> vx(d), vy(d);
  std::vector<float> g0(d), g1(d);
  for (int t = 0; t < draws; ++t) {
    for (int c = 0; c < d; ++c) {
      g0[c] = gaussian(seed, kPurposeCpMc, uint32_t(t), uint32_t(c), 0u);
      g1[c] = gaussian(seed, kPurposeCpMc, uint32_t(t), uint32_t(c), 1u);
    }
    for (int a = 0; a < kAlphaSteps; ++a) {
      const double alpha = double(5 * a - 100) / 100.0;
      const double beta = std::sqrt(1.0 - alpha * alpha);
      for (int c = 0; c < d; ++c) {
        vx[c] = double(g0[c]);
        vy[c] = alpha * double(g0[c]) + beta * double(g1[c]);
      }
      const uint32_t hx = cp_code_of(vx.data(), d, ell);
      const uint32_t hy = cp_code_of(vy.data(), d, ell);
      for (int r = 0; r <= ell; ++r) hits[a * W + r] += (hx >> (ell - r)) == (hy >> (ell - r)) ? 1 : 0;
    }
  }
  for (int a = 0; a < kAlphaSteps; ++a)
    for (int r = 0; r <= ell; ++r) P[a * W + r] = double(hits[a * W + r]) / double(draws);
  for (int a = kAlphaSteps - 2; a >= 0; --a)
    for (int r = 0; r <= ell; ++r) P[a * W + r] = std::fmin(P[a * W + r], P[(a + 1) * W + r]);
}

// ---------------------------------------------------------------------------
// Pseudo-random cross-polytope family (Sec. 4.3: "three applications of the
// fast Hadamard transform", after Andoni et al. 2015).  A function maps x,
// zero-padded to d'' = 2^ceil(log2 d) coordinates, to y = H D3 H D2 H D1 x, with
// H the unnormalised Walsh-Hadamard matrix and D_r diagonal with random +-1
// entries; its value is the index c of the largest |y_c| (first c on ties) and
// the sign of y_c, as for the exact family.  H v is the in-place butterfly: for
// h = 1, 2, 4, ..., d''/2 and every pair (i, i + h) with bit h of i clear,
// (v_i, v_{i+h}) <- (v_i + v_{i+h}, v_i - v_{i+h}).  Every float64 value
// is defined by this order of operations.
// Signs: the generator's counter (block, b, a, purpose) with the seed as key
// yields 128 bits per block; bit i of a vector is bit i % 32 of word
// (i % 128) / 32 of block i / 128, and a set bit means -1.  The index's
// function f of table j uses (a, b) = (j, 3 f + r) for D_{r+1}, purpose
// kPurposeFht; draw t of the collision table uses (t, r), kPurposeFhtMc.
// ---------------------------------------------------------------------------
namespace {
void fht_sign_words(uint64_t seed, uint32_t purpose, uint32_t a, uint32_t b, int words, uint32_t* out) {
  for (int blk = 0; blk * 4 < words; ++blk) {
    uint32_t w[4] = {uint32_t(blk), b, a, purpose};
    Philox4x32::block(w, uint32_t(seed), uint32_t(seed >> 32));
    for (int q = 0; q < 4 && blk * 4 + q < words; ++q) out[blk * 4 + q] = w[q];
  }
}

// y = H D3 H D2 H D1 v in float64 (v: n2 values, overwritten), signs[r][words]
void fht_rotate64(double* v, int n2, const uint32_t* signs, int words) {
  for (int r = 0; r < 3; ++r) {
    const uint32_t* sg = signs + size_t(r) * words;
    for (int i = 0; i < n2; ++i)
      if ((sg[i / 32] >> (i % 32)) & 1u) v[i] = -v[i];
    for (int h = 1; h < n2; h *= 2)
      for (int i = 0; i < n2; ++i)
        if (!(i & h)) {
          const double a = v[i], b = v[i + h];
          v[i] = a + b;
          v[i + h] = a - b;
        }
  }
}
}  // namespace

void gen_fht_signs(uint64_t seed, int L, const Layout& lay, uint32_t* out) {
  const int W = lay.fht_words;
  parallel_for(L, [&](int64_t j) {
    for (int f = 0; f < lay.fns; ++f)
      for (int r = 0; r < 3; ++r)
        fht_sign_words(seed, kPurposeFht, uint32_t(j), uint32_t(3 * f + r), W,
                       out + ((size_t(j) * lay.fns + f) * 3 + r) * W);
  });
}

// Sec. 4.3 Monte-Carlo table for this family: x = e_1 and y = (alpha,
// sqrt(1 - alpha^2), 0, ...) on the 0.05 grid, one random function per draw
// (the same draws for every alpha), then made non-decreasing in alpha.
void fht_collision_table(uint64_t seed, const Layout& lay, int draws, double* P) {
  const int n2 = lay.fht_n, ell = lay.ell, W = lay.fht_words, WP = ell + 1;
  std::vector<int64_t> hits(size_t(kAlphaSteps) * WP, 0);
  std::vector<uint32_t> sg(size_t(3) * W);
  std::vector<double> vx(n2), vy(n2);
  for (int t = 0; t < draws; ++t) {
    for (int r = 0; r < 3; ++r) fht_sign_words(seed, kPurposeFhtMc, uint32_t(t), uint32_t(r), W, &sg[size_t(r) * W]);
    std::fill(vx.begin(), vx.end(), 0.0);
    vx[0] = 1.0;
    fht_rotate64(vx.data(), n2, sg.data(), W);
    const uint32_t hx = cp_code_of(vx.data(), n2, ell);
    for (int a = 0; a < kAlphaSteps; ++a) {
      const double alpha = double(5 * a - 100) / 100.0;
      std::fill(vy.begin(), vy.end(), 0.0);
      vy[0] = alpha;
      if (n2 > 1) vy[1] = std::sqrt(1.0 - alpha * alpha);
      fht_rotate64(vy.data(), n2, sg.data(), W);
      const uint32_t hy = cp_code_of(vy.data(), n2, ell);
      for (int r = 0; r <= ell; ++r) hits[a * WP + r] += (hx >> (ell - r)) == (hy >> (ell - r)) ? 1 : 0;
    }
  }
  for (int a = 0; a < kAlphaSteps; ++a)
    for (int r = 0; r <= ell; ++r) P[a * WP + r] = double(hits[a * WP + r]) / double(draws);
  for (int a = kAlphaSteps - 2; a >= 0; --a)
    for (int r = 0; r <= ell; ++r) P[a * WP + r] = std::fmin(P[a * WP + r], P[(a + 1) * WP + r]);
}

// Error of the float32 transform for |x|_2 <= 1 + 2^-20 (a normalised row):
// with u the unit roundoff and m = log2 d'', one butterfly pass of an input v
// errs by at most g |v|_1 per output, g = m u / (1 - m u) (every output is a
// depth-m tree of additions of +-v_i).  An error e of the input reaches an
// output as at most |e|_1 <= d'' |e|_inf.  With |x|_1 <= sqrt(d) |x|_2 and
// |v_r|_1 <= sqrt(d'') |v_r|_2 = d''^((r+1)/2) |x|_2 after pass r:
//   e1 <= g sqrt(d) |x|,  e_{r+1} <= d'' e_r (1 + g) + g d''^((r+1)/2) |x|.
// A decision is redone in float64 when the top two |y| (float32) are within
// 2 (e3 + e3') of each other or the top |y| is within e3 + e3' of zero, e3'
// the same bound for float64.
void fht_bands(int d, const Layout& lay, float* gap, float* sign) {
  const double N = lay.fht_n;
  int m = 0;
  while ((1 << m) < lay.fht_n) ++m;
  auto e3 = [&](double u) {
    const double g = m * u / (1.0 - m * u), x = 1.0 + std::ldexp(1.0, -20);
    double e = g * std::sqrt(double(d)) * x;
    e = N * e * (1.0 + g) + g * N * x;
    e = N * e * (1.0 + g) + g * N * std::sqrt(N) * x;
    return e;
  };
  const double t = (e3(std::ldexp(1.0, -24)) + e3(std::ldexp(1.0, -53))) * 1.01;
  *gap = float(2.0 * t);
  *sign = float(t);
}

// cos(t*pi/(64 (1 + eps))), t = 0..64: the sketch threshold is the largest t
// whose entry is >= s_k (= floor((1 + eps) 64 arccos(s_k)/pi), Sec. 4.2 and the
// footnote of Fig. 2; eps = 0 in Sec. 5.1).
void filter_cos_table(double* c, double eps) {
  for (int t = 0; t <= 64; ++t) c[t] = std::cos(double(t) * M_PI / (64.0 * (1.0 + eps)));
}

// Device bytes the index keeps resident for L repetitions; the budget rule
// picks the largest L whose total fits (Sec. 5: the index size covers the
// data, the hash functions and the tables).  Per repetition: sorted codes and
// ids, the prefix table, the hash rows (float32 + their exact bfloat16 copy) and,
// with per-repetition sketches, one uint64 per entry.  Fixed: the rows
// (float32 + bfloat16), the sketch planes and, with per-point sketches, the M
// sketches of every point.
uint64_t resident_bytes(int family, int64_t n, int d, int M, int L, int sketch_layout, int row_storage, int fp8_rows,
                        int pool_fns) {
  const Layout lay = make_layout(family, d);
  const int64_t dp = lay.d_pad;
  const bool per_point = sketch_layout == PF_SKETCH_PER_POINT;
  const int64_t row_bytes = row_storage == PF_ROWS_F16 ? 4 : 6;  // rows (4 or 2 B) + the bfloat16 copy (2 B)
  int64_t fixed = n * dp * row_bytes + 64LL * M * dp * 6 + (per_point ? n * int64_t(M) * 8 : 0) +
                  (fp8_rows ? n * (dp + 8) : 0);  // e4m3 rows + (scale, bound) per row
  // pooling: the pool's rows (whole groups of fns functions) are fixed; a
  // table keeps its fns indices instead of rows
  int64_t rows_table = lay.rows_table, sel_bytes = 0;
  if (pool_fns > 0) {
    fixed += int64_t((pool_fns + lay.fns - 1) / lay.fns) * lay.rows_table * dp * 6;
    rows_table = 0;
    sel_bytes = int64_t(lay.fns) * 4;
  }
  // pseudo-random CP: three sign vectors per function instead of rows
  const int64_t fht = family == PF_CROSSPOLYTOPE_FHT ? int64_t(lay.fns) * 3 * lay.fht_words * 4 : 0;
  const int64_t per_table =
      n * (per_point ? 8 : 16) + int64_t(kPrefixSize) * 4 + rows_table * dp * 6 + fht + sel_bytes;
  return uint64_t(fixed + per_table * L);
}

int64_t budget_tables(int family, int64_t n, int d, int M, uint64_t budget, int sketch_layout, int row_storage,
                      int fp8_rows, int pool_fns) {
  const uint64_t fixed = resident_bytes(family, n, d, M, 0, sketch_layout, row_storage, fp8_rows, pool_fns);
  if (budget <= fixed) return 0;
  const uint64_t per_table =
      resident_bytes(family, n, d, M, 1, sketch_layout, row_storage, fp8_rows, pool_fns) - fixed;
  return int64_t((budget - fixed) / per_table);
}

}  // namespace pf
