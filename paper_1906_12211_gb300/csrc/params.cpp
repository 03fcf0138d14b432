// Host-side random parameters, collision tables and the budget rule.
//
// Compiled with -ffp-contract=off: every expression below is evaluated as
// written (no fused multiply-add), so the same seed gives the same bits on any
// host, whichever compiler built this file.
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "pf_internal.h"

namespace pf {

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
// Box-Muller cosine branch in double, rounded once to float.
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
  return float(z);
}

Layout make_layout(int family, int d) {
  Layout L;
  L.d_pad = (d + 15) / 16 * 16;
  if (family == PF_CROSSPOLYTOPE) {
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
// 2^-12 * |a_row|_2 (for CP the largest band of the function, on every row of
// it): projections closer to a decision boundary than that are recomputed in
// float64 by the kernels.
void gen_hash_rows(uint64_t seed, int family, int L, int M, int d, const Layout& lay, float* W, float* thr) {
  const int dp = lay.d_pad;
  const int64_t rows = int64_t(L) * lay.rows_table + 64LL * M;
  std::memset(W, 0, sizeof(float) * size_t(rows) * dp);
  auto norm_band = [&](const float* row) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) s = s + double(row[i]) * double(row[i]);
    return float(std::ldexp(std::sqrt(s), -12));
  };
  parallel_for(L, [&](int64_t j) {
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

// cos(t*pi/64), t = 0..64: the sketch threshold is the largest t whose entry
// is >= s_k (= floor(64 arccos(s_k)/pi), Sec. 4.2).
void filter_cos_table(double* c) {
  for (int t = 0; t <= 64; ++t) c[t] = std::cos(double(t) * M_PI / 64.0);
}

// Device bytes the index keeps resident for L repetitions; the budget rule
// picks the largest L whose total fits (Sec. 5: the index size covers the
// data, the hash functions and the tables).  Per repetition: sorted codes and
// ids, the prefix table, the hash rows (float32 + two bfloat16 halves) and,
// with per-repetition sketches, one uint64 per entry.  Fixed: the rows
// (float32 + bfloat16), the sketch planes and, with per-point sketches, the M
// sketches of every point.
uint64_t resident_bytes(int family, int64_t n, int d, int M, int L, int sketch_layout, int row_storage) {
  const Layout lay = make_layout(family, d);
  const int64_t dp = lay.d_pad;
  const bool per_point = sketch_layout == PF_SKETCH_PER_POINT;
  const int64_t row_bytes = row_storage == PF_ROWS_F16 ? 4 : 6;  // rows (4 or 2 B) + the bfloat16 copy (2 B)
  const int64_t fixed = n * dp * row_bytes + 64LL * M * dp * 8 + (per_point ? n * int64_t(M) * 8 : 0);
  const int64_t per_table = n * (per_point ? 8 : 16) + int64_t(kPrefixSize) * 4 + int64_t(lay.rows_table) * dp * 8;
  return uint64_t(fixed + per_table * L);
}

int64_t budget_tables(int family, int64_t n, int d, int M, uint64_t budget, int sketch_layout, int row_storage) {
  const uint64_t fixed = resident_bytes(family, n, d, M, 0, sketch_layout, row_storage);
  if (budget <= fixed) return 0;
  const uint64_t per_table = resident_bytes(family, n, d, M, 1, sketch_layout, row_storage) - fixed;
  return int64_t((budget - fixed) / per_table);
}

}  // namespace pf
