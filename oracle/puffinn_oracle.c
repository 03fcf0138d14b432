/*
 * puffinn_oracle.c -- plain CPU oracle for PUFFINN's index and adaptive k-NN
 * query.  TEST INFRASTRUCTURE ONLY (see puffinn_oracle.h): only the tests, the
 * smoke check and the benchmark's CPU-baseline leg use it.
 *
 * Compiled with -ffp-contract=off so that every floating-point expression is
 * evaluated exactly as written.  OpenMP is used only across independent
 * points, tables and queries; the arithmetic of each item is sequential.
 *
 * Section references are to the ESA 2019 paper:
 *   Sec. 2.2  LSH families (HP: sign of a Gaussian projection; CP: index and
 *             sign of the largest |projection| over d Gaussian hyperplanes)
 *   Sec. 3.1  LSH forest, Algorithm 1 (adaptive-kNN) and Lemma 1
 *   Sec. 3.3  1-bit sketches
 *   Sec. 4.1  the query is answered in rounds of decreasing prefix length,
 *             the stop test runs after all repetitions of a round
 *   Sec. 4.2  normalisation, sorted (code, pos) arrays, 13-bit prefix table,
 *             segment size B, sketch filter, accumulator
 *   Sec. 4.3  bit strings of length l, dropping the last bit per round,
 *             Monte-Carlo collision table on a 0.05 similarity grid
 */
#include "puffinn_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Host threads of the OpenMP loops (n <= 0: all processors).  One thread runs
 * the queries one after another, as the paper measures them (Sec. 5). */
void orc_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC 2011): 10 rounds of the 4x32 multiply/xor bijection */
/* with the Weyl key schedule.                                               */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Round a float to the nearest bfloat16 value (ties to even), kept as a float. */
static float round_to_bfloat16(float f) {
  uint32_t u;
  memcpy(&u, &f, sizeof(u));
  u += 0x7FFFu + ((u >> 16) & 1u);
  u &= 0xFFFF0000u;
  memcpy(&f, &u, sizeof(f));
  return f;
}

/* Reading (the paper fixes no generator): counter = (c, b, a, purpose),
 * key = the 64-bit seed.  u1 in (0,1] from words 0,1 and u2 in [0,1) from
 * words 2,3 (53 bits each); z = sqrt(-2 ln u1) cos(2 pi u2), rounded to float and
 * then to bfloat16 (nearest, ties to even): every hyperplane entry is a
 * bfloat16 value. */
float orc_gauss(uint64_t seed, uint32_t purpose, uint32_t a, uint32_t b, uint32_t c) {
  uint32_t ctr[4] = {c, b, a, purpose};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  orc_philox4x32_10(ctr, key, r);
  uint64_t w1 = ((uint64_t)r[0] << 32) | r[1];
  uint64_t w2 = ((uint64_t)r[2] << 32) | r[3];
  double u1 = (double)((w1 >> 11) + 1) * (1.0 / 9007199254740992.0);
  double u2 = (double)(w2 >> 11) * (1.0 / 9007199254740992.0);
  double rad = sqrt(-2.0 * log(u1));
  double z = rad * cos(2.0 * M_PI * u2);
  return round_to_bfloat16((float)z);
}

/* Sec. 4.3: l = 1 for HP, l = ceil(log2(2d)) for CP.  Reading: codes are 32
 * bits wide, so a table concatenates floor(32/l) functions (K = 32 for HP). */
void orc_layout(int family, int d, int* ell, int* fns, int* Kb, int* rows_per_table) {
  int l = 1;
  if (family == ORC_CROSSPOLYTOPE) {
    l = 0;
    while ((1L << l) < 2L * d) ++l;
  }
  int F = 32 / l;
  if (ell) *ell = l;
  if (fns) *fns = F;
  if (Kb) *Kb = F * l;
  if (rows_per_table) *rows_per_table = (family == ORC_CROSSPOLYTOPE) ? F * d : 32;
}

void orc_gen_hash_params(uint64_t seed, int family, int L, int d, float* A) {
  int rows;
  orc_layout(family, d, NULL, NULL, NULL, &rows);
#pragma omp parallel for schedule(static)
  for (int j = 0; j < L; ++j)
    for (int r = 0; r < rows; ++r)
      for (int i = 0; i < d; ++i)
        A[((int64_t)j * rows + r) * d + i] = orc_gauss(seed, ORC_PURPOSE_HASH, (uint32_t)j, (uint32_t)r, (uint32_t)i);
}

void orc_gen_sketch_params(uint64_t seed, int M, int d, float* S) {
#pragma omp parallel for schedule(static)
  for (int r = 0; r < M * 64; ++r)
    for (int i = 0; i < d; ++i)
      S[(int64_t)r * d + i] = orc_gauss(seed, ORC_PURPOSE_SKETCH, 0u, (uint32_t)r, (uint32_t)i);
}

/* Sec. 4.2 "Vector storage": all vectors are normalised.  Reading: the squared
 * norm is summed in FP64 in index order (float*float products are exact in
 * FP64), sqrt and the division are correctly rounded FP64, the quotient is
 * rounded once to float.  A zero vector stays zero. */
void orc_normalize(const float* x, int64_t n, int d, float* out) {
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < n; ++p) {
    const float* row = x + p * d;
    double ss = 0.0;
    for (int i = 0; i < d; ++i) ss = ss + (double)row[i] * (double)row[i];
    double nrm = sqrt(ss);
    for (int i = 0; i < d; ++i) out[p * d + i] = (nrm > 0.0) ? (float)((double)row[i] / nrm) : 0.0f;
  }
}

/* FP64 projection <a, x>, index order. */
static double dot64(const float* a, const float* x, int d) {
  double s = 0.0;
  for (int i = 0; i < d; ++i) s = s + (double)a[i] * (double)x[i];
  return s;
}

/* out[r] = <A_r, x> in FP64 for the rows r = 0..nrows-1 of A ([nrows][d]), each
 * sum formed in index order exactly as dot64 forms it; the rows' sums are
 * independent and are simply advanced side by side. */
static void dot64_rows(const float* A, int nrows, const float* x, int d, double* out) {
  int r = 0;
  for (; r + 4 <= nrows; r += 4) {
    const float* a0 = A + (int64_t)r * d;
    const float* a1 = a0 + d;
    const float* a2 = a1 + d;
    const float* a3 = a2 + d;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int i = 0; i < d; ++i) {
      const double xi = (double)x[i];
      s0 = s0 + (double)a0[i] * xi;
      s1 = s1 + (double)a1[i] * xi;
      s2 = s2 + (double)a2[i] * xi;
      s3 = s3 + (double)a3[i] * xi;
    }
    out[r] = s0; out[r + 1] = s1; out[r + 2] = s2; out[r + 3] = s3;
  }
  for (; r < nrows; ++r) out[r] = dot64(A + (int64_t)r * d, x, d);
}

/* Sec. 2.2: HP bit = 1 iff <a, x> >= 0.  CP: the index c of the hyperplane
 * with the largest |<a_c, x>| and whether that projection is negative.
 * Reading: the l-bit CP value is (sign << (l-1)) | c with sign = [v_c < 0];
 * ties of |v| go to the smaller c.  Function 0 occupies the most significant
 * bits of the 32-bit code (so "dropping the last bit", Sec. 4.3, drops the
 * least significant used bit). */
void orc_hash_one(int family, int L, int d, const float* A, const float* x, uint32_t* codes_out) {
  int ell, F, Kb, rows;
  orc_layout(family, d, &ell, &F, &Kb, &rows);
  double* v = (double*)malloc(sizeof(double) * (size_t)(rows > d ? rows : d));
  for (int j = 0; j < L; ++j) {
    const float* Aj = A + (int64_t)j * rows * d;
    uint32_t code = 0;
    for (int f = 0; f < F; ++f) {
      uint32_t value;
      if (family == ORC_SIMHASH) {
        dot64_rows(Aj + (int64_t)f * d, 1, x, d, v);
        value = v[0] >= 0.0 ? 1u : 0u;
      } else {
        dot64_rows(Aj + (int64_t)f * d * d, d, x, d, v); /* the d projections of function f */
        int best = 0;
        double best_abs = -1.0, best_v = 0.0;
        for (int c = 0; c < d; ++c)
          if (fabs(v[c]) > best_abs) { best_abs = fabs(v[c]); best = c; best_v = v[c]; }
        value = ((best_v < 0.0 ? 1u : 0u) << (ell - 1)) | (uint32_t)best;
      }
      code |= value << (32 - ell * (f + 1));
    }
    codes_out[j] = code;
  }
  free(v);
}

/* v[r] = <row r, x> in FP64 for the rows of one table, the table given
 * transposed (At[i][r] = (double)A[r][i]).  Each v[r] is summed in index order
 * exactly as dot64 sums it; eight rows are advanced side by side. */
#define ORC_ROW_BLOCK 8
static void project_rows_t(const double* At, int rows, const float* x, int d, double* v) {
  int r0 = 0;
  for (; r0 + ORC_ROW_BLOCK <= rows; r0 += ORC_ROW_BLOCK) {
    double acc[ORC_ROW_BLOCK] = {0.0};
    for (int i = 0; i < d; ++i) {
      const double xi = (double)x[i];
      const double* a = At + (int64_t)i * rows + r0;
      for (int u = 0; u < ORC_ROW_BLOCK; ++u) acc[u] = acc[u] + a[u] * xi;
    }
    for (int u = 0; u < ORC_ROW_BLOCK; ++u) v[r0 + u] = acc[u];
  }
  for (int r = r0; r < rows; ++r) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) s = s + At[(int64_t)i * rows + r] * (double)x[i];
    v[r] = s;
  }
}

/* The code of one table from its rows' projections v (the decisions of
 * orc_hash_one). */
static uint32_t code_from_projections(int family, int ell, int F, int d, const double* v) {
  uint32_t code = 0;
  for (int f = 0; f < F; ++f) {
    uint32_t value;
    if (family == ORC_SIMHASH) {
      value = v[f] >= 0.0 ? 1u : 0u;
    } else {
      const double* vf = v + (int64_t)f * d;
      int best = 0;
      double best_abs = -1.0, best_v = 0.0;
      for (int c = 0; c < d; ++c)
        if (fabs(vf[c]) > best_abs) { best_abs = fabs(vf[c]); best = c; best_v = vf[c]; }
      value = ((best_v < 0.0 ? 1u : 0u) << (ell - 1)) | (uint32_t)best;
    }
    code |= value << (32 - ell * (f + 1));
  }
  return code;
}

/* The same codes as orc_hash_one, for n points: points are taken in blocks,
 * and each table's rows are transposed to float64 once per block. */
void orc_hash_codes(int family, int L, int d, const float* A, const float* x, int64_t n, uint32_t* codes) {
  int ell, F, Kb, rows;
  orc_layout(family, d, &ell, &F, &Kb, &rows);
  const int64_t P = 256;
  const int64_t nblocks = (n + P - 1) / P;
#pragma omp parallel
  {
    double* At = (double*)malloc(sizeof(double) * (size_t)rows * (size_t)d);
    double* v = (double*)malloc(sizeof(double) * (size_t)rows);
#pragma omp for schedule(dynamic, 1)
    for (int64_t b = 0; b < nblocks; ++b) {
      const int64_t p0 = b * P, p1 = (p0 + P < n) ? p0 + P : n;
      for (int j = 0; j < L; ++j) {
        const float* Aj = A + (int64_t)j * rows * d;
        for (int r = 0; r < rows; ++r)
          for (int i = 0; i < d; ++i) At[(int64_t)i * rows + r] = (double)Aj[(int64_t)r * d + i];
        for (int64_t p = p0; p < p1; ++p) {
          project_rows_t(At, rows, x + p * d, d, v);
          codes[(int64_t)j * n + p] = code_from_projections(family, ell, F, d, v);
        }
      }
    }
    free(At);
    free(v);
  }
}

/* Sec. 3.3 / 4.2: M sketches of 64 HP bits each. */
void orc_sketches(int M, int d, const float* S, const float* x, int64_t n, uint64_t* sk) {
  const int rows = 64 * M;
  double* St = (double*)malloc(sizeof(double) * (size_t)rows * (size_t)d);
  for (int r = 0; r < rows; ++r)
    for (int i = 0; i < d; ++i) St[(int64_t)i * rows + r] = (double)S[(int64_t)r * d + i];
#pragma omp parallel
  {
    double* v = (double*)malloc(sizeof(double) * (size_t)rows);
#pragma omp for schedule(dynamic, 64)
    for (int64_t p = 0; p < n; ++p) {
      project_rows_t(St, rows, x + p * d, d, v);
      for (int m = 0; m < M; ++m) {
        uint64_t w = 0;
        for (int b = 0; b < 64; ++b)
          if (v[m * 64 + b] >= 0.0) w |= (uint64_t)1 << b;
        sk[(int64_t)m * n + p] = w;
      }
    }
    free(v);
  }
  free(St);
}

/* Sec. 3.2 "Pooling" / App. B.2: the tables share a pool of m functions; table
 * j uses F of them, an independent uniformly random subset.  Reading: the
 * subset is drawn by a partial Fisher-Yates shuffle of 0..m-1 whose swap
 * partner at step s is s + floor(w * (m - s) / 2^32), w the first word of the
 * generator at counter (s, j, 0, purpose 7); position s of the subset gives the
 * value in bits 32 - l(s+1) .. 32 - l s - 1 of the code. */
void orc_pool_select(uint64_t seed, int L, int F, int m, int32_t* sel) {
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  for (int j = 0; j < L; ++j) {
    for (int t = 0; t < m; ++t) perm[t] = t;
    for (int st = 0; st < F && st < m; ++st) {
      uint32_t ctr[4] = {(uint32_t)st, (uint32_t)j, 0u, ORC_PURPOSE_POOL_SELECT};
      uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
      uint32_t w[4];
      orc_philox4x32_10(ctr, key, w);
      int r = st + (int)(((uint64_t)w[0] * (uint64_t)(m - st)) >> 32);
      int32_t tmp = perm[st]; perm[st] = perm[r]; perm[r] = tmp;
      sel[(int64_t)j * F + st] = perm[st];
    }
  }
  free(perm);
}

/* The pool's functions: CP function f has hyperplanes (f, c), c < d; HP
 * function f one hyperplane; entries N(0,1) at counter (i, c, f, purpose 6). */
void orc_gen_pool_params(uint64_t seed, int family, int m, int d, float* A) {
  const int R = family == ORC_CROSSPOLYTOPE ? d : 1;
#pragma omp parallel for schedule(static)
  for (int f = 0; f < m; ++f)
    for (int c = 0; c < R; ++c)
      for (int i = 0; i < d; ++i)
        A[((int64_t)f * R + c) * d + i] = orc_gauss(seed, ORC_PURPOSE_POOL, (uint32_t)f, (uint32_t)c, (uint32_t)i);
}

void orc_pool_codes(int family, int m, int d, const float* A, int L, const int32_t* sel, const float* x, int64_t n,
                    uint32_t* codes) {
  int ell, F;
  orc_layout(family, d, &ell, &F, NULL, NULL);
  const int R = family == ORC_CROSSPOLYTOPE ? d : 1;
#pragma omp parallel
  {
    uint32_t* val = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)m);
    double* v = (double*)malloc(sizeof(double) * (size_t)R);
#pragma omp for schedule(dynamic, 64)
    for (int64_t p = 0; p < n; ++p) {
      for (int f = 0; f < m; ++f) { /* every pool function's value (Sec. 2.2) */
        dot64_rows(A + (int64_t)f * R * d, R, x + p * d, d, v);
        if (family == ORC_SIMHASH) {
          val[f] = v[0] >= 0.0 ? 1u : 0u;
        } else {
          int best = 0;
          double best_abs = -1.0;
          for (int c = 0; c < d; ++c)
            if (fabs(v[c]) > best_abs) { best_abs = fabs(v[c]); best = c; }
          val[f] = ((v[best] < 0.0 ? 1u : 0u) << (ell - 1)) | (uint32_t)best;
        }
      }
      for (int j = 0; j < L; ++j) {
        uint32_t code = 0;
        for (int st = 0; st < F; ++st) code |= val[sel[(int64_t)j * F + st]] << (32 - ell * (st + 1));
        codes[(int64_t)j * n + p] = code;
      }
    }
    free(val);
    free(v);
  }
}

/* Sec. 4.2: repetition j is the array of (code, pos) sorted by code; equal
 * codes keep increasing pos (reading: ties ordered by position). */
typedef struct { uint32_t code, id; } orc_pair;
static int cmp_pair(const void* a, const void* b) {
  const orc_pair* x = (const orc_pair*)a;
  const orc_pair* y = (const orc_pair*)b;
  if (x->code != y->code) return x->code < y->code ? -1 : 1;
  if (x->id != y->id) return x->id < y->id ? -1 : 1;
  return 0;
}

void orc_sort_tables(int L, int64_t n, const uint32_t* codes, uint32_t* sorted_codes, uint32_t* ids) {
#pragma omp parallel
  {
    orc_pair* buf = (orc_pair*)malloc(sizeof(orc_pair) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 1)
    for (int j = 0; j < L; ++j) {
      for (int64_t p = 0; p < n; ++p) { buf[p].code = codes[(int64_t)j * n + p]; buf[p].id = (uint32_t)p; }
      qsort(buf, (size_t)n, sizeof(orc_pair), cmp_pair);
      for (int64_t p = 0; p < n; ++p) { sorted_codes[(int64_t)j * n + p] = buf[p].code; ids[(int64_t)j * n + p] = buf[p].id; }
    }
    free(buf);
  }
}

/* Sec. 4.2: the lexicographic position of every 13-bit prefix is tabulated.
 * pfx[t] = number of entries whose top 13 bits are < t, t = 0..8192. */
void orc_prefix_table(int L, int64_t n, const uint32_t* sorted_codes, uint32_t* pfx) {
  const int T = 1 << ORC_PREFIX_BITS;
#pragma omp parallel for schedule(static)
  for (int j = 0; j < L; ++j) {
    uint32_t* out = pfx + (int64_t)j * (T + 1);
    const uint32_t* c = sorted_codes + (int64_t)j * n;
    int64_t p = 0;
    for (int t = 0; t <= T; ++t) {
      while (p < n && (int64_t)(c[p] >> (32 - ORC_PREFIX_BITS)) < t) ++p;
      out[t] = (uint32_t)p;
    }
  }
}

/* Sec. 4.3: similarities enumerated in windows of 0.05 from -1 to 1. */
double orc_alpha(int t) { return (double)(5 * t - 100) / 100.0; }

/* Sec. 4.3 "round the distance down": reading = round the similarity down to
 * the grid (the smaller similarity bounds the collision probability from
 * below, which is what the stop test of Lemma 1 needs). */
int orc_alpha_index(double s) {
  int t = 0;
  for (int u = 0; u < ORC_ALPHA_STEPS; ++u)
    if (orc_alpha(u) <= s) t = u;
  return t;
}

/* CP value of a vector whose projections are v[0..d). */
static uint32_t cp_value(const double* v, int d, int ell) {
  int best = 0;
  double best_abs = -1.0;
  for (int c = 0; c < d; ++c)
    if (fabs(v[c]) > best_abs) { best_abs = fabs(v[c]); best = c; }
  return ((v[best] < 0.0 ? 1u : 0u) << (ell - 1)) | (uint32_t)best;
}

/* Sec. 4.3: x = (1,0,...,0), y = (alpha, sqrt(1-alpha^2), 0, ...); draw CP
 * functions and count how often the first r bits of h(x) and h(y) agree, for
 * every r = 0..l.  Readings: the same draws serve every alpha; the table is
 * then made non-decreasing in alpha by taking, at each grid point, the minimum
 * over all larger grid points (a lower bound on a monotone function). */
void orc_cp_table(uint64_t seed, int d, int draws, double* P) {
  int ell;
  orc_layout(ORC_CROSSPOLYTOPE, d, &ell, NULL, NULL, NULL);
  const int W = ell + 1;
  double* vx = (double*)malloc(sizeof(double) * (size_t)d);
  double* vy = (double*)malloc(sizeof(double) * (size_t)d);
  float* a0 = (float*)malloc(sizeof(float) * (size_t)d);
  float* a1 = (float*)malloc(sizeof(float) * (size_t)d);
  int64_t* hits = (int64_t*)calloc((size_t)(ORC_ALPHA_STEPS * W), sizeof(int64_t));
  for (int t = 0; t < draws; ++t) {
    for (int c = 0; c < d; ++c) {
      a0[c] = orc_gauss(seed, ORC_PURPOSE_CPMC, (uint32_t)t, (uint32_t)c, 0u);
      a1[c] = orc_gauss(seed, ORC_PURPOSE_CPMC, (uint32_t)t, (uint32_t)c, 1u);
    }
    for (int g = 0; g < ORC_ALPHA_STEPS; ++g) {
      double alpha = orc_alpha(g);
      double beta = sqrt(1.0 - alpha * alpha);
      for (int c = 0; c < d; ++c) {
        vx[c] = (double)a0[c];
        vy[c] = alpha * (double)a0[c] + beta * (double)a1[c];
      }
      uint32_t hx = cp_value(vx, d, ell), hy = cp_value(vy, d, ell);
      for (int r = 0; r <= ell; ++r)
        if ((hx >> (ell - r)) == (hy >> (ell - r))) hits[g * W + r] += 1;
    }
  }
  for (int g = 0; g < ORC_ALPHA_STEPS; ++g)
    for (int r = 0; r <= ell; ++r) P[g * W + r] = (double)hits[g * W + r] / (double)draws;
  for (int g = ORC_ALPHA_STEPS - 2; g >= 0; --g)
    for (int r = 0; r <= ell; ++r)
      if (P[(g + 1) * W + r] < P[g * W + r]) P[g * W + r] = P[(g + 1) * W + r];
  free(vx); free(vy); free(a0); free(a1); free(hits);
}

/* x^e by binary exponentiation (square-and-multiply), pinned order. */
double orc_ipow(double x, int64_t e) {
  double result = 1.0, base = x;
  while (e > 0) {
    if (e & 1) result = result * base;
    base = base * base;
    e >>= 1;
  }
  return result;
}

/* Probability that a point at similarity s collides with the query on the
 * first `depth` bits of one table.  HP (Sec. 4.3: "easy to derive"):
 * p = 1 - arccos(s)/pi per bit.  CP: the tabulated probability of the full
 * l-bit value for each complete function and the r-bit entry for the partial
 * last one (functions are independent). */
double orc_collision_prob(int family, int ell, const double* P, double s, int depth) {
  if (family == ORC_SIMHASH) {
    double sc = s > 1.0 ? 1.0 : (s < -1.0 ? -1.0 : s);
    double p = 1.0 - acos(sc) / M_PI;
    return orc_ipow(p, depth);
  }
  int g = orc_alpha_index(s);
  const double* row = P + g * (ell + 1);
  return orc_ipow(row[ell], depth / ell) * row[depth % ell];
}

/* App. B.2 adapted to general delta.  X = number of the j tables, searched to
 * prefix length i, in which x_k collides with the query; E[X] = mu = j p_i
 * (the functions within one table are distinct pool members, so independent).
 * For two tables, each of the f = ceil(i/l) functions behind the first i bits
 * of the second is one of the first's with probability <= f/(m - f), so
 * E[X_1 X_2] <= p_i^2 (1 + f / ((m - f) P))^f <= p_i^2 e^c, c = f^2/((m - f) P),
 * P = the collision probability of one whole function (the smallest factor).
 * Hence Var X <= mu + mu^2 (e^c - 1), and Cantelli's inequality gives
 * Pr[X = 0] <= Var/(mu^2 + Var).  Reading: e^c - 1 is replaced by its upper
 * bound c/(1 - c) (c < 1), so the test needs no exponential; stop iff that
 * bound is <= delta.  (With c -> 0 the bound is 1/(1 + mu); the paper's
 * rule for delta = 1/2 is mu >= 2 and m >= 5 i^2 / P.) */
int orc_pool_stop(int family, int ell, const double* P, int m, double s_k, int depth, int64_t j, double delta) {
  const int f = (depth + ell - 1) / ell;
  if (f <= 0 || f >= m || j <= 0) return 0;
  const double p = orc_collision_prob(family, ell, P, s_k, depth);
  const double p1 = orc_collision_prob(family, ell, P, s_k, ell);
  if (!(p1 > 0.0)) return 0;
  const double c = ((double)f * (double)f) / ((double)(m - f) * p1);
  if (!(c < 1.0)) return 0;
  const double mu = (double)j * p;
  if (!(mu > 0.0)) return 0;
  const double var = mu + (mu * mu) * (c / (1.0 - c));
  return var / (mu * mu + var) <= delta;
}

/* Sec. 4.2 + Fig. 2 footnote: the sketch threshold is (1+eps) times the
 * expected number of differing bits, 64 * arccos(s_k)/pi, with eps = 0
 * (Sec. 5.1); a candidate passes if its Hamming distance is at most that.
 * Since the distance is an integer this is floor(64 arccos(s_k)/pi), computed
 * without arccos as the largest t with cos(t pi / 64) >= s_k. */
int orc_filter_tau(double s_k) { return orc_filter_tau_eps(s_k, 0.0); }

/* With the footnote's slack eps >= 0: the largest t with
 * t <= (1 + eps) 64 arccos(s_k)/pi, i.e. cos(t pi / (64 (1 + eps))) >= s_k. */
int orc_filter_tau_eps(double s_k, double eps) {
  int tau = 0;
  for (int t = 0; t <= 64; ++t)
    if (cos((double)t * M_PI / (64.0 * (1.0 + eps))) >= s_k) tau = t;
  return tau;
}

/* Sec. 5 ("Influence of the Index Size"): the budget covers the stored data,
 * the hash functions and the tables.  Reading: bytes of the layout the GPU
 * library keeps resident, with d' = d rounded up to a multiple of 16:
 *   fixed     = n d' (4 + 2)   rows as float32 and bfloat16
 *             + 64 M d' 6      sketch planes (float32 + their exact bfloat16 copy)
 *             + n M 8          the M sketches of every point (layout 1 only)
 *   per table = n (4 + 4)      sorted codes and positions
 *             + n 8            the sketch of each entry (layout 0 only)
 *             + 8193 * 4       prefix table
 *             + R d' 6         hash rows (float32 + their exact bfloat16 copy),
 *               R = F * d' for CP (rows of a function padded to d'), 32 for HP
 *   L = floor((budget - fixed) / per_table). */
int64_t orc_budget_L(int family, int64_t n, int d, int M, uint64_t budget_bytes, int sketch_layout,
                     int row_storage, int fp8_rows, int pool_fns) {
  int64_t dp = ((int64_t)d + 15) / 16 * 16;
  int F;
  orc_layout(family == ORC_CROSSPOLYTOPE_FHT ? ORC_CROSSPOLYTOPE : family, d, NULL, &F, NULL, NULL);
  int64_t R = (family == ORC_CROSSPOLYTOPE) ? (int64_t)F * dp : (family == ORC_SIMHASH ? 32 : 0);
  /* pseudo-random CP (Sec. 4.3): a function keeps three random sign vectors
   * of d'' = 2^ceil(log2 d) bits, in 32-bit words (at least one) */
  int64_t fht_bytes = 0;
  if (family == ORC_CROSSPOLYTOPE_FHT) {
    int64_t dpp = 1;
    while (dpp < d) dpp *= 2;
    fht_bytes = (int64_t)F * 3 * (dpp < 32 ? 1 : dpp / 32) * 4;
  }
  /* rows: float32 (4 B) or binary16 (2 B) per element, plus the bfloat16 copy (2 B) */
  int64_t row_bytes = row_storage == 1 ? 4 : 6;
  int64_t fixed = n * dp * row_bytes + 64 * (int64_t)M * dp * 6 + (sketch_layout == 1 ? n * (int64_t)M * 8 : 0);
  /* an 8-bit float copy of the rows, with a scale and an error bound each */
  if (fp8_rows) fixed += n * (dp + 8);
  /* pooled functions (Sec. 3.2): the pool's rows, stored in whole groups of F
   * functions, are fixed; a table keeps only its F indices */
  if (pool_fns > 0) {
    int64_t groups = (pool_fns + F - 1) / F;
    fixed += groups * R * dp * 6;
    R = 0;
  }
  int64_t per_table = n * (sketch_layout == 1 ? 8 : 16) + (int64_t)((1 << ORC_PREFIX_BITS) + 1) * 4 + R * dp * 6 +
                      fht_bytes + (pool_fns > 0 ? (int64_t)F * 4 : 0);
  if ((int64_t)budget_bytes <= fixed) return 0;
  return ((int64_t)budget_bytes - fixed) / per_table;
}

/* Canonical float32 inner product (reading: the paper's 16-bit fixed point
 * product is replaced by float32): 32 partial sums, partial c accumulating the
 * coordinates i = c (mod 32) in increasing i with fused multiply-add, then
 * combined pairwise as s[c] += s[c + w] for w = 16, 8, 4, 2, 1. */
float orc_sim(const float* q, const float* x, int d) {
  float s[32];
  for (int c = 0; c < 32; ++c) s[c] = 0.0f;
  for (int i = 0; i < d; ++i) s[i & 31] = fmaf(q[i], x[i], s[i & 31]);
  for (int w = 16; w >= 1; w >>= 1)
    for (int c = 0; c < w; ++c) s[c] = s[c] + s[c + w];
  return s[0];
}

/* ---- accumulator (Sec. 4.2 "Computing distances"): the k best unique
 *      points, ordered by similarity descending and position ascending ---- */
static int better(float s1, uint32_t id1, float s2, uint32_t id2) {
  return s1 > s2 || (s1 == s2 && id1 < id2);
}

static void pq_insert(float* ps, uint32_t* pid, int* size, int k, float s, uint32_t id) {
  for (int t = 0; t < *size; ++t)
    if (pid[t] == id) return; /* de-duplicate */
  if (*size == k && !better(s, id, ps[k - 1], pid[k - 1])) return;
  int pos = (*size < k) ? (*size)++ : k - 1;
  while (pos > 0 && better(s, id, ps[pos - 1], pid[pos - 1])) {
    ps[pos] = ps[pos - 1];
    pid[pos] = pid[pos - 1];
    --pos;
  }
  ps[pos] = s;
  pid[pos] = id;
}

static int64_t lower_bound_u32(const uint32_t* a, int64_t n, uint32_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

static int64_t upper_bound_u32(const uint32_t* a, int64_t n, uint32_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (a[mid] <= key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

static int popcount64(uint64_t w) {
  int c = 0;
  while (w) { w &= w - 1; ++c; }
  return c;
}

/* Algorithm 1 as implemented in Sec. 4.1-4.2, one query:
 *   - rounds at prefix length i = i0, i0-1, ..., 0 with i0 = K (Sec. 4.1) or
 *     a given start depth in [0, K) (the first round then takes the whole
 *     block at i0, so every candidate of the skipped rounds is still seen);
 *   - in a round every repetition j extends its range [l, r) to cover the
 *     block of codes sharing the first i bits with the query, growing each
 *     side in whole segments of B entries (Sec. 4.2, App. C), and visits the
 *     new positions;
 *   - a visited point is dropped if i > 0 and the Hamming distance of sketch
 *     (j mod M) exceeds tau; otherwise its similarity is computed and it is
 *     offered to the accumulator;
 *   - after the round: stop at i = 0 (a linear scan, Lemma 1), or when the
 *     accumulator holds k points and (1 - p_i(s_k))^L <= delta (Lemma 1).
 * Readings: the paper refreshes the accumulator (and so tau) after every k
 * insertions, in the order repetitions are inspected (Sec. 4.2); here tau is
 * taken from the accumulator at the start of each round and, in a query's first
 * round (which starts with an empty accumulator), also before repetitions
 * 1, 2, 4, 8, 16 and every 32 after that, so within a group the visiting order
 * does not matter.  The stop test runs once per round (Sec. 4.1); the
 * initial range of a repetition is empty at the first position whose code is
 * >= the query code. */
/* Reading of the accumulator's refresh in a first round (Sec. 4.2): snapshots
 * before repetitions 1, 2, 4, 8, 16 and then every 32 (the first repetitions'
 * blocks fill the top-k, so the threshold tightens early). */
static int first_round_snapshot(int j) {
  return j < ORC_SNAPSHOT_GROUP ? (j & (j - 1)) == 0 : j % ORC_SNAPSHOT_GROUP == 0;
}

static void search_one(const orc_index* ix, const float* q, const uint32_t* qcode, const uint64_t* qsk,
                       int k, double recall, int k_max, int32_t start_depth, int filter, int stop_every,
                       uint32_t* out_ids, float* out_sims, orc_stats* st,
                       uint32_t* trace, int64_t trace_cap, int64_t* trace_len) {
  const int64_t n = ix->n;
  const int L = ix->L, Kb = ix->Kb, B = ix->B, M = ix->M;
  const double delta = 1.0 - recall;
  int64_t* l = (int64_t*)malloc(sizeof(int64_t) * (size_t)L);
  int64_t* r = (int64_t*)malloc(sizeof(int64_t) * (size_t)L);
  float* ps = (float*)malloc(sizeof(float) * (size_t)(k > 0 ? k : 1));
  uint32_t* pid = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(k > 0 ? k : 1));
  int size = 0;
  int64_t tl = 0;
  orc_stats s = {0, 0, 0, -1, 0, 0, 0, 0};

  for (int j = 0; j < L; ++j) {
    l[j] = r[j] = lower_bound_u32(ix->codes + (int64_t)j * n, n, qcode[j]);
  }
  int i0 = Kb;
  if (start_depth >= 0 && start_depth < Kb) i0 = start_depth;
  s.start_depth = i0;

  int depth = i0;
  int stopped = 0;
  for (;;) {
    const uint32_t mask = depth == 0 ? 0u : (0xFFFFFFFFu << (32 - depth));
    int tau = 64;
    for (int j = 0; j < L; ++j) {
      if (j == 0 || (stop_every > 0 ? j % stop_every == 0
                                    : (s.rounds == 0 && first_round_snapshot(j)))) { /* threshold snapshot */
        const int full = (size == k);
        tau = full ? orc_filter_tau_eps((double)ps[k - 1], ix->filter_eps) : 64;
      }
      const uint32_t* cj = ix->codes + (int64_t)j * n;
      const uint32_t* idj = ix->ids + (int64_t)j * n;
      int64_t lo = lower_bound_u32(cj, n, qcode[j] & mask);
      int64_t hi = upper_bound_u32(cj, n, qcode[j] | ~mask);
      int64_t nl = l[j], nr = r[j];
      if (lo < l[j]) { nl = l[j] - (int64_t)B * ((l[j] - lo + B - 1) / B); if (nl < 0) nl = 0; }
      if (hi > r[j]) { nr = r[j] + (int64_t)B * ((hi - r[j] + B - 1) / B); if (nr > n) nr = n; }
      for (int side = 0; side < 2; ++side) {
        int64_t a = side == 0 ? nl : r[j];
        int64_t b = side == 0 ? l[j] : nr;
        for (int64_t p = a; p < b; ++p) {
          uint32_t id = idj[p];
          s.retrieved += 1;
          const int64_t slot = tl++;
          if (trace && slot < trace_cap) trace[2 * slot] = ((uint32_t)depth << 24) | (uint32_t)j, trace[2 * slot + 1] = id;
          if (filter && depth > 0) {
            int ham = popcount64(qsk[j % M] ^ ix->sk[(int64_t)(j % M) * n + id]);
            if (ham > tau) continue;
          }
          if (trace && slot < trace_cap) trace[2 * slot] |= 0x80000000u; /* scored */
          s.passed_filter += 1;
          s.scored += 1;
          float sim = orc_sim(q, ix->x + (int64_t)id * ix->d, ix->d);
          pq_insert(ps, pid, &size, k, sim, id);
        }
      }
      l[j] = nl;
      r[j] = nr;
      if (stop_every > 0 && depth > 0 && size == k && ((j + 1) % stop_every == 0 || j + 1 == L)) {
        /* Alg. 1 tests after repetitions, not rounds: repetitions 0..j have
         * now been searched to prefix length `depth`, the others to depth + 1
         * (to nothing yet in the first round, whose factor is 1) */
        int stop_now;
        if (ix->pool_fns > 0 && !ix->pool_as_independent) { /* pooled functions: only the j + 1 tables at this depth are counted */
          stop_now = orc_pool_stop(ix->family, ix->ell, ix->P, ix->pool_fns, (double)ps[k - 1], depth, j + 1, delta);
        } else {
          double fail =
              orc_ipow(1.0 - orc_collision_prob(ix->family, ix->ell, ix->P, (double)ps[k - 1], depth), j + 1);
          if (s.rounds > 0)
            fail = fail * orc_ipow(1.0 - orc_collision_prob(ix->family, ix->ell, ix->P, (double)ps[k - 1], depth + 1),
                                   L - j - 1);
          stop_now = fail <= delta;
        }
        if (stop_now) { stopped = j + 1; break; }
      }
    }
    s.last_reps = stopped ? stopped : L;
    s.rounds += 1;
    s.stop_depth = depth;
    if (size == k && s.full_depth < 0) s.full_depth = depth;
    if (stopped) break;
    if (depth == 0) break;
    if (size == k) {
      if (ix->pool_fns > 0 && !ix->pool_as_independent) {
        if (orc_pool_stop(ix->family, ix->ell, ix->P, ix->pool_fns, (double)ps[k - 1], depth, L, delta)) break;
      } else {
        double p = orc_collision_prob(ix->family, ix->ell, ix->P, (double)ps[k - 1], depth);
        double fail = orc_ipow(1.0 - p, L);
        if (fail <= delta) break;
      }
    }
    depth -= 1;
  }
  for (int t = 0; t < k_max; ++t) {
    out_ids[t] = t < size ? pid[t] : 0xFFFFFFFFu;
    out_sims[t] = t < size ? ps[t] : -INFINITY;
  }
  if (st) *st = s;
  if (trace_len) *trace_len = tl;
  free(l); free(r); free(ps); free(pid);
}

void orc_search(const orc_index* ix, const float* q, const uint32_t* qcodes, const uint64_t* qsk,
                int64_t Q, const int32_t* k, const double* recall, int32_t k_max,
                const int32_t* start_depth, int filter, int stop_every,
                uint32_t* out_ids, float* out_sims, orc_stats* stats,
                uint32_t* trace, int64_t trace_cap, int64_t* trace_len) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t t = 0; t < Q; ++t) {
    search_one(ix, q + t * ix->d, qcodes + t * ix->L, qsk + t * ix->M, k[t], recall[t], k_max,
               start_depth ? start_depth[t] : -1, filter, stop_every, out_ids + t * k_max, out_sims + t * k_max,
               stats ? stats + t : NULL, trace ? trace + 2 * t * trace_cap : NULL, trace_cap,
               trace_len ? trace_len + t : NULL);
  }
}

void orc_brute_force(const float* x, int64_t n, int d, const float* q, int64_t Q, int k,
                     uint32_t* out_ids, float* out_sims) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t t = 0; t < Q; ++t) {
    float* ps = (float*)malloc(sizeof(float) * (size_t)(k > 0 ? k : 1));
    uint32_t* pid = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(k > 0 ? k : 1));
    int size = 0;
    for (int64_t p = 0; p < n; ++p)
      pq_insert(ps, pid, &size, k, orc_sim(q + t * d, x + p * d, d), (uint32_t)p);
    for (int u = 0; u < k; ++u) {
      out_ids[t * k + u] = u < size ? pid[u] : 0xFFFFFFFFu;
      out_sims[t * k + u] = u < size ? ps[u] : -INFINITY;
    }
    free(ps); free(pid);
  }
}
