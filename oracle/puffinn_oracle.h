/*
 * puffinn_oracle.h -- plain, slow, obviously-correct CPU statement of PUFFINN's
 * LSH-forest index and adaptive k-NN query (Aumueller, Christiani, Pagh,
 * Vesterli, "PUFFINN: Parameterless and Universally Fast FInding of Nearest
 * Neighbors", ESA 2019).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this code; only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no source, header, table or helper with the
 * CUDA library: both sides were written separately from the paper.
 *
 * Every function states the passage of the paper it follows.  Where the paper
 * leaves a detail open, the reading taken is stated next to the function.
 *
 * Conventions
 *   - points / queries: row-major float32 [n][d] (no padding here).
 *   - codes: uint32, first hash function in the most significant bits,
 *     unused low bits zero.
 *   - sketches: uint64, sketch m of point x at sk[m*n + x], bit b (LSB first)
 *     is the b-th hyperplane bit.
 *   - all floating point decisions in FP64 unless stated.
 */
#ifndef PUFFINN_ORACLE_H
#define PUFFINN_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_SIMHASH = 0, ORC_CROSSPOLYTOPE = 1, ORC_CROSSPOLYTOPE_FHT = 2 /* budget rule only (oracle/fht.py) */ };
enum { ORC_PURPOSE_HASH = 1, ORC_PURPOSE_SKETCH = 2, ORC_PURPOSE_CPMC = 3,
       ORC_PURPOSE_POOL = 6 /* rows of the pooled functions */, ORC_PURPOSE_POOL_SELECT = 7 /* their subsets */ };
#define ORC_PREFIX_BITS 13
#define ORC_ALPHA_STEPS 41 /* similarity grid -1, -0.95, ..., 1 (Sec. 4.3) */
#define ORC_SNAPSHOT_GROUP 32 /* repetitions per sketch-threshold snapshot in a query's first round, after the
                                 geometric start 1, 2, 4, 8, 16 */

/* Host threads of the OpenMP loops (n <= 0: all processors). */
void orc_set_threads(int n);

/* ---- random parameters (counter-based generator, Salmon et al. SC'11) ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* One standard normal per counter (purpose, a, b, c), Box-Muller in FP64,
 * rounded to float32. */
float orc_gauss(uint64_t seed, uint32_t purpose, uint32_t a, uint32_t b, uint32_t c);

/* ---- layout of one table's code (Sec. 4.3: l-bit strings, l=1 for HP,
 *      l=ceil(log2 2d) for CP) ---- */
void orc_layout(int family, int d, int* ell, int* fns, int* Kb, int* rows_per_table);

/* Hash-function parameters: A[L][rows_per_table][d] float32.
 * CP: row f*d + c is hyperplane c of function f.  HP: row b is function b. */
void orc_gen_hash_params(uint64_t seed, int family, int L, int d, float* A);
/* Sketch planes S[M*64][d] float32 (Sec. 3.3 / 4.2). */
void orc_gen_sketch_params(uint64_t seed, int M, int d, float* S);

/* ---- step a1: normalisation (Sec. 4.2 "Vector storage") ---- */
void orc_normalize(const float* x, int64_t n, int d, float* out);

/* ---- hashing (Sec. 2.2 HP and CP definitions, Sec. 4.3 bit strings) ---- */
/* hash one normalised vector under all L tables */
void orc_hash_one(int family, int L, int d, const float* A, const float* x, uint32_t* codes_out /*[L]*/);
/* codes[L][n] for n normalised points (OpenMP over points) */
void orc_hash_codes(int family, int L, int d, const float* A, const float* x, int64_t n, uint32_t* codes);
/* sk[M][n] */
void orc_sketches(int M, int d, const float* S, const float* x, int64_t n, uint64_t* sk);

/* ---- sorted repetition arrays and 13-bit prefix table (Sec. 4.2) ---- */
void orc_sort_tables(int L, int64_t n, const uint32_t* codes, uint32_t* sorted_codes, uint32_t* ids);
void orc_prefix_table(int L, int64_t n, const uint32_t* sorted_codes, uint32_t* pfx /*[L][8193]*/);

/* ---- pooling (Sec. 3.2 "Pooling", App. B.2): a pool of m functions, each
 *      table takes an independent random subset of F of them ---- */
/* sel[L][F]: the subset of table j, drawn without replacement (partial
 * Fisher-Yates driven by the counter-based generator, purpose 7) */
void orc_pool_select(uint64_t seed, int L, int F, int m, int32_t* sel);
/* rows of the pool's functions [m][R][d], R = d (CP) or 1 (HP), purpose 6 */
void orc_gen_pool_params(uint64_t seed, int family, int m, int d, float* A);
/* codes[L][n] of normalised points: table j concatenates the values of its
 * selected functions, the first in the most significant bits */
void orc_pool_codes(int family, int m, int d, const float* A, int L, const int32_t* sel, const float* x, int64_t n,
                    uint32_t* codes);
/* the stop test of a pooled index after j tables searched to prefix length
 * `depth`: Cantelli's bound on Pr[x_k never collided] <= delta (the reading of
 * App. B.2 for general delta) */
int orc_pool_stop(int family, int ell, const double* P, int m, double s_k, int depth, int64_t j, double delta);

/* ---- collision probabilities (Sec. 4.3 "Estimating Collision Probabilities") ---- */
double orc_alpha(int t); /* grid value alpha_t */
int orc_alpha_index(double s);
void orc_cp_table(uint64_t seed, int d, int draws, double* P /*[41][ell+1]*/);
double orc_collision_prob(int family, int ell, const double* P, double s, int depth);
double orc_ipow(double x, int64_t e);

/* ---- sketch filter threshold (Sec. 4.2 "Filtering", Fig. 2 footnote) ---- */
int orc_filter_tau(double s_k);
int orc_filter_tau_eps(double s_k, double eps); /* threshold with slack eps (Fig. 2) */

/* ---- memory budget -> number of repetitions (Sec. 5, index size) ----
 * sketch_layout 0: one sketch copy per repetition entry; 1: M per point.
 * row_storage 0: normalised rows kept in float32; 1: in binary16 (Sec. 4.2
 * keeps 16-bit vectors); a bfloat16 copy is kept either way.  fp8_rows 1: an
 * 8-bit float copy with a scale and a bound per row is kept too.  pool_fns
 * > 0: the tables draw their functions from a pool of that many. */
int64_t orc_budget_L(int family, int64_t n, int d, int M, uint64_t budget_bytes, int sketch_layout,
                     int row_storage, int fp8_rows, int pool_fns);

/* ---- canonical float32 inner product ---- */
float orc_sim(const float* q, const float* x, int d);

/* ---- the query (Algorithm 1, Sec. 4.1) ---- */
typedef struct {
  int32_t start_depth, stop_depth, rounds;
  int32_t full_depth; /* prefix length of the first round after which k points were held, -1 if none */
  int64_t retrieved, passed_filter, scored;
  int32_t last_reps;  /* repetitions searched in the last round (L unless the stop test ran after a group) */
} orc_stats;

typedef struct {
  int family, d, ell, Kb, L, M, B;
  int64_t n;
  const float* x;          /* normalised points [n][d] */
  const uint32_t* codes;   /* sorted codes [L][n] */
  const uint32_t* ids;     /* ids [L][n] */
  const uint64_t* sk;      /* sketches [M][n] */
  const double* P;         /* CP table [41][ell+1] or NULL for HP */
  int pool_fns;            /* 0: independent functions; m > 0: each table draws its functions from a pool of m */
  int pool_as_independent; /* pooled index, 1: stop by Lemma 1's rule as if the functions were independent */
  double filter_eps;       /* slack of the sketch threshold (Fig. 2 footnote; Sec. 5.1 uses 0) */
} orc_index;

/* Search Q normalised queries.  qcodes[Q][L], qsk[Q][M], k[Q], recall[Q].
 * start_depth: NULL (plain schedule K, K-1, ..., 0) or per-query start depth
 * i0 (schedule i0, i0-1, ..., 0; i0 outside [0, K) means K).
 * filter: 0/1.  stop_every: 0 = the stop test once per round (Sec. 4.1);
 * G >= 1 = the test after every G repetitions and after the last (Alg. 1
 * tests after every repetition: G = 1), with fail =
 * (1 - p_i)^j (1 - p_{i+1})^(L - j) after j repetitions at depth i; the
 * threshold is then also refreshed at every group of G repetitions.
 * Outputs [Q][k_max]; stats may be NULL.
 * trace (may be NULL): per query up to trace_cap entries
 * (scored<<31 | depth<<24 | table, id) of every retrieved candidate in the order
 * visited, scored = 1 when it passed the sketch filter and was scored; count
 * in trace_len[q]. */
void orc_search(const orc_index* ix, const float* q, const uint32_t* qcodes, const uint64_t* qsk,
                int64_t Q, const int32_t* k, const double* recall, int32_t k_max,
                const int32_t* start_depth, int filter, int stop_every,
                uint32_t* out_ids, float* out_sims, orc_stats* stats,
                uint32_t* trace, int64_t trace_cap, int64_t* trace_len);

/* exact top-k by canonical similarity, ties by smaller id */
void orc_brute_force(const float* x, int64_t n, int d, const float* q, int64_t Q, int k,
                     uint32_t* out_ids, float* out_sims);

#ifdef __cplusplus
}
#endif
#endif
