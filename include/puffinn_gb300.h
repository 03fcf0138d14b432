/*
 * puffinn_gb300.h -- C ABI of the GB300 (sm_103a) implementation of PUFFINN's
 * LSH-forest index and adaptive k-NN query (Aumueller, Christiani, Pagh,
 * Vesterli, ESA 2019).
 *
 * The user supplies only the points, a memory budget and the hash family at
 * build time, and k plus the recall target 1 - delta at query time (Sec. 1.1,
 * Sec. 5 "Parameter Choices"; Definition 1 of the (k, delta)-NN problem).
 *
 * General conventions
 *   - Pointers are plain host or device addresses; the library detects which
 *     with cudaPointerGetAttributes.  Device pointers must be on the device
 *     that is current when the call is made.  Host inputs are copied to the
 *     device inside the call; host outputs are written before the call returns.
 *   - The caller owns every buffer it passes in; the library never frees or
 *     retains caller memory.  Everything the index needs is copied into
 *     library-owned device memory by pf_index_build.
 *   - stream: a cudaStream_t (NULL = the legacy default stream).  Device work
 *     is ordered on it.  Calls return after synchronising that stream, and the
 *     returned status includes asynchronous device errors.
 *   - No C++ exception, abort or exit crosses this boundary.  On error the
 *     status is negative and pf_last_error_message() (thread-local) explains.
 *   - Layouts are row-major.  n, Q <= 2^31 - 1; ids are uint32 row numbers of
 *     the build input.
 */
#ifndef PUFFINN_GB300_H
#define PUFFINN_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pf_index pf_index; /* opaque, owned by the library */

typedef enum {
  PF_OK = 0,
  PF_ERR_INVALID_ARG = -1,      /* a size, pointer or option is out of range */
  PF_ERR_BUDGET_TOO_SMALL = -2, /* the memory budget leaves room for no repetition */
  PF_ERR_OOM = -3,              /* a device allocation failed */
  PF_ERR_CUDA = -4,             /* a CUDA runtime / driver call or a kernel failed */
  PF_ERR_DEVICE_TIMEOUT = -5,   /* a bounded device-side wait gave up */
  PF_ERR_NOT_TRAINED = -6       /* learned start requested before pf_learned_train */
} pf_status;

typedef enum {
  PF_SIMHASH = 0,       /* random hyperplane LSH, 1 bit per function (Sec. 2.2) */
  PF_CROSSPOLYTOPE = 1,     /* cross-polytope LSH, ceil(log2 2d) bits per function (Sec. 2.2, 4.3) */
  PF_CROSSPOLYTOPE_FHT = 2  /* pseudo-random cross-polytope (Sec. 4.3, after Andoni et al. 2015): the d Gaussian
                               hyperplanes replaced by H D3 H D2 H D1, three Walsh-Hadamard transforms of length
                               d'' = 2^ceil(log2 d) with random sign diagonals; same bits per function */
} pf_family;

typedef enum { PF_F32 = 0 } pf_dtype;

/* Where the 1-bit sketches live (Sec. 4.2 stores M sketches per point and lets
 * repetition j use sketch j mod M).  Both layouts hold the same values and give
 * the same results for the same L; they differ in memory and access pattern. */
typedef enum {
  PF_SKETCH_PER_TABLE = 0, /* default: repetition j keeps, next to its sorted ids, the sketch j mod M of the
                              point at each position (8 more bytes per entry, read contiguously) */
  PF_SKETCH_PER_POINT = 1  /* M sketches per point, gathered by id during the search */
} pf_sketch_layout;

/* Precision in which the normalised rows are kept (Sec. 4.2 keeps 16-bit
 * vectors).  With binary16 the stored point is the round-to-nearest-even
 * binary16 copy of the float64-normalised row: it is what is hashed, and the
 * canonical float32 similarity is taken of it (read back exactly as float32). */
typedef enum {
  PF_ROWS_F32 = 0,  /* default: float32 rows */
  PF_ROWS_F16 = 1   /* binary16 rows: half the row bytes */
} pf_row_storage;

/* Build parameters (Sec. 4.2-4.3).  Zero-initialise and set what you need;
 * zero means "default" for the optional fields. */
typedef struct {
  int64_t n;                    /* number of points, >= 1 */
  int32_t d;                    /* dimension, 1..320 */
  int32_t dtype;                /* pf_dtype of `points` */
  int32_t family;               /* pf_family */
  int32_t num_sketches;         /* M 64-bit sketches per point (Sec. 4.2); 0 -> 32 */
  uint64_t memory_budget_bytes; /* index size budget (Sec. 5); sets the number of repetitions L */
  uint64_t seed;                /* seed of every random draw of the index (hash functions, sketches, CP table) */
  int32_t segment_B;            /* segment size B (Sec. 4.2, App. C); 0 -> 12 */
  int32_t cp_draws;             /* Monte-Carlo draws per similarity for the CP table (Sec. 4.3); 0 -> 1000 */
  int32_t num_tables;           /* if > 0, use exactly this L instead of the budget (tests, sweeps) */
  int32_t sketch_layout;        /* pf_sketch_layout; 0 -> PF_SKETCH_PER_TABLE */
  int32_t row_storage;          /* pf_row_storage; 0 -> PF_ROWS_F32 */
  int32_t fp8_rows;             /* 1: also keep an 8-bit float (e4m3) copy of the rows with a scale and an error
                                   bound per row, for scoring 2; counted in the budget (n * (d_pad + 8) bytes) */
  int32_t pool_bits;            /* 0: independent functions in every table.  m > 0: pooling (Sec. 3.2, App. B.2):
                                   a pool of floor(m / l) functions shared by the tables, each table using a random
                                   subset of fns of them (the paper uses m = 3072).  PF_SIMHASH and
                                   PF_CROSSPOLYTOPE only; the pool must hold at least fns functions */
} pf_build_params;

/* Per-call search options.  NULL = defaults (FP32 scoring, filter on). */
typedef struct {
  int32_t scoring;             /* 0: float32 scoring; 1: bfloat16 estimate + exact float32 rerank; 2: 8-bit float
                                  (e4m3, per-row scale) estimate + exact float32 rerank (an index built with
                                  fp8_rows).  Estimates only drop candidates that provably cannot enter the top-k,
                                  so every mode returns the float32 mode's results */
  int32_t filter;              /* 1: sketch filter on (Sec. 4.2); 0: off.  Set by pf_search_opts_default */
  int32_t learned_start;       /* 1: start depth from the trained model (needs pf_learned_train) */
  int32_t timing;              /* 1: record CUDA events around each phase (see pf_index_last_timing) */
  const int32_t* start_depth;  /* optional [Q] per-query start depth i0 (host or device): rounds i0, i0-1, ..., 0,
                                  the first taking the whole block at i0; values outside [0, K) mean K */
  int32_t pool_rule;           /* pooled index: 0 = stop when Cantelli's bound on missing the k-th point is <= delta
                                  (the guarantee carried to general delta); 1 = Lemma 1's test as if the pooled
                                  functions were independent (no guarantee).  Ignored otherwise */
  double filter_eps;           /* slack of the sketch threshold (Fig. 2 footnote): a candidate passes when its
                                  Hamming distance is <= (1 + eps) 64 arccos(s_k)/pi; 0 (Sec. 5.1's choice) by
                                  default; larger values trade speed for recall */
  int32_t stop_every;          /* 0: the stop test after each round (Sec. 4.1).  G >= 1: also after every G
                                  repetitions (Alg. 1 tests after each one: G = 1): after j repetitions of the round
                                  at prefix length i the test is (1 - p_i)^j (1 - p_{i+1})^(L - j) <= delta (no second
                                  factor in the first round); the filter threshold is then refreshed at every group
                                  of G repetitions, in every round */
} pf_search_opts;

/* Per-query statistics (Sec. 5 reports recall and throughput; these counts
 * explain both). */
typedef struct {
  int32_t start_depth;   /* prefix length of the first round */
  int32_t stop_depth;    /* prefix length of the last round */
  int32_t rounds;        /* rounds run */
  int32_t full_depth;    /* prefix length of the first round after which k points were held, -1 if none */
  int64_t retrieved;     /* candidate positions read from the repetitions (with repeats) */
  int64_t passed_filter; /* of those, how many passed the sketch filter */
  int64_t scored;        /* similarities computed (float32, or bfloat16 estimates) */
  int64_t reranked;      /* exact float32 similarities recomputed after a bfloat16 estimate */
  int32_t last_reps;     /* repetitions searched in the last round: L, or fewer when the stop test ran after
                            groups of repetitions (pf_search_opts.stop_every) and held mid-round */
  int32_t reserved;      /* always 0 (keeps the struct free of padding) */
} pf_query_stats;

typedef struct {
  int64_t n;
  int32_t d, d_pad;         /* d_pad = d rounded up to 16 */
  int32_t family;
  int32_t L;                /* repetitions */
  int32_t Kb;               /* bits per code = maximum prefix length K */
  int32_t ell;              /* bits per hash function */
  int32_t fns;              /* hash functions per repetition */
  int32_t M;                /* sketches per point */
  int32_t B;                /* segment size */
  int32_t trained;          /* a start-depth model is present */
  int32_t sketch_layout;    /* pf_sketch_layout */
  int32_t row_storage;      /* pf_row_storage */
  uint64_t bytes_used;      /* device bytes the index keeps resident */
  uint64_t budget_bytes;    /* budget it was built for */
} pf_index_info_t;

/* Internal arrays exposed read-only for verification (pf_index_array). */
typedef enum {
  PF_ARRAY_ROWS_F32 = 0,   /* float [n][d_pad]: normalised points (Sec. 4.2 "Vector storage") */
  PF_ARRAY_ROWS_BF16 = 1,  /* bfloat16 [n][d_pad]: RNE copy used by bfloat16 scoring */
  PF_ARRAY_CODES = 2,      /* uint32 [L][n]: sorted codes of each repetition (Sec. 4.2) */
  PF_ARRAY_IDS = 3,        /* uint32 [L][n]: positions pos(p) in the same order */
  PF_ARRAY_PREFIX = 4,     /* uint32 [L][8193]: lexicographic start of each 13-bit prefix */
  PF_ARRAY_SKETCHES = 5,   /* uint64 [M][n]: 1-bit sketches (Sec. 3.3, 4.2); PF_SKETCH_PER_POINT only */
  PF_ARRAY_HASH_ROWS = 6,  /* float [L*R + 64*M][d_pad]: Gaussian rows (R = fns*d_pad for CP, 32 for HP) */
  PF_ARRAY_CP_TABLE = 7,   /* double [41][ell+1]: CP collision table (Sec. 4.3); absent for HP */
  PF_ARRAY_TABLE_SKETCHES = 8, /* uint64 [L][n]: sketch (j mod M) of the point at each position of repetition j;
                                  PF_SKETCH_PER_TABLE only */
  PF_ARRAY_ROWS_F16 = 9,       /* binary16 [n][d_pad]: normalised points; PF_ROWS_F16 only (PF_ARRAY_ROWS_F32 is
                                  then absent) */
  /* the start-depth perceptron (after pf_learned_train; PF_ERR_NOT_TRAINED
     before), F = d_pad + 64 features, H = 256 hidden units, C = K + 1 classes */
  PF_ARRAY_MLP_F32 = 10,       /* float: W1 [H][F], b1 [H], W2 [C][H], b2 [C], one after another (the biases are
                                  also what inference uses) */
  PF_ARRAY_MLP_W1_BF16 = 11,   /* bfloat16 [F][H]: W1 rounded to nearest even, transposed, as inference reads it */
  PF_ARRAY_MLP_W2_BF16 = 12,   /* bfloat16 [C][H]: W2 rounded to nearest even, as inference reads it */
  PF_ARRAY_FHT_SIGNS = 13,     /* uint32 [L][fns][3][W]: sign bits of D1, D2, D3 of every pseudo-random CP function,
                                  W = max(1, d''/32) words, bit i of a vector set = -1 (PF_CROSSPOLYTOPE_FHT only) */
  PF_ARRAY_ROWS_FP8 = 14,      /* e4m3 [n][d_pad]: x_i / scale rounded to nearest even, saturated (fp8_rows only) */
  PF_ARRAY_FP8_META = 15,      /* float [n][2]: scale, and the bound on |<q, x> - scale <q, x8>| + rounding for
                                  any unit q (fp8_rows only) */
  PF_ARRAY_POOL_SELECT = 16    /* int32 [L][fns]: the pool functions of each table, first in the most significant
                                  bits (pool_bits only) */
} pf_array;

/* Build the index over `points` ([n][d] row-major, host or device).
 * Sec. 4: normalise (Sec. 4.2), draw L*K hash functions and M*64 sketch
 * hyperplanes from `seed`, hash every point, sort each repetition's
 * (code, pos) array and tabulate its 13-bit prefixes, and estimate the CP
 * collision table (Sec. 4.3).  L is the largest count whose resident bytes fit
 * memory_budget_bytes (PF_ERR_BUDGET_TOO_SMALL if none), clamped to 2048 (a
 * query keeps its per-repetition state in shared memory); an explicit
 * num_tables above 2048 is PF_ERR_INVALID_ARG.  The bytes counted are
 * those of the chosen sketch layout and row storage.  On success *out
 * receives a new index that the caller releases with pf_index_free. */
pf_status pf_index_build(const pf_build_params* params, const void* points, pf_index** out, void* stream);

/* Answer Q queries ([Q][d] float32, host or device) with Algorithm 1 as
 * implemented in Sec. 4.1-4.2: rounds of decreasing prefix length, segment-
 * wise range growth, sketch filter, exact similarity, top-k accumulator, and
 * the stop test of Lemma 1 after each round.
 *   k[Q]       (host or device) neighbours wanted per query, 1..k_max
 *   recall[Q]  (host or device) target 1 - delta per query, in (0, 1)
 *   k_max      row stride of the outputs, 1..128
 *   out_ids    [Q][k_max] uint32, out_sims [Q][k_max] float32 (host or
 *              device): sorted by similarity descending then id ascending;
 *              slots >= min(k, n) hold id 0xFFFFFFFF and similarity -inf
 *   stats      [Q] (host or device) or NULL
 *   opts       NULL for defaults
 * Each returned point is among the true k nearest with probability >= 1-delta
 * when the filter is off (Lemma 1); with the filter on this holds empirically
 * (Sec. 5.1). */
pf_status pf_index_search(pf_index* index, const float* queries, int64_t Q, const int32_t* k,
                          const double* recall, int32_t k_max, uint32_t* out_ids, float* out_sims,
                          pf_query_stats* stats, const pf_search_opts* opts, void* stream);

/* pf_index_search for callers that cannot allocate device memory while they
 * run: a serving process whose device memory is handed out up front by another
 * allocator, or a path where an allocation's latency or failure is not
 * acceptable.  The paper has no counterpart; this is a deployment variant.
 *   - Same arguments, semantics and results as pf_index_search, except that
 *     queries, k, recall, out_ids, out_sims, stats (if not NULL) and
 *     opts->start_depth (if set) must all be device memory, and that
 *     opts->learned_start is rejected (PF_ERR_INVALID_ARG: the learned start
 *     uses the index's own workspace); give opts->start_depth instead.
 *   - Scratch (normalised queries, query codes and sketches, work counter)
 *     lives in one 32 MiB file-scope device array that every GPU loading the
 *     library holds until the process exits.  A batch must satisfy
 *     Q*(8*d_pad + 4*L + 8*M) + 2048 <= 32 MiB; larger batches are rejected with
 *     PF_ERR_INVALID_ARG and a message giving the limit (split the batch).
 *   - No cudaMalloc, cudaFree or other allocating call is made.
 *   - All calls share the array: calls whose device work overlaps (other
 *     streams, other threads) race and must be serialised by the caller.
 *   - The first call on a device looks up the array's device address.  The
 *     call synchronises `stream` before it returns, so it cannot be captured
 *     in a CUDA graph; pf_search_plan_* is the capturable search.
 *   - A bounded device-side wait that expired is reported as
 *     PF_ERR_DEVICE_TIMEOUT and cleared, as pf_index_search does. */
pf_status pf_index_search_noalloc(pf_index* index, const float* queries, int64_t Q, const int32_t* k,
                                  const double* recall, int32_t k_max, uint32_t* out_ids, float* out_sims,
                                  pf_query_stats* stats, const pf_search_opts* opts, void* stream);

/* ---- learned start depth (the paper has no counterpart: an optional
 *      predictor layered on Algorithm 1's depth schedule) ----
 * A 2-layer perceptron (hidden 256, ReLU) maps a query's features -- its
 * normalised vector and its first 64-bit sketch as +-1 -- to a distribution
 * over the prefix length at which the plain schedule K, K-1, ... stops.  With
 * opts->learned_start the search starts at min(K, q + m), q the smallest depth
 * with P(stop depth > q) <= 0.05 and m = 0 (both settable with
 * pf_learned_set_start_rule): the first round takes the block at that depth
 * at once (its sketch threshold refreshed before repetitions 1, 2, 4, 8, 16
 * and every 32 after), later rounds drop one bit each.  The stop test of Lemma 1 still ends every query, so the
 * recall guarantee is that of the plain method. */
typedef struct {
  float final_loss;      /* mean cross-entropy of the last epoch */
  float train_accuracy;  /* fraction of training queries whose predicted quantile >= their stop depth */
  float mean_stop;       /* mean stop depth of the training traces */
  float mean_start;      /* mean predicted start depth on the training queries */
  int32_t samples;       /* training queries */
  int32_t epochs;
} pf_learned_report;

/* Train the start-depth model of `index` on Qt training queries ([Qt][d],
 * host or device): trace the plain search of each (k, recall) to get its stop
 * depth, then `epochs` passes of mini-batch Adam (batch 1024, learning rate
 * 1e-3, weights drawn from `seed`) with this library's kernels.  Replaces any
 * previous model.  report may be NULL. */
pf_status pf_learned_train(pf_index* index, const float* train_queries, int64_t Qt, int32_t k, double recall,
                           int32_t epochs, uint64_t seed, pf_learned_report* report, void* stream);

/* Start depths the trained model picks for Q queries (int32 [Q], host or
 * device).  PF_ERR_NOT_TRAINED without a model. */
pf_status pf_learned_predict(pf_index* index, const float* queries, int64_t Q, int32_t* start_depth, void* stream);

/* The rule that turns the model's distribution over stop depths into a start
 * depth: the smallest depth q with P(stop depth > q) <= tail, plus `margin`
 * bits, capped at K (defaults 0.05 and 0).  A lower start costs only time (the
 * first round takes the whole block at its depth), never recall.  Applies to
 * later predictions and searches; not while plans exist (they captured the
 * rule).  Errors: PF_ERR_INVALID_ARG (tail outside (0, 1), margin outside
 * [0, 32], plans exist). */
pf_status pf_learned_set_start_rule(pf_index* index, float tail, int32_t margin);

/* One forward + backward pass of the start-depth perceptron on caller data
 * (all device pointers, float32, row-major): X [B][F], y [B] class labels in
 * [0, C), W1 [H][F], b1 [H], W2 [C][H], b2 [C].  Writes the mean
 * cross-entropy to *loss (device) and its gradients dW1, db1, dW2, db2.
 * Exposed so that the gradients can be checked against an independent CPU
 * implementation. */
pf_status pf_mlp_forward_backward(const float* X, const int32_t* y, int32_t B, int32_t F, int32_t H, int32_t C,
                                  const float* W1, const float* b1, const float* W2, const float* b2, float* loss,
                                  float* dW1, float* db1, float* dW2, float* db2, void* stream);

/* Hash Q queries only (the first step of every query, Sec. 4.1): normalise,
 * then codes [Q][L] uint32 and sketches [Q][M] uint64 (host or device). */
pf_status pf_hash_queries(pf_index* index, const float* queries, int64_t Q, uint32_t* qcodes,
                          uint64_t* qsketches, void* stream);

/* Device time in milliseconds, measured with CUDA events on the call's stream,
 * of the phases of the last pf_index_search on this index that ran with
 * opts->timing = 1: t[0] query normalisation and hashing, t[1] the search
 * kernel, t[2] all device work of the call.  count = entries to write (<= 3). */
pf_status pf_index_last_timing(const pf_index* index, float* t, int32_t count);

/* Sizes and resident bytes of an index. */
pf_status pf_index_info(const pf_index* index, pf_index_info_t* info);

/* Read-only device pointer and byte size of one internal array
 * (PF_ERR_INVALID_ARG if the index has no such array). */
pf_status pf_index_array(const pf_index* index, int32_t which, const void** device_ptr, uint64_t* bytes);

/* Copy one internal array (pf_array) into dst (host or device), which must
 * hold at least the array's byte size (see pf_index_array). */
pf_status pf_index_read_array(const pf_index* index, int32_t which, void* dst, uint64_t dst_bytes, void* stream);

/* Defaults: FP32 scoring, filter on, no learned start, no start depths. */
void pf_search_opts_default(pf_search_opts* opts);

/* ---- Launch-shape tuning (the shape is not part of the method of Sec. 4:
 * results and their order are the same for every shape; so are the statistics
 * for one number of warps per query) ----
 * Times the search kernel of a batch (Q queries of one k and recall, opts as
 * in pf_index_search: scoring, filter, learned start) for each candidate shape
 * -- 4 warps per query with 4 or 8 positions per lane per streaming step, or
 * 8 warps with 8 positions, times the largest resident CTAs per SM and one or
 * two fewer, times streaming rule flat_fill 0 or 3 -- and keeps the fastest for the index's later searches and
 * plans.  queries: host or device, [Q][d] float32.
 * report (may be NULL) receives the choice.  Errors: PF_ERR_INVALID_ARG (bad
 * sizes, or search plans bound to the index exist), PF_ERR_NOT_TRAINED, CUDA. */
typedef struct {
  int32_t unroll;       /* chosen positions per lane per streaming step */
  int32_t warps;        /* chosen warps per query (4 or 8) */
  int32_t ctas_per_sm;  /* chosen CTAs per SM */
  int32_t flat_fill;    /* chosen streaming rule (see pf_index_set_shape) */
  int32_t candidates;   /* shapes timed */
  float best_ms;        /* search-kernel time of the chosen shape on the batch */
  float default_ms;     /* ... of the default shape (8 positions, full occupancy) */
} pf_tune_report;
pf_status pf_index_tune(pf_index* index, const float* queries, int64_t Q, int32_t k, double recall,
                        const pf_search_opts* opts, pf_tune_report* report, void* stream);
/* Set the launch shape of the index's later searches and plans directly:
 * unroll 4 or 8 positions per lane, warps 4 or 8 per query (8 only with unroll
 * 8), ctas_per_sm a cap on resident CTAs per SM (0: as many as fit),
 * flat_fill the streaming rule: 0 = every round streams its new positions in
 * chunks of one run; F in 1..64 = a round whose chunks would be less than 1/F
 * full streams them as one flat sequence instead (short runs; the same
 * candidates either way).  Errors: PF_ERR_INVALID_ARG (other values, or search
 * plans bound to the index). */
pf_status pf_index_set_shape(pf_index* index, int32_t unroll, int32_t warps, int32_t ctas_per_sm, int32_t flat_fill);

/* ---- Captured search (a CUDA graph of one batch shape) ----
 * pf_index_search for a fixed Q, k_max and options, bound to caller-owned
 * DEVICE buffers: normalisation, hashing (with its float64 fix-up), the
 * learned start (if opts->learned_start) and the search kernel are captured
 * once into a CUDA graph; pf_search_plan_run launches it (one graph launch,
 * asynchronous on `stream`), reading whatever the buffers hold at that time.
 * Each buffer may be device memory or page-locked host memory
 * (cudaHostAlloc / cudaHostRegister): for a host buffer the plan keeps a
 * device copy, and its graph copies host inputs in before the search and host
 * outputs out after it, on the run's stream (pageable host memory is
 * rejected: it cannot be copied asynchronously inside a graph).
 * The plan owns its own workspace, so plans and plain searches of one index
 * do not share scratch; runs of one plan must not overlap.  A plan is bound to
 * the index's state at creation: while plans exist, pf_learned_train and
 * pf_index_tune fail with PF_ERR_INVALID_ARG and pf_index_free does nothing
 * (it sets the error message), so free plans first. */
typedef struct pf_search_plan pf_search_plan;
typedef struct {
  const float* queries;        /* [Q][d] float32 */
  const int32_t* k;            /* [Q] in [1, k_max] */
  const double* recall;        /* [Q] in (0, 1) */
  const int32_t* start_depth;  /* [Q] per-query start depths, or NULL (see pf_search_opts) */
  uint32_t* out_ids;           /* [Q][k_max] */
  float* out_sims;             /* [Q][k_max] */
  pf_query_stats* stats;       /* [Q], or NULL */
} pf_plan_io;
/* opts: scoring, filter, learned_start (timing and opts->start_depth are
 * ignored: the start depths, if any, are io->start_depth).  Errors:
 * PF_ERR_INVALID_ARG (Q < 1, k_max outside [1, 128], a null or pageable host pointer),
 * PF_ERR_NOT_TRAINED, PF_ERR_OOM, CUDA. */
pf_status pf_search_plan_create(pf_index* index, int64_t Q, int32_t k_max, const pf_plan_io* io,
                                const pf_search_opts* opts, pf_search_plan** out);
/* Launch the captured graph on `stream`; returns without waiting. */
pf_status pf_search_plan_run(pf_search_plan* plan, void* stream);
/* Wait for `stream` and report what the last run found: PF_ERR_INVALID_ARG if
 * some k or recall was out of range (those queries return empty rows),
 * PF_ERR_DEVICE_TIMEOUT if a bounded device-side wait expired. */
pf_status pf_search_plan_check(pf_search_plan* plan, void* stream);
/* Release a plan (NULL is accepted). */
void pf_search_plan_free(pf_search_plan* plan);

/* ---- Diagnostics of the bounded device-side waits ----
 * Every wait of the tensor-core hashing kernel (Sec. 2.2 hashing of the
 * queries) on one of its pipeline barriers gives up after 1 s, records an
 * error word and leaves the kernel; the call that launched it then returns
 * PF_ERR_DEVICE_TIMEOUT and clears the word, and the index stays usable.
 * This call hashes the Q queries (host or device, [Q][d] float32) with the
 * kernel's weight-tile loads withheld, so that the waits on them expire (about
 * 1 s), and returns what the library reports for it: PF_ERR_DEVICE_TIMEOUT
 * when the time-out path works.  No output is written.  Errors:
 * PF_ERR_INVALID_ARG (null argument, Q < 1, or search plans bound to the
 * index), CUDA. */
pf_status pf_index_selftest_timeout(pf_index* index, const float* queries, int64_t Q, void* stream);
/* Withhold (hold != 0) or restore (hold == 0) the weight-tile loads of every
 * later tensor-core hashing launch of this index, so that a whole entry point
 * (pf_index_search, pf_index_search_noalloc, ...) can be driven through its
 * time-out path: while held, each such call returns PF_ERR_DEVICE_TIMEOUT
 * after about 1 s, with its outputs unspecified.  Captured plans keep the
 * setting they were captured with.  Errors: PF_ERR_INVALID_ARG (null index). */
pf_status pf_index_selftest_hold(pf_index* index, int32_t hold);

/* ---- Diagnostics of the search kernel's range pass (Sec. 4.2 "Retrieving
 *      candidate points": the range of a repetition grows to the block of
 *      codes sharing the first i bits with the query) ----
 * With enable != 0, later searches of this index count how each range step
 * was settled: counts[0] steps at prefix length <= 13 read from the 13-bit
 * prefix table, counts[1] sides settled within the first four segment
 * boundaries probed together, counts[2] sides that galloped past them,
 * counts[3] rounds whose new positions were streamed in chunks of one run,
 * counts[4] rounds streamed as one flat sequence (short runs).  Each call waits
 * for the device, writes the 5 counts since the previous call into counts
 * (NULL: not read) and resets them; enable == 0 stops counting (not
 * while search plans exist: they were captured with the counters).  The
 * counters cost device atomics: leave them off outside tests.  Errors:
 * PF_ERR_INVALID_ARG (null index, plans exist), PF_ERR_OOM, CUDA. */
pf_status pf_index_count_range_paths(pf_index* index, int32_t enable, uint64_t* counts);

/* Release an index (NULL is accepted).  Does nothing while search plans bound
 * to it exist (pf_last_error_message says so). */
void pf_index_free(pf_index* index);

/* Static description of a status code. */
const char* pf_status_string(pf_status status);

/* Message of the last failed call on this thread ("" if none). */
const char* pf_last_error_message(void);

#ifdef __cplusplus
}
#endif
#endif /* PUFFINN_GB300_H */
