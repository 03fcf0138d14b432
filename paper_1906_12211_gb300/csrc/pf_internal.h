// Internal declarations of the GB300 PUFFINN library (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "puffinn_gb300.h"

namespace pf {

constexpr int kPrefixBits = 13;                     // Sec. 4.2: 13-bit prefix table
constexpr int kPrefixSize = (1 << kPrefixBits) + 1;
constexpr int kAlphaSteps = 41;                     // Sec. 4.3: similarity grid step 0.05
constexpr int kMaxK = 128;
constexpr int kMaxD = 320;
constexpr int kMaxL = 2048;
constexpr int kMlpHidden = 256;                     // start-depth model hidden units
constexpr float kMlpTail = 0.05f;                   // quantile: P(stop depth > q) <= this
constexpr int kMlpMargin = 0;                       // start depth = quantile + this many bits (capped at K)

enum Purpose : uint32_t {
  kPurposeHash = 1,
  kPurposeSketch = 2,
  kPurposeCpMc = 3,
  kPurposeFht = 4,    // sign vectors of the pseudo-random cross-polytope functions
  kPurposeFhtMc = 5,  // sign vectors of its Monte-Carlo collision draws
  kPurposePool = 6,   // hyperplanes of the pooled functions
  kPurposePoolSelect = 7,  // each table's subset of the pool
};

// Shape of one repetition's code (Sec. 4.3): l bits per function, floor(32/l)
// functions, K = fns * l bits.  Hash rows are padded so that every CP function
// owns d_pad rows (rows c >= d are zero and never win the argmax).
struct Layout {
  int ell = 1, fns = 32, Kb = 32, d_pad = 16;
  int rows_fn = 1;      // rows per hash function in the padded row matrix
  int rows_table = 32;  // rows per repetition (0 for the pseudo-random family: no rows)
  int fht_n = 0;        // pseudo-random family: transform length 2^ceil(log2 d)
  int fht_words = 0;    // 32-bit words of one sign vector (at least one)
};
Layout make_layout(int family, int d);

// Launch shape of the search kernel (not part of the method): positions per
// lane per streaming step (4 or 8), a cap on CTAs per SM (0: occupancy) and
// warps per query (4, or 8 with 8 positions).
struct SearchShape {
  int unroll = 0;       // 0 in SearchArgs: the index's tuned shape
  int ctas_per_sm = 0;
  int warps = 4;
  int flat_fill = 0;    // 0: rounds stream in chunks of one run; F: flat when the chunks are < 1/F full
};

// ---------------------------------------------------------------- host params
float gaussian(uint64_t seed, uint32_t purpose, uint32_t a, uint32_t b, uint32_t c);
// W[(L*rows_table + 64*M)][d_pad] float32 and per-row recheck band thr[]
void gen_hash_rows(uint64_t seed, int family, int L, int M, int d, const Layout& lay, float* W, float* thr);
void cp_collision_table(uint64_t seed, int d, int ell, int draws, double* P /*[41][ell+1]*/);
void filter_cos_table(double* c /*[65]*/, double eps = 0.0);
// pseudo-random cross-polytope family (Sec. 4.3): sign bits [L][fns][3][fht_words]
void gen_fht_signs(uint64_t seed, int L, const Layout& lay, uint32_t* out);
void fht_collision_table(uint64_t seed, const Layout& lay, int draws, double* P /*[41][ell+1]*/);
// bounds on the float32 transform's error for unit inputs: decisions whose top
// two |y| are closer than *gap, or whose top |y| is below *sign, are redone in float64
void fht_bands(int d, const Layout& lay, float* gap, float* sign);
// pooling (Sec. 3.2): rows of m pooled functions laid out as ceil(m / fns)
// groups shaped like tables (W [(groups*rows_table + 64*M)][d_pad], sketch
// planes after them, as gen_hash_rows lays them out), and each table's subset
void gen_pool_rows(uint64_t seed, int family, int m, int M, int d, const Layout& lay, float* W, float* thr);
void pool_select(uint64_t seed, int L, int F, int m, int32_t* sel /*[L][F]*/);
int64_t budget_tables(int family, int64_t n, int d, int M, uint64_t budget, int sketch_layout, int row_storage,
                      int fp8_rows, int pool_fns);
uint64_t resident_bytes(int family, int64_t n, int d, int M, int L, int sketch_layout, int row_storage, int fp8_rows,
                        int pool_fns);

// A hash decision the tensor-core kernel leaves to the float64 fix-up pass.
struct RecheckReq {
  uint32_t p;     // point (row of the normalised matrix)
  uint32_t row0;  // CP: first hash row of the function; one-bit decisions: the hash row
  uint32_t info;  // bits 0-19 repetition / sketch, 20-25 function / bit, 26-27 CP candidate mask, 30-31 kind
  uint16_t c[2];  // CP candidate hyperplanes (rows of the function)
};

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
struct Error {
  pf_status status;
  std::string msg;
};

}  // namespace pf

// Workspace for one search call (grown on demand, owned by the index).
struct pf_workspace {
  size_t cap_q = 0;  // queries the buffers hold
  float* qraw = nullptr;       // [Q][d] staged host queries
  float* qx = nullptr;         // [Q][d_pad] normalised queries
  __nv_bfloat16* qxh = nullptr;  // [Q][d_pad] bfloat16 high half of qx
  __nv_bfloat16* qxl = nullptr;  // [Q][d_pad] bfloat16 low half (qx - qxh)
  uint32_t* qcodes = nullptr;  // [Q][L]
  uint32_t* qgcodes = nullptr;  // [Q][pool groups] (pooled index only)
  uint64_t* qsk = nullptr;     // [Q][M]
  int32_t* k = nullptr;
  double* recall = nullptr;
  int32_t* start = nullptr;
  uint32_t* ids = nullptr;     // [Q][k_max] staged outputs
  float* sims = nullptr;
  pf_query_stats* stats = nullptr;
  int32_t* counter = nullptr;  // work queue head + error word
  double* cos_eps = nullptr;   // [65] threshold table of the last nonzero filter slack
  pf::RecheckReq* rq = nullptr;  // deferred hash rechecks
  uint32_t* rq_count = nullptr;
  size_t cap_kmax = 0;
};

struct pf_index {
  int device = 0;
  int64_t n = 0;
  int d = 0, family = 0, L = 0, M = 32, B = 12;
  int sketch_layout = PF_SKETCH_PER_TABLE;
  pf::Layout lay;
  uint64_t budget = 0, bytes_used = 0;
  int64_t hash_rows = 0;  // L*rows_table + 64*M
  // resident device arrays
  float* x32 = nullptr;            // [n][d_pad] (float32 rows; null with binary16 rows)
  __half* xf16 = nullptr;          // [n][d_pad] (binary16 rows; null with float32 rows)
  int row_storage = PF_ROWS_F32;
  __nv_bfloat16* x16 = nullptr;    // [n][d_pad]
  uint8_t* x8 = nullptr;           // [n][d_pad] e4m3 copy (fp8_rows only)
  float2* x8_meta = nullptr;       // [n] (scale, error bound) of the e4m3 copy
  uint64_t* sk = nullptr;          // [M][n] (per-point layout)
  uint64_t* skc = nullptr;         // [L][n] sketch j mod M of the point at each position (per-table layout)
  float* W32 = nullptr;            // [hash_rows][d_pad]
  __nv_bfloat16* Whi = nullptr;    // [hash_rows][d_pad]
  float* Wthr = nullptr;           // [hash_rows]
  uint32_t* codes = nullptr;       // [L][n]
  uint32_t* ids = nullptr;         // [L][n]
  uint32_t* pfx = nullptr;         // [L][8193]
  double* cpP = nullptr;           // [41][ell+1]
  uint32_t* fht_signs = nullptr;   // [L][fns][3][fht_words] (pseudo-random family only)
  int pool_fns = 0, pool_tables = 0;  // pooling: functions in the pool, groups of fns of them
  int32_t* pool_sel = nullptr;     // [L][fns] each table's pool functions
  float fht_gap = 0.f, fht_sign = 0.f;  // its float64 recheck bands
  double* cos_tab = nullptr;       // [65]
  float bf16_err = 0.f;            // bound on |bf16 estimate - float32 canonical similarity|
  int32_t* dev_error = nullptr;    // device error word (bit 1: a bounded wait timed out)
  int num_sms = 0;
  pf::SearchShape search_shape{8, 0, 4};  // chosen by pf_index_tune (default: 8 positions per lane, full occupancy)
  int live_plans = 0;                   // captured search plans bound to this index
  int hold_weight_loads = 0;            // diagnostics only (pf_index_selftest_timeout)
  unsigned long long* path_count = nullptr;  // diagnostics only (pf_index_count_range_paths)
  pf_workspace ws;
  // start-depth model: params = [W1 (H x F) | b1 (H) | W2 (C x H) | b2 (C)], float32
  int mlp_trained = 0, mlp_F = 0, mlp_C = 0;
  float mlp_tail = pf::kMlpTail;  // start rule: smallest q with P(stop depth > q) <= tail ...
  int mlp_margin = pf::kMlpMargin;  // ... plus this many bits (capped at K)
  float* mlp_w = nullptr;
  __nv_bfloat16* mlp_w1h = nullptr;  // bfloat16 W1 for inference, transposed: [F][H]
  __nv_bfloat16* mlp_w2h = nullptr;  // bfloat16 W2 for inference
  float* mlp_x = nullptr;            // [cap_q][F] feature scratch of the search path
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // phase timing events
  float last_ms[3] = {0.f, 0.f, 0.f};
};

// ---------------------------------------------------------------- launchers
namespace pf {

// round normalised rows x32 [rows][d_pad] in place to binary16 (nearest, ties to
// even), keep the binary16 copy, and redo the bfloat16 split xh + xl (xl may be
// null) of the rounded rows
cudaError_t launch_round_rows_f16(float* x32, int64_t rows, int d_pad, __half* xf16, __nv_bfloat16* xh,
                                  __nv_bfloat16* xl, cudaStream_t s);
// normalise rows (Sec. 4.2) -> x32 [rows][d_pad], and optionally its bfloat16
// split x32 = xh + xl (xh is the round-to-nearest bfloat16 copy)
cudaError_t launch_normalize(const float* in, int64_t rows, int d, int d_pad, float* x32, __nv_bfloat16* xh,
                             __nv_bfloat16* xl, cudaStream_t s);
// e4m3 copy of normalised rows x32 [rows][d_pad] with per-row (scale, error bound)
cudaError_t launch_quantize_fp8(const float* x32, int64_t rows, int d, int d_pad, uint8_t* x8, float2* meta,
                                cudaStream_t s);

// Hash rows x32 [npts][d_pad] (with its bfloat16 split xh + xl) under all L
// repetitions and M sketches.  Codes written at codes[j*cj + p*cp], sketches
// at sk[m*sm + p*sp].  Uses the tensor-core kernel when d_pad <= 128.
// rq: optional queue of deferred float64 rechecks (capacity rq_cap, split
// into one region per CTA of the hashing kernel; rq_count holds one counter per
// region, at least ix->num_sms of them); without a queue, or where a region is
// full, rechecks run inline.
// tables: row-based repetitions to hash (-1: ix->L; a pooled index passes its
// pool groups, whose codes pool_gather then combines)
cudaError_t launch_hash(const pf_index* ix, const float* x32, const __nv_bfloat16* xh, const __nv_bfloat16* xl,
                        int64_t npts, uint32_t* codes, int64_t cj, int64_t cp, uint64_t* sk, int64_t sm,
                        int64_t sp, RecheckReq* rq, uint32_t* rq_count, uint32_t rq_cap, cudaStream_t s,
                        int tables = -1);
// codes[j*cj + p*cp] of a pooled index from its pool groups' codes
// gcodes[g*gj + p*gp] (group g holds pool functions g*fns .. g*fns + fns - 1)
cudaError_t launch_pool_gather(const pf_index* ix, const uint32_t* gcodes, int64_t gj, int64_t gp, int64_t npts,
                               uint32_t* codes, int64_t cj, int64_t cp, cudaStream_t s);
// recheck-queue entries to provision for npts points
// Entries of the deferred-recheck queue for hashing npts points with `tables`
// row-function tables: on the order of 1 % of cross-polytope decisions and
// 0.2 % of one-bit decisions fall inside the band, so a twentieth of the
// table decisions plus a 256th of the sketch bits per point (at least 48)
// leaves room for a CTA's uneven share; requests beyond a CTA's region are
// rechecked inline (slower, the same codes).
uint32_t recheck_capacity(const pf_index* ix, int64_t npts, int tables);
// the recheck band of a hash row is its norm times 2^-band_exponent(d_pad) (params.cpp)
int band_exponent(int d_pad);
// tables: repetitions hashed with row-based functions (ix->L; 0 hashes sketches only)
cudaError_t launch_hash_tc(const pf_index* ix, const __nv_bfloat16* xh, const __nv_bfloat16* xl, const float* x32,
                           int64_t npts, uint32_t* codes, int64_t cj, int64_t cp, uint64_t* sk, int64_t sm,
                           int64_t sp, int32_t* error, RecheckReq* rq, uint32_t* rq_count, uint32_t rq_cap,
                           cudaStream_t s, int tables);
// pseudo-random cross-polytope codes (kernels_fht.cu): codes[j*cj + p*cp]
cudaError_t launch_hash_fht(const pf_index* ix, const float* x32, int64_t npts, uint32_t* codes, int64_t cj,
                            int64_t cp, cudaStream_t s);

// Sort every repetition's (code, position) pairs and build the prefix tables.
cudaError_t sort_tables(pf_index* ix, const uint32_t* codes_unsorted, cudaStream_t s);
// skc[j][pos] = sk[j mod M][ids[j][pos]] for every repetition
cudaError_t gather_table_sketches(const pf_index* ix, const uint64_t* sk, uint64_t* skc, cudaStream_t s);

struct SearchArgs {
  int Q = 0;
  SearchShape shape;   // launch shape override (unroll 0: the index's)
  const float* qx = nullptr;
  const uint32_t* qcodes = nullptr;
  const uint64_t* qsk = nullptr;
  const int32_t* k = nullptr;
  const double* recall = nullptr;
  const int32_t* start = nullptr;
  int k_max = 0;
  int filter = 1;
  int scoring = 0;
  uint32_t* out_ids = nullptr;
  float* out_sims = nullptr;
  pf_query_stats* stats = nullptr;
  int32_t* counter = nullptr;
  int stop_every = 0;  // pf_search_opts.stop_every
  int pool_rule = 0;   // pf_search_opts.pool_rule
  const double* cos_tab = nullptr;  // threshold table of a nonzero filter slack (null: the index's)
};
cudaError_t launch_search(const pf_index* ix, const SearchArgs& a, cudaStream_t s);
// CTAs per SM the search kernel can keep resident for this index (0 on error)
int search_max_ctas_per_sm(const pf_index* ix, int k_max, int unroll, int warps);

// start-depth perceptron (kernels_mlp.cu)
cudaError_t mlp_features(const float* qx, const uint64_t* qsk, int Q, int d_pad, int M, float* x, cudaStream_t s);
cudaError_t mlp_forward_backward(const float* X, const int32_t* y, int B, int F, int H, int C, const float* W1,
                                 const float* b1, const float* W2, const float* b2, float* loss, float* dW1,
                                 float* db1, float* dW2, float* db2, float* h, float* z, float* dz, float* dh,
                                 cudaStream_t s);
cudaError_t adam_step(float* w, const float* g, float* m, float* v, int64_t count, float lr, int t, cudaStream_t s);
cudaError_t to_bf16(const float* a, __nv_bfloat16* b, int64_t count, cudaStream_t s);
cudaError_t to_bf16_transposed(const float* a, __nv_bfloat16* b, int rows, int cols, cudaStream_t s);
cudaError_t mlp_predict(const float* qx, const uint64_t* qsk, int Q, int d_pad, int M, const __nv_bfloat16* W1t,
                        const float* b1, const __nv_bfloat16* W2, const float* b2, int C, float tail, int margin,
                        int32_t* start, cudaStream_t s);
cudaError_t gather_rows(const float* src, const int32_t* idx, int rows, int cols, float* dst, cudaStream_t s);

}  // namespace pf
