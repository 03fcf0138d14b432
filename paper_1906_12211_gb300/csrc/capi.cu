// C ABI of the library: argument checks, device memory ownership, host/device
// staging, and the order of the build and search steps.  Every step of the
// computation runs in this library's CUDA kernels.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <random>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pf_internal.h"

namespace pf {

namespace {
thread_local std::string g_last_error;

struct CudaFail {
  cudaError_t err;
  std::string where;
};

#define PF_CK(expr)                                                       \
  do {                                                                    \
    cudaError_t _e = (expr);                                              \
    if (_e != cudaSuccess) throw CudaFail{_e, std::string(#expr)};        \
  } while (0)

template <class T>
void dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * count);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error{PF_ERR_OOM, "cudaMalloc of " + std::to_string(sizeof(T) * count) + " bytes failed: " +
                                cudaGetErrorString(e)};
  }
}

template <class T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

pf_status fail(pf_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

template <class F>
pf_status guarded(F&& body) {
  try {
    g_last_error.clear();
    return body();
  } catch (const Error& e) {
    return fail(e.status, e.msg);
  } catch (const CudaFail& e) {
    return fail(PF_ERR_CUDA, e.where + ": " + cudaGetErrorString(e.err));
  } catch (const std::bad_alloc&) {
    return fail(PF_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(PF_ERR_CUDA, "unexpected exception");
  }
}

// bfloat16 hi/lo split of the float32 hash rows (for the tensor-core path)
// the hyperplanes' entries are bfloat16 values (R2): their bfloat16 copy is exact
__global__ void to_bf16_exact_kernel(const float* __restrict__ w, int64_t count, __nv_bfloat16* __restrict__ hi) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
    hi[i] = __float2bfloat16_rn(w[i]);
}

void free_ws(pf_workspace& ws) {
  dfree(ws.qraw);
  dfree(ws.qx);
  dfree(ws.qxh);
  dfree(ws.qxl);
  dfree(ws.qcodes);
  dfree(ws.qsk);
  dfree(ws.qgcodes);
  dfree(ws.k);
  dfree(ws.recall);
  dfree(ws.start);
  dfree(ws.ids);
  dfree(ws.sims);
  dfree(ws.stats);
  dfree(ws.counter);
  dfree(ws.cos_eps);
  dfree(ws.rq);
  dfree(ws.rq_count);
  ws.cap_q = 0;
  ws.cap_kmax = 0;
}

// (re)allocate a workspace for q queries of up to km results
void alloc_ws(pf_index* ix, pf_workspace& ws, size_t q, size_t km) {
  free_ws(ws);
  const int dp = ix->lay.d_pad;
  dalloc(&ws.qraw, q * ix->d);
  dalloc(&ws.qx, q * dp);
  dalloc(&ws.qxh, q * dp);
  dalloc(&ws.qxl, q * dp);
  dalloc(&ws.qcodes, q * ix->L);
  if (ix->pool_tables > 0) dalloc(&ws.qgcodes, q * ix->pool_tables);
  dalloc(&ws.qsk, q * ix->M);
  dalloc(&ws.k, q);
  dalloc(&ws.recall, q);
  dalloc(&ws.start, q);
  dalloc(&ws.ids, q * km);
  dalloc(&ws.sims, q * km);
  dalloc(&ws.stats, q);
  dalloc(&ws.counter, 64);
  dalloc(&ws.cos_eps, 65);
  dalloc(&ws.rq, recheck_capacity(ix, int64_t(q), ix->pool_tables > 0 ? ix->pool_tables : ix->L));
  dalloc(&ws.rq_count, size_t(ix->num_sms));
  ws.cap_q = q;
  ws.cap_kmax = km;
}

void ensure_ws(pf_index* ix, int64_t Q, int k_max) {
  pf_workspace& ws = ix->ws;
  if (size_t(Q) <= ws.cap_q && size_t(k_max) <= ws.cap_kmax) return;
  alloc_ws(ix, ws, std::max<size_t>(size_t(Q), ws.cap_q), std::max<size_t>(size_t(k_max), ws.cap_kmax));
}

void destroy(pf_index* ix) {
  if (!ix) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ix->device);
  dfree(ix->x32);
  dfree(ix->xf16);
  dfree(ix->x16);
  dfree(ix->sk);
  dfree(ix->skc);
  dfree(ix->W32);
  dfree(ix->Whi);
  dfree(ix->Wthr);
  dfree(ix->codes);
  dfree(ix->ids);
  dfree(ix->pfx);
  dfree(ix->cpP);
  dfree(ix->cos_tab);
  dfree(ix->dev_error);
  dfree(ix->path_count);
  dfree(ix->fht_signs);
  dfree(ix->x8);
  dfree(ix->x8_meta);
  dfree(ix->pool_sel);
  dfree(ix->mlp_w);
  dfree(ix->mlp_w1h);
  dfree(ix->mlp_w2h);
  free_ws(ix->ws);
  for (auto& e : ix->ev)
    if (e) cudaEventDestroy(e);
  cudaSetDevice(prev);
  delete ix;
}

// Copy `bytes` from a host or device pointer into device buffer dst.
void stage_in(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (bytes == 0) return;
  PF_CK(cudaMemcpyAsync(dst, src, bytes, on_device(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
}

// The threshold table of a nonzero filter slack, copied into the workspace on
// `s` (null for eps = 0: the index's own table).  capture: the copy must not be
// recorded into a graph, so it is made synchronously.
const double* slack_table(pf_workspace& ws, double eps, cudaStream_t s, bool capture = false) {
  if (eps == 0.0) return nullptr;
  double tab[65];
  filter_cos_table(tab, eps);
  if (capture)
    PF_CK(cudaMemcpy(ws.cos_eps, tab, sizeof(tab), cudaMemcpyHostToDevice));
  else
    PF_CK(cudaMemcpyAsync(ws.cos_eps, tab, sizeof(tab), cudaMemcpyHostToDevice, s));  // pageable: staged on return
  return ws.cos_eps;
}

// Hash and normalise Q queries (device pointer qsrc) into the workspace.
void hash_queries_ws(pf_index* ix, pf_workspace& ws, const float* qdev, int64_t Q, cudaStream_t s) {
  PF_CK(launch_normalize(qdev, Q, ix->d, ix->lay.d_pad, ws.qx, ws.qxh, ws.qxl, s));
  if (ix->pool_tables > 0) {  // the pool's functions once, then each table's subset
    PF_CK(launch_hash(ix, ws.qx, ws.qxh, ws.qxl, Q, ws.qgcodes, 1, ix->pool_tables, ws.qsk, 1, ix->M, ws.rq,
                      ws.rq_count, recheck_capacity(ix, Q, ix->pool_tables), s, ix->pool_tables));
    PF_CK(launch_pool_gather(ix, ws.qgcodes, 1, ix->pool_tables, Q, ws.qcodes, 1, ix->L, s));
    return;
  }
  PF_CK(launch_hash(ix, ws.qx, ws.qxh, ws.qxl, Q, ws.qcodes, 1, ix->L, ws.qsk, 1, ix->M, ws.rq, ws.rq_count,
                    recheck_capacity(ix, Q, ix->L), s));
}

// start depths of the model for the Q hashed queries of the workspace -> ws.start
void predict_ws(pf_index* ix, pf_workspace& ws, int64_t Q, cudaStream_t s) {
  const int F = ix->mlp_F, H = kMlpHidden, C = ix->mlp_C;
  const float* b1 = ix->mlp_w + size_t(H) * F;
  const float* b2 = b1 + H + size_t(C) * H;
  PF_CK(mlp_predict(ws.qx, ws.qsk, int(Q), ix->lay.d_pad, ix->M, ix->mlp_w1h, b1, ix->mlp_w2h, b2, C, ix->mlp_tail,
                    ix->mlp_margin, ws.start, s));
}

const float* stage_queries(pf_index* ix, const float* queries, int64_t Q, cudaStream_t s) {
  if (on_device(queries)) return queries;
  stage_in(ix->ws.qraw, queries, sizeof(float) * size_t(Q) * ix->d, s);
  return ix->ws.qraw;
}

// After the stream has been synchronised: did a bounded device-side wait give
// up since the last check?  The error word is cleared, so the index stays
// usable (a call's outputs are its own; the index itself is not written).
bool device_timed_out(pf_index* ix) {
  int32_t herr = 0;
  PF_CK(cudaMemcpy(&herr, ix->dev_error, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (herr) PF_CK(cudaMemset(ix->dev_error, 0, sizeof(int32_t)));
  return herr != 0;
}

}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

}  // namespace pf

using namespace pf;

extern "C" {

void pf_search_opts_default(pf_search_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->filter = 1;
}

const char* pf_status_string(pf_status s) {
  switch (s) {
    case PF_OK: return "ok";
    case PF_ERR_INVALID_ARG: return "invalid argument";
    case PF_ERR_BUDGET_TOO_SMALL: return "memory budget too small for one repetition";
    case PF_ERR_OOM: return "out of device memory";
    case PF_ERR_CUDA: return "CUDA error";
    case PF_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case PF_ERR_NOT_TRAINED: return "start-depth model not trained";
  }
  return "unknown status";
}

const char* pf_last_error_message(void) { return g_last_error.c_str(); }

pf_status pf_index_build(const pf_build_params* prm, const void* points, pf_index** out, void* stream) {
  return guarded([&]() -> pf_status {
    if (!prm || !points || !out) return fail(PF_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (prm->n < 1 || prm->n > 0x7fffffffLL) return fail(PF_ERR_INVALID_ARG, "n must be in [1, 2^31-1]");
    if (prm->d < 1 || prm->d > kMaxD) return fail(PF_ERR_INVALID_ARG, "d must be in [1, 320]");
    if (prm->dtype != PF_F32) return fail(PF_ERR_INVALID_ARG, "points must be float32");
    if (prm->family != PF_SIMHASH && prm->family != PF_CROSSPOLYTOPE && prm->family != PF_CROSSPOLYTOPE_FHT)
      return fail(PF_ERR_INVALID_ARG, "unknown hash family");
    const int M = prm->num_sketches ? prm->num_sketches : 32;
    const int B = prm->segment_B ? prm->segment_B : 12;
    const int draws = prm->cp_draws ? prm->cp_draws : 1000;
    if (M < 1 || M > 256) return fail(PF_ERR_INVALID_ARG, "num_sketches must be in [1, 256]");
    if (B < 1 || B > 4096) return fail(PF_ERR_INVALID_ARG, "segment_B must be in [1, 4096]");
    if (draws < 1) return fail(PF_ERR_INVALID_ARG, "cp_draws must be >= 1");
    if (prm->sketch_layout != PF_SKETCH_PER_TABLE && prm->sketch_layout != PF_SKETCH_PER_POINT)
      return fail(PF_ERR_INVALID_ARG, "unknown sketch layout");
    if (prm->row_storage != PF_ROWS_F32 && prm->row_storage != PF_ROWS_F16)
      return fail(PF_ERR_INVALID_ARG, "unknown row storage");
    int pool_fns = 0;
    if (prm->pool_bits != 0) {
      if (prm->pool_bits < 0 || prm->family == PF_CROSSPOLYTOPE_FHT)
        return fail(PF_ERR_INVALID_ARG, "pool_bits must be >= 0, and pooling needs PF_SIMHASH or PF_CROSSPOLYTOPE");
      const Layout lay0 = make_layout(prm->family, prm->d);
      pool_fns = prm->pool_bits / lay0.ell;
      if (pool_fns < lay0.fns) return fail(PF_ERR_INVALID_ARG, "the pool must hold at least one table's functions");
    }
    int64_t L = prm->num_tables > 0 ? prm->num_tables
                                    : budget_tables(prm->family, prm->n, prm->d, M, prm->memory_budget_bytes,
                                                    prm->sketch_layout, prm->row_storage, prm->fp8_rows, pool_fns);
    if (L < 1) return fail(PF_ERR_BUDGET_TOO_SMALL, "memory budget leaves room for no repetition");
    if (prm->num_tables > kMaxL)
      return fail(PF_ERR_INVALID_ARG, "num_tables above " + std::to_string(kMaxL) + " is not supported");
    if (L > kMaxL) L = kMaxL;  // only a budget-derived L is clamped
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    pf_index* ix = new pf_index();
    try {
      PF_CK(cudaGetDevice(&ix->device));
      PF_CK(cudaDeviceGetAttribute(&ix->num_sms, cudaDevAttrMultiProcessorCount, ix->device));
      ix->n = prm->n;
      ix->d = prm->d;
      ix->family = prm->family;
      ix->L = int(L);
      ix->M = M;
      ix->B = B;
      ix->lay = make_layout(prm->family, prm->d);
      ix->budget = prm->memory_budget_bytes;
      ix->sketch_layout = prm->sketch_layout;
      ix->row_storage = prm->row_storage;
      ix->bytes_used =
          resident_bytes(prm->family, prm->n, prm->d, M, ix->L, prm->sketch_layout, prm->row_storage, prm->fp8_rows,
                         pool_fns);
      const int dp = ix->lay.d_pad;
      const int64_t n = ix->n;
      ix->pool_fns = pool_fns;
      ix->pool_tables = pool_fns > 0 ? (pool_fns + ix->lay.fns - 1) / ix->lay.fns : 0;
      ix->hash_rows = int64_t(pool_fns > 0 ? ix->pool_tables : ix->L) * ix->lay.rows_table + 64LL * M;
      // bound on |bfloat16 estimate - canonical float32 similarity| for unit
      // vectors: 2^-8 from rounding the row to bfloat16, plus the float32
      // accumulation error of both sums (each <= d_pad * 2^-24 * |q||x|)
      ix->bf16_err = float(std::ldexp(1.0, -8) * (1.0 + std::ldexp(1.0, -20)) + 2.2 * dp * std::ldexp(1.0, -24));

      if (ix->row_storage == PF_ROWS_F16)
        dalloc(&ix->xf16, size_t(n) * dp);
      else
        dalloc(&ix->x32, size_t(n) * dp);
      dalloc(&ix->x16, size_t(n) * dp);
      if (prm->fp8_rows) {
        dalloc(&ix->x8, size_t(n) * dp);
        dalloc(&ix->x8_meta, size_t(n));
      }
      if (ix->sketch_layout == PF_SKETCH_PER_POINT)
        dalloc(&ix->sk, size_t(n) * M);
      else
        dalloc(&ix->skc, size_t(n) * ix->L);
      dalloc(&ix->W32, size_t(ix->hash_rows) * dp);
      dalloc(&ix->Whi, size_t(ix->hash_rows) * dp);
      dalloc(&ix->Wthr, size_t(ix->hash_rows));
      dalloc(&ix->codes, size_t(n) * ix->L);
      dalloc(&ix->ids, size_t(n) * ix->L);
      dalloc(&ix->pfx, size_t(kPrefixSize) * ix->L);
      dalloc(&ix->cos_tab, 65);
      dalloc(&ix->dev_error, 16);
      PF_CK(cudaMemsetAsync(ix->dev_error, 0, 16 * sizeof(int32_t), s));
      const bool cp_table = ix->family == PF_CROSSPOLYTOPE || ix->family == PF_CROSSPOLYTOPE_FHT;
      if (cp_table) dalloc(&ix->cpP, size_t(kAlphaSteps) * (ix->lay.ell + 1));
      if (ix->family == PF_CROSSPOLYTOPE_FHT) {
        const size_t words = size_t(ix->L) * ix->lay.fns * 3 * ix->lay.fht_words;
        dalloc(&ix->fht_signs, words);
        std::vector<uint32_t> sg(words);
        gen_fht_signs(prm->seed, ix->L, ix->lay, sg.data());
        PF_CK(cudaMemcpy(ix->fht_signs, sg.data(), sizeof(uint32_t) * words, cudaMemcpyHostToDevice));
        fht_bands(prm->d, ix->lay, &ix->fht_gap, &ix->fht_sign);
      }

      // random parameters on the host (bit-reproducible from the seed)
      std::vector<float> W(size_t(ix->hash_rows) * dp), thr(size_t(ix->hash_rows));
      if (pool_fns > 0) {
        gen_pool_rows(prm->seed, prm->family, pool_fns, M, prm->d, ix->lay, W.data(), thr.data());
        std::vector<int32_t> sel(size_t(ix->L) * ix->lay.fns);
        pool_select(prm->seed, ix->L, ix->lay.fns, pool_fns, sel.data());
        dalloc(&ix->pool_sel, sel.size());
        PF_CK(cudaMemcpy(ix->pool_sel, sel.data(), sizeof(int32_t) * sel.size(), cudaMemcpyHostToDevice));
      } else {
        gen_hash_rows(prm->seed, prm->family, ix->L, M, prm->d, ix->lay, W.data(), thr.data());
      }
      PF_CK(cudaMemcpyAsync(ix->W32, W.data(), sizeof(float) * W.size(), cudaMemcpyHostToDevice, s));
      PF_CK(cudaMemcpyAsync(ix->Wthr, thr.data(), sizeof(float) * thr.size(), cudaMemcpyHostToDevice, s));
      to_bf16_exact_kernel<<<1024, 256, 0, s>>>(ix->W32, int64_t(W.size()), ix->Whi);
      PF_CK(cudaGetLastError());
      std::vector<double> cosv(65);
      filter_cos_table(cosv.data());
      PF_CK(cudaMemcpyAsync(ix->cos_tab, cosv.data(), sizeof(double) * 65, cudaMemcpyHostToDevice, s));
      std::vector<double> P;
      if (cp_table) {
        P.resize(size_t(kAlphaSteps) * (ix->lay.ell + 1));
        if (ix->family == PF_CROSSPOLYTOPE_FHT)
          fht_collision_table(prm->seed, ix->lay, draws, P.data());
        else
          cp_collision_table(prm->seed, prm->d, ix->lay.ell, draws, P.data());
        PF_CK(cudaMemcpyAsync(ix->cpP, P.data(), sizeof(double) * P.size(), cudaMemcpyHostToDevice, s));
      }

      // points -> device, normalise, hash, sort
      const float* pin = static_cast<const float*>(points);
      float* staged = nullptr;
      if (!on_device(points)) {
        dalloc(&staged, size_t(n) * prm->d);
        PF_CK(cudaMemcpyAsync(staged, points, sizeof(float) * size_t(n) * prm->d, cudaMemcpyHostToDevice, s));
        pin = staged;
      }
      uint32_t* raw_codes = nullptr;
      uint32_t* gcodes = nullptr;    // codes of the pool's groups, only while hashing a pooled index
      __nv_bfloat16* xlo = nullptr;  // low bfloat16 half of the rows, only while hashing
      RecheckReq* rq = nullptr;      // deferred float64 rechecks, only while hashing
      uint32_t* rq_count = nullptr;
      uint64_t* sk_tmp = nullptr;    // per-point sketches, only while building a per-table layout
      float* x32_tmp = nullptr;      // float32 rows, only while hashing binary16 rows
      int32_t herr = 0;
      try {
        uint64_t* sk_out = ix->sk;
        if (!sk_out) {
          dalloc(&sk_tmp, size_t(n) * M);
          sk_out = sk_tmp;
        }
        dalloc(&xlo, size_t(n) * dp);
        float* x32 = ix->x32;
        if (ix->row_storage == PF_ROWS_F16) {
          dalloc(&x32_tmp, size_t(n) * dp);
          x32 = x32_tmp;
        }
        PF_CK(launch_normalize(pin, n, prm->d, dp, x32, ix->x16, xlo, s));
        if (ix->row_storage == PF_ROWS_F16)  // the stored point is the binary16 row: hash that
          PF_CK(launch_round_rows_f16(x32, n, dp, ix->xf16, ix->x16, xlo, s));
        if (ix->x8) PF_CK(launch_quantize_fp8(x32, n, prm->d, dp, ix->x8, ix->x8_meta, s));
        dalloc(&raw_codes, size_t(n) * ix->L);
        const int hashed_tables = ix->pool_tables > 0 ? ix->pool_tables : ix->L;
        dalloc(&rq, recheck_capacity(ix, n, hashed_tables));
        dalloc(&rq_count, size_t(ix->num_sms));
        if (ix->pool_tables > 0) {  // the pool's functions once, then each table's subset
          dalloc(&gcodes, size_t(n) * ix->pool_tables);
          PF_CK(launch_hash(ix, x32, ix->x16, xlo, n, gcodes, n, 1, sk_out, n, 1, rq, rq_count,
                            recheck_capacity(ix, n, hashed_tables), s, ix->pool_tables));
          PF_CK(launch_pool_gather(ix, gcodes, n, 1, n, raw_codes, n, 1, s));
        } else {
          PF_CK(launch_hash(ix, x32, ix->x16, xlo, n, raw_codes, n, 1, sk_out, n, 1, rq, rq_count,
                            recheck_capacity(ix, n, hashed_tables), s));
        }
        PF_CK(sort_tables(ix, raw_codes, s));
        if (ix->skc) PF_CK(gather_table_sketches(ix, sk_out, ix->skc, s));
        PF_CK(cudaMemcpyAsync(&herr, ix->dev_error, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PF_CK(cudaStreamSynchronize(s));
      } catch (...) {
        cudaStreamSynchronize(s);
        dfree(staged);
        dfree(raw_codes);
        dfree(gcodes);
        dfree(xlo);
        dfree(rq);
        dfree(rq_count);
        dfree(sk_tmp);
        dfree(x32_tmp);
        throw;
      }
      dfree(staged);
      dfree(raw_codes);
      dfree(gcodes);
      dfree(xlo);
      dfree(rq);
      dfree(rq_count);
      dfree(sk_tmp);
      dfree(x32_tmp);
      PF_CK(cudaGetLastError());
      if (herr) throw Error{PF_ERR_DEVICE_TIMEOUT, "a bounded device-side wait of the hashing kernel timed out"};
    } catch (...) {
      destroy(ix);
      throw;
    }
    *out = ix;
    return PF_OK;
  });
}

pf_status pf_hash_queries(pf_index* ix, const float* queries, int64_t Q, uint32_t* qcodes, uint64_t* qsk,
                          void* stream) {
  return guarded([&]() -> pf_status {
    if (!ix) return fail(PF_ERR_INVALID_ARG, "null index");
    if (Q < 0 || Q > 0x7fffffffLL) return fail(PF_ERR_INVALID_ARG, "Q out of range");
    if (Q == 0) return PF_OK;  // an empty batch may pass null buffers
    if (!queries || !qcodes || !qsk) return fail(PF_ERR_INVALID_ARG, "null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PF_CK(cudaSetDevice(ix->device));
    ensure_ws(ix, Q, 1);
    const float* qd = stage_queries(ix, queries, Q, s);
    hash_queries_ws(ix, ix->ws, qd, Q, s);
    PF_CK(cudaMemcpyAsync(qcodes, ix->ws.qcodes, sizeof(uint32_t) * size_t(Q) * ix->L, cudaMemcpyDefault, s));
    PF_CK(cudaMemcpyAsync(qsk, ix->ws.qsk, sizeof(uint64_t) * size_t(Q) * ix->M, cudaMemcpyDefault, s));
    PF_CK(cudaStreamSynchronize(s));
    PF_CK(cudaGetLastError());
    if (device_timed_out(ix)) return fail(PF_ERR_DEVICE_TIMEOUT, "a bounded device-side wait timed out");
    return PF_OK;
  });
}

pf_status pf_index_search(pf_index* ix, const float* queries, int64_t Q, const int32_t* k, const double* recall,
                          int32_t k_max, uint32_t* out_ids, float* out_sims, pf_query_stats* stats,
                          const pf_search_opts* opts, void* stream) {
  return guarded([&]() -> pf_status {
    if (!ix) return fail(PF_ERR_INVALID_ARG, "null index");
    if (Q < 0 || Q > 0x7fffffffLL) return fail(PF_ERR_INVALID_ARG, "Q out of range");
    if (k_max < 1 || k_max > kMaxK) return fail(PF_ERR_INVALID_ARG, "k_max must be in [1, 128]");
    if (Q == 0) return PF_OK;  // an empty batch may pass null buffers
    if (!queries || !k || !recall || !out_ids || !out_sims) return fail(PF_ERR_INVALID_ARG, "null argument");
    pf_search_opts o;
    pf_search_opts_default(&o);
    if (opts) o = *opts;
    if (o.scoring < 0 || o.scoring > 2) return fail(PF_ERR_INVALID_ARG, "scoring must be 0, 1 or 2");
    if (o.scoring == 2 && !ix->x8) return fail(PF_ERR_INVALID_ARG, "scoring 2 needs an index built with fp8_rows");
    if (o.stop_every < 0) return fail(PF_ERR_INVALID_ARG, "stop_every must be >= 0");
    if (o.pool_rule != 0 && o.pool_rule != 1) return fail(PF_ERR_INVALID_ARG, "pool_rule must be 0 or 1");
    if (!(o.filter_eps >= 0.0 && o.filter_eps <= 1e6)) return fail(PF_ERR_INVALID_ARG, "filter_eps must be in [0, 1e6]");
    if (o.learned_start && !ix->mlp_trained) return fail(PF_ERR_NOT_TRAINED, "no start-depth model has been trained");
    if (Q == 0) return PF_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PF_CK(cudaSetDevice(ix->device));
    ensure_ws(ix, Q, k_max);
    pf_workspace& ws = ix->ws;
    // per-query k and recall are checked by the search kernel (error word 1)
    const float* qd = stage_queries(ix, queries, Q, s);
    const int32_t* kd = k;
    const double* rd = recall;
    const int32_t* sd = o.start_depth;
    if (!on_device(k)) { stage_in(ws.k, k, sizeof(int32_t) * Q, s); kd = ws.k; }
    if (!on_device(recall)) { stage_in(ws.recall, recall, sizeof(double) * Q, s); rd = ws.recall; }
    if (sd && !on_device(sd)) { stage_in(ws.start, sd, sizeof(int32_t) * Q, s); sd = ws.start; }
    const bool timing = o.timing != 0;
    if (timing) {
      for (auto& e : ix->ev)
        if (!e) PF_CK(cudaEventCreate(&e));
      PF_CK(cudaEventRecord(ix->ev[0], s));
    }
    hash_queries_ws(ix, ix->ws, qd, Q, s);
    if (o.learned_start) {
      predict_ws(ix, ix->ws, Q, s);
      sd = ws.start;
    }
    if (timing) PF_CK(cudaEventRecord(ix->ev[1], s));

    const bool ids_dev = on_device(out_ids), sims_dev = on_device(out_sims);
    const bool st_dev = stats && on_device(stats);
    SearchArgs a;
    a.Q = int(Q);
    a.qx = ws.qx;
    a.qcodes = ws.qcodes;
    a.qsk = ws.qsk;
    a.k = kd;
    a.recall = rd;
    a.start = sd;
    a.k_max = k_max;
    a.filter = o.filter ? 1 : 0;
    a.scoring = o.scoring;
    a.stop_every = o.stop_every;
    a.pool_rule = o.pool_rule;
    a.cos_tab = slack_table(ws, o.filter_eps, s);
    a.out_ids = ids_dev ? out_ids : ws.ids;
    a.out_sims = sims_dev ? out_sims : ws.sims;
    a.stats = stats ? (st_dev ? stats : ws.stats) : nullptr;
    a.counter = ws.counter;
    PF_CK(cudaMemsetAsync(ws.counter, 0, sizeof(int32_t) * 64, s));
    PF_CK(launch_search(ix, a, s));
    if (timing) PF_CK(cudaEventRecord(ix->ev[2], s));
    if (!ids_dev)
      PF_CK(cudaMemcpyAsync(out_ids, ws.ids, sizeof(uint32_t) * size_t(Q) * k_max, cudaMemcpyDeviceToHost, s));
    if (!sims_dev)
      PF_CK(cudaMemcpyAsync(out_sims, ws.sims, sizeof(float) * size_t(Q) * k_max, cudaMemcpyDeviceToHost, s));
    if (stats && !st_dev)
      PF_CK(cudaMemcpyAsync(stats, ws.stats, sizeof(pf_query_stats) * size_t(Q), cudaMemcpyDeviceToHost, s));
    int32_t flags = 0;
    PF_CK(cudaMemcpyAsync(&flags, ws.counter + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PF_CK(cudaStreamSynchronize(s));
    PF_CK(cudaGetLastError());
    if (device_timed_out(ix)) return fail(PF_ERR_DEVICE_TIMEOUT, "a bounded device-side wait timed out");
    if (flags & 1) return fail(PF_ERR_INVALID_ARG, "some k not in [1, k_max] or recall not in (0, 1)");
    if (timing) {
      PF_CK(cudaEventElapsedTime(&ix->last_ms[0], ix->ev[0], ix->ev[1]));
      PF_CK(cudaEventElapsedTime(&ix->last_ms[1], ix->ev[1], ix->ev[2]));
      PF_CK(cudaEventElapsedTime(&ix->last_ms[2], ix->ev[0], ix->ev[2]));
    }
    return PF_OK;
  });
}

pf_status pf_index_last_timing(const pf_index* ix, float* t, int32_t count) {
  if (!ix || !t || count < 0 || count > 3) return fail(PF_ERR_INVALID_ARG, "bad argument");
  for (int i = 0; i < count; ++i) t[i] = ix->last_ms[i];
  return PF_OK;
}

pf_status pf_index_info(const pf_index* ix, pf_index_info_t* info) {
  if (!ix || !info) return fail(PF_ERR_INVALID_ARG, "null argument");
  std::memset(info, 0, sizeof(*info));
  info->n = ix->n;
  info->d = ix->d;
  info->d_pad = ix->lay.d_pad;
  info->family = ix->family;
  info->L = ix->L;
  info->Kb = ix->lay.Kb;
  info->ell = ix->lay.ell;
  info->fns = ix->lay.fns;
  info->M = ix->M;
  info->B = ix->B;
  info->trained = ix->mlp_trained;
  info->sketch_layout = ix->sketch_layout;
  info->row_storage = ix->row_storage;
  info->bytes_used = ix->bytes_used;
  info->budget_bytes = ix->budget;
  return PF_OK;
}

pf_status pf_index_array(const pf_index* ix, int32_t which, const void** ptr, uint64_t* bytes) {
  if (!ix || !ptr || !bytes) return fail(PF_ERR_INVALID_ARG, "null argument");
  const uint64_t n = uint64_t(ix->n), dp = uint64_t(ix->lay.d_pad), L = uint64_t(ix->L);
  switch (which) {
    case PF_ARRAY_ROWS_F32:
      if (!ix->x32) return fail(PF_ERR_INVALID_ARG, "index keeps its rows in binary16");
      *ptr = ix->x32;
      *bytes = n * dp * 4;
      break;
    case PF_ARRAY_ROWS_F16:
      if (!ix->xf16) return fail(PF_ERR_INVALID_ARG, "index keeps its rows in float32");
      *ptr = ix->xf16;
      *bytes = n * dp * 2;
      break;
    case PF_ARRAY_ROWS_BF16: *ptr = ix->x16; *bytes = n * dp * 2; break;
    case PF_ARRAY_CODES: *ptr = ix->codes; *bytes = n * L * 4; break;
    case PF_ARRAY_IDS: *ptr = ix->ids; *bytes = n * L * 4; break;
    case PF_ARRAY_PREFIX: *ptr = ix->pfx; *bytes = uint64_t(kPrefixSize) * L * 4; break;
    case PF_ARRAY_SKETCHES:
      if (!ix->sk) return fail(PF_ERR_INVALID_ARG, "index keeps its sketches per repetition");
      *ptr = ix->sk;
      *bytes = n * uint64_t(ix->M) * 8;
      break;
    case PF_ARRAY_TABLE_SKETCHES:
      if (!ix->skc) return fail(PF_ERR_INVALID_ARG, "index keeps its sketches per point");
      *ptr = ix->skc;
      *bytes = n * L * 8;
      break;
    case PF_ARRAY_HASH_ROWS: *ptr = ix->W32; *bytes = uint64_t(ix->hash_rows) * dp * 4; break;
    case PF_ARRAY_CP_TABLE:
      if (!ix->cpP) return fail(PF_ERR_INVALID_ARG, "index has no CP table");
      *ptr = ix->cpP;
      *bytes = uint64_t(kAlphaSteps) * (ix->lay.ell + 1) * 8;
      break;
    case PF_ARRAY_FHT_SIGNS:
      if (!ix->fht_signs) return fail(PF_ERR_INVALID_ARG, "index is not of the pseudo-random cross-polytope family");
      *ptr = ix->fht_signs;
      *bytes = uint64_t(ix->L) * ix->lay.fns * 3 * ix->lay.fht_words * 4;
      break;
    case PF_ARRAY_ROWS_FP8:
    case PF_ARRAY_FP8_META:
      if (!ix->x8) return fail(PF_ERR_INVALID_ARG, "index was built without fp8_rows");
      *ptr = which == PF_ARRAY_ROWS_FP8 ? static_cast<const void*>(ix->x8) : static_cast<const void*>(ix->x8_meta);
      *bytes = which == PF_ARRAY_ROWS_FP8 ? n * dp : n * 8;
      break;
    case PF_ARRAY_POOL_SELECT:
      if (!ix->pool_sel) return fail(PF_ERR_INVALID_ARG, "index does not pool its functions");
      *ptr = ix->pool_sel;
      *bytes = uint64_t(ix->L) * ix->lay.fns * 4;
      break;
    case PF_ARRAY_MLP_F32:
    case PF_ARRAY_MLP_W1_BF16:
    case PF_ARRAY_MLP_W2_BF16: {
      if (!ix->mlp_trained) return fail(PF_ERR_NOT_TRAINED, "no start-depth model has been trained");
      const uint64_t F = uint64_t(ix->mlp_F), H = uint64_t(kMlpHidden), C = uint64_t(ix->mlp_C);
      if (which == PF_ARRAY_MLP_F32) {
        *ptr = ix->mlp_w;
        *bytes = (H * F + H + C * H + C) * 4;
      } else if (which == PF_ARRAY_MLP_W1_BF16) {
        *ptr = ix->mlp_w1h;
        *bytes = F * H * 2;
      } else {
        *ptr = ix->mlp_w2h;
        *bytes = C * H * 2;
      }
      break;
    }
    default: return fail(PF_ERR_INVALID_ARG, "unknown array");
  }
  return PF_OK;
}

pf_status pf_index_read_array(const pf_index* ix, int32_t which, void* dst, uint64_t dst_bytes, void* stream) {
  return guarded([&]() -> pf_status {
    const void* src = nullptr;
    uint64_t nb = 0;
    const pf_status st = pf_index_array(ix, which, &src, &nb);
    if (st != PF_OK) return st;
    if (!dst || dst_bytes < nb) return fail(PF_ERR_INVALID_ARG, "destination too small");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PF_CK(cudaMemcpyAsync(dst, src, nb, cudaMemcpyDefault, s));
    PF_CK(cudaStreamSynchronize(s));
    return PF_OK;
  });
}

pf_status pf_mlp_forward_backward(const float* X, const int32_t* y, int32_t B, int32_t F, int32_t H, int32_t C,
                                  const float* W1, const float* b1, const float* W2, const float* b2, float* loss,
                                  float* dW1, float* db1, float* dW2, float* db2, void* stream) {
  return guarded([&]() -> pf_status {
    if (!X || !y || !W1 || !b1 || !W2 || !b2 || !loss || !dW1 || !db1 || !dW2 || !db2)
      return fail(PF_ERR_INVALID_ARG, "null argument");
    if (B < 1 || F < 1 || H < 1 || C < 1) return fail(PF_ERR_INVALID_ARG, "sizes must be >= 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float *h = nullptr, *z = nullptr, *dz = nullptr, *dh = nullptr;
    try {
      dalloc(&h, size_t(B) * H);
      dalloc(&z, size_t(B) * C);
      dalloc(&dz, size_t(B) * C);
      dalloc(&dh, size_t(B) * H);
      PF_CK(mlp_forward_backward(X, y, B, F, H, C, W1, b1, W2, b2, loss, dW1, db1, dW2, db2, h, z, dz, dh, s));
      PF_CK(cudaStreamSynchronize(s));
    } catch (...) {
      cudaStreamSynchronize(s);
      dfree(h); dfree(z); dfree(dz); dfree(dh);
      throw;
    }
    dfree(h); dfree(z); dfree(dz); dfree(dh);
    return PF_OK;
  });
}

pf_status pf_learned_train(pf_index* ix, const float* train_queries, int64_t Qt, int32_t k, double recall,
                           int32_t epochs, uint64_t seed, pf_learned_report* report, void* stream) {
  return guarded([&]() -> pf_status {
    if (!ix || !train_queries) return fail(PF_ERR_INVALID_ARG, "null argument");
    if (Qt < 1 || Qt > 0x7fffffffLL) return fail(PF_ERR_INVALID_ARG, "Qt out of range");
    if (k < 1 || k > kMaxK) return fail(PF_ERR_INVALID_ARG, "k must be in [1, 128]");
    if (!(recall > 0.0 && recall < 1.0)) return fail(PF_ERR_INVALID_ARG, "recall not in (0, 1)");
    if (epochs < 1 || epochs > 100000) return fail(PF_ERR_INVALID_ARG, "epochs must be in [1, 100000]");
    if (ix->live_plans > 0) return fail(PF_ERR_INVALID_ARG, "search plans bound to the index exist");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PF_CK(cudaSetDevice(ix->device));
    const int F = ix->lay.d_pad + 64, H = kMlpHidden, C = ix->lay.Kb + 1;
    const int64_t nW1 = int64_t(H) * F, nW2 = int64_t(C) * H, nparam = nW1 + H + nW2 + C;
    const int Bt = 1024;
    // traces of the plain schedule: the stop depth of every training query
    const int64_t chunk = std::min<int64_t>(Qt, 32768);
    float *X = nullptr, *Xp = nullptr, *P = nullptr, *G = nullptr, *Mo = nullptr, *Vo = nullptr;
    float *h = nullptr, *z = nullptr, *dz = nullptr, *dh = nullptr, *losses = nullptr;
    int32_t *y = nullptr, *yp = nullptr, *perm = nullptr, *kk = nullptr;
    double* rr = nullptr;
    __nv_bfloat16 *w1h = nullptr, *w2h = nullptr;
    auto cleanup = [&]() {
      dfree(X); dfree(Xp); dfree(P); dfree(G); dfree(Mo); dfree(Vo); dfree(h); dfree(z); dfree(dz); dfree(dh);
      dfree(losses); dfree(y); dfree(yp); dfree(perm); dfree(kk); dfree(rr); dfree(w1h); dfree(w2h);
    };
    std::vector<int32_t> hy(Qt);
    try {
      dalloc(&X, size_t(Qt) * F);
      dalloc(&Xp, size_t(Qt) * F);
      dalloc(&y, size_t(Qt));
      dalloc(&yp, size_t(Qt));
      dalloc(&perm, size_t(Qt));
      dalloc(&kk, size_t(chunk));
      dalloc(&rr, size_t(chunk));
      ensure_ws(ix, chunk, k);
      pf_workspace& ws = ix->ws;
      {
        std::vector<int32_t> kv(chunk, k);
        std::vector<double> rv(chunk, recall);
        PF_CK(cudaMemcpyAsync(kk, kv.data(), sizeof(int32_t) * chunk, cudaMemcpyHostToDevice, s));
        PF_CK(cudaMemcpyAsync(rr, rv.data(), sizeof(double) * chunk, cudaMemcpyHostToDevice, s));
        PF_CK(cudaStreamSynchronize(s));
      }
      std::vector<pf_query_stats> st(chunk);
      for (int64_t q0 = 0; q0 < Qt; q0 += chunk) {
        const int64_t nq = std::min(chunk, Qt - q0);
        const float* src = train_queries + size_t(q0) * ix->d;
        const float* qd = stage_queries(ix, src, nq, s);
        hash_queries_ws(ix, ix->ws, qd, nq, s);
        SearchArgs a;
        a.Q = int(nq);
        a.qx = ws.qx;
        a.qcodes = ws.qcodes;
        a.qsk = ws.qsk;
        a.k = kk;
        a.recall = rr;
        a.k_max = k;
        a.filter = 1;
        a.scoring = 1;
        a.out_ids = ws.ids;
        a.out_sims = ws.sims;
        a.stats = ws.stats;
        a.counter = ws.counter;
        PF_CK(cudaMemsetAsync(ws.counter, 0, sizeof(int32_t) * 64, s));
        PF_CK(launch_search(ix, a, s));
        PF_CK(mlp_features(ws.qx, ws.qsk, int(nq), ix->lay.d_pad, ix->M, X + size_t(q0) * F, s));
        PF_CK(cudaMemcpyAsync(st.data(), ws.stats, sizeof(pf_query_stats) * nq, cudaMemcpyDeviceToHost, s));
        PF_CK(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < nq; ++i) hy[q0 + i] = st[i].stop_depth;
      }
      if (device_timed_out(ix)) throw Error{PF_ERR_DEVICE_TIMEOUT, "a bounded device-side wait timed out"};
      PF_CK(cudaMemcpyAsync(y, hy.data(), sizeof(int32_t) * Qt, cudaMemcpyHostToDevice, s));
      // weights: W1 ~ N(0, 2/F), W2 ~ N(0, 1/H), zero biases (host, from the seed)
      std::vector<float> hp(nparam, 0.f);
      const float s1 = std::sqrt(2.f / float(F)), s2 = std::sqrt(1.f / float(H));
      for (int64_t i = 0; i < nW1; ++i) hp[i] = s1 * gaussian(seed, 4u, 0u, uint32_t(i / F), uint32_t(i % F));
      for (int64_t i = 0; i < nW2; ++i)
        hp[nW1 + H + i] = s2 * gaussian(seed, 4u, 1u, uint32_t(i / H), uint32_t(i % H));
      dalloc(&P, size_t(nparam));
      dalloc(&G, size_t(nparam));
      dalloc(&Mo, size_t(nparam));
      dalloc(&Vo, size_t(nparam));
      PF_CK(cudaMemcpyAsync(P, hp.data(), sizeof(float) * nparam, cudaMemcpyHostToDevice, s));
      PF_CK(cudaMemsetAsync(Mo, 0, sizeof(float) * nparam, s));
      PF_CK(cudaMemsetAsync(Vo, 0, sizeof(float) * nparam, s));
      dalloc(&h, size_t(Bt) * H);
      dalloc(&z, size_t(Bt) * C);
      dalloc(&dz, size_t(Bt) * C);
      dalloc(&dh, size_t(Bt) * H);
      const int nb = int((Qt + Bt - 1) / Bt);
      dalloc(&losses, size_t(nb));
      float *W1 = P, *b1 = P + nW1, *W2 = b1 + H, *b2 = W2 + nW2;
      float *gW1 = G, *gb1 = G + nW1, *gW2 = gb1 + H, *gb2 = gW2 + nW2;
      std::mt19937_64 rng(seed ^ 0x5DEECE66DULL);
      std::vector<int32_t> order(Qt);
      std::iota(order.begin(), order.end(), 0);
      int t = 0;
      float last_loss = 0.f;
      for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(order.begin(), order.end(), rng);
        PF_CK(cudaMemcpyAsync(perm, order.data(), sizeof(int32_t) * Qt, cudaMemcpyHostToDevice, s));
        PF_CK(gather_rows(X, perm, int(Qt), F, Xp, s));
        PF_CK(gather_rows(reinterpret_cast<const float*>(y), perm, int(Qt), 1, reinterpret_cast<float*>(yp), s));
        for (int b = 0; b < nb; ++b) {
          const int B = int(std::min<int64_t>(Bt, Qt - int64_t(b) * Bt));
          PF_CK(mlp_forward_backward(Xp + size_t(b) * Bt * F, yp + size_t(b) * Bt, B, F, H, C, W1, b1, W2, b2,
                                     losses + b, gW1, gb1, gW2, gb2, h, z, dz, dh, s));
          PF_CK(adam_step(P, G, Mo, Vo, nparam, 1e-3f, ++t, s));
        }
        if (ep == epochs - 1) {
          std::vector<float> hl(nb);
          PF_CK(cudaMemcpyAsync(hl.data(), losses, sizeof(float) * nb, cudaMemcpyDeviceToHost, s));
          PF_CK(cudaStreamSynchronize(s));
          double sum = 0.0, wsum = 0.0;
          for (int b = 0; b < nb; ++b) {
            const double wgt = double(std::min<int64_t>(Bt, Qt - int64_t(b) * Bt));
            sum += hl[b] * wgt;
            wsum += wgt;
          }
          last_loss = float(sum / wsum);
        }
      }
      dalloc(&w1h, size_t(nW1));
      dalloc(&w2h, size_t(nW2));
      PF_CK(to_bf16_transposed(W1, w1h, H, F, s));  // [H][F] -> [F][H]
      PF_CK(to_bf16(W2, w2h, nW2, s));
      PF_CK(cudaStreamSynchronize(s));
      // install the model
      dfree(ix->mlp_w);
      dfree(ix->mlp_w1h);
      dfree(ix->mlp_w2h);
      ix->mlp_w = P;
      P = nullptr;
      ix->mlp_w1h = w1h;
      w1h = nullptr;
      ix->mlp_w2h = w2h;
      w2h = nullptr;
      ix->mlp_F = F;
      ix->mlp_C = C;
      ix->mlp_trained = 1;
      if (report) {
        // predicted start depths on the training queries
        int64_t covered = 0;
        double sum_start = 0.0, sum_stop = 0.0;
        std::vector<int32_t> sd(chunk);
        for (int64_t q0 = 0; q0 < Qt; q0 += chunk) {
          const int64_t nq = std::min(chunk, Qt - q0);
          const float* qd = stage_queries(ix, train_queries + size_t(q0) * ix->d, nq, s);
          hash_queries_ws(ix, ix->ws, qd, nq, s);
          predict_ws(ix, ix->ws, nq, s);
          PF_CK(cudaMemcpyAsync(sd.data(), ws.start, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, s));
          PF_CK(cudaStreamSynchronize(s));
          for (int64_t i = 0; i < nq; ++i) {
            covered += sd[i] - ix->mlp_margin >= hy[q0 + i] || sd[i] == ix->lay.Kb ? 1 : 0;
            sum_start += sd[i];
            sum_stop += hy[q0 + i];
          }
        }
        if (device_timed_out(ix)) throw Error{PF_ERR_DEVICE_TIMEOUT, "a bounded device-side wait timed out"};
        report->final_loss = last_loss;
        report->train_accuracy = float(double(covered) / double(Qt));
        report->mean_stop = float(sum_stop / double(Qt));
        report->mean_start = float(sum_start / double(Qt));
        report->samples = int32_t(Qt);
        report->epochs = epochs;
      }
    } catch (...) {
      cudaStreamSynchronize(s);
      cleanup();
      throw;
    }
    cleanup();
    return PF_OK;
  });
}

pf_status pf_learned_predict(pf_index* ix, const float* queries, int64_t Q, int32_t* start_depth, void* stream) {
  return guarded([&]() -> pf_status {
    if (!ix) return fail(PF_ERR_INVALID_ARG, "null index");
    if (!ix->mlp_trained) return fail(PF_ERR_NOT_TRAINED, "no start-depth model has been trained");
    if (Q < 0 || Q > 0x7fffffffLL) return fail(PF_ERR_INVALID_ARG, "Q out of range");
    if (Q == 0) return PF_OK;
    if (!queries || !start_depth) return fail(PF_ERR_INVALID_ARG, "null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PF_CK(cudaSetDevice(ix->device));
    ensure_ws(ix, Q, 1);
    const float* qd = stage_queries(ix, queries, Q, s);
    hash_queries_ws(ix, ix->ws, qd, Q, s);
    predict_ws(ix, ix->ws, Q, s);
    PF_CK(cudaMemcpyAsync(start_depth, ix->ws.start, sizeof(int32_t) * size_t(Q), cudaMemcpyDefault, s));
    PF_CK(cudaStreamSynchronize(s));
    if (device_timed_out(ix)) return fail(PF_ERR_DEVICE_TIMEOUT, "a bounded device-side wait timed out");
    return PF_OK;
  });
}

pf_status pf_index_selftest_timeout(pf_index* ix, const float* queries, int64_t Q, void* stream) {
  return guarded([&]() -> pf_status {
    if (!ix || !queries) return fail(PF_ERR_INVALID_ARG, "null argument");
    if (Q < 1 || Q > 0x7fffffffLL) return fail(PF_ERR_INVALID_ARG, "Q out of range");
    if (ix->live_plans > 0) return fail(PF_ERR_INVALID_ARG, "search plans bound to the index exist");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PF_CK(cudaSetDevice(ix->device));
    ensure_ws(ix, Q, 1);
    const float* qd = stage_queries(ix, queries, Q, s);
    struct Hold {
      pf_index* ix;
      ~Hold() { ix->hold_weight_loads = 0; }
    } hold{ix};
    ix->hold_weight_loads = 1;
    hash_queries_ws(ix, ix->ws, qd, Q, s);
    PF_CK(cudaStreamSynchronize(s));
    ix->hold_weight_loads = 0;
    PF_CK(cudaGetLastError());
    if (device_timed_out(ix)) return fail(PF_ERR_DEVICE_TIMEOUT, "a bounded device-side wait timed out");
    return PF_OK;
  });
}

pf_status pf_learned_set_start_rule(pf_index* ix, float tail, int32_t margin) {
  return guarded([&]() -> pf_status {
    if (!ix) return fail(PF_ERR_INVALID_ARG, "null index");
    if (!(tail > 0.f && tail < 1.f) || margin < 0 || margin > 32)
      return fail(PF_ERR_INVALID_ARG, "tail must be in (0, 1) and margin in [0, 32]");
    if (ix->live_plans > 0) return fail(PF_ERR_INVALID_ARG, "search plans bound to the index exist");
    ix->mlp_tail = tail;
    ix->mlp_margin = margin;
    return PF_OK;
  });
}

pf_status pf_index_count_range_paths(pf_index* ix, int32_t enable, uint64_t* counts) {
  return guarded([&]() -> pf_status {
    if (!ix) return fail(PF_ERR_INVALID_ARG, "null index");
    PF_CK(cudaSetDevice(ix->device));
    PF_CK(cudaDeviceSynchronize());
    uint64_t c[5] = {0, 0, 0, 0, 0};
    if (ix->path_count) {
      PF_CK(cudaMemcpy(c, ix->path_count, sizeof(c), cudaMemcpyDeviceToHost));
      PF_CK(cudaMemset(ix->path_count, 0, sizeof(c)));
    }
    if (counts)
      for (int i = 0; i < 5; ++i) counts[i] = c[i];
    if (enable && !ix->path_count) {
      dalloc(&ix->path_count, 5);
      PF_CK(cudaMemset(ix->path_count, 0, 5 * sizeof(unsigned long long)));
    } else if (!enable && ix->path_count) {
      if (ix->live_plans > 0) return fail(PF_ERR_INVALID_ARG, "search plans bound to the index exist");
      dfree(ix->path_count);
    }
    return PF_OK;
  });
}

pf_status pf_index_selftest_hold(pf_index* ix, int32_t hold) {
  return guarded([&]() -> pf_status {
    if (!ix) return fail(PF_ERR_INVALID_ARG, "null index");
    ix->hold_weight_loads = hold ? 1 : 0;
    return PF_OK;
  });
}

void pf_index_free(pf_index* ix) {
  if (ix && ix->live_plans > 0) {
    set_error("pf_index_free: search plans bound to the index still exist; free them first");
    return;
  }
  destroy(ix);
}

// ---------------------------------------------------------------- tuning
pf_status pf_index_tune(pf_index* ix, const float* queries, int64_t Q, int32_t k, double recall,
                        const pf_search_opts* opts, pf_tune_report* report, void* stream) {
  return guarded([&]() -> pf_status {
    if (!ix || !queries) return fail(PF_ERR_INVALID_ARG, "null argument");
    if (Q < 1 || Q > 0x7fffffffLL) return fail(PF_ERR_INVALID_ARG, "Q must be in [1, 2^31-1]");
    if (k < 1 || k > kMaxK) return fail(PF_ERR_INVALID_ARG, "k must be in [1, 128]");
    if (!(recall > 0.0 && recall < 1.0)) return fail(PF_ERR_INVALID_ARG, "recall must be in (0, 1)");
    if (ix->live_plans > 0) return fail(PF_ERR_INVALID_ARG, "search plans bound to the index exist");
    pf_search_opts o;
    pf_search_opts_default(&o);
    if (opts) o = *opts;
    if (o.scoring < 0 || o.scoring > 2) return fail(PF_ERR_INVALID_ARG, "scoring must be 0, 1 or 2");
    if (o.scoring == 2 && !ix->x8) return fail(PF_ERR_INVALID_ARG, "scoring 2 needs an index built with fp8_rows");
    if (o.stop_every < 0) return fail(PF_ERR_INVALID_ARG, "stop_every must be >= 0");
    if (o.pool_rule != 0 && o.pool_rule != 1) return fail(PF_ERR_INVALID_ARG, "pool_rule must be 0 or 1");
    if (!(o.filter_eps >= 0.0 && o.filter_eps <= 1e6)) return fail(PF_ERR_INVALID_ARG, "filter_eps must be in [0, 1e6]");
    if (o.learned_start && !ix->mlp_trained) return fail(PF_ERR_NOT_TRAINED, "no start-depth model has been trained");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PF_CK(cudaSetDevice(ix->device));
    ensure_ws(ix, Q, k);
    pf_workspace& ws = ix->ws;
    const float* qd = stage_queries(ix, queries, Q, s);
    {
      std::vector<int32_t> kv(size_t(Q), k);
      std::vector<double> rv(size_t(Q), recall);
      PF_CK(cudaMemcpyAsync(ws.k, kv.data(), sizeof(int32_t) * size_t(Q), cudaMemcpyHostToDevice, s));
      PF_CK(cudaMemcpyAsync(ws.recall, rv.data(), sizeof(double) * size_t(Q), cudaMemcpyHostToDevice, s));
      PF_CK(cudaStreamSynchronize(s));
    }
    const int32_t* sd = o.start_depth;
    if (sd && !on_device(sd)) {
      stage_in(ws.start, sd, sizeof(int32_t) * size_t(Q), s);
      sd = ws.start;
    }
    hash_queries_ws(ix, ws, qd, Q, s);
    if (o.learned_start) {
      predict_ws(ix, ws, Q, s);
      sd = ws.start;
    }
    SearchArgs a;
    a.Q = int(Q);
    a.qx = ws.qx;
    a.qcodes = ws.qcodes;
    a.qsk = ws.qsk;
    a.k = ws.k;
    a.recall = ws.recall;
    a.start = sd;
    a.k_max = k;
    a.filter = o.filter ? 1 : 0;
    a.scoring = o.scoring;
    a.stop_every = o.stop_every;
    a.pool_rule = o.pool_rule;
    a.cos_tab = slack_table(ws, o.filter_eps, s);
    a.out_ids = ws.ids;
    a.out_sims = ws.sims;
    a.stats = nullptr;
    a.counter = ws.counter;
    std::vector<SearchShape> cand;
    for (const auto& uw : {std::pair<int, int>{8, 4}, {4, 4}, {8, 8}}) {
      const int mx = search_max_ctas_per_sm(ix, k, uw.first, uw.second);
      for (int c = mx; c >= 1 && c >= mx - 2; --c)
        for (int ff : {0, 3}) cand.push_back(SearchShape{uw.first, c, uw.second, ff});
    }
    if (cand.empty()) return fail(PF_ERR_CUDA, "no launchable search shape");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PF_CK(cudaEventCreate(&e0));
    PF_CK(cudaEventCreate(&e1));
    float best = 0.f, dflt = 0.f;
    SearchShape pick = cand[0];
    try {
      for (size_t i = 0; i < cand.size(); ++i) {
        a.shape = cand[i];
        float t = 0.f;
        for (int rep = 0; rep < 3; ++rep) {  // the first run warms up; the best of two timed runs
          PF_CK(cudaMemsetAsync(ws.counter, 0, sizeof(int32_t) * 64, s));
          PF_CK(cudaEventRecord(e0, s));
          PF_CK(launch_search(ix, a, s));
          PF_CK(cudaEventRecord(e1, s));
          PF_CK(cudaEventSynchronize(e1));
          float ms = 0.f;
          PF_CK(cudaEventElapsedTime(&ms, e0, e1));
          if (rep == 1 || (rep == 2 && ms < t)) t = ms;
        }
        if (i == 0) dflt = t;
        if (i == 0 || t < best) {
          best = t;
          pick = cand[i];
        }
      }
    } catch (...) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (device_timed_out(ix)) return fail(PF_ERR_DEVICE_TIMEOUT, "a bounded device-side wait timed out");
    ix->search_shape = pick;
    if (report) {
      report->unroll = pick.unroll;
      report->warps = pick.warps;
      report->ctas_per_sm = pick.ctas_per_sm;
      report->flat_fill = pick.flat_fill;
      report->candidates = int32_t(cand.size());
      report->best_ms = best;
      report->default_ms = dflt;
    }
    return PF_OK;
  });
}

pf_status pf_index_set_shape(pf_index* ix, int32_t unroll, int32_t warps, int32_t ctas_per_sm, int32_t flat_fill) {
  return guarded([&]() -> pf_status {
    if (!ix) return fail(PF_ERR_INVALID_ARG, "null index");
    if ((unroll != 4 && unroll != 8) || (warps != 4 && warps != 8) || (warps == 8 && unroll != 8) || ctas_per_sm < 0 ||
        flat_fill < 0 || flat_fill > 64)
      return fail(PF_ERR_INVALID_ARG,
                  "unroll must be 4 or 8, warps 4 or 8 (8 only with unroll 8), ctas_per_sm >= 0, flat_fill in [0, 64]");
    if (ix->live_plans > 0) return fail(PF_ERR_INVALID_ARG, "search plans bound to the index exist");
    ix->search_shape = SearchShape{unroll, ctas_per_sm, warps, flat_fill};
    return PF_OK;
  });
}

}  // extern "C"

// ---------------------------------------------------------------- plans
struct pf_search_plan {
  pf_index* ix = nullptr;
  int64_t Q = 0;
  int k_max = 0;
  pf_search_opts opts{};
  pf_plan_io io{};   // the caller's buffers (device or page-locked host)
  pf_plan_io dio{};  // the device buffers the kernels use: the caller's, or the plan's staging copies
  unsigned char* stage[7] = {};  // staging of the host buffers, in pf_plan_io's field order
  pf_workspace ws;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

// The captured sequence: the same steps as pf_index_search on device buffers.
// Host buffer -> staging copy size in bytes, per pf_plan_io field.
size_t io_bytes(const pf_search_plan* pl, int field) {
  const size_t Q = size_t(pl->Q), km = size_t(pl->k_max);
  switch (field) {
    case 0: return Q * size_t(pl->ix->d) * sizeof(float);
    case 1: return Q * sizeof(int32_t);
    case 2: return Q * sizeof(double);
    case 3: return Q * sizeof(int32_t);
    case 4: return Q * km * sizeof(uint32_t);
    case 5: return Q * km * sizeof(float);
    default: return Q * sizeof(pf_query_stats);
  }
}

void* io_field(pf_plan_io& io, int field) {
  switch (field) {
    case 0: return const_cast<float*>(io.queries);
    case 1: return const_cast<int32_t*>(io.k);
    case 2: return const_cast<double*>(io.recall);
    case 3: return const_cast<int32_t*>(io.start_depth);
    case 4: return io.out_ids;
    case 5: return io.out_sims;
    default: return io.stats;
  }
}

void set_io_field(pf_plan_io& io, int field, void* p) {
  switch (field) {
    case 0: io.queries = static_cast<const float*>(p); break;
    case 1: io.k = static_cast<const int32_t*>(p); break;
    case 2: io.recall = static_cast<const double*>(p); break;
    case 3: io.start_depth = static_cast<const int32_t*>(p); break;
    case 4: io.out_ids = static_cast<uint32_t*>(p); break;
    case 5: io.out_sims = static_cast<float*>(p); break;
    default: io.stats = static_cast<pf_query_stats*>(p); break;
  }
}

bool page_locked_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

void plan_sequence(pf_search_plan* pl, cudaStream_t s) {
  pf_index* ix = pl->ix;
  pf_workspace& ws = pl->ws;
  for (int f = 0; f <= 3; ++f)  // inputs held in host memory: copied in first
    if (pl->stage[f]) PF_CK(cudaMemcpyAsync(pl->stage[f], io_field(pl->io, f), io_bytes(pl, f), cudaMemcpyHostToDevice, s));
  const pf_plan_io& io = pl->dio;
  hash_queries_ws(ix, ws, io.queries, pl->Q, s);
  const int32_t* sd = io.start_depth;
  if (pl->opts.learned_start) {
    predict_ws(ix, ws, pl->Q, s);
    sd = ws.start;
  }
  SearchArgs a;
  a.Q = int(pl->Q);
  a.qx = ws.qx;
  a.qcodes = ws.qcodes;
  a.qsk = ws.qsk;
  a.k = io.k;
  a.recall = io.recall;
  a.start = sd;
  a.k_max = pl->k_max;
  a.filter = pl->opts.filter ? 1 : 0;
  a.scoring = pl->opts.scoring;
  a.stop_every = pl->opts.stop_every;
  a.pool_rule = pl->opts.pool_rule;
  a.cos_tab = pl->opts.filter_eps != 0.0 ? ws.cos_eps : nullptr;  // filled before the capture
  a.out_ids = io.out_ids;
  a.out_sims = io.out_sims;
  a.stats = io.stats;
  a.counter = ws.counter;
  PF_CK(cudaMemsetAsync(ws.counter, 0, sizeof(int32_t) * 64, s));
  PF_CK(launch_search(ix, a, s));
  for (int f = 4; f <= 6; ++f)  // outputs held in host memory: copied out last
    if (pl->stage[f]) PF_CK(cudaMemcpyAsync(io_field(pl->io, f), pl->stage[f], io_bytes(pl, f), cudaMemcpyDeviceToHost, s));
}

void plan_release(pf_search_plan* pl) {
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  free_ws(pl->ws);
  for (unsigned char*& p : pl->stage) dfree(p);
  delete pl;
}

}  // namespace

extern "C" {

pf_status pf_search_plan_create(pf_index* ix, int64_t Q, int32_t k_max, const pf_plan_io* io,
                                const pf_search_opts* opts, pf_search_plan** out) {
  return guarded([&]() -> pf_status {
    if (!ix || !io || !out) return fail(PF_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (Q < 1 || Q > 0x7fffffffLL) return fail(PF_ERR_INVALID_ARG, "Q must be in [1, 2^31-1]");
    if (k_max < 1 || k_max > kMaxK) return fail(PF_ERR_INVALID_ARG, "k_max must be in [1, 128]");
    PF_CK(cudaSetDevice(ix->device));
    const void* need[] = {io->queries, io->k, io->recall, io->out_ids, io->out_sims};
    for (const void* p : need)
      if (!p) return fail(PF_ERR_INVALID_ARG, "null plan buffer");
    const void* all[] = {io->queries, io->k, io->recall, io->start_depth, io->out_ids, io->out_sims, io->stats};
    bool host[7] = {};
    for (int f = 0; f < 7; ++f) {
      if (!all[f] || on_device(all[f])) continue;
      if (!page_locked_host(all[f]))
        return fail(PF_ERR_INVALID_ARG, "plan buffers must be device memory or page-locked host memory");
      host[f] = true;
    }
    pf_search_opts o;
    pf_search_opts_default(&o);
    if (opts) o = *opts;
    if (o.scoring < 0 || o.scoring > 2) return fail(PF_ERR_INVALID_ARG, "scoring must be 0, 1 or 2");
    if (o.scoring == 2 && !ix->x8) return fail(PF_ERR_INVALID_ARG, "scoring 2 needs an index built with fp8_rows");
    if (o.stop_every < 0) return fail(PF_ERR_INVALID_ARG, "stop_every must be >= 0");
    if (o.pool_rule != 0 && o.pool_rule != 1) return fail(PF_ERR_INVALID_ARG, "pool_rule must be 0 or 1");
    if (!(o.filter_eps >= 0.0 && o.filter_eps <= 1e6)) return fail(PF_ERR_INVALID_ARG, "filter_eps must be in [0, 1e6]");
    if (o.learned_start && !ix->mlp_trained) return fail(PF_ERR_NOT_TRAINED, "no start-depth model has been trained");
    o.start_depth = nullptr;
    o.timing = 0;
    pf_search_plan* pl = new pf_search_plan;
    pl->ix = ix;
    pl->Q = Q;
    pl->k_max = k_max;
    pl->opts = o;
    pl->io = *io;
    pl->dio = *io;
    cudaStream_t cs = nullptr;
    try {
      for (int f = 0; f < 7; ++f)
        if (host[f]) {
          dalloc(&pl->stage[f], io_bytes(pl, f));
          set_io_field(pl->dio, f, pl->stage[f]);
        }
      alloc_ws(ix, pl->ws, size_t(Q), size_t(k_max));
      slack_table(pl->ws, o.filter_eps, nullptr, true);
      PF_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      PF_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
      try {
        plan_sequence(pl, cs);
      } catch (...) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(cs, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      PF_CK(cudaStreamEndCapture(cs, &pl->graph));
      PF_CK(cudaGraphInstantiate(&pl->exec, pl->graph, 0));
      PF_CK(cudaStreamDestroy(cs));
      cs = nullptr;
    } catch (...) {
      if (cs) cudaStreamDestroy(cs);
      plan_release(pl);
      throw;
    }
    ix->live_plans += 1;
    *out = pl;
    return PF_OK;
  });
}

pf_status pf_search_plan_run(pf_search_plan* pl, void* stream) {
  return guarded([&]() -> pf_status {
    if (!pl) return fail(PF_ERR_INVALID_ARG, "null plan");
    PF_CK(cudaSetDevice(pl->ix->device));
    PF_CK(cudaGraphLaunch(pl->exec, static_cast<cudaStream_t>(stream)));
    return PF_OK;
  });
}

pf_status pf_search_plan_check(pf_search_plan* pl, void* stream) {
  return guarded([&]() -> pf_status {
    if (!pl) return fail(PF_ERR_INVALID_ARG, "null plan");
    PF_CK(cudaSetDevice(pl->ix->device));
    PF_CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int32_t flags = 0;
    PF_CK(cudaMemcpy(&flags, pl->ws.counter + 1, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (device_timed_out(pl->ix)) return fail(PF_ERR_DEVICE_TIMEOUT, "a bounded device-side wait timed out");
    if (flags & 1) return fail(PF_ERR_INVALID_ARG, "some k not in [1, k_max] or recall not in (0, 1)");
    return PF_OK;
  });
}

void pf_search_plan_free(pf_search_plan* pl) {
  if (!pl) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(pl->ix->device);
  cudaDeviceSynchronize();  // a launched graph may still be running
  pl->ix->live_plans -= 1;
  plan_release(pl);
  cudaSetDevice(prev);
}

}  // extern "C"
