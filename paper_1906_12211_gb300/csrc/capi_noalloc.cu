// pf_index_search_noalloc: the batched search for callers that cannot
// allocate device memory while they run -- for example a serving process whose
// device memory is handed out up front by another allocator, or a real-time
// path where an allocation's latency or failure is not acceptable.  The
// ordinary pf_index_search grows a per-index workspace with cudaMalloc; this
// entry point instead keeps its scratch (normalised queries, query codes and
// sketches, the work counter and error word) in one file-scope device array of
// fixed size, and calls no allocating routine.
//
// The array lives on every GPU on which the library is loaded, for the life of
// the process.  All calls share it and it keeps the previous call's contents;
// the parts that must start at zero are cleared by each call.  Two calls whose
// device work overlaps (different streams, or different host threads) race on
// the array: serialise them.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "pf_internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};

size_t round_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

size_t scratch_bytes(const pf_index* ix, int64_t Q) {
  return round_up(size_t(Q) * ix->lay.d_pad * sizeof(float)) + 2 * round_up(size_t(Q) * ix->lay.d_pad * 2) +
         round_up(size_t(Q) * ix->L * sizeof(uint32_t)) + round_up(size_t(Q) * ix->M * sizeof(uint64_t)) +
         round_up(64 + 65 * sizeof(double));  // work counter, error word, threshold table
}

bool device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

pf_status reject(pf_status s, const std::string& msg) {
  pf::set_error(msg);
  return s;
}

pf_status cuda_fail(cudaError_t e, const char* what) {
  return reject(PF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Device address of the scratch array on the current device (looked up once
// per device, on that device's first call).
cudaError_t scratch_address(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" pf_status pf_index_search_noalloc(pf_index* ix, const float* queries, int64_t Q, const int32_t* k,
                                             const double* recall, int32_t k_max, uint32_t* out_ids,
                                             float* out_sims, pf_query_stats* stats, const pf_search_opts* opts,
                                             void* stream) {
  try {
    pf::set_error("");
    if (!ix) return reject(PF_ERR_INVALID_ARG, "null index");
    if (Q < 0 || Q > 0x7fffffffLL) return reject(PF_ERR_INVALID_ARG, "Q out of range");
    if (k_max < 1 || k_max > pf::kMaxK) return reject(PF_ERR_INVALID_ARG, "k_max must be in [1, 128]");
    if (Q == 0) return PF_OK;
    pf_search_opts o;
    pf_search_opts_default(&o);
    if (opts) o = *opts;
    if (o.scoring < 0 || o.scoring > 2) return reject(PF_ERR_INVALID_ARG, "scoring must be 0, 1 or 2");
    if (o.scoring == 2 && !ix->x8) return reject(PF_ERR_INVALID_ARG, "scoring 2 needs an index built with fp8_rows");
    if (o.stop_every < 0) return reject(PF_ERR_INVALID_ARG, "stop_every must be >= 0");
    if (o.pool_rule != 0 && o.pool_rule != 1) return reject(PF_ERR_INVALID_ARG, "pool_rule must be 0 or 1");
    if (!(o.filter_eps >= 0.0 && o.filter_eps <= 1e6))
      return reject(PF_ERR_INVALID_ARG, "filter_eps must be in [0, 1e6]");
    if (ix->pool_tables > 0)
      return reject(PF_ERR_INVALID_ARG, "a pooled index needs pf_index_search (its pool codes use the index workspace)");
    if (o.learned_start)
      return reject(PF_ERR_INVALID_ARG, "the learned start depth needs pf_index_search (it uses the index workspace)");
    const size_t need = scratch_bytes(ix, Q);
    if (need > kScratchBytes) {
      const size_t per_q = size_t(ix->lay.d_pad) * 8 + size_t(ix->L) * 4 + size_t(ix->M) * 8;
      return reject(PF_ERR_INVALID_ARG,
                    "batch too large for the fixed 32 MiB search scratch: this index allows about " +
                        std::to_string((kScratchBytes - 8 * kAlign) / per_q) + " queries per call, got " +
                        std::to_string(Q));
    }
    if (ix->device < 0 || ix->device >= kMaxDevices) return reject(PF_ERR_INVALID_ARG, "device ordinal too large");
    cudaError_t e = cudaSetDevice(ix->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const void* must_be_device[] = {queries, k, recall, out_ids, out_sims};
    for (const void* p : must_be_device)
      if (!p || !device_pointer(p)) return reject(PF_ERR_INVALID_ARG, "all buffers must be device memory");
    if (stats && !device_pointer(stats)) return reject(PF_ERR_INVALID_ARG, "stats must be device memory");
    if (o.start_depth && !device_pointer(o.start_depth))
      return reject(PF_ERR_INVALID_ARG, "start_depth must be device memory");

    unsigned char* base = nullptr;
    if ((e = scratch_address(ix->device, &base)) != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
    float* qx = reinterpret_cast<float*>(base);
    base += round_up(size_t(Q) * ix->lay.d_pad * sizeof(float));
    __nv_bfloat16* qxh = reinterpret_cast<__nv_bfloat16*>(base);
    base += round_up(size_t(Q) * ix->lay.d_pad * 2);
    __nv_bfloat16* qxl = reinterpret_cast<__nv_bfloat16*>(base);
    base += round_up(size_t(Q) * ix->lay.d_pad * 2);
    uint32_t* qcodes = reinterpret_cast<uint32_t*>(base);
    base += round_up(size_t(Q) * ix->L * sizeof(uint32_t));
    uint64_t* qsk = reinterpret_cast<uint64_t*>(base);
    base += round_up(size_t(Q) * ix->M * sizeof(uint64_t));
    int32_t* counter = reinterpret_cast<int32_t*>(base);  // [0] work queue head, [1] error word
    double* cos_eps = reinterpret_cast<double*>(base + 64);  // [65] threshold table of a nonzero filter slack

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((e = cudaMemsetAsync(counter, 0, 64, s)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if ((e = pf::launch_normalize(queries, Q, ix->d, ix->lay.d_pad, qx, qxh, qxl, s)) != cudaSuccess)
      return cuda_fail(e, "normalize");
    // no deferred-recheck queue here: near-boundary hash decisions are rechecked inline
    if ((e = pf::launch_hash(ix, qx, qxh, qxl, Q, qcodes, 1, ix->L, qsk, 1, ix->M, nullptr, nullptr, 0, s)) !=
        cudaSuccess)
      return cuda_fail(e, "hash");
    pf::SearchArgs a;
    a.Q = int(Q);
    a.qx = qx;
    a.qcodes = qcodes;
    a.qsk = qsk;
    a.k = k;
    a.recall = recall;
    a.start = o.start_depth;
    a.k_max = k_max;
    a.filter = o.filter ? 1 : 0;
    a.scoring = o.scoring;
    a.stop_every = o.stop_every;
    a.pool_rule = o.pool_rule;
    if (o.filter_eps != 0.0) {
      double tab[65];
      pf::filter_cos_table(tab, o.filter_eps);
      if ((e = cudaMemcpyAsync(cos_eps, tab, sizeof(tab), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync");
      a.cos_tab = cos_eps;
    }
    a.out_ids = out_ids;
    a.out_sims = out_sims;
    a.stats = stats;
    a.counter = counter;
    if ((e = pf::launch_search(ix, a, s)) != cudaSuccess) return cuda_fail(e, "search");
    int32_t flags = 0;
    if ((e = cudaMemcpyAsync(&flags, counter + 1, sizeof(flags), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return cuda_fail(e, "cudaMemcpyAsync");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    int32_t herr = 0;
    if ((e = cudaMemcpy(&herr, ix->dev_error, sizeof(herr), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "cudaMemcpy");
    if (herr) {
      // clear the word (a memset allocates nothing), so that the next call on
      // this index is not reported as timed out too
      if ((e = cudaMemset(ix->dev_error, 0, sizeof(int32_t))) != cudaSuccess) return cuda_fail(e, "cudaMemset");
      return reject(PF_ERR_DEVICE_TIMEOUT, "a bounded device-side wait timed out");
    }
    if (flags & 1) return reject(PF_ERR_INVALID_ARG, "some k not in [1, k_max] or recall not in (0, 1)");
    return PF_OK;
  } catch (...) {
    return reject(PF_ERR_CUDA, "unexpected exception");
  }
}
