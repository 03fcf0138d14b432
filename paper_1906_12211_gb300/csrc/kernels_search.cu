// The adaptive k-NN query (Algorithm 1 as implemented in Sec. 4.1-4.2), one
// warp per query, persistent CTAs pulling queries from an atomic counter so
// queries of very different cost share one launch.
//
// Per round at prefix length i, for every repetition j the warp extends the
// range [l, r) of positions around the query's code so that it covers the
// block of codes sharing the first i bits, growing each side in whole
// segments of B entries (Sec. 4.2, App. C).  The new positions are streamed
// lane-parallel: position -> id -> sketch Hamming filter (Sec. 4.2) -> exact
// similarity -> top-k accumulator (unique ids, ordered by similarity then id).
// After the round the stop test of Lemma 1 runs in float64.
//
// Readings shared with the oracle: the sketch threshold and s_k are taken at
// the start of each round; the stop test runs once per round (Sec. 4.1); the
// canonical similarity is float32 with 32 partial sums (partial c takes the
// coordinates = c mod 32 in index order by fused multiply-add) combined as
// s[c] += s[c + w] for w = 16, 8, 4, 2, 1.  Because only the filter depends on
// the order of insertion and it uses the round's snapshot, the result does not
// depend on the order in which lanes visit candidates.
#include <cuda_bf16.h>

#include "pf_internal.h"

namespace pf {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 4;          // warps (queries in flight) per CTA
constexpr int kCandBuf = 64;       // compacted candidate ids per warp

struct Dev {
  int64_t n;
  int d, d_pad, L, Kb, M, B, family, ell;
  const float* x32;
  const __nv_bfloat16* x16;
  const uint32_t* codes;
  const uint32_t* ids;
  const uint32_t* pfx;
  const uint64_t* sk;
  const double* cpP;
  const double* cos_tab;
  float bf16_err;
  // queries
  int Q;
  const float* qx;
  const uint32_t* qcodes;
  const uint64_t* qsk;
  const int32_t* k;
  const double* recall;
  const int32_t* start;
  int k_max, filter, scoring;
  uint32_t* out_ids;
  float* out_sims;
  pf_query_stats* stats;
  int32_t* counter;
};

__device__ __forceinline__ bool better(float s1, uint32_t i1, float s2, uint32_t i2) {
  return s1 > s2 || (s1 == s2 && i1 < i2);
}

__device__ __forceinline__ double ipow(double x, int64_t e) {
  double r = 1.0, b = x;
  while (e > 0) {
    if (e & 1) r = __dmul_rn(r, b);
    b = __dmul_rn(b, b);
    e >>= 1;
  }
  return r;
}

// probability that a point at similarity s collides with the query on the
// first `depth` bits of one repetition (Sec. 4.3)
__device__ double collision_prob(const Dev& P, double s, int depth) {
  if (P.family == PF_SIMHASH) {
    const double sc = s > 1.0 ? 1.0 : (s < -1.0 ? -1.0 : s);
    const double p = 1.0 - acos(sc) / M_PI;
    return ipow(p, depth);
  }
  int t = 0;
  for (int u = 0; u < kAlphaSteps; ++u)
    if (double(5 * u - 100) / 100.0 <= s) t = u;
  const double* row = P.cpP + t * (P.ell + 1);
  return __dmul_rn(ipow(row[P.ell], depth / P.ell), row[depth % P.ell]);
}

__device__ __forceinline__ int filter_tau(const Dev& P, float s_k) {
  int tau = 0;
  const double s = double(s_k);
  for (int t = 0; t <= 64; ++t)
    if (P.cos_tab[t] >= s) tau = t;
  return tau;
}

__device__ __forceinline__ bool prefix_match(uint32_t a, uint32_t b, uint32_t mask) { return ((a ^ b) & mask) == 0; }

// first position in [lo, hi) of codes with code >= key
__device__ __forceinline__ int64_t lower_bound(const uint32_t* c, int64_t lo, int64_t hi, uint32_t key) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (c[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Canonical float32 similarity of the query (shared memory, d_pad floats) and
// row `id`, computed by the 8 lanes of a group (lane g8 owns partials
// 4*g8 .. 4*g8+3, i.e. float4 chunks g8, g8+8, ...).  Valid in all 8 lanes.
__device__ __forceinline__ float sim_canonical(const float* __restrict__ q, const float* __restrict__ row,
                                               int d_pad, int g8, unsigned gmask) {
  const float4* q4 = reinterpret_cast<const float4*>(q);
  const float4* r4 = reinterpret_cast<const float4*>(row);
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int ch = g8; ch * 4 < d_pad; ch += 8) {
    const float4 a = q4[ch];
    const float4 b = __ldg(r4 + ch);
    s.x = __fmaf_rn(a.x, b.x, s.x);
    s.y = __fmaf_rn(a.y, b.y, s.y);
    s.z = __fmaf_rn(a.z, b.z, s.z);
    s.w = __fmaf_rn(a.w, b.w, s.w);
  }
  // s[c] += s[c+16], s[c] += s[c+8], s[c] += s[c+4]: partner lanes 4, 2, 1 away
#pragma unroll
  for (int off = 4; off >= 1; off >>= 1) {
    s.x = __fadd_rn(s.x, __shfl_xor_sync(gmask, s.x, off, 8));
    s.y = __fadd_rn(s.y, __shfl_xor_sync(gmask, s.y, off, 8));
    s.z = __fadd_rn(s.z, __shfl_xor_sync(gmask, s.z, off, 8));
    s.w = __fadd_rn(s.w, __shfl_xor_sync(gmask, s.w, off, 8));
  }
  return __fadd_rn(__fadd_rn(s.x, s.z), __fadd_rn(s.y, s.w));
}

// bfloat16 estimate: float32 query against the bfloat16 row; any order.
__device__ __forceinline__ float sim_bf16(const float* __restrict__ q, const __nv_bfloat16* __restrict__ row,
                                          int d_pad, int g8, unsigned gmask) {
  const uint4* r8 = reinterpret_cast<const uint4*>(row);
  float acc = 0.f;
  for (int ch = g8; ch * 8 < d_pad; ch += 8) {
    const uint4 u = __ldg(r8 + ch);
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float lo = __uint_as_float(w[t] << 16);
      const float hi = __uint_as_float(w[t] & 0xffff0000u);
      acc = fmaf(q[ch * 8 + 2 * t], lo, acc);
      acc = fmaf(q[ch * 8 + 2 * t + 1], hi, acc);
    }
  }
#pragma unroll
  for (int off = 4; off >= 1; off >>= 1) acc += __shfl_xor_sync(gmask, acc, off, 8);
  return acc;
}

struct WarpState {
  float* q;        // [d_pad]
  uint32_t* l;     // [L]
  uint32_t* r;     // [L]
  float* pq_s;     // [k_max]
  uint32_t* pq_id; // [k_max]
  uint32_t* cbuf;  // [kCandBuf]
};

// Offer (s, id) to the sorted top-k of the warp (all lanes call with the same
// arguments).  Returns the new size.
__device__ int pq_offer(WarpState& w, int size, int k, float s, uint32_t id, int lane) {
  bool dup = false;
  int cnt = 0;
  for (int t = lane; t < size; t += 32) {
    dup |= w.pq_id[t] == id;
    cnt += better(w.pq_s[t], w.pq_id[t], s, id) ? 1 : 0;
  }
  if (__any_sync(kFull, dup)) return size;
  if (size == k && !better(s, id, w.pq_s[k - 1], w.pq_id[k - 1])) return size;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) cnt += __shfl_xor_sync(kFull, cnt, off);
  const int pos = cnt;
  const int nsize = size < k ? size + 1 : k;
  // shift [pos, nsize-1) one slot right
  float vs[kMaxK / 32];
  uint32_t vi[kMaxK / 32];
#pragma unroll
  for (int u = 0; u < kMaxK / 32; ++u) {
    const int t = lane + 32 * u;
    if (t > pos && t < nsize) {
      vs[u] = w.pq_s[t - 1];
      vi[u] = w.pq_id[t - 1];
    }
  }
  __syncwarp();
#pragma unroll
  for (int u = 0; u < kMaxK / 32; ++u) {
    const int t = lane + 32 * u;
    if (t > pos && t < nsize) {
      w.pq_s[t] = vs[u];
      w.pq_id[t] = vi[u];
    }
  }
  if (lane == 0) {
    w.pq_s[pos] = s;
    w.pq_id[pos] = id;
  }
  __syncwarp();
  return nsize;
}

struct Counters {
  int64_t retrieved = 0, passed = 0, scored = 0, reranked = 0;
};

// Score the buffered candidate ids and offer them to the top-k.
__device__ int flush_candidates(const Dev& P, WarpState& w, int cnt, int size, int k, int lane, Counters& ct) {
  const int g = lane >> 3, g8 = lane & 7;
  const unsigned gmask = 0xffu << (lane & ~7);  // the 8 lanes scoring one candidate
  for (int c0 = 0; c0 < cnt; c0 += 4) {
    const int c = c0 + g;
    const bool valid = c < cnt;
    const uint32_t id = valid ? w.cbuf[c] : 0u;
    float s;
    bool need = valid;
    if (P.scoring == 1) {
      const float est = sim_bf16(w.q, P.x16 + int64_t(id) * P.d_pad, P.d_pad, g8, gmask);
      // the running k-th similarity only rises, so a candidate whose
      // estimate plus the error bound is below it cannot enter the top-k
      if (size == k && est + P.bf16_err < w.pq_s[k - 1]) need = false;
      const unsigned rr = __ballot_sync(kFull, need && g8 == 0);
      if (lane == 0) ct.reranked += __popc(rr);
    }
    s = need ? sim_canonical(w.q, P.x32 + int64_t(id) * P.d_pad, P.d_pad, g8, gmask) : 0.f;
    const unsigned vb = __ballot_sync(kFull, valid && g8 == 0);
    if (lane == 0) ct.scored += __popc(vb);
    // offer in candidate order (the result is order independent)
#pragma unroll
    for (int gg = 0; gg < 4; ++gg) {
      const float ss = __shfl_sync(kFull, s, gg * 8);
      const uint32_t ii = __shfl_sync(kFull, id, gg * 8);
      const bool nn = __shfl_sync(kFull, need ? 1 : 0, gg * 8) != 0;
      if (nn) size = pq_offer(w, size, k, ss, ii, lane);
    }
  }
  return size;
}

__global__ void __launch_bounds__(kWarps * 32) search_kernel(Dev P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int d_pad = P.d_pad, L = P.L, kmax = P.k_max;
  // per-warp shared memory: q | l | r | pq_s | pq_id | cbuf
  const size_t per_warp = size_t(d_pad) * 4 + size_t(L) * 8 + size_t(kmax) * 8 + kCandBuf * 4;
  const size_t per_warp_al = (per_warp + 15) & ~size_t(15);
  unsigned char* base = smem_raw + per_warp_al * warp;
  WarpState w;
  w.q = reinterpret_cast<float*>(base);
  w.l = reinterpret_cast<uint32_t*>(base + size_t(d_pad) * 4);
  w.r = w.l + L;
  w.pq_s = reinterpret_cast<float*>(w.r + L);
  w.pq_id = reinterpret_cast<uint32_t*>(w.pq_s + kmax);
  w.cbuf = w.pq_id + kmax;
  const int64_t n = P.n;

  for (;;) {
    int qi = 0;
    if (lane == 0) qi = atomicAdd(P.counter, 1);
    qi = __shfl_sync(kFull, qi, 0);
    if (qi >= P.Q) break;

    const float* qg = P.qx + int64_t(qi) * d_pad;
    for (int i = lane; i < d_pad; i += 32) w.q[i] = qg[i];
    const uint32_t* qc = P.qcodes + int64_t(qi) * L;
    const uint64_t* qs = P.qsk + int64_t(qi) * P.M;
    const int k = P.k[qi];
    const double rec = P.recall[qi];
    if (k < 1 || k > kmax || !(rec > 0.0 && rec < 1.0)) {
      if (lane == 0) atomicOr(P.counter + 1, 1);
      for (int t = lane; t < kmax; t += 32) {
        P.out_ids[int64_t(qi) * kmax + t] = 0xffffffffu;
        P.out_sims[int64_t(qi) * kmax + t] = -INFINITY;
      }
      continue;
    }
    const double delta = 1.0 - rec;
    int i0 = P.Kb;
    if (P.start) {
      const int sd = P.start[qi];
      if (sd >= 0 && sd < P.Kb - 1) i0 = sd;
    }
    // initial empty range at the first code >= the query's code
    for (int j = lane; j < L; j += 32) {
      const uint32_t c = qc[j];
      const uint32_t* pj = P.pfx + int64_t(j) * kPrefixSize;
      const uint32_t t = c >> (32 - kPrefixBits);
      const int64_t lb = lower_bound(P.codes + int64_t(j) * n, pj[t], pj[t + 1], c);
      w.l[j] = uint32_t(lb);
      w.r[j] = uint32_t(lb);
    }
    __syncwarp();

    int size = 0, rounds = 0, depth = P.Kb, prev = -1, stop_depth = P.Kb;  // prev < 0: probe both sides
    Counters ct;
    for (;;) {
      const bool full = size == k;
      const float s_snap = full ? w.pq_s[k - 1] : -INFINITY;
      const int tau = full ? filter_tau(P, s_snap) : 64;
      if (depth == 0) {
        // prefix length 0: every point collides in every repetition, so the
        // round is a linear scan of all points (Lemma 1, i = 0), unfiltered.
        int nb = 0;
        for (int64_t b0 = 0; b0 < n; b0 += 32) {
          const int64_t id = b0 + lane;
          const unsigned m = __ballot_sync(kFull, id < n);
          if (id < n) w.cbuf[nb + __popc(m & ((1u << lane) - 1u))] = uint32_t(id);
          nb += __popc(m);
          if (lane == 0) { ct.retrieved += __popc(m); ct.passed += __popc(m); }
          __syncwarp();
          if (nb >= kCandBuf - 32) {
            size = flush_candidates(P, w, nb, size, k, lane, ct);
            nb = 0;
          }
        }
        if (nb) size = flush_candidates(P, w, nb, size, k, lane, ct);
        ++rounds;
        stop_depth = 0;
        break;
      }
      const uint32_t mask = 0xffffffffu << (32 - depth);
      const bool single = prev == depth + 1;
      // side that can grow when only bit `depth` (0-based from the top) is dropped
      int nb = 0;
      for (int jb = 0; jb < L; jb += 32) {
        const int j = jb + lane;
        uint32_t l = 0, r = 0, nl = 0, nr = 0;
        if (j < L) {
          const uint32_t qcj = qc[j];
          const uint32_t* cj = P.codes + int64_t(j) * n;
          l = w.l[j];
          r = w.r[j];
          nl = l;
          nr = r;
          const bool dropped_one = (qcj >> (31 - depth)) & 1u;
          const bool try_left = !single || dropped_one;
          const bool try_right = !single || !dropped_one;
          const uint32_t B = uint32_t(P.B);
          if (try_left && l > 0 && prefix_match(cj[l - 1], qcj, mask)) {
            // smallest m >= 1 with l - B*m <= 0 or codes[l - B*m - 1] outside the block
            uint32_t lo = 0, hi = 1;  // f(lo) false, search f(hi)
            for (;;) {
              const int64_t pos = int64_t(l) - int64_t(B) * hi;
              if (pos <= 0 || !prefix_match(cj[pos - 1], qcj, mask)) break;
              lo = hi;
              hi *= 2;
            }
            while (hi - lo > 1) {
              const uint32_t mid = (lo + hi) >> 1;
              const int64_t pos = int64_t(l) - int64_t(B) * mid;
              if (pos <= 0 || !prefix_match(cj[pos - 1], qcj, mask)) hi = mid; else lo = mid;
            }
            const int64_t pos = int64_t(l) - int64_t(B) * hi;
            nl = pos < 0 ? 0u : uint32_t(pos);
          }
          if (try_right && r < n && prefix_match(cj[r], qcj, mask)) {
            uint32_t lo = 0, hi = 1;
            for (;;) {
              const int64_t pos = int64_t(r) + int64_t(B) * hi;
              if (pos >= n || !prefix_match(cj[pos], qcj, mask)) break;
              lo = hi;
              hi *= 2;
            }
            while (hi - lo > 1) {
              const uint32_t mid = (lo + hi) >> 1;
              const int64_t pos = int64_t(r) + int64_t(B) * mid;
              if (pos >= n || !prefix_match(cj[pos], qcj, mask)) hi = mid; else lo = mid;
            }
            const int64_t pos = int64_t(r) + int64_t(B) * hi;
            nr = pos > n ? uint32_t(n) : uint32_t(pos);
          }
          w.l[j] = nl;
          w.r[j] = nr;
        }
        const uint32_t cl = l - nl;
        const uint32_t cnt = cl + (nr - r);
        // inclusive warp scan of cnt
        uint32_t inc = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const uint32_t v = __shfl_up_sync(kFull, inc, off);
          if (lane >= off) inc += v;
        }
        const uint32_t ex = inc - cnt;
        const uint32_t total = __shfl_sync(kFull, inc, 31);
        if (lane == 0) ct.retrieved += total;
        for (uint32_t e0 = 0; e0 < total; e0 += 32) {
          const uint32_t idx = e0 + lane;
          // owner lane: largest o with ex_o <= idx
          int o = 0;
#pragma unroll
          for (int step = 16; step >= 1; step >>= 1) {
            const uint32_t v = __shfl_sync(kFull, ex, o + step);
            if (v <= idx) o += step;
          }
          const uint32_t ex_o = __shfl_sync(kFull, ex, o);
          const uint32_t cl_o = __shfl_sync(kFull, cl, o);
          const uint32_t nl_o = __shfl_sync(kFull, nl, o);
          const uint32_t r_o = __shfl_sync(kFull, r, o);
          bool pass = false;
          uint32_t id = 0;
          if (idx < total) {
            const uint32_t off = idx - ex_o;
            const int jo = jb + o;
            const uint32_t pos = off < cl_o ? nl_o + off : r_o + (off - cl_o);
            id = __ldg(P.ids + int64_t(jo) * n + pos);
            pass = true;
            if (P.filter) {
              const int m = jo % P.M;
              const uint64_t h = __ldg(P.sk + int64_t(m) * n + id) ^ qs[m];
              pass = __popcll(h) <= tau;
            }
          }
          const unsigned pm = __ballot_sync(kFull, pass);
          if (pass) w.cbuf[nb + __popc(pm & ((1u << lane) - 1u))] = id;
          nb += __popc(pm);
          if (lane == 0) ct.passed += __popc(pm);
          __syncwarp();
          if (nb > kCandBuf - 32) {
            size = flush_candidates(P, w, nb, size, k, lane, ct);
            nb = 0;
          }
        }
      }
      if (nb) size = flush_candidates(P, w, nb, size, k, lane, ct);
      ++rounds;
      stop_depth = depth;
      int stop = 0;
      if (lane == 0 && size == k) {
        const double p = collision_prob(P, double(w.pq_s[k - 1]), depth);
        const double fail = ipow(__dsub_rn(1.0, p), L);
        stop = fail <= delta ? 1 : 0;
      }
      stop = __shfl_sync(kFull, stop, 0);
      if (stop) break;
      prev = depth;
      depth = (depth == P.Kb && i0 < P.Kb) ? i0 : depth - 1;
    }

    for (int t = lane; t < kmax; t += 32) {
      P.out_ids[int64_t(qi) * kmax + t] = t < size ? w.pq_id[t] : 0xffffffffu;
      P.out_sims[int64_t(qi) * kmax + t] = t < size ? w.pq_s[t] : -INFINITY;
    }
    if (P.stats && lane == 0) {
      pf_query_stats st;
      st.start_depth = i0;
      st.stop_depth = stop_depth;
      st.rounds = rounds;
      st.reserved = 0;
      st.retrieved = ct.retrieved;
      st.passed_filter = ct.passed;
      st.scored = ct.scored;
      st.reranked = P.scoring == 1 ? ct.reranked : 0;
      P.stats[qi] = st;
    }
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_search(const pf_index* ix, const SearchArgs& a, cudaStream_t s) {
  if (a.Q <= 0) return cudaSuccess;
  Dev P;
  P.n = ix->n;
  P.d = ix->d;
  P.d_pad = ix->lay.d_pad;
  P.L = ix->L;
  P.Kb = ix->lay.Kb;
  P.M = ix->M;
  P.B = ix->B;
  P.family = ix->family;
  P.ell = ix->lay.ell;
  P.x32 = ix->x32;
  P.x16 = ix->x16;
  P.codes = ix->codes;
  P.ids = ix->ids;
  P.pfx = ix->pfx;
  P.sk = ix->sk;
  P.cpP = ix->cpP;
  P.cos_tab = ix->cos_tab;
  P.bf16_err = ix->bf16_err;
  P.Q = a.Q;
  P.qx = a.qx;
  P.qcodes = a.qcodes;
  P.qsk = a.qsk;
  P.k = a.k;
  P.recall = a.recall;
  P.start = a.start;
  P.k_max = a.k_max;
  P.filter = a.filter;
  P.scoring = a.scoring;
  P.out_ids = a.out_ids;
  P.out_sims = a.out_sims;
  P.stats = a.stats;
  P.counter = a.counter;
  const size_t per_warp = size_t(P.d_pad) * 4 + size_t(P.L) * 8 + size_t(P.k_max) * 8 + kCandBuf * 4;
  const size_t smem = ((per_warp + 15) & ~size_t(15)) * kWarps;
  cudaError_t e = cudaFuncSetAttribute(search_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, search_kernel, kWarps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int blocks = ix->num_sms * per_sm;
  const int need = (a.Q + kWarps - 1) / kWarps;
  if (blocks > need) blocks = need;
  search_kernel<<<blocks, kWarps * 32, smem, s>>>(P);
  return cudaGetLastError();
}

}  // namespace pf
