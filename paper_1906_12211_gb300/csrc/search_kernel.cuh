// The adaptive k-NN query (Algorithm 1 as implemented in Sec. 4.1-4.2), one
// CTA of QW warps per query (four, or eight for batches too small to fill the
// GPU), persistent CTAs pulling queries from an atomic counter so queries of
// very different cost share one launch.
//
// Per round at prefix length i, for every repetition j the CTA extends the
// range [l, r) of positions around the query's code so that it covers the
// block of codes sharing the first i bits, growing each side in whole
// segments of B entries (Sec. 4.2, App. C).  The round's new positions form at
// most two runs per repetition; the runs are cut into chunks of up to 256
// positions (32 U) and the warps take the chunks in turn, one chunk per warp
// step (U lane-strided, coalesced loads of ids and of sketches per lane):
// position -> id and sketch -> Hamming filter (Sec. 4.2) -> the warp's
// compacted candidate buffer.
// Buffered candidates are scored (float32 canonical, or a bfloat16 estimate
// followed by an exact float32 rerank of those whose estimate plus its error
// bound can still reach the k-th similarity known so far) and offered to the
// warp's own top-k list (unique ids, ordered by similarity then id).  At every
// threshold snapshot the warp lists are merged into the query's top-k, which
// is the top-k of all candidates offered so far; after the round the stop test
// of Lemma 1 runs in float64.
//
// Readings shared with the oracle: the sketch threshold is taken from the
// top-k at the start of each round and, in a query's first round (which starts
// with an empty top-k), also at the start of every group of 32 repetitions (the
// paper refreshes it every k insertions, Sec. 4.2; all candidates of the
// previous group have been offered by then); the stop test runs once per round
// (Sec. 4.1); the canonical similarity is float32 with 32 partial sums
// (partial c takes the coordinates = c mod 32 in index order by fused
// multiply-add) combined as s[c] += s[c + w] for w = 16, 8, 4, 2, 1.  Only the
// filter depends on s_k and it uses the snapshot, so the result does not
// depend on which warp or lane visits a candidate, nor in which order.
//
// This header holds the kernel template and its device helpers; each
// kernels_search_*.cu instantiates one family of launch shapes and
// kernels_search.cu launches them.
#pragma once

#include <cuda_bf16.h>

#include <cuda_fp8.h>

#include "pf_internal.h"

namespace pf {
namespace skern {

constexpr unsigned kFull = 0xffffffffu;
// warps per query (one CTA): QW = 4 by default; 8 halves a query's latency
// for batches too small to fill the GPU with one CTA per query
// U = positions per lane per streaming step (a template parameter: 4 or 8,
// chosen by the tuner); a chunk is 32*U positions of one run
constexpr int kFlushAt = 256;   // a warp scores its buffer once it holds more than this
__host__ __device__ constexpr int cand_buf(int U) { return kFlushAt + 32 * U; }  // compacted ids per warp
constexpr int kGroup = 32;      // repetitions per threshold snapshot in a first round (after 1, 2, 4, 8, 16)

// first repetition of threshold-snapshot group g of a first round: 0, 1, 2,
// 4, 8, 16, then every kGroup
__device__ __forceinline__ int first_round_group_start(int g) {
  return g == 0 ? 0 : (g <= 5 ? 1 << (g - 1) : kGroup * (g - 5));
}
constexpr int kSub = 64;        // candidates per bfloat16 sub-batch (the pruning bound is refreshed between)

struct Dev {
  int n;
  int d, d_pad, L, Kb, M, B, family, ell;
  const float* x32;     // float32 rows, or null
  const __half* xf16;   // binary16 rows (read back exactly as float32), or null
  const __nv_bfloat16* x16;
  const uint8_t* x8;     // e4m3 rows (scoring 2), or null
  const float2* x8_meta;  // their (scale, error bound)
  const uint32_t* codes;
  const uint32_t* ids;
  const uint32_t* pfx;
  const uint64_t* sk;   // [M][n] per-point sketches, or null
  const uint64_t* skc;  // [L][n] per-repetition sketches, or null
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
  // diagnostics, or null: [0] range steps served by the prefix table (depth
  // <= 13), [1] sides settled within the first probed boundaries, [2] sides
  // that galloped past them, [3] rounds streamed in chunks of one run, [4]
  // rounds streamed flat
  unsigned long long* path_count;
  int stop_every;  // 0: stop test per round; G: also after every G repetitions (Alg. 1)
  int pool_fns;    // pooled index: functions in the pool (0: independent functions)
  int pool_rule;   // pooled index: 0 Cantelli's bound, 1 Lemma 1 as if independent
  int flat_fill;   // launch shape: stream a round flat when its chunks are < 1/flat_fill full (0: never)
};

__device__ __forceinline__ bool better(float s1, uint32_t i1, float s2, uint32_t i2) {
  return s1 > s2 || (s1 == s2 && i1 < i2);
}

__device__ __forceinline__ double ipow(double x, int e) {
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
// s_k: a k-th similarity (float32).  alpha_up[u]: the grid value (5u - 100)/100
// (a float64 division) rounded up to float32, so that alpha <= s_k exactly when
// alpha_up <= s_k; the grid point is the largest u with alpha <= s_k (or 0).
// The grid search runs in float32: the float64 pipe of sm_103 is narrow.
static __device__ __noinline__ double collision_prob(const Dev& P, const float* alpha_up, float s_k, int depth) {
  if (P.family == PF_SIMHASH) {
    const double s = double(s_k);
    const double sc = s > 1.0 ? 1.0 : (s < -1.0 ? -1.0 : s);
    const double p = 1.0 - acos(sc) / M_PI;
    return ipow(p, depth);
  }
  int t = 0;
  for (int u = 0; u < kAlphaSteps; ++u)
    if (alpha_up[u] <= s_k) t = u;
  const double* row = P.cpP + t * (P.ell + 1);
  return __dmul_rn(ipow(row[P.ell], depth / P.ell), row[depth % P.ell]);
}

// The largest t in [0, 64] with cos(t pi / 64) >= s_k (0 if none), from the
// table cosf[t] = the float64 cos(t pi / 64) rounded down to float32: for a
// float32 s_k, c >= s_k holds exactly when round_down(c) >= s_k, and the table
// does not increase, so a binary search for the first t with cosf[t] < s_k
// gives the same t as a scan of the float64 table (every thread computes it at
// every snapshot, and float64 compares are slow on sm_103).
__device__ __forceinline__ int filter_tau(const float* cosf, float s_k) {
  int lo = 0, hi = 65;  // first t with !(cosf[t] >= s_k) lies in [lo, hi]
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cosf[mid] >= s_k) lo = mid + 1; else hi = mid;
  }
  return lo > 0 ? lo - 1 : 0;
}

__device__ __forceinline__ bool prefix_match(uint32_t a, uint32_t b, uint32_t mask) { return ((a ^ b) & mask) == 0; }

// first position in [lo, hi) of codes with code >= key
__device__ __forceinline__ uint32_t lower_bound(const uint32_t* c, uint32_t lo, uint32_t hi, uint32_t key) {
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(c + mid) < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Offer (s, id) to the sorted top-k list (ps, pid) of `size` entries (all
// lanes of the warp call with the same arguments).  Returns the new size.
__device__ __forceinline__ int pq_offer(float* ps, uint32_t* pid, int size, int k, float s, uint32_t id, int lane) {
  if (size == k && !better(s, id, ps[k - 1], pid[k - 1])) return size;
  bool dup = false;
  int cnt = 0;
  for (int t = lane; t < size; t += 32) {
    const uint32_t it = pid[t];
    dup |= it == id;
    cnt += better(ps[t], it, s, id) ? 1 : 0;
  }
  if (__any_sync(kFull, dup)) return size;
  const int pos = __reduce_add_sync(kFull, cnt);
  const int nsize = size < k ? size + 1 : k;
  // shift [pos, nsize - 1) one slot right, the highest block of 32 slots
  // first (a block reads only slots of its own or of the next lower block)
  for (int base = ((nsize - 1) >> 5) << 5; base >= 0; base -= 32) {
    const int t = base + lane;
    const bool mv = t > pos && t < nsize;
    float vs = 0.f;
    uint32_t vi = 0u;
    if (mv) {
      vs = ps[t - 1];
      vi = pid[t - 1];
    }
    __syncwarp();
    if (mv) {
      ps[t] = vs;
      pid[t] = vi;
    }
    __syncwarp();
  }
  if (lane == 0) {
    ps[pos] = s;
    pid[pos] = id;
  }
  __syncwarp();
  return nsize;
}

// Canonical float32 similarities of the query with two rows, computed by the
// 8 lanes of a group (lane g8 owns partials 4*g8 .. 4*g8+3, i.e. float4
// chunks g8, g8+8, ...); the loads of up to 4 chunks of both rows are issued
// before their arithmetic.  Chunks wholly beyond the d coordinates (the zero
// padding up to d') are neither read nor added.
// four consecutive coordinates (chunk ch) of a float32 or a binary16 row
__device__ __forceinline__ float4 row_chunk(const float* __restrict__ r32, const __half* __restrict__ r16, int ch) {
  if (r32) return __ldg(reinterpret_cast<const float4*>(r32) + ch);
  const uint2 u = __ldg(reinterpret_cast<const uint2*>(r16) + ch);
  const float2 lo = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
  const float2 hi = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}

template <int NT>
__device__ __forceinline__ void sim_canonical2(const float* __restrict__ q, const float* __restrict__ ra,
                                               const float* __restrict__ rb, const __half* __restrict__ ha,
                                               const __half* __restrict__ hb, int d, int g8, unsigned gmask,
                                               float& out_a, float& out_b) {
  const float4* q4 = reinterpret_cast<const float4*>(q);
  constexpr int kBatch = NT < 4 ? NT : 4;  // chunks of both rows loaded before their arithmetic
  float4 sa = make_float4(0.f, 0.f, 0.f, 0.f), sb = sa;
#pragma unroll
  for (int t0 = 0; t0 < NT; t0 += kBatch) {
    float4 va[kBatch], vb[kBatch];
#pragma unroll
    for (int t = 0; t < kBatch; ++t) {
      const int ch = g8 + 8 * (t0 + t);
      va[t] = ch * 4 < d ? row_chunk(ra, ha, ch) : make_float4(0.f, 0.f, 0.f, 0.f);
      vb[t] = ch * 4 < d ? row_chunk(rb, hb, ch) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int t = 0; t < kBatch; ++t) {
      const int ch = g8 + 8 * (t0 + t);
      if (ch * 4 < d) {
        const float4 x = q4[ch];
        sa.x = __fmaf_rn(x.x, va[t].x, sa.x);
        sa.y = __fmaf_rn(x.y, va[t].y, sa.y);
        sa.z = __fmaf_rn(x.z, va[t].z, sa.z);
        sa.w = __fmaf_rn(x.w, va[t].w, sa.w);
        sb.x = __fmaf_rn(x.x, vb[t].x, sb.x);
        sb.y = __fmaf_rn(x.y, vb[t].y, sb.y);
        sb.z = __fmaf_rn(x.z, vb[t].z, sb.z);
        sb.w = __fmaf_rn(x.w, vb[t].w, sb.w);
      }
    }
  }
  // s[c] += s[c+16], s[c] += s[c+8], s[c] += s[c+4]: partner lanes 4, 2, 1 away
#pragma unroll
  for (int off = 4; off >= 1; off >>= 1) {
    sa.x = __fadd_rn(sa.x, __shfl_xor_sync(gmask, sa.x, off, 8));
    sa.y = __fadd_rn(sa.y, __shfl_xor_sync(gmask, sa.y, off, 8));
    sa.z = __fadd_rn(sa.z, __shfl_xor_sync(gmask, sa.z, off, 8));
    sa.w = __fadd_rn(sa.w, __shfl_xor_sync(gmask, sa.w, off, 8));
    sb.x = __fadd_rn(sb.x, __shfl_xor_sync(gmask, sb.x, off, 8));
    sb.y = __fadd_rn(sb.y, __shfl_xor_sync(gmask, sb.y, off, 8));
    sb.z = __fadd_rn(sb.z, __shfl_xor_sync(gmask, sb.z, off, 8));
    sb.w = __fadd_rn(sb.w, __shfl_xor_sync(gmask, sb.w, off, 8));
  }
  // s[c] += s[c+2], then s[0] += s[1]
  out_a = __fadd_rn(__fadd_rn(sa.x, sa.z), __fadd_rn(sa.y, sa.w));
  out_b = __fadd_rn(__fadd_rn(sb.x, sb.z), __fadd_rn(sb.y, sb.w));
}

// bfloat16 estimate of <q, x> by a pair of lanes: float32 query against the
// bfloat16 row, lane h of the pair takes the 8-element chunks h, h+2, ... below
// d (the rest is zero padding); any summation order (the error bound covers
// every order).
template <int NT2>
__device__ __forceinline__ float sim_bf16_pair(const float* __restrict__ q, const __nv_bfloat16* __restrict__ row,
                                               int d, int h) {
  const uint4* r8 = reinterpret_cast<const uint4*>(row);
  constexpr int kBatch = NT2 < 8 ? NT2 : 8;  // chunks loaded before their arithmetic
  float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
  for (int t0 = 0; t0 < NT2; t0 += kBatch) {
    uint4 v[kBatch];
#pragma unroll
    for (int t = 0; t < kBatch; ++t) {
      const int ch = h + 2 * (t0 + t);
      v[t] = ch * 8 < d ? __ldg(r8 + ch) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int t = 0; t < kBatch; ++t) {
      const int ch = h + 2 * (t0 + t);
      if (ch * 8 < d) {
        const float4 qa = reinterpret_cast<const float4*>(q)[2 * ch];
        const float4 qb = reinterpret_cast<const float4*>(q)[2 * ch + 1];
        acc0 = fmaf(qa.x, __uint_as_float(v[t].x << 16), acc0);
        acc1 = fmaf(qa.y, __uint_as_float(v[t].x & 0xffff0000u), acc1);
        acc0 = fmaf(qa.z, __uint_as_float(v[t].y << 16), acc0);
        acc1 = fmaf(qa.w, __uint_as_float(v[t].y & 0xffff0000u), acc1);
        acc0 = fmaf(qb.x, __uint_as_float(v[t].z << 16), acc0);
        acc1 = fmaf(qb.y, __uint_as_float(v[t].z & 0xffff0000u), acc1);
        acc0 = fmaf(qb.z, __uint_as_float(v[t].w << 16), acc0);
        acc1 = fmaf(qb.w, __uint_as_float(v[t].w & 0xffff0000u), acc1);
      }
    }
  }
  const float acc = acc0 + acc1;
  return acc + __shfl_xor_sync(kFull, acc, 1);
}

// 8-bit float (e4m3) estimate of <q, dec(row)> by a pair of lanes (scale not
// applied): lane h takes the 16-element chunks h, h+2, ... below d.
template <int NT2>
__device__ __forceinline__ float sim_fp8_pair(const float* __restrict__ q, const uint8_t* __restrict__ row, int d,
                                              int h) {
  constexpr int kChunks = (NT2 + 1) / 2;            // 16-byte chunks per lane
  constexpr int kBatch = kChunks < 2 ? kChunks : 2;  // chunks loaded before their arithmetic
  const uint4* r16 = reinterpret_cast<const uint4*>(row);
  float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
  for (int t0 = 0; t0 < kChunks; t0 += kBatch) {
    uint4 v[kBatch];
#pragma unroll
    for (int t = 0; t < kBatch; ++t) {
      const int ch = h + 2 * (t0 + t);
      v[t] = ch * 16 < d ? __ldg(r16 + ch) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int t = 0; t < kBatch; ++t) {
      const int ch = h + 2 * (t0 + t);
      if (ch * 16 < d) {
        const uint32_t w[4] = {v[t].x, v[t].y, v[t].z, v[t].w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float4 qv = reinterpret_cast<const float4*>(q)[4 * ch + u];
          const float2 lo = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(
              __nv_fp8x2_storage_t(w[u] & 0xffffu), __NV_E4M3)));
          const float2 hi = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(
              __nv_fp8x2_storage_t(w[u] >> 16), __NV_E4M3)));
          acc0 = fmaf(qv.x, lo.x, acc0);
          acc1 = fmaf(qv.y, lo.y, acc1);
          acc0 = fmaf(qv.z, hi.x, acc0);
          acc1 = fmaf(qv.w, hi.y, acc1);
        }
      }
    }
  }
  const float acc = acc0 + acc1;
  return acc + __shfl_xor_sync(kFull, acc, 1);
}

// Stop test of a pooled index (Sec. 3.2, App. B.2, read for general delta):
// j tables searched to prefix length `depth`, mu = j p_i, f = ceil(depth / l)
// pool functions behind those bits, c = f^2 / ((m - f) P) with P one whole
// function's collision probability; stop iff c < 1 and
// (mu + mu^2 c/(1-c)) / (mu^2 + mu + mu^2 c/(1-c)) <= delta (Cantelli).  Every
// operation is a correctly rounded float64 one, in the oracle's order.
__device__ __forceinline__ bool pool_stop(const Dev& P, const float* s_alpha, float s_k, int depth, int j,
                                          double delta) {
  const int f = (depth + P.ell - 1) / P.ell;
  const int m = P.pool_fns;
  if (f <= 0 || f >= m || j <= 0) return false;
  const double p = collision_prob(P, s_alpha, s_k, depth);
  const double p1 = collision_prob(P, s_alpha, s_k, P.ell);
  if (!(p1 > 0.0)) return false;
  const double c = __ddiv_rn(double(f) * double(f), __dmul_rn(double(m - f), p1));
  if (!(c < 1.0)) return false;
  const double mu = __dmul_rn(double(j), p);
  if (!(mu > 0.0)) return false;
  const double var = __dadd_rn(mu, __dmul_rn(__dmul_rn(mu, mu), __ddiv_rn(c, __dsub_rn(1.0, c))));
  return __ddiv_rn(var, __dadd_rn(__dmul_rn(mu, mu), var)) <= delta;
}

struct Counters {
  uint32_t retrieved = 0, passed = 0, scored = 0, reranked = 0;
};

// Exact float32 similarities of the `cnt` ids at the front of cbuf, each
// offered to the list (ps, pid) (8 candidates per step: 4 groups of 8 lanes,
// 2 rows each).
template <int NT>
__device__ __forceinline__ int canonical_and_offer(const Dev& P, const float* q, const uint32_t* cbuf, int cnt,
                                                   float* ps, uint32_t* pid, int size, int k, int lane) {
  const int g = lane >> 3, g8 = lane & 7;
  const unsigned gmask = 0xffu << (lane & ~7);
  for (int c0 = 0; c0 < cnt; c0 += 8) {
    const int ca = c0 + g, cb = c0 + 4 + g;
    const uint32_t ida = ca < cnt ? cbuf[ca] : cbuf[c0];
    const uint32_t idb = cb < cnt ? cbuf[cb] : cbuf[c0];
    float sa, sb;
    const size_t oa = size_t(ida) * P.d_pad, ob = size_t(idb) * P.d_pad;
    if (P.x32)
      sim_canonical2<NT>(q, P.x32 + oa, P.x32 + ob, nullptr, nullptr, P.d, g8, gmask, sa, sb);
    else
      sim_canonical2<NT>(q, nullptr, nullptr, P.xf16 + oa, P.xf16 + ob, P.d, g8, gmask, sa, sb);
    const int m = min(8, cnt - c0);
    for (int t = 0; t < m; ++t) {
      const int src = (t & 3) * 8;
      const float s = __shfl_sync(kFull, t < 4 ? sa : sb, src);
      const uint32_t id = __shfl_sync(kFull, t < 4 ? ida : idb, src);
      size = pq_offer(ps, pid, size, k, s, id, lane);
    }
  }
  return size;
}

// Score the cnt buffered candidate ids of a warp and offer them to its list.
// kth_known: a k-th similarity already reached by the query (or -inf).
template <int NT, int NT2>
__device__ __forceinline__ int flush_candidates(const Dev& P, const float* q, uint32_t* cbuf, int cnt, float* ps,
                                                uint32_t* pid, int size, int k, float kth_known, int lane,
                                                Counters& ct) {
  if (lane == 0) ct.scored += cnt;
  if (P.scoring == 0) return canonical_and_offer<NT>(P, q, cbuf, cnt, ps, pid, size, k, lane);
  // bfloat16 (or e4m3) estimates, 16 rows per step (a pair of lanes each).  A candidate
  // can enter the final top-k only if its exact similarity reaches every k-th
  // similarity the query has already reached (that of the merged top-k at the
  // last snapshot, or of this warp's list: each is a k-th of a subset of the
  // candidates); the estimate is within its bound of the exact value (bf16_err,
  // or the row's own bound for e4m3), so candidates whose estimate + bound is
  // below it are dropped and the
  // others are compacted in place at the front of cbuf.  Each warp takes a
  // fixed share of the chunks, so the work done (and its count) does not
  // depend on timing.
  // The buffer is taken in sub-batches of kSub so that the bound rises as soon
  // as the reranked candidates of one sub-batch are in the list.
  const int g = lane >> 1, h = lane & 1;
  for (int b0 = 0; b0 < cnt; b0 += kSub) {
    const int b1 = min(cnt, b0 + kSub);
    const float kth = fmaxf(kth_known, size == k ? ps[k - 1] : -INFINITY);
    int nr = 0;
    for (int c0 = b0; c0 < b1; c0 += 16) {
      const int c = c0 + g;
      const bool valid = c < b1;
      const uint32_t id = valid ? cbuf[c] : cbuf[c0];
      bool need;
      if (P.scoring == 2) {  // e4m3 estimate: per-row scale and error bound
        const float2 m = __ldg(P.x8_meta + id);
        const float est = sim_fp8_pair<NT2>(q, P.x8 + size_t(id) * P.d_pad, P.d, h) * m.x;
        need = valid && est + m.y >= kth;
      } else {
        const float est = sim_bf16_pair<NT2>(q, P.x16 + size_t(id) * P.d_pad, P.d, h);
        need = valid && est + P.bf16_err >= kth;
      }
      const unsigned b = __ballot_sync(kFull, need && h == 0);
      __syncwarp();
      if (need && h == 0) cbuf[b0 + nr + __popc(b & ((1u << lane) - 1u))] = id;
      nr += __popc(b);
      __syncwarp();
    }
    if (lane == 0) ct.reranked += nr;
    size = canonical_and_offer<NT>(P, q, cbuf + b0, nr, ps, pid, size, k, lane);
  }
  return size;
}

// A flat round's streaming (see the launch shape's flat_fill): warp `warp`
// takes the spans of kSpan consecutive positions warp, warp + QW, ... of the
// group's runs laid end to end (repetition by repetition, left run before right
// run); a lane finds the repetition of its first position by binary search over
// ppre (the position prefix), then walks on.  Only the kernel instantiations
// with FLAT = true contain it, so that the chunked loop, the common case, is
// compiled as if this did not exist.
template <int NT, int NT2, int U, int QW>
__device__ __forceinline__ void flat_stream(const Dev& P, const float* q, const uint64_t* qsk, const uint4* runs,
                                         const uint32_t* ppre, uint32_t* cbuf, float* my_s, uint32_t* my_id, int j0,
                                         int j1, int tau, float gkth, int k, int lane, int warp, int& nb_io,
                                         int& wsize_io, Counters& ct) {
  constexpr int kUnroll = U;
  constexpr uint32_t kSpan = 32u * U;
  constexpr int kQW = QW;
  const uint32_t n = uint32_t(P.n);
  const int M = P.M;
  const uint32_t lt_mask = (1u << lane) - 1u;
  int nb = nb_io, wsize = wsize_io;
  const uint32_t p_end = ppre[j1];
  for (uint32_t b = ppre[j0] + uint32_t(warp) * kSpan; b < p_end; b += kQW * kSpan) {
    int jl = j0, jh = j1;  // ppre[jl] <= b + lane < ppre[jh]
    const uint32_t p0 = min(b + uint32_t(lane), p_end - 1u);
    while (jh - jl > 1) {
      const int mid = (jl + jh) >> 1;
      if (ppre[mid] <= p0) jl = mid; else jh = mid;
    }
    int jr = jl;
    uint32_t id[kUnroll];
    bool pass[kUnroll];
    size_t at[kUnroll];
    int jof[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint32_t pos = b + 32u * u + uint32_t(lane);
      const bool valid = pos < p_end;
      if (valid)
        while (ppre[jr + 1] <= pos) ++jr;
      const uint4 ru = runs[jr];
      const uint32_t o = pos - ppre[jr];
      const uint32_t ap = o < ru.y ? ru.x + o : ru.z + (o - ru.y);
      at[u] = size_t(jr) * n + ap;
      jof[u] = jr;
      id[u] = valid ? __ldcs(P.ids + at[u]) : 0u;
      pass[u] = valid;
    }
    if (P.filter) {
      uint64_t hd[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const uint64_t sk = !pass[u] ? 0ull
                            : P.skc ? __ldcs(P.skc + at[u])
                                    : __ldg(P.sk + size_t(jof[u] % M) * n + id[u]);
        hd[u] = sk ^ qsk[jof[u] % M];
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) pass[u] = pass[u] && __popcll(hd[u]) <= tau;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const unsigned pm = __ballot_sync(kFull, pass[u]);
      if (pass[u]) cbuf[nb + __popc(pm & lt_mask)] = id[u];
      nb += __popc(pm);
    }
    if (lane == 0) ct.retrieved += min(kSpan, p_end - b);
    __syncwarp();
    if (nb > kFlushAt) {
      if (lane == 0) ct.passed += uint32_t(nb);  // every buffered candidate passed the filter
      wsize = flush_candidates<NT, NT2>(P, q, cbuf, nb, my_s, my_id, wsize, k, gkth, lane, ct);
      nb = 0;
    }
  }
  nb_io = nb;
  wsize_io = wsize;
}

// NT = d_pad / 32 rounded up: float4 chunks of a float32 row per lane of an
// 8-lane group; NT2 = d_pad / 16 rounded up: 16-byte chunks of a bfloat16 row
// per lane of a pair
// FLAT: the instantiation that can stream a round flat (the launch shape's
// flat_fill > 0); the others never do and carry none of its code
template <int NT, int NT2, int U, int QW, bool FLAT>
__global__ void __launch_bounds__(32 * QW, 32 / QW) search_kernel(Dev P) {
  constexpr int kQW = QW;
  constexpr int kThreads = 32 * QW;
  constexpr int kUnroll = U;
  constexpr uint32_t kSpan = 32u * U;
  constexpr int kCandBuf = cand_buf(U);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int d_pad = P.d_pad, L = P.L, kmax = P.k_max, M = P.M;
  // shared memory: q | runs | range | qsk | cpre | gs | gid | ws | wid | cbuf
  // (q is read as float4 and runs as uint4: both 16-byte aligned, d_pad is a
  // multiple of 16)
  float* q = reinterpret_cast<float*>(smem_raw);
  uint4* runs = reinterpret_cast<uint4*>(q + d_pad);  // [L] this round's (left start, left count, right start, right count)
  uint2* range = reinterpret_cast<uint2*>(runs + L);  // [L] current [l, r)
  uint64_t* qsk = reinterpret_cast<uint64_t*>(range + L);
  uint32_t* cpre = reinterpret_cast<uint32_t*>(qsk + M);  // [L + 1] chunk prefix
  uint32_t* ppre = cpre + L + 1;                           // [L + 1] position prefix
  float* gs = reinterpret_cast<float*>(ppre + L + 1);
  uint32_t* gid = reinterpret_cast<uint32_t*>(gs + kmax);
  float* ws = reinterpret_cast<float*>(gid + kmax);              // [kQW][kmax]
  uint32_t* wid = reinterpret_cast<uint32_t*>(ws + kQW * kmax);  // [kQW][kmax]
  uint32_t* cbuf = wid + kQW * kmax + warp * kCandBuf;           // this warp's buffer
  float* my_s = ws + warp * kmax;
  uint32_t* my_id = wid + warp * kmax;
  __shared__ int s_qi, s_size, s_stop, s_wsize[kQW];
  __shared__ uint32_t s_scan[kQW], s_pscan[kQW];
  __shared__ float s_cosf[65];
  __shared__ float s_alpha[kAlphaSteps];
  __shared__ uint32_t s_ct[kQW][4];
  const uint32_t n = uint32_t(P.n);
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int per = (L + kThreads - 1) / kThreads;  // repetitions per thread in the range pass
  for (int t = tid; t < 65; t += kThreads) s_cosf[t] = __double2float_rd(P.cos_tab[t]);
  for (int u = tid; u < kAlphaSteps; u += kThreads) s_alpha[u] = __double2float_ru(double(5 * u - 100) / 100.0);
  __syncthreads();

  for (;;) {
    if (tid == 0) s_qi = atomicAdd(P.counter, 1);
    __syncthreads();
    const int qi = s_qi;
    if (qi >= P.Q) break;

    const int k = P.k[qi];
    const double rec = P.recall[qi];
    if (k < 1 || k > kmax || !(rec > 0.0 && rec < 1.0)) {
      if (tid == 0) atomicOr(P.counter + 1, 1);
      for (int t = tid; t < kmax; t += kThreads) {
        P.out_ids[size_t(qi) * kmax + t] = 0xffffffffu;
        P.out_sims[size_t(qi) * kmax + t] = -INFINITY;
      }
      __syncthreads();  // s_qi is rewritten by the next fetch
      continue;
    }
    const double delta = 1.0 - rec;
    const float* qg = P.qx + size_t(qi) * d_pad;
    for (int i = tid; i < d_pad; i += kThreads) q[i] = qg[i];
    for (int m = tid; m < M; m += kThreads) qsk[m] = P.qsk[size_t(qi) * M + m];
    const uint32_t* qc = P.qcodes + size_t(qi) * L;
    // start depth: the plain schedule starts at K (Sec. 4.1); a given start i0
    // in [0, K) takes the whole block at i0 in the first round
    int i0 = P.Kb;
    if (P.start) {
      const int sd = P.start[qi];
      if (sd >= 0 && sd < P.Kb) i0 = sd;
    }
    // initial empty range at the first code >= the query's code
    for (int j = tid; j < L; j += kThreads) {
      const uint32_t c = qc[j];
      const uint32_t* pj = P.pfx + size_t(j) * kPrefixSize;
      const uint32_t t = c >> (32 - kPrefixBits);
      const uint32_t lb = lower_bound(P.codes + size_t(j) * n, __ldg(pj + t), __ldg(pj + t + 1), c);
      range[j] = make_uint2(lb, lb);
    }
    if (tid == 0) s_size = 0;
    if (lane == 0) s_wsize[warp] = 0;
    __syncthreads();

    int rounds = 0, depth = i0, prev = -1, stop_depth = i0;  // prev < 0: probe both sides
    int full_depth = -1;  // first depth after whose round k points were held
    int last_reps = L;    // repetitions searched in the last round
    Counters ct;
    int wsize = 0;  // entries of this warp's list
    for (;;) {
      if (depth == 0) {
        // prefix length 0: every point collides in every repetition, so the
        // round is a linear scan of all points (Lemma 1, i = 0), unfiltered.
        const float kth0 = s_size == k ? gs[k - 1] : -INFINITY;
        int nb = 0;
        for (uint32_t b0 = uint32_t(warp) * 32u; b0 < n; b0 += kThreads) {
          const uint32_t id = b0 + lane;
          const unsigned m = __ballot_sync(kFull, id < n);
          if (id < n) cbuf[nb + __popc(m & lt_mask)] = id;
          nb += __popc(m);
          if (lane == 0) {
            ct.retrieved += __popc(m);
            ct.passed += __popc(m);
          }
          __syncwarp();
          if (nb > kFlushAt) {
            wsize = flush_candidates<NT, NT2>(P, q, cbuf, nb, my_s, my_id, wsize, k, kth0, lane, ct);
            nb = 0;
          }
        }
        if (nb) wsize = flush_candidates<NT, NT2>(P, q, cbuf, nb, my_s, my_id, wsize, k, kth0, lane, ct);
        if (lane == 0) s_wsize[warp] = wsize;
        __syncthreads();
        if (warp == 0) {
          int size = s_size;
          for (int w = 0; w < kQW; ++w)
            for (int t = 0; t < s_wsize[w]; ++t) size = pq_offer(gs, gid, size, k, ws[w * kmax + t], wid[w * kmax + t], lane);
          if (lane == 0) s_size = size;
        }
        __syncthreads();
        ++rounds;
        stop_depth = 0;
        if (s_size == k && full_depth < 0) full_depth = 0;
        break;
      }
      // ---- range pass: thread t extends repetitions [t*per, (t+1)*per)
      const uint32_t mask = 0xffffffffu << (32 - depth);
      const bool single = prev == depth + 1;
      uint32_t my_chunks = 0, my_pos = 0;
      const int jlo = min(L, tid * per), jhi = min(L, jlo + per);
      for (int j = jlo; j < jhi; ++j) {
        const uint32_t qcj = qc[j];
        const uint32_t* cj = P.codes + size_t(j) * n;
        const uint2 lr = range[j];
        const uint32_t l = lr.x, r = lr.y;
        uint32_t nl = l, nr = r;
        // in a one-bit step only the side of the dropped bit can grow
        // (bit `depth`, counted from the top, of the query's code)
        const bool dropped_one = (qcj >> (31 - depth)) & 1u;
        const bool try_left = !single || dropped_one;
        const bool try_right = !single || !dropped_one;
        const uint32_t B = uint32_t(P.B);
        if (depth <= kPrefixBits) {
          // the block [blo, bhi) of codes sharing the first `depth` bits is a
          // run of 13-bit prefix buckets: two table reads.  A side grows by the
          // smallest whole number of segments that reaches the block's end
          // (or the array's end): the same positions as probing segment by
          // segment until the entry beyond the range is outside the block.
          const uint32_t* pj = P.pfx + size_t(j) * kPrefixSize;
          const uint32_t span = 1u << (kPrefixBits - depth);
          const uint32_t t0 = (qcj >> (32 - kPrefixBits)) & ~(span - 1u);
          const uint32_t blo = __ldg(pj + t0), bhi = __ldg(pj + t0 + span);
          if (P.path_count) atomicAdd(P.path_count + 0, 1ull);  // diagnostics only
          if (try_left && l > blo) {
            const uint32_t m = (l - blo + B - 1) / B;
            nl = l >= B * m ? l - B * m : 0u;
          }
          if (try_right && r < bhi) {
            const uint32_t m = (bhi - r + B - 1) / B;
            nr = min(n, r + B * m);
          }
        } else {
          // above 13 bits: a side grows by m* segments, m* the smallest m >= 1
          // whose position is outside the array or whose code is outside the
          // block.  The entry next to the range and the first kProbe segment
          // boundaries of both sides are read together (one round trip in the
          // common case); past them the search gallops on.  A position outside
          // the array reads as a code outside the block (~qcj).
          constexpr int kProbe = 4;
          const bool lv = try_left && l > 0, rv = try_right && r < n;
          uint32_t cl[kProbe + 1], cr[kProbe + 1];
#pragma unroll
          for (int m = 0; m <= kProbe; ++m) {
            const int64_t pl = int64_t(l) - int64_t(B) * m - 1, pr = int64_t(r) + int64_t(B) * m;
            cl[m] = lv && pl >= 0 ? __ldg(cj + pl) : ~qcj;
            cr[m] = rv && pr < int64_t(n) ? __ldg(cj + pr) : ~qcj;
          }
          if (lv && prefix_match(cl[0], qcj, mask)) {
            uint32_t lo = 0, hi = 0;
#pragma unroll
            for (int m = kProbe; m >= 1; --m)
              if (!prefix_match(cl[m], qcj, mask)) hi = m;
            if (hi == 0) {  // the first kProbe boundaries are all inside the block
              if (P.path_count) atomicAdd(P.path_count + 2, 1ull);
              lo = kProbe;
              hi = 2 * kProbe;
              for (;;) {
                const int64_t pos = int64_t(l) - int64_t(B) * hi;
                if (pos <= 0 || !prefix_match(__ldg(cj + pos - 1), qcj, mask)) break;
                lo = hi;
                hi *= 2;
              }
              while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                const int64_t pos = int64_t(l) - int64_t(B) * mid;
                if (pos <= 0 || !prefix_match(__ldg(cj + pos - 1), qcj, mask)) hi = mid; else lo = mid;
              }
            }
            const int64_t pos = int64_t(l) - int64_t(B) * hi;
            nl = pos < 0 ? 0u : uint32_t(pos);
            if (P.path_count && hi <= kProbe) atomicAdd(P.path_count + 1, 1ull);
          }
          if (rv && prefix_match(cr[0], qcj, mask)) {
            uint32_t lo = 0, hi = 0;
#pragma unroll
            for (int m = kProbe; m >= 1; --m)
              if (!prefix_match(cr[m], qcj, mask)) hi = m;
            if (hi == 0) {
              if (P.path_count) atomicAdd(P.path_count + 2, 1ull);
              lo = kProbe;
              hi = 2 * kProbe;
              for (;;) {
                const int64_t pos = int64_t(r) + int64_t(B) * hi;
                if (pos >= int64_t(n) || !prefix_match(__ldg(cj + pos), qcj, mask)) break;
                lo = hi;
                hi *= 2;
              }
              while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                const int64_t pos = int64_t(r) + int64_t(B) * mid;
                if (pos >= int64_t(n) || !prefix_match(__ldg(cj + pos), qcj, mask)) hi = mid; else lo = mid;
              }
            }
            const int64_t pos = int64_t(r) + int64_t(B) * hi;
            nr = pos > int64_t(n) ? n : uint32_t(pos);
            if (P.path_count && hi <= kProbe) atomicAdd(P.path_count + 1, 1ull);
          }
        }
        range[j] = make_uint2(nl, nr);
        runs[j] = make_uint4(nl, l - nl, r, nr - r);
        my_chunks += (l - nl + kSpan - 1) / kSpan + (nr - r + kSpan - 1) / kSpan;
        my_pos += (l - nl) + (nr - r);
      }
      // exclusive scans over the repetitions of the chunk counts -> cpre and
      // of the new positions -> ppre
      uint32_t inc = my_chunks, pinc = FLAT ? my_pos : 0u;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, inc, off);
        if (lane >= off) inc += v;
        if constexpr (FLAT) {
          const uint32_t pv = __shfl_up_sync(kFull, pinc, off);
          if (lane >= off) pinc += pv;
        }
      }
      if (lane == 31) {
        s_scan[warp] = inc;
        if constexpr (FLAT) s_pscan[warp] = pinc;
      }
      __syncthreads();
      uint32_t run = inc - my_chunks, prun = pinc - my_pos;
      for (int w = 0; w < warp; ++w) {
        run += s_scan[w];
        if constexpr (FLAT) prun += s_pscan[w];
      }
      for (int j = jlo; j < jhi; ++j) {
        cpre[j] = run;
        const uint4 ru = runs[j];
        run += (ru.y + kSpan - 1) / kSpan + (ru.w + kSpan - 1) / kSpan;
        if constexpr (FLAT) {
          ppre[j] = prun;
          prun += ru.y + ru.w;
        }
      }
      if (tid == kThreads - 1) {
        cpre[L] = run;
        if constexpr (FLAT) ppre[L] = prun;
      }
      __syncthreads();
      // short runs leave most of a chunk's lanes idle: the round then streams
      // its positions as one flat sequence instead (the same candidates)
      const bool flat = FLAT && P.flat_fill > 0 && uint64_t(cpre[L]) * kSpan > uint64_t(P.flat_fill) * ppre[L];
      if (P.path_count && tid == 0) atomicAdd(P.path_count + (flat ? 4 : 3), 1ull);  // diagnostics only

      // ---- stream the chunks, group by group
      // groups of repetitions: in a first round (threshold snapshots), and in
      // every round when the stop test also runs after groups of G repetitions
      const bool every = P.stop_every > 0;
      const bool grouped = rounds == 0 || every;
      const int G = P.stop_every;
      bool stopped_mid = false;
      for (int grp = 0;; ++grp) {
        const int j0 = !grouped ? (grp == 0 ? 0 : L) : every ? grp * G : first_round_group_start(grp);
        if (j0 >= L) break;
        const int j1 = !grouped ? L : min(L, every ? j0 + G : first_round_group_start(grp + 1));
        // threshold snapshot: every earlier candidate is in the merged top-k
        const int gsize = s_size;
        const float gkth = gsize == k ? gs[k - 1] : -INFINITY;
        const int tau = gsize == k ? filter_tau(s_cosf, gkth) : 64;
        const uint32_t c_end = flat ? cpre[j0] : cpre[j1];  // the chunk loop is skipped in a flat round
        int jc = j0;
        uint64_t qh = qsk[j0 % M];  // the query's sketch for repetition jc
        int nb = 0;
        if constexpr (FLAT) {
          if (flat)
            flat_stream<NT, NT2, U, QW>(P, q, qsk, runs, ppre, cbuf, my_s, my_id, j0, j1, tau, gkth, k, lane, warp,
                                        nb, wsize, ct);
        }
        // warp w takes chunks w, w + 4, ...: up to kSpan positions of one run,
        // lane-strided so that every load instruction is coalesced.  Ids and
        // sketches are read once per round: their loads are marked evict-first,
        // so that L2 keeps the rows that the scoring gathers instead
        for (uint32_t c = cpre[j0] + uint32_t(warp); c < c_end; c += kQW) {
          if (cpre[jc + 1] <= c) {  // chunk -> repetition (c only grows)
            do ++jc; while (cpre[jc + 1] <= c);
            qh = qsk[jc % M];
          }
          const uint32_t lk = c - cpre[jc];
          const uint4 ru = runs[jc];
          const uint32_t nlc = (ru.y + kSpan - 1) / kSpan;
          const bool left = lk < nlc;
          const uint32_t off = (left ? lk : lk - nlc) * kSpan;
          const uint32_t start = (left ? ru.x : ru.z) + off;
          const uint32_t cnt = min((left ? ru.y : ru.w) - off, kSpan);
          const size_t rowbase = size_t(jc) * n + start;
          uint32_t id[kUnroll];
          bool pass[kUnroll];
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            const uint32_t o = 32u * u + uint32_t(lane);
            id[u] = o < cnt ? __ldcs(P.ids + rowbase + o) : 0u;
          }
          if (P.filter) {
            uint64_t hd[kUnroll];
            if (P.skc) {  // the sketch sits at the same position as the id
#pragma unroll
              for (int u = 0; u < kUnroll; ++u) {
                const uint32_t o = 32u * u + uint32_t(lane);
                hd[u] = o < cnt ? __ldcs(P.skc + rowbase + o) ^ qh : 0ull;
              }
            } else {
              const uint64_t* skm = P.sk + size_t(jc % M) * n;
#pragma unroll
              for (int u = 0; u < kUnroll; ++u) {
                const uint32_t o = 32u * u + uint32_t(lane);
                hd[u] = o < cnt ? __ldg(skm + id[u]) ^ qh : 0ull;
              }
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) pass[u] = 32u * u + uint32_t(lane) < cnt && __popcll(hd[u]) <= tau;
          } else {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) pass[u] = 32u * u + uint32_t(lane) < cnt;
          }
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            const unsigned pm = __ballot_sync(kFull, pass[u]);
            if (pass[u]) cbuf[nb + __popc(pm & lt_mask)] = id[u];
            nb += __popc(pm);
          }
          if (lane == 0) ct.retrieved += cnt;
          __syncwarp();
          if (nb > kFlushAt) {
            if (lane == 0) ct.passed += uint32_t(nb);  // every buffered candidate passed the filter
            wsize = flush_candidates<NT, NT2>(P, q, cbuf, nb, my_s, my_id, wsize, k, gkth, lane, ct);
            nb = 0;
          }
        }
        if (lane == 0) ct.passed += uint32_t(nb);
        if (nb) wsize = flush_candidates<NT, NT2>(P, q, cbuf, nb, my_s, my_id, wsize, k, gkth, lane, ct);
        // merge the warp lists into the query's top-k
        if (lane == 0) s_wsize[warp] = wsize;
        __syncthreads();
        if (warp == 0) {
          int size = s_size;
          for (int w = 0; w < kQW; ++w)
            for (int t = 0; t < s_wsize[w]; ++t) size = pq_offer(gs, gid, size, k, ws[w * kmax + t], wid[w * kmax + t], lane);
          if (lane == 0) s_size = size;
        }
        wsize = 0;
        __syncthreads();
        if (P.stop_every > 0 && j1 < L) {
          // Alg. 1: the stop test after repetitions 0..j1-1 searched to this
          // prefix length and the others to depth + 1 (to nothing yet in a
          // first round); after the last group it is the round's test below
          if (tid == 0) {
            int stop = 0;
            if (s_size == k) {
              const float skf = gs[k - 1];
              if (P.pool_fns > 0 && P.pool_rule == 0) {  // only the j1 tables at this depth count
                stop = pool_stop(P, s_alpha, skf, depth, j1, delta) ? 1 : 0;
              } else {
                double fail = ipow(__dsub_rn(1.0, collision_prob(P, s_alpha, skf, depth)), j1);
                if (rounds > 0)
                  fail = __dmul_rn(fail, ipow(__dsub_rn(1.0, collision_prob(P, s_alpha, skf, depth + 1)), L - j1));
                stop = fail <= delta ? 1 : 0;
              }
            }
            s_stop = stop;
          }
          __syncthreads();
          if (s_stop) {
            stopped_mid = true;
            last_reps = j1;
            break;
          }
        }
      }
      ++rounds;
      stop_depth = depth;
      const int size = s_size;
      if (size == k && full_depth < 0) full_depth = depth;
      if (stopped_mid) break;
      if (tid == 0) {
        int stop = 0;
        if (size == k) {
          if (P.pool_fns > 0 && P.pool_rule == 0) {
            stop = pool_stop(P, s_alpha, gs[k - 1], depth, L, delta) ? 1 : 0;
          } else {
            const double p = collision_prob(P, s_alpha, gs[k - 1], depth);
            const double fail = ipow(__dsub_rn(1.0, p), L);
            stop = fail <= delta ? 1 : 0;
          }
        }
        s_stop = stop;
      }
      __syncthreads();
      const int stop = s_stop;
      if (stop) break;
      prev = depth;
      depth -= 1;
    }

    const int size = s_size;
    for (int t = tid; t < kmax; t += kThreads) {
      P.out_ids[size_t(qi) * kmax + t] = t < size ? gid[t] : 0xffffffffu;
      P.out_sims[size_t(qi) * kmax + t] = t < size ? gs[t] : -INFINITY;
    }
    if (lane == 0) {
      s_ct[warp][0] = ct.retrieved;
      s_ct[warp][1] = ct.passed;
      s_ct[warp][2] = ct.scored;
      s_ct[warp][3] = ct.reranked;
    }
    __syncthreads();
    if (P.stats && tid == 0) {
      pf_query_stats st;
      st.start_depth = i0;
      st.stop_depth = stop_depth;
      st.rounds = rounds;
      st.full_depth = full_depth;
      int64_t sum[4] = {0, 0, 0, 0};
      for (int w = 0; w < kQW; ++w)
        for (int c = 0; c < 4; ++c) sum[c] += s_ct[w][c];
      st.retrieved = sum[0];
      st.passed_filter = sum[1];
      st.scored = sum[2];
      st.reranked = P.scoring != 0 ? sum[3] : 0;
      st.last_reps = last_reps;
      st.reserved = 0;
      P.stats[qi] = st;
    }
  }
}


using Kernel = void (*)(Dev);

// the instantiation for d_pad (NT = d_pad / 32 rounded up to a power of two)
template <int U, int QW, bool FLAT>
Kernel pick_nt(int d_pad) {
  const int nt = (d_pad + 31) / 32;
  return nt <= 1   ? search_kernel<1, 2, U, QW, FLAT>
         : nt <= 2 ? search_kernel<2, 4, U, QW, FLAT>
         : nt <= 4 ? search_kernel<4, 8, U, QW, FLAT>
         : nt <= 8 ? search_kernel<8, 16, U, QW, FLAT>
                   : search_kernel<16, 32, U, QW, FLAT>;
}

// defined one per translation unit (kernels_search_u*w*[_flat].cu)
Kernel pick_u8w4(int d_pad);
Kernel pick_u4w4(int d_pad);
Kernel pick_u8w8(int d_pad);
Kernel pick_u8w4_flat(int d_pad);
Kernel pick_u4w4_flat(int d_pad);
Kernel pick_u8w8_flat(int d_pad);

}  // namespace skern
}  // namespace pf
