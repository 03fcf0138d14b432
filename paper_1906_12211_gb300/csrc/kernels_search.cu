// The adaptive k-NN query (Algorithm 1 as implemented in Sec. 4.1-4.2), one
// warp per query, persistent CTAs pulling queries from an atomic counter so
// queries of very different cost share one launch.
//
// Per round at prefix length i, for every repetition j the warp extends the
// range [l, r) of positions around the query's code so that it covers the
// block of codes sharing the first i bits, growing each side in whole
// segments of B entries (Sec. 4.2, App. C).  The new positions of 32
// repetitions are flattened and streamed lane-parallel, four per lane per step
// so that many independent loads are in flight: position -> id -> sketch
// Hamming filter (Sec. 4.2) -> compacted candidate buffer.  Buffered
// candidates are scored (float32 canonical, or a bfloat16 estimate followed by
// an exact float32 rerank of those whose estimate plus its error bound can
// still reach the running k-th similarity) and offered to the top-k
// accumulator (unique ids, ordered by similarity then id).  After the round
// the stop test of Lemma 1 runs in float64.
//
// Readings shared with the oracle: the sketch threshold is taken from the
// top-k at the start of each round and, in a query's first round (which starts
// with an empty top-k), also at the start of every group of 32 repetitions (the
// paper refreshes it every k insertions, Sec. 4.2; a group is one warp step,
// and all candidates of the previous group have been offered by then); the
// stop test runs once per round (Sec. 4.1); the
// canonical similarity is float32 with 32 partial sums (partial c takes the
// coordinates = c mod 32 in index order by fused multiply-add) combined as
// s[c] += s[c + w] for w = 16, 8, 4, 2, 1.  Only the filter depends on s_k and
// it uses the round's snapshot, so the result does not depend on the order in
// which lanes visit candidates.
#include <cuda_bf16.h>

#include "pf_internal.h"

namespace pf {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 4;      // warps (queries in flight) per CTA
constexpr int kUnroll = 4;     // candidate positions per lane per step
constexpr int kCandBuf = 256;  // compacted candidate ids per warp
constexpr int kFlushAt = kCandBuf - 32 * kUnroll;

struct Dev {
  int n;
  int d, d_pad, L, Kb, M, B, family, ell;
  const float* x32;
  const __nv_bfloat16* x16;
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
__device__ __noinline__ double collision_prob(const Dev& P, double s, int depth) {
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
__device__ __forceinline__ uint32_t lower_bound(const uint32_t* c, uint32_t lo, uint32_t hi, uint32_t key) {
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(c + mid) < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

struct WarpState {
  float* q;         // [d_pad]
  uint32_t* l;      // [L]
  uint32_t* r;      // [L]
  float* pq_s;      // [k_max]
  uint32_t* pq_id;  // [k_max]
  uint32_t* cbuf;   // [kCandBuf]
};

struct Counters {
  uint32_t retrieved = 0, passed = 0, scored = 0, reranked = 0;
};

// Offer (s, id) to the sorted top-k of the warp (all lanes call with the same
// arguments).  Returns the new size.
__device__ __forceinline__ int pq_offer(WarpState& w, int size, int k, float s, uint32_t id, int lane) {
  if (size == k && !better(s, id, w.pq_s[k - 1], w.pq_id[k - 1])) return size;
  bool dup = false;
  int cnt = 0;
  for (int t = lane; t < size; t += 32) {
    const uint32_t it = w.pq_id[t];
    dup |= it == id;
    cnt += better(w.pq_s[t], it, s, id) ? 1 : 0;
  }
  if (__any_sync(kFull, dup)) return size;
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

// Canonical float32 similarities of the query with two rows, computed by the
// 8 lanes of a group (lane g8 owns partials 4*g8 .. 4*g8+3, i.e. float4
// chunks g8, g8+8, ...).  Both rows' loads are issued before the arithmetic.
template <int NT>
__device__ __forceinline__ void sim_canonical2(const float* __restrict__ q, const float* __restrict__ ra,
                                               const float* __restrict__ rb, int d_pad, int g8, unsigned gmask,
                                               float& out_a, float& out_b) {
  const float4* q4 = reinterpret_cast<const float4*>(q);
  const float4* a4 = reinterpret_cast<const float4*>(ra);
  const float4* b4 = reinterpret_cast<const float4*>(rb);
  float4 va[NT], vb[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int ch = g8 + 8 * t;
    va[t] = ch * 4 < d_pad ? __ldg(a4 + ch) : make_float4(0.f, 0.f, 0.f, 0.f);
    vb[t] = ch * 4 < d_pad ? __ldg(b4 + ch) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  float4 sa = make_float4(0.f, 0.f, 0.f, 0.f), sb = sa;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int ch = g8 + 8 * t;
    if (ch * 4 < d_pad) {
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

// bfloat16 estimate of <q, x> by the 4 lanes of a group: float32 query against
// the bfloat16 row (chunks of 8 elements g4, g4+4, ...), any summation order.
template <int NT>
__device__ __forceinline__ float sim_bf16(const float* __restrict__ q, const __nv_bfloat16* __restrict__ row,
                                          int d_pad, int g4, unsigned gmask) {
  const uint4* r8 = reinterpret_cast<const uint4*>(row);
  uint4 v[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int ch = g4 + 4 * t;
    v[t] = ch * 8 < d_pad ? __ldg(r8 + ch) : make_uint4(0u, 0u, 0u, 0u);
  }
  float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int ch = g4 + 4 * t;
    if (ch * 8 < d_pad) {
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
  float acc = acc0 + acc1;
  acc += __shfl_xor_sync(gmask, acc, 2, 4);
  acc += __shfl_xor_sync(gmask, acc, 1, 4);
  return acc;
}

// Exact float32 similarities of the `cnt` ids at the front of cbuf, each
// offered to the top-k (8 candidates per step: 4 groups of 8 lanes, 2 rows
// each).
template <int NT>
__device__ __forceinline__ int canonical_and_offer(const Dev& P, WarpState& w, int cnt, int size, int k, int lane) {
  const int g = lane >> 3, g8 = lane & 7;
  const unsigned gmask = 0xffu << (lane & ~7);
  for (int c0 = 0; c0 < cnt; c0 += 8) {
    const int ca = c0 + g, cb = c0 + 4 + g;
    const uint32_t ida = ca < cnt ? w.cbuf[ca] : w.cbuf[c0];
    const uint32_t idb = cb < cnt ? w.cbuf[cb] : w.cbuf[c0];
    float sa, sb;
    sim_canonical2<NT>(w.q, P.x32 + size_t(ida) * P.d_pad, P.x32 + size_t(idb) * P.d_pad, P.d_pad, g8, gmask, sa, sb);
    const int m = min(8, cnt - c0);
    for (int t = 0; t < m; ++t) {
      const int src = (t & 3) * 8;
      const float s = __shfl_sync(kFull, t < 4 ? sa : sb, src);
      const uint32_t id = __shfl_sync(kFull, t < 4 ? ida : idb, src);
      size = pq_offer(w, size, k, s, id, lane);
    }
  }
  return size;
}

// Score the cnt buffered candidate ids and offer them to the top-k.
template <int NT>
__device__ __forceinline__ int flush_candidates(const Dev& P, WarpState& w, int cnt, int size, int k, int lane,
                                                Counters& ct) {
  if (lane == 0) ct.scored += cnt;
  if (P.scoring != 1) return canonical_and_offer<NT>(P, w, cnt, size, k, lane);
  // bfloat16 estimates, 8 rows per step (4 lanes each).  A candidate can enter
  // the top-k only if its exact similarity reaches the running k-th, which
  // never decreases; the estimate is within bf16_err of the exact value, so
  // candidates with estimate + bf16_err below the current k-th are dropped and
  // the others are compacted in place at the front of cbuf.
  const int g = lane >> 2, g4 = lane & 3;
  const unsigned gmask = 0xfu << (lane & ~3);
  const bool full = size == k;
  const float kth = full ? w.pq_s[k - 1] : -INFINITY;
  int nr = 0;
  for (int c0 = 0; c0 < cnt; c0 += 8) {
    const int c = c0 + g;
    const bool valid = c < cnt;
    const uint32_t id = valid ? w.cbuf[c] : w.cbuf[c0];
    const float est = sim_bf16<NT>(w.q, P.x16 + size_t(id) * P.d_pad, P.d_pad, g4, gmask);
    const bool need = valid && (!full || est + P.bf16_err >= kth);
    const unsigned b = __ballot_sync(kFull, need && g4 == 0);
    __syncwarp();
    if (need && g4 == 0) w.cbuf[nr + __popc(b & ((1u << lane) - 1u))] = id;
    nr += __popc(b);
    __syncwarp();
  }
  if (lane == 0) ct.reranked += nr;
  return canonical_and_offer<NT>(P, w, nr, size, k, lane);
}

// NT = d_pad / 32 rounded up: float4 chunks of a float32 row per lane of an
// 8-lane group (and 16-byte chunks of a bfloat16 row per lane of a 4-lane group)
template <int NT>
__global__ void __launch_bounds__(kWarps * 32, 8) search_kernel(Dev P) {
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
  const uint32_t n = uint32_t(P.n);
  const uint32_t lt_mask = (1u << lane) - 1u;

  for (;;) {
    int qi = 0;
    if (lane == 0) qi = atomicAdd(P.counter, 1);
    qi = __shfl_sync(kFull, qi, 0);
    if (qi >= P.Q) break;

    const int k = P.k[qi];
    const double rec = P.recall[qi];
    if (k < 1 || k > kmax || !(rec > 0.0 && rec < 1.0)) {
      if (lane == 0) atomicOr(P.counter + 1, 1);
      for (int t = lane; t < kmax; t += 32) {
        P.out_ids[size_t(qi) * kmax + t] = 0xffffffffu;
        P.out_sims[size_t(qi) * kmax + t] = -INFINITY;
      }
      continue;
    }
    const double delta = 1.0 - rec;
    const float* qg = P.qx + size_t(qi) * d_pad;
    for (int i = lane; i < d_pad; i += 32) w.q[i] = qg[i];
    const uint32_t* qc = P.qcodes + size_t(qi) * L;
    const uint64_t* qs = P.qsk + size_t(qi) * P.M;
    // start depth: the plain schedule starts at K (Sec. 4.1); a given start i0
    // in [0, K) takes the whole block at i0 in the first round
    int i0 = P.Kb;
    if (P.start) {
      const int sd = P.start[qi];
      if (sd >= 0 && sd < P.Kb) i0 = sd;
    }
    // initial empty range at the first code >= the query's code
    for (int j = lane; j < L; j += 32) {
      const uint32_t c = qc[j];
      const uint32_t* pj = P.pfx + size_t(j) * kPrefixSize;
      const uint32_t t = c >> (32 - kPrefixBits);
      const uint32_t lb = lower_bound(P.codes + size_t(j) * n, __ldg(pj + t), __ldg(pj + t + 1), c);
      w.l[j] = lb;
      w.r[j] = lb;
    }
    __syncwarp();

    int size = 0, rounds = 0, depth = i0, prev = -1, stop_depth = i0;  // prev < 0: probe both sides
    int full_depth = -1;  // first depth after whose round k points were held
    Counters ct;
    for (;;) {
      if (depth == 0) {
        // prefix length 0: every point collides in every repetition, so the
        // round is a linear scan of all points (Lemma 1, i = 0), unfiltered.
        int nb = 0;
        for (uint32_t b0 = 0; b0 < n; b0 += 32) {
          const uint32_t id = b0 + lane;
          const unsigned m = __ballot_sync(kFull, id < n);
          if (id < n) w.cbuf[nb + __popc(m & lt_mask)] = id;
          nb += __popc(m);
          if (lane == 0) {
            ct.retrieved += __popc(m);
            ct.passed += __popc(m);
          }
          __syncwarp();
          if (nb > kFlushAt) {
            size = flush_candidates<NT>(P, w, nb, size, k, lane, ct);
            nb = 0;
          }
        }
        if (nb) size = flush_candidates<NT>(P, w, nb, size, k, lane, ct);
        ++rounds;
        stop_depth = 0;
        if (size == k && full_depth < 0) full_depth = 0;
        break;
      }
      const uint32_t mask = 0xffffffffu << (32 - depth);
      const bool single = prev == depth + 1;
      int nb = 0;
      int tau = 64;
      for (int jb = 0; jb < L; jb += 32) {
        if (jb == 0 || rounds == 0) {
          // threshold snapshot; the previous group's candidates go into the top-k first
          if (nb) {
            size = flush_candidates<NT>(P, w, nb, size, k, lane, ct);
            nb = 0;
          }
          tau = size == k ? filter_tau(P, w.pq_s[k - 1]) : 64;
        }
        const int j = jb + lane;
        uint32_t l = 0, r = 0, nl = 0, nr = 0;
        if (j < L) {
          const uint32_t qcj = qc[j];
          const uint32_t* cj = P.codes + size_t(j) * n;
          l = w.l[j];
          r = w.r[j];
          nl = l;
          nr = r;
          // in a one-bit step only the side of the dropped bit can grow
          // (bit `depth`, counted from the top, of the query's code)
          const bool dropped_one = (qcj >> (31 - depth)) & 1u;
          const bool try_left = !single || dropped_one;
          const bool try_right = !single || !dropped_one;
          const uint32_t B = uint32_t(P.B);
          if (try_left && l > 0 && prefix_match(__ldg(cj + l - 1), qcj, mask)) {
            // smallest m >= 1 with l - B*m <= 0 or codes[l - B*m - 1] outside the block
            uint32_t lo = 0, hi = 1;
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
            const int64_t pos = int64_t(l) - int64_t(B) * hi;
            nl = pos < 0 ? 0u : uint32_t(pos);
          }
          if (try_right && r < n && prefix_match(__ldg(cj + r), qcj, mask)) {
            uint32_t lo = 0, hi = 1;
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
            const int64_t pos = int64_t(r) + int64_t(B) * hi;
            nr = pos > int64_t(n) ? n : uint32_t(pos);
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
        for (uint32_t e0 = 0; e0 < total; e0 += 32 * kUnroll) {
          uint32_t id[kUnroll], pos[kUnroll];
          int jo[kUnroll];
          bool valid[kUnroll];
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            const uint32_t idx = e0 + 32 * u + lane;
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
            valid[u] = idx < total;
            const uint32_t off = idx - ex_o;
            jo[u] = jb + o;
            pos[u] = off < cl_o ? nl_o + off : r_o + (off - cl_o);
          }
#pragma unroll
          for (int u = 0; u < kUnroll; ++u)
            id[u] = valid[u] ? __ldg(P.ids + size_t(jo[u]) * n + pos[u]) : 0u;
          bool pass[kUnroll];
          if (P.filter) {
            uint64_t h[kUnroll];
            if (P.skc) {  // the sketch sits at the same position as the id
#pragma unroll
              for (int u = 0; u < kUnroll; ++u)
                h[u] = valid[u] ? __ldg(P.skc + size_t(jo[u]) * n + pos[u]) ^ qs[jo[u] % P.M] : 0ull;
            } else {
#pragma unroll
              for (int u = 0; u < kUnroll; ++u) {
                const int m = jo[u] % P.M;
                h[u] = valid[u] ? __ldg(P.sk + size_t(m) * n + id[u]) ^ qs[m] : 0ull;
              }
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) pass[u] = valid[u] && __popcll(h[u]) <= tau;
          } else {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) pass[u] = valid[u];
          }
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            const unsigned pm = __ballot_sync(kFull, pass[u]);
            if (pass[u]) w.cbuf[nb + __popc(pm & lt_mask)] = id[u];
            nb += __popc(pm);
            if (lane == 0) ct.passed += __popc(pm);
          }
          __syncwarp();
          if (nb > kFlushAt) {
            size = flush_candidates<NT>(P, w, nb, size, k, lane, ct);
            nb = 0;
          }
        }
      }
      if (nb) size = flush_candidates<NT>(P, w, nb, size, k, lane, ct);
      ++rounds;
      stop_depth = depth;
      if (size == k && full_depth < 0) full_depth = depth;
      int stop = 0;
      if (lane == 0 && size == k) {
        const double p = collision_prob(P, double(w.pq_s[k - 1]), depth);
        const double fail = ipow(__dsub_rn(1.0, p), L);
        stop = fail <= delta ? 1 : 0;
      }
      stop = __shfl_sync(kFull, stop, 0);
      if (stop) break;
      prev = depth;
      depth -= 1;
    }

    for (int t = lane; t < kmax; t += 32) {
      P.out_ids[size_t(qi) * kmax + t] = t < size ? w.pq_id[t] : 0xffffffffu;
      P.out_sims[size_t(qi) * kmax + t] = t < size ? w.pq_s[t] : -INFINITY;
    }
    if (P.stats && lane == 0) {
      pf_query_stats st;
      st.start_depth = i0;
      st.stop_depth = stop_depth;
      st.rounds = rounds;
      st.full_depth = full_depth;
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
  P.n = int(ix->n);
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
  P.skc = ix->skc;
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
  const int nt = (P.d_pad + 31) / 32;
  auto kern = nt <= 1 ? search_kernel<1> : nt <= 2 ? search_kernel<2> : nt <= 4 ? search_kernel<4> : search_kernel<8>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int blocks = ix->num_sms * per_sm;
  const int need = (a.Q + kWarps - 1) / kWarps;
  if (blocks > need) blocks = need;
  kern<<<blocks, kWarps * 32, smem, s>>>(P);
  return cudaGetLastError();
}

}  // namespace pf
