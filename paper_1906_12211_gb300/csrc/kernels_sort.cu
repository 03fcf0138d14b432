// Per-repetition sort of (code, position) pairs into the sorted arrays and the
// 13-bit prefix table (Sec. 4.2), most-significant bits first:
//   1. bucket_hist_kernel: per repetition, how many codes fall in each of the
//      8192 buckets of their top 13 bits;
//   2. bucket_scan_kernel: the exclusive scan of those counts is the prefix
//      table itself (pfx[t] = the first position whose top 13 bits are >= t);
//      it also seeds one write cursor per bucket and flags a repetition whose
//      largest bucket exceeds kBigBucket;
//   3. bucket_scatter_kernel: every pair goes to its bucket's region through
//      the bucket's cursor (an atomic add, so the order inside a bucket is
//      arbitrary at this point);
//   4. bucket_sort_warp_kernel / bucket_sort_cta_kernel: each bucket is sorted
//      in shared memory by the 64-bit key (code, position) with a bitonic
//      network.  The keys are distinct (positions are), so whatever order the
//      scatter left, the result is the stable (code, position) order,
//      deterministic.
// A repetition flagged in step 2 (a bucket of more than kBigBucket pairs, e.g.
// many identical points) is sorted instead by the stable LSD radix sort of
// kernels_build.cu, whose cost does not depend on the codes' distribution.
// The 4 + 4 + 8 + 16 bytes each pair moves are two passes over the arrays
// where four 8-bit LSD passes move about 121.
#include <algorithm>

#include "pf_internal.h"

namespace pf {

namespace {

constexpr int kTopBits = kPrefixBits;          // buckets = the prefix table's entries
constexpr int kBuckets = 1 << kTopBits;        // 8192
constexpr int kShift = 32 - kTopBits;          // bucket of a code = code >> kShift
constexpr int kHistThreads = 256;
constexpr int kHistItems = 64;                 // codes per thread in the histogram (few, large CTAs: one
constexpr int kHistTile = kHistThreads * kHistItems;  // flush of 8192 counters each)
constexpr int kScatterItems = 8;               // codes per thread in the scatter (many CTAs hide the
constexpr int kScatterTile = kHistThreads * kScatterItems;  // latency of its atomic adds)
constexpr int kWarpBucket = 512;               // a warp sorts buckets of up to this many pairs
constexpr int kBigBucket = 4096;               // a CTA sorts buckets of up to this many pairs
constexpr int kSortCtaThreads = 256;

// counts[tab][b] += the codes of this tile in bucket b (a shared histogram per CTA)
__global__ void __launch_bounds__(kHistThreads) bucket_hist_kernel(const uint32_t* __restrict__ codes, int64_t n,
                                                                   uint32_t* __restrict__ counts) {
  __shared__ uint32_t h[kBuckets];
  const int tab = blockIdx.y;
  for (int b = threadIdx.x; b < kBuckets; b += kHistThreads) h[b] = 0;
  __syncthreads();
  const uint32_t* c = codes + int64_t(tab) * n;
  const int64_t base = int64_t(blockIdx.x) * kHistTile;
  for (int t = 0; t < kHistItems; ++t) {
    const int64_t i = base + int64_t(t) * kHistThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[c[i] >> kShift], 1u);
  }
  __syncthreads();
  uint32_t* out = counts + int64_t(tab) * kBuckets;
  for (int b = threadIdx.x; b < kBuckets; b += kHistThreads)
    if (h[b]) atomicAdd(out + b, h[b]);
}

// One CTA per repetition: pfx[tab][b] = exclusive scan of counts (pfx[tab][8192]
// = n), cursor[tab][b] = pfx[tab][b], big[tab] = whether a bucket holds more than
// kBigBucket pairs.
__global__ void __launch_bounds__(1024) bucket_scan_kernel(const uint32_t* __restrict__ counts, int64_t n,
                                                           uint32_t* __restrict__ pfx, uint32_t* __restrict__ cursor,
                                                           int32_t* __restrict__ big) {
  constexpr int kPer = kBuckets / 1024;  // 8 buckets per thread
  __shared__ uint32_t part[1024];
  __shared__ int s_big;
  const int tab = blockIdx.x, t = threadIdx.x;
  const uint32_t* c = counts + int64_t(tab) * kBuckets;
  uint32_t v[kPer], sum = 0;
  int bigl = 0;
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    v[u] = c[t * kPer + u];
    sum += v[u];
    bigl |= v[u] > uint32_t(kBigBucket);
  }
  if (t == 0) s_big = 0;
  part[t] = sum;
  __syncthreads();
  if (bigl) s_big = 1;
  for (int off = 1; off < 1024; off <<= 1) {
    const uint32_t x = t >= off ? part[t - off] : 0u;
    __syncthreads();
    part[t] += x;
    __syncthreads();
  }
  uint32_t run = part[t] - sum;
  uint32_t* p = pfx + int64_t(tab) * kPrefixSize;
  uint32_t* cu = cursor + int64_t(tab) * kBuckets;
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    p[t * kPer + u] = run;
    cu[t * kPer + u] = run;
    run += v[u];
  }
  if (t == 1023) p[kBuckets] = uint32_t(n);
  __syncthreads();
  if (t == 0) big[tab] = s_big;
}

// Every (code, position) of an unflagged repetition to the next free slot of its
// bucket; lanes of a warp with the same bucket share one atomic add.
__global__ void __launch_bounds__(kHistThreads) bucket_scatter_kernel(const uint32_t* __restrict__ codes, int64_t n,
                                                                      uint32_t* __restrict__ cursor,
                                                                      const int32_t* __restrict__ big,
                                                                      uint32_t* __restrict__ kout,
                                                                      uint32_t* __restrict__ vout) {
  const int tab = blockIdx.y;
  if (big[tab]) return;
  const uint32_t* c = codes + int64_t(tab) * n;
  uint32_t* cu = cursor + int64_t(tab) * kBuckets;
  uint32_t* ko = kout + int64_t(tab) * n;
  uint32_t* vo = vout + int64_t(tab) * n;
  const int lane = threadIdx.x & 31;
  const int64_t base = int64_t(blockIdx.x) * kScatterTile;
  for (int t = 0; t < kScatterItems; ++t) {
    const int64_t i = base + int64_t(t) * kHistThreads + threadIdx.x;
    const bool valid = i < n;
    const uint32_t key = valid ? c[i] : 0u;
    const uint32_t b = valid ? key >> kShift : uint32_t(kBuckets);  // an invalid lane matches only invalid lanes
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int leader = __ffs(peers) - 1;
    uint32_t slot = 0;
    if (valid && lane == leader) slot = atomicAdd(cu + b, uint32_t(__popc(peers)));
    slot = __shfl_sync(0xffffffffu, slot, leader);
    if (valid) {
      const uint32_t pos = slot + __popc(peers & ((1u << lane) - 1u));
      ko[pos] = key;
      vo[pos] = uint32_t(i);
    }
  }
}

// Sort keys[0, s) in shared memory ascending with a bitonic network over the
// next power of two >= s (the slots beyond s hold the largest key), by `nthr`
// threads of which this is `tid`; SYNC() orders the stages.
#define PF_BITONIC(keys, s, tid, nthr, SYNC)                                        \
  do {                                                                              \
    int P_ = 2;                                                                     \
    while (P_ < (s)) P_ <<= 1;                                                      \
    for (int e_ = (s) + (tid); e_ < P_; e_ += (nthr)) (keys)[e_] = ~0ull;          \
    SYNC();                                                                         \
    for (int k_ = 2; k_ <= P_; k_ <<= 1)                                            \
      for (int j_ = k_ >> 1; j_ > 0; j_ >>= 1) {                                    \
        for (int i_ = (tid); i_ < P_ / 2; i_ += (nthr)) {                           \
          const int lo_ = (i_ / j_) * 2 * j_ + (i_ % j_), hi_ = lo_ + j_;           \
          const uint64_t a_ = (keys)[lo_], b_ = (keys)[hi_];                        \
          if ((a_ > b_) == ((lo_ & k_) == 0)) {                                     \
            (keys)[lo_] = b_;                                                       \
            (keys)[hi_] = a_;                                                       \
          }                                                                         \
        }                                                                           \
        SYNC();                                                                     \
      }                                                                             \
  } while (0)

__device__ __forceinline__ void warp_sync() { __syncwarp(); }
__device__ __forceinline__ void cta_sync() { __syncthreads(); }

// A warp per bucket of 2 .. kWarpBucket pairs of an unflagged repetition: load
// the bucket's (code << 32 | position) keys, sort them, write them back.
__global__ void __launch_bounds__(256) bucket_sort_warp_kernel(const uint32_t* __restrict__ pfx, int64_t n, int tables,
                                                               const int32_t* __restrict__ big,
                                                               uint32_t* __restrict__ kio, uint32_t* __restrict__ vio) {
  __shared__ uint64_t keys[8][kWarpBucket];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t* kw = keys[w];
  const int64_t total = int64_t(tables) * kBuckets;
  for (int64_t g = int64_t(blockIdx.x) * 8 + w; g < total; g += int64_t(gridDim.x) * 8) {
    const int tab = int(g / kBuckets), b = int(g - int64_t(tab) * kBuckets);
    if (big[tab]) continue;
    const uint32_t* p = pfx + int64_t(tab) * kPrefixSize;
    const uint32_t lo = p[b];
    const int s = int(p[b + 1] - lo);
    if (s < 2 || s > kWarpBucket) continue;  // uniform in the warp
    uint32_t* kb = kio + int64_t(tab) * n + lo;
    uint32_t* vb = vio + int64_t(tab) * n + lo;
    for (int e = lane; e < s; e += 32) kw[e] = (uint64_t(kb[e]) << 32) | vb[e];
    PF_BITONIC(kw, s, lane, 32, warp_sync);
    for (int e = lane; e < s; e += 32) {
      kb[e] = uint32_t(kw[e] >> 32);
      vb[e] = uint32_t(kw[e]);
    }
    __syncwarp();
  }
}

// A CTA per bucket of kWarpBucket+1 .. kBigBucket pairs: the same with the
// CTA's threads.
__global__ void __launch_bounds__(kSortCtaThreads) bucket_sort_cta_kernel(const uint32_t* __restrict__ pfx, int64_t n,
                                                                          int tables, const int32_t* __restrict__ big,
                                                                          uint32_t* __restrict__ kio,
                                                                          uint32_t* __restrict__ vio) {
  __shared__ uint64_t keys[kBigBucket];
  const int64_t total = int64_t(tables) * kBuckets;
  for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
    const int tab = int(g / kBuckets), b = int(g - int64_t(tab) * kBuckets);
    if (big[tab]) continue;
    const uint32_t* p = pfx + int64_t(tab) * kPrefixSize;
    const uint32_t lo = p[b];
    const int s = int(p[b + 1] - lo);
    if (s <= kWarpBucket) continue;  // uniform in the CTA
    uint32_t* kb = kio + int64_t(tab) * n + lo;
    uint32_t* vb = vio + int64_t(tab) * n + lo;
    const int tid = int(threadIdx.x);
    for (int e = tid; e < s; e += kSortCtaThreads) keys[e] = (uint64_t(kb[e]) << 32) | vb[e];
    PF_BITONIC(keys, s, tid, kSortCtaThreads, cta_sync);
    for (int e = tid; e < s; e += kSortCtaThreads) {
      kb[e] = uint32_t(keys[e] >> 32);
      vb[e] = uint32_t(keys[e]);
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t sort_tables(pf_index* ix, uint32_t* codes_unsorted, cudaStream_t s) {
  const int64_t n = ix->n;
  const int L = ix->L;
  if (L <= 0 || n <= 0) return cudaSuccess;
  // repetitions per group: their sorted arrays (8 bytes per pair) stay within
  // about 64 MB, so the scatter's writes gather in L2
  const int G = int(std::max<int64_t>(1, std::min<int64_t>(L, (int64_t(64) << 20) / std::max<int64_t>(1, n * 8))));
  const int tiles = int((n + kHistTile - 1) / kHistTile);
  const int stiles = int((n + kScatterTile - 1) / kScatterTile);
  uint32_t *counts = nullptr, *cursor = nullptr;
  int32_t* big = nullptr;
  cudaError_t e;
  if ((e = cudaMallocAsync(&counts, sizeof(uint32_t) * size_t(kBuckets) * G, s)) != cudaSuccess) return e;
  if ((e = cudaMallocAsync(&cursor, sizeof(uint32_t) * size_t(kBuckets) * G, s)) != cudaSuccess) return e;
  if ((e = cudaMallocAsync(&big, sizeof(int32_t) * size_t(L), s)) != cudaSuccess) return e;
  const int sort_blocks = ix->num_sms * 8;
  for (int j0 = 0; j0 < L && e == cudaSuccess; j0 += G) {
    const int g = std::min(G, L - j0);
    const uint32_t* keys = codes_unsorted + int64_t(j0) * n;
    uint32_t* outk = ix->codes + int64_t(j0) * n;
    uint32_t* outv = ix->ids + int64_t(j0) * n;
    uint32_t* pfx = ix->pfx + int64_t(j0) * kPrefixSize;
    if ((e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * size_t(kBuckets) * g, s)) != cudaSuccess) break;
    bucket_hist_kernel<<<dim3(tiles, g), kHistThreads, 0, s>>>(keys, n, counts);
    bucket_scan_kernel<<<g, 1024, 0, s>>>(counts, n, pfx, cursor, big + j0);
    bucket_scatter_kernel<<<dim3(stiles, g), kHistThreads, 0, s>>>(keys, n, cursor, big + j0, outk, outv);
    bucket_sort_warp_kernel<<<sort_blocks, 256, 0, s>>>(pfx, n, g, big + j0, outk, outv);
    bucket_sort_cta_kernel<<<sort_blocks, kSortCtaThreads, 0, s>>>(pfx, n, g, big + j0, outk, outv);
    e = cudaGetLastError();
  }
  // repetitions with a bucket too large for shared memory: the LSD radix sort
  std::vector<int32_t> hbig(size_t(L), 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hbig.data(), big, sizeof(int32_t) * size_t(L), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(counts, s);
  cudaFreeAsync(cursor, s);
  cudaFreeAsync(big, s);
  for (int j = 0; j < L && e == cudaSuccess; ++j) {
    if (!hbig[size_t(j)]) continue;
    int j1 = j + 1;
    while (j1 < L && hbig[size_t(j1)]) ++j1;
    e = lsd_sort_tables(ix, codes_unsorted, j, j1, s);
    j = j1 - 1;
  }
  return e;
}

}  // namespace pf
