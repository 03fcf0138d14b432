// Index-build kernels: normalisation, hashing (projection + sign/argmax with
// float64 recheck), per-repetition LSD radix sort of (code, position) pairs,
// and the 13-bit prefix tables.
#include <cuda_bf16.h>

#include <algorithm>

#include <cuda_fp8.h>

#include "pf_internal.h"

namespace pf {

// ---------------------------------------------------------------------------
// Normalisation (Sec. 4.2 "Vector storage"): squared norm summed in float64 in
// index order (float*float products are exact in float64), correctly rounded
// sqrt and division in float64, one rounding to float.  One thread per row;
// padding columns are zero; a zero row stays zero.
// ---------------------------------------------------------------------------
__global__ void normalize_kernel(const float* __restrict__ in, int64_t rows, int d, int d_pad,
                                 float* __restrict__ x32, __nv_bfloat16* __restrict__ xh,
                                 __nv_bfloat16* __restrict__ xl) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const float* row = in + r * d;
  double ss = 0.0;
  for (int i = 0; i < d; ++i) {
    const double v = double(row[i]);
    ss = __dadd_rn(ss, __dmul_rn(v, v));
  }
  const double nrm = __dsqrt_rn(ss);
  float* o = x32 + r * d_pad;
  for (int i = 0; i < d_pad; ++i) {
    const float y = (i < d && nrm > 0.0) ? __double2float_rn(__ddiv_rn(double(row[i]), nrm)) : 0.0f;
    o[i] = y;
    if (xh) {
      const __nv_bfloat16 h = __float2bfloat16_rn(y);
      xh[r * d_pad + i] = h;
      if (xl) xl[r * d_pad + i] = __float2bfloat16_rn(y - __bfloat162float(h));
    }
  }
}

// e4m3 copy of a normalised row: scale = max |x_i| / 448 (the largest finite
// e4m3 value), code_i = e4m3(x_i / scale) rounded to nearest even, saturated.
// meta = (scale, bound) with bound >= |<q, x> - scale * <q, dec(code)>| plus
// the float32 rounding of the estimate and of the canonical similarity, for
// any q with |q|_2 <= 1 + 2^-16: by Cauchy-Schwarz the first part is at most
// |q| |x - scale dec(code)|_2, the residual norm taken here in float64.
__global__ void quantize_fp8_kernel(const float* __restrict__ x32, int64_t rows, int d, int d_pad,
                                    uint8_t* __restrict__ x8, float2* __restrict__ meta) {
  const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const float* row = x32 + r * d_pad;
  float mx = 0.f;
  for (int i = 0; i < d; ++i) mx = fmaxf(mx, fabsf(row[i]));
  const float scale = mx > 0.f ? mx / 448.f : 1.f;
  double res = 0.0;
  for (int i = 0; i < d_pad; ++i) {
    uint8_t c = 0;
    if (i < d) c = __nv_cvt_float_to_fp8(row[i] / scale, __NV_SATFINITE, __NV_E4M3);
    x8[r * d_pad + i] = c;
    const float dec = __half2float(__half(__nv_cvt_fp8_to_halfraw(c, __NV_E4M3)));
    const double e = double(row[i]) - double(scale) * double(dec);  // the product is exact in float64
    res += e * e;
  }
  const double en = sqrt(res) * (1.0 + 1e-12);
  const double bound = (1.0 + ldexp(1.0, -16)) * (en + (2.0 * d_pad + 2.0) * ldexp(1.0, -24) * (1.0 + en));
  meta[r] = make_float2(scale, __double2float_ru(bound));
}

__global__ void round_rows_f16_kernel(float* __restrict__ x32, int64_t count, __half* __restrict__ xf16,
                                      __nv_bfloat16* __restrict__ xh, __nv_bfloat16* __restrict__ xl) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x) {
    const __half h = __float2half_rn(x32[i]);
    const float y = __half2float(h);  // exact
    x32[i] = y;
    xf16[i] = h;
    const __nv_bfloat16 b = __float2bfloat16_rn(y);
    xh[i] = b;
    if (xl) xl[i] = __float2bfloat16_rn(y - __bfloat162float(b));
  }
}

cudaError_t launch_round_rows_f16(float* x32, int64_t rows, int d_pad, __half* xf16, __nv_bfloat16* xh,
                                  __nv_bfloat16* xl, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  round_rows_f16_kernel<<<1024, 256, 0, s>>>(x32, rows * d_pad, xf16, xh, xl);
  return cudaGetLastError();
}

cudaError_t launch_normalize(const float* in, int64_t rows, int d, int d_pad, float* x32, __nv_bfloat16* xh,
                             __nv_bfloat16* xl, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  const int tb = 128;
  normalize_kernel<<<unsigned((rows + tb - 1) / tb), tb, 0, s>>>(in, rows, d, d_pad, x32, xh, xl);
  return cudaGetLastError();
}

// Pooling (Sec. 3.2): table j's code concatenates the values of its pool
// functions sel[j][0..F), the first in the most significant bits; function f is
// slot f % F of pool group f / F, whose code holds it in bits
// 32 - l (slot + 1) .. 32 - l slot - 1.
__global__ void pool_gather_kernel(const uint32_t* __restrict__ gcodes, int64_t gj, int64_t gp, int64_t npts,
                                   const int32_t* __restrict__ sel, int L, int F, int ell, uint32_t* __restrict__ codes,
                                   int64_t cj, int64_t cp) {
  const uint32_t mask = (1u << ell) - 1u;
  const int64_t total = npts * L;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t j = e / npts, p = e % npts;
    uint32_t code = 0;
    for (int st = 0; st < F; ++st) {
      const int f = __ldg(sel + j * F + st);
      const int g = f / F, slot = f % F;
      const uint32_t v = (__ldg(gcodes + g * gj + p * gp) >> (32 - ell * (slot + 1))) & mask;
      code |= v << (32 - ell * (st + 1));
    }
    codes[j * cj + p * cp] = code;
  }
}

cudaError_t launch_pool_gather(const pf_index* ix, const uint32_t* gcodes, int64_t gj, int64_t gp, int64_t npts,
                               uint32_t* codes, int64_t cj, int64_t cp, cudaStream_t s) {
  if (npts <= 0) return cudaSuccess;
  const int64_t total = npts * ix->L;
  const int blocks = int(std::min<int64_t>((total + 255) / 256, int64_t(ix->num_sms) * 32));
  pool_gather_kernel<<<blocks, 256, 0, s>>>(gcodes, gj, gp, npts, ix->pool_sel, ix->L, ix->lay.fns, ix->lay.ell,
                                            codes, cj, cp);
  return cudaGetLastError();
}

cudaError_t launch_quantize_fp8(const float* x32, int64_t rows, int d, int d_pad, uint8_t* x8, float2* meta,
                                cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  quantize_fp8_kernel<<<unsigned((rows + 255) / 256), 256, 0, s>>>(x32, rows, d, d_pad, x8, meta);
  return cudaGetLastError();
}

cudaError_t launch_hash(const pf_index* ix, const float* x32, const __nv_bfloat16* xh, const __nv_bfloat16* xl,
                        int64_t npts, uint32_t* codes, int64_t cj, int64_t cp, uint64_t* sk, int64_t sm,
                        int64_t sp, RecheckReq* rq, uint32_t* rq_count, uint32_t rq_cap, cudaStream_t s,
                        int tables) {
  if (npts <= 0) return cudaSuccess;
  // repetitions hashed from rows; the pseudo-random family has its own kernel
  // and leaves only the sketches to the row kernels
  if (tables < 0) tables = ix->L;
  if (ix->family == PF_CROSSPOLYTOPE_FHT) {
    const cudaError_t e = launch_hash_fht(ix, x32, npts, codes, cj, cp, s);
    if (e != cudaSuccess) return e;
    tables = 0;
  }
  // every projection runs on the tensor cores; the caller provides the
  // bfloat16 halves of the rows
  if (!xh || !xl) return cudaErrorInvalidValue;
  return launch_hash_tc(ix, xh, xl, x32, npts, codes, cj, cp, sk, sm, sp, ix->dev_error, rq, rq_count, rq_cap, s,
                        tables);
}

// ---------------------------------------------------------------------------
// Per-repetition stable LSD radix sort of (code, position), 4 passes of 8 bits
// (positions start as 0..n-1, so equal codes stay in position order, Sec. 4.2).
// Each pass: per-tile digit histograms -> one exclusive scan per repetition in
// (digit, tile) order -> stable scatter.  Within a tile, each warp ranks its
// own contiguous slice with warp match masks, so equal digits keep their input
// order.  No kernel waits on another CTA.
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;

__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint32_t* __restrict__ keys, int64_t n,
                                                                 int shift, int ntiles,
                                                                 uint32_t* __restrict__ counts) {
  __shared__ uint32_t h[256];
  const int tile = blockIdx.x, tab = blockIdx.y;
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t* k = keys + int64_t(tab) * n;
  const int64_t base = int64_t(tile) * kSortTile;
  for (int t = 0; t < kSortItems; ++t) {
    const int64_t i = base + int64_t(t) * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(k[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[(int64_t(tab) * 256 + threadIdx.x) * ntiles + tile] = h[threadIdx.x];
}

// exclusive scan of counts[tab][256*ntiles] (digit-major), one CTA per table
__global__ void __launch_bounds__(1024) radix_scan_kernel(uint32_t* __restrict__ counts, int ntiles) {
  __shared__ uint32_t part[1024];
  const int64_t len = int64_t(256) * ntiles;
  uint32_t* c = counts + int64_t(blockIdx.x) * len;
  const int64_t per = (len + 1023) / 1024;
  const int64_t b = threadIdx.x * per, e = min(len, b + per);
  uint32_t sum = 0;
  for (int64_t i = b; i < e; ++i) sum += c[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - sum;
  for (int64_t i = b; i < e; ++i) {
    const uint32_t v = c[i];
    c[i] = run;
    run += v;
  }
}

// Stable scatter of one tile: warp w ranks the keys of its contiguous 512-key
// slice (item t of lane l is key w*512 + t*32 + l, so (w, t, l) is the input
// order) with match masks against its own running digit counts, without
// waiting for the other warps; then one CTA-wide pass turns the warps' digit
// counts into offsets (the tile's offset of the digit, plus the counts of the
// earlier warps), and every key goes to offset + its rank in its warp.
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t n, int shift, int ntiles, const uint32_t* __restrict__ offsets) {
  constexpr int kWarps = kSortThreads / 32;
  __shared__ uint32_t wcount[kWarps][256];  // per warp: digit counts, then digit offsets
  const int tile = blockIdx.x, tab = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t* ki = kin + int64_t(tab) * n;
  const uint32_t* vi = vin ? vin + int64_t(tab) * n : nullptr;
  uint32_t* ko = kout + int64_t(tab) * n;
  uint32_t* vo = vout + int64_t(tab) * n;
  for (int w = 0; w < kWarps; ++w) wcount[w][threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = int64_t(tile) * kSortTile + int64_t(warp) * 32 * kSortItems;
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
#pragma unroll
  for (int t = 0; t < kSortItems; ++t) {
    const int64_t i = base + int64_t(t) * 32 + lane;
    const bool valid = i < n;
    key[t] = valid ? ki[i] : 0u;
    val[t] = valid ? (vi ? vi[i] : uint32_t(i)) : 0u;
    const uint32_t dig = valid ? ((key[t] >> shift) & 255u) : 256u;
    const uint32_t peers = __match_any_sync(0xffffffffu, dig);
    rank[t] = valid ? wcount[warp][dig] + __popc(peers & lt_mask) : 0u;
    __syncwarp();
    if (valid && (peers & lt_mask) == 0) wcount[warp][dig] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {  // per digit: the tile's offset plus the counts of the earlier warps
    const int dg = threadIdx.x;
    uint32_t run = offsets[(int64_t(tab) * 256 + dg) * ntiles + tile];
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = wcount[w][dg];
      wcount[w][dg] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < kSortItems; ++t) {
    const int64_t i = base + int64_t(t) * 32 + lane;
    if (i < n) {
      const uint32_t pos = wcount[warp][(key[t] >> shift) & 255u] + rank[t];
      ko[pos] = key[t];
      vo[pos] = val[t];
    }
  }
}

// pfx[t] = first position whose top 13 bits are >= t (t = 0..8192)
__global__ void prefix_kernel(const uint32_t* __restrict__ codes, int64_t n, uint32_t* __restrict__ pfx) {
  const int tab = blockIdx.y;
  const uint32_t* c = codes + int64_t(tab) * n;
  uint32_t* out = pfx + int64_t(tab) * kPrefixSize;
  for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < n; p += int64_t(gridDim.x) * blockDim.x) {
    const int top = int(c[p] >> (32 - kPrefixBits));
    const int prev = p == 0 ? -1 : int(c[p - 1] >> (32 - kPrefixBits));
    for (int t = prev + 1; t <= top; ++t) out[t] = uint32_t(p);
    if (p == n - 1)
      for (int t = top + 1; t < kPrefixSize; ++t) out[t] = uint32_t(n);
  }
}

// Per-repetition copy of the sketches in the repetition's sorted order, so the
// search reads a candidate's id and sketch from the same position.
__global__ void table_sketch_kernel(const uint32_t* __restrict__ ids, const uint64_t* __restrict__ sk, int64_t n,
                                    int L, int M, uint64_t* __restrict__ skc) {
  const int64_t total = n * L;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t j = e / n;
    skc[e] = sk[(j % M) * n + ids[e]];
  }
}

cudaError_t gather_table_sketches(const pf_index* ix, const uint64_t* sk, uint64_t* skc, cudaStream_t s) {
  const int64_t total = ix->n * ix->L;
  const int blocks = int(std::min<int64_t>(int64_t(ix->num_sms) * 16, (total + 255) / 256));
  table_sketch_kernel<<<blocks, 256, 0, s>>>(ix->ids, sk, ix->n, ix->L, ix->M, skc);
  return cudaGetLastError();
}

cudaError_t sort_tables(pf_index* ix, const uint32_t* codes_unsorted, cudaStream_t s) {
  const int64_t n = ix->n;
  const int j_begin = 0, j_end = ix->L, nt = ix->L;
  if (nt <= 0) return cudaSuccess;
  const int ntiles = int((n + kSortTile - 1) / kSortTile);
  // tables per group: bound the temporary buffers to ~1 GiB
  int G = int(std::max<int64_t>(1, std::min<int64_t>(nt, (int64_t(1) << 30) / std::max<int64_t>(1, n * 16))));
  uint32_t *tk = nullptr, *tv = nullptr, *cnt = nullptr;
  cudaError_t e;
  if ((e = cudaMallocAsync(&tk, sizeof(uint32_t) * size_t(n) * G, s)) != cudaSuccess) return e;
  if ((e = cudaMallocAsync(&tv, sizeof(uint32_t) * size_t(n) * G, s)) != cudaSuccess) return e;
  if ((e = cudaMallocAsync(&cnt, sizeof(uint32_t) * size_t(256) * ntiles * G, s)) != cudaSuccess) return e;
  for (int j0 = j_begin; j0 < j_end && e == cudaSuccess; j0 += G) {
    const int g = std::min(G, j_end - j0);
    const uint32_t* keys0 = codes_unsorted + int64_t(j0) * n;
    uint32_t* outk = ix->codes + int64_t(j0) * n;
    uint32_t* outv = ix->ids + int64_t(j0) * n;
    // pass buffers: in -> tmp -> out -> tmp -> out
    const uint32_t* kin = keys0;
    const uint32_t* vin = nullptr;
    for (int pass = 0; pass < 4; ++pass) {
      uint32_t* ko = (pass % 2 == 0) ? tk : outk;
      uint32_t* vo = (pass % 2 == 0) ? tv : outv;
      dim3 grid(ntiles, g);
      radix_hist_kernel<<<grid, kSortThreads, 0, s>>>(kin, n, pass * 8, ntiles, cnt);
      radix_scan_kernel<<<g, 1024, 0, s>>>(cnt, ntiles);
      radix_scatter_kernel<<<grid, kSortThreads, 0, s>>>(kin, vin, ko, vo, n, pass * 8, ntiles, cnt);
      kin = ko;
      vin = vo;
    }
    prefix_kernel<<<dim3(unsigned(std::min<int64_t>(1024, (n + 255) / 256)), g), 256, 0, s>>>(
        outk, n, ix->pfx + int64_t(j0) * kPrefixSize);
    e = cudaGetLastError();
  }
  cudaFreeAsync(tk, s);
  cudaFreeAsync(tv, s);
  cudaFreeAsync(cnt, s);
  return e;
}

}  // namespace pf
