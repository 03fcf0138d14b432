// Pseudo-random cross-polytope hashing (Sec. 4.3: the family that applies the
// fast Hadamard transform three times, after Andoni et al. 2015).
//
// A function of repetition j maps the normalised point x, zero-padded to
// d'' = 2^ceil(log2 d) coordinates, to y = H D3 H D2 H D1 x (H the unnormalised
// Walsh-Hadamard matrix, D_r random +-1 diagonals); its l-bit value is the index
// of the largest |y_c| (first c on ties) and the sign of y_c.  A table's code
// concatenates floor(32 / l) functions, function 0 in the most significant bits.
//
// One warp per point: lane t holds V = max(1, d''/32) consecutive coordinates
// t*V .. t*V + V - 1 in registers; the butterfly passes h < V run inside a lane,
// the passes h >= V pair lane t with lane t ^ (h / V) through shuffles.  Two
// functions are transformed together, so that the shuffle chain of one hides
// the latency of the other's.  Each
// pass is the same pairwise operation (a, b) -> (a + b, a - b), lower index
// first, as the float64 definition, so a recomputation in float64 in the same
// order gives the definition's values bit for bit.  The transform runs in
// float32; a function whose top two |y| lie within the float32 error bound of
// each other (params.cpp: fht_bands), or whose top |y| lies within it of zero,
// is recomputed in float64 by the same warp, so every code equals the float64
// definition.
#include "pf_internal.h"

namespace pf {

namespace {

constexpr int kFhtWarps = 8;  // warps (points) per CTA

struct FhtArgs {
  const float* x32;
  int64_t npts;
  int d, d_pad, n2, L, fns, ell, words;
  const uint32_t* signs;  // [L][fns][3][words]
  float gap, sign;        // float64 recheck bands
  uint32_t* codes;
  int64_t cj, cp;
};

// v <- D_r v for the lane's V coordinates (a set bit means -1)
template <int V, class T>
__device__ __forceinline__ void apply_signs(T (&v)[V], uint32_t bits) {
#pragma unroll
  for (int k = 0; k < V; ++k)
    if ((bits >> k) & 1u) v[k] = -v[k];
}

// One pass of H over the warp's values (value i = lane * V + k).
template <int V, class T>
__device__ __forceinline__ void wht_pass(T (&v)[V], int lane, int n2) {
#pragma unroll
  for (int h = 1; h < V; h *= 2) {
#pragma unroll
    for (int k = 0; k < V; ++k)
      if (!(k & h)) {
        const T a = v[k], b = v[k + h];
        v[k] = a + b;
        v[k + h] = a - b;
      }
  }
  const int lanes = n2 / V;  // lanes that hold coordinates (a power of two, <= 32)
#pragma unroll
  for (int t = 1; t < 32; t *= 2) {
    if (t >= lanes) break;  // uniform in the warp
    const bool upper = lane & t;
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const T p = __shfl_xor_sync(0xffffffffu, v[k], t);
      v[k] = upper ? p - v[k] : v[k] + p;  // the upper element of a pair takes (lower - upper)
    }
  }
}

// The float32 transform of two functions at once (independent chains, so the
// latency of one's shuffles hides behind the other's), signs given.
template <int V>
__device__ __forceinline__ void transform2(float (&a)[V], float (&b)[V], const uint32_t (&sa)[3],
                                           const uint32_t (&sb)[3], int lane, int n2) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    apply_signs<V>(a, sa[r]);
    apply_signs<V>(b, sb[r]);
#pragma unroll
    for (int h = 1; h < V; h *= 2) {
#pragma unroll
      for (int k = 0; k < V; ++k)
        if (!(k & h)) {
          const float a0 = a[k], a1 = a[k + h], b0 = b[k], b1 = b[k + h];
          a[k] = a0 + a1;
          a[k + h] = a0 - a1;
          b[k] = b0 + b1;
          b[k + h] = b0 - b1;
        }
    }
    const int lanes = n2 / V;
#pragma unroll
    for (int t = 1; t < 32; t *= 2) {
      if (t >= lanes) break;  // uniform in the warp
      const bool upper = lane & t;
#pragma unroll
      for (int k = 0; k < V; ++k) {
        const float pa = __shfl_xor_sync(0xffffffffu, a[k], t);
        const float pb = __shfl_xor_sync(0xffffffffu, b[k], t);
        a[k] = upper ? pa - a[k] : a[k] + pa;
        b[k] = upper ? pb - b[k] : b[k] + pb;
      }
    }
  }
}

// The warp's largest |y| (a1, at index i1 with sign n1: first index on ties)
// and the runner-up a2, of the lane's V values of a transform.
struct Top2 {
  float a1, a2;
  uint32_t in;  // index | sign << 31
};

template <int V>
__device__ __forceinline__ Top2 lane_top2(const float (&v)[V], int lane, bool live) {
  Top2 t;
  t.a1 = -1.f;
  t.a2 = -1.f;
  t.in = 0u;
#pragma unroll
  for (int k = 0; k < V; ++k) {
    const float a = fabsf(v[k]);
    if (!live) continue;
    if (a > t.a1) {
      t.a2 = t.a1;
      t.a1 = a;
      t.in = uint32_t(lane * V + k) | (v[k] < 0.f ? 0x80000000u : 0u);
    } else if (a > t.a2) {
      t.a2 = a;
    }
  }
  return t;
}

__device__ __forceinline__ void merge_top2(Top2& t, int off) {
  const float o1 = __shfl_xor_sync(0xffffffffu, t.a1, off);
  const float o2 = __shfl_xor_sync(0xffffffffu, t.a2, off);
  const uint32_t oi = __shfl_xor_sync(0xffffffffu, t.in, off);
  if (o1 > t.a1 || (o1 == t.a1 && (oi & 0x7FFFFFFFu) < (t.in & 0x7FFFFFFFu))) {
    t.a2 = fmaxf(t.a1, o2);
    t.a1 = o1;
    t.in = oi;
  } else {
    t.a2 = fmaxf(t.a2, o1);
  }
}

template <int V>
__device__ __forceinline__ uint32_t lane_sign_bits(const FhtArgs& A, int j, int f, int r, int lane) {
  const uint32_t w = __ldg(A.signs + ((size_t(j) * A.fns + f) * 3 + r) * A.words + (lane * V) / 32);
  return w >> ((lane * V) & 31);
}

// Value (sign << (l - 1)) | c of the largest |y_c| over the warp, first c on
// ties, in float64 (no band: this is the definition).
template <int V>
__device__ uint32_t value64(const FhtArgs& A, const float (&x)[V], int j, int f, int lane) {
  double v[V];
#pragma unroll
  for (int k = 0; k < V; ++k) v[k] = double(x[k]);
  for (int r = 0; r < 3; ++r) {
    apply_signs<V>(v, lane_sign_bits<V>(A, j, f, r, lane));
    wht_pass<V>(v, lane, A.n2);
  }
  double best = -1.0;
  int idx = 0;
  bool neg = false;
  const bool live = lane * V < A.n2;
#pragma unroll
  for (int k = 0; k < V; ++k) {
    const double a = fabs(v[k]);
    if (live && a > best) {
      best = a;
      idx = lane * V + k;
      neg = v[k] < 0.0;
    }
  }
  for (int t = 16; t >= 1; t >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, t);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, t);
    const int on = __shfl_xor_sync(0xffffffffu, int(neg), t);
    if (ob > best || (ob == best && oi < idx)) {
      best = ob;
      idx = oi;
      neg = on != 0;
    }
  }
  return (uint32_t(neg) << (A.ell - 1)) | uint32_t(idx);
}

template <int V>
__global__ void __launch_bounds__(32 * kFhtWarps) hash_fht_kernel(FhtArgs A) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = int64_t(blockIdx.x) * kFhtWarps + (threadIdx.x >> 5);
  const int64_t nwarps = int64_t(gridDim.x) * kFhtWarps;
  const bool live = lane * V < A.n2;  // lanes past d'' (d'' < 32) take no part in the argmax
  for (int64_t p = warp0; p < A.npts; p += nwarps) {
    float x[V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const int i = lane * V + k;
      x[k] = i < A.d ? __ldg(A.x32 + p * A.d_pad + i) : 0.f;
    }
    for (int j = 0; j < A.L; ++j) {
      uint32_t code = 0;
      // two functions at a time (the second a copy of the first when fns is odd)
      for (int f = 0; f < A.fns; f += 2) {
        const int f2 = f + 1 < A.fns ? f + 1 : f;
        uint32_t sa[3], sb[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          sa[r] = lane_sign_bits<V>(A, j, f, r, lane);
          sb[r] = lane_sign_bits<V>(A, j, f2, r, lane);
        }
        float va[V], vb[V];
#pragma unroll
        for (int k = 0; k < V; ++k) va[k] = vb[k] = x[k];
        transform2<V>(va, vb, sa, sb, lane, A.n2);
        Top2 ta = lane_top2<V>(va, lane, live), tb = lane_top2<V>(vb, lane, live);
#pragma unroll
        for (int t = 16; t >= 1; t >>= 1) {
          merge_top2(ta, t);
          merge_top2(tb, t);
        }
        const Top2 tt[2] = {ta, tb};
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int fu = u == 0 ? f : f2;
          if (u == 1 && f2 == f) break;
          uint32_t value;
          if (tt[u].a1 - tt[u].a2 < A.gap || tt[u].a1 <= A.sign)  // warp-uniform: every lane holds the reduced values
            value = value64<V>(A, x, j, fu, lane);
          else
            value = ((tt[u].in >> 31) << (A.ell - 1)) | (tt[u].in & 0x7FFFFFFFu);
          code |= value << (32 - A.ell * (fu + 1));
        }
      }
      if (lane == 0) A.codes[int64_t(j) * A.cj + p * A.cp] = code;
    }
  }
}

}  // namespace

cudaError_t launch_hash_fht(const pf_index* ix, const float* x32, int64_t npts, uint32_t* codes, int64_t cj,
                            int64_t cp, cudaStream_t s) {
  if (npts <= 0 || ix->L <= 0) return cudaSuccess;
  FhtArgs A;
  A.x32 = x32;
  A.npts = npts;
  A.d = ix->d;
  A.d_pad = ix->lay.d_pad;
  A.n2 = ix->lay.fht_n;
  A.L = ix->L;
  A.fns = ix->lay.fns;
  A.ell = ix->lay.ell;
  A.words = ix->lay.fht_words;
  A.signs = ix->fht_signs;
  A.gap = ix->fht_gap;
  A.sign = ix->fht_sign;
  A.codes = codes;
  A.cj = cj;
  A.cp = cp;
  const int64_t blocks64 = (npts + kFhtWarps - 1) / kFhtWarps;
  const int blocks = int(blocks64 < 65536 * 16 ? blocks64 : 65536 * 16);
  const dim3 grid(blocks), block(32 * kFhtWarps);
  switch (A.n2 <= 32 ? 1 : A.n2 / 32) {
    case 1: hash_fht_kernel<1><<<grid, block, 0, s>>>(A); break;
    case 2: hash_fht_kernel<2><<<grid, block, 0, s>>>(A); break;
    case 4: hash_fht_kernel<4><<<grid, block, 0, s>>>(A); break;
    case 8: hash_fht_kernel<8><<<grid, block, 0, s>>>(A); break;
    case 16: hash_fht_kernel<16><<<grid, block, 0, s>>>(A); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace pf
