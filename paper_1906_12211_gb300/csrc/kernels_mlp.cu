// Learned start depth: a 2-layer perceptron that predicts, from a query's
// normalised vector and its first 64-bit sketch, the prefix length at which
// the plain depth schedule (Sec. 4.1: K, K-1, ...) stops.  The search starts a
// few bits above a high quantile of that prediction: the first round takes the
// block at the start depth at once (its sketch threshold refreshed every 32
// repetitions), later rounds drop one bit each.  The stop test of Lemma 1 still
// decides termination, so the recall guarantee is unchanged.
//
//   x = [q (d_pad floats), sketch-0 bits as +-1 (64)]         F_in = d_pad + 64
//   h = relu(W1 x + b1)                                        H = 256
//   z = W2 h + b2                                              C = K + 1 classes
//   loss = mean over the batch of -log softmax(z)[y]           y = stop depth
//
// Training: float32 master weights, forward / backward with the tiled GEMM
// and elementwise kernels below, Adam.  Inference: bfloat16 copies of W1 and
// W2 with float32 accumulation, one warp per query; the start depth is
// min(K, q + margin) with q the smallest d with P(stop depth > d) <= tail under
// the predicted distribution (the index's start rule: 0.05 and 0 by default).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "pf_internal.h"

namespace pf {

namespace {

// C[M][N] = op(A)[M][K] * op(B)[K][N] (+ C if accumulate); op(A) = A or A^T
// (A stored [K][M]), same for B.  64x64 tile per CTA, 256 threads, 4x4 each.
constexpr int kG = 64, kGK = 16;

__global__ void __launch_bounds__(256) gemm_f32_kernel(int M, int N, int K, const float* __restrict__ A, int lda,
                                                       bool ta, const float* __restrict__ B, int ldb, bool tb,
                                                       float* __restrict__ C, int ldc, bool accumulate) {
  __shared__ float As[kGK][kG + 1];
  __shared__ float Bs[kGK][kG + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * kG, n0 = blockIdx.x * kG;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += kGK) {
    for (int e = threadIdx.x; e < kGK * kG; e += 256) {
      const int kk = e / kG, mm = e % kG;
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < K) ? (ta ? A[size_t(k) * lda + m] : A[size_t(m) * lda + k]) : 0.f;
      const int n = n0 + mm;
      Bs[kk][mm] = (n < N && k < K) ? (tb ? B[size_t(n) * ldb + k] : B[size_t(k) * ldb + n]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
      if (m < M && n < N) C[size_t(m) * ldc + n] = accumulate ? C[size_t(m) * ldc + n] + acc[i][j] : acc[i][j];
    }
}

cudaError_t gemm(int M, int N, int K, const float* A, int lda, bool ta, const float* B, int ldb, bool tb, float* C,
                 int ldc, bool accumulate, cudaStream_t s) {
  dim3 grid((N + kG - 1) / kG, (M + kG - 1) / kG);
  gemm_f32_kernel<<<grid, 256, 0, s>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, accumulate);
  return cudaGetLastError();
}

__global__ void bias_relu_kernel(float* __restrict__ h, const float* __restrict__ b, int rows, int cols) {
  const int64_t total = int64_t(rows) * cols;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x)
    h[e] = fmaxf(h[e] + b[e % cols], 0.f);
}

// softmax cross-entropy per row (one warp per row): adds b2, accumulates the
// mean loss, writes dZ = (softmax - onehot) / rows
__global__ void softmax_ce_kernel(const float* __restrict__ z, const float* __restrict__ b, const int32_t* __restrict__ y,
                                  int rows, int C, float* __restrict__ dz, float* __restrict__ loss) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= rows) return;
  float mx = -INFINITY;
  for (int c = lane; c < C; c += 32) mx = fmaxf(mx, z[size_t(r) * C + c] + b[c]);
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  float se = 0.f;
  for (int c = lane; c < C; c += 32) se += expf(z[size_t(r) * C + c] + b[c] - mx);
  for (int o = 16; o; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
  const int yr = y[r];
  for (int c = lane; c < C; c += 32) {
    const float p = expf(z[size_t(r) * C + c] + b[c] - mx) / se;
    dz[size_t(r) * C + c] = (p - (c == yr ? 1.f : 0.f)) / float(rows);
  }
  if (lane == 0) {
    const float ly = -(z[size_t(r) * C + yr] + b[yr] - mx - logf(se));
    atomicAdd(loss, ly / float(rows));
  }
}

__global__ void relu_backward_kernel(float* __restrict__ dh, const float* __restrict__ h, int64_t total) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x)
    if (h[e] <= 0.f) dh[e] = 0.f;
}

// out[c] = sum over rows of a[r][c]
__global__ void colsum_kernel(const float* __restrict__ a, int rows, int cols, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += a[size_t(r) * cols + c];
  out[c] = s;
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t count, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// features of Q queries: normalised vector (d_pad) then sketch-0 bits as +-1
__global__ void features_kernel(const float* __restrict__ qx, const uint64_t* __restrict__ qsk, int Q, int d_pad, int M,
                                float* __restrict__ x) {
  const int F = d_pad + 64;
  const int64_t total = int64_t(Q) * F;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t q = e / F;
    const int i = int(e % F);
    x[e] = i < d_pad ? qx[q * d_pad + i] : (((qsk[q * M] >> (i - d_pad)) & 1ull) ? 1.f : -1.f);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t count) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

// Inference for a tile of kPredQ queries per CTA of 256 threads (= hidden
// units): thread u accumulates its hidden unit for all queries of the tile
// (the bfloat16 first layer is stored transposed, [F][H], so one feature step
// is one coalesced row shared by the tile); float32 accumulation.  The start
// depth is min(C - 1, q + margin), q the smallest d with P(stop depth > d) <= tail.
constexpr int kPredQ = 16;
__global__ void __launch_bounds__(kMlpHidden) predict_kernel(const float* __restrict__ qx,
                                                             const uint64_t* __restrict__ qsk, int Q, int d_pad,
                                                             int M, const __nv_bfloat16* __restrict__ W1t,
                                                             const float* __restrict__ b1,
                                                             const __nv_bfloat16* __restrict__ W2,
                                                             const float* __restrict__ b2, int C, float tail,
                                                             int margin, int32_t* __restrict__ start) {
  // xs holds the features, then (once the hidden layer is done) the output
  // layer's C <= 33 rows of bfloat16 weights
  __shared__ __align__(16) float xs[kPredQ][kMaxD + 64];
  __shared__ float hs[kPredQ][kMlpHidden];
  __shared__ float zs[kPredQ][64];
  __nv_bfloat16* w2s = reinterpret_cast<__nv_bfloat16*>(&xs[0][0]);
  const int tid = threadIdx.x;
  const int q0 = blockIdx.x * kPredQ;
  const int nq = min(kPredQ, Q - q0);
  const int F = d_pad + 64;
  for (int e = tid; e < nq * F; e += kMlpHidden) {
    const int t = e / F, i = e % F;
    const int64_t q = q0 + t;
    xs[t][i] = i < d_pad ? qx[q * d_pad + i] : (((qsk[q * M] >> (i - d_pad)) & 1ull) ? 1.f : -1.f);
  }
  __syncthreads();
  const int u = tid;
  float acc[kPredQ];
#pragma unroll
  for (int t = 0; t < kPredQ; ++t) acc[t] = b1[u];
  // F is a multiple of 16 (d_pad + 64): eight weight loads in flight per step
  for (int i0 = 0; i0 < F; i0 += 8) {
    float w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) w[j] = __bfloat162float(W1t[size_t(i0 + j) * kMlpHidden + u]);
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int t = 0; t < kPredQ; ++t) acc[t] = fmaf(w[j], xs[t][i0 + j], acc[t]);
  }
#pragma unroll
  for (int t = 0; t < kPredQ; ++t) hs[t][u] = fmaxf(acc[t], 0.f);
  __syncthreads();
  for (int e = tid; e < C * kMlpHidden; e += kMlpHidden) w2s[e] = W2[e];
  __syncthreads();
  for (int e = tid; e < nq * C; e += kMlpHidden) {
    const int t = e / C, c = e % C;
    const __nv_bfloat16* row = w2s + c * kMlpHidden;
    float a = b2[c];
    for (int h = 0; h < kMlpHidden; ++h) a = fmaf(__bfloat162float(row[h]), hs[t][h], a);
    zs[t][c] = a;
  }
  __syncthreads();
  if (tid < nq) {
    const float* z = zs[tid];
    float mx = -INFINITY;
    for (int c = 0; c < C; ++c) mx = fmaxf(mx, z[c]);
    float se = 0.f;
    for (int c = 0; c < C; ++c) se += expf(z[c] - mx);
    // P(stop depth > d) = sum over c > d; scan from the top
    float above = 0.f;
    int dsel = C - 1;
    for (int d = C - 1; d >= 0; --d) {
      if (above > tail * se) break;
      dsel = d;
      above += expf(z[d] - mx);
    }
    start[q0 + tid] = min(C - 1, dsel + margin);
  }
}

__global__ void gather_rows_kernel(const float* __restrict__ src, const int32_t* __restrict__ idx, int rows, int cols,
                                   float* __restrict__ dst) {
  const int64_t total = int64_t(rows) * cols;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x)
    dst[e] = src[int64_t(idx[e / cols]) * cols + e % cols];
}

}  // namespace

cudaError_t gather_rows(const float* src, const int32_t* idx, int rows, int cols, float* dst, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  gather_rows_kernel<<<512, 256, 0, s>>>(src, idx, rows, cols, dst);
  return cudaGetLastError();
}

cudaError_t mlp_features(const float* qx, const uint64_t* qsk, int Q, int d_pad, int M, float* x, cudaStream_t s) {
  if (Q <= 0) return cudaSuccess;
  features_kernel<<<1024, 256, 0, s>>>(qx, qsk, Q, d_pad, M, x);
  return cudaGetLastError();
}

// loss and gradients of the mean cross-entropy over a batch (all device
// pointers); scratch: h [B][H], z [B][C], dz [B][C], dh [B][H]
cudaError_t mlp_forward_backward(const float* X, const int32_t* y, int B, int F, int H, int C, const float* W1,
                                 const float* b1, const float* W2, const float* b2, float* loss, float* dW1,
                                 float* db1, float* dW2, float* db2, float* h, float* z, float* dz, float* dh,
                                 cudaStream_t s) {
  cudaError_t e;
  if ((e = gemm(B, H, F, X, F, false, W1, F, true, h, H, false, s)) != cudaSuccess) return e;  // X W1^T
  bias_relu_kernel<<<256, 256, 0, s>>>(h, b1, B, H);
  if ((e = gemm(B, C, H, h, H, false, W2, H, true, z, C, false, s)) != cudaSuccess) return e;  // h W2^T
  if ((e = cudaMemsetAsync(loss, 0, sizeof(float), s)) != cudaSuccess) return e;
  softmax_ce_kernel<<<(B + 3) / 4, 128, 0, s>>>(z, b2, y, B, C, dz, loss);
  if ((e = gemm(C, H, B, dz, C, true, h, H, false, dW2, H, false, s)) != cudaSuccess) return e;  // dz^T h
  colsum_kernel<<<(C + 127) / 128, 128, 0, s>>>(dz, B, C, db2);
  if ((e = gemm(B, H, C, dz, C, false, W2, H, false, dh, H, false, s)) != cudaSuccess) return e;  // dz W2
  relu_backward_kernel<<<256, 256, 0, s>>>(dh, h, int64_t(B) * H);
  if ((e = gemm(H, F, B, dh, H, true, X, F, false, dW1, F, false, s)) != cudaSuccess) return e;  // dh^T X
  colsum_kernel<<<(H + 127) / 128, 128, 0, s>>>(dh, B, H, db1);
  return cudaGetLastError();
}

cudaError_t adam_step(float* w, const float* g, float* m, float* v, int64_t count, float lr, int t, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, float(t)), c2 = 1.f - std::pow(b2, float(t));
  adam_kernel<<<256, 256, 0, s>>>(w, g, m, v, count, lr, b1, b2, 1e-8f, c1, c2);
  return cudaGetLastError();
}

__global__ void to_bf16_transposed_kernel(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int rows,
                                          int cols) {
  const int64_t count = int64_t(rows) * cols;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < count; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = e / cols, c = e % cols;
    b[c * rows + r] = __float2bfloat16_rn(a[e]);
  }
}

// b[c][r] = bfloat16(a[r][c]) for a [rows][cols]
cudaError_t to_bf16_transposed(const float* a, __nv_bfloat16* b, int rows, int cols, cudaStream_t s) {
  to_bf16_transposed_kernel<<<256, 256, 0, s>>>(a, b, rows, cols);
  return cudaGetLastError();
}

cudaError_t to_bf16(const float* a, __nv_bfloat16* b, int64_t count, cudaStream_t s) {
  to_bf16_kernel<<<256, 256, 0, s>>>(a, b, count);
  return cudaGetLastError();
}

cudaError_t mlp_predict(const float* qx, const uint64_t* qsk, int Q, int d_pad, int M, const __nv_bfloat16* W1t,
                        const float* b1, const __nv_bfloat16* W2, const float* b2, int C, float tail, int margin,
                        int32_t* start, cudaStream_t s) {
  if (Q <= 0) return cudaSuccess;
  predict_kernel<<<(Q + kPredQ - 1) / kPredQ, kMlpHidden, 0, s>>>(qx, qsk, Q, d_pad, M, W1t, b1, W2, b2, C, tail,
                                                                  margin, start);
  return cudaGetLastError();
}

}  // namespace pf
