// Per-element MLP preconditioner: inference and training kernels.
//
// Network (shared by all elements): x (2n) -> relu(W1 x + b1) (h) -> relu(W2 . + b2) (h)
// -> W3 . + b3 + Ws x_v (n), n = n_cu * n_pe, with a learned linear skip map Ws acting
// on the scaled vector block x_v. Its input is the element block scaled to unit
// 2-norm followed by the element's state block, x = [v_K / ||v_K||, u_K], and the
// output is rescaled: M(v)_K = ||v_K|| net(v_K / ||v_K||, u_K), positively
// homogeneous in v. Trained by mean-squared error with Adam; FP32 master weights,
// BF16 weights for inference, FP32 arithmetic. Parameter order: W1 [h][2n], b1,
// W2 [h][h], b2, W3 [n][h], b3, Ws [n][n].
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace ldg {

__device__ __forceinline__ float tof(float x) { return x; }
__device__ __forceinline__ float tof(__nv_bfloat16 x) { return __bfloat162float(x); }

// C[M][N] (+)= op(A) op(B) + bias[n] (relu optional), FP32 accumulate, row-major;
// acc adds the product to the existing C.
// op(A) = A (M x K, lda) or A^T (A stored K x M); op(B) = B (K x N, ldb) or B^T
// (B stored N x K). 64 x 64 tiles, 16-deep k steps, 4 x 4 outputs per thread.
template <bool TA, bool TB, class TBt>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                             const TBt* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                             const float* __restrict__ bias, int relu, const int* skip, int acc_c) {
  if (skip && *skip) return;
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int l = threadIdx.x; l < 1024; l += 256) {
      int mm, kk;
      if (TA) { mm = l & 63; kk = l >> 6; } else { kk = l & 15; mm = l >> 4; }
      const int m = m0 + mm, k = k0 + kk;
      float a = 0.f;
      if (m < M && k < K) a = TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
      As[kk][mm] = a;
      int nn, kb;
      if (TB) { kb = l & 15; nn = l >> 4; } else { nn = l & 63; kb = l >> 6; }
      const int n = n0 + nn, kb2 = k0 + kb;
      float b = 0.f;
      if (n < N && kb2 < K) b = TB ? tof(B[(size_t)n * ldb + kb2]) : tof(B[(size_t)kb2 * ldb + n]);
      Bs[kb][nn] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
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
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j];
      if (acc_c) v += C[(size_t)m * ldc + n];
      if (bias) v += bias[n];
      if (relu) v = fmaxf(v, 0.f);
      C[(size_t)m * ldc + n] = v;
    }
  }
}

// Rows r < rows: Xn[r] = [X[src] / ||X[src]||, S[src]] (width 2n), Tn[r] = T[src]
// scaled by the same norm (if T), mask[r] = (norm > tiny), norms[r] = norm;
// *count += number of valid rows. One warp per row; src = idx[r] (idx == null: r).
// With Xbf the row goes out in BF16 (the tensor-core operand) instead of FP32 Xn.
// The norm is formed in FP32: the network's inputs are FP32 or BF16 anyway, and FP64
// square roots and divisions would occupy this part's FP64 pipe for most of the kernel
// (a row whose entries are all below about 1e-19 in magnitude reads as zero).
__global__ void k_mlp_prep(const double* __restrict__ X, const double* __restrict__ T, const double* __restrict__ S,
                           const int* __restrict__ idx, int64_t rows, int n, float* __restrict__ Xn,
                           __nv_bfloat16* __restrict__ Xbf, float* __restrict__ Tn, float* __restrict__ mask,
                           double* __restrict__ norms, int* count, const int* skip) {
  if (skip && *skip) return;
  const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  const int64_t src = idx ? (int64_t)idx[r] : r;
  const double* x = X + src * n;
  float s = 0.f;
  for (int i = lane; i < n; i += 32) {
    const float xi = (float)x[i];
    s = fmaf(xi, xi, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const float nrm = sqrtf(s);
  const bool ok = nrm > 1e-30f;
  const float inv = ok ? 1.f / nrm : 0.f;
  for (int i = lane; i < n; i += 32) {
    const float a = (float)x[i] * inv, b = (float)S[src * n + i];
    if (Xbf) {
      Xbf[r * 2 * n + i] = __float2bfloat16(a);
      Xbf[r * 2 * n + n + i] = __float2bfloat16(b);
    } else {
      Xn[r * 2 * n + i] = a;
      Xn[r * 2 * n + n + i] = b;
    }
    if (T) Tn[r * n + i] = (float)T[src * n + i] * inv;
  }
  if (lane == 0) {
    if (mask) mask[r] = ok ? 1.f : 0.f;
    if (norms) norms[r] = (double)nrm;
    if (count && ok) atomicAdd(count, 1);
  }
}

// dY = 2 mask (Y - Tn) / count, loss += sum mask |Y - Tn|^2 / count (per-block partials)
__global__ void k_mlp_dloss(const float* __restrict__ Y, const float* __restrict__ Tn, const float* __restrict__ mask,
                            int64_t rows, int n, const int* count, float* __restrict__ dY, double* loss) {
  const int64_t total = rows * n;
  const float c = (float)max(*count, 1);
  double part = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const float mk = mask[i / n];
    const float e = (Y[i] - Tn[i]) * mk;
    dY[i] = 2.f * e / c;
    part += (double)e * e;
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, part / c);
}

// dH *= (H > 0)
__global__ void k_relu_back(float* __restrict__ dH, const float* __restrict__ H, int64_t total) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    if (!(H[i] > 0.f)) dH[i] = 0.f;
}

// out[c] = sum_r D[r][c] (one block per column, fixed summation order)
__global__ void k_colsum(const float* __restrict__ D, int64_t rows, int cols, float* __restrict__ out) {
  __shared__ float red[256];
  const int c = blockIdx.x;
  float s = 0.f;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) s += D[r * cols + c];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = red[0];
}

// Adam (Kingma & Ba 2015), step t >= 1
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, int t) {
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void k_to_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16(src[i]);
}

// Normal equations of the least-squares skip map: dst (FP64, n x n) = G (FP32) with
// a relative ridge `reg` * trace(G) / n added to the diagonal (one block).
__global__ void k_gram_to_f64(const float* __restrict__ G, int n, double reg, double* __restrict__ dst) {
  __shared__ double tr;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += G[i * n + i];
    tr = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n * n; i += blockDim.x)
    dst[i] = (double)G[i] + ((i / n == i % n) ? reg * tr / n : 0.0);
}
__global__ void k_f64_to_f32(const double* __restrict__ src, float* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

// z[r][i] = norms[r] * Y[r][i]
// z[r] = norms[r] Y[r], one warp per row (the product in FP32, the precision of Y)
__global__ void k_mlp_unprep(const float* __restrict__ Y, const double* __restrict__ norms, int64_t rows, int n,
                             double* __restrict__ z, const int* skip) {
  if (skip && *skip) return;
  const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  const float nr = (float)norms[r];
  for (int i = lane; i < n; i += 32) z[r * n + i] = (double)(nr * Y[r * n + i]);
}

}  // namespace ldg
