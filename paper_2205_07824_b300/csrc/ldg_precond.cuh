// Block-Jacobi preconditioner of the Newton-GMRES solve: the exact element
// diagonal blocks dR_K/du_K of the Jacobian, inverted per element.
//
// Blocks are extracted in FP64 storage (column-major per element, n = n_cu * n_pe),
// inverted by Gauss-Jordan elimination with partial pivoting in FP32 (the
// preconditioner only has to be a good approximate inverse; the Krylov solve and
// the Newton residual stay FP64), and applied as one dense block-vector product
// per element.
#pragma once
#include <cuda_runtime.h>

namespace ldg {

// inv[e] = blocks[e]^{-1} in precision T. One CTA per element; smem holds the
// augmented [n x 2n] matrix (row-major) plus n pivot factors. A zero pivot sets *status = 1.
template <class T>
__global__ void k_block_inverse(const double* __restrict__ blocks, T* __restrict__ inv, int n, int* status) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* A = (T*)sm_raw;            // [n][2n]
  T* fac = A + 2 * n * n;       // [n]
  __shared__ int piv;
  const int e = blockIdx.x, w2 = 2 * n;
  const double* B = blocks + (size_t)e * n * n;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int col = idx / n, row = idx - col * n;
    A[row * w2 + col] = (T)B[idx];
    A[col * w2 + n + row] = (col == row) ? T(1) : T(0);
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x < 32) {
      T best = T(-1);
      int bi = k;
      for (int i = k + threadIdx.x; i < n; i += 32) {
        const T v = fabs(A[i * w2 + k]);
        if (v > best) { best = v; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) piv = bi;
    }
    __syncthreads();
    const int p = piv;
    if (p != k)
      for (int j = threadIdx.x; j < w2; j += blockDim.x) {
        const T t = A[k * w2 + j];
        A[k * w2 + j] = A[p * w2 + j];
        A[p * w2 + j] = t;
      }
    __syncthreads();
    const T pv = A[k * w2 + k];
    if (pv == T(0) && threadIdx.x == 0) *status = 1;
    const T ip = pv != T(0) ? T(1) / pv : T(0);
    __syncthreads();
    for (int j = threadIdx.x; j < w2; j += blockDim.x) A[k * w2 + j] *= ip;
    for (int i = threadIdx.x; i < n; i += blockDim.x) fac[i] = (i == k) ? T(0) : A[i * w2 + k];
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * w2; idx += blockDim.x) {
      const int i = idx / w2, j = idx - i * w2;
      if (i != k) A[idx] -= fac[i] * A[k * w2 + j];
    }
    __syncthreads();
  }
  T* Iv = inv + (size_t)e * n * n;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int col = idx / n, row = idx - col * n;
    Iv[idx] = A[row * w2 + n + col];   // column-major
  }
}

// y_e = inv_e x_e for every element (arithmetic in T, FP64 vectors).
template <class T>
__global__ void k_block_apply(const T* __restrict__ inv, const double* __restrict__ x, double* __restrict__ y,
                              int n, const int* skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* xs = (T*)sm_raw;
  const int e = blockIdx.x;
  const double* xe = x + (size_t)e * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) xs[i] = (T)xe[i];
  __syncthreads();
  const T* Iv = inv + (size_t)e * n * n;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    T s = T(0);
    for (int c = 0; c < n; ++c) s = fma(Iv[(size_t)c * n + r], xs[c], s);
    y[(size_t)e * n + r] = (double)s;
  }
}

// probe[e][l'] = 1 where colour[e] == colour and l' == l, else 0
__global__ void k_probe(double* probe, const int* colour, int c, int l, int nloc, int64_t E) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= E * nloc) return;
  const int64_t e = i / nloc;
  const int lp = (int)(i - e * nloc);
  probe[i] = (colour[e] == c && lp == l) ? 1.0 : 0.0;
}

// blocks[e][l][:] = jp[e][:] for the elements of colour c (column l of their diagonal block)
__global__ void k_extract(const double* jp, const int* colour, int c, int l, int nloc, int64_t E, double* blocks) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= E * nloc) return;
  const int64_t e = i / nloc;
  if (colour[e] != c) return;
  const int row = (int)(i - e * nloc);
  blocks[((size_t)e * nloc + l) * nloc + row] = jp[i];
}

}  // namespace ldg
