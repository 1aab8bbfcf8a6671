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

// inv[e] = blocks[e]^{-1} in precision T: in-place Gauss-Jordan elimination with
// partial (row) pivoting, the row interchanges undone as column interchanges at the
// end. One CTA per element; thread t owns columns t, t + blockDim, ... of the n x n
// matrix held row-major in shared memory, so every update is one FMA per owned
// entry with no index arithmetic in the inner loop. A zero pivot sets *status = 1.
template <class T>
__global__ void k_block_inverse(const double* __restrict__ blocks, T* __restrict__ inv, int n, int* status) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* A = (T*)sm_raw;            // [n][n] row-major
  T* fac = A + n * n;           // [n] column k before the update
  int* ipiv = (int*)(fac + n);  // [n] row interchanges
  __shared__ int piv;
  const int e = blockIdx.x;
  const double* B = blocks + (size_t)e * n * n;   // column-major
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int col = idx / n, row = idx - col * n;
    A[row * n + col] = (T)B[idx];
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x < 32) {
      T best = T(-1);
      int bi = k;
      for (int i = k + threadIdx.x; i < n; i += 32) {
        const T v = fabs(A[i * n + k]);
        if (v > best) { best = v; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) { piv = bi; ipiv[k] = bi; }
    }
    __syncthreads();
    const int p = piv;
    if (p != k)
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const T t = A[k * n + j];
        A[k * n + j] = A[p * n + j];
        A[p * n + j] = t;
      }
    __syncthreads();
    const T pv = A[k * n + k];
    if (pv == T(0) && threadIdx.x == 0) *status = 1;
    const T ip = pv != T(0) ? T(1) / pv : T(0);
    for (int i = threadIdx.x; i < n; i += blockDim.x) fac[i] = (i == k) ? T(0) : A[i * n + k];
    __syncthreads();
    // pivot row: A[k][j] *= 1/pivot, with A[k][k] := 1/pivot
    for (int j = threadIdx.x; j < n; j += blockDim.x) A[k * n + j] = (j == k ? T(1) : A[k * n + j]) * ip;
    __syncthreads();
    // other rows: A[i][j] -= fac[i] A[k][j], with column k taking -fac[i] / pivot
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const T akj = A[k * n + j];
      const bool colk = (j == k);
      for (int i = 0; i < n; ++i) {
        if (i == k) continue;
        const T aij = colk ? T(0) : A[i * n + j];
        A[i * n + j] = aij - fac[i] * akj;
      }
    }
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, last first; store column-major
  T* Iv = inv + (size_t)e * n * n;
  for (int row = threadIdx.x; row < n; row += blockDim.x)
    for (int k = n - 1; k >= 0; --k) {
      const int p = ipiv[k];
      if (p != k) {
        const T t = A[row * n + k];
        A[row * n + k] = A[row * n + p];
        A[row * n + p] = t;
      }
    }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int col = idx / n, row = idx - col * n;
    Iv[idx] = A[row * n + col];
  }
}

// shared memory of k_block_inverse<T> for block size n
template <class T> constexpr size_t block_inverse_smem(int n) {
  return (size_t)(n * n + n) * sizeof(T) + (size_t)n * sizeof(int) + 16;
}

// y_e = inv_e x_e for every element (arithmetic in T, FP64 vectors). Optional skips:
// the whole launch (*skip != 0), or element e when inst_skip[inst[e]] != 0.
template <class T>
__global__ void k_block_apply(const T* __restrict__ inv, const double* __restrict__ x, double* __restrict__ y,
                              int n, const int* skip, const int* inst, const int* inst_skip) {
  if (skip && *skip) return;
  const int e = blockIdx.x;
  if (inst_skip && inst_skip[inst[e]]) return;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* xs = (T*)sm_raw;
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

// y_e = inv_e x_e with one warp per element (n <= 32 RW): lane r holds x_e rows
// r, r + 32, ... and computes the same output rows; column c of the block is read as
// one coalesced run of n values while x_e[c] is broadcast by a warp shuffle. Skips
// as k_block_apply. 8 elements per CTA.
template <class T, int RW>
__global__ void __launch_bounds__(256) k_block_apply_warp(const T* __restrict__ inv, const double* __restrict__ x,
                                                         double* __restrict__ y, int n, int64_t E, const int* skip,
                                                         const int* inst, const int* inst_skip) {
  if (skip && *skip) return;
  const int64_t e = blockIdx.x * (int64_t)8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= E) return;
  if (inst_skip && inst_skip[inst[e]]) return;
  const double* xe = x + e * n;
  T xr[RW], acc[RW];
#pragma unroll
  for (int t = 0; t < RW; ++t) {
    const int r = lane + 32 * t;
    xr[t] = r < n ? (T)xe[r] : T(0);
    acc[t] = T(0);
  }
  const T* Iv = inv + e * n * n;
#pragma unroll
  for (int tb = 0; tb < RW; ++tb) {
    const int cn = min(32, n - 32 * tb);
#pragma unroll 4
    for (int cc = 0; cc < cn; ++cc) {
      const T xc = __shfl_sync(0xffffffffu, xr[tb], cc);
      const T* col = Iv + (size_t)(32 * tb + cc) * n;
#pragma unroll
      for (int t = 0; t < RW; ++t) {
        const int r = lane + 32 * t;
        if (r < n) acc[t] = fma(col[r], xc, acc[t]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < RW; ++t) {
    const int r = lane + 32 * t;
    if (r < n) y[e * n + r] = (double)acc[t];
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
