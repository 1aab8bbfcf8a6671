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

#include <type_traits>

namespace ldg {

// inv[e] = blocks[e]^{-1} in precision T: in-place Gauss-Jordan elimination with
// partial (row) pivoting, the row interchanges undone as column interchanges at the
// end. One CTA per element, the n x n matrix row-major in shared memory; in each
// elimination step thread t updates column t mod n in every (blockDim / n)-th row,
// consecutive threads on consecutive columns. A zero pivot sets *status = 1.
template <class T>
__global__ void k_block_inverse(const double* __restrict__ blocks, T* __restrict__ inv, int n, int* status) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* A = (T*)sm_raw;            // [n][n] row-major
  T* fac = A + n * n;           // [n] column k before the update
  int* ipiv = (int*)(fac + n);  // [n] row interchanges
  __shared__ int piv;
  const int e = blockIdx.x;
  const double* B = blocks + (size_t)e * n * n;   // column-major
  // elimination mapping: thread t updates column jc = t mod n in rows rg, rg + ng, ...
  const int ng = max(1, (int)blockDim.x / n);
  const int jc = n <= (int)blockDim.x ? ((int)threadIdx.x < ng * n ? (int)threadIdx.x % n : n) : (int)threadIdx.x;
  const int rg = n <= (int)blockDim.x ? (int)threadIdx.x / n : 0;
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
    // (row k is not written here, so its entries are read unchanged)
    // (blocks wider than the CTA: each thread takes columns t, t + blockDim, ... in all rows)
    for (int j = jc; j < n; j += (n <= (int)blockDim.x ? n : (int)blockDim.x)) {
      const T akj = A[k * n + j];
      const bool colk = (j == k);
      for (int i = rg; i < n; i += ng) {
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

// |x| as an integer with the same order as the magnitudes (IEEE bit pattern without
// the sign); NaN maps to -1
__device__ __forceinline__ int abs_key(float x) {
  const int b = __float_as_int(x) & 0x7fffffff;
  return b > 0x7f800000 ? -1 : b;
}
__device__ __forceinline__ long long abs_key(double x) {
  const long long b = __double_as_longlong(x) & 0x7fffffffffffffffLL;
  return b > 0x7ff0000000000000LL ? -1LL : b;
}

// f(integral_constant<int, I>) for I = I0 .. I1 - 1, in order
template <int I0, int I1, class F> __device__ __forceinline__ void unrolled_for(F& f) {
  if constexpr (I0 < I1) {
    f(std::integral_constant<int, I0>());
    unrolled_for<I0 + 1, I1>(f);
  }
}

// The same Gauss-Jordan inversion with partial pivoting for a compile-time block size
// N (a multiple of CPT, N <= 128; NT threads) with the matrix held in registers:
// thread t owns columns CPT (t mod N/CPT) .. +CPT-1 in rows rg, rg + NG, ...
// (rg = t div N/CPT, NG row groups). Rows are not interchanged; the pivot of step k
// is the largest |A(i, k)| over the rows i not yet used as pivots (ties to the smaller
// i), found by every warp from the same shared copy of column k (on integer keys of
// the magnitudes), so all warps agree without a broadcast. Step k, with p the pivot row and r_p = A(p, :) / A(p, k),
// r_p(k) = 1 / A(p, k):
//   * column k was zeroed in registers when its owners published it, and row p is
//     zeroed by its owners when they publish r_p;
//   * every row then takes A(i, :) -= f_i r_p with f_i = A(i, k), f_p = -1, so row p
//     becomes r_p and column k becomes -A(i, k) / A(p, k): no per-element selects;
//   * the owners of column k + 1 publish it for the next step at once (the column
//     buffer is double-buffered by the parity of k), two barriers per step.
// The k loop is unrolled by CPT so that the published column is a fixed register.
// At the end, with p_k the pivot row of step k and c(p_k) = k, the inverse is
// A^{-1}(k, m) = X(p_k, c(m)), read from the padded [N][N+1] shared tile that also
// stages the block on the way in (16-byte global loads and stores).
template <class T, int N, int NT, int CPT> struct BInvN {
  static constexpr int CG = N / CPT;                             // column groups
  static constexpr int NG = (NT / CG) < N ? (NT / CG) : N;       // row groups
  static constexpr int RPT = (N + NG - 1) / NG;                  // rows per thread
  static constexpr int NS = (N + 31) / 32;                       // pivot-search rows per lane
  static constexpr size_t SMEM = (size_t)N * (N + 1) * sizeof(T) + 3 * N * sizeof(T) + 2 * N * sizeof(int) + 64;
};

template <class T, int N, int NT, int CPT>
__global__ void __launch_bounds__(NT) k_block_inverse_n(const double* __restrict__ blocks, T* __restrict__ inv,
                                                        int* status) {
  static_assert(N % CPT == 0 && N % 4 == 0 && N <= 128 && NT % 32 == 0 && NT / (N / CPT) >= 1 &&
                    (CPT * sizeof(T)) % 16 == 0, "block size");
  typedef BInvN<T, N, NT, CPT> L;
  constexpr int CG = L::CG, NG = L::NG, RPT = L::RPT, NS = L::NS, LD = N + 1;
  constexpr int VW = 16 / sizeof(T);   // values per 16-byte shared load
  typedef typename std::conditional<sizeof(T) == 4, int, long long>::type PivotKey;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* S = (T*)sm_raw;                   // [N][N+1] staging tile
  T* colbuf = S + N * LD;              // [2][N] column k (parity of k)
  T* prow = colbuf + 2 * N;            // [N] scaled pivot row (16-byte aligned: N (N + 3) % 4 == 0)
  int* pivrow = (int*)(prow + N);      // [N] pivot row of step k
  int* colof = pivrow + N;             // [N] step whose pivot was row i
  const int e = blockIdx.x;
  const int lane = threadIdx.x & 31;
  // column-major FP64 block -> row-major padded tile; N even, so each 16-byte pair
  // holds rows r, r + 1 of one column
  {
    const double2* B2 = (const double2*)(blocks + (size_t)e * N * N);
    constexpr int P2 = N * N / 2, IT = (P2 + NT - 1) / NT;
    double2 v[IT];
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int i2 = threadIdx.x + it * NT;
      if (i2 < P2) v[it] = B2[i2];
    }
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int i2 = threadIdx.x + it * NT;
      if (i2 < P2) {
        const int col = (2 * i2) / N, row = 2 * i2 - col * N;
        S[row * LD + col] = (T)v[it].x;
        S[(row + 1) * LD + col] = (T)v[it].y;
      }
    }
  }
  const int cg = threadIdx.x % CG, rg = threadIdx.x / CG;
  const bool act = rg < NG;
  __syncthreads();
  T a[RPT][CPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int i = rg + NG * r;
#pragma unroll
    for (int c = 0; c < CPT; ++c) a[r][c] = (act && i < N) ? S[i * LD + CPT * cg + c] : T(0);
  }
  // the owners of column CPT kq + KC write it to buf and zero it in registers
  auto publish_column = [&](int kq, auto kc_const, T* buf) {
    constexpr int KC = decltype(kc_const)::value;
    if (act && cg == kq) {
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const int i = rg + NG * r;
        if (i < N) {
          buf[i] = a[r][KC];
          a[r][KC] = T(0);
        }
      }
    }
  };
  publish_column(0, std::integral_constant<int, 0>(), colbuf);
  bool used[NS];
#pragma unroll
  for (int t = 0; t < NS; ++t) used[t] = false;
  __syncthreads();
  for (int kq = 0; kq < CG; ++kq) {
    auto step = [&](auto kc_const) {
      constexpr int KC = decltype(kc_const)::value;
      const int k = CPT * kq + KC;
      const T* col = colbuf + (k & 1) * N;
      // pivot row, on integer keys of |A(i, k)| (the order of the magnitudes; NaN
      // counts as -1, and a lane without unused rows offers row N at -2), so that no
      // floating-point instruction is spent on the search
      PivotKey best = -2;
      int bi = N;
#pragma unroll
      for (int t = 0; t < NS; ++t) {
        const int i = lane + 32 * t;
        if (i < N && !used[t]) {
          const PivotKey key = abs_key(col[i]);
          if (key > best) { best = key; bi = i; }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const PivotKey ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      const int p = bi;
#pragma unroll
      for (int t = 0; t < NS; ++t)
        if (lane + 32 * t == p) used[t] = true;
      if (threadIdx.x == 0) {
        pivrow[k] = p;
        colof[p] = k;
      }
      // the owners of row p publish it scaled (column k: 1 / pivot) and zero it; only
      // they form the reciprocal
      if (act && p >= rg && (p - rg) % NG == 0) {
        const T pv = col[p];
        if (pv == T(0) && cg == 0) *status = 1;
        const T ip = pv != T(0) ? T(1) / pv : T(0);
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          if (rg + NG * r == p) {
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
              prow[CPT * cg + c] = (c == KC && cg == kq ? T(1) : a[r][c]) * ip;
              a[r][c] = T(0);
            }
          }
        }
      }
      __syncthreads();
      // elimination: A(i, :) -= f_i r_p, f_p = -1
      if (act) {
        T pk[CPT];
#pragma unroll
        for (int c = 0; c < CPT; c += VW) {
          if constexpr (sizeof(T) == 4) {
            const float4 w = *(const float4*)(prow + CPT * cg + c);
            pk[c] = w.x; pk[c + 1] = w.y; pk[c + 2] = w.z; pk[c + 3] = w.w;
          } else {
            const double2 w = *(const double2*)(prow + CPT * cg + c);
            pk[c] = w.x; pk[c + 1] = w.y;
          }
        }
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          const int i = rg + NG * r;
          if (i < N) {
            const T f = i == p ? T(-1) : col[i];
#pragma unroll
            for (int c = 0; c < CPT; ++c) a[r][c] = fma(-f, pk[c], a[r][c]);
          }
        }
      }
      // the next column, for the next step
      if (k + 1 < N) {
        constexpr int KN = (KC + 1) % CPT;
        publish_column(KC + 1 < CPT ? kq : kq + 1, std::integral_constant<int, KN>(), colbuf + ((k + 1) & 1) * N);
      }
      __syncthreads();
    };
    unrolled_for<0, CPT>(step);
  }
  // X to the shared tile (its last reads precede the elimination's barriers)
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int i = rg + NG * r;
    if (act && i < N)
#pragma unroll
      for (int c = 0; c < CPT; ++c) S[i * LD + CPT * cg + c] = a[r][c];
  }
  __syncthreads();
  // A^{-1}(k, m) = X(p_k, c(m)), column-major, 16 bytes per store (N is a multiple of 4)
  T* Iv = inv + (size_t)e * N * N;
  if constexpr (sizeof(T) == 4) {
    for (int i4 = threadIdx.x; i4 < N * N / 4; i4 += NT) {
      const int m = (4 * i4) / N, k = 4 * i4 - m * N, sc = colof[m];
      ((float4*)Iv)[i4] = make_float4(S[pivrow[k] * LD + sc], S[pivrow[k + 1] * LD + sc],
                                      S[pivrow[k + 2] * LD + sc], S[pivrow[k + 3] * LD + sc]);
    }
  } else {
    for (int i2 = threadIdx.x; i2 < N * N / 2; i2 += NT) {
      const int m = (2 * i2) / N, k = 2 * i2 - m * N, sc = colof[m];
      ((double2*)Iv)[i2] = make_double2(S[pivrow[k] * LD + sc], S[pivrow[k + 1] * LD + sc]);
    }
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

// y_e = inv_e x_e (FP32 blocks) for block sizes n that divide 128 (n >= 16): one warp per
// element reads the column-major block as a flat array with 16-byte loads, 128
// consecutive values (128 / n columns) per warp instruction, so every lane keeps the
// same 4 rows r = 4 lane mod n throughout; lanes holding the same rows are summed by
// shuffles at the end. x_e is staged in shared memory. 8 elements per CTA.
__global__ void __launch_bounds__(256) k_block_apply_vec(const float* __restrict__ inv, const double* __restrict__ x,
                                                        double* __restrict__ y, int n, int64_t E, const int* skip,
                                                        const int* inst, const int* inst_skip) {
  if (skip && *skip) return;
  __shared__ float xs[8][128];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e = blockIdx.x * (int64_t)8 + wid;
  const bool live = e < E && !(inst_skip && inst_skip[inst[e]]);
  if (live)
    for (int i = lane; i < n; i += 32) xs[wid][i] = (float)x[e * n + i];
  __syncwarp();
  if (!live) return;
  const float4* blk = reinterpret_cast<const float4*>(inv + e * n * n);
  const int per = n * n / 128;                 // float4 loads per lane
  const int cpi = 128 / n;                     // columns per warp instruction
  const int c_lane = (4 * lane) / n;           // the lane's column within the instruction
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
  for (int k = 0; k < per; ++k) {
    const float4 b = __ldg(blk + k * 32 + lane);
    const float xc = xs[wid][k * cpi + c_lane];
    acc.x = fmaf(b.x, xc, acc.x);
    acc.y = fmaf(b.y, xc, acc.y);
    acc.z = fmaf(b.z, xc, acc.z);
    acc.w = fmaf(b.w, xc, acc.w);
  }
  // lanes l and l + n/4, l + 2n/4, ... hold partial sums of the same rows
  for (int off = n / 4; off < 32; off <<= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, off);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, off);
    acc.z += __shfl_down_sync(0xffffffffu, acc.z, off);
    acc.w += __shfl_down_sync(0xffffffffu, acc.w, off);
  }
  if (lane < n / 4) {
    double* ye = y + e * n + 4 * lane;
    ye[0] = (double)acc.x;
    ye[1] = (double)acc.y;
    ye[2] = (double)acc.z;
    ye[3] = (double)acc.w;
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
