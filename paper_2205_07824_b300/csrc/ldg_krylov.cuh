// Device kernels of the restarted GMRES(m) solve (Section 3.3): FP64 dot
// products, vector updates, Givens rotations and the triangular solve.
//
// Every grid-wide reduction is finished by the last block to arrive (threadfence
// + atomic ticket), which sums the per-block partials in block order, so results
// are deterministic and no separate reduction launch is needed. Each kernel
// returns at once when the solve's `done` flag is set, so the host can queue
// Arnoldi steps ahead of the GPU without waiting for the convergence test.
#pragma once
#include <cuda_runtime.h>

namespace ldg {

constexpr int KRY_T = 256;

// Forcing term of an inexact Newton step at ||R(u_k)|| = rn: gmres_rtol, or with
// LDG_FORCING_LAST at least half of what the Newton tolerance still asks for, so that
// the last linear solve is not taken further than the Newton test needs.
__host__ __device__ inline double newton_forcing_eta(int forcing, double gmres_rtol, double newton_rtol, double r0,
                                                     double rn) {
  if (forcing != 1 || !(rn > 0.0)) return gmres_rtol;
  const double need = 0.5 * newton_rtol * r0 / rn;
  return need > gmres_rtol ? need : gmres_rtol;
}

// Layout of the small FP64 work area of one GMRES(m) solve.
struct KrySmall {
  int m;
  __host__ __device__ size_t H() const { return 0; }                      // (m+1) x m, column-major
  __host__ __device__ size_t cs() const { return (size_t)(m + 1) * m; }
  __host__ __device__ size_t sn() const { return cs() + m; }
  __host__ __device__ size_t g() const { return sn() + m; }               // m+1
  __host__ __device__ size_t y() const { return g() + m + 1; }            // m
  __host__ __device__ size_t h1() const { return y() + m; }               // m+2
  __host__ __device__ size_t h2() const { return h1() + m + 2; }          // m+2
  __host__ __device__ size_t sc() const { return h2() + m + 2; }          // 16 scalars
  __host__ __device__ size_t total() const { return sc() + 16; }
};
// scalars sc[]: 0 ||w||^2 (last norm), 1 |g_{j+1}|, 2 h_{j+1,j}, 3 convergence threshold,
//               4 ||r||^2 (true residual), 5 spare, 6 -1.0 (axpy coefficient)
// int flags[]: 0 done, 1 number of Arnoldi columns, 2 breakdown

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce `NV` accumulators into part[blockIdx.x][k]; returns true in the
// last block (after all partials are visible).
template <int NV>
__device__ __forceinline__ bool block_partials(double (&acc)[NV], int nvec, double* part, int ldp,
                                               unsigned int* ticket) {
  __shared__ double red[KRY_T / 32][NV];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double v = warp_sum(acc[k]);
    if (lane == 0) red[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < nvec) {
    double s = 0.0;
    for (int q = 0; q < KRY_T / 32; ++q) s += red[q][threadIdx.x];
    part[(size_t)blockIdx.x * ldp + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  return last;
}

// Sum of column k of the partials, in block order (single thread; small grids).
__device__ __forceinline__ double sum_partials(const double* part, int ldp, int k) {
  double s = 0.0;
  for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(part + (size_t)b * ldp + k);
  return s;
}

// out[k] = sum over blocks of part[b][k], k < nvec, by the whole last block: the
// threads form KRY_T / kw groups of kw lanes (kw = nvec rounded up to a power of
// two), each group strides over the blocks, then a fixed-shape tree sums the groups.
// The summation order is fixed, so the result is deterministic.
__device__ __forceinline__ void reduce_partials(const double* part, int ldp, int nvec, double* out) {
  __shared__ double gred[KRY_T];
  int kw = 1;
  while (kw < nvec) kw <<= 1;
  const int groups = KRY_T / kw;
  const int k = threadIdx.x % kw, grp = threadIdx.x / kw;
  double s = 0.0;
  if (k < nvec) {
    const int nb = (int)gridDim.x;
#pragma unroll 4
    for (int b = grp; b < nb; b += groups) s += __ldcg(part + (size_t)b * ldp + k);
  }
  gred[threadIdx.x] = s;
  __syncthreads();
  // fixed-shape tree over the groups (groups is a power of two)
  for (int st = groups >> 1; st > 0; st >>= 1) {
    if (grp < st) gred[threadIdx.x] += gred[threadIdx.x + st * kw];
    __syncthreads();
  }
  if (threadIdx.x < nvec) out[threadIdx.x] = gred[threadIdx.x];
}

// Completes Arnoldi column j from the two Gram-Schmidt passes' projections h1 + h2 and
// ||w||^2: H(:, j) = h1 + h2, H(j+1, j) = ||w||, applies the previous Givens rotations,
// forms rotation j, rotates g, and sets flags[0] (done) when |g_{j+1}| <= sc[3] or on
// breakdown (flags[2]); flags[1] = j + 1 columns. The previous rotations and h1 + h2 are
// staged in shared memory by the whole CTA, so the one-thread rotation loop reads no
// global memory. Call from all threads of the CTA; returns flags[0] in every thread.
__device__ __forceinline__ int arnoldi_column_block(double* small, int m, int j, double nrm2, int* flags) {
  __shared__ double cs_s[32], sn_s[32], col_s[34];
  __shared__ int done_s;
  KrySmall S{m};
  const int t = threadIdx.x;
  if (t < j) {
    cs_s[t] = small[S.cs() + t];
    sn_s[t] = small[S.sn() + t];
  }
  if (t <= j) col_s[t] = small[S.h1() + t] + small[S.h2() + t];
  __syncthreads();
  if (t == 0) {
    double* sc = small + S.sc();
    double* g = small + S.g();
    const double hn = sqrt(nrm2);
    sc[0] = nrm2;
    col_s[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
      const double a = col_s[i], b = col_s[i + 1];
      col_s[i] = cs_s[i] * a + sn_s[i] * b;
      col_s[i + 1] = -sn_s[i] * a + cs_s[i] * b;
    }
    const double a = col_s[j], b = col_s[j + 1];
    const double den = sqrt(a * a + b * b);
    const double cj = den > 0.0 ? a / den : 1.0, sj = den > 0.0 ? b / den : 0.0;
    small[S.cs() + j] = cj;
    small[S.sn() + j] = sj;
    col_s[j] = den;
    col_s[j + 1] = 0.0;
    const double gj = g[j];
    g[j + 1] = -sj * gj;
    g[j] = cj * gj;
    const double est = fabs(g[j + 1]);
    sc[1] = est;
    sc[2] = hn;
    flags[1] = j + 1;
    const bool breakdown = !(hn > 1e-14 * den);
    if (!(est > sc[3]) || breakdown) flags[0] = 1;   // NaN also ends the cycle
    if (breakdown) flags[2] = 1;
    done_s = flags[0];
  }
  __syncthreads();
  if (t <= j + 1) small[S.H() + (size_t)j * (m + 1) + t] = col_s[t];
  return done_s;
}

// out[k] = sum_i V[k][i] w[i] for k < nvec (NV >= nvec). Loads of all nvec vectors
// are issued together (compile-time bucket NV), two entries per thread per pass.
template <int NV>
__global__ void __launch_bounds__(KRY_T) k_dots(const double* __restrict__ V, int64_t ldv, int nvec,
                                               const double* __restrict__ w, int64_t n, double* part, int ldp,
                                               unsigned int* ticket, double* out, const int* flags) {
  if (flags && flags[0]) return;
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  const int64_t stride = (int64_t)gridDim.x * KRY_T;
  int64_t i = blockIdx.x * (int64_t)KRY_T + threadIdx.x;
  if constexpr (NV <= 16) {
    for (; i + stride < n; i += 2 * stride) {
      const double w0 = w[i], w1 = w[i + stride];
#pragma unroll
      for (int k = 0; k < NV; ++k)
        if (k < nvec) {
          const double a = V[k * ldv + i], b = V[k * ldv + i + stride];
          acc[k] = fma(b, w1, fma(a, w0, acc[k]));
        }
    }
  }
  for (; i < n; i += stride) {
    const double wi = w[i];
#pragma unroll
    for (int k = 0; k < NV; ++k)
      if (k < nvec) acc[k] = fma(V[k * ldv + i], wi, acc[k]);
  }
  if (!block_partials<NV>(acc, nvec, part, ldp, ticket)) return;
  reduce_partials(part, ldp, nvec, out);
  if (threadIdx.x == 0) *ticket = 0u;
}

// w -= sum_k V[k] h[k] (one classical Gram-Schmidt pass).
// DOTS: the same loop, which already holds V[k][i] in registers, also forms the
// next pass's projections out[k] = V[k] . w_new (the second Gram-Schmidt pass
// needs nothing else), saving a separate sweep over V.
// givens: forms ||w_new||^2 and the last block completes Arnoldi column j:
// H(:, j) = h1 + h2, H(j+1, j) = ||w||, applies the previous rotations, forms
// rotation j, rotates g and sets the done flag when |g_{j+1}| <= sc[3] or on breakdown.
template <int NV, bool DOTS>
__global__ void __launch_bounds__(KRY_T) k_orth_update(const double* __restrict__ V, int64_t ldv, int nvec,
                                                      const double* __restrict__ h, double* __restrict__ w,
                                                      int64_t n, double* part, int ldp, unsigned int* ticket,
                                                      double* small, int m, int j, int givens, int* flags,
                                                      double* dots_out) {
  if (flags[0]) return;
  __shared__ double hs[NV];
  if (threadIdx.x < NV) hs[threadIdx.x] = threadIdx.x < nvec ? h[threadIdx.x] : 0.0;
  __syncthreads();
  constexpr int NA = DOTS ? NV : 1;
  double acc[NA];
#pragma unroll
  for (int k = 0; k < NA; ++k) acc[k] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)KRY_T + threadIdx.x; i < n; i += (int64_t)gridDim.x * KRY_T) {
    double vv[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) vv[k] = k < nvec ? V[k * ldv + i] : 0.0;
    double s = w[i];
#pragma unroll
    for (int k = 0; k < NV; ++k) s = fma(-vv[k], hs[k], s);
    w[i] = s;
    if constexpr (DOTS) {
#pragma unroll
      for (int k = 0; k < NV; ++k) acc[k] = fma(vv[k], s, acc[k]);
    } else {
      acc[0] = fma(s, s, acc[0]);
    }
  }
  if constexpr (DOTS) {
    if (!block_partials<NA>(acc, nvec, part, ldp, ticket)) return;
    reduce_partials(part, ldp, nvec, dots_out);
    if (threadIdx.x == 0) *ticket = 0u;
    return;
  } else {
    if (!givens) return;
    if (!block_partials<1>(acc, 1, part, ldp, ticket)) return;
    __shared__ double nrm_s[1];
    reduce_partials(part, ldp, 1, nrm_s);
    __syncthreads();
    if (threadIdx.x == 0) *ticket = 0u;
    arnoldi_column_block(small, m, j, nrm_s[0], flags);
  }
}

// out = in / sqrt(sc[0]) (the factor formed once per CTA: FP64 square roots and divisions
// in every thread would cost the FP64 pipe more than the scaling)
static __global__ void k_scale_by_norm(const double* in, const double* small_sc, double* out, int64_t n, const int* flags) {
  if (flags && flags[0]) return;
  __shared__ double f_s;
  if (threadIdx.x == 0) {
    const double s = sqrt(small_sc[0]);
    f_s = s > 0.0 ? 1.0 / s : 0.0;
  }
  __syncthreads();
  const double f = f_s;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i] * f;
}

// Cycle start: V0 = r / ||r|| (||r||^2 in sc[4]); g = (||r||, 0, ...); flags cleared.
static __global__ void k_cycle_start(const double* r, double* V0, int64_t n, double* small, int m, int* flags) {
  KrySmall S{m};
  const double* sc = small + S.sc();
  __shared__ double s_s, f_s;
  if (threadIdx.x == 0) {
    s_s = sqrt(sc[4]);
    f_s = s_s > 0.0 ? 1.0 / s_s : 0.0;
  }
  __syncthreads();
  const double s = s_s, f = f_s;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    V0[i] = r[i] * f;
  if (blockIdx.x == 0) {
    double* g = small + S.g();
    for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = i == 0 ? s : 0.0;
    if (threadIdx.x == 0) { flags[0] = 0; flags[1] = 0; flags[2] = 0; }
  }
}

// y = H(0:k, 0:k)^{-1} g(0:k), k = flags[1]
static __global__ void k_backsolve(double* small, int m, const int* flags) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  KrySmall S{m};
  const double* H = small + S.H();
  const double* g = small + S.g();
  double* y = small + S.y();
  const int k = flags[1];
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int l = i + 1; l < k; ++l) s -= H[(size_t)l * (m + 1) + i] * y[l];
    y[i] = s / H[(size_t)i * (m + 1) + i];
  }
}

// x += sum_{k < flags[1]} V[k] y[k]
static __global__ void k_solution_update(const double* __restrict__ V, int64_t ldv, const double* small, int m,
                                  const int* flags, double* __restrict__ x, int64_t n) {
  __shared__ double ys[32];
  KrySmall S{m};
  const int k = flags[1];
  if (threadIdx.x < k) ys[threadIdx.x] = small[S.y() + threadIdx.x];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = x[i];
    for (int l = 0; l < k; ++l) s = fma(V[l * ldv + i], ys[l], s);
    x[i] = s;
  }
}

// r = b - a and ||r||^2 -> *out
static __global__ void __launch_bounds__(KRY_T) k_sub_norm(const double* __restrict__ b, const double* __restrict__ a,
                                                   double* __restrict__ r, int64_t n, double* part, int ldp,
                                                   unsigned int* ticket, double* out) {
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)KRY_T + threadIdx.x; i < n; i += (int64_t)gridDim.x * KRY_T) {
    const double s = b[i] - a[i];
    r[i] = s;
    acc[0] = fma(s, s, acc[0]);
  }
  if (!block_partials<1>(acc, 1, part, ldp, ticket)) return;
  reduce_partials(part, ldp, 1, out);
  if (threadIdx.x == 0) *ticket = 0u;
}

// x += alpha * y with alpha read from device memory
static __global__ void k_axpy_dev(const double* __restrict__ y, const double* alpha, double* __restrict__ x, int64_t n) {
  const double a = *alpha;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fma(a, y[i], x[i]);
}

}  // namespace ldg
