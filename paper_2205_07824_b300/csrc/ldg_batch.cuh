// Device kernels of the batched Newton-GMRES solve (Section 3.3 applied to many
// independent parametrised problems at once).
//
// The batch vector holds every instance's state; instance s is the contiguous
// segment [off_s, off_s + n_s). Streaming kernels run one CTA per chunk (a
// contiguous piece of one segment, at most KB_CHUNK entries). Per-instance
// reductions (dot products, norms) are finished by the last chunk of the segment
// to arrive (threadfence + per-segment atomic ticket), which sums the segment's
// chunk partials in chunk order, so every result is deterministic.
//
// All instances advance in lock step through the same Newton iteration, restart
// cycle and Arnoldi step; each keeps its own Hessenberg matrix, Givens rotations
// and convergence state, and an instance that has converged is skipped by every
// kernel (skip arrays indexed by instance). The loop control kernels run in one
// CTA, decide the next trip of each loop from the per-instance state, and, inside
// a CUDA graph, set the WHILE node's condition with cudaGraphSetConditional. The
// Arnoldi step index lives in device memory (BatchCtl::j), so one captured body
// serves every step.
#pragma once
#include <cuda_runtime.h>

#include "ldg_krylov.cuh"

namespace ldg {

constexpr int KB_CHUNK = 4096;   // entries per chunk (16 per thread)
constexpr int KB_LDP = 32;       // leading dimension of the chunk partials
constexpr int KB_NV = 32;        // Gram-Schmidt bucket: up to 32 basis vectors (m <= 30)

struct SegView {
  const int* chunk_seg;     // [n_chunk] segment of each chunk
  const int64_t* chunk_lo;  // [n_chunk] first entry
  const int64_t* chunk_hi;  // [n_chunk] one past the last entry
  const int* seg_c0;        // [n_seg] first chunk of the segment
  const int* seg_nc;        // [n_seg] number of chunks
  double* part;             // [n_chunk][KB_LDP] reduction partials
  unsigned int* tick;       // [n_seg] arrival tickets (zero between kernels)
  double* small;            // [n_seg][ks] per-instance KrySmall areas
  int64_t ks;               // KrySmall{m}.total()
  int m;
  int* sflags;              // [n_seg][4]: 0 Arnoldi done, 1 columns, 2 breakdown
  int nseg;
  int nchunk;
};

// Per-instance Newton state.
struct SegState {
  double r0, rn, bnorm, lin_resid;
  int newton_done, gmres_active, status, newton_iters, gmres_iters, jv_calls, residual_calls, cycles;
  double rprev;      // ||R|| at the last accepted iterate
  int halvings;      // consecutive step halvings at the current iterate
  int backtracks;    // step halvings over the solve
};

// Newton step control: a step after which ||R|| grew more than NEWTON_GROWTH times, or
// became non-finite, is halved (u = u_accepted - delta / 2^h), at most NEWTON_HALVINGS
// times in a row and while Newton iterations remain; a step that cannot be halved any
// more is discarded (u = u_accepted) and the solve ends with LDG_ERR_MAXIT.
constexpr double NEWTON_GROWTH = 10.0;
constexpr int NEWTON_HALVINGS = 10;

// Loop state of the batched solve (one record).
struct BatchCtl {
  int k;          // Newton iteration
  int restart;    // restart cycle within the current linear solve
  int j;          // Arnoldi step within the current cycle
  int cond_a, cond_b, cond_c;        // last decision of each loop (read by the host-driven form)
  int n_newton, n_gmres, n_arn;      // instances active in each loop
  int max_newton, max_restarts, m;
  double newton_rtol, gmres_rtol;
  int forcing;    // ldg_options::newton_forcing
  long long trips_a, trips_b, trips_c;   // loop bodies executed
};

// Block-reduce NV accumulators of chunk c into part[c][:]; true in the last chunk of
// segment s to arrive (after every partial of the segment is visible).
template <int NV>
__device__ __forceinline__ bool seg_partials(double (&acc)[NV], int nvec, const SegView& sv, int c, int s) {
  __shared__ double red[KRY_T / 32][NV];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) red[wid][k] = v;
  }
  __syncthreads();
  if ((int)threadIdx.x < nvec) {
    double t = 0.0;
    for (int q = 0; q < KRY_T / 32; ++q) t += red[q][threadIdx.x];
    sv.part[(size_t)c * KB_LDP + threadIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(sv.tick + s, 1u) == (unsigned)(sv.seg_nc[s] - 1);
  __syncthreads();
  return last;
}

// out[k] = sum over the segment's chunks of part[c][k] in chunk order (whole CTA).
__device__ __forceinline__ void seg_reduce(const SegView& sv, int s, int nvec, double* out) {
  __shared__ double gred[KRY_T];
  int kw = 1;
  while (kw < nvec) kw <<= 1;
  const int groups = KRY_T / kw;
  const int k = threadIdx.x % kw, grp = threadIdx.x / kw;
  const int c0 = sv.seg_c0[s], nc = sv.seg_nc[s];
  double t = 0.0;
  if (k < nvec)
    for (int b = grp; b < nc; b += groups) t += __ldcg(sv.part + (size_t)(c0 + b) * KB_LDP + k);
  gred[threadIdx.x] = t;
  __syncthreads();
  // fixed-shape tree over the groups (groups is a power of two)
  for (int st = groups >> 1; st > 0; st >>= 1) {
    if (grp < st) gred[threadIdx.x] += gred[threadIdx.x + st * kw];
    __syncthreads();
  }
  if ((int)threadIdx.x < nvec) out[threadIdx.x] = gred[threadIdx.x];
}

// small_s[out_off] = ||x_s||^2 for every segment not skipped.
__global__ void __launch_bounds__(KRY_T) kb_norm2(SegView sv, const double* __restrict__ x, int out_off,
                                                 const int* skip) {
  const int c = blockIdx.x, s = sv.chunk_seg[c];
  if (skip && skip[s]) return;
  double acc[1] = {0.0};
  for (int64_t i = sv.chunk_lo[c] + threadIdx.x; i < sv.chunk_hi[c]; i += KRY_T) acc[0] = fma(x[i], x[i], acc[0]);
  if (!seg_partials<1>(acc, 1, sv, c, s)) return;
  seg_reduce(sv, s, 1, sv.small + (size_t)s * sv.ks + out_off);
  if (threadIdx.x == 0) sv.tick[s] = 0u;
}

// ------------------------------------------------------------ Arnoldi step
// One classical Gram-Schmidt step with re-orthogonalisation is five launches:
//   kb_mdot(part1)  kb_update(h1 <- part1; w -= V h1)  kb_mdot(part2)
//   kb_update(h2 <- part2; w -= V h2; ||w||^2 -> part3)  kb_scale(||w|| <- part3; v_{j+1})
// (kb_update can also form the next projections in its own sweep, part_dots; the
// per-column warp sums inside the row loop measured slower than the separate kb_mdot.)
// A kernel only writes per-chunk partials; the next kernel's CTAs each sum the
// partials of their own instance in chunk order (every CTA gets the same bits), so
// no atomics, tickets or serial last-block tails are needed. The CTA owning an
// instance's first chunk also keeps h1, h2 in the instance's small area, and in
// kb_scale completes the Arnoldi column and its Givens rotation.

// out[k] (shared memory) = sum over the chunks of segment s of part[c][k], in chunk
// order (whole CTA; every CTA computes the same bits).
__device__ __forceinline__ void seg_sum(const SegView& sv, const double* part, int s, int nvec, double* out) {
  __shared__ double gred[KRY_T];
  int kw = 1;
  while (kw < nvec) kw <<= 1;
  const int groups = KRY_T / kw;
  const int k = threadIdx.x % kw, grp = threadIdx.x / kw;
  const int c0 = sv.seg_c0[s], nc = sv.seg_nc[s];
  double t = 0.0;
  if (k < nvec)
    for (int b = grp; b < nc; b += groups) t += part[(size_t)(c0 + b) * KB_LDP + k];
  gred[threadIdx.x] = t;
  __syncthreads();
  // fixed-shape tree over the groups (groups is a power of two)
  for (int st = groups >> 1; st > 0; st >>= 1) {
    if (grp < st) gred[threadIdx.x] += gred[threadIdx.x + st * kw];
    __syncthreads();
  }
  if ((int)threadIdx.x < nvec) out[threadIdx.x] = gred[threadIdx.x];
  __syncthreads();
}

constexpr int KB_RB = 512;   // rows of one multi-dot work unit (16 per lane)

// part[c][k] = V[k] . w over chunk c, k <= j = ctl->j. The chunk of w is staged in
// shared memory; the work units (column k, 512-row block) are spread over the warps,
// each lane keeping 16 independent loads in flight, so a step with few columns still
// fills the memory pipeline. With zsrc, the staging also stores Z[j] = zsrc (flexible
// GMRES).
__global__ void __launch_bounds__(KRY_T) kb_mdot(SegView sv, const BatchCtl* ctl, const double* __restrict__ V,
                                                int64_t ldv, const double* __restrict__ w, double* __restrict__ part,
                                                const double* __restrict__ zsrc, double* __restrict__ Z,
                                                const int* skip) {
  const int c = blockIdx.x, s = sv.chunk_seg[c];
  if (skip[s]) return;
  __shared__ double ws[KB_CHUNK];
  __shared__ double red[KB_NV][KB_CHUNK / KB_RB];
  const int j = ctl->j, nvec = j + 1;
  const int64_t lo = sv.chunk_lo[c];
  const int len = (int)(sv.chunk_hi[c] - lo);
  for (int t = threadIdx.x; t < len; t += KRY_T) {
    ws[t] = w[lo + t];
    if (zsrc) Z[j * ldv + lo + t] = zsrc[lo + t];
  }
  __syncthreads();
  const int nb = (len + KB_RB - 1) / KB_RB;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int u = warp; u < nvec * nb; u += KRY_T / 32) {
    const int k = u / nb, b = u - k * nb;
    const int r0 = b * KB_RB + lane;
    const double* col = V + k * ldv + lo;
    double a = 0.0;
#pragma unroll
    for (int t = 0; t < KB_RB / 32; ++t) {
      const int r = r0 + 32 * t;
      if (r < len) a = fma(col[r], ws[r], a);
    }
    a = warp_sum(a);
    if (lane == 0) red[k][b] = a;
  }
  __syncthreads();
  if ((int)threadIdx.x < nvec) {
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += red[threadIdx.x][b];
    part[(size_t)c * KB_LDP + threadIdx.x] = t;
  }
}

// h_s = sum of part_in over the instance's chunks (kept at small_s + h_off by the
// instance's first chunk), then w_s -= V[0..j]_s h_s (4 rows per thread per pass, the
// column loop unrolled so 16 loads are in flight). With part_norm, the chunk's share
// of ||w_new||^2 goes to part_norm[c][0]. With part_dots, the same sweep also forms
// the next pass's projections V[k] . w_new over the chunk (the rows of V it just read,
// read again from L1) into part_dots[c][k].
__global__ void __launch_bounds__(KRY_T) kb_update(SegView sv, const BatchCtl* ctl, const double* __restrict__ V,
                                                  int64_t ldv, const double* __restrict__ part_in, int h_off,
                                                  double* __restrict__ w, double* __restrict__ part_norm,
                                                  double* __restrict__ part_dots, const int* skip) {
  const int c = blockIdx.x, s = sv.chunk_seg[c];
  if (skip[s]) return;
  const int j = ctl->j, nvec = j + 1;
  __shared__ double hs[KB_NV];
  seg_sum(sv, part_in, s, nvec, hs);
  if (c == sv.seg_c0[s] && (int)threadIdx.x < nvec) sv.small[(size_t)s * sv.ks + h_off + threadIdx.x] = hs[threadIdx.x];
  const int64_t lo = sv.chunk_lo[c], hi = sv.chunk_hi[c];
  __shared__ double dred[KB_NV][KRY_T / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (part_dots && lane < KB_NV) dred[lane][warp] = 0.0;
  __syncwarp();
  double acc = 0.0;
  // the trip count depends on the warp's first row only, so every lane of a warp takes
  // part in the shuffles below (rows past the chunk end are masked per lane)
  for (int64_t base0 = lo + (threadIdx.x - lane); base0 < hi; base0 += 4 * KRY_T) {
    const int64_t base = base0 + lane;
    double t[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i = base + q * KRY_T;
      t[q] = i < hi ? w[i] : 0.0;
    }
#pragma unroll 4
    for (int k = 0; k < nvec; ++k) {
      const double hk = hs[k];
      const double* col = V + k * ldv;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t i = base + q * KRY_T;
        if (i < hi) t[q] = fma(-col[i], hk, t[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i = base + q * KRY_T;
      if (i < hi) {
        w[i] = t[q];
        acc = fma(t[q], t[q], acc);
      }
    }
    if (part_dots) {
      // warp sums per column, accumulated per warp in a fixed order
      for (int k = 0; k < nvec; ++k) {
        const double* col = V + k * ldv;
        double d = 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t i = base + q * KRY_T;
          if (i < hi) d = fma(col[i], t[q], d);
        }
        d = warp_sum(d);
        if (lane == 0) dred[k][warp] += d;
      }
    }
  }
  if (part_dots) {
    __syncthreads();
    if ((int)threadIdx.x < nvec) {
      double t = 0.0;
      for (int q = 0; q < KRY_T / 32; ++q) t += dred[threadIdx.x][q];
      part_dots[(size_t)c * KB_LDP + threadIdx.x] = t;
    }
  }
  if (part_norm) {
    __shared__ double red[KRY_T / 32];
    const double v = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < KRY_T / 32; ++q) t += red[q];
      part_norm[(size_t)c * KB_LDP] = t;
    }
  }
}

// ||w_s||^2 = sum of part_norm over the instance's chunks; V[j+1]_s = vcur_s = w_s /
// ||w_s||. CTAs 0 .. nseg-1 (scheduled first) complete Arnoldi column j of one instance
// each (from h1, h2 in its small area), its Givens rotation and the convergence test,
// and set skip[s] when the instance is done; the other CTAs scale one chunk each
// (a chunk of an instance that is done at this step may be left unscaled: its v_{j+1}
// is never used).
__global__ void __launch_bounds__(KRY_T) kb_scale(SegView sv, const BatchCtl* ctl, const double* __restrict__ w,
                                                 const double* __restrict__ part_norm, double* __restrict__ V,
                                                 int64_t ldv, double* __restrict__ vcur, int* skip) {
  const int b = blockIdx.x;
  const bool givens = b < sv.nseg;
  const int c = givens ? -1 : b - sv.nseg;
  const int s = givens ? b : sv.chunk_seg[c];
  if (skip[s]) return;
  __shared__ double nrm_s[1];
  seg_sum(sv, part_norm, s, 1, nrm_s);
  const double nrm2 = nrm_s[0];
  const int j = ctl->j;
  if (givens) {
    const int done = arnoldi_column_block(sv.small + (size_t)s * sv.ks, sv.m, j, nrm2, sv.sflags + 4 * s);
    if (threadIdx.x == 0 && done) skip[s] = 1;
    return;
  }
  // 1 / ||w|| once per CTA: FP64 square roots and divisions in every thread would
  // cost the FP64 pipe more than the scaling itself
  __shared__ double f_s;
  if (threadIdx.x == 0) {
    const double nr = sqrt(nrm2);
    f_s = nr > 0.0 ? 1.0 / nr : 0.0;
  }
  __syncthreads();
  const double f = f_s;
  double* out = V + (size_t)(j + 1) * ldv;
  for (int64_t i = sv.chunk_lo[c] + threadIdx.x; i < sv.chunk_hi[c]; i += KRY_T) {
    const double t = w[i] * f;
    out[i] = t;
    vcur[i] = t;
  }
}

// ------------------------------------------------ double-FP32 Krylov basis
// With ldg_options::krylov_basis = LDG_BASIS_F32X2 the Arnoldi basis V and the vector
// being orthogonalised are held as pairs of floats, value = hi + lo, and the
// Gram-Schmidt sweeps run on the FP32 pipes. A pair carries about 48 significand bits
// (emulated FP64). Building blocks, from the published error-free transformations:
// Knuth's TwoSum, the FMA form of Dekker's exact product, Dekker's pair addition, and
// the compensated dot product of Ogita, Rump and Oishi (2005).
struct f32x2 {
  float hi, lo;
};

// a + b = s + e exactly (Knuth)
__device__ __forceinline__ f32x2 ff_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
// a + b = s + e exactly when |a| >= |b| or a = 0
__device__ __forceinline__ f32x2 ff_quick_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ f32x2 ff_normalise(f32x2 a) { return ff_quick_two_sum(a.hi, a.lo); }
__device__ __forceinline__ f32x2 ff_from_double(double x) {
  const float hi = __double2float_rn(x);
  return {hi, __double2float_rn(x - (double)hi)};
}
__device__ __forceinline__ double ff_to_double(f32x2 a) { return (double)a.hi + (double)a.lo; }
// a * b as an unnormalised pair: the exact product of the leading parts (p + e, e from
// one FMA) plus the two cross terms; the lo * lo term is below the pair's precision
__device__ __forceinline__ f32x2 ff_prod(f32x2 a, f32x2 b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p);
  return {p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e))};
}
// compensated accumulation s += t: the leading parts by TwoSum, every error term into
// s.lo (normalise once at the end)
__device__ __forceinline__ void ff_accumulate(f32x2& s, f32x2 t) {
  const f32x2 u = ff_two_sum(s.hi, t.hi);
  s.hi = u.hi;
  s.lo += u.lo + t.lo;
}
// the sum of two normalised pairs, normalised (Dekker's addition with both error terms)
__device__ __forceinline__ f32x2 ff_add(f32x2 a, f32x2 b) {
  f32x2 s = ff_two_sum(a.hi, b.hi);
  const f32x2 t = ff_two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = ff_quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return ff_quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ f32x2 ff_load(const float2* p, int64_t i) {
  const float2 v = p[i];
  return {v.x, v.y};
}
__device__ __forceinline__ void ff_store(float2* p, int64_t i, f32x2 a) { p[i] = make_float2(a.hi, a.lo); }
__device__ __forceinline__ f32x2 ff_warp_sum(f32x2 a) {
  a = ff_normalise(a);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const f32x2 b = {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
    a = ff_add(a, b);
  }
  return a;
}

// out[k] (shared memory) = sum over the chunks of segment s of the pair partials
// part[c][k], in chunk order with a fixed-shape tree (every CTA gets the same bits)
__device__ __forceinline__ void seg_sum_ff(const SegView& sv, const float2* part, int s, int nvec, f32x2* out) {
  __shared__ f32x2 gred[KRY_T];
  int kw = 1;
  while (kw < nvec) kw <<= 1;
  const int groups = KRY_T / kw;
  const int k = threadIdx.x % kw, grp = threadIdx.x / kw;
  const int c0 = sv.seg_c0[s], nc = sv.seg_nc[s];
  f32x2 t = {0.f, 0.f};
  if (k < nvec)
    for (int b = grp; b < nc; b += groups) t = ff_add(t, ff_load(part, (int64_t)(c0 + b) * KB_LDP + k));
  gred[threadIdx.x] = t;
  __syncthreads();
  for (int st = groups >> 1; st > 0; st >>= 1) {
    if (grp < st) gred[threadIdx.x] = ff_add(gred[threadIdx.x], gred[threadIdx.x + st * kw]);
    __syncthreads();
  }
  if ((int)threadIdx.x < nvec) out[threadIdx.x] = gred[threadIdx.x];
  __syncthreads();
}

// kb_mdot on the pair basis: part[c][k] = V[k] . w over chunk c, k <= j, as pairs. With
// wsrc (the first pass), the chunk of the FP64 vector w is split into pairs and also
// stored to wf for the kernels after it; otherwise w is read from wf. zsrc/Z as kb_mdot.
__global__ void __launch_bounds__(KRY_T) kb_mdot_ff(SegView sv, const BatchCtl* ctl, const float2* __restrict__ V,
                                                   int64_t ldv, const double* __restrict__ wsrc,
                                                   float2* __restrict__ wf, float2* __restrict__ part,
                                                   const double* __restrict__ zsrc, double* __restrict__ Z,
                                                   const int* skip) {
  const int c = blockIdx.x, s = sv.chunk_seg[c];
  if (skip[s]) return;
  __shared__ f32x2 ws[KB_CHUNK];
  __shared__ f32x2 red[KB_NV][KB_CHUNK / KB_RB];
  const int j = ctl->j, nvec = j + 1;
  const int64_t lo = sv.chunk_lo[c];
  const int len = (int)(sv.chunk_hi[c] - lo);
  for (int t = threadIdx.x; t < len; t += KRY_T) {
    if (wsrc) {
      ws[t] = ff_from_double(wsrc[lo + t]);
      ff_store(wf, lo + t, ws[t]);
    } else {
      ws[t] = ff_load(wf, lo + t);
    }
    if (zsrc) Z[j * ldv + lo + t] = zsrc[lo + t];
  }
  __syncthreads();
  const int nb = (len + KB_RB - 1) / KB_RB;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int u = warp; u < nvec * nb; u += KRY_T / 32) {
    const int k = u / nb, b = u - k * nb;
    const int r0 = b * KB_RB + lane;
    const float2* col = V + k * ldv + lo;
    // four independent compensated accumulators per lane (the chains are latency-bound)
    f32x2 acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
    for (int t = 0; t < KB_RB / 32; ++t) {
      const int r = r0 + 32 * t;
      if (r < len) ff_accumulate(acc[t & 3], ff_prod(ff_load(col, r), ws[r]));
    }
    f32x2 a = ff_add(ff_add(ff_normalise(acc[0]), ff_normalise(acc[1])),
                     ff_add(ff_normalise(acc[2]), ff_normalise(acc[3])));
    a = ff_warp_sum(a);
    if (lane == 0) red[k][b] = a;
  }
  __syncthreads();
  if ((int)threadIdx.x < nvec) {
    f32x2 t = {0.f, 0.f};
    for (int b = 0; b < nb; ++b) t = ff_add(t, red[threadIdx.x][b]);
    ff_store(part, (int64_t)c * KB_LDP + threadIdx.x, t);
  }
}

// kb_update on the pair basis: h_s = sum of the pair partials (kept at small_s + h_off in
// FP64 by the instance's first chunk), then wf_s -= V[0..j]_s h_s; with part_norm, the
// chunk's share of ||w_new||^2 goes to part_norm[c][0].
__global__ void __launch_bounds__(KRY_T) kb_update_ff(SegView sv, const BatchCtl* ctl, const float2* __restrict__ V,
                                                     int64_t ldv, const float2* __restrict__ part_in, int h_off,
                                                     float2* __restrict__ wf, float2* __restrict__ part_norm,
                                                     const int* skip) {
  const int c = blockIdx.x, s = sv.chunk_seg[c];
  if (skip[s]) return;
  const int j = ctl->j, nvec = j + 1;
  __shared__ f32x2 hs[KB_NV];
  seg_sum_ff(sv, part_in, s, nvec, hs);
  if (c == sv.seg_c0[s] && (int)threadIdx.x < nvec)
    sv.small[(size_t)s * sv.ks + h_off + threadIdx.x] = ff_to_double(hs[threadIdx.x]);
  const int64_t lo = sv.chunk_lo[c], hi = sv.chunk_hi[c];
  f32x2 nacc = {0.f, 0.f};
  for (int64_t base = lo + threadIdx.x; base < hi; base += 4 * KRY_T) {
    // per row two independent compensated accumulators, over the even and the odd
    // columns (the chains are latency-bound), added at the end
    f32x2 t[4], t2[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i = base + q * KRY_T;
      t[q] = i < hi ? ff_load(wf, i) : f32x2{0.f, 0.f};
      t2[q] = f32x2{0.f, 0.f};
    }
#pragma unroll 2
    for (int k = 0; k < nvec; k += 2) {
      const bool two = k + 1 < nvec;
      const f32x2 hk = hs[k], hk1 = two ? hs[k + 1] : f32x2{0.f, 0.f};
      const float2* col = V + k * ldv;
      const float2* col1 = col + ldv;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t i = base + q * KRY_T;
        if (i < hi) {
          const f32x2 p = ff_prod(ff_load(col, i), hk);
          ff_accumulate(t[q], f32x2{-p.hi, -p.lo});
          if (two) {
            const f32x2 p1 = ff_prod(ff_load(col1, i), hk1);
            ff_accumulate(t2[q], f32x2{-p1.hi, -p1.lo});
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i = base + q * KRY_T;
      if (i < hi) {
        t[q] = ff_add(ff_normalise(t[q]), ff_normalise(t2[q]));
        ff_store(wf, i, t[q]);
        if (part_norm) ff_accumulate(nacc, ff_prod(t[q], t[q]));
      }
    }
  }
  if (part_norm) {
    __shared__ f32x2 red[KRY_T / 32];
    const f32x2 v = ff_warp_sum(nacc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      f32x2 t = {0.f, 0.f};
      for (int q = 0; q < KRY_T / 32; ++q) t = ff_add(t, red[q]);
      ff_store(part_norm, (int64_t)c * KB_LDP, t);
    }
  }
}

// kb_scale on the pair basis: ||w_s||^2 from the pair partials; V[j+1]_s = w_s / ||w_s||
// as pairs and vcur_s = the same in FP64 for the preconditioner and J.v. CTAs
// 0 .. nseg-1 complete the Arnoldi column and its Givens rotation as in kb_scale.
__global__ void __launch_bounds__(KRY_T) kb_scale_ff(SegView sv, const BatchCtl* ctl, const float2* __restrict__ wf,
                                                    const float2* __restrict__ part_norm, float2* __restrict__ V,
                                                    int64_t ldv, double* __restrict__ vcur, int* skip) {
  const int b = blockIdx.x;
  const bool givens = b < sv.nseg;
  const int c = givens ? -1 : b - sv.nseg;
  const int s = givens ? b : sv.chunk_seg[c];
  if (skip[s]) return;
  __shared__ f32x2 nrm_s[1];
  seg_sum_ff(sv, part_norm, s, 1, nrm_s);
  const double nrm2 = ff_to_double(nrm_s[0]);
  const int j = ctl->j;
  if (givens) {
    const int done = arnoldi_column_block(sv.small + (size_t)s * sv.ks, sv.m, j, nrm2, sv.sflags + 4 * s);
    if (threadIdx.x == 0 && done) skip[s] = 1;
    return;
  }
  __shared__ f32x2 f_s;
  if (threadIdx.x == 0) {
    const double nr = sqrt(nrm2);
    f_s = ff_from_double(nr > 0.0 ? 1.0 / nr : 0.0);
  }
  __syncthreads();
  const f32x2 f = f_s;
  float2* out = V + (size_t)(j + 1) * ldv;
  for (int64_t i = sv.chunk_lo[c] + threadIdx.x; i < sv.chunk_hi[c]; i += KRY_T) {
    const f32x2 t = ff_normalise(ff_prod(ff_load(wf, i), f));
    ff_store(out, i, t);
    vcur[i] = ff_to_double(t);
  }
}

// Cycle start on the pair basis: V[0]_s = r_s / ||r_s|| as pairs, vcur_s in FP64.
__global__ void kb_cycle_start_ff(SegView sv, const double* __restrict__ r, float2* __restrict__ V0,
                                  double* __restrict__ vcur, const int* skip) {
  const int c = blockIdx.x, s = sv.chunk_seg[c];
  if (skip[s]) return;
  KrySmall S{sv.m};
  __shared__ double f_s;
  if (threadIdx.x == 0) {
    const double nr = sqrt(sv.small[(size_t)s * sv.ks + S.sc() + 4]);
    f_s = nr > 0.0 ? 1.0 / nr : 0.0;
  }
  __syncthreads();
  const double f = f_s;
  for (int64_t i = sv.chunk_lo[c] + threadIdx.x; i < sv.chunk_hi[c]; i += blockDim.x) {
    const f32x2 t = ff_from_double(r[i] * f);
    ff_store(V0, i, t);
    vcur[i] = ff_to_double(t);
  }
}

// x_s += sum_{l < k_s} V[l]_s y_s[l] with the pair basis (no preconditioner)
__global__ void kb_solution_update_ff(SegView sv, const float2* __restrict__ V, int64_t ldv, double* __restrict__ x,
                                      const int* skip) {
  const int c = blockIdx.x, s = sv.chunk_seg[c];
  if (skip[s]) return;
  __shared__ double ys[KB_NV];
  KrySmall S{sv.m};
  const int k = sv.sflags[4 * s + 1];
  if ((int)threadIdx.x < k) ys[threadIdx.x] = sv.small[(size_t)s * sv.ks + S.y() + threadIdx.x];
  __syncthreads();
  for (int64_t i = sv.chunk_lo[c] + threadIdx.x; i < sv.chunk_hi[c]; i += blockDim.x) {
    double t = x[i];
    for (int l = 0; l < k; ++l) t = fma(ff_to_double(ff_load(V, l * ldv + i)), ys[l], t);
    x[i] = t;
  }
}

// Cycle start: V[0]_s = vcur_s = r_s / ||r_s|| (||r_s||^2 in sc[4]).
__global__ void kb_cycle_start(SegView sv, const double* __restrict__ r, double* __restrict__ V0,
                               double* __restrict__ vcur, const int* skip) {
  const int c = blockIdx.x, s = sv.chunk_seg[c];
  if (skip[s]) return;
  KrySmall S{sv.m};
  __shared__ double f_s;
  if (threadIdx.x == 0) {
    const double nr = sqrt(sv.small[(size_t)s * sv.ks + S.sc() + 4]);
    f_s = nr > 0.0 ? 1.0 / nr : 0.0;
  }
  __syncthreads();
  const double f = f_s;
  for (int64_t i = sv.chunk_lo[c] + threadIdx.x; i < sv.chunk_hi[c]; i += blockDim.x) {
    const double t = r[i] * f;
    V0[i] = t;
    vcur[i] = t;
  }
}

// y_s = H_s(0:k, 0:k)^{-1} g_s(0:k), k = columns of the instance (one thread per instance)
__global__ void kb_backsolve(SegView sv, const int* skip) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= sv.nseg || skip[s]) return;
  KrySmall S{sv.m};
  double* sm = sv.small + (size_t)s * sv.ks;
  const double* H = sm + S.H();
  const double* g = sm + S.g();
  double* y = sm + S.y();
  const int m = sv.m, k = sv.sflags[4 * s + 1];
  for (int i = k - 1; i >= 0; --i) {
    double t = g[i];
    for (int l = i + 1; l < k; ++l) t -= H[(size_t)l * (m + 1) + i] * y[l];
    y[i] = t / H[(size_t)i * (m + 1) + i];
  }
}

// x_s += sum_{l < k_s} B[l]_s y_s[l]  (B = V, or Z for flexible preconditioning)
__global__ void kb_solution_update(SegView sv, const double* __restrict__ B, int64_t ldb, double* __restrict__ x,
                                   const int* skip) {
  const int c = blockIdx.x, s = sv.chunk_seg[c];
  if (skip[s]) return;
  __shared__ double ys[KB_NV];
  KrySmall S{sv.m};
  const int k = sv.sflags[4 * s + 1];
  if ((int)threadIdx.x < k) ys[threadIdx.x] = sv.small[(size_t)s * sv.ks + S.y() + threadIdx.x];
  __syncthreads();
  for (int64_t i = sv.chunk_lo[c] + threadIdx.x; i < sv.chunk_hi[c]; i += blockDim.x) {
    double t = x[i];
    for (int l = 0; l < k; ++l) t = fma(B[l * ldb + i], ys[l], t);
    x[i] = t;
  }
}

// r_s = b_s - a_s and ||r_s||^2 -> sc[4]
__global__ void __launch_bounds__(KRY_T) kb_sub_norm(SegView sv, const double* __restrict__ b,
                                                    const double* __restrict__ a, double* __restrict__ r,
                                                    const int* skip) {
  const int c = blockIdx.x, s = sv.chunk_seg[c];
  if (skip[s]) return;
  double acc[1] = {0.0};
  for (int64_t i = sv.chunk_lo[c] + threadIdx.x; i < sv.chunk_hi[c]; i += KRY_T) {
    const double t = b[i] - a[i];
    r[i] = t;
    acc[0] = fma(t, t, acc[0]);
  }
  if (!seg_partials<1>(acc, 1, sv, c, s)) return;
  KrySmall S{sv.m};
  seg_reduce(sv, s, 1, sv.small + (size_t)s * sv.ks + S.sc() + 4);
  if (threadIdx.x == 0) sv.tick[s] = 0u;
}

// Start of a linear solve: r_s = res_s, x_s = 0
__global__ void kb_prep_linear(SegView sv, const double* __restrict__ res, double* __restrict__ r,
                               double* __restrict__ x, const int* skip) {
  const int c = blockIdx.x, s = sv.chunk_seg[c];
  if (skip[s]) return;
  for (int64_t i = sv.chunk_lo[c] + threadIdx.x; i < sv.chunk_hi[c]; i += blockDim.x) {
    r[i] = res[i];
    x[i] = 0.0;
  }
}

// Newton update u_s -= x_s (not where the step is being halved: bt[s])
__global__ void kb_newton_update(SegView sv, const double* __restrict__ x, double* __restrict__ u, const int* skip,
                                 const int* bt) {
  // (bt[s] == 2 instances are done: skip[s] is set)
  const int c = blockIdx.x, s = sv.chunk_seg[c];
  if (skip[s] || bt[s]) return;
  for (int64_t i = sv.chunk_lo[c] + threadIdx.x; i < sv.chunk_hi[c]; i += blockDim.x) u[i] -= x[i];
}

// After the Newton check: where the step is halved, x_s /= 2 and u_s = ub_s - x_s; at an
// accepted iterate of an active instance, ub_s = u_s.
// bt[s] == 2: the step is discarded, u_s = ub_s.
__global__ void kb_newton_step_control(SegView sv, double* __restrict__ x, double* __restrict__ u,
                                       double* __restrict__ ub, const int* skip_newt, const int* bt) {
  const int c = blockIdx.x, s = sv.chunk_seg[c];
  if (bt[s] == 2) {
    for (int64_t i = sv.chunk_lo[c] + threadIdx.x; i < sv.chunk_hi[c]; i += blockDim.x) u[i] = ub[i];
    return;
  }
  if (skip_newt[s]) return;
  const bool half = bt[s] != 0;
  for (int64_t i = sv.chunk_lo[c] + threadIdx.x; i < sv.chunk_hi[c]; i += blockDim.x) {
    if (half) {
      const double h = 0.5 * x[i];
      x[i] = h;
      u[i] = ub[i] - h;
    } else {
      ub[i] = u[i];
    }
  }
}

// ------------------------------------------------------------ loop control (one CTA)
__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle h, int use, unsigned v) {
  if (use) cudaGraphSetConditional(h, v);
}

// Solve start: every instance active, counters cleared.
__global__ void kb_init(BatchCtl* ctl, SegState* st, int nseg, int* skip_newt, int* skip_gm, int* skip_arn) {
  for (int s = threadIdx.x; s < nseg; s += blockDim.x) {
    SegState z;
    z.r0 = z.rn = z.bnorm = z.lin_resid = 0.0;
    z.newton_done = 0; z.gmres_active = 0; z.status = 0; z.newton_iters = 0; z.gmres_iters = 0;
    z.jv_calls = 0; z.residual_calls = 0; z.cycles = 0;
    z.rprev = 0.0; z.halvings = 0; z.backtracks = 0;
    st[s] = z;
    skip_newt[s] = 0; skip_gm[s] = 1; skip_arn[s] = 1;
  }
  if (threadIdx.x == 0) {
    ctl->k = 0; ctl->restart = 0; ctl->j = 0;
    ctl->cond_a = 1; ctl->cond_b = 0; ctl->cond_c = 0;
    ctl->n_newton = nseg; ctl->n_gmres = 0; ctl->n_arn = 0;
    ctl->trips_a = 0; ctl->trips_b = 0; ctl->trips_c = 0;
  }
}

// After R(u_k) and ||R_s||^2 (sc[5]): Newton convergence test per instance; the ones
// still active start a linear solve J delta = R with threshold eta_k ||R_s||, eta_k the
// forcing term (newton_forcing_eta).
// bt[s] = 1 where the last step is halved instead (no linear solve this iteration).
__global__ void kb_newton_check(BatchCtl* ctl, SegView sv, SegState* st, int* skip_newt, int* skip_gm, int* bt,
                                cudaGraphConditionalHandle hb, int use_cond) {
  const int k = ctl->k;
  KrySmall S{sv.m};
  int active = 0;
  for (int s = threadIdx.x; s < sv.nseg; s += blockDim.x) {
    SegState& q = st[s];
    skip_gm[s] = 1;
    bt[s] = 0;
    if (q.newton_done) continue;
    double* sc = sv.small + (size_t)s * sv.ks + S.sc();
    const double rn = sqrt(sc[5]);
    q.residual_calls++;
    if (k == 0) { q.r0 = rn; q.rprev = rn; }
    q.rn = rn;
    if (k > 0 && !(rn <= NEWTON_GROWTH * q.rprev)) {
      if (q.halvings < NEWTON_HALVINGS && k < ctl->max_newton) {
        bt[s] = 1;
        q.halvings++;
        q.backtracks++;
      } else {
        // no acceptable step within the limits: back to the last accepted iterate
        bt[s] = 2;
        q.rn = q.rprev;
        q.status = -5;                                                // LDG_ERR_MAXIT
        q.newton_done = 1;
        skip_newt[s] = 1;
      }
      continue;
    }
    q.halvings = 0;
    q.rprev = rn;
    int done = 0;
    if (!isfinite(rn)) { q.status = -4; done = 1; }                 // LDG_ERR_NONFINITE
    else if (rn <= ctl->newton_rtol * q.r0) { q.status = 0; done = 1; }
    else if (k >= ctl->max_newton) { q.status = -5; done = 1; }     // LDG_ERR_MAXIT
    if (done) { q.newton_done = 1; skip_newt[s] = 1; continue; }
    q.gmres_active = 1;
    q.bnorm = rn;
    q.newton_iters++;
    sc[3] = newton_forcing_eta(ctl->forcing, ctl->gmres_rtol, ctl->newton_rtol, q.r0, rn) * rn;
    sc[4] = rn * rn;
    skip_gm[s] = 0;
    ++active;
  }
  const int cnt = __syncthreads_count(active > 0) > 0 ? 1 : 0;
  __shared__ int tot;
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  if (active) atomicAdd(&tot, active);
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl->n_newton = tot;
    ctl->restart = 0;
    ctl->trips_a++;
    ctl->cond_b = cnt;
    set_cond(hb, use_cond, (unsigned)cnt);
  }
}

// Restart cycle start: g_s = (||r_s||, 0, ...), flags cleared, Arnoldi active for the
// instances whose linear solve continues.
__global__ void kb_cycle_init(BatchCtl* ctl, SegView sv, const int* skip_gm, int* skip_arn,
                              cudaGraphConditionalHandle hc, int use_cond) {
  KrySmall S{sv.m};
  int active = 0;
  for (int s = threadIdx.x; s < sv.nseg; s += blockDim.x) {
    if (skip_gm[s]) { skip_arn[s] = 1; continue; }
    double* sm = sv.small + (size_t)s * sv.ks;
    double* g = sm + S.g();
    g[0] = sqrt(sm[S.sc() + 4]);
    for (int i = 1; i <= sv.m; ++i) g[i] = 0.0;
    int* fl = sv.sflags + 4 * s;
    fl[0] = 0; fl[1] = 0; fl[2] = 0;
    skip_arn[s] = 0;
    ++active;
  }
  const int any = __syncthreads_count(active > 0) > 0 ? 1 : 0;
  if (threadIdx.x == 0) {
    ctl->j = 0;
    ctl->n_arn = any;
    ctl->trips_b++;
    ctl->cond_c = any;
    set_cond(hc, use_cond, (unsigned)any);
  }
}

// End of an Arnoldi step: j += 1; continue while j < m and an instance is active.
__global__ void kb_arnoldi_end(BatchCtl* ctl, const int* skip_arn, int nseg, cudaGraphConditionalHandle hc,
                               int use_cond) {
  int active = 0;
  for (int s = threadIdx.x; s < nseg; s += blockDim.x) active += skip_arn[s] ? 0 : 1;
  const int any = __syncthreads_count(active > 0) > 0 ? 1 : 0;
  if (threadIdx.x == 0) {
    const int j = ctl->j + 1;
    ctl->j = j;
    ctl->trips_c++;
    const int go = (j < ctl->m && any) ? 1 : 0;
    ctl->cond_c = go;
    set_cond(hc, use_cond, (unsigned)go);
  }
}

// End of a restart cycle (true residual ||b - J x||^2 in sc[4]): an instance has
// converged when the true residual meets its threshold (or the Arnoldi estimate did
// and the true residual is within 10x of it); a cycle without columns or a
// non-finite residual ends its solve. Continue while some instance is unconverged
// and fewer than max_restarts cycles ran.
__global__ void kb_cycle_end(BatchCtl* ctl, SegView sv, SegState* st, int* skip_gm, int* skip_newt,
                             cudaGraphConditionalHandle hb, int use_cond) {
  KrySmall S{sv.m};
  const int restart = ctl->restart + 1;
  const bool last_cycle = restart >= ctl->max_restarts;
  int active = 0;
  for (int s = threadIdx.x; s < sv.nseg; s += blockDim.x) {
    if (skip_gm[s]) continue;
    SegState& q = st[s];
    const double* sc = sv.small + (size_t)s * sv.ks + S.sc();
    const int* fl = sv.sflags + 4 * s;
    const int cols = fl[1];
    const double beta = sqrt(sc[4]), thr = sc[3];
    q.gmres_iters += cols;
    q.jv_calls += cols + 1;
    q.cycles++;
    q.lin_resid = q.bnorm > 0.0 ? beta / q.bnorm : 0.0;
    const bool est = fl[0] && !fl[2];
    bool stop = false;
    if (!isfinite(beta)) {
      q.status = -4; q.newton_done = 1; skip_newt[s] = 1; stop = true;
    } else if (beta <= thr * (1.0 + 1e-6) || (est && beta <= thr * 10.0)) {
      stop = true;
    } else if (cols == 0 || last_cycle) {
      stop = true;   // no progress or out of cycles: Newton continues with this update
    }
    if (stop) { q.gmres_active = 0; skip_gm[s] = 1; }
    else ++active;
  }
  const int any = __syncthreads_count(active > 0) > 0 ? 1 : 0;
  if (threadIdx.x == 0) {
    ctl->restart = restart;
    ctl->n_gmres = any;
    const int go = (any && !last_cycle) ? 1 : 0;
    ctl->cond_b = go;
    set_cond(hb, use_cond, (unsigned)go);
  }
}

// End of a Newton iteration: k += 1; continue while an instance is unconverged
// (bounded by max_newton + 2 iterations).
__global__ void kb_newton_end(BatchCtl* ctl, const int* skip_newt, int nseg, cudaGraphConditionalHandle ha,
                              int use_cond) {
  int active = 0;
  for (int s = threadIdx.x; s < nseg; s += blockDim.x) active += skip_newt[s] ? 0 : 1;
  const int any = __syncthreads_count(active > 0) > 0 ? 1 : 0;
  if (threadIdx.x == 0) {
    const int k = ctl->k + 1;
    ctl->k = k;
    const int go = (any && k <= ctl->max_newton + 1) ? 1 : 0;
    ctl->cond_a = go;
    set_cond(ha, use_cond, (unsigned)go);
  }
}

}  // namespace ldg
