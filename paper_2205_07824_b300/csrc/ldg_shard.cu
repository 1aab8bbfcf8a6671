// Element-sharded operators and GMRES (Section 3.5: the paper partitions the mesh over
// MPI ranks, one GPU each). Each rank holds a context on its local mesh: the elements it
// owns first, then ghost copies of the face neighbours other ranks own. A sharded R or
// J.v exchanges the ghosts' u before the q-stage and their q before the residual stage,
// and computes the owned elements only; the GMRES sums its dot products over the ranks.
// Communication is the caller's: two callbacks of ldg_comm move the ghost blocks and sum
// the partial dot products (NCCL, or any transport), ordered after the stream has drained.
#include <cmath>
#include <string>
#include <vector>

#include "../../include/ldg.h"
#include "ldg_ctx.h"

using namespace ldg;

namespace {

constexpr int kT = 256;
constexpr int kBlocks = 296;   // partial sums per dot product (two per SM)

int fail_sh(ldg_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CKS(call)                                                                                \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return fail_sh(ctx, LDG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

// part[k * gridDim.x + b] = block b's share of V[k] . w over n entries
__global__ void __launch_bounds__(kT) k_sh_dots(const double* __restrict__ V, int64_t ldv, int nvec,
                                                const double* __restrict__ w, int64_t n, double* __restrict__ part) {
  __shared__ double red[kT];
  for (int k = 0; k < nvec; ++k) {
    const double* vk = V + (size_t)k * ldv;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) s += vk[i] * w[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = kT / 2; h > 0; h >>= 1) {
      if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)k * gridDim.x + blockIdx.x] = red[0];
    __syncthreads();
  }
}

// out[k] = sum of the G partials of vector k, in block order (one warp per vector)
__global__ void k_sh_reduce(const double* __restrict__ part, int G, int nvec, double* __restrict__ out) {
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (k >= nvec) return;
  double s = 0.0;
  for (int b = lane; b < G; b += 32) s += part[(size_t)k * G + b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[k] = s;
}

// w[i] -= sum_k h[k] V[k][i]
__global__ void k_sh_orth(const double* __restrict__ V, int64_t ldv, int nvec, const double* __restrict__ h,
                          double* __restrict__ w, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = w[i];
    for (int k = 0; k < nvec; ++k) s -= h[k] * V[(size_t)k * ldv + i];
    w[i] = s;
  }
}

// y[i] = a x[i] + b y[i] (y is not read when b = 0)
__global__ void k_sh_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = b == 0.0 ? a * x[i] : a * x[i] + b * y[i];
}

unsigned grid_n(int64_t n) { return (unsigned)std::min<int64_t>(148 * 8, std::max<int64_t>(1, (n + kT - 1) / kT)); }

int exchange(ldg_ctx* ctx, double* x, int block) {
  CKS(cudaStreamSynchronize(ctx->stream));
  const int rc = ctx->shard_comm.exchange_ghosts(ctx->shard_comm.user, x, block, (void*)ctx->stream);
  if (rc) return fail_sh(ctx, LDG_ERR_CUDA, "ldg_comm exchange_ghosts failed (" + std::to_string(rc) + ")");
  return LDG_OK;
}

// out[0..nvec) = sum over ranks of V[k] . w (owned entries), on the host in ctx->h_shdot
// and on the device in ctx->d_shdot
int gdots(ldg_ctx* ctx, const double* V, int64_t ldv, int nvec, const double* w) {
  const int64_t n = ctx->shard_owned * ctx->nloc;
  k_sh_dots<<<kBlocks, kT, 0, ctx->stream>>>(V, ldv, nvec, w, n, ctx->d_shpart);
  count_launch();
  k_sh_reduce<<<(nvec + 7) / 8, 256, 0, ctx->stream>>>(ctx->d_shpart, kBlocks, nvec, ctx->d_shdot);
  count_launch();
  CKS(cudaGetLastError());
  CKS(cudaStreamSynchronize(ctx->stream));
  const int rc = ctx->shard_comm.allreduce_sum(ctx->shard_comm.user, ctx->d_shdot, nvec, (void*)ctx->stream);
  if (rc) return fail_sh(ctx, LDG_ERR_CUDA, "ldg_comm allreduce_sum failed (" + std::to_string(rc) + ")");
  CKS(cudaMemcpyAsync(ctx->h_shdot.data(), ctx->d_shdot, nvec * sizeof(double), cudaMemcpyDeviceToHost,
                      ctx->stream));
  CKS(cudaStreamSynchronize(ctx->stream));
  return LDG_OK;
}

// R (mode R) or J.v of a linear model (mode HOM) on the owned elements; x's ghost blocks
// are refreshed first (x is written there).
int shard_apply(ldg_ctx* ctx, int mode, double* x, double* out) {
  int rc;
  if ((rc = exchange(ctx, x, ctx->nloc))) return rc;
  if (ctx->ks->qstage) {
    if ((rc = ldg_q_stage(ctx, mode, ctx->shard_owned, x, ctx->d_shq))) return rc;
    if ((rc = exchange(ctx, ctx->d_shq, ctx->nloc * ctx->dim))) return rc;
  }
  return ldg_residual_stage(ctx, mode, ctx->shard_owned, x, ctx->ks->qstage ? ctx->d_shq : nullptr, out);
}

bool sharded(const ldg_ctx* ctx) { return ctx && ctx->shard_owned > 0; }

}  // namespace

extern "C" {

int ldg_shard_setup(ldg_ctx* ctx, int64_t n_owned, const ldg_comm* comm) {
  if (!ctx || !ctx->ks || !comm || !comm->exchange_ghosts || !comm->allreduce_sum || n_owned <= 0 || n_owned > ctx->E)
    return LDG_ERR_ARG;
  ctx->shard_owned = n_owned;
  ctx->shard_comm = *comm;
  if (!ctx->d_shq && ctx->ks->qstage) CKS(cudaMalloc(&ctx->d_shq, (size_t)ctx->ndof * ctx->dim * sizeof(double)));
  if (!ctx->d_shpart) CKS(cudaMalloc(&ctx->d_shpart, (size_t)kBlocks * 32 * sizeof(double)));
  if (!ctx->d_shdot) CKS(cudaMalloc(&ctx->d_shdot, 32 * sizeof(double)));
  ctx->h_shdot.assign(32, 0.0);
  return LDG_OK;
}

int ldg_shard_residual(ldg_ctx* ctx, double* u, double* r) {
  if (!sharded(ctx) || !u || !r) return LDG_ERR_ARG;
  return shard_apply(ctx, LDG_STAGE_R, u, r);
}

int ldg_shard_jvp(ldg_ctx* ctx, double* v, double* jv) {
  if (!sharded(ctx) || !v || !jv) return LDG_ERR_ARG;
  if (!ctx->ks->linear) return fail_sh(ctx, LDG_ERR_ARG, "ldg_shard_jvp: linear models only");
  return shard_apply(ctx, LDG_STAGE_HOM, v, jv);
}

int ldg_shard_gmres(ldg_ctx* ctx, const double* b, double* x, ldg_solve_report* rep) {
  if (!sharded(ctx) || !b || !x) return LDG_ERR_ARG;
  if (!ctx->ks->linear) return fail_sh(ctx, LDG_ERR_ARG, "ldg_shard_gmres: linear models only");
  if (rep) *rep = ldg_solve_report{};
  const int m = ctx->m;
  const int64_t N = ctx->ndof, n = ctx->shard_owned * ctx->nloc;
  const double rtol = ctx->opt.gmres_rtol;
  double* V = ctx->d_V;                 // (m + 1) full-length vectors: J.v inputs carry ghost slots
  double* w = ctx->d_w;
  double* r = ctx->d_r;
  int rc;
  CKS(cudaMemsetAsync(x, 0, N * sizeof(double), ctx->stream));
  CKS(cudaMemcpyAsync(r, b, N * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  if ((rc = gdots(ctx, r, N, 1, r))) return rc;
  const double bnorm = std::sqrt(ctx->h_shdot[0]);
  if (!std::isfinite(bnorm)) return fail_sh(ctx, LDG_ERR_NONFINITE, "non-finite right-hand side");
  if (bnorm == 0.0) return LDG_OK;
  double beta = bnorm;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  for (int cycle = 0; cycle < ctx->opt.max_restarts; ++cycle) {
    k_sh_axpby<<<grid_n(n), kT, 0, ctx->stream>>>(1.0 / beta, r, 0.0, V, n);
    count_launch();
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int cols = 0;
    for (int j = 0; j < m; ++j) {
      double* vj = V + (size_t)j * N;
      double* wj = V + (size_t)(j + 1) * N;
      if ((rc = shard_apply(ctx, LDG_STAGE_HOM, vj, wj))) return rc;
      if (rep) rep->jv_calls++;
      // two passes of classical Gram-Schmidt, each with one summed multi-dot
      double* h = &H[(size_t)j * (m + 1)];
      for (int i = 0; i <= j; ++i) h[i] = 0.0;
      for (int pass = 0; pass < 2; ++pass) {
        // the summed projections stay in d_shdot for the update
        if ((rc = gdots(ctx, V, N, j + 1, wj))) return rc;
        for (int i = 0; i <= j; ++i) h[i] += ctx->h_shdot[i];
        k_sh_orth<<<grid_n(n), kT, 0, ctx->stream>>>(V, N, j + 1, ctx->d_shdot, wj, n);
        count_launch();
      }
      if ((rc = gdots(ctx, wj, N, 1, wj))) return rc;
      const double hn = std::sqrt(ctx->h_shdot[0]);
      h[j + 1] = hn;
      if (!std::isfinite(hn)) return fail_sh(ctx, LDG_ERR_NONFINITE, "non-finite Arnoldi vector");
      if (hn > 0.0) {
        k_sh_axpby<<<grid_n(n), kT, 0, ctx->stream>>>(1.0 / hn, wj, 0.0, wj, n);
        count_launch();
      }
      // Givens rotations of the new column
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * h[i] + sn[i] * h[i + 1];
        h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
        h[i] = t;
      }
      const double den = std::hypot(h[j], h[j + 1]);
      cs[j] = den > 0.0 ? h[j] / den : 1.0;
      sn[j] = den > 0.0 ? h[j + 1] / den : 0.0;
      h[j] = den;
      h[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      cols = j + 1;
      if (rep) rep->gmres_iters++;
      if (std::fabs(g[j + 1]) <= rtol * bnorm || hn == 0.0) break;
    }
    // y = H^{-1} g (upper triangular), x += V y
    for (int i = cols - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < cols; ++k) s -= H[(size_t)k * (m + 1) + i] * y[k];
      y[i] = s / H[(size_t)i * (m + 1) + i];
    }
    for (int i = 0; i < cols; ++i) {
      k_sh_axpby<<<grid_n(n), kT, 0, ctx->stream>>>(y[i], V + (size_t)i * N, 1.0, x, n);
      count_launch();
    }
    // true residual r = b - J x
    if ((rc = shard_apply(ctx, LDG_STAGE_HOM, x, w))) return rc;
    if (rep) rep->jv_calls++;
    CKS(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    k_sh_axpby<<<grid_n(n), kT, 0, ctx->stream>>>(-1.0, w, 1.0, r, n);
    count_launch();
    CKS(cudaGetLastError());
    if ((rc = gdots(ctx, r, N, 1, r))) return rc;
    beta = std::sqrt(ctx->h_shdot[0]);
    if (rep) rep->lin_resid = beta / bnorm;
    if (!std::isfinite(beta)) return fail_sh(ctx, LDG_ERR_NONFINITE, "non-finite GMRES residual");
    if (beta <= rtol * bnorm * (1.0 + 1e-6)) return LDG_OK;
  }
  return fail_sh(ctx, LDG_ERR_MAXIT, "sharded GMRES did not reach its tolerance within max_restarts cycles");
}

}  // extern "C"
