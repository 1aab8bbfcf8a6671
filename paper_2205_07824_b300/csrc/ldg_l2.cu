// L2 projection of the analytic field and relative L2 errors of u_h and q_h
// (Section 4.1: the errors E(u_h), E(q_h) of Table 3), on affine elements.
//
// Both use a richer reference rule than the operator's: Gauss with p + 3 points per
// direction (collapsed on simplices), built once per context. On an affine element
// the mass matrix is det J times the reference one, so the projection is
//   u_K = Mref^{-1} B^T W g(x_K(xi))      (one reference operator for every element)
// and the errors are
//   E(u_h) = sqrt( sum_K sum_k w_k det J |u_h - u|^2 / sum_K sum_k w_k det J |u|^2 ),
//   E(q_h) likewise with q = -grad u, q_h from the q-stage (Eq. 1a).
// One CTA per element evaluates its points; per-element partial sums are added in
// element order by a single CTA, so the result does not depend on the launch.
#include <cmath>
#include <string>
#include <vector>

#include "../../include/ldg.h"
#include "ldg_ctx.h"
#include "ldg_host.h"

using namespace ldg;

namespace {

constexpr int kThreads = 128;

int fail_l2(ldg_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CKL(call)                                                                                \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return fail_l2(ctx, LDG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

// physical point x = x(0) + J xi of an affine element's geometry record
template <int DIM> __device__ __forceinline__ void affine_x(const double* g, const double* xi, double* x) {
  for (int d = 0; d < DIM; ++d) {
    double s = g[Geo<DIM>::XM + d];
    for (int k = 0; k < DIM; ++k) s += g[Geo<DIM>::JAC + d * DIM + k] * xi[k];
    x[d] = s;
  }
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) k_project(int npe, int ncu, int nqp, int GEO, const double* geo,
                                                     const double* xi, const double* P, ModelParams mp, double t,
                                                     double* u) {
  extern __shared__ double gq[];   // [ncu][nqp] exact field at the rule's points
  const int64_t e = blockIdx.x;
  const double* g = geo + e * GEO;
  for (int k = threadIdx.x; k < nqp; k += blockDim.x) {
    double x[3] = {0.0, 0.0, 0.0}, st[4] = {0.0, 0.0, 0.0, 0.0};
    affine_x<DIM>(g, xi + (size_t)k * DIM, x);
    exact_state<DIM>(mp, ncu, x, t, st);
    for (int c = 0; c < ncu; ++c) gq[c * nqp + k] = st[c];
  }
  __syncthreads();
  for (int it = threadIdx.x; it < ncu * npe; it += blockDim.x) {
    const int c = it / npe, i = it - c * npe;
    const double* Pi = P + (size_t)i * nqp;
    const double* gc = gq + c * nqp;
    double s = 0.0;
    for (int k = 0; k < nqp; ++k) s += Pi[k] * gc[k];
    u[((size_t)e * ncu + c) * npe + i] = s;
  }
}

// part[e][0..3] = element sums of w det J (|u_h - u|^2, |u|^2, |q_h - q|^2, |q|^2)
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_l2_err(int npe, int ncu, int nqp, int GEO, const double* geo,
                                                    const double* xi, const double* w, const double* B,
                                                    const double* u, const double* q, ModelParams mp, double t,
                                                    double* part) {
  __shared__ double red[4][kThreads];
  const int64_t e = blockIdx.x;
  const double* g = geo + e * GEO;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = threadIdx.x; k < nqp; k += blockDim.x) {
    double x[3] = {0.0, 0.0, 0.0}, st[4] = {0.0, 0.0, 0.0, 0.0};
    affine_x<DIM>(g, xi + (size_t)k * DIM, x);
    exact_state<DIM>(mp, ncu, x, t, st);
    const double wj = w[k] * g[Geo<DIM>::DETJ];
    const double* Bk = B + (size_t)k * npe;
    for (int c = 0; c < ncu; ++c) {
      const double* uc = u + ((size_t)e * ncu + c) * npe;
      double uh = 0.0;
      for (int i = 0; i < npe; ++i) uh += Bk[i] * uc[i];
      s[0] += wj * (uh - st[c]) * (uh - st[c]);
      s[1] += wj * st[c] * st[c];
    }
    if (q) {
      double grad[3], lap;
      scalar_derivs<DIM>(mp, x, grad, lap);
      for (int d = 0; d < DIM; ++d) {
        const double* qd = q + ((size_t)e * DIM + d) * npe;
        double qh = 0.0;
        for (int i = 0; i < npe; ++i) qh += Bk[i] * qd[i];
        const double qe = -grad[d];
        s[2] += wj * (qh - qe) * (qh - qe);
        s[3] += wj * qe * qe;
      }
    }
  }
  for (int j = 0; j < 4; ++j) red[j][threadIdx.x] = s[j];
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int j = 0; j < 4; ++j) red[j][threadIdx.x] += red[j][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < 4) part[e * 4 + threadIdx.x] = red[threadIdx.x][0];
}

// out[0] = E(u_h), out[1] = E(q_h) (0 without q): the element partials summed in a fixed order
__global__ void __launch_bounds__(256) k_l2_finish(int64_t E, const double* part, int hasq, double* out) {
  __shared__ double red[4][256];
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t e = threadIdx.x; e < E; e += blockDim.x)
    for (int j = 0; j < 4; ++j) s[j] += part[e * 4 + j];
  for (int j = 0; j < 4; ++j) red[j][threadIdx.x] = s[j];
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
      for (int j = 0; j < 4; ++j) red[j][threadIdx.x] += red[j][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sqrt(red[0][0] / (red[1][0] > 0.0 ? red[1][0] : 1.0));
    out[1] = hasq ? sqrt(red[2][0] / (red[3][0] > 0.0 ? red[3][0] : 1.0)) : 0.0;
  }
}

// Builds and uploads the context's error rule on first use.
int ensure_err_rule(ldg_ctx* ctx) {
  if (ctx->d_er_P) return LDG_OK;
  if (ctx->pg > 0)
    return fail_l2(ctx, LDG_ERR_UNSUPPORTED, "L2 projection and errors are built for affine elements only");
  ErrRule R;
  std::string err;
  if (!build_err_rule(ctx->etype, ctx->p, ctx->p + 3, R, err)) return fail_l2(ctx, LDG_ERR_UNSUPPORTED, err);
  auto up = [&](double** dst, const std::vector<double>& v) -> cudaError_t {
    cudaError_t e = cudaMalloc(dst, v.size() * sizeof(double));
    return e ? e : cudaMemcpy(*dst, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice);
  };
  CKL(up(&ctx->d_er_xi, R.xi));
  CKL(up(&ctx->d_er_w, R.w));
  CKL(up(&ctx->d_er_B, R.B));
  CKL(up(&ctx->d_er_P, R.P));
  CKL(cudaMalloc(&ctx->d_l2, ((size_t)ctx->E * 4 + 2) * sizeof(double)));
  ctx->er_nqp = R.nqp;
  return LDG_OK;
}

int geo_len(const ldg_ctx* ctx) { return ctx->dim == 2 ? Geo<2>::size(ctx->nf) : Geo<3>::size(ctx->nf); }

}  // namespace

extern "C" {

int ldg_project(ldg_ctx* ctx, double t, double* u) {
  if (!ctx || !ctx->ks || !u) return LDG_ERR_ARG;
  int rc = ensure_err_rule(ctx);
  if (rc) return rc;
  const size_t smem = (size_t)ctx->ncu * ctx->er_nqp * sizeof(double);
  if (ctx->dim == 2)
    k_project<2><<<(unsigned)ctx->E, kThreads, smem, ctx->stream>>>(ctx->npe, ctx->ncu, ctx->er_nqp, geo_len(ctx),
                                                                    ctx->d_geo, ctx->d_er_xi, ctx->d_er_P, ctx->mp,
                                                                    t, u);
  else
    k_project<3><<<(unsigned)ctx->E, kThreads, smem, ctx->stream>>>(ctx->npe, ctx->ncu, ctx->er_nqp, geo_len(ctx),
                                                                    ctx->d_geo, ctx->d_er_xi, ctx->d_er_P, ctx->mp,
                                                                    t, u);
  count_launch();
  CKL(cudaGetLastError());
  return LDG_OK;
}

int ldg_l2_error(ldg_ctx* ctx, const double* u, double t, double* err_u, double* err_q) {
  if (!ctx || !ctx->ks || !u || !err_u) return LDG_ERR_ARG;
  int rc = ensure_err_rule(ctx);
  if (rc) return rc;
  const bool hasq = ctx->model == LDG_POISSON || ctx->model == LDG_CONVDIFF;
  if (hasq && (rc = ldg_q(ctx, u, ctx->d_q))) return rc;
  const double* q = hasq ? ctx->d_q : nullptr;
  if (ctx->dim == 2)
    k_l2_err<2><<<(unsigned)ctx->E, kThreads, 0, ctx->stream>>>(ctx->npe, ctx->ncu, ctx->er_nqp, geo_len(ctx),
                                                               ctx->d_geo, ctx->d_er_xi, ctx->d_er_w, ctx->d_er_B, u,
                                                               q, ctx->mp, t, ctx->d_l2);
  else
    k_l2_err<3><<<(unsigned)ctx->E, kThreads, 0, ctx->stream>>>(ctx->npe, ctx->ncu, ctx->er_nqp, geo_len(ctx),
                                                               ctx->d_geo, ctx->d_er_xi, ctx->d_er_w, ctx->d_er_B, u,
                                                               q, ctx->mp, t, ctx->d_l2);
  count_launch();
  CKL(cudaGetLastError());
  double* out = ctx->d_l2 + (size_t)ctx->E * 4;
  k_l2_finish<<<1, 256, 0, ctx->stream>>>(ctx->E, ctx->d_l2, hasq ? 1 : 0, out);
  count_launch();
  CKL(cudaGetLastError());
  double h[2];
  CKL(cudaMemcpyAsync(h, out, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CKL(cudaStreamSynchronize(ctx->stream));
  *err_u = h[0];
  if (err_q) *err_q = h[1];
  return LDG_OK;
}

}  // extern "C"
