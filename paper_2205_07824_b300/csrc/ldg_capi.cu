// C-ABI of the LDG hot path (include/ldg.h): context set-up, kernel dispatch,
// residual / J.v entry points, and the matrix-free Newton-GMRES solve of
// Section 3.3 with a device-resident Arnoldi process (classical Gram-Schmidt
// with one re-orthogonalisation pass, Givens rotations, FP64 throughout).
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ldg.h"
#include "ldg_host.h"
#include "ldg_launch.cuh"

using namespace ldg;

struct ldg_ctx {
  int etype = 0, p = 0, nq = 0, dim = 0, npe = 0, ncu = 0, nf = 0, nfq = 0, model = 0;
  int64_t E = 0, ndof = 0;
  ModelParams mp{};
  ldg_options opt{};
  cudaStream_t stream = nullptr;
  const KernelSet* ks = nullptr;
  // device data
  double* d_ops = nullptr;
  double* d_geo = nullptr;
  int* d_nbr = nullptr;
  unsigned char* d_nbf = nullptr;
  unsigned char* d_perm = nullptr;
  double* d_xn = nullptr;      // reference node coordinates [npe][dim]
  double* d_q = nullptr;       // q(u) scratch [E][ncu][dim][npe]
  double* d_dq = nullptr;      // q(v) scratch
  double* d_hist = nullptr;    // BDF history term
  // time scheme
  int scheme = LDG_STEADY;
  double t = 0.0, dt = 1.0, a0dt = 0.0;
  // Krylov work space
  int m = 0;
  double* d_V = nullptr;       // [(m+1)][ndof]
  double* d_r = nullptr;       // [ndof]
  double* d_w = nullptr;       // [ndof]
  double* d_res = nullptr;     // [ndof] Newton residual
  double* d_x = nullptr;       // [ndof] Newton update
  double* d_small = nullptr;   // H, cs, sn, g, y, h, scalars
  double* d_part = nullptr;    // reduction partials [nblk][m+2]
  double* h_pin = nullptr;     // pinned host scalars
  int nblk = 0;
  std::string err;
};

namespace ldg {
long long& launch_counter() {
  static long long n = 0;
  return n;
}
}  // namespace ldg

namespace {

const std::vector<KernelSet>& registry() {
  static std::vector<KernelSet> reg = [] {
    std::vector<KernelSet> r;
    register_tri(r);
    register_quad(r);
    register_hex(r);
    return r;
  }();
  return reg;
}

// Static scratch of ldg_jvp_noalloc: q of the direction v for diffusion models.
// Host code must not use `noalloc_scratch` as an address; the device address is
// looked up once per device with cudaGetSymbolAddress.
constexpr size_t kNoAllocScratchDoubles = (size_t)LDG_NOALLOC_SCRATCH_DOUBLES;
__device__ __align__(256) double noalloc_scratch[kNoAllocScratchDoubles];
constexpr int kMaxDevices = 64;
double* noalloc_addr[kMaxDevices] = {nullptr};

int fail(ldg_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(ctx, LDG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

// small-array offsets in d_small
struct Small {
  int m;
  __host__ __device__ size_t H() const { return 0; }                              // (m+1) x m, column-major
  __host__ __device__ size_t cs() const { return (size_t)(m + 1) * m; }
  __host__ __device__ size_t sn() const { return cs() + m; }
  __host__ __device__ size_t g() const { return sn() + m; }                       // m+1
  __host__ __device__ size_t y() const { return g() + m + 1; }                    // m
  __host__ __device__ size_t h() const { return y() + m; }                        // m+2: first Gram-Schmidt pass
  __host__ __device__ size_t h2() const { return h() + m + 2; }                   // m+2: second pass
  __host__ __device__ size_t sc() const { return h2() + m + 2; }                  // scalars: [0] ||w||^2, [1] |g_{j+1}|, [2] h_{j+1,j}
  __host__ __device__ size_t total() const { return sc() + 8; }
};

// ---------------------------------------------------------------- aux kernels
__global__ void k_interp_nodes(int dim, int npe, int ncu, int64_t E, const double* geo, int GEO, const double* xn,
                               ModelParams mp, double t, double* u) {
  int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (it >= E * npe) return;
  int64_t e = it / npe;
  int n = (int)(it % npe);
  const double* g = geo + e * GEO;
  double x[3] = {0, 0, 0}, st[4] = {0, 0, 0, 0};
  for (int d = 0; d < dim; ++d) {
    double s = g[dim * dim + 1 + d];
    for (int k = 0; k < dim; ++k) s += g[dim * dim + 1 + dim + d * dim + k] * xn[n * dim + k];
    x[d] = s;
  }
  if (dim == 2) exact_state<2>(mp, ncu, x, t, st);
  else exact_state<3>(mp, ncu, x, t, st);
  for (int c = 0; c < ncu; ++c) u[(e * ncu + c) * npe + n] = st[c];
}

__global__ void k_hist(int64_t n, double c1, const double* a, double c2, const double* b, double* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = c1 * a[i] + (b ? c2 * b[i] : 0.0);
}

// Partial dot products of the nvec vectors V[k] (stride ldv) with w:
// part[block][k] = sum over this block's slice of V[k][i] * w[i].
constexpr int RED_T = 256;
__global__ void __launch_bounds__(RED_T) k_multidot(const double* __restrict__ V, int64_t ldv, int nvec,
                                                    const double* __restrict__ w, int64_t n, double* part, int ldp) {
  double acc[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) acc[k] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)RED_T + threadIdx.x; i < n; i += (int64_t)gridDim.x * RED_T) {
    double wi = w[i];
#pragma unroll
    for (int k = 0; k < 32; ++k)
      if (k < nvec) acc[k] += V[k * ldv + i] * wi;
  }
  __shared__ double red[RED_T / 32][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k >= nvec) break;
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < nvec) {
    double s = 0.0;
    for (int q = 0; q < RED_T / 32; ++q) s += red[q][threadIdx.x];
    part[blockIdx.x * (int64_t)ldp + threadIdx.x] = s;
  }
}
// out[k] (=|+=) sum over blocks of part[b][k]; one block, deterministic order.
__global__ void k_reduce_part(const double* part, int nblk, int ldp, int nvec, double* out, int add) {
  __shared__ double red[RED_T];
  for (int k = 0; k < nvec; ++k) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += RED_T) s += part[b * (int64_t)ldp + k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = RED_T / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = add ? out[k] + red[0] : red[0];
    __syncthreads();
  }
}
// w[i] += sgn * sum_k V[k][i] * h[k]
__global__ void k_update(const double* __restrict__ V, int64_t ldv, int nvec, const double* __restrict__ h,
                         double sgn, double* __restrict__ w, int64_t n) {
  __shared__ double hs[32];
  if (threadIdx.x < nvec) hs[threadIdx.x] = sgn * h[threadIdx.x];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = w[i];
    for (int k = 0; k < nvec; ++k) s += V[k * ldv + i] * hs[k];
    w[i] = s;
  }
}
// out = in / sqrt(*nrm2)   (nrm2 holds a squared norm; zero leaves out = 0)
__global__ void k_scale_inv(const double* in, const double* nrm2, double* out, int64_t n) {
  double s = sqrt(*nrm2);
  double f = s > 0.0 ? 1.0 / s : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i] * f;
}
// out = a - b
__global__ void k_sub(const double* a, const double* b, double* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i] - b[i];
}
// Arnoldi column j: H[:, j] = h[0..j], H[j+1][j] = ||w||; apply the previous rotations,
// form the new one, rotate g, and record |g_{j+1}| in sc[1].
__global__ void k_givens(double* small, int m, int j) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Small S{m};
  double* H = small + S.H();
  double* cs = small + S.cs();
  double* sn = small + S.sn();
  double* g = small + S.g();
  const double* h = small + S.h();
  const double* h2 = small + S.h2();
  double* sc = small + S.sc();
  double* col = H + (size_t)j * (m + 1);
  for (int i = 0; i <= j; ++i) col[i] = h[i] + h2[i];
  double hn = sqrt(sc[0]);
  col[j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    double a = col[i], b = col[i + 1];
    col[i] = cs[i] * a + sn[i] * b;
    col[i + 1] = -sn[i] * a + cs[i] * b;
  }
  double a = col[j], b = col[j + 1];
  double den = sqrt(a * a + b * b);
  cs[j] = den > 0.0 ? a / den : 1.0;
  sn[j] = den > 0.0 ? b / den : 0.0;
  col[j] = den;
  col[j + 1] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  sc[1] = fabs(g[j + 1]);
  sc[2] = hn;
}
// y = H[0:k, 0:k]^{-1} g[0:k] (upper triangular)
__global__ void k_backsolve(double* small, int m, int k) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Small S{m};
  const double* H = small + S.H();
  const double* g = small + S.g();
  double* y = small + S.y();
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int l = i + 1; l < k; ++l) s -= H[(size_t)l * (m + 1) + i] * y[l];
    y[i] = s / H[(size_t)i * (m + 1) + i];
  }
}
__global__ void k_init_g(double* small, int m, const double* nrm2) {
  Small S{m};
  double* g = small + S.g();
  for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = 0.0;
  if (threadIdx.x == 0) g[0] = sqrt(*nrm2);
}

KArgs base_args(ldg_ctx* c) {
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.geo = c->d_geo; a.nbr = c->d_nbr; a.nbf = c->d_nbf; a.ops = c->d_ops; a.perm = c->d_perm;
  a.a0dt = c->a0dt; a.t = c->t; a.mp = c->mp; a.E = (int)c->E;
  return a;
}

int64_t grid_for(int64_t n, int t = 256) { return (n + t - 1) / t; }

// ||x||^2 into dst (device scalar)
int dot_into(ldg_ctx* ctx, const double* V, int64_t ldv, int nvec, const double* w, double* dst, int add) {
  k_multidot<<<ctx->nblk, RED_T, 0, ctx->stream>>>(V, ldv, nvec, w, ctx->ndof, ctx->d_part, ctx->m + 2);
  count_launch();
  CK(cudaGetLastError());
  k_reduce_part<<<1, RED_T, 0, ctx->stream>>>(ctx->d_part, ctx->nblk, ctx->m + 2, nvec, dst, add);
  count_launch();
  CK(cudaGetLastError());
  return LDG_OK;
}

int read_scalars(ldg_ctx* ctx, const double* src, int n) {
  CK(cudaMemcpyAsync(ctx->h_pin, src, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return LDG_OK;
}

int do_residual(ldg_ctx* ctx, const double* u, double* r) {
  KArgs a = base_args(ctx);
  if (ctx->ks->qstage) {
    a.u = u; a.out = ctx->d_q;
    CK(ctx->ks->qstage(MODE_R, a, ctx->stream));
    a = base_args(ctx);
    a.q = ctx->d_q;
  }
  a.u = u; a.out = r;
  a.hist = ctx->scheme != LDG_STEADY ? ctx->d_hist : nullptr;
  CK(ctx->ks->residual(MODE_R, a, ctx->stream));
  return LDG_OK;
}

int do_jvp(ldg_ctx* ctx, const double* u, const double* v, double* jv) {
  KArgs a = base_args(ctx);
  if (ctx->ks->qstage) {
    // linear model: J v = R(v) - R(0), the homogeneous operator applied to v
    a.u = v; a.out = ctx->d_dq;
    CK(ctx->ks->qstage(MODE_HOM, a, ctx->stream));
    a = base_args(ctx);
    a.u = v; a.q = ctx->d_dq; a.out = jv;
    CK(ctx->ks->residual(MODE_HOM, a, ctx->stream));
  } else {
    a.u = u; a.v = v; a.out = jv;
    CK(ctx->ks->residual(MODE_JV, a, ctx->stream));
  }
  return LDG_OK;
}

// GMRES(m) on J(u) x = b, x0 = 0, to ||b - J x|| <= rtol ||b||.
int do_gmres(ldg_ctx* ctx, const double* u, const double* b, double* x, double rtol, ldg_solve_report* rep) {
  const int m = ctx->m;
  const int64_t n = ctx->ndof;
  Small S{m};
  double* sm = ctx->d_small;
  double* V = ctx->d_V;
  int rc;
  CK(cudaMemsetAsync(x, 0, n * sizeof(double), ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  if ((rc = dot_into(ctx, ctx->d_r, n, 1, ctx->d_r, sm + S.sc(), 0))) return rc;
  if ((rc = read_scalars(ctx, sm + S.sc(), 1))) return rc;
  const double bnorm = std::sqrt(ctx->h_pin[0]);
  if (!std::isfinite(bnorm)) return fail(ctx, LDG_ERR_NONFINITE, "non-finite right-hand side");
  if (rep) rep->lin_resid = 0.0;
  if (bnorm == 0.0) return LDG_OK;
  const int64_t g1 = std::min<int64_t>(grid_for(n), 148 * 8);
  double beta = bnorm;
  for (int cycle = 0; cycle < ctx->opt.max_restarts; ++cycle) {
    // V[0] = r / ||r||, g = (||r||, 0, ...); sc[0] holds ||r||^2
    k_scale_inv<<<g1, 256, 0, ctx->stream>>>(ctx->d_r, sm + S.sc(), V, n);
    count_launch();
    k_init_g<<<1, 64, 0, ctx->stream>>>(sm, m, sm + S.sc());
    count_launch();
    CK(cudaGetLastError());
    int j = 0;
    bool done = false;
    for (; j < m; ++j) {
      double* w = V + (size_t)(j + 1) * n;
      if ((rc = do_jvp(ctx, u, V + (size_t)j * n, w))) return rc;
      if (rep) { rep->jv_calls++; rep->gmres_iters++; }
      // classical Gram-Schmidt with one re-orthogonalisation pass
      if ((rc = dot_into(ctx, V, n, j + 1, w, sm + S.h(), 0))) return rc;
      k_update<<<g1, 256, 0, ctx->stream>>>(V, n, j + 1, sm + S.h(), -1.0, w, n);
      count_launch();
      CK(cudaGetLastError());
      if ((rc = dot_into(ctx, V, n, j + 1, w, sm + S.h2(), 0))) return rc;
      k_update<<<g1, 256, 0, ctx->stream>>>(V, n, j + 1, sm + S.h2(), -1.0, w, n);
      count_launch();
      CK(cudaGetLastError());
      if ((rc = dot_into(ctx, w, n, 1, w, sm + S.sc(), 0))) return rc;
      k_givens<<<1, 1, 0, ctx->stream>>>(sm, m, j);
      count_launch();
      k_scale_inv<<<g1, 256, 0, ctx->stream>>>(w, sm + S.sc(), w, n);
      count_launch();
      CK(cudaGetLastError());
      if ((rc = read_scalars(ctx, sm + S.sc(), 3))) return rc;
      const double est = ctx->h_pin[1], hn = ctx->h_pin[2];
      if (!std::isfinite(est)) return fail(ctx, LDG_ERR_NONFINITE, "non-finite Arnoldi quantity");
      if (est <= rtol * bnorm || hn == 0.0) { ++j; done = true; break; }
    }
    if (j == m) done = false;
    // x += V y
    k_backsolve<<<1, 1, 0, ctx->stream>>>(sm, m, j);
    count_launch();
    k_update<<<g1, 256, 0, ctx->stream>>>(V, n, j, sm + S.y(), 1.0, x, n);
    count_launch();
    CK(cudaGetLastError());
    // true residual r = b - J x
    if ((rc = do_jvp(ctx, u, x, ctx->d_w))) return rc;
    if (rep) rep->jv_calls++;
    k_sub<<<g1, 256, 0, ctx->stream>>>(b, ctx->d_w, ctx->d_r, n);
    count_launch();
    CK(cudaGetLastError());
    if ((rc = dot_into(ctx, ctx->d_r, n, 1, ctx->d_r, sm + S.sc(), 0))) return rc;
    if ((rc = read_scalars(ctx, sm + S.sc(), 1))) return rc;
    beta = std::sqrt(ctx->h_pin[0]);
    if (rep) rep->lin_resid = beta / bnorm;
    if (!std::isfinite(beta)) return fail(ctx, LDG_ERR_NONFINITE, "non-finite GMRES residual");
    if (beta <= rtol * bnorm * (1.0 + 1e-6) || (done && beta <= rtol * bnorm * 10.0)) return LDG_OK;
  }
  return fail(ctx, LDG_ERR_MAXIT, "GMRES did not reach its tolerance within max_restarts cycles");
}

int do_newton(ldg_ctx* ctx, double* u, ldg_solve_report* rep) {
  const int64_t n = ctx->ndof;
  Small S{ctx->m};
  double* sm = ctx->d_small;
  int rc;
  auto t0 = std::chrono::steady_clock::now();
  double* res = ctx->d_res;   // R(u_k), the right-hand side of each linear solve
  double* del = ctx->d_x;     // Newton update
  if ((rc = do_residual(ctx, u, res))) return rc;
  if (rep) rep->residual_calls++;
  if ((rc = dot_into(ctx, res, n, 1, res, sm + S.sc() + 4, 0))) return rc;
  if ((rc = read_scalars(ctx, sm + S.sc() + 4, 1))) return rc;
  const double r0 = std::sqrt(ctx->h_pin[0]);
  double rn = r0;
  if (rep) rep->r0 = r0;
  if (!std::isfinite(r0)) return fail(ctx, LDG_ERR_NONFINITE, "non-finite initial residual");
  int k = 0;
  const int64_t g1 = std::min<int64_t>(grid_for(n), 148 * 8);
  while (rn > ctx->opt.newton_rtol * r0 && k < ctx->opt.max_newton) {
    if ((rc = do_gmres(ctx, u, res, del, ctx->opt.gmres_rtol, rep)) && rc != LDG_ERR_MAXIT) return rc;
    // u <- u - delta   (sc[6] holds -1)
    k_update<<<g1, 256, 0, ctx->stream>>>(del, n, 1, sm + S.sc() + 6, 1.0, u, n);
    count_launch();
    CK(cudaGetLastError());
    if ((rc = do_residual(ctx, u, res))) return rc;
    if (rep) rep->residual_calls++;
    if ((rc = dot_into(ctx, res, n, 1, res, sm + S.sc() + 4, 0))) return rc;
    if ((rc = read_scalars(ctx, sm + S.sc() + 4, 1))) return rc;
    rn = std::sqrt(ctx->h_pin[0]);
    if (!std::isfinite(rn)) return fail(ctx, LDG_ERR_NONFINITE, "non-finite residual after a Newton step");
    ++k;
  }
  if (rep) {
    rep->newton_iters = k;
    rep->rfinal = rn;
    rep->elapsed_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  if (rn > ctx->opt.newton_rtol * r0) return fail(ctx, LDG_ERR_MAXIT, "Newton did not converge within max_newton");
  return LDG_OK;
}

}  // namespace

// ===================================================================== C ABI
extern "C" {

const char* ldg_version(void) { return "ldg-b300 0.1 (sm_103a)"; }

int64_t ldg_kernel_launches(void) { return (int64_t)launch_counter(); }

const char* ldg_last_error(const ldg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int ldg_destroy(ldg_ctx* ctx) {
  if (!ctx) return LDG_OK;
  cudaFree(ctx->d_ops); cudaFree(ctx->d_geo); cudaFree(ctx->d_nbr); cudaFree(ctx->d_nbf); cudaFree(ctx->d_perm);
  cudaFree(ctx->d_xn); cudaFree(ctx->d_q); cudaFree(ctx->d_dq); cudaFree(ctx->d_hist);
  cudaFree(ctx->d_V); cudaFree(ctx->d_r); cudaFree(ctx->d_w); cudaFree(ctx->d_res); cudaFree(ctx->d_x); cudaFree(ctx->d_small); cudaFree(ctx->d_part);
  if (ctx->h_pin) cudaFreeHost(ctx->h_pin);
  delete ctx;
  return LDG_OK;
}

int ldg_create(ldg_ctx** out, const ldg_mesh_desc* mesh, int p, const ldg_model_desc* model, const ldg_options* opts,
               void* cuda_stream) {
  if (!out || !mesh || !model || !mesh->xyz || !mesh->vid || mesh->n_elem <= 0) return LDG_ERR_ARG;
  *out = nullptr;
  ldg_ctx* ctx = new ldg_ctx();
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->etype = mesh->elem_type;
  ctx->model = model->model;
  if (ctx->etype < 0 || ctx->etype > 2 || ctx->model < 0 || ctx->model > 2) {
    ldg_destroy(ctx);
    return LDG_ERR_ARG;
  }
  ctx->dim = ctx->etype == LDG_HEX ? 3 : 2;
  if (ctx->model == LDG_EULER && ctx->dim != 2) { ldg_destroy(ctx); return LDG_ERR_UNSUPPORTED; }
  ctx->ncu = ctx->model == LDG_EULER ? 4 : 1;
  ldg_options o{};
  if (opts) o = *opts;
  if (o.nq1 <= 0) o.nq1 = (ctx->model == LDG_EULER || ctx->etype == LDG_TRI) ? p + 2 : p + 1;
  if (o.gmres_m <= 0) o.gmres_m = 30;
  if (o.gmres_m > 30) o.gmres_m = 30;
  if (o.max_restarts <= 0) o.max_restarts = 50;
  if (o.max_newton <= 0) o.max_newton = 20;
  if (o.newton_rtol <= 0) o.newton_rtol = 1e-8;
  if (o.gmres_rtol <= 0) o.gmres_rtol = 1e-3;
  ctx->opt = o;
  ctx->p = p; ctx->nq = o.nq1;
  // model parameters
  ModelParams mp{};
  mp.kappa = 1.0; mp.tau = 1.0; mp.gamma = 1.4; mp.cas = model->case_id;
  const double* mu = model->mu;
  int nmu = mu ? model->n_mu : 0;
  if (ctx->model == LDG_EULER) { if (nmu > 0) mp.gamma = mu[0]; }
  else {
    if (nmu > 0) mp.kappa = mu[0];
    if (nmu > 1) mp.tau = mu[1];
    for (int d = 0; d < 3; ++d) if (nmu > 2 + d) mp.beta[d] = mu[2 + d];
  }
  ctx->mp = mp;
  for (const KernelSet& k : registry())
    if (k.etype == ctx->etype && k.p == p && k.nq == o.nq1 && k.model == ctx->model) ctx->ks = &k;
  if (!ctx->ks) {
    ctx->err = "no compiled kernel for element " + std::to_string(ctx->etype) + ", p " + std::to_string(p) +
               ", nq1 " + std::to_string(o.nq1) + ", model " + std::to_string(ctx->model);
    *out = ctx;
    return LDG_ERR_UNSUPPORTED;
  }
  RefOps ref;
  MeshPrep mp_;
  std::string err;
  if (!build_ref_ops(ctx->etype, p, o.nq1, ref, err)) { ctx->err = err; *out = ctx; return LDG_ERR_ARG; }
  if (!prepare_mesh(ref, mesh->n_elem, mesh->xyz, mesh->vid, mp_, err)) { ctx->err = err; *out = ctx; return LDG_ERR_MESH; }
  if (mesh->n_elem > (int64_t)0x7fffffff) { ctx->err = "too many elements"; *out = ctx; return LDG_ERR_ARG; }
  ctx->E = mesh->n_elem;
  ctx->npe = ref.npe; ctx->nf = ref.nf; ctx->nfq = ref.nfq;
  ctx->ndof = ctx->E * ctx->npe * ctx->ncu;
  ctx->m = o.gmres_m;
  std::vector<double> xn;
  ref_nodes(ref, xn);
  *out = ctx;
  const int64_t n = ctx->ndof;
  CK(cudaMalloc(&ctx->d_ops, ref.blob.size() * sizeof(double)));
  CK(cudaMalloc(&ctx->d_geo, mp_.geo.size() * sizeof(double)));
  CK(cudaMalloc(&ctx->d_nbr, mp_.nbr.size() * sizeof(int)));
  CK(cudaMalloc(&ctx->d_nbf, mp_.nbf.size()));
  CK(cudaMalloc(&ctx->d_perm, mp_.perm.size()));
  CK(cudaMalloc(&ctx->d_xn, xn.size() * sizeof(double)));
  CK(cudaMemcpy(ctx->d_ops, ref.blob.data(), ref.blob.size() * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_geo, mp_.geo.data(), mp_.geo.size() * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_nbr, mp_.nbr.data(), mp_.nbr.size() * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_nbf, mp_.nbf.data(), mp_.nbf.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_perm, mp_.perm.data(), mp_.perm.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_xn, xn.data(), xn.size() * sizeof(double), cudaMemcpyHostToDevice));
  if (ctx->ks->qstage) {
    CK(cudaMalloc(&ctx->d_q, n * ctx->dim * sizeof(double)));
    CK(cudaMalloc(&ctx->d_dq, n * ctx->dim * sizeof(double)));
  }
  CK(cudaMalloc(&ctx->d_hist, n * sizeof(double)));
  CK(cudaMalloc(&ctx->d_V, (size_t)(ctx->m + 1) * n * sizeof(double)));
  CK(cudaMalloc(&ctx->d_r, n * sizeof(double)));
  CK(cudaMalloc(&ctx->d_w, n * sizeof(double)));
  CK(cudaMalloc(&ctx->d_res, n * sizeof(double)));
  CK(cudaMalloc(&ctx->d_x, n * sizeof(double)));
  Small S{ctx->m};
  CK(cudaMalloc(&ctx->d_small, S.total() * sizeof(double)));
  CK(cudaMemset(ctx->d_small, 0, S.total() * sizeof(double)));
  ctx->nblk = 148 * 4;
  CK(cudaMalloc(&ctx->d_part, (size_t)ctx->nblk * (ctx->m + 2) * sizeof(double)));
  CK(cudaMallocHost(&ctx->h_pin, 16 * sizeof(double)));
  // the Newton update uses sc[6] = -1 as its axpy coefficient
  double minus1 = -1.0;
  CK(cudaMemcpy(ctx->d_small + S.sc() + 6, &minus1, sizeof(double), cudaMemcpyHostToDevice));
  return LDG_OK;
}

int ldg_set_stream(ldg_ctx* ctx, void* s) {
  if (!ctx) return LDG_ERR_ARG;
  ctx->stream = (cudaStream_t)s;
  return LDG_OK;
}

int ldg_sizes(const ldg_ctx* ctx, int64_t* n_dof, int* n_pe, int* n_cu, int* dim) {
  if (!ctx || !ctx->ks) return LDG_ERR_ARG;
  if (n_dof) *n_dof = ctx->ndof;
  if (n_pe) *n_pe = ctx->npe;
  if (n_cu) *n_cu = ctx->ncu;
  if (dim) *dim = ctx->dim;
  return LDG_OK;
}

int ldg_set_time(ldg_ctx* ctx, int scheme, double t, double dt, const double* un, const double* unm1) {
  if (!ctx || !ctx->ks) return LDG_ERR_ARG;
  ctx->t = t;
  if (scheme == LDG_STEADY) { ctx->scheme = scheme; ctx->a0dt = 0.0; return LDG_OK; }
  if ((scheme != LDG_BDF1 && scheme != LDG_BDF2) || !(dt > 0) || !un || (scheme == LDG_BDF2 && !unm1))
    return fail(ctx, LDG_ERR_ARG, "ldg_set_time: bad scheme, step or history");
  ctx->scheme = scheme;
  ctx->dt = dt;
  double a0 = scheme == LDG_BDF1 ? 1.0 : 1.5, a1 = scheme == LDG_BDF1 ? -1.0 : -2.0, a2 = scheme == LDG_BDF1 ? 0.0 : 0.5;
  ctx->a0dt = a0 / dt;
  k_hist<<<grid_for(ctx->ndof), 256, 0, ctx->stream>>>(ctx->ndof, a1 / dt, un, a2 / dt, scheme == LDG_BDF2 ? unm1 : nullptr,
                                                      ctx->d_hist);
  count_launch();
  CK(cudaGetLastError());
  return LDG_OK;
}

int ldg_residual(ldg_ctx* ctx, const double* u, double* r) {
  if (!ctx || !ctx->ks || !u || !r) return LDG_ERR_ARG;
  return do_residual(ctx, u, r);
}

int ldg_jvp(ldg_ctx* ctx, const double* u, const double* v, double* jv) {
  if (!ctx || !ctx->ks || !u || !v || !jv) return LDG_ERR_ARG;
  return do_jvp(ctx, u, v, jv);
}

int ldg_q(ldg_ctx* ctx, const double* u, double* q) {
  if (!ctx || !ctx->ks || !u || !q) return LDG_ERR_ARG;
  if (!ctx->ks->qstage) return fail(ctx, LDG_ERR_ARG, "the model has no q (convection model)");
  KArgs a = base_args(ctx);
  a.u = u; a.out = q;
  CK(ctx->ks->qstage(MODE_R, a, ctx->stream));
  return LDG_OK;
}

int ldg_interpolate(ldg_ctx* ctx, double t, double* u) {
  if (!ctx || !ctx->ks || !u) return LDG_ERR_ARG;
  const int GEO = ctx->dim * ctx->dim * 2 + 1 + ctx->dim + ctx->nf * (ctx->dim + 1);
  k_interp_nodes<<<grid_for(ctx->E * ctx->npe), 256, 0, ctx->stream>>>(ctx->dim, ctx->npe, ctx->ncu, ctx->E, ctx->d_geo,
                                                                      GEO, ctx->d_xn, ctx->mp, t, u);
  count_launch();
  CK(cudaGetLastError());
  return LDG_OK;
}

int ldg_gmres(ldg_ctx* ctx, const double* u, const double* b, double* x, ldg_solve_report* rep) {
  if (!ctx || !ctx->ks || !u || !b || !x) return LDG_ERR_ARG;
  if (rep) std::memset(rep, 0, sizeof(*rep));
  auto t0 = std::chrono::steady_clock::now();
  int rc = do_gmres(ctx, u, b, x, ctx->opt.gmres_rtol, rep);
  if (rep) {
    rep->status = rc;
    rep->elapsed_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return rc;
}

int ldg_newton_gmres(ldg_ctx* ctx, double* u, ldg_solve_report* rep) {
  if (!ctx || !ctx->ks || !u) return LDG_ERR_ARG;
  ldg_solve_report local{};
  if (!rep) rep = &local;
  std::memset(rep, 0, sizeof(*rep));
  int rc = do_newton(ctx, u, rep);
  rep->status = rc;
  return rc;
}

int ldg_jvp_noalloc(ldg_ctx* ctx, const double* u, const double* v, double* jv) {
  if (!ctx || !ctx->ks || !u || !v || !jv) return LDG_ERR_ARG;
  if (!ctx->ks->qstage) {
    // convection models need no scratch: the dual-number kernel reads u, v and writes jv only
    KArgs a = base_args(ctx);
    a.u = u; a.v = v; a.out = jv;
    CK(ctx->ks->residual(MODE_JV, a, ctx->stream));
    return LDG_OK;
  }
  const size_t need = (size_t)ctx->ndof * ctx->dim;
  if (need > kNoAllocScratchDoubles)
    return fail(ctx, LDG_ERR_ARG, "ldg_jvp_noalloc: this operator needs " + std::to_string(need) +
                                      " doubles of scratch (n_dof * dim), more than the static maximum of " +
                                      std::to_string(kNoAllocScratchDoubles));
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(ctx, LDG_ERR_ARG, "ldg_jvp_noalloc: device ordinal out of range");
  if (!noalloc_addr[dev]) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, noalloc_scratch));
    noalloc_addr[dev] = (double*)p;
  }
  double* dq = noalloc_addr[dev];
  // q(v) of the homogeneous operator overwrites every entry it later reads: nothing to clear
  KArgs a = base_args(ctx);
  a.u = v; a.out = dq;
  CK(ctx->ks->qstage(MODE_HOM, a, ctx->stream));
  a = base_args(ctx);
  a.u = v; a.q = dq; a.out = jv;
  CK(ctx->ks->residual(MODE_HOM, a, ctx->stream));
  return LDG_OK;
}

int ldg_newton_gmres_host(ldg_ctx* ctx, double* u_host, ldg_solve_report* rep) {
  if (!ctx || !ctx->ks || !u_host) return LDG_ERR_ARG;
  const size_t bytes = ctx->ndof * sizeof(double);
  double* du = nullptr;
  CK(cudaMallocAsync(&du, bytes, ctx->stream));
  CK(cudaMemcpyAsync(du, u_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
  int rc = ldg_newton_gmres(ctx, du, rep);
  cudaError_t e1 = cudaMemcpyAsync(u_host, du, bytes, cudaMemcpyDeviceToHost, ctx->stream);
  cudaError_t e2 = cudaFreeAsync(du, ctx->stream);
  cudaError_t e3 = cudaStreamSynchronize(ctx->stream);
  if (rc) return rc;
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) return fail(ctx, LDG_ERR_CUDA, "host copy-back failed");
  return LDG_OK;
}

}  // extern "C"
