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
#include "ldg_krylov.cuh"
#include "ldg_precond.cuh"
#include "ldg_mlp.cuh"
#include "ldg_tc.cuh"
#include <cudaTypedefs.h>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <random>
#include <map>
#include <numeric>
#include <tuple>
#include <type_traits>
#include "ldg_launch.cuh"
#include "ldg_ctx.h"

using namespace ldg;


namespace ldg {
void register_all(std::vector<KernelSet>& reg) {
  // Tile0 first: the default instance of every (element, order, model)
  register_tri_t<Tile0>(reg); register_quad_t<Tile0>(reg); register_hex_t<Tile0>(reg); register_ns_t<Tile0>(reg);
  register_tri_t<Tile1>(reg); register_quad_t<Tile1>(reg); register_hex_t<Tile1>(reg); register_ns_t<Tile1>(reg);
  register_tri_t<Tile2>(reg); register_quad_t<Tile2>(reg); register_hex_t<Tile2>(reg); register_ns_t<Tile2>(reg);
  register_tri_t<Tile3>(reg); register_quad_t<Tile3>(reg); register_hex_t<Tile3>(reg); register_ns_t<Tile3>(reg);
  // tetrahedra and curved elements: two tile shapes
  register_tet_t<Tile0>(reg); register_tet_t<Tile1>(reg);
  register_curved_scalar_t<Tile0>(reg); register_curved_gas_t<Tile0>(reg); register_curved_tri_t<Tile0>(reg);
  register_curved_scalar_t<Tile1>(reg); register_curved_gas_t<Tile1>(reg); register_curved_tri_t<Tile1>(reg);
}
std::atomic<long long>& launch_counter() {
  static std::atomic<long long> n{0};
  return n;
}
}  // namespace ldg

namespace ldg {
namespace impl {

const std::vector<KernelSet>& registry() {
  static std::vector<KernelSet> reg = [] {
    std::vector<KernelSet> r;
    register_all(r);
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
// Per-device address cache, filled under a lock on the first call on that device
// (two host threads may make their first calls at once).
std::atomic<double*> noalloc_addr[kMaxDevices];
std::mutex noalloc_lock;

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

// ---------------------------------------------------------------- aux kernels
// xnode (curved elements): physical node coordinates [E][npe][dim]; else the affine map
__global__ void k_interp_nodes(int dim, int npe, int ncu, int64_t E, const double* geo, int GEO, const double* xn,
                               ModelParams mp, double t, double* u, const double* xnode) {
  int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (it >= E * npe) return;
  int64_t e = it / npe;
  int n = (int)(it % npe);
  const double* g = geo + e * GEO;
  double x[3] = {0, 0, 0}, st[4] = {0, 0, 0, 0};
  for (int d = 0; d < dim; ++d) {
    double s = g[dim * dim + 1 + d];
    for (int k = 0; k < dim; ++k) s += g[dim * dim + 1 + dim + d * dim + k] * xn[n * dim + k];
    x[d] = xnode ? xnode[it * dim + d] : s;
  }
  if (dim == 2) exact_state<2>(mp, ncu, x, t, st);
  else exact_state<3>(mp, ncu, x, t, st);
  for (int c = 0; c < ncu; ++c) u[(e * ncu + c) * npe + n] = st[c];
}

__global__ void k_set_scalar(double* dst, double v) { *dst = v; }

__global__ void k_hist(int64_t n, double c1, const double* a, double c2, const double* b, double* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = c1 * a[i] + (b ? c2 * b[i] : 0.0);
}

// Finite-difference step eps = sqrt(2^-52) (1 + ||u||) / ||v|| from the squared norms
// nn = (u.u, v.v): eps[0] = eps, eps[1] = -eps, eps[2] = the difference's weight.
__global__ void k_fd_eps(const double* nn, double* eps, int order) {
  const double nu = sqrt(nn[0]), nv = sqrt(nn[1]);
  const double e = nv > 0.0 ? 1.4901161193847656e-08 * (1.0 + nu) / nv : 0.0;
  eps[0] = e;
  eps[1] = -e;
  eps[2] = e > 0.0 ? (order == 2 ? 0.5 / e : 1.0 / e) : 0.0;
}
// out = (a - b) * s[0]
__global__ void k_fd_diff(const double* a, const double* b, const double* s, double* out, int64_t n) {
  const double w = *s;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (a[i] - b[i]) * w;
}

KArgs base_args(ldg_ctx* c) {
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.geo = c->d_geo; a.nbr = c->d_nbr; a.nbf = c->d_nbf; a.ops = c->d_ops; a.opsf = c->d_opsf; a.perm = c->d_perm;
  a.lops = c->d_lops; a.lopsf = c->d_lopsf; a.lops_host = c->h_lops.empty() ? nullptr : c->h_lops.data();
  a.a0dt = c->a0dt; a.t = c->t; a.mp = c->mp; a.E = (int)c->E;
  a.inst = c->ext_inst; a.mtab = c->ext_mtab; a.t_dev = c->d_t;
  a.cgeo = c->d_cgeo; a.cgeof = c->d_cgeof; a.cx = c->d_cx; a.minv = c->d_minv; a.minvf = c->d_minvf;
  a.radd = c->radd_on ? c->d_radd : nullptr;
  a.blk_col = -1;
  return a;
}

int64_t grid_for(int64_t n, int t) { return (n + t - 1) / t; }

constexpr int LDP = 32;   // leading dimension of the reduction partials

// out[k] = V[k] . w for k < nvec (device), optionally skipped when flags[0] is set
int dots(ldg_ctx* ctx, const double* V, int64_t ldv, int nvec, const double* w, double* out, const int* flags) {
  const int64_t n = ctx->ndof;
  if (nvec <= 1)
    k_dots<1><<<ctx->nblk_d, KRY_T, 0, ctx->stream>>>(V, ldv, nvec, w, n, ctx->d_part, LDP, ctx->d_ticket, out, flags);
  else if (nvec <= 4)
    k_dots<4><<<ctx->nblk_d, KRY_T, 0, ctx->stream>>>(V, ldv, nvec, w, n, ctx->d_part, LDP, ctx->d_ticket, out, flags);
  else if (nvec <= 8)
    k_dots<8><<<ctx->nblk_d, KRY_T, 0, ctx->stream>>>(V, ldv, nvec, w, n, ctx->d_part, LDP, ctx->d_ticket, out, flags);
  else if (nvec <= 16)
    k_dots<16><<<ctx->nblk_d, KRY_T, 0, ctx->stream>>>(V, ldv, nvec, w, n, ctx->d_part, LDP, ctx->d_ticket, out, flags);
  else
    k_dots<32><<<ctx->nblk_d, KRY_T, 0, ctx->stream>>>(V, ldv, nvec, w, n, ctx->d_part, LDP, ctx->d_ticket, out, flags);
  count_launch();
  CK(cudaGetLastError());
  return LDG_OK;
}

// w -= V h (nvec vectors). dots_out != null: also V . w_new into dots_out (DOTS form);
// otherwise with givens, also completes Arnoldi column j.
template <int NV>
void launch_orth(ldg_ctx* ctx, const double* V, int nvec, const double* h, double* w, int j, int givens,
                 double* dots_out) {
  const int64_t n = ctx->ndof;
  if (dots_out)
    k_orth_update<NV, true><<<ctx->nblk_d, KRY_T, 0, ctx->stream>>>(V, n, nvec, h, w, n, ctx->d_part, LDP,
                                                                   ctx->d_ticket, ctx->d_small, ctx->m, j, givens,
                                                                   ctx->d_flags, dots_out);
  else
    k_orth_update<NV, false><<<ctx->nblk, KRY_T, 0, ctx->stream>>>(V, n, nvec, h, w, n, ctx->d_part, LDP,
                                                                  ctx->d_ticket, ctx->d_small, ctx->m, j, givens,
                                                                  ctx->d_flags, nullptr);
}
int orth_update(ldg_ctx* ctx, const double* V, int nvec, const double* h, double* w, int j, int givens,
                double* dots_out = nullptr) {
  if (nvec <= 4) launch_orth<4>(ctx, V, nvec, h, w, j, givens, dots_out);
  else if (nvec <= 8) launch_orth<8>(ctx, V, nvec, h, w, j, givens, dots_out);
  else if (nvec <= 16) launch_orth<16>(ctx, V, nvec, h, w, j, givens, dots_out);
  else launch_orth<32>(ctx, V, nvec, h, w, j, givens, dots_out);
  count_launch();
  CK(cudaGetLastError());
  return LDG_OK;
}

int read_scalars(ldg_ctx* ctx, const double* src, int n) {
  CK(cudaMemcpyAsync(ctx->h_pin, src, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return LDG_OK;
}

void state_copies(ldg_ctx* ctx, KArgs& a) {
  a.q32_out = ctx->d_q32;
  a.u32_out = ctx->d_u32;
}

int do_residual(ldg_ctx* ctx, const double* u, double* r) {
  KArgs a = base_args(ctx);
  if (ctx->ks->qstage) {
    a.u = u; a.out = ctx->d_q;
    state_copies(ctx, a);
    CK(ctx->ks->qstage(MODE_R, a, ctx->stream));
    a = base_args(ctx);
    a.q = ctx->d_q;
  }
  a.u = u; a.out = r;
  a.hist = ctx->scheme != LDG_STEADY ? ctx->d_hist : nullptr;
  CK(ctx->ks->residual(MODE_R, a, ctx->stream));
  return LDG_OK;
}

int jvp_args(ldg_ctx* ctx, KArgs a, const double* u, const double* v, double* jv, int prec, bool q_ready) {
  if (prec == LDG_TC_BF16X3 || prec == LDG_TC_BF16) {
    if (!ctx->tcjv)
      return fail(ctx, LDG_ERR_ARG,
                  "the tensor-core J.v exists for the Euler model on affine quadrilaterals, p = 1..4, with p + 2 "
                  "Gauss points");
    KArgs b = a;
    b.u = u; b.v = v; b.out = jv;
    CK(ctx->tcjv(b, ctx->d_tcimg, prec == LDG_TC_BF16X3 ? 3 : 1, ctx->d_tcerr, ctx->stream));
    return LDG_OK;
  }
  if (prec == LDG_F32X2) {
    // float-pair arithmetic: the nodal kernels of the linear models only
    if (!(ctx->ks->linear && ctx->ks->qstage && ctx->linff))
      return fail(ctx, LDG_ERR_ARG,
                  "LDG_F32X2: the float-pair J.v exists for the nodal kernels of the linear models only (affine "
                  "quadrilaterals and hexahedra with p + 1 Gauss points, triangles and tetrahedra with at least "
                  "p + 2)");
    KArgs b = a;
    b.u = v; b.out = jv;
    CK(ctx->linff(b, ctx->d_dq, ctx->stream));
    return LDG_OK;
  }
  const bool f32 = prec == LDG_FP32;
  StageFn qs = f32 ? ctx->ks->qstage32 : ctx->ks->qstage;
  StageFn rs = f32 ? ctx->ks->residual32 : ctx->ks->residual;
  KArgs b = a;   // skip flags, instance map and model data of the caller
  if (ctx->ks->linear && ctx->ks->qstage && (f32 ? ctx->lin32 : ctx->lin64)) {
    // linear model on affine tensor elements: the nodal form of the same operator
    b.u = v; b.out = jv;
    CK((f32 ? ctx->lin32 : ctx->lin64)(b, ctx->d_dq, ctx->stream));
  } else if (ctx->ks->linear && ctx->ks->qstage) {
    // linear model: J v = R(v) - R(0), the homogeneous operator applied to v
    b.u = v; b.out = ctx->d_dq;
    CK(qs(MODE_HOM, b, ctx->stream));
    b = a;
    b.u = v; b.q = ctx->d_dq; b.out = jv;
    CK(rs(MODE_HOM, b, ctx->stream));
  } else if (ctx->ks->qstage) {
    // nonlinear model with q: dual numbers (u, v) and (q(u), Q v). q(u) is the FP64
    // q-stage of the residual (reused when the caller has just evaluated R(u))
    // q-stage of the residual (reused when the caller has just evaluated R(u)). The FP32
    // J.v reads the FP32 copies of u and q(u) that this q-stage writes beside q(u).
    if (!q_ready) {
      b.u = u; b.out = ctx->d_q;
      state_copies(ctx, b);
      CK(ctx->ks->qstage(MODE_R, b, ctx->stream));
      b = a;
    }
    b.u = v; b.out = ctx->d_dq;
    CK(qs(MODE_HOM, b, ctx->stream));
    b = a;
    if (f32) {
      b.u = ctx->d_u32; b.q = ctx->d_q32;
    } else {
      b.u = u; b.q = ctx->d_q;
    }
    b.v = v; b.dq = ctx->d_dq; b.out = jv;
    CK(rs(MODE_JV, b, ctx->stream));
  } else {
    b.u = u; b.v = v; b.out = jv;
    CK(rs(MODE_JV, b, ctx->stream));
  }
  return LDG_OK;
}

// ------------------------------------------------------- block-Jacobi
// Greedy colouring such that no two elements of one colour are within `dist`
// face steps (dist 2 for diffusion models: R_K depends on u up to two faces away
// through q).
void colour_mesh(ldg_ctx* ctx, int dist, std::vector<int>& col) {
  const int64_t E = ctx->E;
  const int nf = ctx->nf;
  col.assign(E, -1);
  std::vector<int> mark;
  for (int64_t e = 0; e < E; ++e) {
    std::vector<int64_t> near;
    for (int f = 0; f < nf; ++f) {
      int a = ctx->h_nbr[e * nf + f];
      if (a < 0) continue;
      near.push_back(a);
      if (dist >= 2)
        for (int g = 0; g < nf; ++g) {
          int b = ctx->h_nbr[(int64_t)a * nf + g];
          if (b >= 0 && b != e) near.push_back(b);
        }
    }
    std::vector<char> used(near.size() + 1, 0);
    for (int64_t x : near)
      if (col[x] >= 0 && col[x] < (int)used.size()) used[col[x]] = 1;
    int c = 0;
    while (used[c]) ++c;   // at most near.size() colours are taken
    col[e] = c;
  }
}

int ensure_pc_storage(ldg_ctx* ctx) {
  const int64_t E = ctx->E, n = ctx->nloc;
  if (!ctx->d_blocks) CK(cudaMalloc(&ctx->d_blocks, (size_t)E * n * n * sizeof(double)));
  if (!ctx->d_Z && !ctx->lean) CK(cudaMalloc(&ctx->d_Z, (size_t)ctx->m * ctx->ndof * sizeof(double)));
  if (!ctx->d_status) {
    CK(cudaMalloc(&ctx->d_status, sizeof(int)));
    CK(cudaMemset(ctx->d_status, 0, sizeof(int)));
  }
  if (ctx->ks->qstage && !ctx->d_colour) {
    std::vector<int> col;
    colour_mesh(ctx, 2, col);
    int nc = 0;
    for (int c : col) nc = std::max(nc, c + 1);
    ctx->ncolour = nc;
    CK(cudaMalloc(&ctx->d_colour, col.size() * sizeof(int)));
    CK(cudaMemcpy(ctx->d_colour, col.data(), col.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_probe, ctx->ndof * sizeof(double)));
    CK(cudaMalloc(&ctx->d_jp, ctx->ndof * sizeof(double)));
  }
  return LDG_OK;
}

const KernelSet* find_set(const ldg_ctx* ctx, int tile);

// Exact diagonal blocks dR_K/du_K at state u, computed in the given arithmetic.
int do_blocks(ldg_ctx* ctx, const double* u, int prec, double* blocks) {
  int rc;
  if ((rc = ensure_pc_storage(ctx))) return rc;
  if (!blocks) return fail(ctx, LDG_ERR_ARG, "block extraction: null output buffer");
  const int nloc = ctx->nloc;
  const int64_t E = ctx->E;
  if (!ctx->ks->qstage) {
    if (prec == LDG_FP32 && !ctx->ks->blocks32) {
      // curved elements: one unit tangent per launch in FP32 arithmetic
      for (int l = 0; l < nloc; ++l) {
        KArgs a = base_args(ctx);
        a.u = u; a.v = u; a.out = nullptr;
        a.blk_col = l;
        a.blk_out = blocks;
        CK(ctx->ks->residual32(MODE_JV, a, ctx->stream));
      }
    } else if (prec == LDG_FP32) {
      // dual numbers with BLK_KT unit tangents on every element and none on its neighbours;
      // the default tile (the J.v's tuned tile suits one tangent, not eight)
      const KernelSet* k0 = find_set(ctx, 0);
      for (int l = 0; l < nloc; l += BLK_KT) {
        KArgs a = base_args(ctx);
        a.u = u; a.v = u; a.out = nullptr;
        a.blk_out = blocks;
        CK(k0->blocks32(l, a, ctx->stream));
      }
    } else {
      // FP64: one unit tangent per launch (the FP64 multi-tangent kernel needs one
      // element per CTA at over 200 registers per thread, and measured slower)
      for (int l = 0; l < nloc; ++l) {
        KArgs a = base_args(ctx);
        a.u = u; a.v = u; a.out = nullptr;
        a.blk_col = l;
        a.blk_out = blocks;
        CK(ctx->ks->residual(MODE_JV, a, ctx->stream));
      }
    }
    return LDG_OK;
  }
  // models with q: coloured probing, J applied to the sum of unit vectors of one colour;
  // a nonlinear model's q(u) is formed once for all probes
  if (!ctx->ks->linear) {
    KArgs a = base_args(ctx);
    a.u = u; a.out = ctx->d_q;
    state_copies(ctx, a);
    CK(ctx->ks->qstage(MODE_R, a, ctx->stream));
  }
  for (int c = 0; c < ctx->ncolour; ++c)
    for (int l = 0; l < nloc; ++l) {
      k_probe<<<grid_for(E * nloc), 256, 0, ctx->stream>>>(ctx->d_probe, ctx->d_colour, c, l, nloc, E);
      count_launch();
      if ((rc = jvp_args(ctx, base_args(ctx), u, ctx->d_probe, ctx->d_jp, prec, true))) return rc;
      k_extract<<<grid_for(E * nloc), 256, 0, ctx->stream>>>(ctx->d_jp, ctx->d_colour, c, l, nloc, E, blocks);
      count_launch();
      CK(cudaGetLastError());
    }
  return LDG_OK;
}

// Build the block-Jacobi preconditioner at state u: blocks in the Krylov arithmetic,
// inverses in FP32 when the Krylov J.v is FP32 (or the block is too large for an FP64
// elimination in shared memory), else FP64.
int do_pc_setup(ldg_ctx* ctx, const double* u) {
  int rc;
  // (a float-pair Krylov J.v takes FP64 blocks, the tensor-core forms FP32 ones)
  const int kp = ctx->opt.krylov_precision;
  const int prec = kp == LDG_FP32 || kp == LDG_TC_BF16X3 || kp == LDG_TC_BF16 ? LDG_FP32 : LDG_FP64;
  ctx->pc_kappa = ctx->mp.kappa;
  ctx->pc_a0dt = ctx->a0dt;
  // the block storage must exist before its address is handed to the extraction
  if ((rc = ensure_pc_storage(ctx))) return rc;
  if ((rc = do_blocks(ctx, u, prec, ctx->d_blocks))) return rc;
  const int n = ctx->nloc;
  const bool fp64 = prec == LDG_FP64 && block_inverse_smem<double>(n) <= 200 * 1024;
  const int want = fp64 ? LDG_FP64 : LDG_FP32;
  if (ctx->binv_prec != want) {
    cudaFree(ctx->d_binv);
    ctx->d_binv = nullptr;
    CK(cudaMalloc(&ctx->d_binv, (size_t)ctx->E * n * n * (fp64 ? sizeof(double) : sizeof(float))));
    ctx->binv_prec = want;
  }
  const int threads = n >= 16 ? 256 : ((n + 31) / 32) * 32;
  // compile-time block sizes of the common element blocks (quadrilateral Euler p = 1..4,
  // scalar models p = 3); threads and columns per thread as measured fastest on a B300
  // for each size and precision (4,096 to 65,536 random blocks)
  auto fixed = [&](auto tag, auto nconst, auto ntconst, auto cptconst) -> int {
    typedef decltype(tag) T;
    constexpr int NN = decltype(nconst)::value, NT = decltype(ntconst)::value, CPT = decltype(cptconst)::value;
    const size_t smem = BInvN<T, NN, NT, CPT>::SMEM;
    CK(cudaFuncSetAttribute(k_block_inverse_n<T, NN, NT, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)smem));
    k_block_inverse_n<T, NN, NT, CPT><<<(unsigned)ctx->E, NT, smem, ctx->stream>>>(ctx->d_blocks, (T*)ctx->d_binv,
                                                                                    ctx->d_status);
    count_launch();
    CK(cudaGetLastError());
    ctx->pc_ready = true;
    return LDG_OK;
  };
  typedef std::integral_constant<int, 4> C4;
  if (n == 16)
    return fp64 ? fixed(0.0, std::integral_constant<int, 16>(), std::integral_constant<int, 64>(), C4())
                : fixed(0.f, std::integral_constant<int, 16>(), std::integral_constant<int, 32>(), C4());
  if (n == 36)
    return fp64 ? fixed(0.0, std::integral_constant<int, 36>(), std::integral_constant<int, 64>(), C4())
                : fixed(0.f, std::integral_constant<int, 36>(), std::integral_constant<int, 64>(), C4());
  if (n == 64)
    return fp64 ? fixed(0.0, std::integral_constant<int, 64>(), std::integral_constant<int, 256>(), C4())
                : fixed(0.f, std::integral_constant<int, 64>(), std::integral_constant<int, 128>(),
                        std::integral_constant<int, 8>());
  if (n == 100 && !fp64)
    return fixed(0.f, std::integral_constant<int, 100>(), std::integral_constant<int, 256>(), C4());
  if (fp64) {
    const size_t smem = block_inverse_smem<double>(n);
    CK(cudaFuncSetAttribute(k_block_inverse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_block_inverse<double><<<(unsigned)ctx->E, threads, smem, ctx->stream>>>(ctx->d_blocks, (double*)ctx->d_binv, n,
                                                                             ctx->d_status);
  } else {
    const size_t smem = block_inverse_smem<float>(n);
    CK(cudaFuncSetAttribute(k_block_inverse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_block_inverse<float><<<(unsigned)ctx->E, threads, smem, ctx->stream>>>(ctx->d_blocks, (float*)ctx->d_binv, n,
                                                                            ctx->d_status);
  }
  count_launch();
  CK(cudaGetLastError());
  ctx->pc_ready = true;
  return LDG_OK;
}

int pc_apply(ldg_ctx* ctx, const double* x, double* y, const int* skip, const int* inst_skip) {
  const int n = ctx->nloc;
  const int threads = std::min(256, ((n + 31) / 32) * 32);
  const int* inst = inst_skip ? ctx->ext_inst : nullptr;
  if (inst_skip && !inst) return fail(ctx, LDG_ERR_ARG, "per-instance skip on a context without instances");
  const int64_t E = ctx->E;
  const unsigned gw = (unsigned)((E + 7) / 8);
  const bool f64 = ctx->binv_prec == LDG_FP64;
  const double* bd = (const double*)ctx->d_binv;
  const float* bf = (const float*)ctx->d_binv;
  // FP32 blocks whose size divides 128: flat 16-byte loads; otherwise one warp per
  // element up to 128 rows, one CTA per element beyond
  if (!f64 && n >= 16 && 128 % n == 0) {
    k_block_apply_vec<<<gw, 256, 0, ctx->stream>>>(bf, x, y, n, E, skip, inst, inst_skip);
  } else if (n <= 32) {
    if (f64) k_block_apply_warp<double, 1><<<gw, 256, 0, ctx->stream>>>(bd, x, y, n, E, skip, inst, inst_skip);
    else k_block_apply_warp<float, 1><<<gw, 256, 0, ctx->stream>>>(bf, x, y, n, E, skip, inst, inst_skip);
  } else if (n <= 64) {
    if (f64) k_block_apply_warp<double, 2><<<gw, 256, 0, ctx->stream>>>(bd, x, y, n, E, skip, inst, inst_skip);
    else k_block_apply_warp<float, 2><<<gw, 256, 0, ctx->stream>>>(bf, x, y, n, E, skip, inst, inst_skip);
  } else if (n <= 128) {
    if (f64) k_block_apply_warp<double, 4><<<gw, 256, 0, ctx->stream>>>(bd, x, y, n, E, skip, inst, inst_skip);
    else k_block_apply_warp<float, 4><<<gw, 256, 0, ctx->stream>>>(bf, x, y, n, E, skip, inst, inst_skip);
  } else if (f64) {
    k_block_apply<double><<<(unsigned)E, threads, n * sizeof(double), ctx->stream>>>(bd, x, y, n, skip, inst, inst_skip);
  } else {
    k_block_apply<float><<<(unsigned)E, threads, n * sizeof(float), ctx->stream>>>(bf, x, y, n, skip, inst, inst_skip);
  }
  count_launch();
  CK(cudaGetLastError());
  return LDG_OK;
}

// ------------------------------------------------------ reduced-basis preconditioner
// P^{-1} r = C r + B^{-1} (r - J C r), C = W G^{-1} (J W)^T, G = (J W)^T J W (include/ldg.h).
// Scratch d_rbS: [0, 32) (J W)^T x, [32, 64) y, [64, 64 + 1024) G by columns, then G^{-1}
// (row-major, 1024), then two norms.
constexpr int kRbMax = 32;
constexpr int kRbA = 0, kRbY = 32, kRbM = 64, kRbJi = 64 + 1024, kRbN = 64 + 2048, kRbScratch = 64 + 2048 + 8;

__global__ void k_rb_small(const double* Ji, const double* a, double* y, int k, const int* flags) {
  if (flags && flags[0]) return;
  const int i = threadIdx.x;
  if (i < k) {
    double s = 0.0;
    for (int j = 0; j < k; ++j) s += Ji[i * k + j] * a[j];
    y[i] = s;
  }
}
// c = sum_j y_j W_j, r = x - sum_j y_j (J W)_j
__global__ void k_rb_combine(const double* W, const double* JW, const double* y, int k, const double* x, double* c,
                             double* r, int64_t n, const int* flags) {
  if (flags && flags[0]) return;
  __shared__ double ys[kRbMax];
  if (threadIdx.x < k) ys[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double cs = 0.0, rs = x[i];
    for (int j = 0; j < k; ++j) {
      cs += ys[j] * W[(size_t)j * n + i];
      rs -= ys[j] * JW[(size_t)j * n + i];
    }
    c[i] = cs;
    r[i] = rs;
  }
}
__global__ void k_rb_add(double* z, const double* c, int64_t n, const int* flags) {
  if (flags && flags[0]) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] += c[i];
}
// v -= sum_{j != skip} h_j W_j
__global__ void k_rb_orth(const double* W, const double* h, int k, int skip, double* v, int64_t n) {
  __shared__ double hs[kRbMax];
  if (threadIdx.x < k) hs[threadIdx.x] = (int)threadIdx.x == skip ? 0.0 : h[threadIdx.x];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = v[i];
    for (int j = 0; j < k; ++j) s -= hs[j] * W[(size_t)j * n + i];
    v[i] = s;
  }
}
__global__ void k_rb_scale(const double* v, double a, double* dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = a * v[i];
}

int ensure_rb_storage(ldg_ctx* ctx) {
  if (ctx->d_rbW || ctx->rb_cap <= 0) return LDG_OK;
  const size_t n = (size_t)ctx->ndof;
  CK(cudaMalloc(&ctx->d_rbW, (size_t)ctx->rb_cap * n * sizeof(double)));
  CK(cudaMalloc(&ctx->d_rbJW, (size_t)ctx->rb_cap * n * sizeof(double)));
  CK(cudaMalloc(&ctx->d_rbS, kRbScratch * sizeof(double)));
  CK(cudaMalloc(&ctx->d_rbC, 2 * n * sizeof(double)));
  return LDG_OK;
}

// Inverse of the rb_k x rb_k matrix ctx->h_rbJr (G; Gauss-Jordan with partial pivoting) into
// the device scratch; a matrix singular to rounding leaves block-Jacobi alone.
int rb_invert(ldg_ctx* ctx) {
  const int k = ctx->rb_k;
  ctx->rb_eff = 0;
  if (k == 0) return LDG_OK;
  std::vector<double> A((size_t)k * 2 * k, 0.0);
  double amax = 0.0;
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      A[(size_t)i * 2 * k + j] = ctx->h_rbJr[(size_t)i * kRbMax + j];
      amax = std::max(amax, std::fabs(ctx->h_rbJr[(size_t)i * kRbMax + j]));
    }
  for (int i = 0; i < k; ++i) A[(size_t)i * 2 * k + k + i] = 1.0;
  for (int c = 0; c < k; ++c) {
    int piv = c;
    for (int r = c + 1; r < k; ++r)
      if (std::fabs(A[(size_t)r * 2 * k + c]) > std::fabs(A[(size_t)piv * 2 * k + c])) piv = r;
    const double d = A[(size_t)piv * 2 * k + c];
    if (!(std::fabs(d) > 1e-12 * amax) || !std::isfinite(d)) return LDG_OK;
    if (piv != c)
      for (int j = 0; j < 2 * k; ++j) std::swap(A[(size_t)piv * 2 * k + j], A[(size_t)c * 2 * k + j]);
    for (int j = 0; j < 2 * k; ++j) A[(size_t)c * 2 * k + j] /= d;
    for (int r = 0; r < k; ++r) {
      if (r == c) continue;
      const double f = A[(size_t)r * 2 * k + c];
      if (f != 0.0)
        for (int j = 0; j < 2 * k; ++j) A[(size_t)r * 2 * k + j] -= f * A[(size_t)c * 2 * k + j];
    }
  }
  std::vector<double> Ji((size_t)k * k);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) Ji[(size_t)i * k + j] = A[(size_t)i * 2 * k + k + j];
  CK(cudaMemcpyAsync(ctx->d_rbS + kRbJi, Ji.data(), Ji.size() * sizeof(double), cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->rb_eff = k;
  return LDG_OK;
}

// Enter v (device, n) into the basis: orthogonalised twice against the vectors that stay,
// skipped when nothing of it remains, normalised into a free slot or the oldest one.
// With u given and the set-up current, the new column's J W_s = J(u) W_s and the row and
// column s of G are formed (one J.v), so the set-up stays current; otherwise a later
// rb_setup forms all of it.
int rb_insert(ldg_ctx* ctx, const double* v, const double* u) {
  int rc;
  if (ctx->rb_cap <= 0) return LDG_OK;
  if ((rc = ensure_rb_storage(ctx))) return rc;
  const int64_t n = ctx->ndof;
  const int64_t g1 = std::min<int64_t>(grid_for(n), 148 * 8);
  const int k = ctx->rb_k, full = k == ctx->rb_cap;
  const int slot = full ? ctx->rb_next : k;
  const bool current = u && ctx->rb_eff == k;
  double* t = ctx->d_rbC;
  double* S = ctx->d_rbS;
  CK(cudaMemcpyAsync(t, v, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  if ((rc = dots(ctx, t, n, 1, t, S + kRbN, nullptr))) return rc;
  for (int pass = 0; pass < 2 && k > 0; ++pass) {
    if ((rc = dots(ctx, ctx->d_rbW, n, k, t, S + kRbA, nullptr))) return rc;
    k_rb_orth<<<g1, 256, 0, ctx->stream>>>(ctx->d_rbW, S + kRbA, k, full ? slot : -1, t, n);
    count_launch();
    CK(cudaGetLastError());
  }
  if ((rc = dots(ctx, t, n, 1, t, S + kRbN + 1, nullptr))) return rc;
  if ((rc = read_scalars(ctx, S + kRbN, 2))) return rc;
  const double n0 = std::sqrt(ctx->h_pin[0]), n1 = std::sqrt(ctx->h_pin[1]);
  if (!(n1 > 1e-10 * n0) || !std::isfinite(n1)) return LDG_OK;   // nothing new in v
  double* ws = ctx->d_rbW + (size_t)slot * n;
  k_rb_scale<<<g1, 256, 0, ctx->stream>>>(t, 1.0 / n1, ws, n);
  count_launch();
  CK(cudaGetLastError());
  if (full) ctx->rb_next = (ctx->rb_next + 1) % ctx->rb_cap;
  else ++ctx->rb_k;
  const int k1 = ctx->rb_k;
  if (!current) { ctx->rb_eff = 0; return LDG_OK; }
  // row and column s of G: (J W)_i . (J W)_s
  double* jws = ctx->d_rbJW + (size_t)slot * n;
  if ((rc = jvp_args(ctx, base_args(ctx), u, ws, jws, ctx->opt.krylov_precision))) return rc;
  if ((rc = dots(ctx, ctx->d_rbJW, n, k1, jws, S + kRbM, nullptr))) return rc;
  double cr[kRbMax];
  CK(cudaMemcpyAsync(cr, S + kRbM, kRbMax * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->h_rbJr.empty()) ctx->h_rbJr.assign((size_t)kRbMax * kRbMax, 0.0);
  for (int i = 0; i < k1; ++i) {
    ctx->h_rbJr[(size_t)i * kRbMax + slot] = cr[i];
    ctx->h_rbJr[(size_t)slot * kRbMax + i] = cr[i];
  }
  return rb_invert(ctx);
}

// J W at state u for every vector and G = (J W)^T J W, then its inverse.
int rb_setup(ldg_ctx* ctx, const double* u) {
  int rc;
  ctx->rb_eff = 0;
  const int k = ctx->rb_k;
  if (k == 0) return LDG_OK;
  const int64_t n = ctx->ndof;
  double* S = ctx->d_rbS;
  for (int j = 0; j < k; ++j) {
    if ((rc = jvp_args(ctx, base_args(ctx), u, ctx->d_rbW + (size_t)j * n, ctx->d_rbJW + (size_t)j * n,
                       ctx->opt.krylov_precision)))
      return rc;
  }
  for (int j = 0; j < k; ++j)
    if ((rc = dots(ctx, ctx->d_rbJW, n, k, ctx->d_rbJW + (size_t)j * n, S + kRbM + j * kRbMax, nullptr))) return rc;
  std::vector<double> colmaj((size_t)k * kRbMax);
  CK(cudaMemcpyAsync(colmaj.data(), S + kRbM, colmaj.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->h_rbJr.empty()) ctx->h_rbJr.assign((size_t)kRbMax * kRbMax, 0.0);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) ctx->h_rbJr[(size_t)i * kRbMax + j] = colmaj[(size_t)j * kRbMax + i];
  return rb_invert(ctx);
}

// z = C x + B^{-1} (x - J C x); block-Jacobi alone while no reduced set-up is in force
int rb_apply(ldg_ctx* ctx, const double* x, double* z, const int* flags) {
  int rc;
  const int k = ctx->rb_eff;
  if (k == 0) return pc_apply(ctx, x, z, flags);
  const int64_t n = ctx->ndof;
  const int64_t g1 = std::min<int64_t>(grid_for(n), 148 * 8);
  double* S = ctx->d_rbS;
  double* c = ctx->d_rbC;
  double* r = c + n;
  if ((rc = dots(ctx, ctx->d_rbJW, n, k, x, S + kRbA, flags))) return rc;
  k_rb_small<<<1, kRbMax, 0, ctx->stream>>>(S + kRbJi, S + kRbA, S + kRbY, k, flags);
  k_rb_combine<<<g1, 256, 0, ctx->stream>>>(ctx->d_rbW, ctx->d_rbJW, S + kRbY, k, x, c, r, n, flags);
  count_launch();
  count_launch();
  CK(cudaGetLastError());
  if ((rc = pc_apply(ctx, r, z, flags))) return rc;
  k_rb_add<<<g1, 256, 0, ctx->stream>>>(z, c, n, flags);
  count_launch();
  CK(cudaGetLastError());
  return LDG_OK;
}

// ------------------------------------------------------------ MLP preconditioner
int mlp_reserve(ldg_ctx* ctx, int64_t rows) {
  auto& M = ctx->mlp;
  if (rows <= M.cap) return LDG_OK;
  for (float** p : {&M.T, &M.Y, &M.dY}) { cudaFree(*p); *p = nullptr; CK(cudaMalloc(p, rows * M.n * sizeof(float))); }
  cudaFree(M.X); M.X = nullptr;
  CK(cudaMalloc(&M.X, rows * 2 * M.n * sizeof(float)));
  for (float** p : {&M.H1, &M.H2, &M.dH1, &M.dH2}) { cudaFree(*p); *p = nullptr; CK(cudaMalloc(p, rows * M.h * sizeof(float))); }
  cudaFree(M.mask); M.mask = nullptr;
  CK(cudaMalloc(&M.mask, rows * sizeof(float)));
  cudaFree(M.norms); M.norms = nullptr;
  CK(cudaMalloc(&M.norms, rows * sizeof(double)));
  M.cap = rows;
  return LDG_OK;
}

int mlp_alloc(ldg_ctx* ctx) {
  auto& M = ctx->mlp;
  if (M.theta) return LDG_OK;
  M.n = ctx->nloc;
  M.nparam = (int64_t)M.h * 2 * M.n + M.h + (int64_t)M.h * M.h + M.h + (int64_t)M.n * M.h + M.n + (int64_t)M.n * M.n;
  for (float** p : {&M.theta, &M.grad, &M.m, &M.v}) CK(cudaMalloc(p, M.nparam * sizeof(float)));
  CK(cudaMalloc(&M.theta_bf, M.nparam * sizeof(__nv_bfloat16)));
  CK(cudaMalloc(&M.loss, sizeof(double)));
  CK(cudaMalloc(&M.count, sizeof(int)));
  CK(cudaMemset(M.m, 0, M.nparam * sizeof(float)));
  CK(cudaMemset(M.v, 0, M.nparam * sizeof(float)));
  return mlp_reserve(ctx, ctx->E);
}

// parameter offsets: W1 [h][2n], b1 [h], W2 [h][h], b2 [h], W3 [n][h], b3 [n], Ws [n][n]
struct MlpOff {
  int64_t W1, b1, W2, b2, W3, b3, Ws;
  MlpOff(int n, int h) {
    W1 = 0; b1 = W1 + (int64_t)h * 2 * n; W2 = b1 + h; b2 = W2 + (int64_t)h * h; W3 = b2 + h;
    b3 = W3 + (int64_t)n * h; Ws = b3 + n;
  }
};

template <bool TA, bool TB, class TBt>
void gemm(ldg_ctx* ctx, int M_, int N_, int K_, const float* A, int lda, const TBt* B, int ldb, float* C, int ldc,
          const float* bias, int relu, const int* skip, int acc_c = 0) {
  dim3 grid((N_ + 63) / 64, (M_ + 63) / 64);
  k_gemm<TA, TB, TBt><<<grid, 256, 0, ctx->stream>>>(M_, N_, K_, A, lda, B, ldb, C, ldc, bias, relu, skip, acc_c);
  count_launch();
}

// forward pass on `rows` prepared rows (Xn in M.X); weights FP32 (train) or BF16 (inference)
template <class TW>
void mlp_forward(ldg_ctx* ctx, int64_t rows, const TW* th, const float* thf, const int* skip) {
  auto& M = ctx->mlp;
  MlpOff o(M.n, M.h);
  const int r = (int)rows;
  gemm<false, true, TW>(ctx, r, M.h, 2 * M.n, M.X, 2 * M.n, th + o.W1, 2 * M.n, M.H1, M.h, thf + o.b1, 1, skip);
  gemm<false, true, TW>(ctx, r, M.h, M.h, M.H1, M.h, th + o.W2, M.h, M.H2, M.h, thf + o.b2, 1, skip);
  gemm<false, true, TW>(ctx, r, M.n, M.h, M.H2, M.h, th + o.W3, M.h, M.Y, M.n, thf + o.b3, 0, skip);
  // linear skip path on the scaled vector block (first n input columns)
  gemm<false, true, TW>(ctx, r, M.n, M.n, M.X, 2 * M.n, th + o.Ws, M.n, M.Y, M.n, nullptr, 0, skip, 1);
}

// loss and gradient (into M.grad) of the prepared batch in M.X / M.T / M.mask
int mlp_backward(ldg_ctx* ctx, int64_t rows) {
  auto& M = ctx->mlp;
  MlpOff o(M.n, M.h);
  const int r = (int)rows;
  const int64_t g1 = std::min<int64_t>(grid_for(rows * M.n), 148 * 8);
  k_mlp_dloss<<<g1, 256, 0, ctx->stream>>>(M.Y, M.T, M.mask, rows, M.n, M.count, M.dY, M.loss);
  count_launch();
  float* G = M.grad;
  gemm<true, false, float>(ctx, M.n, M.h, r, M.dY, M.n, M.H2, M.h, G + o.W3, M.h, nullptr, 0, nullptr);
  gemm<true, false, float>(ctx, M.n, M.n, r, M.dY, M.n, M.X, 2 * M.n, G + o.Ws, M.n, nullptr, 0, nullptr);
  k_colsum<<<M.n, 256, 0, ctx->stream>>>(M.dY, rows, M.n, G + o.b3);
  count_launch();
  gemm<false, false, float>(ctx, r, M.h, M.n, M.dY, M.n, M.theta + o.W3, M.h, M.dH2, M.h, nullptr, 0, nullptr);
  k_relu_back<<<std::min<int64_t>(grid_for(rows * M.h), 148 * 8), 256, 0, ctx->stream>>>(M.dH2, M.H2, rows * M.h);
  count_launch();
  gemm<true, false, float>(ctx, M.h, M.h, r, M.dH2, M.h, M.H1, M.h, G + o.W2, M.h, nullptr, 0, nullptr);
  k_colsum<<<M.h, 256, 0, ctx->stream>>>(M.dH2, rows, M.h, G + o.b2);
  count_launch();
  gemm<false, false, float>(ctx, r, M.h, M.h, M.dH2, M.h, M.theta + o.W2, M.h, M.dH1, M.h, nullptr, 0, nullptr);
  k_relu_back<<<std::min<int64_t>(grid_for(rows * M.h), 148 * 8), 256, 0, ctx->stream>>>(M.dH1, M.H1, rows * M.h);
  count_launch();
  gemm<true, false, float>(ctx, M.h, 2 * M.n, r, M.dH1, M.h, M.X, 2 * M.n, G + o.W1, 2 * M.n, nullptr, 0, nullptr);
  k_colsum<<<M.h, 256, 0, ctx->stream>>>(M.dH1, rows, M.h, G + o.b1);
  count_launch();
  CK(cudaGetLastError());
  return LDG_OK;
}

// prepare rows idx (or 0..rows-1) of the pair set X / T into the work buffers (the
// input rows in FP32, or in BF16 into xbf for the tensor-core path)
int mlp_prep(ldg_ctx* ctx, const double* X, const double* T, const double* U, const int* idx, int64_t rows,
             const int* skip, __nv_bfloat16* xbf) {
  auto& M = ctx->mlp;
  int rc;
  if ((rc = mlp_reserve(ctx, rows))) return rc;
  if (!skip) {
    CK(cudaMemsetAsync(M.count, 0, sizeof(int), ctx->stream));
    CK(cudaMemsetAsync(M.loss, 0, sizeof(double), ctx->stream));
  }
  k_mlp_prep<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, ctx->stream>>>(X, T, U, idx, rows, M.n, M.X, xbf,
                                                                          T ? M.T : nullptr,
                                                                          M.mask, M.norms, skip ? nullptr : M.count,
                                                                          skip);
  count_launch();
  CK(cudaGetLastError());
  return LDG_OK;
}

// ------------------------------------------------- tensor-core inference (tcgen05)
// BF16 row-major [rows][cols] with row stride ld elements, as a TMA map with
// 64 x box_rows boxes and 128-byte swizzle.
int tc_map(ldg_ctx* ctx, CUtensorMap* map, const void* base, int64_t rows, int cols, int ld, int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&encode, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !encode) return fail(ctx, LDG_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  }
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, LDG_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return LDG_OK;
}

// Buffers and TMA maps of the tensor-core inference over the context's E elements.
int mlp_tc_setup(ldg_ctx* ctx) {
  auto& M = ctx->mlp;
  const char* simt = getenv("LDG_MLP_SIMT");
  M.tc = M.n % 64 == 0 && M.n <= 128 && M.h % 64 == 0 && M.h <= 256 && !(simt && simt[0] == '1');
  if (!M.tc || M.tc_rows == ctx->E) return LDG_OK;
  const int n = M.n, h = M.h;
  const int64_t E = ctx->E;
  for (__nv_bfloat16** p : {&M.Xbf, &M.H1bf, &M.H2bf, &M.wtc}) { cudaFree(*p); *p = nullptr; }
  CK(cudaMalloc(&M.Xbf, (size_t)E * 2 * n * sizeof(__nv_bfloat16)));
  CK(cudaMalloc(&M.H1bf, (size_t)E * h * sizeof(__nv_bfloat16)));
  CK(cudaMalloc(&M.H2bf, (size_t)E * h * sizeof(__nv_bfloat16)));
  // W1 [h][2n], W2 [h][h], W3 [n][h], Ws [n][n], each at a 256-byte boundary
  const int64_t w1 = 0, w2 = w1 + (((int64_t)h * 2 * n + 127) & ~127), w3 = w2 + (((int64_t)h * h + 127) & ~127),
                ws = w3 + (((int64_t)n * h + 127) & ~127), wend = ws + (((int64_t)n * n + 127) & ~127);
  CK(cudaMalloc(&M.wtc, wend * sizeof(__nv_bfloat16)));
  if (!M.d_err) {
    CK(cudaMalloc(&M.d_err, sizeof(int)));
    CK(cudaMemset(M.d_err, 0, sizeof(int)));
  }
  int rc;
  if ((rc = tc_map(ctx, &M.maps[0], M.Xbf, E, 2 * n, 2 * n, TC_BM)) ||
      (rc = tc_map(ctx, &M.maps[1], M.Xbf, E, n, 2 * n, TC_BM)) ||
      (rc = tc_map(ctx, &M.maps[2], M.H1bf, E, h, h, TC_BM)) ||
      (rc = tc_map(ctx, &M.maps[3], M.H2bf, E, h, h, TC_BM)) ||
      (rc = tc_map(ctx, &M.maps[4], M.wtc + w1, h, 2 * n, 2 * n, h)) ||
      (rc = tc_map(ctx, &M.maps[5], M.wtc + w2, h, h, h, h)) ||
      (rc = tc_map(ctx, &M.maps[6], M.wtc + w3, n, h, h, n)) ||
      (rc = tc_map(ctx, &M.maps[7], M.wtc + ws, n, n, n, n)))
    return rc;
  M.tc_rows = E;
  return LDG_OK;
}

int mlp_refresh_bf16(ldg_ctx* ctx) {
  auto& M = ctx->mlp;
  k_to_bf16<<<std::min<int64_t>(grid_for(M.nparam), 148 * 4), 256, 0, ctx->stream>>>(M.theta, M.theta_bf, M.nparam);
  count_launch();
  CK(cudaGetLastError());
  int rc;
  if ((rc = mlp_tc_setup(ctx))) return rc;
  if (M.tc) {
    const int n = M.n, h = M.h;
    MlpOff o(n, h);
    const int64_t w1 = 0, w2 = w1 + (((int64_t)h * 2 * n + 127) & ~127), w3 = w2 + (((int64_t)h * h + 127) & ~127),
                  ws = w3 + (((int64_t)n * h + 127) & ~127);
    const struct { int64_t src, dst; int rows, cols; } part[4] = {
        {o.W1, w1, h, 2 * n}, {o.W2, w2, h, h}, {o.W3, w3, n, h}, {o.Ws, ws, n, n}};
    for (const auto& q : part) {
      k_to_bf16_2d<<<148, 256, 0, ctx->stream>>>(M.theta + q.src, q.cols, M.wtc + q.dst, q.cols, q.rows, q.cols,
                                                 nullptr);
      count_launch();
    }
    CK(cudaGetLastError());
  }
  M.ready = true;
  return LDG_OK;
}

// One tcgen05 GEMM launch: C = act(A1 B1^T [+ A2 B2^T] + bias), maps by index.
int tc_gemm(ldg_ctx* ctx, int a1, int b1, int a2, int b2, int N, int K1, int K2, const float* bias, int relu,
            void* C, int ldc, int out_bf16, const int* skip) {
  auto& M = ctx->mlp;
  TcGemmArgs g;
  g.M = (int)ctx->E; g.N = N; g.K1 = K1; g.K2 = K2; g.bias = bias; g.relu = relu; g.C = C; g.ldc = ldc;
  g.out_bf16 = out_bf16; g.err = M.d_err; g.skip = skip;
  const size_t smem = tc_gemm_smem(N, K1, K2, out_bf16);
  static int smem_set = 0;
  if (smem_set < (int)smem) {
    CK(cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    smem_set = 200 * 1024;
  }
  if (smem > 200 * 1024) return fail(ctx, LDG_ERR_UNSUPPORTED, "tensor-core GEMM tile too large");
  const unsigned grid = (unsigned)((ctx->E + TC_BM - 1) / TC_BM);
  k_tc_gemm<<<grid, 128, smem, ctx->stream>>>(M.maps[a1], M.maps[b1], M.maps[a2 >= 0 ? a2 : a1],
                                              M.maps[b2 >= 0 ? b2 : b1], g);
  count_launch();
  CK(cudaGetLastError());
  return LDG_OK;
}

// y = M(x) on a full n_dof vector (element blocks) at state u, BF16 weights. With the
// tensor-core path the input and hidden activations are stored in BF16 as well, and
// the output layer accumulates W3 h2 and the skip map Ws x_v in one TMEM accumulator.
int mlp_apply(ldg_ctx* ctx, const double* u, const double* x, double* y, const int* skip) {
  auto& M = ctx->mlp;
  int rc;
  MlpOff o(M.n, M.h);
  const bool tc = M.tc && M.tc_rows == ctx->E;
  if ((rc = mlp_prep(ctx, x, nullptr, u, nullptr, ctx->E, skip, tc ? M.Xbf : nullptr))) return rc;
  if (tc) {
    const int n = M.n, h = M.h;
    if ((rc = tc_gemm(ctx, 0, 4, -1, -1, h, 2 * n, 0, M.theta + o.b1, 1, M.H1bf, h, 1, skip))) return rc;
    if ((rc = tc_gemm(ctx, 2, 5, -1, -1, h, h, 0, M.theta + o.b2, 1, M.H2bf, h, 1, skip))) return rc;
    if ((rc = tc_gemm(ctx, 3, 6, 1, 7, n, h, n, M.theta + o.b3, 0, M.Y, n, 0, skip))) return rc;
  } else {
    mlp_forward<__nv_bfloat16>(ctx, ctx->E, M.theta_bf, M.theta, skip);
  }
  k_mlp_unprep<<<(unsigned)((ctx->E * 32 + 255) / 256), 256, 0, ctx->stream>>>(M.Y, M.norms, ctx->E, M.n, y,
                                                                                       skip);
  count_launch();
  CK(cudaGetLastError());
  return LDG_OK;
}

// ------------------------------------------ learned correction of block-Jacobi
// h[K][c][i] = (sum over the faces of K holding node i of the face neighbour's z at the
// same place) / ||z_K||; one warp per element.
__global__ void k_halo_feat(const double* __restrict__ z, const int* __restrict__ src, int64_t E, int npe, int ncu,
                            double* __restrict__ h, const int* skip) {
  if (skip && *skip) return;
  const int64_t K = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (K >= E) return;
  const int nloc = npe * ncu;
  const double* zk = z + K * nloc;
  double s2 = 0.0;
  for (int i = lane; i < nloc; i += 32) s2 += zk[i] * zk[i];
  for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  const double nrm = sqrt(s2);
  const double inv = nrm > 1e-30 ? 1.0 / nrm : 0.0;
  for (int i = lane; i < nloc; i += 32) {
    const int c = i / npe, n = i - c * npe;
    const int* sk = src + (K * npe + n) * 3;
    double acc = 0.0;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int sidx = sk[t];
      if (sidx >= 0) {
        const int64_t nb = sidx / npe, nn = sidx - nb * npe;
        acc += z[(nb * ncu + c) * npe + nn];
      }
    }
    h[K * nloc + i] = acc * inv;
  }
}

// The neighbour-node table of the halo features, built on the host at first use.
int ensure_halo(ldg_ctx* ctx) {
  if (ctx->d_halo) return LDG_OK;
  const int et = ctx->etype, p = ctx->p, npe = ctx->npe, nf = ctx->nf;
  const int nfn = et == LDG_QUAD ? p + 1 : (et == LDG_HEX ? (p + 1) * (p + 1) :
                  (et == LDG_TRI ? p + 1 : (p + 1) * (p + 2) / 2));
  const int nfq = ctx->nfq;
  if (et == LDG_HEX && ctx->nq != p + 1)
    return fail(ctx, LDG_ERR_UNSUPPORTED, "halo features on hexahedra need p + 1 quadrature points");
  std::vector<int> tab((size_t)ctx->E * npe * 3, -1);
  for (int64_t K = 0; K < ctx->E; ++K)
    for (int f = 0; f < nf; ++f) {
      const int nb = ctx->h_nbr[K * nf + f];
      if (nb < 0) continue;
      const int code = ctx->h_nbf[K * nf + f], nface = code & 7, orient = code >> 3;
      for (int j = 0; j < nfn; ++j) {
        int jn;
        if (et == LDG_TET) jn = ctx->h_perm[(size_t)orient * nfn + j];
        else if (et == LDG_HEX) jn = ctx->h_perm[(size_t)orient * nfq + j];
        else jn = ctx->h_perm[(size_t)orient * nfq] != 0 ? nfn - 1 - j : j;   // edges (also curved): same or reversed
        const int own = face_node_host(et, p, f, j), other = face_node_host(et, p, nface, jn);
        int* slot = &tab[((size_t)K * npe + own) * 3];
        int t = 0;
        while (t < 3 && slot[t] >= 0) ++t;
        if (t == 3) return fail(ctx, LDG_ERR_MESH, "a node on more than three faces");
        slot[t] = (int)(nb * npe + other);
      }
    }
  CK(cudaMalloc(&ctx->d_halo, tab.size() * sizeof(int)));
  CK(cudaMemcpy(ctx->d_halo, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice));
  return LDG_OK;
}

int halo_features(ldg_ctx* ctx, const double* z, double* h, const int* skip) {
  int rc;
  if ((rc = ensure_halo(ctx))) return rc;
  k_halo_feat<<<(unsigned)((ctx->E * 32 + 255) / 256), 256, 0, ctx->stream>>>(z, ctx->d_halo, ctx->E, ctx->npe,
                                                                             ctx->ncu, h, skip);
  count_launch();
  CK(cudaGetLastError());
  return LDG_OK;
}

// y = M(x) of the learned block-Jacobi correction: z = BJ^{-1} x, h = halo(z), network.
int mlp_bj_apply(ldg_ctx* ctx, const double* x, double* y, const int* skip) {
  int rc;
  if (!ctx->d_pcz) {
    CK(cudaMalloc(&ctx->d_pcz, ctx->ndof * sizeof(double)));
    CK(cudaMalloc(&ctx->d_pch, ctx->ndof * sizeof(double)));
  }
  if ((rc = pc_apply(ctx, x, ctx->d_pcz, skip))) return rc;
  if ((rc = halo_features(ctx, ctx->d_pcz, ctx->d_pch, skip))) return rc;
  return mlp_apply(ctx, ctx->d_pch, ctx->d_pcz, y, skip);
}

// GMRES(m) on J(u) x = b, x0 = 0, to ||b - J x|| <= rtol ||b||.
// The host queues Arnoldi steps up to LAG steps ahead of the GPU; each step's
// kernels return at once after the device-side convergence test has fired.
int do_gmres(ldg_ctx* ctx, const double* u, const double* b, double* x, double rtol, ldg_solve_report* rep) {
  const int m = ctx->m;
  const int64_t n = ctx->ndof;
  KrySmall S{m};
  double* sm = ctx->d_small;
  double* sc = sm + S.sc();
  double* V = ctx->d_V;
  int* flags = ctx->d_flags;
  const int LAG = 2;
  int rc;
  CK(cudaMemsetAsync(x, 0, n * sizeof(double), ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  if ((rc = dots(ctx, ctx->d_r, n, 1, ctx->d_r, sc + 4, nullptr))) return rc;
  if ((rc = read_scalars(ctx, sc + 4, 1))) return rc;
  const double bnorm = std::sqrt(ctx->h_pin[0]);
  if (!std::isfinite(bnorm)) return fail(ctx, LDG_ERR_NONFINITE, "non-finite right-hand side");
  if (rep) rep->lin_resid = 0.0;
  if (bnorm == 0.0) return LDG_OK;
  const double thr = rtol * bnorm;
  CK(cudaMemcpyAsync(sc + 3, &thr, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  const bool pc = ((ctx->opt.precond == LDG_PC_BJACOBI || ctx->opt.precond == LDG_PC_RB_BJ) && ctx->pc_ready) ||
                  (ctx->opt.precond == LDG_PC_MLP && ctx->mlp.ready) ||
                  (ctx->opt.precond == LDG_PC_MLP_BJ && ctx->mlp.ready && ctx->pc_ready);
  // the preconditioned Krylov vectors Z must exist before their addresses are used
  if (pc && (rc = ensure_pc_storage(ctx))) return rc;
  const int64_t g1 = std::min<int64_t>(grid_for(n), 148 * 8);
  for (int cycle = 0; cycle < ctx->opt.max_restarts; ++cycle) {
    k_cycle_start<<<g1, 256, 0, ctx->stream>>>(ctx->d_r, V, n, sm, m, flags);
    count_launch();
    CK(cudaGetLastError());
    bool stop = false;
    for (int j = 0; j < m && !stop; ++j) {
      if (j >= LAG) {
        CK(cudaEventSynchronize(ctx->ev[j - LAG]));
        if (ctx->h_flags[(j - LAG) * 4]) { stop = true; break; }
      }
      double* w = V + (size_t)(j + 1) * n;
      KArgs a = base_args(ctx);
      a.skip = flags;
      const double* dir = V + (size_t)j * n;
      if (pc) {
        // flexible right preconditioning: z_j = M^{-1} v_j, w = J z_j, x += Z y
        double* z = ctx->d_Z + (size_t)j * n;
        if (ctx->opt.precond == LDG_PC_MLP) {
          if ((rc = mlp_apply(ctx, u, dir, z, flags))) return rc;
        } else if (ctx->opt.precond == LDG_PC_MLP_BJ) {
          if ((rc = mlp_bj_apply(ctx, dir, z, flags))) return rc;
        } else if (ctx->opt.precond == LDG_PC_RB_BJ) {
          if ((rc = rb_apply(ctx, dir, z, flags))) return rc;
        } else {
          if ((rc = pc_apply(ctx, dir, z, flags))) return rc;
        }
        dir = z;
      }
      if ((rc = jvp_args(ctx, a, u, dir, w, ctx->opt.krylov_precision))) return rc;
      if ((rc = dots(ctx, V, n, j + 1, w, sm + S.h1(), flags))) return rc;
      // pass 1 projects and forms the pass-2 projections in the same sweep
      if ((rc = orth_update(ctx, V, j + 1, sm + S.h1(), w, j, 0, sm + S.h2()))) return rc;
      if ((rc = orth_update(ctx, V, j + 1, sm + S.h2(), w, j, 1))) return rc;
      k_scale_by_norm<<<g1, 256, 0, ctx->stream>>>(w, sc, w, n, flags);
      count_launch();
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(ctx->h_flags + j * 4, flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaEventRecord(ctx->ev[j], ctx->stream));
    }
    k_backsolve<<<1, 32, 0, ctx->stream>>>(sm, m, flags);
    count_launch();
    k_solution_update<<<g1, 256, 0, ctx->stream>>>(pc ? ctx->d_Z : V, n, sm, m, flags, x, n);
    count_launch();
    CK(cudaGetLastError());
    // true residual r = b - J x (with the operator the Arnoldi process used)
    if ((rc = jvp_args(ctx, base_args(ctx), u, x, ctx->d_w, ctx->opt.krylov_precision))) return rc;
    k_sub_norm<<<ctx->nblk, KRY_T, 0, ctx->stream>>>(b, ctx->d_w, ctx->d_r, n, ctx->d_part, LDP, ctx->d_ticket, sc + 4);
    count_launch();
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ctx->h_pin, sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_flags + 60 * 4, flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int cols = ctx->h_flags[60 * 4 + 1];
    if (rep) { rep->gmres_iters += cols; rep->jv_calls += cols + 1; }
    if (pc && ctx->col_X && (ctx->col_mode & 2) && ctx->opt.precond == LDG_PC_BJACOBI) {
      // exact inverse pairs of the learned correction's training set: r = J z_j, d = z_j
      // for the cycle's block-Jacobi-preconditioned directions z_j
      if (!ctx->d_pcz) {
        CK(cudaMalloc(&ctx->d_pcz, n * sizeof(double)));
        CK(cudaMalloc(&ctx->d_pch, n * sizeof(double)));
      }
      for (int jj = 0; jj < cols && ctx->col_count < ctx->col_cap; ++jj, ++ctx->col_count) {
        const size_t o = (size_t)ctx->col_count * n;
        const double* zj = ctx->d_Z + (size_t)jj * n;
        if ((rc = jvp_args(ctx, base_args(ctx), u, zj, ctx->d_pcz, ctx->opt.krylov_precision))) return rc;
        if ((rc = pc_apply(ctx, ctx->d_pcz, ctx->col_X + o, nullptr))) return rc;
        if ((rc = halo_features(ctx, ctx->col_X + o, ctx->col_U + o, nullptr))) return rc;
        CK(cudaMemcpyAsync(ctx->col_T + o, zj, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
      }
    }
    if (pc && ctx->col_X && ctx->col_mode == 0 && ctx->opt.precond == LDG_PC_BJACOBI) {
      // training triples for the learned preconditioner: (v_j, M^{-1} v_j, u)
      for (int jj = 0; jj < cols && ctx->col_count < ctx->col_cap; ++jj, ++ctx->col_count) {
        const size_t o = (size_t)ctx->col_count * n;
        CK(cudaMemcpyAsync(ctx->col_X + o, V + (size_t)jj * n, n * sizeof(double), cudaMemcpyDeviceToDevice,
                           ctx->stream));
        CK(cudaMemcpyAsync(ctx->col_T + o, ctx->d_Z + (size_t)jj * n, n * sizeof(double), cudaMemcpyDeviceToDevice,
                           ctx->stream));
        CK(cudaMemcpyAsync(ctx->col_U + o, u, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
      }
    }
    const double beta = std::sqrt(ctx->h_pin[4]);
    if (rep) rep->lin_resid = beta / bnorm;
    if (!std::isfinite(beta)) return fail(ctx, LDG_ERR_NONFINITE, "non-finite GMRES residual");
    const bool converged_est = ctx->h_flags[60 * 4] && !ctx->h_flags[60 * 4 + 2];
    if (beta <= thr * (1.0 + 1e-6) || (converged_est && beta <= thr * 10.0)) return LDG_OK;
    if (cols == 0) return fail(ctx, LDG_ERR_NONFINITE, "GMRES made no progress");
  }
  return fail(ctx, LDG_ERR_MAXIT, "GMRES did not reach its tolerance within max_restarts cycles");
}

constexpr int kLearnedRestarts = 2;

int do_newton(ldg_ctx* ctx, double* u, ldg_solve_report* rep) {
  const int64_t n = ctx->ndof;
  KrySmall S{ctx->m};
  double* sc = ctx->d_small + S.sc();
  int rc;
  auto t0 = std::chrono::steady_clock::now();
  double* res = ctx->d_res;   // R(u_k), the right-hand side of each linear solve
  double* del = ctx->d_x;     // Newton update
  if ((rc = do_residual(ctx, u, res))) return rc;
  if (rep) rep->residual_calls++;
  if ((rc = dots(ctx, res, n, 1, res, sc + 5, nullptr))) return rc;
  if ((rc = read_scalars(ctx, sc + 5, 1))) return rc;
  const double r0 = std::sqrt(ctx->h_pin[0]);
  double rn = r0;
  if (rep) rep->r0 = r0;
  if (!std::isfinite(r0)) return fail(ctx, LDG_ERR_NONFINITE, "non-finite initial residual");
  int k = 0;
  const int64_t g1 = std::min<int64_t>(grid_for(n), 148 * 8);
  while (rn > ctx->opt.newton_rtol * r0 && k < ctx->opt.max_newton) {
    if ((ctx->opt.precond == LDG_PC_BJACOBI || ctx->opt.precond == LDG_PC_MLP_BJ ||
         ctx->opt.precond == LDG_PC_RB_BJ) &&
        ((k == 0 && !(ctx->pc_hold && ctx->pc_ready)) || (ctx->opt.pc_refresh > 0 && k % ctx->opt.pc_refresh == 0))) {
      if ((rc = do_pc_setup(ctx, u))) return rc;
      if (rep) rep->pc_setups++;
    }
    // the reduced Jacobian: formed in full at the first Newton step of a solve (J at its
    // initial state), then kept up to date as updates enter the basis
    if (ctx->opt.precond == LDG_PC_RB_BJ && (k == 0 || ctx->rb_eff != ctx->rb_k) && (rc = rb_setup(ctx, u)))
      return rc;
    if (ctx->opt.precond == LDG_PC_MLP && k == 0 && (rc = ensure_pc_storage(ctx))) return rc;
    const double eta = newton_forcing_eta(ctx->opt.newton_forcing, ctx->opt.gmres_rtol, ctx->opt.newton_rtol, r0, rn);
    const bool learned = ctx->opt.precond == LDG_PC_MLP || ctx->opt.precond == LDG_PC_MLP_BJ;
    // a learned preconditioner gets two restart cycles to reach the tolerance before the
    // solve is redone with block-Jacobi, so that a network that does not fit the operator
    // costs at most 2 m extra Krylov steps per linear solve
    const int restarts = ctx->opt.max_restarts;
    if (learned) ctx->opt.max_restarts = std::min(restarts, kLearnedRestarts);
    rc = do_gmres(ctx, u, res, del, eta, rep);
    ctx->opt.max_restarts = restarts;
    if (rc == LDG_ERR_MAXIT && learned) {
      // the learned preconditioner did not reach the tolerance: fall back to block-Jacobi
      const int learned = ctx->opt.precond;
      ctx->opt.precond = LDG_PC_BJACOBI;
      rc = learned == LDG_PC_MLP_BJ ? LDG_OK : do_pc_setup(ctx, u);
      if (!rc) rc = do_gmres(ctx, u, res, del, eta, rep);
      ctx->opt.precond = learned;
      if (rep) { rep->pc_fallbacks++; if (learned == LDG_PC_MLP) rep->pc_setups++; }
    }
    if (rc && rc != LDG_ERR_MAXIT) return rc;
    // the Newton update enters the reduced basis
    if (ctx->opt.precond == LDG_PC_RB_BJ) {
      const int rc2 = rb_insert(ctx, del, u);
      if (rc2) return rc2;
    }
    if (ctx->col_X && (ctx->col_mode & 1) && ctx->col_count < ctx->col_cap && ctx->pc_ready) {
      // training data of the learned block-Jacobi correction: z = BJ^{-1} R(u_k), its
      // neighbour traces h, and the Newton update delta_k
      const size_t o = (size_t)ctx->col_count * n;
      if ((rc = pc_apply(ctx, res, ctx->col_X + o, nullptr))) return rc;
      if ((rc = halo_features(ctx, ctx->col_X + o, ctx->col_U + o, nullptr))) return rc;
      CK(cudaMemcpyAsync(ctx->col_T + o, del, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
      ++ctx->col_count;
    }
    // u <- u - delta   (sc[6] holds -1)
    k_axpy_dev<<<g1, 256, 0, ctx->stream>>>(del, sc + 6, u, n);
    count_launch();
    CK(cudaGetLastError());
    const double rprev = rn;
    if ((rc = do_residual(ctx, u, res))) return rc;
    if (rep) rep->residual_calls++;
    if ((rc = dots(ctx, res, n, 1, res, sc + 5, nullptr))) return rc;
    if ((rc = read_scalars(ctx, sc + 5, 1))) return rc;
    rn = std::sqrt(ctx->h_pin[0]);
    // step control (as in the batched engine): where ||R|| grew more than tenfold or
    // became non-finite, halve the step (u += delta / 2, delta /= 2), up to ten times
    for (int h = 0; h < 10 && !(rn <= 10.0 * rprev) && k + 1 < ctx->opt.max_newton; ++h) {
      k_hist<<<grid_for(n), 256, 0, ctx->stream>>>(n, 0.5, del, 0.0, nullptr, del);
      k_hist<<<grid_for(n), 256, 0, ctx->stream>>>(n, 1.0, u, 1.0, del, u);
      count_launch();
      count_launch();
      if ((rc = do_residual(ctx, u, res))) return rc;
      if (rep) { rep->residual_calls++; rep->newton_backtracks++; }
      if ((rc = dots(ctx, res, n, 1, res, sc + 5, nullptr))) return rc;
      if ((rc = read_scalars(ctx, sc + 5, 1))) return rc;
      rn = std::sqrt(ctx->h_pin[0]);
    }
    if (!(rn <= 10.0 * rprev)) {
      // no acceptable step within the limits: back to the last accepted iterate
      k_hist<<<grid_for(n), 256, 0, ctx->stream>>>(n, 1.0, u, 1.0, del, u);
      count_launch();
      if (rep) { rep->newton_iters = k + 1; rep->rfinal = rprev; }
      return fail(ctx, LDG_ERR_MAXIT, "no acceptable Newton step within the step-halving limits");
    }
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

// Model parameters from the ABI description (defaults: kappa = tau = 1, beta = 0, gamma = 1.4).
ModelParams make_params(const ldg_model_desc* model) {
  ModelParams mp{};
  mp.kappa = 1.0; mp.tau = 1.0; mp.gamma = 1.4; mp.cas = model->case_id;
  const double* mu = model->mu;
  const int nmu = mu ? model->n_mu : 0;
  mp.pr = 0.72;
  if (model->model == LDG_EULER) { if (nmu > 0) mp.gamma = mu[0]; }
  else if (model->model == LDG_NS) {
    // mu = {gamma, Re, Pr, tau}: viscosity 1/Re, penalty tau = 1/Re unless given
    const double re = nmu > 1 ? mu[1] : 100.0;
    if (nmu > 0) mp.gamma = mu[0];
    mp.kappa = 1.0 / re;
    if (nmu > 2) mp.pr = mu[2];
    mp.tau = nmu > 3 ? mu[3] : 1.0 / re;
  } else {
    if (nmu > 0) mp.kappa = mu[0];
    if (nmu > 1) mp.tau = mu[1];
    for (int d = 0; d < 3; ++d) if (nmu > 2 + d) mp.beta[d] = mu[2 + d];
  }
  return mp;
}

// ------------------------------------------------------------------ autotuner
// Deterministic direction for timing: v_i = sin(0.37 i + 0.5).
__global__ void k_tune_pattern(double* v, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) v[i] = sin(0.37 * (double)i + 0.5);
}

const KernelSet* find_set(const ldg_ctx* ctx, int tile) {
  for (const KernelSet& k : registry())
    if (k.etype == ctx->etype && k.p == ctx->p && k.nq == ctx->nq && k.model == ctx->model && k.tile == tile &&
        k.curved == (ctx->pg > 0))
      return &k;
  return nullptr;
}

int autotune(ldg_ctx* ctx, int force, int* tile, double* best_ms) {
  static std::map<std::tuple<int, int, int, int, int, int>, int> cache;
  const int kp = ctx->opt.krylov_precision;
  const int prec = kp == LDG_FP32 || kp == LDG_TC_BF16X3 || kp == LDG_TC_BF16 ? LDG_FP32 : LDG_FP64;
  int eb = 0;
  while ((int64_t(1) << eb) < ctx->E) ++eb;
  // (curved elements are keyed apart from the affine ones of the same element type)
  const auto key = std::make_tuple(ctx->etype + (ctx->pg > 0 ? 8 : 0), ctx->p, ctx->nq, ctx->model, prec, eb);
  if (best_ms) *best_ms = -1.0;
  if (!force) {
    auto it = cache.find(key);
    if (it != cache.end()) {
      if (const KernelSet* k = find_set(ctx, it->second)) {
        ctx->ks = k;
        if (tile) *tile = k->tile;
        return LDG_OK;
      }
    }
  }
  // candidates: the compiled tiles with distinct elements-per-CTA counts
  std::vector<const KernelSet*> cand;
  for (const KernelSet& k : registry()) {
    if (k.etype != ctx->etype || k.p != ctx->p || k.nq != ctx->nq || k.model != ctx->model ||
        k.curved != (ctx->pg > 0))
      continue;
    bool dup = false;
    for (const KernelSet* c : cand) dup |= (c->ne_q == k.ne_q && c->ne_j == k.ne_j && c->ne_r == k.ne_r);
    if (!dup) cand.push_back(&k);
  }
  if (cand.empty()) return fail(ctx, LDG_ERR_UNSUPPORTED, "autotune: no compiled kernels");
  const int64_t n = ctx->ndof;
  double *u = nullptr, *v = nullptr, *jv = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto release = [&]() {
    cudaFree(u); cudaFree(v); cudaFree(jv);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  int rc = LDG_OK;
  double best = 1e300;
  const KernelSet* pick = cand[0];
  do {
    cudaError_t ce;
    if ((ce = cudaMalloc(&u, n * sizeof(double))) || (ce = cudaMalloc(&v, n * sizeof(double))) ||
        (ce = cudaMalloc(&jv, n * sizeof(double))) || (ce = cudaEventCreate(&e0)) || (ce = cudaEventCreate(&e1))) {
      rc = fail(ctx, LDG_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(ce));
      break;
    }
    const int GEO = ctx->dim == 2 ? Geo<2>::size(ctx->nf) : Geo<3>::size(ctx->nf);
    k_interp_nodes<<<grid_for(ctx->E * ctx->npe), 256, 0, ctx->stream>>>(ctx->dim, ctx->npe, ctx->ncu, ctx->E, ctx->d_geo,
                                                                        GEO, ctx->d_xn, ctx->mp, ctx->t, u,
                                                                        ctx->d_xnode);
    k_tune_pattern<<<grid_for(n), 256, 0, ctx->stream>>>(v, n);
    count_launch();
    count_launch();
    for (const KernelSet* k : cand) {
      ctx->ks = k;
      const int reps = 10;
      for (int w = 0; w < 3 && !rc; ++w) rc = jvp_args(ctx, base_args(ctx), u, v, jv, prec);
      if (!rc && (ce = cudaEventRecord(e0, ctx->stream))) rc = fail(ctx, LDG_ERR_CUDA, cudaGetErrorString(ce));
      for (int r = 0; r < reps && !rc; ++r) rc = jvp_args(ctx, base_args(ctx), u, v, jv, prec);
      if (!rc && (ce = cudaEventRecord(e1, ctx->stream))) rc = fail(ctx, LDG_ERR_CUDA, cudaGetErrorString(ce));
      if (!rc && (ce = cudaEventSynchronize(e1))) rc = fail(ctx, LDG_ERR_CUDA, cudaGetErrorString(ce));
      if (rc) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms / reps < best) { best = ms / reps; pick = k; }
    }
  } while (false);
  release();
  ctx->ks = pick;
  if (rc) return rc;
  cache[key] = pick->tile;
  if (tile) *tile = pick->tile;
  if (best_ms) *best_ms = best;
  return LDG_OK;
}

}  // namespace impl
}  // namespace ldg

using namespace ldg::impl;

// ===================================================================== C ABI
extern "C" {

const char* ldg_version(void) { return "ldg-b300 0.1 (sm_103a)"; }

int64_t ldg_kernel_launches(void) { return (int64_t)launch_counter().load(); }

const char* ldg_last_error(const ldg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int ldg_destroy(ldg_ctx* ctx) {
  if (!ctx) return LDG_OK;
  if (ctx->engine) batch_free(ctx->engine);
  cudaFree(ctx->d_ops); cudaFree(ctx->d_opsf); cudaFree(ctx->d_geo); cudaFree(ctx->d_nbr); cudaFree(ctx->d_nbf); cudaFree(ctx->d_perm);
  cudaFree(ctx->d_xn); cudaFree(ctx->d_q); cudaFree(ctx->d_dq); cudaFree(ctx->d_hist);
  cudaFree(ctx->d_q32); cudaFree(ctx->d_u32);
  cudaFree(ctx->d_rbW); cudaFree(ctx->d_rbJW); cudaFree(ctx->d_rbS); cudaFree(ctx->d_rbC);
  cudaFree(ctx->d_tcimg); cudaFree(ctx->d_tcerr);
  cudaFree(ctx->d_cgeo); cudaFree(ctx->d_cgeof); cudaFree(ctx->d_cx); cudaFree(ctx->d_minv); cudaFree(ctx->d_minvf);
  cudaFree(ctx->d_xnode); cudaFree(ctx->d_fd); cudaFree(ctx->d_radd); cudaFree(ctx->d_dirk);
  cudaFree(ctx->d_wave);
  cudaFree(ctx->d_V); cudaFree(ctx->d_r); cudaFree(ctx->d_w); cudaFree(ctx->d_res); cudaFree(ctx->d_x); cudaFree(ctx->d_small); cudaFree(ctx->d_part);
  cudaFree(ctx->d_flags); cudaFree(ctx->d_ticket); cudaFree(ctx->d_t);
  cudaFree(ctx->d_colour); cudaFree(ctx->d_blocks); cudaFree(ctx->d_binv); cudaFree(ctx->d_Z);
  cudaFree(ctx->d_probe); cudaFree(ctx->d_jp); cudaFree(ctx->d_status);
  cudaFree(ctx->d_stage); cudaFree(ctx->d_lops); cudaFree(ctx->d_lopsf); cudaFree(ctx->d_stage_many);
  if (ctx->s_in) cudaStreamDestroy(ctx->s_in);
  if (ctx->s_out) cudaStreamDestroy(ctx->s_out);
  for (int k = 0; k < 2; ++k) {
    if (ctx->ev_in[k]) cudaEventDestroy(ctx->ev_in[k]);
    if (ctx->ev_done[k]) cudaEventDestroy(ctx->ev_done[k]);
    if (ctx->ev_out[k]) cudaEventDestroy(ctx->ev_out[k]);
  }
  cudaFree(ctx->d_halo); cudaFree(ctx->d_pcz); cudaFree(ctx->d_pch);
  cudaFree(ctx->d_shq); cudaFree(ctx->d_shpart); cudaFree(ctx->d_shdot);
  cudaFree(ctx->d_er_xi); cudaFree(ctx->d_er_w); cudaFree(ctx->d_er_B); cudaFree(ctx->d_er_P); cudaFree(ctx->d_l2);
  {
    auto& M = ctx->mlp;
    for (void* p : {(void*)M.Xbf, (void*)M.H1bf, (void*)M.H2bf, (void*)M.wtc, (void*)M.d_err})
      cudaFree(p);
    for (void* p : {(void*)M.theta, (void*)M.grad, (void*)M.m, (void*)M.v, (void*)M.theta_bf, (void*)M.X, (void*)M.T,
                    (void*)M.mask, (void*)M.H1, (void*)M.H2, (void*)M.Y, (void*)M.dY, (void*)M.dH1, (void*)M.dH2,
                    (void*)M.norms, (void*)M.loss, (void*)M.count, (void*)M.idx})
      cudaFree(p);
  }
  if (ctx->h_pin) cudaFreeHost(ctx->h_pin);
  if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
  for (int i = 0; i < 64; ++i) if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  delete ctx;
  return LDG_OK;
}

int ldg_create(ldg_ctx** out, const ldg_mesh_desc* mesh, int p, const ldg_model_desc* model, const ldg_options* opts,
               void* cuda_stream) {
  return create_ctx(out, mesh, p, model, opts, cuda_stream, false);
}

}  // extern "C"

namespace ldg {
namespace impl {
// Every element is an axis-aligned box: the off-diagonal entries of J^{-1} and the
// off-axis components of each face normal (face f lies on local axis f / 2) are exactly
// zero in the geometry records (layout of Geo<DIM>).
static bool cartesian_elements(const std::vector<double>& geo, int dim, int64_t nelem) {
  const int nf = 2 * dim, stride = dim * dim + 1 + dim + dim * dim + nf * (dim + 1);
  const int face = dim * dim + 1 + dim + dim * dim;
  if (nelem <= 0 || (int64_t)geo.size() < nelem * stride) return false;
  for (int64_t e = 0; e < nelem; ++e) {
    const double* g = geo.data() + e * stride;
    for (int k = 0; k < dim; ++k)
      for (int d = 0; d < dim; ++d)
        if (k != d && g[k * dim + d] != 0.0) return false;
    for (int f = 0; f < nf; ++f)
      for (int d = 0; d < dim; ++d)
        if (d != f / 2 && g[face + f * (dim + 1) + d] != 0.0) return false;
  }
  return true;
}

int create_ctx(ldg_ctx** out, const ldg_mesh_desc* mesh, int p, const ldg_model_desc* model, const ldg_options* opts,
               void* cuda_stream, bool lean) {
  if (!out || !mesh || !model || !mesh->xyz || !mesh->vid || mesh->n_elem <= 0) return LDG_ERR_ARG;
  *out = nullptr;
  ldg_ctx* ctx = new ldg_ctx();
  ctx->lean = lean;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->etype = mesh->elem_type;
  ctx->model = model->model;
  if (ctx->etype < 0 || ctx->etype > 3 || ctx->model < 0 || ctx->model > 3) {
    ldg_destroy(ctx);
    return LDG_ERR_ARG;
  }
  ctx->dim = (ctx->etype == LDG_HEX || ctx->etype == LDG_TET) ? 3 : 2;
  const bool gas = ctx->model == LDG_EULER || ctx->model == LDG_NS;
  if (gas && ctx->dim != 2) { ldg_destroy(ctx); return LDG_ERR_UNSUPPORTED; }
  ctx->pg = mesh->geom_order > 0 ? mesh->geom_order : 0;
  if (ctx->pg > 0 && ((ctx->etype != LDG_QUAD && ctx->etype != LDG_TRI) || !mesh->xgeo)) {
    ldg_destroy(ctx);
    return LDG_ERR_UNSUPPORTED;
  }
  ctx->ncu = gas ? 4 : 1;
  ldg_options o{};
  if (opts) o = *opts;
  if (o.nq1 <= 0) o.nq1 = (gas || ctx->etype == LDG_TRI || ctx->etype == LDG_TET) ? p + 2 : p + 1;
  if (o.gmres_m <= 0) o.gmres_m = 30;
  if (o.gmres_m > 30) o.gmres_m = 30;
  if (o.max_restarts <= 0) o.max_restarts = 50;
  if (o.max_newton <= 0) o.max_newton = 20;
  if (o.newton_rtol <= 0) o.newton_rtol = 1e-8;
  if (o.gmres_rtol <= 0) o.gmres_rtol = 1e-3;
  if (o.krylov_precision != LDG_FP32 && o.krylov_precision != LDG_F32X2 && o.krylov_precision != LDG_TC_BF16X3 &&
      o.krylov_precision != LDG_TC_BF16)
    o.krylov_precision = LDG_FP64;
  if (o.precond != LDG_PC_BJACOBI && o.precond != LDG_PC_MLP && o.precond != LDG_PC_MLP_BJ &&
      o.precond != LDG_PC_RB_BJ)
    o.precond = LDG_PC_NONE;
  if (o.rb_size <= 0) o.rb_size = 8;
  if (o.rb_size > kRbMax) o.rb_size = kRbMax;
  if (o.pc_refresh < 0) o.pc_refresh = 0;
  if (o.newton_forcing != LDG_FORCING_LAST) o.newton_forcing = LDG_FORCING_FIXED;
  if (o.pc_reuse < 1) o.pc_reuse = 1;
  if (o.krylov_basis != LDG_BASIS_F32X2) o.krylov_basis = LDG_BASIS_FP64;
  ctx->opt = o;
  ctx->rb_cap = o.precond == LDG_PC_RB_BJ ? o.rb_size : 0;
  ctx->p = p; ctx->nq = o.nq1;
  ctx->mp = make_params(model);
  for (const KernelSet& k : registry())
    if (!ctx->ks && k.etype == ctx->etype && k.p == p && k.nq == o.nq1 && k.model == ctx->model &&
        k.curved == (ctx->pg > 0))
      ctx->ks = &k;
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
  if (!prepare_mesh(ref, mesh->n_elem, mesh->xyz, mesh->vid, mp_, err, ctx->pg, mesh->xgeo)) {
    ctx->err = err;
    *out = ctx;
    return LDG_ERR_MESH;
  }
  CurvedPrep cp;
  if (ctx->pg > 0 && !prepare_curved(ref, mesh->n_elem, ctx->pg, mesh->xgeo, cp, err)) {
    ctx->err = err;
    *out = ctx;
    return LDG_ERR_MESH;
  }
  // wall faces (gas models): boundary faces marked 1 in mesh->bc become neighbour -2
  if (mesh->bc && gas)
    for (size_t i = 0; i < mp_.nbr.size(); ++i)
      if (mp_.nbr[i] < 0 && mesh->bc[i] == 1) mp_.nbr[i] = -2;
  if (mesh->n_elem > (int64_t)0x7fffffff) { ctx->err = "too many elements"; *out = ctx; return LDG_ERR_ARG; }
  ctx->E = mesh->n_elem;
  ctx->npe = ref.npe; ctx->nf = ref.nf; ctx->nfq = ref.nfq;
  ctx->ndof = ctx->E * ctx->npe * ctx->ncu;
  ctx->nloc = ctx->npe * ctx->ncu;
  ctx->h_nbr = mp_.nbr;
  ctx->h_nbf = mp_.nbf;
  ctx->h_perm = mp_.perm;
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
  {
    std::vector<float> bf(ref.blob.begin(), ref.blob.end());
    CK(cudaMalloc(&ctx->d_opsf, bf.size() * sizeof(float)));
    CK(cudaMemcpy(ctx->d_opsf, bf.data(), bf.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  // nodal J.v kernels of the linear models on affine tensor elements (exact when the
  // quadrature has at least p + 1 points; the face-node permutations equal the face-point
  // ones when it has exactly p + 1)
  if ((ctx->etype == LDG_QUAD || ctx->etype == LDG_HEX) && ctx->pg == 0 &&
      (ctx->model == LDG_POISSON || ctx->model == LDG_CONVDIFF) && o.nq1 == p + 1 && o.jv_form != LDG_JV_STAGE) {
    const bool conv = ctx->model == LDG_CONVDIFF;
    ctx->lin_cart = cartesian_elements(mp_.geo, ctx->dim, ctx->E);
    ctx->lin64 = lin_launcher(ctx->dim, p, conv, 0, ctx->lin_cart);
    ctx->lin32 = lin_launcher(ctx->dim, p, conv, 1, ctx->lin_cart);
    ctx->linff = lin_df_launcher(ctx->dim, p, conv, ctx->lin_cart);
    std::vector<double> lb;
    if (ctx->lin64 && ctx->lin32 && build_lin_ops(p, lb, err)) {
      ctx->h_lops = lb;
      std::vector<float> lf(lb.begin(), lb.end());
      CK(cudaMalloc(&ctx->d_lops, lb.size() * sizeof(double)));
      CK(cudaMemcpy(ctx->d_lops, lb.data(), lb.size() * sizeof(double), cudaMemcpyHostToDevice));
      CK(cudaMalloc(&ctx->d_lopsf, lf.size() * sizeof(float)));
      CK(cudaMemcpy(ctx->d_lopsf, lf.data(), lf.size() * sizeof(float), cudaMemcpyHostToDevice));
    } else {
      ctx->lin64 = ctx->lin32 = ctx->linff = nullptr;
    }
  }
  // the same on triangles and tetrahedra, whose stage kernels integrate exactly with at
  // least p + 2 collapsed points per direction
  if ((ctx->etype == LDG_TRI || ctx->etype == LDG_TET) && ctx->pg == 0 &&
      (ctx->model == LDG_POISSON || ctx->model == LDG_CONVDIFF) && o.nq1 >= p + 2 && o.jv_form != LDG_JV_STAGE) {
    const bool conv = ctx->model == LDG_CONVDIFF;
    ctx->lin64 = lin_simplex_launcher(ctx->etype, p, conv, 0);
    ctx->lin32 = lin_simplex_launcher(ctx->etype, p, conv, 1);
    ctx->linff = lin_simplex_launcher(ctx->etype, p, conv, 2);
    std::vector<double> lb;
    if (ctx->lin64 && ctx->lin32 && build_lin_simplex_ops(ctx->etype, p, lb, err)) {
      std::vector<float> lf(lb.begin(), lb.end());
      CK(cudaMalloc(&ctx->d_lops, lb.size() * sizeof(double)));
      CK(cudaMemcpy(ctx->d_lops, lb.data(), lb.size() * sizeof(double), cudaMemcpyHostToDevice));
      CK(cudaMalloc(&ctx->d_lopsf, lf.size() * sizeof(float)));
      CK(cudaMemcpy(ctx->d_lopsf, lf.data(), lf.size() * sizeof(float), cudaMemcpyHostToDevice));
    } else {
      ctx->lin64 = ctx->lin32 = ctx->linff = nullptr;
    }
  }
  // the tensor-core Euler J.v: affine quadrilaterals with p + 2 Gauss points
  if (ctx->model == LDG_EULER && ctx->etype == LDG_QUAD && ctx->pg == 0 && o.nq1 == p + 2 && tcjv_launcher(p)) {
    std::vector<unsigned char> img;
    if (build_tcjv_image(p, ref.blob, img)) {
      ctx->tcjv = tcjv_launcher(p);
      CK(cudaMalloc(&ctx->d_tcimg, img.size()));
      CK(cudaMemcpy(ctx->d_tcimg, img.data(), img.size(), cudaMemcpyHostToDevice));
      CK(cudaMalloc(&ctx->d_tcerr, sizeof(int)));
      CK(cudaMemset(ctx->d_tcerr, 0, sizeof(int)));
    }
  }
  if ((o.krylov_precision == LDG_TC_BF16X3 || o.krylov_precision == LDG_TC_BF16) && !ctx->tcjv) {
    ctx->err = "krylov_precision LDG_TC_BF16X3 / LDG_TC_BF16 needs the tensor-core J.v: the Euler model on affine "
               "quadrilaterals, p = 1..4, with p + 2 Gauss points";
    return LDG_ERR_ARG;
  }
  if (o.krylov_precision == LDG_F32X2 && !(ctx->ks->linear && ctx->linff)) {
    ctx->err = "krylov_precision LDG_F32X2 needs the float-pair nodal J.v kernels: a linear model on affine "
               "quadrilaterals or hexahedra with p + 1 Gauss points, or on triangles or tetrahedra with at least "
               "p + 2";
    return LDG_ERR_ARG;
  }
  CK(cudaMemcpy(ctx->d_geo, mp_.geo.data(), mp_.geo.size() * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_nbr, mp_.nbr.data(), mp_.nbr.size() * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_nbf, mp_.nbf.data(), mp_.nbf.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_perm, mp_.perm.data(), mp_.perm.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_xn, xn.data(), xn.size() * sizeof(double), cudaMemcpyHostToDevice));
  if (ctx->pg > 0) {
    auto up64 = [&](double** dst, const std::vector<double>& v) -> cudaError_t {
      cudaError_t e = cudaMalloc(dst, v.size() * sizeof(double));
      return e ? e : cudaMemcpy(*dst, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice);
    };
    auto up32 = [&](float** dst, const std::vector<double>& v) -> cudaError_t {
      std::vector<float> f(v.begin(), v.end());
      cudaError_t e = cudaMalloc(dst, f.size() * sizeof(float));
      return e ? e : cudaMemcpy(*dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice);
    };
    CK(up64(&ctx->d_cgeo, cp.geo));
    CK(up32(&ctx->d_cgeof, cp.geo));
    CK(up64(&ctx->d_cx, cp.x));
    CK(up64(&ctx->d_minv, cp.minv));
    CK(up32(&ctx->d_minvf, cp.minv));
    CK(up64(&ctx->d_xnode, cp.xnode));
  }
  if (ctx->ks->qstage) {
    CK(cudaMalloc(&ctx->d_q, n * ctx->dim * sizeof(double)));
    CK(cudaMalloc(&ctx->d_dq, n * ctx->dim * sizeof(double)));
    if (!ctx->ks->linear) {
      // FP32 copies of u and q(u) for the FP32 Krylov J.v (written by the residual's q-stage)
      CK(cudaMalloc(&ctx->d_q32, n * ctx->dim * sizeof(float)));
      CK(cudaMalloc(&ctx->d_u32, n * sizeof(float)));
    }
  }
  CK(cudaMalloc(&ctx->d_hist, n * sizeof(double)));
  if (!lean) CK(cudaMalloc(&ctx->d_V, (size_t)(ctx->m + 1) * n * sizeof(double)));
  CK(cudaMalloc(&ctx->d_t, sizeof(double)));
  CK(cudaMemset(ctx->d_t, 0, sizeof(double)));
  CK(cudaMalloc(&ctx->d_r, n * sizeof(double)));
  CK(cudaMalloc(&ctx->d_w, n * sizeof(double)));
  CK(cudaMalloc(&ctx->d_res, n * sizeof(double)));
  CK(cudaMalloc(&ctx->d_x, n * sizeof(double)));
  KrySmall S{ctx->m};
  CK(cudaMalloc(&ctx->d_small, S.total() * sizeof(double)));
  CK(cudaMemset(ctx->d_small, 0, S.total() * sizeof(double)));
  ctx->nblk = (int)std::min<int64_t>(148 * 4, std::max<int64_t>(1, (n + 511) / 512));
  ctx->nblk_d = (int)std::min<int64_t>(148, std::max<int64_t>(1, (n + 2047) / 2048));
  CK(cudaMalloc(&ctx->d_part, (size_t)ctx->nblk * LDP * sizeof(double)));
  CK(cudaMalloc(&ctx->d_flags, 8 * sizeof(int)));
  CK(cudaMemset(ctx->d_flags, 0, 8 * sizeof(int)));
  CK(cudaMalloc(&ctx->d_ticket, 8 * sizeof(unsigned int)));
  CK(cudaMemset(ctx->d_ticket, 0, 8 * sizeof(unsigned int)));
  CK(cudaMallocHost(&ctx->h_pin, 16 * sizeof(double)));
  CK(cudaMallocHost(&ctx->h_flags, 64 * 4 * sizeof(int)));
  for (int i = 0; i < 64; ++i) CK(cudaEventCreateWithFlags(&ctx->ev[i], cudaEventDisableTiming));
  // the Newton update uses sc[6] = -1 as its axpy coefficient
  double minus1 = -1.0;
  CK(cudaMemcpy(ctx->d_small + S.sc() + 6, &minus1, sizeof(double), cudaMemcpyHostToDevice));
  return LDG_OK;
}
}  // namespace impl
}  // namespace ldg

extern "C" {

int ldg_autotune(ldg_ctx* ctx, int force, int* tile, double* best_ms) {
  if (!ctx || !ctx->ks) return LDG_ERR_ARG;
  return autotune(ctx, force, tile, best_ms);
}

int ldg_set_tile(ldg_ctx* ctx, int tile) {
  if (!ctx || !ctx->ks) return LDG_ERR_ARG;
  const KernelSet* k = find_set(ctx, tile);
  if (!k) return fail(ctx, LDG_ERR_UNSUPPORTED, "no compiled kernel with tile " + std::to_string(tile));
  ctx->ks = k;
  return LDG_OK;
}

int ldg_get_tile(const ldg_ctx* ctx, int* tile, int* ne_q, int* ne_r, int* ne_j) {
  if (!ctx || !ctx->ks) return LDG_ERR_ARG;
  if (tile) *tile = ctx->ks->tile;
  if (ne_q) *ne_q = ctx->ks->ne_q;
  if (ne_r) *ne_r = ctx->ks->ne_r;
  if (ne_j) *ne_j = ctx->ks->ne_j;
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
  if (ctx->d_t) {
    k_set_scalar<<<1, 1, 0, ctx->stream>>>(ctx->d_t, t);
    count_launch();
    CK(cudaGetLastError());
  }
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

int ldg_q_stage(ldg_ctx* ctx, int mode, int64_t n_owned, const double* u, double* q) {
  if (!ctx || !ctx->ks || !u || !q || (mode != LDG_STAGE_R && mode != LDG_STAGE_HOM) || n_owned < 0 ||
      n_owned > ctx->E)
    return LDG_ERR_ARG;
  if (!ctx->ks->qstage) return fail(ctx, LDG_ERR_ARG, "ldg_q_stage: the model has no q (convection model)");
  KArgs a = base_args(ctx);
  a.E = (int)n_owned;
  a.u = u; a.out = q;
  CK(ctx->ks->qstage(mode == LDG_STAGE_R ? MODE_R : MODE_HOM, a, ctx->stream));
  return LDG_OK;
}

int ldg_residual_stage(ldg_ctx* ctx, int mode, int64_t n_owned, const double* u, const double* q, double* r) {
  if (!ctx || !ctx->ks || !u || !r || (mode != LDG_STAGE_R && mode != LDG_STAGE_HOM) || n_owned < 0 ||
      n_owned > ctx->E)
    return LDG_ERR_ARG;
  if (ctx->ks->qstage && !q) return fail(ctx, LDG_ERR_ARG, "ldg_residual_stage: the model needs q");
  if (mode == LDG_STAGE_HOM && !ctx->ks->linear)
    return fail(ctx, LDG_ERR_ARG, "ldg_residual_stage: the homogeneous stage is the J.v of linear models only");
  KArgs a = base_args(ctx);
  a.E = (int)n_owned;
  a.u = u; a.q = q; a.out = r;
  if (mode == LDG_STAGE_R) a.hist = ctx->scheme != LDG_STEADY ? ctx->d_hist : nullptr;
  CK(ctx->ks->residual(mode == LDG_STAGE_R ? MODE_R : MODE_HOM, a, ctx->stream));
  return LDG_OK;
}

int ldg_jvp(ldg_ctx* ctx, const double* u, const double* v, double* jv) {
  if (!ctx || !ctx->ks || !u || !v || !jv) return LDG_ERR_ARG;
  return jvp_args(ctx, base_args(ctx), u, v, jv, LDG_FP64);
}

static bool jv_precision_ok(int precision) {
  return precision == LDG_FP64 || precision == LDG_FP32 || precision == LDG_F32X2 || precision == LDG_TC_BF16X3 ||
         precision == LDG_TC_BF16;
}

int ldg_jvp_prec(ldg_ctx* ctx, int precision, const double* u, const double* v, double* jv) {
  if (!ctx || !ctx->ks || !u || !v || !jv || !jv_precision_ok(precision)) return LDG_ERR_ARG;
  return jvp_args(ctx, base_args(ctx), u, v, jv, precision);
}

// the nodal J.v kernels of the context's element type in `precision` (hexahedra: one
// thread per line in FP32 and float pairs, one per node in FP64)
static std::string nodal_names(const ldg_ctx* ctx, int precision) {
  if (ctx->etype == LDG_TRI || ctx->etype == LDG_TET) return "k_sim_q + k_sim_r [";
  if (ctx->etype == LDG_HEX && precision != LDG_FP64) return ctx->lin_cart ? "k_hex_qt + k_hex_rt [" : "k_hex_q + k_hex_r [";
  return ctx->lin_cart ? "k_lin_qt + k_lin_rt [" : "k_lin_q + k_lin_r [";
}

const char* ldg_jv_describe(const ldg_ctx* ctx, int precision) {
  if (!ctx || !ctx->ks) return "";
  static thread_local std::string s;
  const bool f32 = precision == LDG_FP32;
  static const char* el[] = {"tri", "quad", "hex", "tet"};
  static const char* md[] = {"poisson", "convdiff", "euler", "ns"};
  std::string what = std::string(el[ctx->etype]) + (ctx->pg ? " curved" : "") + " p=" + std::to_string(ctx->p) +
                     " nq=" + std::to_string(ctx->nq) + " " + md[ctx->model];
  if (precision == LDG_F32X2) {
    s = ctx->ks->linear && ctx->linff ? nodal_names(ctx, precision) + what +
                                            (ctx->lin_cart && ctx->etype == LDG_QUAD ? " cartesian" : "") +
                                            " f32x2, q scratch f32x2]"
                                      : "";
    return s.c_str();
  }
  if (precision == LDG_TC_BF16X3 || precision == LDG_TC_BF16) {
    s = ctx->tcjv ? "k_euler_jv_tc [" + what + (precision == LDG_TC_BF16X3 ? " bf16x3" : " bf16") +
                        " tcgen05 contractions, fp32 pointwise, 32 elements per CTA]"
                  : "";
    return s.c_str();
  }
  what += f32 ? " fp32" : " fp64";
  if (ctx->ks->linear && (f32 ? ctx->lin32 : ctx->lin64))
    s = nodal_names(ctx, precision) + what + (ctx->lin_cart && !(f32 && ctx->etype == LDG_HEX) ? " cartesian" : "") +
        ", q scratch " + (f32 ? "fp32" : "fp64") + "]";
  else if (ctx->ks->qstage)
    s = std::string(ctx->pg ? "k_qstage_curved" : "k_qstage") + " + k_residual [" + what + ", tile " +
        std::to_string(ctx->ks->tile) + "]";
  else
    s = "k_residual [" + what + ", tile " + std::to_string(ctx->ks->tile) + "]";
  return s.c_str();
}

int ldg_jvp_host(ldg_ctx* ctx, int precision, const double* u_host, const double* v_host, double* jv_host) {
  if (!ctx || !ctx->ks || !v_host || !jv_host || !jv_precision_ok(precision)) return LDG_ERR_ARG;
  if (!u_host && !ctx->ks->linear)
    return fail(ctx, LDG_ERR_ARG, "ldg_jvp_host: u_host may be NULL only for linear models");
  const size_t n = (size_t)ctx->ndof, bytes = n * sizeof(double);
  if (!ctx->d_stage) CK(cudaMalloc(&ctx->d_stage, 3 * bytes));
  double *du = ctx->d_stage, *dv = du + n, *djv = dv + n;
  if (u_host) CK(cudaMemcpyAsync(du, u_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(dv, v_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
  // a linear model's J.v does not read u: the direction stands in for it
  int rc = jvp_args(ctx, base_args(ctx), u_host ? du : dv, dv, djv, precision);
  if (rc) return rc;
  CK(cudaMemcpyAsync(jv_host, djv, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return LDG_OK;
}

int ldg_jvp_host_many(ldg_ctx* ctx, int precision, const double* u_host, int count, const double* const* v_host,
                      double* const* jv_host) {
  if (!ctx || !ctx->ks || count < 1 || !v_host || !jv_host || !jv_precision_ok(precision)) return LDG_ERR_ARG;
  for (int i = 0; i < count; ++i)
    if (!v_host[i] || !jv_host[i]) return fail(ctx, LDG_ERR_ARG, "ldg_jvp_host_many: null direction or output");
  if (!u_host && !ctx->ks->linear)
    return fail(ctx, LDG_ERR_ARG, "ldg_jvp_host_many: u_host may be NULL only for linear models");
  const size_t n = (size_t)ctx->ndof, bytes = n * sizeof(double);
  if (!ctx->d_stage_many) CK(cudaMalloc(&ctx->d_stage_many, 5 * bytes));
  if (!ctx->s_in) {
    CK(cudaStreamCreateWithFlags(&ctx->s_in, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&ctx->s_out, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
      CK(cudaEventCreateWithFlags(&ctx->ev_in[k], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ctx->ev_done[k], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ctx->ev_out[k], cudaEventDisableTiming));
    }
  }
  double* du = ctx->d_stage_many;
  double* dv[2] = {du + n, du + 2 * n};
  double* djv[2] = {du + 3 * n, du + 4 * n};
  // the copy streams start after the work already queued on the context's stream
  CK(cudaEventRecord(ctx->ev_done[0], ctx->stream));
  CK(cudaStreamWaitEvent(ctx->s_in, ctx->ev_done[0], 0));
  CK(cudaStreamWaitEvent(ctx->s_out, ctx->ev_done[0], 0));
  if (u_host) CK(cudaMemcpyAsync(du, u_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
  for (int i = 0; i < count; ++i) {
    const int s = i & 1;
    // slot s: its v is free once the J.v of direction i - 2 has run, its J.v once that
    // result has been copied out
    if (i >= 2) CK(cudaStreamWaitEvent(ctx->s_in, ctx->ev_done[s], 0));
    CK(cudaMemcpyAsync(dv[s], v_host[i], bytes, cudaMemcpyHostToDevice, ctx->s_in));
    CK(cudaEventRecord(ctx->ev_in[s], ctx->s_in));
    CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_in[s], 0));
    if (i >= 2) CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_out[s], 0));
    int rc = jvp_args(ctx, base_args(ctx), u_host ? du : dv[s], dv[s], djv[s], precision);
    if (rc) {
      cudaStreamSynchronize(ctx->stream);
      cudaStreamSynchronize(ctx->s_in);
      cudaStreamSynchronize(ctx->s_out);
      return rc;
    }
    CK(cudaEventRecord(ctx->ev_done[s], ctx->stream));
    CK(cudaStreamWaitEvent(ctx->s_out, ctx->ev_done[s], 0));
    CK(cudaMemcpyAsync(jv_host[i], djv[s], bytes, cudaMemcpyDeviceToHost, ctx->s_out));
    CK(cudaEventRecord(ctx->ev_out[s], ctx->s_out));
  }
  CK(cudaStreamSynchronize(ctx->s_out));
  CK(cudaStreamSynchronize(ctx->s_in));
  CK(cudaStreamSynchronize(ctx->stream));
  return LDG_OK;
}

// out = sum_k c[k] x[k] over the non-null x[k] (k < 4); out may alias none of them
__global__ void k_lincomb4(double* out, int64_t n, double c0, const double* x0, double c1, const double* x1, double c2,
                           const double* x2, double c3, const double* x3) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    if (x0) s += c0 * x0[i];
    if (x1) s += c1 * x1[i];
    if (x2) s += c2 * x2[i];
    if (x3) s += c3 * x3[i];
    out[i] = s;
  }
}

namespace {
// Singly diagonally implicit Runge-Kutta tableaus: backward Euler; the L-stable,
// stiffly accurate two- and three-stage schemes of Alexander (1977) (orders 2, 3);
// the three-stage order-4 A-stable scheme of Crouzeix (1975).
struct Dirk {
  int s = 0;
  double A[3][3] = {}, b[3] = {}, c[3] = {};
};
bool dirk_tableau(int scheme, Dirk& d) {
  if (scheme == LDG_DIRK11) {
    d.s = 1; d.A[0][0] = 1.0; d.b[0] = 1.0; d.c[0] = 1.0;
  } else if (scheme == LDG_DIRK22) {
    const double g = 1.0 - std::sqrt(0.5);            // g^2 - 2 g + 1/2 = 0
    d.s = 2;
    d.A[0][0] = g; d.A[1][0] = 1.0 - g; d.A[1][1] = g;
    d.b[0] = 1.0 - g; d.b[1] = g; d.c[0] = g; d.c[1] = 1.0;
  } else if (scheme == LDG_DIRK33) {
    // g: the root in (1/3, 1/2) of g^3 - 3 g^2 + 3 g / 2 - 1/6 (bisection)
    auto f = [](double x) { return ((x - 3.0) * x + 1.5) * x - 1.0 / 6.0; };
    double lo = 1.0 / 3.0, hi = 0.5;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (f(mid) * f(lo) > 0.0) lo = mid; else hi = mid;
    }
    const double g = 0.5 * (lo + hi), t2 = 0.5 * (1.0 + g);
    const double b1 = -(6.0 * g * g - 16.0 * g + 1.0) / 4.0, b2 = (6.0 * g * g - 20.0 * g + 5.0) / 4.0;
    d.s = 3;
    d.A[0][0] = g; d.A[1][0] = t2 - g; d.A[1][1] = g; d.A[2][0] = b1; d.A[2][1] = b2; d.A[2][2] = g;
    d.b[0] = b1; d.b[1] = b2; d.b[2] = g; d.c[0] = g; d.c[1] = t2; d.c[2] = 1.0;
  } else if (scheme == LDG_DIRK34) {
    const double g = std::cos(M_PI / 18.0) / std::sqrt(3.0) + 0.5;
    const double del = 1.0 / (6.0 * (2.0 * g - 1.0) * (2.0 * g - 1.0));
    d.s = 3;
    d.A[0][0] = g; d.A[1][0] = 0.5 - g; d.A[1][1] = g; d.A[2][0] = 2.0 * g; d.A[2][1] = 1.0 - 4.0 * g; d.A[2][2] = g;
    d.b[0] = del; d.b[1] = 1.0 - 2.0 * del; d.b[2] = del; d.c[0] = g; d.c[1] = 0.5; d.c[2] = 1.0 - g;
  } else {
    return false;
  }
  return true;
}
}  // namespace

// Spatial residual R_s(u): no time term, no stage constant.
int do_residual_spatial(ldg_ctx* ctx, const double* u, double* r) {
  KArgs a = base_args(ctx);
  if (ctx->ks->qstage) {
    a.u = u; a.out = ctx->d_q;
    state_copies(ctx, a);
    CK(ctx->ks->qstage(MODE_R, a, ctx->stream));
    a = base_args(ctx);
    a.q = ctx->d_q;
  }
  a.u = u; a.out = r;
  a.hist = nullptr; a.a0dt = 0.0; a.radd = nullptr;
  CK(ctx->ks->residual(MODE_R, a, ctx->stream));
  return LDG_OK;
}

int ldg_dirk_step(ldg_ctx* ctx, int scheme, double t, double dt, double* u, ldg_solve_report* rep) {
  Dirk d;
  if (!ctx || !ctx->ks || !u || !(dt > 0) || !dirk_tableau(scheme, d)) return LDG_ERR_ARG;
  const int64_t n = ctx->ndof;
  if (!ctx->d_radd) CK(cudaMalloc(&ctx->d_radd, n * sizeof(double)));
  if (!ctx->d_dirk) CK(cudaMalloc(&ctx->d_dirk, (size_t)7 * n * sizeof(double)));
  double* un = ctx->d_dirk;                      // u at the start of the step
  double* Rs[3] = {un + n, un + 2 * n, un + 3 * n};      // spatial residuals of the stages
  double* K[3] = {un + 4 * n, un + 5 * n, un + 6 * n};   // stage slopes
  const int64_t g1 = std::min<int64_t>(grid_for(n), 148 * 8);
  CK(cudaMemcpyAsync(un, u, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  ldg_solve_report total{};
  int rc = LDG_OK;
  for (int i = 0; i < d.s && !rc; ++i) {
    const double g = d.A[i][i];
    // radd = sum_{j<i} (a_ij / a_ii) R_s(U_j)
    const double* x[3] = {nullptr, nullptr, nullptr};
    double cf[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < i; ++j) { x[j] = Rs[j]; cf[j] = d.A[i][j] / g; }
    k_lincomb4<<<g1, 256, 0, ctx->stream>>>(ctx->d_radd, n, cf[0], x[0], cf[1], x[1], cf[2], x[2], 0.0, nullptr);
    count_launch();
    CK(cudaGetLastError());
    // stage residual: M (U - u^n) / (g dt) + R_s(U) + radd, at t + c_i dt
    if ((rc = ldg_set_time(ctx, LDG_BDF1, t + d.c[i] * dt, g * dt, un, nullptr))) break;
    ctx->radd_on = true;
    ldg_solve_report r{};
    rc = ldg_newton_gmres(ctx, u, &r);
    ctx->radd_on = false;
    total.newton_iters += r.newton_iters;
    total.gmres_iters += r.gmres_iters;
    total.jv_calls += r.jv_calls;
    total.residual_calls += r.residual_calls;
    total.pc_setups += r.pc_setups;
    total.pc_fallbacks += r.pc_fallbacks;
    total.newton_backtracks += r.newton_backtracks;
    if (i == 0) total.r0 = r.r0;
    total.rfinal = std::max(total.rfinal, r.rfinal / (r.r0 > 0 ? r.r0 : 1.0));
    total.lin_resid = std::max(total.lin_resid, r.lin_resid);
    if (rc) break;
    if ((rc = do_residual_spatial(ctx, u, Rs[i]))) break;
    // K_i = (U_i - u^n) / (g dt) - sum_{j<i} (a_ij / g) K_j
    const double* kx[3] = {nullptr, nullptr, nullptr};
    double kc[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < i; ++j) { kx[j] = K[j]; kc[j] = -d.A[i][j] / g; }
    k_lincomb4<<<g1, 256, 0, ctx->stream>>>(K[i], n, 1.0 / (g * dt), u, -1.0 / (g * dt), un, kc[0], kx[0],
                                            kc[1], kx[1]);
    count_launch();
    CK(cudaGetLastError());
  }
  if (!rc) {
    // u^{n+1} = u^n + dt sum_i b_i K_i
    k_lincomb4<<<g1, 256, 0, ctx->stream>>>(u, n, 1.0, un, dt * d.b[0], K[0], d.s > 1 ? dt * d.b[1] : 0.0,
                                            d.s > 1 ? K[1] : nullptr, d.s > 2 ? dt * d.b[2] : 0.0,
                                            d.s > 2 ? K[2] : nullptr);
    count_launch();
    CK(cudaGetLastError());
  }
  // the context is left steady at the end time
  const int rc2 = ldg_set_time(ctx, LDG_STEADY, t + dt, 1.0, nullptr, nullptr);
  if (rep) {
    total.status = rc;
    total.elapsed_ms = 0.0;
    *rep = total;
  }
  return rc ? rc : rc2;
}

// ------------------------------------------------------------------ wave model
// The wave model of Section 2.1: Eq. 1a becomes dq/dt + grad u = 0, Eq. 1b keeps
// M du/dt + R_s(u, q) = 0, and the ODE Eq. 2, alpha dw/dt + beta w = u, recovers the
// displacement. One step of a singly diagonally implicit DIRK scheme (Section 2.2).
//
// With f = kappa q linear in q, R_s(u, q) = A u + B q with B proportional to kappa, and the
// q-stage of the diffusion model is the LDG form Qop(u) of -grad u. Stage i has
//   Q_i = Qh_i + g dt Qop(U_i),  Qh_i = q^n + dt sum_{j<i} a_ij Qop(U_j),
//   M (U_i - u^n) / (g dt) + R_s(U_i, Q_i) + sum_{j<i} (a_ij / g) R_s(U_j, Q_j) = 0,
// and R_s(U, Qh + g dt Qop(U)) = R'(U) + B Qh, where R' is the diffusion residual with
// kappa' = g dt kappa. So each stage is the context's own implicit solve with kappa'
// and the constant radd = B Qh_i + sum_{j<i} (a_ij / g) R_s(U_j, Q_j); q and w follow node by
// node. All a_ii are equal (g), so kappa' and the block-Jacobi blocks hold for every stage.
namespace {

// R_s(u, q) with the context's current kappa: the homogeneous residual stage, no time term
int wave_rs(ldg_ctx* ctx, const double* u, const double* q, double* out) {
  KArgs a = base_args(ctx);
  a.u = u; a.q = q; a.out = out;
  a.a0dt = 0.0; a.hist = nullptr; a.radd = nullptr;
  CK(ctx->ks->residual(MODE_HOM, a, ctx->stream));
  return LDG_OK;
}

}  // namespace

int ldg_wave_step(ldg_ctx* ctx, int scheme, double t, double dt, double alpha, double beta, double* u, double* q,
                  double* w, ldg_solve_report* rep) {
  Dirk d;
  if (!ctx || !ctx->ks || !u || !q || !(dt > 0) || !dirk_tableau(scheme, d)) return LDG_ERR_ARG;
  const bool diffusion = ctx->model == LDG_POISSON ||
                         (ctx->model == LDG_CONVDIFF && ctx->mp.beta[0] == 0.0 && ctx->mp.beta[1] == 0.0 &&
                          ctx->mp.beta[2] == 0.0);
  if (!diffusion || ctx->mp.cas != LDG_CASE_ZERO || ctx->ncu != 1)
    return fail(ctx, LDG_ERR_ARG,
                "ldg_wave_step: the context must be a Poisson model (or convection-diffusion with beta = 0) of case "
                "LDG_CASE_ZERO");
  const double g = d.A[0][0];
  for (int i = 1; i < d.s; ++i)
    if (d.A[i][i] != g) return fail(ctx, LDG_ERR_ARG, "ldg_wave_step: the scheme is not singly diagonally implicit");
  if (w && !(std::fabs(alpha + beta * g * dt) > 0.0))
    return fail(ctx, LDG_ERR_ARG, "ldg_wave_step: alpha + beta a_ii dt must not vanish");
  const int64_t n = ctx->ndof, nq = n * ctx->dim;
  if (!ctx->d_radd) CK(cudaMalloc(&ctx->d_radd, n * sizeof(double)));
  if (!ctx->d_wave) CK(cudaMalloc(&ctx->d_wave, (size_t)(12 * n + 6 * nq) * sizeof(double)));
  double* un = ctx->d_wave;
  double* wn = un + n;
  double* zero = wn + n;
  double* Ku[3] = {zero + n, zero + 2 * n, zero + 3 * n};      // slopes of u
  double* Rs[3] = {zero + 4 * n, zero + 5 * n, zero + 6 * n};  // R_s(U_j, Q_j)
  double* Kw[3] = {zero + 7 * n, zero + 8 * n, zero + 9 * n};  // slopes of w
  double* qn = zero + 10 * n;
  double* Qs = qn + nq;                                        // Qh_i / (g dt)
  double* Qt = Qs + nq;                                        // Q_i / (g dt)
  double* Kq[3] = {Qt + nq, Qt + 2 * nq, Qt + 3 * nq};          // slopes of q: Qop(U_j)
  const int64_t g1 = std::min<int64_t>(grid_for(n), 148 * 8), gq = std::min<int64_t>(grid_for(nq), 148 * 8);
  CK(cudaMemcpyAsync(un, u, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaMemcpyAsync(qn, q, nq * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  if (w) CK(cudaMemcpyAsync(wn, w, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaMemsetAsync(zero, 0, n * sizeof(double), ctx->stream));
  const double c2 = ctx->mp.kappa;
  const double kp = g * dt * c2;
  ctx->mp.kappa = kp;
  // the blocks of an earlier step of the same operator are kept
  ctx->pc_hold = ctx->pc_ready && ctx->pc_kappa == kp && ctx->pc_a0dt == 1.0 / (g * dt);
  ldg_solve_report total{};
  int rc = LDG_OK;
  auto lin = [&](double* out, int64_t len, double c0, const double* x0, double c1, const double* x1, double cc2,
                 const double* x2, double c3, const double* x3) -> int {
    k_lincomb4<<<len == n ? g1 : gq, 256, 0, ctx->stream>>>(out, len, c0, x0, c1, x1, cc2, x2, c3, x3);
    count_launch();
    CK(cudaGetLastError());
    return LDG_OK;
  };
  for (int i = 0; i < d.s && !rc; ++i) {
    const double* kx[3] = {nullptr, nullptr, nullptr};
    double kc[3] = {0.0, 0.0, 0.0};
    // Qs = (q^n + dt sum_{j<i} a_ij Kq_j) / (g dt)
    for (int j = 0; j < i; ++j) { kx[j] = Kq[j]; kc[j] = d.A[i][j] / g; }
    if ((rc = lin(Qs, nq, 1.0 / (g * dt), qn, kc[0], kx[0], kc[1], kx[1], 0.0, nullptr))) break;
    // radd = B Qh_i + sum_{j<i} (a_ij / g) R_s(U_j, Q_j); B Qh_i = R_s(0, Qs) with kappa'
    if ((rc = wave_rs(ctx, zero, Qs, Ku[i]))) break;
    for (int j = 0; j < 3; ++j) { kx[j] = j < i ? Rs[j] : nullptr; kc[j] = j < i ? d.A[i][j] / g : 0.0; }
    if ((rc = lin(ctx->d_radd, n, 1.0, Ku[i], kc[0], kx[0], kc[1], kx[1], kc[2], kx[2]))) break;
    // the stage solve: M (U - u^n) / (g dt) + R'(U) + radd = 0 at t + c_i dt
    if ((rc = ldg_set_time(ctx, LDG_BDF1, t + d.c[i] * dt, g * dt, un, nullptr))) break;
    ctx->radd_on = true;
    ldg_solve_report r{};
    rc = do_newton(ctx, u, &r);
    ctx->radd_on = false;
    ctx->pc_hold = true;
    total.newton_iters += r.newton_iters;
    total.gmres_iters += r.gmres_iters;
    total.jv_calls += r.jv_calls;
    total.residual_calls += r.residual_calls;
    total.pc_setups += r.pc_setups;
    total.pc_fallbacks += r.pc_fallbacks;
    if (i == 0) total.r0 = r.r0;
    total.rfinal = std::max(total.rfinal, r.rfinal / (r.r0 > 0 ? r.r0 : 1.0));
    total.lin_resid = std::max(total.lin_resid, r.lin_resid);
    if (rc) break;
    // Kq_i = Qop(U_i); Q_i / (g dt) = Qs + Kq_i; R_s(U_i, Q_i)
    {
      KArgs a = base_args(ctx);
      a.u = u; a.out = Kq[i];
      cudaError_t e = ctx->ks->qstage(MODE_HOM, a, ctx->stream);
      if (e != cudaSuccess) { rc = fail(ctx, LDG_ERR_CUDA, cudaGetErrorString(e)); break; }
    }
    if ((rc = lin(Qt, nq, 1.0, Qs, 1.0, Kq[i], 0.0, nullptr, 0.0, nullptr))) break;
    if ((rc = wave_rs(ctx, u, Qt, Rs[i]))) break;
    // Ku_i = (U_i - u^n) / (g dt) - sum_{j<i} (a_ij / g) Ku_j
    for (int j = 0; j < 3; ++j) { kx[j] = j < i ? Ku[j] : nullptr; kc[j] = j < i ? -d.A[i][j] / g : 0.0; }
    if ((rc = lin(Ku[i], n, 1.0 / (g * dt), u, -1.0 / (g * dt), un, kc[0], kx[0], kc[1], kx[1]))) break;
    if (w) {
      // alpha Kw_i + beta (w^n + dt sum_{j<=i} a_ij Kw_j) = U_i
      const double den = alpha + beta * g * dt;
      for (int j = 0; j < 3; ++j) { kx[j] = j < i ? Kw[j] : nullptr; kc[j] = j < i ? -beta * dt * d.A[i][j] / den : 0.0; }
      if ((rc = lin(Kw[i], n, 1.0 / den, u, -beta / den, wn, kc[0], kx[0], kc[1], kx[1]))) break;
    }
  }
  if (!rc) {
    // y^{n+1} = y^n + dt sum_i b_i K_i for u, q and w
    const double b1 = d.s > 1 ? dt * d.b[1] : 0.0, b2 = d.s > 2 ? dt * d.b[2] : 0.0;
    rc = lin(u, n, 1.0, un, dt * d.b[0], Ku[0], b1, d.s > 1 ? Ku[1] : nullptr, b2, d.s > 2 ? Ku[2] : nullptr);
    if (!rc) rc = lin(q, nq, 1.0, qn, dt * d.b[0], Kq[0], b1, d.s > 1 ? Kq[1] : nullptr, b2, d.s > 2 ? Kq[2] : nullptr);
    if (!rc && w)
      rc = lin(w, n, 1.0, wn, dt * d.b[0], Kw[0], b1, d.s > 1 ? Kw[1] : nullptr, b2, d.s > 2 ? Kw[2] : nullptr);
  }
  ctx->mp.kappa = c2;
  ctx->pc_hold = false;
  const int rc2 = ldg_set_time(ctx, LDG_STEADY, t + dt, 1.0, nullptr, nullptr);
  if (rep) {
    total.status = rc;
    *rep = total;
  }
  return rc ? rc : rc2;
}

int ldg_jvp_fd(ldg_ctx* ctx, int order, const double* u, const double* v, double* jv) {
  if (!ctx || !ctx->ks || !u || !v || !jv || (order != 1 && order != 2)) return LDG_ERR_ARG;
  const int64_t n = ctx->ndof;
  if (!ctx->d_fd) CK(cudaMalloc(&ctx->d_fd, (3 * n + 4) * sizeof(double)));
  double* w = ctx->d_fd;
  double* rp = w + n;
  double* rm = w + 2 * n;
  double* sc = w + 3 * n;   // u.u, v.v, then (eps, -eps, weight) from sc + 2 on
  int rc;
  if ((rc = dots(ctx, u, n, 1, u, sc, nullptr))) return rc;
  if ((rc = dots(ctx, v, n, 1, v, sc + 1, nullptr))) return rc;
  // scalars move to sc[0..2] only after both norms are read
  double* eps = sc;
  k_fd_eps<<<1, 1, 0, ctx->stream>>>(sc, eps, order);
  count_launch();
  const int64_t g1 = std::min<int64_t>(grid_for(n), 148 * 8);
  CK(cudaMemcpyAsync(w, u, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  k_axpy_dev<<<g1, 256, 0, ctx->stream>>>(v, eps, w, n);
  count_launch();
  if ((rc = do_residual(ctx, w, rp))) return rc;
  if (order == 2) {
    CK(cudaMemcpyAsync(w, u, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    k_axpy_dev<<<g1, 256, 0, ctx->stream>>>(v, eps + 1, w, n);
    count_launch();
    if ((rc = do_residual(ctx, w, rm))) return rc;
  } else {
    if ((rc = do_residual(ctx, u, rm))) return rc;
  }
  k_fd_diff<<<g1, 256, 0, ctx->stream>>>(rp, rm, eps + 2, jv, n);
  count_launch();
  CK(cudaGetLastError());
  return LDG_OK;
}

int ldg_jvp_after_residual(ldg_ctx* ctx, int precision, const double* u, const double* v, double* jv) {
  if (!ctx || !ctx->ks || !u || !v || !jv || !jv_precision_ok(precision)) return LDG_ERR_ARG;
  return jvp_args(ctx, base_args(ctx), u, v, jv, precision, true);
}

int ldg_diag_blocks(ldg_ctx* ctx, int precision, const double* u, double* blocks) {
  if (!ctx || !ctx->ks || !u || !blocks || (precision != LDG_FP64 && precision != LDG_FP32)) return LDG_ERR_ARG;
  return do_blocks(ctx, u, precision, blocks);
}

int ldg_precond_setup(ldg_ctx* ctx, const double* u) {
  if (!ctx || !ctx->ks || !u) return LDG_ERR_ARG;
  int rc = do_pc_setup(ctx, u);
  if (!rc && ctx->opt.precond == LDG_PC_RB_BJ) rc = rb_setup(ctx, u);
  return rc;
}

int ldg_precond_apply(ldg_ctx* ctx, const double* x, double* y) {
  if (!ctx || !ctx->ks || !x || !y) return LDG_ERR_ARG;
  if (!ctx->pc_ready) return fail(ctx, LDG_ERR_ARG, "ldg_precond_apply: call ldg_precond_setup first");
  if (ctx->opt.precond == LDG_PC_RB_BJ) return rb_apply(ctx, x, y, nullptr);
  return pc_apply(ctx, x, y, nullptr);
}

int ldg_rb_set_basis(ldg_ctx* ctx, const double* W, int k) {
  if (!ctx || !ctx->ks || k < 0 || (k > 0 && !W)) return LDG_ERR_ARG;
  if (ctx->rb_cap <= 0) ctx->rb_cap = ctx->opt.rb_size;
  if (k > ctx->rb_cap) return fail(ctx, LDG_ERR_ARG, "ldg_rb_set_basis: more vectors than rb_size");
  ctx->rb_k = ctx->rb_next = ctx->rb_eff = 0;
  for (int j = 0; j < k; ++j) {
    const int rc = rb_insert(ctx, W + (size_t)j * ctx->ndof, nullptr);
    if (rc) return rc;
  }
  return LDG_OK;
}

int ldg_rb_count(const ldg_ctx* ctx) { return ctx ? ctx->rb_k : 0; }

int ldg_mlp_init(ldg_ctx* ctx, uint64_t seed) {
  if (!ctx || !ctx->ks) return LDG_ERR_ARG;
  int rc;
  if ((rc = mlp_alloc(ctx))) return rc;
  auto& M = ctx->mlp;
  MlpOff o(M.n, M.h);
  // He initialisation for the ReLU layers, small output layer, zero biases
  std::mt19937_64 gen(seed);
  std::vector<float> th(M.nparam, 0.f);
  auto fill = [&](int64_t off, int rows, int cols, double sd) {
    std::normal_distribution<double> nd(0.0, sd);
    for (int64_t i = 0; i < (int64_t)rows * cols; ++i) th[off + i] = (float)nd(gen);
  };
  fill(o.W1, M.h, M.n, std::sqrt(2.0 / M.n));
  fill(o.W2, M.h, M.h, std::sqrt(2.0 / M.h));
  fill(o.W3, M.n, M.h, 0.1 * std::sqrt(1.0 / M.h));
  CK(cudaMemcpy(M.theta, th.data(), th.size() * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemset(M.m, 0, M.nparam * sizeof(float)));
  CK(cudaMemset(M.v, 0, M.nparam * sizeof(float)));
  M.t = 0;
  return mlp_refresh_bf16(ctx);
}

int ldg_mlp_params(ldg_ctx* ctx, int get, double* host, int64_t* count) {
  if (!ctx || !ctx->ks || !count) return LDG_ERR_ARG;
  int rc;
  if ((rc = mlp_alloc(ctx))) return rc;
  auto& M = ctx->mlp;
  if (!host) { *count = M.nparam; return LDG_OK; }
  if (*count < M.nparam) return fail(ctx, LDG_ERR_ARG, "ldg_mlp_params: buffer too small");
  std::vector<float> th(M.nparam);
  if (get) {
    CK(cudaMemcpy(th.data(), M.theta, M.nparam * sizeof(float), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < M.nparam; ++i) host[i] = th[i];
  } else {
    for (int64_t i = 0; i < M.nparam; ++i) th[i] = (float)host[i];
    CK(cudaMemcpy(M.theta, th.data(), M.nparam * sizeof(float), cudaMemcpyHostToDevice));
    if ((rc = mlp_refresh_bf16(ctx))) return rc;
  }
  *count = M.nparam;
  return LDG_OK;
}

int ldg_mlp_loss_grad(ldg_ctx* ctx, const double* X, const double* T, const double* U, int64_t n_pairs, double* loss,
                      double* grad) {
  if (!ctx || !ctx->ks || !X || !T || !U || n_pairs <= 0 || !loss) return LDG_ERR_ARG;
  auto& M = ctx->mlp;
  if (!M.theta) return fail(ctx, LDG_ERR_ARG, "ldg_mlp_loss_grad: call ldg_mlp_init first");
  int rc;
  if ((rc = mlp_prep(ctx, X, T, U, nullptr, n_pairs, nullptr, nullptr))) return rc;
  mlp_forward<float>(ctx, n_pairs, M.theta, M.theta, nullptr);
  if ((rc = mlp_backward(ctx, n_pairs))) return rc;
  CK(cudaMemcpyAsync(loss, M.loss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  std::vector<float> g(M.nparam);
  CK(cudaMemcpyAsync(g.data(), M.grad, M.nparam * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (grad)
    for (int64_t i = 0; i < M.nparam; ++i) grad[i] = g[i];
  return LDG_OK;
}

int ldg_mlp_train(ldg_ctx* ctx, const double* X, const double* T, const double* U, int64_t n_pairs,
                  const ldg_train_opts* opts, ldg_train_report* rep) {
  if (!ctx || !ctx->ks || !X || !T || !U || n_pairs <= 0) return LDG_ERR_ARG;
  auto& M = ctx->mlp;
  if (!M.theta) return fail(ctx, LDG_ERR_ARG, "ldg_mlp_train: call ldg_mlp_init first");
  ldg_train_opts o{};
  if (opts) o = *opts;
  if (o.epochs <= 0) o.epochs = 50;
  if (o.batch <= 0) o.batch = 4096;
  if (o.lr <= 0) o.lr = 1e-3;
  const int64_t B = std::min<int64_t>(o.batch, n_pairs);
  int rc;
  if ((rc = mlp_reserve(ctx, B))) return rc;
  if (M.idx_cap < n_pairs) {
    cudaFree(M.idx);
    M.idx = nullptr;
    CK(cudaMalloc(&M.idx, n_pairs * sizeof(int)));
    M.idx_cap = n_pairs;
  }
  auto t0 = std::chrono::steady_clock::now();
  if (o.linear_init) {
    // least-squares fit of the linear skip map on all pairs: Ws = (Xn^T Tn)^T (Xn^T Xn)^{-1},
    // with the nonlinear branch's output layer zeroed, so training starts from the best
    // state-independent linear block map
    MlpOff off(M.n, M.h);
    const int n = M.n;
    float *Gm = nullptr, *Cm = nullptr, *Gi32 = nullptr;
    double *G64 = nullptr, *Gi64 = nullptr;
    CK(cudaMalloc(&Gm, (size_t)n * n * sizeof(float)));
    CK(cudaMalloc(&Cm, (size_t)n * n * sizeof(float)));
    CK(cudaMalloc(&Gi32, (size_t)n * n * sizeof(float)));
    CK(cudaMalloc(&G64, (size_t)n * n * sizeof(double)));
    CK(cudaMalloc(&Gi64, (size_t)n * n * sizeof(double)));
    for (int64_t b0 = 0; b0 < n_pairs; b0 += B) {
      const int64_t rows = std::min<int64_t>(B, n_pairs - b0);
      if ((rc = mlp_prep(ctx, X + b0 * n, T + b0 * n, U + b0 * n, nullptr, rows, nullptr, nullptr))) return rc;
      const int acc = b0 > 0;
      gemm<true, false, float>(ctx, n, n, (int)rows, M.X, 2 * n, M.X, 2 * n, Gm, n, nullptr, 0, nullptr, acc);
      gemm<true, false, float>(ctx, n, n, (int)rows, M.X, 2 * n, M.T, n, Cm, n, nullptr, 0, nullptr, acc);
    }
    k_gram_to_f64<<<1, 256, 0, ctx->stream>>>(Gm, n, 1e-6, G64);
    count_launch();
    if ((rc = ensure_pc_storage(ctx))) return rc;
    const size_t smem = block_inverse_smem<double>(n);
    CK(cudaFuncSetAttribute(k_block_inverse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_block_inverse<double><<<1, std::min(256, ((n + 31) / 32) * 32), smem, ctx->stream>>>(G64, Gi64, n, ctx->d_status);
    count_launch();
    k_f64_to_f32<<<grid_for((int64_t)n * n), 256, 0, ctx->stream>>>(Gi64, Gi32, (int64_t)n * n);
    count_launch();
    // Ws[i][j] = sum_k C[k][i] Ginv[k][j]  (Ginv symmetric)
    gemm<true, false, float>(ctx, n, n, n, Cm, n, Gi32, n, M.theta + off.Ws, n, nullptr, 0, nullptr);
    CK(cudaMemsetAsync(M.theta + off.W3, 0, ((size_t)n * M.h + n) * sizeof(float), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(Gm); cudaFree(Cm); cudaFree(Gi32); cudaFree(G64); cudaFree(Gi64);
    CK(cudaGetLastError());
  }
  std::vector<int> perm(n_pairs);
  std::iota(perm.begin(), perm.end(), 0);
  std::mt19937_64 gen(o.seed);
  double first = -1.0, last = 0.0;
  int steps = 0;
  std::vector<double> epoch_loss;
  for (int ep = 0; ep < o.epochs; ++ep) {
    std::shuffle(perm.begin(), perm.end(), gen);
    CK(cudaMemcpyAsync(M.idx, perm.data(), n_pairs * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    double acc = 0.0;
    int nb = 0;
    for (int64_t b0 = 0; b0 + B <= n_pairs; b0 += B) {
      if ((rc = mlp_prep(ctx, X, T, U, M.idx + b0, B, nullptr, nullptr))) return rc;
      mlp_forward<float>(ctx, B, M.theta, M.theta, nullptr);
      if ((rc = mlp_backward(ctx, B))) return rc;
      ++M.t;
      k_adam<<<std::min<int64_t>(grid_for(M.nparam), 148 * 4), 256, 0, ctx->stream>>>(
          M.theta, M.grad, M.m, M.v, M.nparam, (float)o.lr, 0.9f, 0.999f, 1e-8f, M.t);
      count_launch();
      double l = 0.0;
      CK(cudaMemcpyAsync(ctx->h_pin, M.loss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      l = ctx->h_pin[0];
      acc += l;
      ++nb;
      ++steps;
    }
    const double el = nb ? acc / nb : 0.0;
    if (first < 0) first = el;
    last = el;
  }
  if ((rc = mlp_refresh_bf16(ctx))) return rc;
  CK(cudaStreamSynchronize(ctx->stream));
  if (rep) {
    rep->loss_first = first;
    rep->loss_last = last;
    rep->steps = steps;
    rep->elapsed_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return LDG_OK;
}

int ldg_mlp_apply(ldg_ctx* ctx, const double* u, const double* x, double* y) {
  if (!ctx || !ctx->ks || !u || !x || !y) return LDG_ERR_ARG;
  if (!ctx->mlp.ready) return fail(ctx, LDG_ERR_ARG, "ldg_mlp_apply: no trained network (ldg_mlp_init/train)");
  int rc = mlp_apply(ctx, u, x, y, nullptr);
  if (rc || !ctx->mlp.d_err) return rc;
  int err = 0;
  CK(cudaMemcpyAsync(&err, ctx->mlp.d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (err) return fail(ctx, LDG_ERR_CUDA, "tensor-core GEMM: a TMA or MMA wait timed out");
  return LDG_OK;
}

int ldg_newton_gmres_collect(ldg_ctx* ctx, double* u, double* X, double* T, double* U, int capacity, int* count,
                             ldg_solve_report* rep) {
  if (!ctx || !ctx->ks || !u || !X || !T || !U || capacity <= 0 || !count) return LDG_ERR_ARG;
  if (ctx->opt.precond != LDG_PC_BJACOBI)
    return fail(ctx, LDG_ERR_ARG, "ldg_newton_gmres_collect: needs the block-Jacobi preconditioner");
  ctx->col_X = X; ctx->col_T = T; ctx->col_U = U; ctx->col_cap = capacity; ctx->col_count = 0;
  int rc = ldg_newton_gmres(ctx, u, rep);
  *count = ctx->col_count;
  ctx->col_X = nullptr; ctx->col_T = nullptr; ctx->col_U = nullptr; ctx->col_cap = 0;
  return rc;
}

int ldg_newton_collect_updates(ldg_ctx* ctx, double* u, double* X, double* T, double* U, int capacity, int which,
                               int* count, ldg_solve_report* rep) {
  if (!ctx || !ctx->ks || !u || !X || !T || !U || capacity <= 0 || !count || which < 1 || which > 3)
    return LDG_ERR_ARG;
  int rc;
  if ((rc = ensure_halo(ctx))) return rc;
  const int pc = ctx->opt.precond;
  ctx->opt.precond = LDG_PC_BJACOBI;
  ctx->col_X = X; ctx->col_T = T; ctx->col_U = U; ctx->col_cap = capacity; ctx->col_count = 0;
  ctx->col_mode = which;
  rc = ldg_newton_gmres(ctx, u, rep);
  *count = ctx->col_count;
  ctx->col_X = nullptr; ctx->col_T = nullptr; ctx->col_U = nullptr; ctx->col_cap = 0; ctx->col_mode = 0;
  ctx->opt.precond = pc;
  return rc;
}

int ldg_halo_features(ldg_ctx* ctx, const double* z, double* h) {
  if (!ctx || !ctx->ks || !z || !h) return LDG_ERR_ARG;
  return halo_features(ctx, z, h, nullptr);
}

int ldg_mlp_bj_apply(ldg_ctx* ctx, const double* x, double* y) {
  if (!ctx || !ctx->ks || !x || !y) return LDG_ERR_ARG;
  if (!ctx->mlp.ready) return fail(ctx, LDG_ERR_ARG, "ldg_mlp_bj_apply: no trained network (ldg_mlp_init/train)");
  if (!ctx->pc_ready) return fail(ctx, LDG_ERR_ARG, "ldg_mlp_bj_apply: no block-Jacobi blocks (ldg_precond_setup)");
  return mlp_bj_apply(ctx, x, y, nullptr);
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
                                                                      GEO, ctx->d_xn, ctx->mp, t, u, ctx->d_xnode);
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
  int rc;
  // block-Jacobi built once per call, or no preconditioner: the graph-driven solver
  // (the whole Newton-GMRES one CUDA graph launch); otherwise the host-driven loop
  if (ctx->opt.precond != LDG_PC_MLP && ctx->opt.precond != LDG_PC_MLP_BJ && ctx->opt.precond != LDG_PC_RB_BJ &&
      ctx->opt.pc_refresh == 0 && !ctx->col_X) {
    if (!ctx->engine && (rc = batch_wrap(ctx, &ctx->engine))) {
      rep->status = rc;
      return rc;
    }
    rc = batch_solve_one(ctx->engine, u, rep);
    if (rc) ctx->err = batch_error(ctx->engine);
  } else {
    rc = do_newton(ctx, u, rep);
  }
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
  // linear models: Q v; nonlinear models with q: q(u) and Q v
  const size_t nq = (size_t)ctx->ndof * ctx->dim;
  const size_t need = ctx->ks->linear ? nq : 2 * nq;
  if (need > kNoAllocScratchDoubles)
    return fail(ctx, LDG_ERR_ARG, "ldg_jvp_noalloc: this operator needs " + std::to_string(need) +
                                      " doubles of scratch (n_dof * dim per q field), more than the static maximum of " +
                                      std::to_string(kNoAllocScratchDoubles));
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(ctx, LDG_ERR_ARG, "ldg_jvp_noalloc: device ordinal out of range");
  double* dq = noalloc_addr[dev].load(std::memory_order_acquire);
  if (!dq) {
    std::lock_guard<std::mutex> hold(noalloc_lock);
    dq = noalloc_addr[dev].load(std::memory_order_acquire);
    if (!dq) {
      void* p = nullptr;
      CK(cudaGetSymbolAddress(&p, noalloc_scratch));
      dq = (double*)p;
      noalloc_addr[dev].store(dq, std::memory_order_release);
    }
  }
  // each q-stage overwrites every entry that is later read: nothing to clear
  KArgs a = base_args(ctx);
  a.u = v; a.out = dq;
  CK(ctx->ks->qstage(MODE_HOM, a, ctx->stream));
  if (ctx->ks->linear) {
    a = base_args(ctx);
    a.u = v; a.q = dq; a.out = jv;
    CK(ctx->ks->residual(MODE_HOM, a, ctx->stream));
    return LDG_OK;
  }
  double* qu = dq + nq;
  a = base_args(ctx);
  a.u = u; a.out = qu;
  CK(ctx->ks->qstage(MODE_R, a, ctx->stream));
  a = base_args(ctx);
  a.u = u; a.v = v; a.q = qu; a.dq = dq; a.out = jv;
  CK(ctx->ks->residual(MODE_JV, a, ctx->stream));
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
