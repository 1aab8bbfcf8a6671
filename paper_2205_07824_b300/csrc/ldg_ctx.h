// Internal interface shared by the single-problem C-ABI and the batched solver:
// the context record and the helpers both use. Not part of the public ABI.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ldg.h"
#include "ldg_launch.cuh"

struct ldg_ctx {
  int etype = 0, p = 0, nq = 0, dim = 0, npe = 0, ncu = 0, nf = 0, nfq = 0, model = 0;
  int64_t E = 0, ndof = 0;
  ldg::ModelParams mp{};
  ldg_options opt{};
  cudaStream_t stream = nullptr;
  const ldg::KernelSet* ks = nullptr;
  // device data
  double* d_ops = nullptr;
  float* d_opsf = nullptr;
  double* d_geo = nullptr;
  int* d_nbr = nullptr;
  unsigned char* d_nbf = nullptr;
  unsigned char* d_perm = nullptr;
  double* d_xn = nullptr;      // reference node coordinates [npe][dim]
  // curved elements (pg > 0): per-point geometry records (see CurvedPrep)
  int pg = 0;
  double* d_cgeo = nullptr;
  float* d_cgeof = nullptr;
  double* d_cx = nullptr;
  double* d_minv = nullptr;
  float* d_minvf = nullptr;
  double* d_xnode = nullptr;   // [E][npe][dim] physical node coordinates
  double* d_q = nullptr;       // q(u) scratch [E][ncu][dim][npe]
  double* d_dq = nullptr;      // q(v) scratch (FP32 values for the FP32 J.v)
  float* d_q32 = nullptr;      // nonlinear models with q: FP32 copies of q(u) and u, written by
  float* d_u32 = nullptr;      // the residual's q-stage and read by the FP32 J.v
  double* d_hist = nullptr;    // BDF history term
  double* d_radd = nullptr;    // DIRK stage: constant added to the residual (active when radd_on)
  bool radd_on = false;
  double* d_dirk = nullptr;    // DIRK work: u^n, then the stages' spatial residuals and slopes
  double* d_wave = nullptr;    // wave steps: u^n, q^n, w^n and the stages' slopes and residuals
  double pc_kappa = 0.0, pc_a0dt = -1.0;  // kappa and a0/dt the block-Jacobi blocks were built with
  bool pc_hold = false;        // do_newton keeps the built blocks (wave stages of one operator)
  // reduced-basis preconditioner (LDG_PC_RB_BJ)
  int rb_cap = 0, rb_k = 0, rb_next = 0;  // capacity, vectors held, slot replaced next when full
  int rb_eff = 0;              // vectors the current set-up uses (0: block-Jacobi alone)
  double* d_rbW = nullptr;     // [rb_cap][n] orthonormal reduced basis
  double* d_rbJW = nullptr;    // [rb_cap][n] J W at the Newton state of the set-up
  double* d_rbS = nullptr;     // small scratch: W^T x, y, J_r, J_r^{-1}, norms
  double* d_rbC = nullptr;     // [2 n] scratch: C x and the remainder x - J C x
  std::vector<double> h_rbJr;  // [32][32] G = (J W)^T J W (row-major), kept with rb_eff
  // nodal J.v kernels of linear models on affine tensor elements (null when not applicable)
  ldg::LinFn lin64 = nullptr, lin32 = nullptr;
  ldg::LinFn linff = nullptr;
  bool lin_cart = false;   // the nodal kernels' axis-aligned-box instances (every element a box)
  // Euler on affine quadrilaterals: the tensor-core J.v and its constant operand image
  ldg::TcJvFn tcjv = nullptr;
  unsigned char* d_tcimg = nullptr;
  int* d_tcerr = nullptr;
  std::vector<double> h_lops;    // host copy of the nodal kernels' FP64 operator blob   // the same in (hi, lo) float-pair arithmetic (LDG_F32X2)
  double* d_lops = nullptr;
  float* d_lopsf = nullptr;
  // element-sharded use (ldg_shard_*): owned elements, the caller's transport, q and
  // reduction buffers
  int64_t shard_owned = 0;
  ldg_comm shard_comm{};
  double *d_shq = nullptr, *d_shpart = nullptr, *d_shdot = nullptr;
  std::vector<double> h_shdot;
  double* d_stage = nullptr;   // ldg_jvp_host: device copies of u, v and J.v (3 n_dof, first use)
  // ldg_jvp_host_many: u, two (v, J.v) slots (5 n_dof), the copy-in and copy-out streams and
  // per-slot events (copied in, J.v done, copied out); created on first use
  double* d_stage_many = nullptr;
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
  // L2 projection / error rule (built on first use): points, weights, basis values,
  // projection operator, and per-element error partials [E][4]
  int er_nqp = 0;
  double *d_er_xi = nullptr, *d_er_w = nullptr, *d_er_B = nullptr, *d_er_P = nullptr, *d_l2 = nullptr;
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
  double* d_small = nullptr;   // H, cs, sn, g, y, h1, h2, scalars (KrySmall)
  double* d_part = nullptr;    // reduction partials [nblk][32]
  int* d_flags = nullptr;      // done, columns, breakdown
  unsigned int* d_ticket = nullptr;
  double* h_pin = nullptr;     // pinned host scalars
  int* h_flags = nullptr;      // pinned copies of the flags, one slot per Arnoldi step
  cudaEvent_t ev[64] = {};
  int nblk = 0;                // grid of streaming vector kernels
  int nblk_d = 0;              // grid of the many-accumulator reductions (dot products)
  // block-Jacobi preconditioner
  int nloc = 0;
  std::vector<int> h_nbr;      // host copy of the face neighbours (colouring)
  std::vector<unsigned char> h_nbf, h_perm;   // host copies of the neighbour faces and permutations
  int* d_halo = nullptr;       // [E][npe][3] neighbour node (nbr * npe + node) per face holding the node, -1 none
  double* d_pcz = nullptr;     // learned block-Jacobi correction: z = BJ^{-1} v ...
  double* d_pch = nullptr;     // ... and its neighbour-trace features
  int* d_colour = nullptr;
  int ncolour = 0;
  double* d_blocks = nullptr;  // [E][nloc][nloc] exact diagonal blocks, column-major
  void* d_binv = nullptr;      // their inverses (float or double)
  int binv_prec = -1;
  double* d_Z = nullptr;       // [m][ndof] preconditioned Krylov vectors (flexible GMRES)
  double* d_fd = nullptr;      // finite-difference J.v: three work vectors and four scalars
  double* d_probe = nullptr;   // probing work vectors (linear models)
  double* d_jp = nullptr;
  int* d_status = nullptr;
  bool pc_ready = false;
  // learned per-element MLP preconditioner
  struct Mlp {
    int n = 0, h = 128;
    int64_t nparam = 0;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16* theta_bf = nullptr;
    int64_t cap = 0;                       // rows of the work buffers
    float *X = nullptr, *T = nullptr, *mask = nullptr, *H1 = nullptr, *H2 = nullptr, *Y = nullptr;
    float *dY = nullptr, *dH1 = nullptr, *dH2 = nullptr;
    double* norms = nullptr;
    double* loss = nullptr;
    int* count = nullptr;
    int* idx = nullptr;
    int64_t idx_cap = 0;
    int t = 0;
    bool ready = false;
    // tensor-core inference: BF16 activations, aligned BF16 weight copies, TMA maps
    bool tc = false;                       // shapes suit the tcgen05 GEMM (n, 2n, h multiples of 64)
    __nv_bfloat16 *Xbf = nullptr, *H1bf = nullptr, *H2bf = nullptr, *wtc = nullptr;
    int64_t tc_rows = 0;
    CUtensorMap maps[8];                   // A: X, X[:, :n], H1, H2; B: W1, W2, W3, Ws
    int* d_err = nullptr;
  } mlp;
  // pair collection during Newton (training data)
  double* col_X = nullptr;
  double* col_T = nullptr;
  double* col_U = nullptr;
  int col_cap = 0, col_count = 0;
  int col_mode = 0;            // 0: Arnoldi triples (v, BJ^{-1} v, u); else a mask: 1 Newton updates,
                               // 2 Arnoldi inverse pairs (J z_j, z_j), as (BJ^{-1} r, d, halo)
  // batched contexts: per-element instance ids and the per-instance parameter table
  // (owned by the batch, not by this context)
  const int* ext_inst = nullptr;
  const ldg::ModelParams* ext_mtab = nullptr;
  bool lean = false;           // no Krylov basis or preconditioned vectors (batch groups)
  double* d_t = nullptr;       // boundary-data time in device memory (read by captured graphs)
  ldg_batch* engine = nullptr; // graph-driven Newton-GMRES over this context (created on first use)
  std::string err;
};


namespace ldg {
namespace impl {
const std::vector<KernelSet>& registry();
int fail(ldg_ctx* c, int code, const std::string& msg);
// Have a residual's FP64 q-stage (MODE_R into ctx->d_q) write the FP32 copies of u and q(u).
void state_copies(ldg_ctx* ctx, KArgs& a);
KArgs base_args(ldg_ctx* c);
int64_t grid_for(int64_t n, int t = 256);
int do_residual(ldg_ctx* ctx, const double* u, double* r);
// J.v in the given arithmetic; q_ready: ctx->d_q already holds q(u) (nonlinear models
// with q, after a residual evaluation at the same u)
int jvp_args(ldg_ctx* ctx, KArgs a, const double* u, const double* v, double* jv, int prec, bool q_ready = false);
int ensure_pc_storage(ldg_ctx* ctx);
int do_pc_setup(ldg_ctx* ctx, const double* u);
int pc_apply(ldg_ctx* ctx, const double* x, double* y, const int* skip, const int* inst_skip = nullptr);
// ldg_create with `lean` contexts (no Krylov work space) for batch groups
int create_ctx(ldg_ctx** out, const ldg_mesh_desc* mesh, int p, const ldg_model_desc* model, const ldg_options* opts,
               void* cuda_stream, bool lean);
// Times every compiled tile of the context's (element, order, model) on its mesh and
// selects the fastest J.v in the Krylov precision; force = 0 reuses a cached choice.
int autotune(ldg_ctx* ctx, int force, int* tile, double* best_ms);
ModelParams make_params(const ldg_model_desc* model);
// The graph-driven batched solver with one borrowed context as its only instance.
int batch_wrap(ldg_ctx* ctx, ldg_batch** out);
int batch_solve_one(ldg_batch* b, double* u, ldg_solve_report* rep);
void batch_free(ldg_batch* b);
const char* batch_error(const ldg_batch* b);
}  // namespace impl
}  // namespace ldg
