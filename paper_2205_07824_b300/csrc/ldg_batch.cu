// Batched parametrised problems (include/ldg.h, "batched parametrised problems"):
// many independent steady LDG problems solved together by Newton-GMRES
// (Section 3.3), the whole solve one CUDA graph launch.
//
// Instances with the same (element, order, quadrature, model) form a group whose
// meshes are joined into one disjoint mesh (vertex ids shifted per instance), so a
// group is an ordinary context with a per-element instance index into a table of
// model parameters: every residual / J.v / preconditioner launch covers all of its
// instances. The Krylov and Newton kernels (ldg_batch.cuh) work on the batch vector
// with per-instance segmented reductions and per-instance convergence, and the
// Newton, restart and Arnoldi loops are CUDA graph WHILE nodes whose conditions the
// loop-control kernels set on the device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "ldg_batch.cuh"
#include "ldg_ctx.h"

using namespace ldg;
using namespace ldg::impl;

namespace {

struct BGroup {
  ldg_ctx* ctx = nullptr;
  int64_t off = 0, ndof = 0;   // slice of the batch vector
  int* d_inst = nullptr;       // [E] instance (segment) of each element
  int etype = 0, p = 0, nq = 0, model = 0;
  bool pc_built = false;       // blocks built by this batch, with the coefficients below
  int pc_scheme = 0;
  double pc_a0dt = 0.0;
};

}  // namespace

struct ldg_batch {
  int n_inst = 0;
  ldg_options opt{};
  cudaStream_t stream = nullptr;   // the caller's stream
  cudaStream_t cap = nullptr;      // private stream used to capture the graph
  std::vector<BGroup> groups;
  std::vector<int> seg_user;       // segment -> user instance
  std::vector<int64_t> user_off, user_n;
  int64_t ntot = 0;
  int nseg = 0, nchunk = 0, m = 30;
  ModelParams* d_mtab = nullptr;
  int *d_chunk_seg = nullptr, *d_seg_c0 = nullptr, *d_seg_nc = nullptr;
  int64_t *d_chunk_lo = nullptr, *d_chunk_hi = nullptr;
  double* d_part = nullptr;
  int* d_bt = nullptr;         // [n_seg] Newton step being halved at the current iteration
  double* d_ubase = nullptr;   // [n_total] last accepted Newton iterate
  unsigned int* d_tick = nullptr;
  double* d_small = nullptr;
  int* d_sflags = nullptr;
  SegState* d_st = nullptr;
  BatchCtl* d_ctl = nullptr;
  int *d_skip_newt = nullptr, *d_skip_gm = nullptr, *d_skip_arn = nullptr;
  double *d_u = nullptr, *d_res = nullptr, *d_r = nullptr, *d_x = nullptr, *d_w = nullptr;
  double *d_vcur = nullptr, *d_zcur = nullptr, *d_V = nullptr, *d_Z = nullptr;
  float2* d_wf = nullptr;          // pair basis: the vector being orthogonalised, as (hi, lo) floats
  bool ff = false;                 // krylov_basis == LDG_BASIS_F32X2: V holds (hi, lo) float pairs
  bool pc = false;
  long long solves = 0;            // ldg_batch_solve calls (block-Jacobi reuse)
  bool borrowed = false;           // one instance whose context belongs to the caller
  std::vector<const KernelSet*> cap_ks;   // per group: kernels, time scheme and a0/dt the graph holds
  std::vector<int> cap_scheme;
  std::vector<double> cap_a0dt;
  std::vector<char> cap_radd;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long k_pre = 0, k_a = 0, k_b = 0, k_c = 0;   // kernels per graph part (captured)
  long long last_exec = 0;
  std::string err;
};

namespace {

int bfail(ldg_batch* b, int code, const std::string& msg) {
  if (b) b->err = msg;
  return code;
}

#define BK(call)                                                                               \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return bfail(b, LDG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
  } while (0)

// a group helper failed: carry its message over
int gfail(ldg_batch* b, const BGroup& g, int rc) { return bfail(b, rc, g.ctx ? g.ctx->err : "group error"); }

SegView seg_view(const ldg_batch* b) {
  SegView v;
  v.chunk_seg = b->d_chunk_seg; v.chunk_lo = b->d_chunk_lo; v.chunk_hi = b->d_chunk_hi;
  v.seg_c0 = b->d_seg_c0; v.seg_nc = b->d_seg_nc;
  v.part = b->d_part; v.tick = b->d_tick;
  v.small = b->d_small; v.ks = (int64_t)KrySmall{b->m}.total(); v.m = b->m;
  v.sflags = b->d_sflags; v.nseg = b->nseg; v.nchunk = b->nchunk;
  return v;
}

int default_nq(int etype, int model, int p) {
  return (model == LDG_EULER || model == LDG_NS || etype == LDG_TRI || etype == LDG_TET) ? p + 2 : p + 1;
}
int verts_per_elem(int etype) {
  return etype == LDG_TRI ? 3 : (etype == LDG_QUAD || etype == LDG_TET) ? 4 : 8;
}

// ------------------------------------------------------------ stage emission
int emit_residual(ldg_batch* b, cudaStream_t s, const double* u, double* r, const int* skip) {
  for (BGroup& g : b->groups) {
    g.ctx->stream = s;
    // per-instance skipping needs the element -> instance map (absent for one borrowed context)
    const int* sk = g.ctx->ext_inst ? skip : nullptr;
    KArgs a = base_args(g.ctx);
    a.inst_skip = sk;
    if (g.ctx->ks->qstage) {
      a.u = u + g.off; a.out = g.ctx->d_q;
      state_copies(g.ctx, a);
      BK(g.ctx->ks->qstage(MODE_R, a, s));
      a = base_args(g.ctx);
      a.inst_skip = sk;
      a.q = g.ctx->d_q;
    }
    a.u = u + g.off; a.out = r + g.off;
    a.hist = g.ctx->scheme != LDG_STEADY ? g.ctx->d_hist : nullptr;
    BK(g.ctx->ks->residual(MODE_R, a, s));
  }
  return LDG_OK;
}

// q_ready: the last residual was evaluated at u (its q-stage left q(u) in each group)
int emit_jv(ldg_batch* b, cudaStream_t s, const double* u, const double* v, double* jv, int prec, const int* skip,
            bool q_ready) {
  for (BGroup& g : b->groups) {
    g.ctx->stream = s;
    KArgs a = base_args(g.ctx);
    a.inst_skip = g.ctx->ext_inst ? skip : nullptr;
    int rc = jvp_args(g.ctx, a, u + g.off, v + g.off, jv + g.off, prec, q_ready);
    if (rc) return gfail(b, g, rc);
  }
  return LDG_OK;
}

int emit_pc(ldg_batch* b, cudaStream_t s, const double* x, double* y, const int* skip) {
  for (BGroup& g : b->groups) {
    g.ctx->stream = s;
    int rc = pc_apply(g.ctx, x + g.off, y + g.off, nullptr, g.ctx->ext_inst ? skip : nullptr);
    if (rc) return gfail(b, g, rc);
  }
  return LDG_OK;
}

// Newton body, part 1: R(u), ||R_s||, convergence test, linear-solve start.
int emit_newton_head(ldg_batch* b, cudaStream_t s, cudaGraphConditionalHandle hb, int use) {
  int rc;
  const SegView sv = seg_view(b);
  KrySmall S{b->m};
  if ((rc = emit_residual(b, s, b->d_u, b->d_res, b->d_skip_newt))) return rc;
  kb_norm2<<<b->nchunk, KRY_T, 0, s>>>(sv, b->d_res, (int)(S.sc() + 5), b->d_skip_newt);
  kb_newton_check<<<1, 256, 0, s>>>(b->d_ctl, sv, b->d_st, b->d_skip_newt, b->d_skip_gm, b->d_bt, hb, use);
  kb_newton_step_control<<<b->nchunk, 256, 0, s>>>(sv, b->d_x, b->d_u, b->d_ubase, b->d_skip_newt, b->d_bt);
  kb_prep_linear<<<b->nchunk, 256, 0, s>>>(sv, b->d_res, b->d_r, b->d_x, b->d_skip_gm);
  for (int i = 0; i < 4; ++i) count_launch();
  BK(cudaGetLastError());
  return LDG_OK;
}

// Newton body, part 2: u -= delta, loop decision.
int emit_newton_tail(ldg_batch* b, cudaStream_t s, cudaGraphConditionalHandle ha, int use) {
  const SegView sv = seg_view(b);
  kb_newton_update<<<b->nchunk, 256, 0, s>>>(sv, b->d_x, b->d_u, b->d_skip_newt, b->d_bt);
  kb_newton_end<<<1, 256, 0, s>>>(b->d_ctl, b->d_skip_newt, b->nseg, ha, use);
  count_launch();
  count_launch();
  BK(cudaGetLastError());
  return LDG_OK;
}

// Restart body, part 1: cycle start.
int emit_cycle_head(ldg_batch* b, cudaStream_t s, cudaGraphConditionalHandle hc, int use) {
  const SegView sv = seg_view(b);
  kb_cycle_init<<<1, 256, 0, s>>>(b->d_ctl, sv, b->d_skip_gm, b->d_skip_arn, hc, use);
  if (b->ff)
    kb_cycle_start_ff<<<b->nchunk, 256, 0, s>>>(sv, b->d_r, (float2*)b->d_V, b->d_vcur, b->d_skip_gm);
  else
    kb_cycle_start<<<b->nchunk, 256, 0, s>>>(sv, b->d_r, b->d_V, b->d_vcur, b->d_skip_gm);
  count_launch();
  count_launch();
  BK(cudaGetLastError());
  return LDG_OK;
}

// Restart body, part 2: least-squares solution, x update, true residual, decision.
int emit_cycle_tail(ldg_batch* b, cudaStream_t s, cudaGraphConditionalHandle hb, int use) {
  int rc;
  const SegView sv = seg_view(b);
  kb_backsolve<<<(b->nseg + 127) / 128, 128, 0, s>>>(sv, b->d_skip_gm);
  if (b->ff && !b->pc)
    kb_solution_update_ff<<<b->nchunk, 256, 0, s>>>(sv, (const float2*)b->d_V, b->ntot, b->d_x, b->d_skip_gm);
  else
    kb_solution_update<<<b->nchunk, 256, 0, s>>>(sv, b->pc ? b->d_Z : b->d_V, b->ntot, b->d_x, b->d_skip_gm);
  count_launch();
  count_launch();
  BK(cudaGetLastError());
  if ((rc = emit_jv(b, s, b->d_u, b->d_x, b->d_w, b->opt.krylov_precision, b->d_skip_gm, true))) return rc;
  kb_sub_norm<<<b->nchunk, KRY_T, 0, s>>>(sv, b->d_res, b->d_w, b->d_r, b->d_skip_gm);
  kb_cycle_end<<<1, 256, 0, s>>>(b->d_ctl, sv, b->d_st, b->d_skip_gm, b->d_skip_newt, hb, use);
  count_launch();
  count_launch();
  BK(cudaGetLastError());
  return LDG_OK;
}

// Arnoldi body: z = M^{-1} v_j, w = J z, two Gram-Schmidt passes, Givens, v_{j+1}.
int emit_arnoldi(ldg_batch* b, cudaStream_t s, cudaGraphConditionalHandle hc, int use) {
  int rc;
  const SegView sv = seg_view(b);
  const double* dir = b->d_vcur;
  if (b->pc) {
    if ((rc = emit_pc(b, s, b->d_vcur, b->d_zcur, b->d_skip_arn))) return rc;
    dir = b->d_zcur;
  }
  if ((rc = emit_jv(b, s, b->d_u, dir, b->d_w, b->opt.krylov_precision, b->d_skip_arn, true))) return rc;
  // classical Gram-Schmidt, two passes: h1 = V^T w, w -= V h1, h2 = V^T w, w -= V h2,
  // then v_{j+1} = w / ||w|| and the Givens column
  double* part1 = b->d_part;
  double* part2 = b->d_part + (size_t)b->nchunk * KB_LDP;
  double* part3 = b->d_part + (size_t)2 * b->nchunk * KB_LDP;
  KrySmall S{b->m};
  if (b->ff) {
    // the same two passes on the pair basis (emulated FP64 on the FP32 pipes)
    float2* V2 = (float2*)b->d_V;
    float2 *q1 = (float2*)part1, *q2 = (float2*)part2, *q3 = (float2*)part3;
    kb_mdot_ff<<<b->nchunk, KRY_T, 0, s>>>(sv, b->d_ctl, V2, b->ntot, b->d_w, b->d_wf, q1,
                                           b->pc ? b->d_zcur : nullptr, b->d_Z, b->d_skip_arn);
    kb_update_ff<<<b->nchunk, KRY_T, 0, s>>>(sv, b->d_ctl, V2, b->ntot, q1, (int)S.h1(), b->d_wf, nullptr,
                                             b->d_skip_arn);
    kb_mdot_ff<<<b->nchunk, KRY_T, 0, s>>>(sv, b->d_ctl, V2, b->ntot, nullptr, b->d_wf, q2, nullptr, nullptr,
                                           b->d_skip_arn);
    kb_update_ff<<<b->nchunk, KRY_T, 0, s>>>(sv, b->d_ctl, V2, b->ntot, q2, (int)S.h2(), b->d_wf, q3, b->d_skip_arn);
    kb_scale_ff<<<b->nseg + b->nchunk, KRY_T, 0, s>>>(sv, b->d_ctl, b->d_wf, q3, V2, b->ntot, b->d_vcur,
                                                      b->d_skip_arn);
    kb_arnoldi_end<<<1, 256, 0, s>>>(b->d_ctl, b->d_skip_arn, b->nseg, hc, use);
    for (int i = 0; i < 6; ++i) count_launch();
    BK(cudaGetLastError());
    return LDG_OK;
  }
  kb_mdot<<<b->nchunk, KRY_T, 0, s>>>(sv, b->d_ctl, b->d_V, b->ntot, b->d_w, part1, b->pc ? b->d_zcur : nullptr,
                                      b->d_Z, b->d_skip_arn);
  kb_update<<<b->nchunk, KRY_T, 0, s>>>(sv, b->d_ctl, b->d_V, b->ntot, part1, (int)S.h1(), b->d_w, nullptr, nullptr,
                                        b->d_skip_arn);
  kb_mdot<<<b->nchunk, KRY_T, 0, s>>>(sv, b->d_ctl, b->d_V, b->ntot, b->d_w, part2, nullptr, nullptr, b->d_skip_arn);
  kb_update<<<b->nchunk, KRY_T, 0, s>>>(sv, b->d_ctl, b->d_V, b->ntot, part2, (int)S.h2(), b->d_w, part3, nullptr,
                                        b->d_skip_arn);
  kb_scale<<<b->nseg + b->nchunk, KRY_T, 0, s>>>(sv, b->d_ctl, b->d_w, part3, b->d_V, b->ntot, b->d_vcur,
                                                 b->d_skip_arn);
  kb_arnoldi_end<<<1, 256, 0, s>>>(b->d_ctl, b->d_skip_arn, b->nseg, hc, use);
  for (int i = 0; i < 6; ++i) count_launch();
  BK(cudaGetLastError());
  return LDG_OK;
}

int emit_init(ldg_batch* b, cudaStream_t s) {
  kb_init<<<1, 256, 0, s>>>(b->d_ctl, b->d_st, b->nseg, b->d_skip_newt, b->d_skip_gm, b->d_skip_arn);
  count_launch();
  BK(cudaGetLastError());
  return LDG_OK;
}

// A WHILE node created (with its handle) in graph g before the kernels that precede
// it are captured, so those kernels can already set its condition.
struct WhileNode {
  cudaGraphConditionalHandle h = 0;
  cudaGraphNode_t node = nullptr;
  cudaGraph_t body = nullptr;
};

int make_while(ldg_batch* b, cudaGraph_t g, unsigned dflt, unsigned flags, WhileNode* w) {
  BK(cudaGraphConditionalHandleCreate(&w->h, g, dflt, flags));
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = w->h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  BK(cudaGraphAddNode(&w->node, g, nullptr, nullptr, 0, &p));
  w->body = p.conditional.phGraph_out[0];
  return LDG_OK;
}

// During the capture of s: the node runs after everything captured so far, and the
// capture continues after the node.
int join_while(ldg_batch* b, cudaStream_t s, const WhileNode& w) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  BK(cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd));
  if (st != cudaStreamCaptureStatusActive) return bfail(b, LDG_ERR_CUDA, "join_while: stream not capturing");
  std::vector<cudaGraphNode_t> from(deps, deps + nd);
  for (cudaGraphNode_t f : from) BK(cudaGraphAddDependencies(g, &f, &w.node, nullptr, 1));
  cudaGraphNode_t n = w.node;
  BK(cudaStreamUpdateCaptureDependencies(s, &n, nullptr, 1, cudaStreamSetCaptureDependencies));
  return LDG_OK;
}

// Captures the whole solve into one graph:
//   init; WHILE(newton) { head; WHILE(restart) { cycle head; WHILE(arnoldi) { step }; cycle tail }; tail }
// Each loop's condition is set by the control kernel that ends its body (and, on
// entry, by the kernel just before the node); the Newton loop starts with condition 1.
int build_graph(ldg_batch* b) {
  int rc = LDG_OK;
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  cudaStream_t s = b->cap;
  BK(cudaGraphCreate(&b->graph, 0));
  WhileNode wa, wb, wc;
  auto capture = [&](cudaGraph_t g, auto&& fn) -> int {
    BK(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    int r = fn();
    cudaGraph_t out = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &out);
    if (r) return r;
    if (e != cudaSuccess) return bfail(b, LDG_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    if (out && out != g) return bfail(b, LDG_ERR_CUDA, "graph capture ended in an unexpected graph");
    return LDG_OK;
  };
  if ((rc = make_while(b, b->graph, 1u, cudaGraphCondAssignDefault, &wa))) return rc;
  if ((rc = make_while(b, wa.body, 0u, 0u, &wb))) return rc;
  if ((rc = make_while(b, wb.body, 0u, 0u, &wc))) return rc;
  long long c0 = launch_counter().load();
  rc = capture(b->graph, [&]() -> int {
    int r = emit_init(b, s);
    if (!r) r = join_while(b, s, wa);
    return r;
  });
  if (rc) return rc;
  b->k_pre = launch_counter().load() - c0;
  c0 = launch_counter().load();
  rc = capture(wa.body, [&]() -> int {
    int r = emit_newton_head(b, s, wb.h, 1);
    if (!r) r = join_while(b, s, wb);
    if (!r) r = emit_newton_tail(b, s, wa.h, 1);
    return r;
  });
  if (rc) return rc;
  b->k_a = launch_counter().load() - c0;
  c0 = launch_counter().load();
  rc = capture(wb.body, [&]() -> int {
    int r = emit_cycle_head(b, s, wc.h, 1);
    if (!r) r = join_while(b, s, wc);
    if (!r) r = emit_cycle_tail(b, s, wb.h, 1);
    return r;
  });
  if (rc) return rc;
  b->k_b = launch_counter().load() - c0;
  c0 = launch_counter().load();
  rc = capture(wc.body, [&]() -> int { return emit_arnoldi(b, s, wc.h, 1); });
  if (rc) return rc;
  b->k_c = launch_counter().load() - c0;
  // the captured kernels are counted when they execute, not here
  launch_counter() -= b->k_pre + b->k_a + b->k_b + b->k_c;
  BK(cudaGraphInstantiate(&b->exec, b->graph, 0));
  return LDG_OK;
}

// The same loops driven from the host (each decision read back from the device).
int run_eager(ldg_batch* b, cudaStream_t s) {
  int rc;
  BatchCtl ctl;
  auto read_ctl = [&]() -> int {
    BK(cudaMemcpyAsync(&ctl, b->d_ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
    BK(cudaStreamSynchronize(s));
    return LDG_OK;
  };
  if ((rc = emit_init(b, s))) return rc;
  const int cap_a = b->opt.max_newton + 2;
  for (int ia = 0; ia < cap_a; ++ia) {
    if ((rc = emit_newton_head(b, s, 0, 0))) return rc;
    if ((rc = read_ctl())) return rc;
    for (int ib = 0; ctl.cond_b && ib < b->opt.max_restarts; ++ib) {
      if ((rc = emit_cycle_head(b, s, 0, 0))) return rc;
      if ((rc = read_ctl())) return rc;
      for (int ic = 0; ctl.cond_c && ic < b->m; ++ic) {
        if ((rc = emit_arnoldi(b, s, 0, 0))) return rc;
        if ((rc = read_ctl())) return rc;
      }
      if ((rc = emit_cycle_tail(b, s, 0, 0))) return rc;
      if ((rc = read_ctl())) return rc;
    }
    if ((rc = emit_newton_tail(b, s, 0, 0))) return rc;
    if ((rc = read_ctl())) return rc;
    if (!ctl.cond_a) break;
  }
  return LDG_OK;
}

void free_batch(ldg_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (BGroup& g : b->groups) {
    if (g.ctx && !b->borrowed) ldg_destroy(g.ctx);
    cudaFree(g.d_inst);
  }
  for (void* p : {(void*)b->d_mtab, (void*)b->d_chunk_seg, (void*)b->d_seg_c0, (void*)b->d_seg_nc,
                  (void*)b->d_chunk_lo, (void*)b->d_chunk_hi, (void*)b->d_part, (void*)b->d_tick, (void*)b->d_small,
                  (void*)b->d_sflags, (void*)b->d_st, (void*)b->d_ctl, (void*)b->d_skip_newt, (void*)b->d_skip_gm,
                  (void*)b->d_skip_arn, (void*)b->d_u, (void*)b->d_res, (void*)b->d_r, (void*)b->d_x, (void*)b->d_w,
                  (void*)b->d_vcur, (void*)b->d_zcur, (void*)b->d_V, (void*)b->d_Z, (void*)b->d_bt,
                  (void*)b->d_ubase, (void*)b->d_wf})
    cudaFree(p);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

template <class T> int upload(ldg_batch* b, T** dst, const std::vector<T>& src) {
  BK(cudaMalloc(dst, std::max<size_t>(1, src.size()) * sizeof(T)));
  if (!src.empty()) BK(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return LDG_OK;
}

int finish_build(ldg_batch* b, const std::vector<int64_t>& seg_off, const std::vector<int64_t>& seg_n);

int build_batch(ldg_batch* b, int n_inst, const ldg_mesh_desc* meshes, const int* p, const ldg_model_desc* models,
                const ldg_options* opts) {
  int rc;
  ldg_options o{};
  if (opts) o = *opts;
  if (o.gmres_m <= 0) o.gmres_m = 30;
  if (o.gmres_m > 30) o.gmres_m = 30;
  if (o.max_restarts <= 0) o.max_restarts = 50;
  if (o.max_newton <= 0) o.max_newton = 20;
  if (o.newton_rtol <= 0) o.newton_rtol = 1e-8;
  if (o.gmres_rtol <= 0) o.gmres_rtol = 1e-3;
  if (o.krylov_precision == LDG_TC_BF16X3 || o.krylov_precision == LDG_TC_BF16)
    return bfail(b, LDG_ERR_UNSUPPORTED, "the batched solver takes LDG_FP64, LDG_FP32 or LDG_F32X2");
  if (o.krylov_precision != LDG_FP32 && o.krylov_precision != LDG_F32X2) o.krylov_precision = LDG_FP64;
  if (o.precond != LDG_PC_BJACOBI) o.precond = LDG_PC_NONE;
  if (o.newton_forcing != LDG_FORCING_LAST) o.newton_forcing = LDG_FORCING_FIXED;
  if (o.pc_reuse < 1) o.pc_reuse = 1;
  if (o.krylov_basis != LDG_BASIS_F32X2) o.krylov_basis = LDG_BASIS_FP64;
  b->opt = o;
  b->m = o.gmres_m;
  b->pc = o.precond == LDG_PC_BJACOBI;
  b->n_inst = n_inst;
  // groups keyed by (element, p, quadrature, model, curved-map degree), instances in
  // caller order within a group
  std::map<std::tuple<int, int, int, int, int>, std::vector<int>> keyed;
  for (int i = 0; i < n_inst; ++i) {
    const ldg_mesh_desc& M = meshes[i];
    if (!M.xyz || !M.vid || M.n_elem <= 0 || M.elem_type < 0 || M.elem_type > 3)
      return bfail(b, LDG_ERR_ARG, "instance " + std::to_string(i) + ": bad mesh");
    if (models[i].model < 0 || models[i].model > 3)
      return bfail(b, LDG_ERR_ARG, "instance " + std::to_string(i) + ": bad model");
    const int nq = opts && opts->nq1 > 0 ? opts->nq1 : default_nq(M.elem_type, models[i].model, p[i]);
    if (M.geom_order > 0 && !M.xgeo)
      return bfail(b, LDG_ERR_ARG, "instance " + std::to_string(i) + ": curved mesh without map points");
    keyed[std::make_tuple(M.elem_type, p[i], nq, models[i].model, std::max(0, M.geom_order))].push_back(i);
  }
  b->user_off.assign(n_inst, 0);
  b->user_n.assign(n_inst, 0);
  std::vector<ModelParams> mtab;
  std::vector<int64_t> seg_off, seg_n;
  int64_t off = 0;
  for (auto& kv : keyed) {
    BGroup g;
    int pg = 0;
    std::tie(g.etype, g.p, g.nq, g.model, pg) = kv.first;
    const std::vector<int>& ids = kv.second;
    const int nv = verts_per_elem(g.etype), dim = (g.etype == LDG_HEX || g.etype == LDG_TET) ? 3 : 2;
    int64_t E = 0;
    for (int i : ids) E += meshes[i].n_elem;
    if (E > (int64_t)0x7fffffff) return bfail(b, LDG_ERR_ARG, "group too large");
    std::vector<double> xyz;
    std::vector<int64_t> vid;
    std::vector<int> inst;
    std::vector<double> xgeo;            // curved groups: map points, concatenated
    std::vector<unsigned char> bc;       // wall marks (0 where an instance gives none)
    const int nfc = g.etype == LDG_TRI ? 3 : (g.etype == LDG_TET ? 4 : 2 * dim);
    bool any_bc = false;
    for (int i : ids) any_bc |= meshes[i].bc != nullptr;
    xyz.reserve((size_t)E * nv * dim);
    vid.reserve((size_t)E * nv);
    inst.reserve(E);
    int64_t vshift = 0;
    for (int i : ids) {
      const ldg_mesh_desc& M = meshes[i];
      const int seg = (int)b->seg_user.size();
      int64_t vmax = -1;
      xyz.insert(xyz.end(), M.xyz, M.xyz + (size_t)M.n_elem * nv * dim);
      for (int64_t k = 0; k < M.n_elem * nv; ++k) {
        if (M.vid[k] < 0) return bfail(b, LDG_ERR_ARG, "instance " + std::to_string(i) + ": negative vertex id");
        vid.push_back(M.vid[k] + vshift);
        vmax = std::max(vmax, M.vid[k]);
      }
      vshift += vmax + 1;
      inst.insert(inst.end(), (size_t)M.n_elem, seg);
      if (pg > 0) {
        // map points per element: (pg+1)^2 on quadrilaterals, (pg+1)(pg+2)/2 on triangles
        const size_t np = g.etype == LDG_TRI ? (size_t)(pg + 1) * (pg + 2) / 2 : (size_t)(pg + 1) * (pg + 1);
        xgeo.insert(xgeo.end(), M.xgeo, M.xgeo + (size_t)M.n_elem * np * 2);
      }
      if (any_bc) {
        if (M.bc) bc.insert(bc.end(), M.bc, M.bc + (size_t)M.n_elem * nfc);
        else bc.insert(bc.end(), (size_t)M.n_elem * nfc, (unsigned char)0);
      }
      b->seg_user.push_back(i);
      mtab.push_back(make_params(&models[i]));
    }
    ldg_mesh_desc um{g.etype, E, xyz.data(), vid.data(), pg, pg > 0 ? xgeo.data() : nullptr,
                     any_bc ? bc.data() : nullptr};
    ldg_model_desc gm = models[ids[0]];
    ldg_options go = o;
    go.nq1 = g.nq;
    go.precond = o.precond;
    rc = create_ctx(&g.ctx, &um, g.p, &gm, &go, b->stream, true);
    if (rc) {
      std::string msg = g.ctx ? g.ctx->err : "group context";
      if (g.ctx) ldg_destroy(g.ctx);
      return bfail(b, rc, msg);
    }
    g.off = off;
    g.ndof = g.ctx->ndof;
    const int64_t nloc = g.ctx->nloc;
    int64_t eo = 0;
    for (int i : ids) {
      b->user_off[i] = off + eo * nloc;
      b->user_n[i] = meshes[i].n_elem * nloc;
      seg_off.push_back(b->user_off[i]);
      seg_n.push_back(b->user_n[i]);
      eo += meshes[i].n_elem;
    }
    off += g.ndof;
    if ((rc = upload(b, &g.d_inst, inst))) { ldg_destroy(g.ctx); return rc; }
    g.ctx->ext_inst = g.d_inst;
    b->groups.push_back(g);
  }
  b->ntot = off;
  b->nseg = (int)b->seg_user.size();
  if ((rc = upload(b, &b->d_mtab, mtab))) return rc;
  for (BGroup& g : b->groups) g.ctx->ext_mtab = b->d_mtab;
  return finish_build(b, seg_off, seg_n);
}

// Chunk tables, per-instance state and the Krylov work space of a batch whose groups
// and instance segments are set.
int finish_build(ldg_batch* b, const std::vector<int64_t>& seg_off, const std::vector<int64_t>& seg_n) {
  const ldg_options& o = b->opt;
  int rc;
  // chunk tables
  // chunk size: a power of two in [512, KB_CHUNK] giving about two chunks per SM, so
  // small batches still spread over the whole GPU
  int64_t ch = 512;
  while (ch < KB_CHUNK && ch * 148 * 2 < b->ntot) ch *= 2;
  std::vector<int> cseg, c0(b->nseg), nc(b->nseg);
  std::vector<int64_t> clo, chi;
  for (int s = 0; s < b->nseg; ++s) {
    c0[s] = (int)cseg.size();
    for (int64_t lo = seg_off[s]; lo < seg_off[s] + seg_n[s]; lo += ch) {
      cseg.push_back(s);
      clo.push_back(lo);
      chi.push_back(std::min(lo + ch, seg_off[s] + seg_n[s]));
    }
    nc[s] = (int)cseg.size() - c0[s];
  }
  b->nchunk = (int)cseg.size();
  if ((rc = upload(b, &b->d_chunk_seg, cseg)) || (rc = upload(b, &b->d_chunk_lo, clo)) ||
      (rc = upload(b, &b->d_chunk_hi, chi)) || (rc = upload(b, &b->d_seg_c0, c0)) || (rc = upload(b, &b->d_seg_nc, nc)))
    return rc;
  const size_t ks = KrySmall{b->m}.total();
  BK(cudaMalloc(&b->d_part, (size_t)3 * b->nchunk * KB_LDP * sizeof(double)));
  BK(cudaMalloc(&b->d_bt, (size_t)b->nseg * sizeof(int)));
  BK(cudaMemset(b->d_bt, 0, (size_t)b->nseg * sizeof(int)));
  BK(cudaMalloc(&b->d_ubase, (size_t)b->ntot * sizeof(double)));
  BK(cudaMalloc(&b->d_tick, b->nseg * sizeof(unsigned int)));
  BK(cudaMemset(b->d_tick, 0, b->nseg * sizeof(unsigned int)));
  BK(cudaMalloc(&b->d_small, (size_t)b->nseg * ks * sizeof(double)));
  BK(cudaMemset(b->d_small, 0, (size_t)b->nseg * ks * sizeof(double)));
  BK(cudaMalloc(&b->d_sflags, (size_t)b->nseg * 4 * sizeof(int)));
  BK(cudaMemset(b->d_sflags, 0, (size_t)b->nseg * 4 * sizeof(int)));
  BK(cudaMalloc(&b->d_st, (size_t)b->nseg * sizeof(SegState)));
  BK(cudaMalloc(&b->d_ctl, sizeof(BatchCtl)));
  BatchCtl ctl;
  std::memset(&ctl, 0, sizeof(ctl));
  ctl.max_newton = o.max_newton; ctl.max_restarts = o.max_restarts; ctl.m = b->m;
  ctl.newton_rtol = o.newton_rtol; ctl.gmres_rtol = o.gmres_rtol; ctl.forcing = o.newton_forcing;
  BK(cudaMemcpy(b->d_ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice));
  for (int** q : {&b->d_skip_newt, &b->d_skip_gm, &b->d_skip_arn}) {
    BK(cudaMalloc(q, b->nseg * sizeof(int)));
    BK(cudaMemset(*q, 0, b->nseg * sizeof(int)));
  }
  const size_t nb = (size_t)b->ntot * sizeof(double);
  for (double** q : {&b->d_u, &b->d_res, &b->d_r, &b->d_x, &b->d_w, &b->d_vcur, &b->d_zcur}) {
    BK(cudaMalloc(q, nb));
    BK(cudaMemset(*q, 0, nb));
  }
  BK(cudaMalloc(&b->d_V, (size_t)(b->m + 1) * nb));   // FP64 vectors, or float pairs of the same size
  if (b->pc) BK(cudaMalloc(&b->d_Z, (size_t)b->m * nb));
  b->ff = o.krylov_basis == LDG_BASIS_F32X2;
  if (b->ff) BK(cudaMalloc(&b->d_wf, (size_t)b->ntot * sizeof(float2)));
  BK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  return LDG_OK;
}

}  // namespace

// ===================================================================== C ABI
extern "C" {

int ldg_batch_create(ldg_batch** out, int n_inst, const ldg_mesh_desc* meshes, const int* p,
                     const ldg_model_desc* models, const ldg_options* opts, void* cuda_stream) {
  if (!out) return LDG_ERR_ARG;
  *out = nullptr;
  if (n_inst <= 0 || !meshes || !p || !models) return LDG_ERR_ARG;
  ldg_batch* b = new ldg_batch();
  b->stream = (cudaStream_t)cuda_stream;
  const int rc = build_batch(b, n_inst, meshes, p, models, opts);
  *out = b;   // on error the caller reads ldg_batch_last_error, then destroys
  return rc;
}

int ldg_batch_destroy(ldg_batch* b) {
  if (b) free_batch(b);
  return LDG_OK;
}

int ldg_batch_sizes(const ldg_batch* b, int64_t* n_total, int64_t* offsets, int64_t* n_dof, int* n_groups) {
  if (!b || b->groups.empty()) return LDG_ERR_ARG;
  if (n_total) *n_total = b->ntot;
  for (int i = 0; i < b->n_inst; ++i) {
    if (offsets) offsets[i] = b->user_off[i];
    if (n_dof) n_dof[i] = b->user_n[i];
  }
  if (n_groups) *n_groups = (int)b->groups.size();
  return LDG_OK;
}

int ldg_batch_set_time(ldg_batch* b, int scheme, double t, double dt, const double* un, const double* unm1) {
  if (!b || b->groups.empty()) return LDG_ERR_ARG;
  if (scheme != LDG_STEADY && (!un || (scheme == LDG_BDF2 && !unm1))) return bfail(b, LDG_ERR_ARG, "missing history");
  bool changed = false;
  for (BGroup& g : b->groups) {
    g.ctx->stream = b->stream;
    const double a0_before = g.ctx->a0dt;
    const int rc = ldg_set_time(g.ctx, scheme, t, dt, un ? un + g.off : nullptr, unm1 ? unm1 + g.off : nullptr);
    if (rc) return gfail(b, g, rc);
    changed |= g.ctx->a0dt != a0_before;
  }
  // the captured kernels hold a0/dt by value; the time itself is read from device memory
  if (changed) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  }
  return LDG_OK;
}

int ldg_batch_residual(ldg_batch* b, const double* u, double* r) {
  if (!b || b->groups.empty() || !u || !r) return LDG_ERR_ARG;
  return emit_residual(b, b->stream, u, r, nullptr);
}

int ldg_batch_jvp(ldg_batch* b, int precision, const double* u, const double* v, double* jv) {
  if (!b || b->groups.empty() || !u || !v || !jv) return LDG_ERR_ARG;
  if (precision == LDG_TC_BF16X3 || precision == LDG_TC_BF16) return LDG_ERR_UNSUPPORTED;
  return emit_jv(b, b->stream, u, v, jv, precision == LDG_FP32 || precision == LDG_F32X2 ? precision : LDG_FP64,
                 nullptr, false);
}

int ldg_batch_autotune(ldg_batch* b, int force, int* tiles) {
  if (!b || b->groups.empty()) return LDG_ERR_ARG;
  for (size_t i = 0; i < b->groups.size(); ++i) {
    BGroup& g = b->groups[i];
    g.ctx->stream = b->stream;
    int t = 0;
    const int rc = autotune(g.ctx, force, &t, nullptr);
    if (rc) return gfail(b, g, rc);
    if (tiles) tiles[i] = t;
  }
  // the captured graph holds the previous kernels
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  return LDG_OK;
}

int ldg_batch_solve(ldg_batch* b, double* u_dev, int use_graph, ldg_solve_report* reps, double* elapsed_ms) {
  if (!b || b->groups.empty() || !u_dev) return LDG_ERR_ARG;
  int rc;
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = b->stream;
  BK(cudaMemcpyAsync(b->d_u, u_dev, (size_t)b->ntot * sizeof(double), cudaMemcpyDeviceToDevice, s));
  // block-Jacobi: built at this call's initial guess every pc_reuse calls, or when the
  // time-scheme coefficient changed since the blocks were built
  bool pc_built_now = false;
  if (b->pc) {
    const bool due = b->solves % b->opt.pc_reuse == 0;
    for (BGroup& g : b->groups) {
      g.ctx->stream = s;
      if (due || !g.pc_built || !g.ctx->pc_ready || g.pc_scheme != g.ctx->scheme || g.pc_a0dt != g.ctx->a0dt) {
        if ((rc = do_pc_setup(g.ctx, b->d_u + g.off))) return gfail(b, g, rc);
        g.pc_built = true;
        g.pc_scheme = g.ctx->scheme;
        g.pc_a0dt = g.ctx->a0dt;
        pc_built_now = true;
      }
    }
  }
  b->solves++;
  long long before = launch_counter();
  if (b->exec) {
    // the captured kernels hold the tile, the time scheme and a0/dt of every group
    bool stale = false;
    for (size_t i = 0; i < b->groups.size(); ++i) {
      const ldg_ctx* c = b->groups[i].ctx;
      stale |= c->ks != b->cap_ks[i] || c->scheme != b->cap_scheme[i] || c->a0dt != b->cap_a0dt[i] ||
               c->radd_on != (bool)b->cap_radd[i];
    }
    if (stale) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
      cudaGraphDestroy(b->graph);
      b->graph = nullptr;
    }
  }
  if (use_graph) {
    if (!b->exec) {
      // every kernel instance runs once outside the capture (function attributes are set then)
      BK(cudaStreamSynchronize(s));
      if ((rc = emit_residual(b, s, b->d_u, b->d_res, nullptr))) return rc;
      if ((rc = emit_jv(b, s, b->d_u, b->d_res, b->d_w, b->opt.krylov_precision, nullptr, true))) return rc;
      if (b->pc && (rc = emit_pc(b, s, b->d_res, b->d_w, nullptr))) return rc;
      BK(cudaStreamSynchronize(s));
      before = launch_counter();
      rc = build_graph(b);
      for (BGroup& g : b->groups) g.ctx->stream = s;
      if (rc) return rc;
      b->cap_ks.clear(); b->cap_scheme.clear(); b->cap_a0dt.clear(); b->cap_radd.clear();
      for (const BGroup& g : b->groups) {
        b->cap_ks.push_back(g.ctx->ks);
        b->cap_scheme.push_back(g.ctx->scheme);
        b->cap_a0dt.push_back(g.ctx->a0dt);
        b->cap_radd.push_back(g.ctx->radd_on ? 1 : 0);
      }
    }
    BK(cudaGraphLaunch(b->exec, s));
  } else {
    if ((rc = run_eager(b, s))) return rc;
  }
  BK(cudaMemcpyAsync(u_dev, b->d_u, (size_t)b->ntot * sizeof(double), cudaMemcpyDeviceToDevice, s));
  std::vector<SegState> st(b->nseg);
  BatchCtl ctl;
  BK(cudaMemcpyAsync(st.data(), b->d_st, st.size() * sizeof(SegState), cudaMemcpyDeviceToHost, s));
  BK(cudaMemcpyAsync(&ctl, b->d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost, s));
  BK(cudaStreamSynchronize(s));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (use_graph) {
    b->last_exec = b->k_pre + ctl.trips_a * b->k_a + ctl.trips_b * b->k_b + ctl.trips_c * b->k_c;
    launch_counter() += b->last_exec;
  } else {
    b->last_exec = launch_counter() - before;
  }
  if (elapsed_ms) *elapsed_ms = ms;
  int worst = LDG_OK;
  for (int sg = 0; sg < b->nseg; ++sg) {
    const SegState& q = st[sg];
    if (q.status < worst) worst = q.status;
    if (!reps) continue;
    ldg_solve_report& r = reps[b->seg_user[sg]];
    std::memset(&r, 0, sizeof(r));
    r.newton_iters = q.newton_iters;
    r.gmres_iters = q.gmres_iters;
    r.jv_calls = q.jv_calls;
    r.residual_calls = q.residual_calls;
    r.r0 = q.r0;
    r.rfinal = q.rn;
    r.lin_resid = q.lin_resid;
    r.elapsed_ms = ms;
    r.status = q.status;
    r.pc_setups = pc_built_now ? 1 : 0;
    r.newton_backtracks = q.backtracks;
  }
  if (worst != LDG_OK) return bfail(b, worst, "some instances did not converge (see the per-instance reports)");
  return LDG_OK;
}

int64_t ldg_batch_kernel_executions(const ldg_batch* b) { return b ? b->last_exec : 0; }

const char* ldg_batch_last_error(const ldg_batch* b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"

namespace ldg {
namespace impl {

int batch_wrap(ldg_ctx* ctx, ldg_batch** out) {
  *out = nullptr;
  ldg_batch* b = new ldg_batch();
  b->borrowed = true;
  b->stream = ctx->stream;
  b->opt = ctx->opt;
  b->m = ctx->opt.gmres_m;
  b->pc = ctx->opt.precond == LDG_PC_BJACOBI;
  b->n_inst = 1;
  BGroup g;
  g.ctx = ctx;
  g.off = 0;
  g.ndof = ctx->ndof;
  g.etype = ctx->etype; g.p = ctx->p; g.nq = ctx->nq; g.model = ctx->model;
  b->groups.push_back(g);
  b->seg_user = {0};
  b->user_off = {0};
  b->user_n = {ctx->ndof};
  b->ntot = ctx->ndof;
  b->nseg = 1;
  const int rc = finish_build(b, {0}, {ctx->ndof});
  if (rc) {
    ctx->err = b->err;
    free_batch(b);
    return rc;
  }
  *out = b;
  return LDG_OK;
}

int batch_solve_one(ldg_batch* b, double* u, ldg_solve_report* rep) {
  b->stream = b->groups[0].ctx->stream;
  ldg_solve_report r{};
  double ms = 0.0;
  // LDG_SOLVER_HOST_LOOPS=1: the same kernels driven by host loops instead of the
  // graph's WHILE nodes (profilers that do not follow conditional graph nodes)
  const char* host = getenv("LDG_SOLVER_HOST_LOOPS");
  const int rc = ldg_batch_solve(b, u, (host && host[0] == '1') ? 0 : 1, &r, &ms);
  if (rep) {
    *rep = r;
    rep->elapsed_ms = ms;
  }
  return rc;
}

void batch_free(ldg_batch* b) {
  if (b) free_batch(b);
}

const char* batch_error(const ldg_batch* b) { return b ? b->err.c_str() : "no solver"; }

}  // namespace impl
}  // namespace ldg
