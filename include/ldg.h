/* ldg.h — C-ABI of the B300 matrix-free LDG hot path.
 *
 * The library evaluates the local discontinuous Galerkin (LDG) discretisation of
 * the first-order system q + grad u = 0, m du/dt + div f(u, q) = s (Section 2.1,
 * Eq. 1a-1b), its exact Jacobian-vector product, and the matrix-free
 * Newton-GMRES solve built on them (Section 3.3), with hand-written CUDA kernels
 * for sm_103a.
 *
 * Conventions
 *  - Every function returns an ldg_status (0 = LDG_OK, < 0 = error); no C++
 *    exception crosses this boundary. On error, ldg_last_error(ctx) returns a
 *    message that stays valid until the next call on that context.
 *  - Vector arguments named *_dev are DEVICE pointers owned by the caller, at
 *    least n_dof doubles (q: n_dof * dim), 8-byte aligned. Work is queued on
 *    the context's CUDA stream; results are complete when that stream is.
 *    Functions ending in _host take HOST pointers and return after the copy
 *    back to host memory has finished.
 *  - State layout is element-major: u[e][c][i] for element e, component c and
 *    local node i (n_pe nodes); q[e][c][d][i] adds the space direction d.
 *  - Host arrays passed to ldg_create are copied; the caller keeps ownership.
 *  - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef LDG_H
#define LDG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ldg_ctx ldg_ctx;

/* element shapes: triangles and tetrahedra (equispaced Lagrange nodes, collapsed
 * Gauss rules), quadrilaterals and hexahedra (tensor Gauss-Lobatto-Legendre nodes);
 * affine elements, and curved quadrilaterals and triangles (geom_order > 0 below). Tetrahedra
 * (Section 4.1's Poisson study) carry the diffusion models, p = 1..3. */
enum { LDG_TRI = 0, LDG_QUAD = 1, LDG_HEX = 2, LDG_TET = 3 };

/* models of Table 1 (Section 2.1): Poisson and convection-diffusion are diffusion
 * models (with q, Eq. 1a); 2-D Euler is a convection model (no q); 2-D compressible
 * Navier-Stokes is nonlinear with q (its viscous flux takes grad u = -q) */
enum { LDG_POISSON = 0, LDG_CONVDIFF = 1, LDG_EULER = 2, LDG_NS = 3 };

/* analytic data: Dirichlet/far-field boundary values, source terms and initial states */
enum {
  LDG_CASE_ZERO = 0,    /* u = 0, s = 0 */
  LDG_CASE_SINSIN = 1,  /* u = prod_d sin(pi x_d) */
  LDG_CASE_EXPSIN = 2,  /* u = exp(sum_d x_d) sin(pi prod_d x_d) */
  LDG_CASE_POLY2 = 3,   /* a fixed quadratic polynomial (patch test) */
  LDG_CASE_LINEAR = 4,  /* a fixed linear polynomial (patch test) */
  LDG_CASE_VORTEX = 5,  /* isentropic vortex, strength 5, centre (5,5), velocity (1,1), period 10 */
  LDG_CASE_CONST = 6,   /* uniform Euler free stream rho = 1, v = (1,1), p = 1 */
  LDG_CASE_ROTATION = 7, /* rigid rotation v = (-y, x)/2, rho = 1 + x/10 + y/20, internal energy 2 */
  LDG_CASE_CYLINDER = 8, /* cylinder free stream rho = 1, v = (1, 0), Mach 0.2 (p = 1 / (gamma 0.04)) */
  LDG_CASE_REST = 9,     /* gas at rest rho = 1, v = 0, p = 1 */
  LDG_CASE_CYLINDER_START = 10 /* cylinder start: the Mach 0.2 free stream with velocity (tanh((r - 0.5)/0.1), 0) */
};

typedef enum {
  LDG_OK = 0,
  LDG_ERR_ARG = -1,          /* invalid argument (null pointer, bad size or enum) */
  LDG_ERR_CUDA = -2,         /* a CUDA call failed; the message names it */
  LDG_ERR_UNSUPPORTED = -3,  /* no compiled kernel for this (element, p, quadrature, model) */
  LDG_ERR_NONFINITE = -4,    /* NaN/Inf met in a residual or Krylov quantity */
  LDG_ERR_MAXIT = -5,        /* iteration limit reached before the tolerance */
  LDG_ERR_MESH = -6          /* mesh rejected: non-affine without a curved map, inverted or non-conforming */
} ldg_status;

enum { LDG_STEADY = 0, LDG_BDF1 = 1, LDG_BDF2 = 2 };

/* Mesh (Section 3.2): per-element vertex coordinates and topological vertex ids.
 * xyz [n_elem][nv][dim] (host), vid [n_elem][nv] (host). Quadrilaterals and
 * hexahedra list vertices in lexicographic order (x fastest), triangles
 * counter-clockwise, tetrahedra with their three edges from vertex 0 right-handed.
 * Faces whose sorted vertex ids match are neighbours; a periodic mesh shares ids
 * across the period while each element keeps its own
 * (unwrapped) coordinates. Faces without a partner are boundary faces.
 *
 * Curved quadrilaterals (geom_order = pg > 0): element K's map is the degree-pg
 * Lagrange interpolant of the points xgeo [n_elem][(pg+1)^2][2] (host) placed at
 * the equispaced reference points (-1 + 2a/pg, -1 + 2b/pg), a fastest. Curved
 * triangles: the points xgeo [n_elem][(pg+1)(pg+2)/2][2] at the lattice points
 * (-1 + 2a/pg, -1 + 2b/pg), a + b <= pg, numbered b outer, a inner (the element's own
 * node order at degree pg). Poisson and convection-diffusion only, p = 1..4 with
 * p + 2 points (nq1) per direction. Either way the corner points must equal xyz, and
 * neighbouring maps must agree along shared edges
 * (checked at the face quadrature points: LDG_ERR_MESH otherwise). The geometry
 * is sampled at the quadrature points once, at creation (metrics, normals and
 * the element mass matrices, whose inverses the q-stage applies). geom_order = 0
 * (xgeo null): affine elements.
 * bc [n_elem][n_faces] (host, optional): 1 marks a boundary face as a no-slip
 * adiabatic wall for Euler / Navier-Stokes (trace (rho, 0, 0, rho E) from inside,
 * pressure flux, viscous momentum flux and penalty); other boundary faces take the
 * case's data (Dirichlet or far field). Faces are numbered 2 * axis + side. */
typedef struct {
  int elem_type;
  int64_t n_elem;
  const double* xyz;
  const int64_t* vid;
  int geom_order;
  const double* xgeo;
  const unsigned char* bc;
} ldg_mesh_desc;

/* Model and parameters mu (Section 2.1):
 *   Poisson:   mu = {kappa, tau}
 *   ConvDiff:  mu = {kappa, tau, beta_x, beta_y[, beta_z]}
 *   Euler:     mu = {gamma}
 *   NS:        mu = {gamma, Re, Pr[, tau]}: viscosity 1/Re, heat conductivity
 *              gamma / (Re Pr) on the internal energy, jump penalty tau
 *              (default 1/Re); defaults 1.4, 100, 0.72; quadrilaterals only  */
typedef struct {
  int model;
  int case_id;
  int n_mu;
  const double* mu;
} ldg_model_desc;

/* Solver options (Section 3.3). nq1 = Gauss points per direction (0 = default:
 * p + 1 for linear models on quadrilaterals/hexahedra, p + 2 for triangles, Euler and
 * Navier-Stokes). */
typedef struct {
  int nq1;
  int gmres_m;          /* Krylov dimension per restart cycle (default 30) */
  int max_restarts;     /* restart cycles per linear solve (default 50) */
  int max_newton;       /* Newton iterations (default 20) */
  double newton_rtol;   /* stop when ||R(u_k)|| <= newton_rtol ||R(u_0)|| (default 1e-8) */
  double gmres_rtol;    /* linear solve: ||b - J x|| <= gmres_rtol ||b|| (default 1e-3) */
  int krylov_precision; /* LDG_FP64 (default), LDG_FP32, LDG_F32X2, LDG_TC_BF16X3 or LDG_TC_BF16:
                           arithmetic of the J.v inside GMRES, and of the preconditioner for
                           LDG_FP32 and the tensor-core forms (FP32 blocks; LDG_F32X2 builds FP64
                           blocks). Newton residuals, Arnoldi, Givens and all vectors stay FP64,
                           so the outer iteration refines a low-precision J.v to the FP64
                           tolerance. LDG_F32X2 and the tensor-core forms are accepted where their
                           kernels exist (see the precision constants below); ldg_create returns
                           LDG_ERR_ARG elsewhere. */
  int precond;          /* LDG_PC_NONE (default), LDG_PC_BJACOBI, LDG_PC_MLP, LDG_PC_MLP_BJ or
                           LDG_PC_RB_BJ (flexible right preconditioning; a linear solve with a
                           learned one that misses its tolerance within two restart cycles is
                           redone with block-Jacobi; see the learned-preconditioner and the
                           reduced-basis sections below) */
  int pc_refresh;       /* rebuild the preconditioner every pc_refresh Newton iterations
                           (0 = once per ldg_newton_gmres call, at the initial guess) */
  int newton_forcing;   /* linear tolerance eta_k of Newton step k (inexact Newton):
                           LDG_FORCING_FIXED (default): eta_k = gmres_rtol;
                           LDG_FORCING_LAST: eta_k = max(gmres_rtol,
                           1/2 newton_rtol ||R(u_0)|| / ||R(u_k)||), so that no step, in
                           practice the last one, is solved further than the Newton
                           tolerance needs */
  int pc_reuse;         /* graph-driven solves (ldg_newton_gmres without the learned
                           preconditioner, ldg_batch_solve): the block-Jacobi blocks are built
                           at the initial guess of every pc_reuse-th solve call and reused by
                           the calls in between (a preconditioner lagged over time steps);
                           a call whose time-scheme coefficient a0/dt differs from the one
                           the blocks were built with rebuilds them. 0 or 1 (default): every
                           call */
  int krylov_basis;     /* graph-driven solves: storage and arithmetic of the Gram-Schmidt
                           sweeps. LDG_BASIS_FP64 (default): FP64 basis and FP64 FMAs.
                           LDG_BASIS_F32X2: the basis and the vector being orthogonalised as
                           (hi, lo) float pairs, about 48 significand bits (emulated FP64),
                           with error-free products and compensated sums on the FP32 pipes;
                           Hessenberg, Givens, Newton residual and solution stay FP64. The
                           host-driven solves (learned preconditioner, ldg_gmres) always use
                           FP64. */
  int jv_form;          /* linear models on affine quadrilaterals / hexahedra with p + 1 Gauss
                           points: LDG_JV_AUTO (default) takes the nodal J.v kernels (the same
                           operator in exact nodal form, one thread per node, two launches);
                           LDG_JV_STAGE keeps the quadrature-point stage kernels of every
                           other case. Results agree to rounding. */
  int rb_size;          /* LDG_PC_RB_BJ: columns of the reduced basis (default 8, at most 32) */
} ldg_options;

/* Arithmetic of a J.v. LDG_FP64: FP64. LDG_FP32: every operation in FP32 (inputs and
 * output FP64 in memory). LDG_F32X2: every operation on (hi, lo) float pairs carrying
 * about 48 significand bits (Dekker's double-length arithmetic with error-free sums and
 * products on the FP32 pipes: emulated FP64, accurate to a few 1e-14 relative where
 * FP64 gives a few 1e-15); inputs and output FP64 in memory. LDG_F32X2 exists where the
 * nodal J.v kernels serve: the linear models (Poisson, convection-diffusion) on affine
 * quadrilaterals and hexahedra with p + 1 Gauss points per direction, and on triangles
 * and tetrahedra with at least p + 2. */
/* LDG_TC_BF16X3 and LDG_TC_BF16 put the interpolation, integration, lift and mass
 * contractions of the residual of Eq. 1b on the tensor cores (tcgen05, FP32 accumulation
 * in tensor memory), written as dense GEMMs over all nodes and points of an element with
 * the elements' (element, component) pairs as rows; the pointwise Euler and Lax-Friedrichs
 * fluxes with their tangents are FP32 dual numbers on the CUDA cores. LDG_TC_BF16X3 splits
 * every operand into BF16 hi and lo parts and sums three products (about 1e-5 relative),
 * LDG_TC_BF16 keeps one BF16 product (about 1e-2). Inputs and output FP64 in memory. They
 * exist for the Euler model on affine quadrilaterals, p = 1..4, with p + 2 Gauss points
 * per direction (the vortex and cylinder cases; the wall and far-field faces included).
 * A tensor-core wait that runs out (about a second) leaves the affected outputs NaN. */
enum { LDG_FP64 = 0, LDG_FP32 = 1, LDG_F32X2 = 2, LDG_TC_BF16X3 = 3, LDG_TC_BF16 = 4 };
enum { LDG_PC_NONE = 0, LDG_PC_BJACOBI = 1, LDG_PC_MLP = 2, LDG_PC_MLP_BJ = 3, LDG_PC_RB_BJ = 4 };
enum { LDG_FORCING_FIXED = 0, LDG_FORCING_LAST = 1 };
enum { LDG_BASIS_FP64 = 0, LDG_BASIS_F32X2 = 1 };
enum { LDG_JV_AUTO = 0, LDG_JV_STAGE = 1 };

typedef struct {
  int newton_iters;
  int gmres_iters;      /* Arnoldi steps over all linear solves */
  int jv_calls;
  int residual_calls;
  double r0;            /* ||R(u_0)||_2 */
  double rfinal;        /* ||R(u)||_2 at exit (recomputed in FP64) */
  double lin_resid;     /* last linear solve: true relative residual */
  double elapsed_ms;
  int status;
  int pc_setups;        /* preconditioner builds during the call */
  int pc_fallbacks;     /* linear solves redone with block-Jacobi after the learned one failed */
  int newton_backtracks;  /* Newton step halvings: a step after which ||R|| grew more than
                             tenfold (or became non-finite) is halved, up to ten times in a row */
} ldg_solve_report;

typedef struct {
  int epochs;           /* passes over the pairs (default 50) */
  int batch;            /* pairs per Adam step (default 4096) */
  double lr;            /* Adam step size (default 1e-3) */
  uint64_t seed;        /* shuffling seed */
  int linear_init;      /* 1: start from the least-squares fit of the linear skip map (output
                           layer of the nonlinear branch zeroed); 0: from the current weights */
} ldg_train_opts;

typedef struct {
  double loss_first, loss_last;   /* mean loss of the first and last epoch */
  int steps;
  double elapsed_ms;
} ldg_train_report;

const char* ldg_version(void);

/* Number of CUDA kernels this library has launched in this process (all contexts). */
int64_t ldg_kernel_launches(void);

/* Creates a context for the discretisation of Section 2.2: the LDG method of order p
 * on the mesh of Section 3.2 for the model of Section 2.1 (Eq. 1a-1b), solved by the
 * Newton-GMRES of Section 3.3 with `opts`. It builds the reference element, the affine
 * (or sampled curved) geometry, the face connectivity and orientation tables on the
 * host, uploads them, and allocates the work space. `cuda_stream` is a cudaStream_t
 * (NULL = legacy default stream). *out receives the context (NULL on error).
 * Returns LDG_ERR_ARG for null or empty inputs, LDG_ERR_MESH for a rejected mesh,
 * LDG_ERR_UNSUPPORTED when no kernel is compiled for the (element, p, quadrature,
 * model), LDG_ERR_CUDA when an allocation or copy fails. */
int ldg_create(ldg_ctx** out, const ldg_mesh_desc* mesh, int p, const ldg_model_desc* model,
               const ldg_options* opts, void* cuda_stream);
int ldg_destroy(ldg_ctx* ctx);
int ldg_set_stream(ldg_ctx* ctx, void* cuda_stream);

/* n_dof = n_elem * n_cu * n_pe; dim = space dimension. */
int ldg_sizes(const ldg_ctx* ctx, int64_t* n_dof, int* n_pe, int* n_cu, int* dim);

/* Time scheme of the residual (Section 2.2): LDG_STEADY, or BDF1/BDF2 with step dt;
 * R then gains M (a0 u + a1 u^n + a2 u^{n-1}) / dt. u_n_dev / u_nm1_dev are read
 * once here (the history term is formed on the device); u_nm1_dev may be NULL for BDF1.
 * t is the time at which boundary data are evaluated. */
int ldg_set_time(ldg_ctx* ctx, int scheme, double t, double dt, const double* u_n_dev,
                 const double* u_nm1_dev);

/* Residual R(u) of Eq. 1b (with the q-stage of Eq. 1a for diffusion models). */
int ldg_residual(ldg_ctx* ctx, const double* u_dev, double* r_dev);

/* Exact J(u) v = dR/du(u) v (Section 3.3, the automatic-differentiation option):
 * forward-mode dual numbers for nonlinear models, the homogeneous linear operator
 * for linear ones. */
int ldg_jvp(ldg_ctx* ctx, const double* u_dev, const double* v_dev, double* jv_dev);

/* J.v in a chosen arithmetic: LDG_FP64 (same as ldg_jvp), LDG_FP32, LDG_F32X2,
 * LDG_TC_BF16X3 or LDG_TC_BF16 (inputs and output FP64 in memory; see the precision
 * constants). LDG_ERR_ARG for LDG_F32X2 or a tensor-core form on a context without
 * those kernels. */
int ldg_jvp_prec(ldg_ctx* ctx, int precision, const double* u_dev, const double* v_dev, double* jv_dev);

/* Names the kernels that form this context's J.v in `precision` (any of the precision
 * constants; "" where that arithmetic has no kernels) and the case they serve, e.g.
 * "k_lin_q + k_lin_r [hex p=4 nq=5 convdiff fp64, ...]".
 * The string stays valid until the calling thread's next call of this function. */
const char* ldg_jv_describe(const ldg_ctx* ctx, int precision);

/* The same J.v with HOST buffers (end-to-end form): u_host and v_host (n_dof doubles
 * each) are copied to the device, J(u) v is formed in `precision` (as ldg_jvp_prec) and
 * copied back to jv_host; the call returns after the copy back has finished. Pinned
 * (page-locked) host memory gives the fastest copies. u_host may be NULL for linear
 * models, whose J.v does not depend on u. The first call allocates 3 n_dof doubles of
 * context staging memory. Errors: LDG_ERR_ARG (null v_host / jv_host, NULL u_host for a
 * nonlinear model, bad precision), LDG_ERR_CUDA. */
int ldg_jvp_host(ldg_ctx* ctx, int precision, const double* u_host, const double* v_host, double* jv_host);

/* J(u) v_i for `count` directions in HOST memory (the end-to-end form of a sequence of
 * Jacobian-vector products of Section 3.3, e.g. for a Krylov method that keeps its
 * vectors on the host), with the copies of each direction overlapped with the J.v of its
 * neighbours: v_host[i] is copied in on one copy stream while the J.v of direction i - 1
 * runs on the context's stream and J(u) v_{i-2} is copied out to jv_host[i] on another,
 * through two device slots. Each result equals ldg_jvp_host's for that direction.
 * u_host: as in ldg_jvp_host (copied once). v_host[i], jv_host[i]: n_dof doubles of host
 * memory each, caller-owned; pinned (page-locked) memory lets the copies run beside the
 * kernels, pageable memory gives the same results without the overlap. Outputs are
 * written in order, so several jv_host[i] may name one buffer (it keeps the last); an
 * output buffer must not be the input of a later direction. The call returns after the
 * last copy back has finished. The first call allocates 5 n_dof doubles of context
 * staging memory, two streams and six events. Errors: LDG_ERR_ARG (count < 1, null
 * arrays or entries, NULL u_host for a nonlinear model, bad precision), LDG_ERR_CUDA. */
int ldg_jvp_host_many(ldg_ctx* ctx, int precision, const double* u_host, int count, const double* const* v_host,
                      double* const* jv_host);

/* J(u) v reusing the q(u) that the last ldg_residual(ctx, u, ...) call on this context
 * computed: the form of J.v inside Newton-GMRES, where every Krylov product of a
 * Newton step is taken at the state whose residual was just evaluated. Nonlinear
 * models with q (Navier-Stokes) skip their q(u) stage; other models compute exactly
 * what ldg_jvp_prec does. The caller guarantees that u is the state of that residual
 * call, unchanged since, and that no other residual call intervened (the result is
 * otherwise the Jacobian at the other state). precision: as ldg_jvp_prec. */
int ldg_jvp_after_residual(ldg_ctx* ctx, int precision, const double* u_dev, const double* v_dev, double* jv_dev);

/* Finite-difference J(u) v, the variant of Section 3.3 beside the exact derivative:
 * order 1: (R(u + eps v) - R(u)) / eps; order 2: (R(u + eps v) - R(u - eps v)) / (2 eps),
 * eps = 2^-26 (1 + ||u||_2) / ||v||_2 (0 when v = 0, giving J v = 0). Two residual
 * evaluations in FP64, time term included. Truncation error O(eps) (order 1) or
 * O(eps^2) (order 2), plus rounding of order 2^-52 ||R|| / eps. The first call
 * allocates 3 n_dof + 4 doubles of context scratch. order not 1 or 2: LDG_ERR_ARG. */
int ldg_jvp_fd(ldg_ctx* ctx, int order, const double* u_dev, const double* v_dev, double* jv_dev);

/* Exact element-diagonal blocks of J(u): blocks_dev [n_elem][n_loc][n_loc], column-major
 * per element (column l at offset l * n_loc), n_loc = n_cu * n_pe. Convection models use
 * dual numbers with a unit tangent on each element and none on its neighbours; diffusion
 * models use coloured probing (no two elements of one colour within two faces). Needed by
 * the block-Jacobi preconditioner that accelerates GMRES (the paper's own preconditioner,
 * Section 3.3, is a reduced-basis one; this is the plain baseline). */
int ldg_diag_blocks(ldg_ctx* ctx, int precision, const double* u_dev, double* blocks_dev);

/* Builds the block-Jacobi preconditioner M = blockdiag(J(u)) at state u (inverses held by
 * the context), and applies y = M^{-1} x (device vectors, n_dof doubles). */
int ldg_precond_setup(ldg_ctx* ctx, const double* u_dev);
int ldg_precond_apply(ldg_ctx* ctx, const double* x_dev, double* y_dev);

/* ------------------------------------------------------------------------------------
 * Reduced-basis preconditioner (Section 3.3: a preconditioner built by the reduced basis
 * method and a low-rank approximation of the Jacobian; its construction is given in the
 * paper's references, so this is a reading of the passage). The reduced basis W holds up
 * to rb_size orthonormal vectors: the Newton updates of the solves so far (each update
 * is orthogonalised against the basis and enters it, the oldest leaving once it is
 * full), so that over a sequence of time steps it spans the directions the solution
 * keeps moving in. At the first Newton step of a solve the solver forms J W (rb_size
 * J.v in the Krylov arithmetic) and G = (J W)^T J W (its inverse on the host); each update
 * entering the basis adds one J.v and a row and column of G. It applies
 *   P^{-1} r = C r + B^{-1} (r - J C r),   C = W G^{-1} (J W)^T,
 * with B the block-Jacobi preconditioner: C r is the minimal-residual solve on span(W)
 * (J C the orthogonal projector onto span(J W)), block-Jacobi acts on the rest. On span(W)
 * the preconditioned operator is the identity (P^{-1} J w = w). precond = LDG_PC_RB_BJ
 * selects it (host-driven Newton-GMRES). */

/* Replaces the reduced basis by the k columns of W_dev ([k][n_dof], device, row-major;
 * k <= rb_size; orthonormalised on copy; k = 0 empties it). Errors: LDG_ERR_ARG. */
int ldg_rb_set_basis(ldg_ctx* ctx, const double* W_dev, int k);

/* The number of vectors in the reduced basis now. */
int ldg_rb_count(const ldg_ctx* ctx);

/* Learned per-element preconditioner (the learned pattern of this build; the paper's own
 * preconditioner, Section 3.3, is a reduced-basis one). A multilayer perceptron
 * 2n -> 128 -> 128 -> n (ReLU, n = n_cu * n_pe) shared by all elements acts on each
 * element block scaled to unit norm, with the element's state as features:
 *   M(v)_K = ||v_K|| net(v_K / ||v_K||, u_K)        (positively homogeneous in v).
 * It is trained on the GPU (FP32 master weights, Adam) by mean-squared error on
 * triples (v_K, z_K, u_K) where z = (block-Jacobi)^{-1} v is the block correction the
 * plain solver computes; inference uses BF16 weights with FP32 arithmetic.
 * X_dev, T_dev, U_dev: [n_pairs][n] FP64 element blocks (rows of v, z and u).
 * The output layer adds a learned linear map of the scaled block: net = W3 h2 + b3 + Ws v/||v||.
 * Parameters (get/set, FP64 host, *count entries): W1 [128][2n], b1, W2 [128][128],
 * b2, W3 [n][128], b3, Ws [n][n]. ldg_mlp_apply evaluates y = M(x) at state u. */
int ldg_mlp_init(ldg_ctx* ctx, uint64_t seed);
int ldg_mlp_params(ldg_ctx* ctx, int get, double* host_params, int64_t* count);
int ldg_mlp_loss_grad(ldg_ctx* ctx, const double* X_dev, const double* T_dev, const double* U_dev, int64_t n_pairs,
                      double* loss, double* grad_host);
int ldg_mlp_train(ldg_ctx* ctx, const double* X_dev, const double* T_dev, const double* U_dev, int64_t n_pairs,
                  const ldg_train_opts* opts, ldg_train_report* rep);
int ldg_mlp_apply(ldg_ctx* ctx, const double* u_dev, const double* x_dev, double* y_dev);

/* ldg_newton_gmres with the block-Jacobi preconditioner that also stores, for every
 * Arnoldi vector v_j of every linear solve, v_j in X_dev[i], its block correction
 * (block-Jacobi)^{-1} v_j in T_dev[i] and the Newton state u in U_dev[i] (n_dof
 * doubles each, up to `capacity` vectors; *count receives how many): training data
 * for the learned preconditioner. */
int ldg_newton_gmres_collect(ldg_ctx* ctx, double* u_dev, double* X_dev, double* T_dev, double* U_dev, int capacity,
                             int* count, ldg_solve_report* rep);

/* Learned correction of block-Jacobi (LDG_PC_MLP_BJ; the learned pattern of this build,
 * trained on the (residual, Newton update) pairs the plain block-Jacobi solver itself
 * generates). The same network as above acts on the block-Jacobi image z = BJ^{-1} v:
 *   M(v)_K = ||z_K|| net(z_K / ||z_K||, h_K),
 *   h_K[c][i] = (sum over the faces f of K that hold node i of the face neighbour's z at
 *               the node in the same place) / ||z_K||   (0 at interior nodes, on boundary faces),
 * so each element sees its neighbours' block-Jacobi corrections along its faces, the
 * coupling block-Jacobi leaves out. Positively homogeneous in v. The blocks are those of
 * the context's block-Jacobi set-up (built at each solve's initial guess).
 *
 * ldg_newton_collect_updates runs the plain block-Jacobi Newton-GMRES solve from u_dev and
 * stores (residual, update) pairs that solve generates, as features and targets: an input
 * r goes in as X = z = BJ^{-1} r and U = h (the scaled neighbour traces of z), its update
 * d as T. `which` selects the pairs (bit mask):
 *   1: every Newton step k: r = R(u_k), d = the Newton update delta_k (J delta_k = R(u_k),
 *      solved to the linear tolerance);
 *   2: every Arnoldi step j of every linear solve: r = J z_j, d = z_j, where z_j is the
 *      block-Jacobi-preconditioned Krylov direction: exact pairs of J^{-1} on the Krylov
 *      space the solver explores.
 * n_dof doubles per pair in each of X_dev, T_dev, U_dev, up to `capacity` pairs; *count
 * receives how many. Train on them with ldg_mlp_train(X, T, U).
 * ldg_halo_features writes h for a given z (device vectors). ldg_mlp_bj_apply evaluates
 * y = M(x) with the current blocks (after ldg_precond_setup) and BF16 weights.
 * Errors: LDG_ERR_ARG (null pointers, no network for the apply), LDG_ERR_UNSUPPORTED
 * (hexahedra whose quadrature size differs from p + 1: their face nodes cannot be matched). */
int ldg_newton_collect_updates(ldg_ctx* ctx, double* u_dev, double* X_dev, double* T_dev, double* U_dev,
                               int capacity, int which, int* count, ldg_solve_report* rep);
int ldg_halo_features(ldg_ctx* ctx, const double* z_dev, double* h_dev);
int ldg_mlp_bj_apply(ldg_ctx* ctx, const double* x_dev, double* y_dev);

/* Stages of R and J.v for element-sharded use (one context per rank, Section 3.5's MPI
 * design on GPUs): the rank's mesh lists its owned elements first, then ghost copies of
 * the face neighbours that other ranks own. A stage computes elements [0, n_owned) only
 * and reads the neighbours' values, ghosts included, from the input vectors, so that the
 * caller can exchange the ghosts' u before the q-stage and their q before the residual
 * stage (FP64 arithmetic; device vectors laid out as for the whole local mesh).
 *   ldg_q_stage:        q of Eq. 1a of u into q_dev [n_elem][n_cu][dim][n_pe] (models with q);
 *   ldg_residual_stage: R of Eq. 1b from u and q (q_dev may be NULL for Euler).
 * mode LDG_STAGE_R evaluates R(u) with boundary data, source and the time term of
 * ldg_set_time; LDG_STAGE_HOM the homogeneous operator of a linear model, whose value at v
 * is J v. Entries of the outputs beyond n_owned elements are left unchanged.
 * Errors: LDG_ERR_ARG (null pointers, n_owned outside [0, n_elem], bad mode, HOM for a
 * nonlinear model, q missing for a model with q). */
enum { LDG_STAGE_R = 0, LDG_STAGE_HOM = 1 };
int ldg_q_stage(ldg_ctx* ctx, int mode, int64_t n_owned, const double* u_dev, double* q_dev);
int ldg_residual_stage(ldg_ctx* ctx, int mode, int64_t n_owned, const double* u_dev, const double* q_dev,
                       double* r_dev);

/* Element-sharded R, J.v and GMRES over ranks (one context per rank, local mesh as for
 * the stage calls above). The caller supplies the transport:
 *   exchange_ghosts: fill the ghost elements' blocks (elements [n_owned, n_elem) of `block`
 *                    doubles each) of the element-major device vector dev_x from the ranks
 *                    that own them;
 *   allreduce_sum:   replace the `count` doubles at dev_buf by their sum over all ranks.
 * Both are called after the context's stream has drained, must complete before they return
 * and return 0 on success. Every rank must make the same sequence of calls.
 * ldg_shard_setup records n_owned and the transport (allocates a q buffer and reduction
 * scratch). ldg_shard_residual: R(u) (stage R, time term included); ldg_shard_jvp: J v of a
 * linear model; both exchange their input's ghosts first (the input is written there) and
 * write the owned elements of the output. ldg_shard_gmres: GMRES(m) on J x = b (linear
 * models) from x = 0 to gmres_rtol, classical Gram-Schmidt with one re-orthogonalisation,
 * Givens rotations on the host, every dot product summed over the ranks; x full length
 * (its ghost blocks are used as scratch). Errors: LDG_ERR_ARG (no setup, nonlinear model
 * for J.v or GMRES), LDG_ERR_CUDA (a transport call returned non-zero), LDG_ERR_MAXIT. */
typedef struct {
  void* user;
  int (*exchange_ghosts)(void* user, double* dev_x, int block, void* cuda_stream);
  int (*allreduce_sum)(void* user, double* dev_buf, int count, void* cuda_stream);
} ldg_comm;
int ldg_shard_setup(ldg_ctx* ctx, int64_t n_owned, const ldg_comm* comm);
int ldg_shard_residual(ldg_ctx* ctx, double* u_dev, double* r_dev);
int ldg_shard_jvp(ldg_ctx* ctx, double* v_dev, double* jv_dev);
int ldg_shard_gmres(ldg_ctx* ctx, const double* b_dev, double* x_dev, ldg_solve_report* rep);

/* q of Eq. 1a for diffusion models: q_dev [n_elem][n_cu][dim][n_pe]. */
int ldg_q(ldg_ctx* ctx, const double* u_dev, double* q_dev);

/* Nodal interpolant of the context's analytic case at time t. */
int ldg_interpolate(ldg_ctx* ctx, double t, double* u_dev);

/* L2 projection of the context's analytic case at time t onto the element space
 * (the projected initial or exact field beside Section 4.1's error study):
 * u_K = M_K^{-1} (phi, u_exact)_K per element, with integrals by a Gauss rule of
 * p + 3 points per direction (collapsed on simplices). u_dev: n_dof doubles,
 * written. Affine elements only: curved elements return LDG_ERR_UNSUPPORTED.
 * The first call builds the rule (a few host arrays and p + 3-point tables on the
 * device, plus 4 n_elem + 2 doubles of error partials). */
int ldg_project(ldg_ctx* ctx, double t, double* u_dev);

/* Relative L2 errors of Section 4.1 / Table 3 against the analytic case at time t:
 *   err_u = ||u_h - u||_L2 / ||u||_L2 (all components),
 *   err_q = ||q_h - q||_L2 / ||q||_L2 with q = -grad u and q_h from the q-stage of
 *           Eq. 1a (Poisson and convection-diffusion; 0 for the gas models),
 * integrated by the rule of ldg_project (a zero denominator counts as 1). u_dev is a
 * device vector; err_u and err_q (may be NULL) are host doubles, written after the
 * call has synchronised the context's stream. Overwrites the context's q scratch.
 * Affine elements only (LDG_ERR_UNSUPPORTED for curved elements). */
int ldg_l2_error(ldg_ctx* ctx, const double* u_dev, double t, double* err_u, double* err_q);

/* GMRES(m) on J(u) x = b from x = 0 (classical Gram-Schmidt with one
 * re-orthogonalisation, Givens rotations, FP64), to gmres_rtol. */
int ldg_gmres(ldg_ctx* ctx, const double* u_dev, const double* b_dev, double* x_dev, ldg_solve_report* rep);

/* Newton-GMRES (Section 3.3): u <- u - delta with J(u) delta = R(u), until
 * ||R(u)|| <= newton_rtol ||R(u_0)||. u_dev is the initial guess on entry and the
 * solution on return. Without the learned preconditioner (and with pc_refresh = 0)
 * the solve runs as the batched solver's single instance: one CUDA graph launch
 * (see ldg_batch_solve); the environment variable LDG_SOLVER_HOST_LOOPS=1 runs the
 * same kernels from host-driven loops instead (for profilers). */
int ldg_newton_gmres(ldg_ctx* ctx, double* u_dev, ldg_solve_report* rep);

/* The same solve with u in HOST memory: copied to the device, solved, copied back. */
int ldg_newton_gmres_host(ldg_ctx* ctx, double* u_host, ldg_solve_report* rep);

/* DIRK time schemes of ldg_dirk_step (Section 2.2 names DIRK as the paper's scheme):
 * singly diagonally implicit Runge-Kutta with the tableaus of backward Euler, of
 * Alexander (1977; L-stable, stiffly accurate; 2 stages order 2, 3 stages order 3)
 * and of Crouzeix (1975; 3 stages order 4, A-stable). */
enum { LDG_DIRK11 = 1, LDG_DIRK22 = 2, LDG_DIRK33 = 3, LDG_DIRK34 = 4 };

/* One DIRK step of M du/dt + R_s(u) = 0 from time t to t + dt; u_dev (device, n_dof)
 * holds u(t) on entry and u(t + dt) on return. Stage i solves, by the context's
 * Newton-GMRES (same options, preconditioner and graph engine as ldg_newton_gmres),
 *   M (U_i - u(t)) / (dt a_ii) + R_s(U_i) + sum_{j<i} (a_ij / a_ii) R_s(U_j) = 0
 * with boundary data at t + c_i dt and U_i starting from the previous stage; R_s(U_j)
 * is then re-evaluated, the slope K_i follows from U_i = u(t) + dt sum_{j<=i} a_ij K_j,
 * and u(t + dt) = u(t) + dt sum_i b_i K_i. The context is left steady at t + dt
 * (ldg_set_time's BDF state is replaced). rep (optional) sums the stages'
 * iterations; r0 is the first stage's ||R(U_0)||, rfinal the largest stage ratio
 * ||R(U_i)|| / ||R(U_i^0)|| at exit. The first call allocates 8 n_dof doubles of
 * context scratch. Errors: a stage's solver status; LDG_ERR_ARG for a bad scheme/dt. */
int ldg_dirk_step(ldg_ctx* ctx, int scheme, double t, double dt, double* u_dev, ldg_solve_report* rep);

/* Wave model (Section 2.1: the diffusion model with Eq. 1a replaced by dq/dt + grad u = 0,
 * and the ODE of Eq. 2, alpha dw/dt + beta w = s_w, recovering the displacement w; here
 * s_w = u). With u the velocity, q = -grad w and f = kappa q, kappa = c^2, the system
 *   M du/dt + R_s(u, q) = 0,   dq/dt = Q(u),   alpha dw/dt + beta w = u
 * (Q the LDG q-stage map of Eq. 1a, R_s the spatial residual of Eq. 1b with q given)
 * is the scalar wave equation w_tt = c^2 lap w. The context must be a Poisson model, or
 * convection-diffusion with beta = 0 (the same operator), of case LDG_CASE_ZERO (no
 * source, homogeneous Dirichlet or periodic faces): mu = {kappa, tau (, 0, 0, 0)}, the
 * wave speed squared and the jump penalty.
 * One step of a DIRK scheme (LDG_DIRK11..34, all singly diagonally implicit) from t to
 * t + dt: u_dev (n_dof), q_dev (n_dof * dim, layout [E][dim][n_pe]) and w_dev (n_dof;
 * may be NULL to skip the ODE) hold the state at t on entry and at t + dt on return.
 * Each stage eliminates its q: Q_i = Qh_i + a_ii dt Q(U_i), so the stage is the
 * context's own implicit Poisson solve (Newton-GMRES with its options and block-Jacobi,
 * host-driven) with kappa' = a_ii dt kappa and a constant term for Qh_i; q and w then
 * follow node by node. The blocks are built once per operator (kappa', a_ii dt) and kept
 * over stages and steps. The context's kappa is restored and its time scheme left
 * steady on return. rep (optional) sums the stages' iterations. The first call allocates
 * 12 n_dof + 6 n_dof dim doubles of context scratch. Errors: LDG_ERR_ARG (not such a
 * context, bad scheme, dt <= 0, alpha + beta a_ii dt = 0), a stage's solver status. */
int ldg_wave_step(ldg_ctx* ctx, int scheme, double t, double dt, double alpha, double beta, double* u_dev,
                  double* q_dev, double* w_dev, ldg_solve_report* rep);

/* J(u) v without any device allocation (the paper has no counterpart; this is a
 * service for callers that cannot allocate). It computes the same product as
 * ldg_jvp, but the scratch that product needs (q of the direction v for Poisson
 * and convection-diffusion, n_dof * dim doubles; q(u) and q of v for Navier-Stokes,
 * twice that; none for Euler) lives in a static device array inside this library
 * instead of the context's work space.
 *
 * Who needs it: callers that must not call cudaMalloc at this point. An application
 * whose device memory is held entirely by its own pool or caching allocator has no
 * memory left for a library to take, and a host loop with a fixed latency budget
 * cannot wait on an allocation, or on the device-wide synchronisation that cudaFree
 * implies. The call itself performs no cudaMalloc, cudaFree or allocating library
 * routine.
 *
 * Limits and behaviour:
 *  - The static array holds LDG_NOALLOC_SCRATCH_DOUBLES doubles (32 MiB). Every
 *    device that loads this library keeps it for the life of the process.
 *    An operator needing more returns LDG_ERR_ARG with a message naming both sizes.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current and caches it; host threads
 *    may make that first call concurrently. The cached address does not survive
 *    cudaDeviceReset: do not call this function on a device after resetting it.
 *  - All calls, from every context on a device, share the one array and the
 *    array keeps the last call's contents. The kernels overwrite every entry
 *    they read, so nothing needs clearing; but calls whose work overlaps on the
 *    GPU (different streams, or different host threads) race on the array and
 *    must be serialised by the caller.
 *  - Euler (no q) needs no scratch; the call then runs the dual-number kernel alone. */
#define LDG_NOALLOC_SCRATCH_DOUBLES 4194304
int ldg_jvp_noalloc(ldg_ctx* ctx, const double* u_dev, const double* v_dev, double* jv_dev);

const char* ldg_last_error(const ldg_ctx* ctx);

/* ------------------------------------------------------------------ autotuning
 * Every (element, p, quadrature, model) is compiled with several tile shapes (the
 * elements each CTA owns and the shared-memory budget they are sized for; the
 * paper's own code generator tunes its GPU kernels, Section 3.3). Tiles:
 *   0: <= 16 elements in <= 100 KB (the default)   1: <= 8 elements in <= 48 KB
 *   2: <= 32 elements in <= 100 KB                 3: <= 4 elements in <= 24 KB
 * ldg_autotune times the J.v of every distinct tile (in the context's Krylov
 * precision) on the context's own mesh, ten timed calls after three warm-up calls
 * with CUDA events, and keeps the fastest for all kernels of the context. The choice
 * is cached per (element, p, quadrature, model, precision, element-count octave) in
 * the process; force = 1 re-times. *best_ms = mean time of the chosen J.v (-1 when
 * the cached choice was used). The call synchronises the context's stream and
 * allocates three temporary vectors. ldg_set_tile forces a tile (LDG_ERR_UNSUPPORTED
 * when none is compiled); ldg_get_tile reports the current tile and its elements per
 * CTA for the q-stage, the residual and the J.v kernel. */
int ldg_autotune(ldg_ctx* ctx, int force, int* tile, double* best_ms);
int ldg_set_tile(ldg_ctx* ctx, int tile);
int ldg_get_tile(const ldg_ctx* ctx, int* tile, int* ne_q, int* ne_r, int* ne_j);

/* ---------------------------------------------------- batched parametrised problems
 * Many independent steady problems (one per instance: its own mesh, order p and model
 * parameters mu, all of one model and element type) solved together by
 * Newton-GMRES (Section 3.3) — a parameter sweep. Instances with the same
 * (element, p, quadrature) form a group whose meshes are joined into one disjoint
 * mesh, so each kernel launch covers every instance of a group; the model parameters
 * are looked up per element.
 *
 * Batch vector: all instances' states in one device array of n_total doubles.
 * Instance i occupies offsets[i] .. offsets[i] + n_dof[i] - 1 in its own element-major
 * layout (the layout of a single context). Instances are stored group by group, so
 * offsets need not increase with i.
 *
 * The solve runs Newton-GMRES per instance, all instances in lock step: classical
 * Gram-Schmidt with re-orthogonalisation, Givens rotations, restarts, convergence
 * tests and the Newton update are per instance (segmented reductions over the
 * batch vector); an instance that has converged drops out of every kernel. With
 * use_graph = 1 the whole solve is one CUDA graph launch: the Newton, restart and
 * Arnoldi loops are graph WHILE nodes whose conditions the device sets, so the host
 * neither waits nor decides anything until the batch is solved. use_graph = 0 runs
 * the same kernels with host-driven loops (for testing).
 * opts (shared by all instances): gmres_m, max_restarts, max_newton, newton_rtol,
 * gmres_rtol, krylov_precision, precond (LDG_PC_NONE or LDG_PC_BJACOBI; the
 * block-Jacobi blocks are built inside ldg_batch_solve at the initial guess);
 * nq1 = 0 picks the default per order. Time schemes: ldg_batch_set_time (as ldg_set_time,
 * with batch vectors); the default is steady.
 * reps: n_inst reports (host), one per instance. *elapsed_ms: wall time of the whole
 * batched solve, set-up included. */
typedef struct ldg_batch ldg_batch;
int ldg_batch_create(ldg_batch** out, int n_inst, const ldg_mesh_desc* meshes, const int* p,
                     const ldg_model_desc* models, const ldg_options* opts, void* cuda_stream);
int ldg_batch_destroy(ldg_batch* b);
/* n_total doubles in the batch vector; offsets / n_dof: [n_inst] host arrays (may be NULL);
 * n_groups: number of (element, p) groups. */
int ldg_batch_sizes(const ldg_batch* b, int64_t* n_total, int64_t* offsets, int64_t* n_dof, int* n_groups);
/* Time scheme of every instance (see ldg_set_time; u_n_dev / u_nm1_dev are batch vectors).
 * The boundary-data time is kept in device memory, so a captured solve graph stays valid
 * from step to step; a change of scheme or dt re-captures it at the next solve. */
int ldg_batch_set_time(ldg_batch* b, int scheme, double t, double dt, const double* u_n_dev,
                       const double* u_nm1_dev);
/* R(u) and J(u) v of every instance (batch vectors, device). */
int ldg_batch_residual(ldg_batch* b, const double* u_dev, double* r_dev);
int ldg_batch_jvp(ldg_batch* b, int precision, const double* u_dev, const double* v_dev, double* jv_dev);
/* Autotunes each group (see ldg_autotune); tiles: [n_groups] chosen tiles (may be NULL). */
int ldg_batch_autotune(ldg_batch* b, int force, int* tiles);
int ldg_batch_solve(ldg_batch* b, double* u_dev, int use_graph, ldg_solve_report* reps, double* elapsed_ms);
/* Kernel executions of the last ldg_batch_solve (inside the graph, counted from the
 * loop trip counts the device recorded). */
int64_t ldg_batch_kernel_executions(const ldg_batch* b);
const char* ldg_batch_last_error(const ldg_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* LDG_H */
