// Nodal form of the homogeneous operator (J.v) of the linear diffusion models
// (Poisson, convection-diffusion) on affine quadrilaterals and hexahedra with
// Gauss-Lobatto nodes (Section 2.2, Eq. 1a-1b; Section 3.3's J.v).
//
// For a linear model every integrand of R(v) - R(0) is a polynomial of degree <= 2p
// on an affine element, and the quadrature of the stage kernels (p + 1 Gauss points per
// direction) integrates it exactly. The same operator therefore has an exact form on
// the nodal values alone, with the 1-D matrices of the Gauss-Lobatto basis l_i:
//   M1[i][j] = int l_i l_j,   C[i][j] = int l_i' l_j,   Dn[i][j] = l_j'(x_i),
// and the columns L0 = M1^{-1} e_0, L1 = M1^{-1} e_p:
//
//  q-stage (Eq. 1a, strong form): the face mass matrix of face f is sJ (M1 x M1), so
//  lifting the weighted trace difference and applying the element's inverse mass matrix
//  M^{-1} = (M1 x M1 x M1)^{-1} / det J cancels the tangential factors:
//    q_d = -sum_k Jinv[k][d] D_k v + sum_f n_{f,d} (sJ_f / det J) L_f(i_axis) Delta_f,
//    Delta_f = v- - vhat at the face nodes ((v- - v+)/2 inside, v- on Dirichlet faces).
//  residual (Eq. 1b): with the nodal flux g_k = det J sum_d Jinv[k][d] (beta_d v + kappa q_d),
//    R = -(C x M1 x M1) g_0 - (M1 x C x M1) g_1 - (M1 x M1 x C) g_2
//        + sum_f sJ_f (M1 x M1) Fhat_f + a0/dt det J (M1 x M1 x M1) v,
//    Fhat_f = beta.n v_upwind + kappa/2 (q- + q+).n + tau (v- - v+) at the face nodes
//    (Dirichlet faces: beta.n v- if beta.n >= 0, kappa q-.n + tau v-).
// Each stage is one kernel with one thread per node; contractions along an axis read
// the node's line from shared memory. q of the direction is stored in QT (double, or
// float for the FP32-arithmetic J.v: it is internal scratch of the product).
#pragma once
#include <type_traits>

#include "ldg_df.cuh"
#include "ldg_kernels.cuh"

namespace ldg {

// Blob of 1-D operators (N1 = p + 1 values per axis): Dn, M1, C, then L0 and L1, then
// the products C Dn, C L0 and C L1 (for the residual of axis-aligned boxes).
template <int N1> struct LinOff {
  static constexpr int DN = 0, M1 = N1 * N1, C = 2 * N1 * N1, L = 3 * N1 * N1, SIZE = 3 * N1 * N1 + 2 * N1;
  static constexpr int CD = SIZE, CL = CD + N1 * N1;
};

// Elements per CTA (one thread per node, elements packed back to back) and threads.
template <int DIM, int N1> struct LinShape {
  static constexpr int NPE = ipow(N1, DIM), NFN = ipow(N1, DIM - 1), NF = 2 * DIM;
  static constexpr int NE = NPE >= 256 ? 1 : 256 / NPE;
  static constexpr int NT = (NE * NPE + 31) / 32 * 32;
  static constexpr int GEO = Geo<DIM>::size(NF);
};
// Resident 256-thread CTAs asked of the register allocator: eight (32 registers a
// thread) for the FP32 kernels, whose face gathers and barriers want every warp slot;
// six (40 registers) for FP64, whose doubles would spill at 32 (measured on 48^3 p = 4);
// four (64 registers) for double-float, whose accumulators hold two floats and whose
// error-free transformations keep several temporaries live.
template <int NT, class R> struct LinMinBlocks {
  static constexpr int value = NT > 256 ? 1 : (sizeof(R) == 4 ? 8 : (std::is_same<R, df>::value ? 4 : 6));
};

// local node of face-node j on face f = 2 axis + side (free axes ascending, first fastest)
template <int DIM, int N1> __device__ __forceinline__ int lin_face_node(int f, int j) {
  const int ax = f >> 1, fix = (f & 1) ? N1 - 1 : 0;
  if constexpr (DIM == 2) return ax == 0 ? fix + N1 * j : j + N1 * fix;
  else {
    const int a = j % N1, b = j / N1;
    if (ax == 0) return fix + N1 * (a + N1 * b);
    if (ax == 1) return a + N1 * (fix + N1 * b);
    return a + N1 * (b + N1 * fix);
  }
}
// face-node index of node (i0, i1, i2) on a face of axis ax
template <int DIM, int N1> __device__ __forceinline__ int lin_face_index(int ax, const int* id) {
  if constexpr (DIM == 2) return id[1 - ax];
  else return ax == 0 ? id[1] + N1 * id[2] : (ax == 1 ? id[0] + N1 * id[2] : id[0] + N1 * id[1]);
}

// The operator blob a kernel in arithmetic R reads (double-float splits the FP64 one)
template <class R> struct LinBlob { typedef double type; };
template <> struct LinBlob<float> { typedef float type; };
template <class R> __device__ __forceinline__ const typename LinBlob<R>::type* lin_ops(const KArgs& a) {
  if constexpr (std::is_same<R, float>::value) return a.lopsf;
  else return a.lops;
}

// ------------------------------------------------------------------ q-stage
template <int DIM, int N1, class R, class QT>
__global__ void __launch_bounds__(LinShape<DIM, N1>::NT, (LinMinBlocks<LinShape<DIM, N1>::NT, R>::value)) k_lin_q(KArgs a) {
  typedef LinShape<DIM, N1> S;
  typedef LinOff<N1> O;
  typedef Geo<DIM> G;
  constexpr int NPE = S::NPE, NFN = S::NFN, NF = S::NF, NE = S::NE, NT = S::NT, GEO = S::GEO;
  typedef typename AccOf<R>::type A;
  if (a.skip && *a.skip) return;
  const int e0 = blockIdx.x * NE;
  const int ne = min(NE, a.E - e0);
  if (!cta_active(a, e0, ne)) return;
  __shared__ R ops[O::SIZE];
  __shared__ R Gs[NE][GEO];
  __shared__ R Vs[NE][NPE];
  __shared__ R Ds[NE][NF][NFN];
  const int t = threadIdx.x;
  const auto* lo = lin_ops<R>(a);
  for (int i = t; i < O::SIZE; i += NT) ops[i] = R(lo[i]);
  for (int i = t; i < ne * GEO; i += NT) Gs[i / GEO][i % GEO] = R(a.geo[(size_t)e0 * GEO + i]);
  const double* v = (const double*)a.u;
  const int e = t / NPE, n = t - e * NPE;
  const bool own = e < ne;
  // the neighbours' face-node values of this thread's face items, loaded before the
  // first barrier so that their latency overlaps the element's own loads
  constexpr int NFI = NE * NF * NFN, ROUNDS = (NFI + NT - 1) / NT;
  R vpre[ROUNDS];
  int hasnb = 0;
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    const int it = t + r * NT;
    vpre[r] = R(0);
    if (it < NFI) {
      const int j = it % NFN, f = (it / NFN) % NF, el = it / (NFN * NF);
      if (el < ne) {
        const int nb = a.nbr[(size_t)(e0 + el) * NF + f];
        if (nb >= 0) {
          const int code = a.nbf[(size_t)(e0 + el) * NF + f];
          const int jn = a.perm[(code >> 3) * NFN + j];
          vpre[r] = R(v[(size_t)nb * NPE + lin_face_node<DIM, N1>(code & 7, jn)]);
          hasnb |= 1 << r;
        }
      }
    }
  }
  if (own) Vs[e][n] = R(v[(size_t)(e0 + e) * NPE + n]);
  __syncthreads();

  // Delta_f = v- - vhat at the face nodes
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    const int it = t + r * NT;
    if (it >= NFI) break;
    const int j = it % NFN, f = (it / NFN) % NF, el = it / (NFN * NF);
    R d = R(0);
    if (el < ne) {
      const R vm = Vs[el][lin_face_node<DIM, N1>(f, j)];
      d = (hasnb >> r) & 1 ? (vm - vpre[r]) * R(0.5) : vm;
    }
    Ds[el][f][j] = d;
  }
  __syncthreads();
  if (!own) return;

  // On an affine element the outward normal of face xi_k = +-1 times its surface
  // Jacobian is +-det J times row k of J^{-1} (Nanson's formula), so the lift of face
  // 2k + side is +-Jinv[k][d] L_side(i_k) Delta and joins the derivative along axis k:
  //   q_d = -sum_k Jinv[k][d] (D_k v - L_p(i_k) Delta_{2k+1} + L_0(i_k) Delta_{2k}).
  const int id[3] = {n % N1, (n / N1) % N1, DIM == 3 ? n / (N1 * N1) : 0};
  constexpr int STR[3] = {1, N1, N1 * N1};
  R gk[DIM];
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    const R* line = &Vs[e][n - id[k] * STR[k]];
    const R* dn = ops + O::DN + id[k] * N1;
    const int jf = lin_face_index<DIM, N1>(k, id);
    A s = A(ops[O::L + id[k]] * Ds[e][2 * k][jf]);
    s -= ops[O::L + N1 + id[k]] * Ds[e][2 * k + 1][jf];
#pragma unroll
    for (int m = 0; m < N1; ++m) s += dn[m] * line[m * STR[k]];
    gk[k] = R(s);
  }
  R qd[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    A s = A(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) s -= Gs[e][G::JINV + k * DIM + d] * gk[k];
    qd[d] = R(s);
  }
  QT* q = (QT*)a.out;
#pragma unroll
  for (int d = 0; d < DIM; ++d) q[((size_t)(e0 + e) * DIM + d) * NPE + n] = QT(qd[d]);
}

// ----------------------------------------------------------------- residual
// The face terms need no contraction of their own. Face f of axis k carries sJ (M1 x M1)
// over its two free axes, which are the axes other than k, so sJ Fhat_f placed at the
// end nodes of the axis-k lines, beside their C contraction, picks up exactly those two
// factors from the volume passes that follow:
//   R = -[M1_z (M1_y X + M1_x Y) + M1_x M1_y Z],
//   X = C_x g_0 - E_x Fhat_x - M1_x (a0/dt det J v),  Y = C_y g_1 - E_y Fhat_y,
//   Z = C_z g_2 - E_z Fhat_z     (2-D: R = -(M1_y X + M1_x Y)),
// E_k Fhat_k placing the two faces of axis k at the nodes i_k = 0 and i_k = p. The
// fluxes are formed one face node per thread, spread over the whole CTA, and written as
// the initial values of the X, Y, Z accumulators; the other nodes start at zero. The
// FP64 pipe issues whole warps, masked lanes included, so every FP64 instruction here is
// executed by converged warps.
template <int DIM, int N1, bool CONV, class R, class QT>
__global__ void __launch_bounds__(LinShape<DIM, N1>::NT, (LinMinBlocks<LinShape<DIM, N1>::NT, R>::value)) k_lin_r(KArgs a) {
  typedef LinShape<DIM, N1> S;
  typedef LinOff<N1> O;
  typedef Geo<DIM> G;
  constexpr int NPE = S::NPE, NFN = S::NFN, NF = S::NF, NE = S::NE, NT = S::NT, GEO = S::GEO;
  typedef typename AccOf<R>::type A;
  if (a.skip && *a.skip) return;
  const int e0 = blockIdx.x * NE;
  const int ne = min(NE, a.E - e0);
  if (!cta_active(a, e0, ne)) return;
  __shared__ R ops[O::SIZE];
  __shared__ R Ak[NE][DIM][DIM + 1];  // g_k = sum_d Ak[k][d] q_d + Ak[k][DIM] v
  __shared__ R FC[NE][NF][DIM + 2];   // per face: kappa/2 sJ n_d, tau sJ, sJ beta.n
  __shared__ R DJ[NE];                // a0/dt det J
  __shared__ unsigned char FK[NE][NF];  // bit 0: the face has a neighbour; bit 1: beta.n >= 0
  __shared__ R Vs[NE][NPE];           // v
  __shared__ R Qs[NE][DIM][NPE];      // q
  __shared__ R Gk[NE][DIM][NPE];      // nodal fluxes g_k, later the axis-2 inputs (3-D)
  __shared__ R Tk[NE][DIM][NPE];      // X, Y, Z (face fluxes first)
  const int t = threadIdx.x;
  const auto* lo = lin_ops<R>(a);
  for (int i = t; i < O::SIZE; i += NT) ops[i] = R(lo[i]);
  for (int i = t; i < ne; i += NT) DJ[i] = R(a.a0dt * a.geo[(size_t)(e0 + i) * GEO + G::DETJ]);
  for (int i = t; i < ne * DIM; i += NT) {
    // det J Jinv[k][.] (kappa q + beta v): per element kappa det J Jinv[k][d] and det J Jinv[k].beta
    const int el = i / DIM, k = i % DIM;
    const double* g = a.geo + (size_t)(e0 + el) * GEO;
    const ModelParams mp = elem_mp(a, e0 + el);
    double bsum = 0.0;
    for (int d = 0; d < DIM; ++d) {
      const double jd = g[G::DETJ] * g[G::JINV + k * DIM + d];
      Ak[el][k][d] = R(mp.kappa * jd);
      bsum += jd * mp.beta[d];
    }
    Ak[el][k][DIM] = CONV ? R(bsum) : R(0);
  }
  for (int i = t; i < ne * NF; i += NT) {
    const int el = i / NF, f = i % NF;
    const double* g = a.geo + (size_t)(e0 + el) * GEO + G::FACE + f * (DIM + 1);
    const ModelParams mp = elem_mp(a, e0 + el);
    const double sj = g[DIM];
    double bn = 0.0;
    for (int d = 0; d < DIM; ++d) {
      FC[el][f][d] = R(0.5 * mp.kappa * sj * g[d]);
      bn += mp.beta[d] * g[d];
    }
    FC[el][f][DIM] = R(mp.tau * sj);
    FC[el][f][DIM + 1] = CONV ? R(sj * bn) : R(0);
    FK[el][f] = (a.nbr[(size_t)(e0 + el) * NF + f] >= 0 ? 1 : 0) | (!CONV || bn >= 0.0 ? 2 : 0);
  }
  const double* v = (const double*)a.u;
  const QT* q = (const QT*)a.q;
  const bool tterm = a.a0dt != 0.0;
  const int e = t / NPE, n = t - e * NPE;
  const bool own = e < ne;
  const int id[3] = {n % N1, (n / N1) % N1, DIM == 3 ? n / (N1 * N1) : 0};
  constexpr int STR[3] = {1, N1, N1 * N1};
  // the neighbours' v and q at this thread's face items, loaded before the first barrier
  constexpr int NFI = NE * NF * NFN, ROUNDS = (NFI + NT - 1) / NT;
  R vpre[ROUNDS], qpre[ROUNDS][DIM];
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    const int it = t + r * NT;
    vpre[r] = R(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) qpre[r][d] = R(0);
    if (it < NFI) {
      const int j = it % NFN, f = (it / NFN) % NF, el = it / (NFN * NF);
      if (el < ne) {
        const int nb = a.nbr[(size_t)(e0 + el) * NF + f];
        if (nb >= 0) {
          const int code = a.nbf[(size_t)(e0 + el) * NF + f];
          const int node = lin_face_node<DIM, N1>(code & 7, a.perm[(code >> 3) * NFN + j]);
          vpre[r] = R(v[(size_t)nb * NPE + node]);
#pragma unroll
          for (int d = 0; d < DIM; ++d) qpre[r][d] = R(q[((size_t)nb * DIM + d) * NPE + node]);
        }
      }
    }
  }
  R vn = R(0), qn[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) qn[d] = R(0);
  if (own) {
    vn = R(v[(size_t)(e0 + e) * NPE + n]);
#pragma unroll
    for (int d = 0; d < DIM; ++d) qn[d] = R(q[((size_t)(e0 + e) * DIM + d) * NPE + n]);
    Vs[e][n] = vn;
#pragma unroll
    for (int d = 0; d < DIM; ++d) Qs[e][d][n] = qn[d];
  }
  __syncthreads();

  // ---- phase 0: nodal fluxes g_k; zero X, Y, Z off the faces of their axis; sJ fhat =
  //   tau sJ (v- - v+) + kappa/2 sJ (q- + q+).n + sJ beta.n v_upwind
  // at every face node, placed as -sJ fhat into the accumulator of the face's axis
  // (Dirichlet faces: v+ = 0, q+ = q-, and no inflow)
  if (own) {
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      A s = CONV ? A(Ak[e][k][DIM] * vn) : A(0);
#pragma unroll
      for (int d = 0; d < DIM; ++d) s += Ak[e][k][d] * qn[d];
      Gk[e][k][n] = R(s);
      if (id[k] != 0 && id[k] != N1 - 1) Tk[e][k][n] = R(0);
    }
  }
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    const int it = t + r * NT;
    if (it >= NFI) break;
    const int j = it % NFN, f = (it / NFN) % NF, el = it / (NFN * NF);
    if (el >= ne) continue;
    const int node = lin_face_node<DIM, N1>(f, j);
    const R* fc = FC[el][f];
    const int fk = FK[el][f];
    const bool nb = fk & 1;
    const R vm = Vs[el][node];
    A s = A(fc[DIM] * (vm - vpre[r]));
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const R qm = Qs[el][d][node];
      s += fc[d] * (qm + (nb ? qpre[r][d] : qm));
    }
    if (CONV) s += fc[DIM + 1] * ((fk & 2) ? vm : vpre[r]);
    Tk[el][f >> 1][node] = -R(s);
  }
  __syncthreads();

  // ---- phase 1: C along each axis onto the face values, and the time term's M1 along
  // axis 0
  if (own) {
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const R* cr = ops + O::C + id[k] * N1;
      const R* line = &Gk[e][k][n - id[k] * STR[k]];
      A acc = A(Tk[e][k][n]);
#pragma unroll
      for (int m = 0; m < N1; ++m) acc += cr[m] * line[m * STR[k]];
      if (k == 0 && tterm) {
        const R* mr = ops + O::M1 + id[0] * N1;
        const R* vl = &Vs[e][n - id[0]];
        A h = A(0);
#pragma unroll
        for (int m = 0; m < N1; ++m) h += mr[m] * vl[m];
        acc -= DJ[e] * R(h);
      }
      Tk[e][k][n] = R(acc);
    }
  }
  __syncthreads();

  // ---- phase 2: M1 along axis 1 of X and Z, along axis 0 of Y
  R rv = R(0);
  if (own) {
    const R* m1 = ops + O::M1 + id[1] * N1;
    const R* m0 = ops + O::M1 + id[0] * N1;
    const int b1 = n - id[1] * N1, b0 = n - id[0];
    A s = A(0);
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      s += m1[m] * Tk[e][0][b1 + m * N1];
      s += m0[m] * Tk[e][1][b0 + m];
    }
    if constexpr (DIM == 2) {
      rv = -R(s);
    } else {
      A z = A(0);
#pragma unroll
      for (int m = 0; m < N1; ++m) z += m1[m] * Tk[e][2][b1 + m * N1];
      Gk[e][0][n] = R(s);
      Gk[e][1][n] = R(z);
    }
  }
  // ---- phase 3 (3-D): M1 along axis 2 of M1_y X + M1_x Y, along axis 0 of M1_y Z
  if constexpr (DIM == 3) {
    __syncthreads();
    if (own) {
      const R* m2 = ops + O::M1 + id[2] * N1;
      const R* m0 = ops + O::M1 + id[0] * N1;
      const int b2 = n - id[2] * N1 * N1, b0 = n - id[0];
      A s = A(0);
#pragma unroll
      for (int m = 0; m < N1; ++m) {
        s += m2[m] * Gk[e][0][b2 + m * N1 * N1];
        s += m0[m] * Gk[e][1][b0 + m];
      }
      rv = -R(s);
    }
  }
  if (own) ((double*)a.out)[(size_t)(e0 + e) * NPE + n] = (double)rv;
}

// ------------------------------------------- axis-aligned boxes: the trace form
// When every element is an axis-aligned box (J and J^{-1} diagonal, s_k = Jinv[k][k],
// each face normal along its own axis), q enters the residual in two places only:
//  * the volume term C_k g_k with g_k = a_k q_k + b_k v (a_k = kappa det J s_k,
//    b_k = det J s_k beta_k) and q_k = -s_k (D_k v + L0 Delta_{2k} - Lp Delta_{2k+1}):
//      C_k g_k = W_k v + c0_k (C L0) Delta_{2k} - c0_k (C Lp) Delta_{2k+1},
//      W_k = -a_k s_k (C Dn) + b_k C,  c0_k = -a_k s_k,
//    with the 1-D products C Dn, C L0, C Lp formed on the host;
//  * the face fluxes, which need only q_k at the face nodes of the faces of axis k.
// So the q-stage forms q_k at the face nodes only (k_lin_qt, output [E][NF][NFN]) and
// the residual (k_lin_rt) applies W_k to v. The products with the zero entries of J^{-1}
// and of the normals drop out; the rest is the same operator as k_lin_q / k_lin_r.
template <int DIM, int N1, class R, class QT>
__global__ void __launch_bounds__(LinShape<DIM, N1>::NT, (LinShape<DIM, N1>::NT > 256 ? 1 : 8)) k_lin_qt(KArgs a) {
  typedef LinShape<DIM, N1> S;
  typedef LinOff<N1> O;
  typedef Geo<DIM> G;
  constexpr int NPE = S::NPE, NFN = S::NFN, NF = S::NF, NE = S::NE, NT = S::NT, GEO = S::GEO;
  typedef typename AccOf<R>::type A;
  if (a.skip && *a.skip) return;
  const int e0 = blockIdx.x * NE;
  const int ne = min(NE, a.E - e0);
  if (!cta_active(a, e0, ne)) return;
  __shared__ R ops[O::SIZE];
  __shared__ R SK[NE][DIM];           // -Jinv[k][k]
  __shared__ R Vs[NE][NPE];
  __shared__ R Ds[NE][NF][NFN];       // Delta_f = v- - vhat at the face nodes
  const int t = threadIdx.x;
  const auto* lo = lin_ops<R>(a);
  for (int i = t; i < O::SIZE; i += NT) ops[i] = R(lo[i]);
  for (int i = t; i < ne * DIM; i += NT)
    SK[i / DIM][i % DIM] = R(-a.geo[(size_t)(e0 + i / DIM) * GEO + G::JINV + (i % DIM) * (DIM + 1)]);
  const double* v = (const double*)a.u;
  constexpr int NFI = NE * NF * NFN, ROUNDS = (NFI + NT - 1) / NT;
  R vpre[ROUNDS];
  int hasnb = 0;
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    const int it = t + r * NT;
    vpre[r] = R(0);
    if (it < NFI) {
      const int j = it % NFN, f = (it / NFN) % NF, el = it / (NFN * NF);
      if (el < ne) {
        const int nb = a.nbr[(size_t)(e0 + el) * NF + f];
        if (nb >= 0) {
          const int code = a.nbf[(size_t)(e0 + el) * NF + f];
          vpre[r] = R(v[(size_t)nb * NPE + lin_face_node<DIM, N1>(code & 7, a.perm[(code >> 3) * NFN + j])]);
          hasnb |= 1 << r;
        }
      }
    }
  }
  for (int i = t; i < ne * NPE; i += NT) Vs[i / NPE][i % NPE] = R(v[(size_t)e0 * NPE + i]);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    const int it = t + r * NT;
    if (it >= NFI) break;
    const int j = it % NFN, f = (it / NFN) % NF, el = it / (NFN * NF);
    if (el >= ne) continue;
    const R vm = Vs[el][lin_face_node<DIM, N1>(f, j)];
    Ds[el][f][j] = (hasnb >> r) & 1 ? (vm - vpre[r]) * R(0.5) : vm;
  }
  __syncthreads();
  // q_k at face node j of face f = 2k + side: the axis-k line through it, at its end i_k
  constexpr int STR[3] = {1, N1, N1 * N1};
  QT* qt = (QT*)a.out;
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    const int it = t + r * NT;
    if (it >= NFI) break;
    const int j = it % NFN, f = (it / NFN) % NF, el = it / (NFN * NF);
    if (el >= ne) continue;
    const int k = f >> 1, ik = (f & 1) ? N1 - 1 : 0;
    const int node = lin_face_node<DIM, N1>(f, j), base = node - ik * STR[k];
    const R* dn = ops + O::DN + ik * N1;
    A s = A(ops[O::L + ik] * Ds[el][2 * k][j]);
    s -= ops[O::L + N1 + ik] * Ds[el][2 * k + 1][j];
#pragma unroll
    for (int m = 0; m < N1; ++m) s += dn[m] * Vs[el][base + m * STR[k]];
    qt[(size_t)e0 * NF * NFN + it] = QT(SK[el][k] * R(s));
  }
}

template <int DIM, int N1, bool CONV, class R, class QT>
__global__ void __launch_bounds__(LinShape<DIM, N1>::NT, (LinMinBlocks<LinShape<DIM, N1>::NT, R>::value)) k_lin_rt(KArgs a) {
  typedef LinShape<DIM, N1> S;
  typedef LinOff<N1> O;
  typedef Geo<DIM> G;
  constexpr int NPE = S::NPE, NFN = S::NFN, NF = S::NF, NE = S::NE, NT = S::NT, GEO = S::GEO;
  typedef typename AccOf<R>::type A;
  if (a.skip && *a.skip) return;
  const int e0 = blockIdx.x * NE;
  const int ne = min(NE, a.E - e0);
  if (!cta_active(a, e0, ne)) return;
  __shared__ R M1s[N1 * N1];
  __shared__ R AB[NE][DIM][2];        // a_k s_k, b_k
  __shared__ R W[NE][DIM][N1 * N1];   // W_k = -a_k s_k (C Dn) + b_k C
  __shared__ R WL[NE][DIM][2][N1];    // -a_k s_k (C L0), +a_k s_k (C Lp)
  __shared__ R FC[NE][NF][3];         // per face: kappa/2 sJ n_k, tau sJ, sJ beta.n
  __shared__ R DJ[NE];                // a0/dt det J
  __shared__ unsigned char FK[NE][NF];  // bit 0: the face has a neighbour; bit 1: beta.n >= 0
  __shared__ R Vs[NE][NPE];
  __shared__ R Ds[NE][NF][NFN];       // Delta_f (as in the q-stage)
  __shared__ R Tk[NE][DIM][NPE];      // X, Y, Z (face fluxes first)
  __shared__ R Gk[NE][2][NPE];        // axis-2 inputs (3-D)
  const int t = threadIdx.x;
  const auto* lo = lin_ops<R>(a);
  for (int i = t; i < N1 * N1; i += NT) M1s[i] = R(lo[O::M1 + i]);
  for (int i = t; i < ne * DIM; i += NT) {
    const int el = i / DIM, k = i % DIM;
    const double* g = a.geo + (size_t)(e0 + el) * GEO;
    const ModelParams mp = elem_mp(a, e0 + el);
    const double sk = g[G::JINV + k * (DIM + 1)], dj = g[G::DETJ];
    const double bk = k == 0 ? mp.beta[0] : (k == 1 ? mp.beta[1] : mp.beta[DIM - 1]);
    AB[el][k][0] = R(mp.kappa * dj * sk * sk);
    AB[el][k][1] = CONV ? R(dj * sk * bk) : R(0);
  }
  for (int i = t; i < ne * NF; i += NT) {
    const int el = i / NF, f = i % NF, k = f >> 1;
    const double* g = a.geo + (size_t)(e0 + el) * GEO + G::FACE + f * (DIM + 1);
    const ModelParams mp = elem_mp(a, e0 + el);
    const double bk = k == 0 ? mp.beta[0] : (k == 1 ? mp.beta[1] : mp.beta[DIM - 1]);
    const double nk = k == 0 ? g[0] : (k == 1 ? g[1] : g[DIM - 1]);
    const double sj = g[DIM], bn = bk * nk;
    FC[el][f][0] = R(0.5 * mp.kappa * sj * nk);
    FC[el][f][1] = R(mp.tau * sj);
    FC[el][f][2] = CONV ? R(sj * bn) : R(0);
    FK[el][f] = (a.nbr[(size_t)(e0 + el) * NF + f] >= 0 ? 1 : 0) | (!CONV || bn >= 0.0 ? 2 : 0);
  }
  for (int i = t; i < ne; i += NT) DJ[i] = R(a.a0dt * a.geo[(size_t)(e0 + i) * GEO + G::DETJ]);
  const double* v = (const double*)a.u;
  const QT* qt = (const QT*)a.q;
  const bool tterm = a.a0dt != 0.0;
  const int e = t / NPE, n = t - e * NPE;
  const bool own = e < ne;
  const int id[3] = {n % N1, (n / N1) % N1, DIM == 3 ? n / (N1 * N1) : 0};
  constexpr int STR[3] = {1, N1, N1 * N1};
  // the neighbour's v and q_k at this thread's face items, loaded before the first barrier
  constexpr int NFI = NE * NF * NFN, ROUNDS = (NFI + NT - 1) / NT;
  R vpre[ROUNDS], qpre[ROUNDS];
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    const int it = t + r * NT;
    vpre[r] = R(0);
    qpre[r] = R(0);
    if (it < NFI) {
      const int j = it % NFN, f = (it / NFN) % NF, el = it / (NFN * NF);
      if (el < ne) {
        const int nb = a.nbr[(size_t)(e0 + el) * NF + f];
        if (nb >= 0) {
          const int code = a.nbf[(size_t)(e0 + el) * NF + f];
          const int jn = a.perm[(code >> 3) * NFN + j];
          vpre[r] = R(v[(size_t)nb * NPE + lin_face_node<DIM, N1>(code & 7, jn)]);
          qpre[r] = R(qt[((size_t)nb * NF + (code & 7)) * NFN + jn]);
        }
      }
    }
  }
  if (own) Vs[e][n] = R(v[(size_t)(e0 + e) * NPE + n]);
  __syncthreads();

  // ---- phase 0: the element operators W_k and the lift coefficients; Delta and sJ fhat
  // at the face nodes (-sJ fhat into the accumulator of the face's axis); zero X, Y, Z
  // off the faces of their axis
  for (int i = t; i < ne * DIM * N1 * N1; i += NT) {
    const int el = i / (DIM * N1 * N1), k = (i / (N1 * N1)) % DIM, c = i % (N1 * N1);
    const R as = AB[el][k][0], bk = AB[el][k][1];
    W[el][k][c] = bk * R(lo[O::C + c]) + (-(as * R(lo[O::CD + c])));
    if (c < 2 * N1) WL[el][k][c / N1][c % N1] = R((c < N1 ? -as : as) * R(lo[O::CL + c]));
  }
  if (own) {
#pragma unroll
    for (int k = 0; k < DIM; ++k)
      if (id[k] != 0 && id[k] != N1 - 1) Tk[e][k][n] = R(0);
  }
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    const int it = t + r * NT;
    if (it >= NFI) break;
    const int j = it % NFN, f = (it / NFN) % NF, el = it / (NFN * NF);
    if (el >= ne) continue;
    const int node = lin_face_node<DIM, N1>(f, j);
    const R qm = R(qt[(size_t)e0 * NF * NFN + it]);
    const R* fc = FC[el][f];
    const int fk = FK[el][f];
    const bool nb = fk & 1;
    const R vm = Vs[el][node];
    const R dv = vm - vpre[r];
    Ds[el][f][j] = nb ? dv * R(0.5) : vm;
    A s = A(fc[1] * dv);
    s += fc[0] * (qm + (nb ? qpre[r] : qm));
    if (CONV) s += fc[2] * ((fk & 2) ? vm : vpre[r]);
    Tk[el][f >> 1][node] = -R(s);
  }
  __syncthreads();

  // ---- phase 1: W_k along each axis onto the face values, the lift of Delta, and the
  // time term's M1 along axis 0
  if (own) {
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const R* wr = &W[e][k][id[k] * N1];
      const R* line = &Vs[e][n - id[k] * STR[k]];
      const int j = lin_face_index<DIM, N1>(k, id);
      A acc = A(Tk[e][k][n]);
      acc += WL[e][k][0][id[k]] * Ds[e][2 * k][j];
      acc += WL[e][k][1][id[k]] * Ds[e][2 * k + 1][j];
#pragma unroll
      for (int m = 0; m < N1; ++m) acc += wr[m] * line[m * STR[k]];
      if (k == 0 && tterm) {
        const R* mr = M1s + id[0] * N1;
        A h = A(0);
#pragma unroll
        for (int m = 0; m < N1; ++m) h += mr[m] * line[m];
        acc -= DJ[e] * R(h);
      }
      Tk[e][k][n] = R(acc);
    }
  }
  __syncthreads();

  // ---- phase 2: M1 along axis 1 of X and Z, along axis 0 of Y
  R rv = R(0);
  if (own) {
    const R* m1 = M1s + id[1] * N1;
    const R* m0 = M1s + id[0] * N1;
    const int b1 = n - id[1] * N1, b0 = n - id[0];
    A s = A(0);
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      s += m1[m] * Tk[e][0][b1 + m * N1];
      s += m0[m] * Tk[e][1][b0 + m];
    }
    if constexpr (DIM == 2) {
      rv = -R(s);
    } else {
      A z = A(0);
#pragma unroll
      for (int m = 0; m < N1; ++m) z += m1[m] * Tk[e][2][b1 + m * N1];
      Gk[e][0][n] = R(s);
      Gk[e][1][n] = R(z);
    }
  }
  // ---- phase 3 (3-D): M1 along axis 2 of M1_y X + M1_x Y, along axis 0 of M1_y Z
  if constexpr (DIM == 3) {
    __syncthreads();
    if (own) {
      const R* m2 = M1s + id[2] * N1;
      const R* m0 = M1s + id[0] * N1;
      const int b2 = n - id[2] * N1 * N1, b0 = n - id[0];
      A s = A(0);
#pragma unroll
      for (int m = 0; m < N1; ++m) {
        s += m2[m] * Gk[e][0][b2 + m * N1 * N1];
        s += m0[m] * Gk[e][1][b0 + m];
      }
      rv = -R(s);
    }
  }
  if (own) ((double*)a.out)[(size_t)(e0 + e) * NPE + n] = (double)rv;
}

// Both stages of the J.v: v -> q(v) in qbuf (QT), then J v (CART: the trace form for
// axis-aligned boxes, q_k at the face nodes in qbuf).
template <int DIM, int N1, bool CONV, class R, class QT, bool CART>
cudaError_t launch_lin(const KArgs& a, void* qbuf, cudaStream_t s) {
  typedef LinShape<DIM, N1> S;
  if (a.E <= 0) return cudaSuccess;
  const int grid = (a.E + S::NE - 1) / S::NE;
  KArgs b = a;
  b.out = qbuf;
  if constexpr (CART) k_lin_qt<DIM, N1, R, QT><<<grid, S::NT, 0, s>>>(b);
  else k_lin_q<DIM, N1, R, QT><<<grid, S::NT, 0, s>>>(b);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  b = a;
  b.q = qbuf;
  if constexpr (CART) k_lin_rt<DIM, N1, CONV, R, QT><<<grid, S::NT, 0, s>>>(b);
  else k_lin_r<DIM, N1, CONV, R, QT><<<grid, S::NT, 0, s>>>(b);
  count_launch();
  return cudaGetLastError();
}


// ===================================================================== simplices
// The same nodal form on triangles and tetrahedra (equispaced nodes): the element's
// nodes on a face are the face's nodes, so the exact integrals become dense reference
// matrices (built on the host, rows padded to odd lengths):
//   Dn_k[n][m] = d_k phi_m(x_n),  C_k[i][j] = int phi_j d_k phi_i,  M = int phi_i phi_j,
//   LIFT_f = M^{-1} E_f M_f (E_f embeds face f's nodes),  M_f the face mass matrix;
//   q_d = -sum_k Jinv[k][d] Dn_k v + sum_f n_{f,d} (sJ_f / det J) LIFT_f Delta_f,
//   R   = -sum_k C_k g_k + sum_f sJ_f E_f M_f Fhat_f + a0/dt det J M v.
template <class EL> struct SimOff {
  static constexpr int DIM = EL::DIM, NPE = EL::NPE, NFN = EL::NFN, NF = EL::NF;
  static constexpr int LDA = NPE | 1, LDL = NFN | 1;
  static constexpr int DN = 0, C = DIM * NPE * LDA, M = 2 * DIM * NPE * LDA, LIFT = (2 * DIM + 1) * NPE * LDA,
                       MF = LIFT + NF * NPE * LDL, SIZE = MF + NFN * LDL;
};
template <class EL> struct SimShape {
  static constexpr int NPE = EL::NPE;
  static constexpr int NE = NPE >= 256 ? 1 : 256 / NPE;
  static constexpr int NT = (NE * NPE + 31) / 32 * 32;
  static constexpr int GEO = Geo<EL::DIM>::size(EL::NF);
};

// The neighbour's local node that carries face node j of this element's face: the
// permuted face node (tetrahedra), or the edge walked the other way when the edge's
// face points are (triangles).
template <class EL> __device__ __forceinline__ int sim_nbr_node(const KArgs& a, int code, int j) {
  if constexpr (EL::NODE_PERM) {
    return EL::face_node(code & 7, a.perm[(code >> 3) * EL::NFN + j]);
  } else {
    const bool rev = a.perm[(code >> 3) * EL::NFQ] != 0;
    return EL::face_node(code & 7, rev ? EL::NFN - 1 - j : j);
  }
}

template <class EL, class R, class QT>
__global__ void __launch_bounds__(SimShape<EL>::NT) k_sim_q(KArgs a) {
  typedef SimShape<EL> S;
  typedef SimOff<EL> O;
  typedef Geo<EL::DIM> G;
  constexpr int DIM = EL::DIM, NPE = EL::NPE, NFN = EL::NFN, NF = EL::NF, NE = S::NE, NT = S::NT, GEO = S::GEO;
  typedef typename AccOf<R>::type A;
  if (a.skip && *a.skip) return;
  const int e0 = blockIdx.x * NE;
  const int ne = min(NE, a.E - e0);
  if (!cta_active(a, e0, ne)) return;
  extern __shared__ __align__(16) unsigned char sim_dsm[];
  R* ops = (R*)sim_dsm;
  __shared__ R Gs[NE][GEO];
  __shared__ R Cf[NE][NF];            // sJ_f / det J
  __shared__ R Vs[NE][NPE];
  __shared__ R Ds[NE][NF][NFN];
  const int t = threadIdx.x;
  const auto* lo = lin_ops<R>(a);
  for (int i = t; i < O::SIZE; i += NT) ops[i] = R(lo[i]);
  for (int i = t; i < ne * GEO; i += NT) Gs[i / GEO][i % GEO] = R(a.geo[(size_t)e0 * GEO + i]);
  for (int i = t; i < ne * NF; i += NT) {
    const double* g = a.geo + (size_t)(e0 + i / NF) * GEO;
    Cf[i / NF][i % NF] = R(g[G::FACE + (i % NF) * (DIM + 1) + DIM] / g[G::DETJ]);
  }
  const double* v = (const double*)a.u;
  const int e = t / NPE, n = t - e * NPE;
  const bool own = e < ne;
  if (own) Vs[e][n] = R(v[(size_t)(e0 + e) * NPE + n]);
  __syncthreads();
  for (int it = t; it < NE * NF * NFN; it += NT) {
    const int j = it % NFN, f = (it / NFN) % NF, el = it / (NFN * NF);
    R d = R(0);
    if (el < ne) {
      const R vm = Vs[el][EL::face_node(f, j)];
      const int nb = a.nbr[(size_t)(e0 + el) * NF + f];
      if (nb >= 0) {
        const int code = a.nbf[(size_t)(e0 + el) * NF + f];
        d = (vm - R(v[(size_t)nb * NPE + sim_nbr_node<EL>(a, code, j)])) * (R(0.5) * Cf[el][f]);
      } else {
        d = vm * Cf[el][f];
      }
    }
    Ds[el][f][j] = d;
  }
  __syncthreads();
  if (!own) return;
  R gk[DIM];
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    const R* row = ops + O::DN + (k * NPE + n) * O::LDA;
    A s = A(0);
#pragma unroll 8
    for (int m = 0; m < NPE; ++m) s += row[m] * Vs[e][m];
    gk[k] = R(s);
  }
  R qd[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    A s = A(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) s -= Gs[e][G::JINV + k * DIM + d] * gk[k];
    qd[d] = R(s);
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const R* row = ops + O::LIFT + (f * NPE + n) * O::LDL;
    A lf = A(0);
#pragma unroll
    for (int j = 0; j < NFN; ++j) lf += row[j] * Ds[e][f][j];
#pragma unroll
    for (int d = 0; d < DIM; ++d) qd[d] += Gs[e][G::FACE + f * (DIM + 1) + d] * R(lf);
  }
  QT* q = (QT*)a.out;
#pragma unroll
  for (int d = 0; d < DIM; ++d) q[((size_t)(e0 + e) * DIM + d) * NPE + n] = QT(qd[d]);
}

// The face terms are formed one face node per thread over the whole CTA (flux, then its
// face-mass moment), so that the FP64 work runs in converged warps; a node then adds the
// moments of the faces it lies on.
template <class EL, bool CONV, class R, class QT>
__global__ void __launch_bounds__(SimShape<EL>::NT) k_sim_r(KArgs a) {
  typedef SimShape<EL> S;
  typedef SimOff<EL> O;
  typedef Geo<EL::DIM> G;
  constexpr int DIM = EL::DIM, NPE = EL::NPE, NFN = EL::NFN, NF = EL::NF, NE = S::NE, NT = S::NT, GEO = S::GEO;
  typedef typename AccOf<R>::type A;
  if (a.skip && *a.skip) return;
  const int e0 = blockIdx.x * NE;
  const int ne = min(NE, a.E - e0);
  if (!cta_active(a, e0, ne)) return;
  extern __shared__ __align__(16) unsigned char sim_dsm[];
  R* ops = (R*)sim_dsm;
  __shared__ R Ak[NE][DIM][DIM + 1];  // g_k = sum_d Ak[k][d] q_d + Ak[k][DIM] v
  __shared__ R FC[NE][NF][DIM + 2];   // per face: kappa/2 sJ n_d, tau sJ, sJ beta.n
  __shared__ R DJ[NE];                // a0/dt det J
  __shared__ R Gk[NE][DIM][NPE];
  __shared__ R Vs[NE][NPE];
  __shared__ R Qs[NE][DIM][NPE];
  __shared__ R FF[NE][NF][NFN];       // sJ fhat at the face nodes
  __shared__ R FM[NE][NF][NFN];       // its face-mass moments M_f (sJ fhat)
  const int t = threadIdx.x;
  const auto* lo = lin_ops<R>(a);
  for (int i = t; i < O::SIZE; i += NT) ops[i] = R(lo[i]);
  for (int i = t; i < ne; i += NT) DJ[i] = R(a.a0dt * a.geo[(size_t)(e0 + i) * GEO + G::DETJ]);
  for (int i = t; i < ne * DIM; i += NT) {
    const int el = i / DIM, k = i % DIM;
    const double* g = a.geo + (size_t)(e0 + el) * GEO;
    const ModelParams mp = elem_mp(a, e0 + el);
    double bsum = 0.0;
    for (int d = 0; d < DIM; ++d) {
      const double jd = g[G::DETJ] * g[G::JINV + k * DIM + d];
      Ak[el][k][d] = R(mp.kappa * jd);
      bsum += jd * mp.beta[d];
    }
    Ak[el][k][DIM] = CONV ? R(bsum) : R(0);
  }
  for (int i = t; i < ne * NF; i += NT) {
    const int el = i / NF, f = i % NF;
    const double* g = a.geo + (size_t)(e0 + el) * GEO + G::FACE + f * (DIM + 1);
    const ModelParams mp = elem_mp(a, e0 + el);
    const double sj = g[DIM];
    double bn = 0.0;
    for (int d = 0; d < DIM; ++d) {
      FC[el][f][d] = R(0.5 * mp.kappa * sj * g[d]);
      bn += mp.beta[d] * g[d];
    }
    FC[el][f][DIM] = R(mp.tau * sj);
    FC[el][f][DIM + 1] = CONV ? R(sj * bn) : R(0);
  }
  const double* v = (const double*)a.u;
  const QT* q = (const QT*)a.q;
  const bool tterm = a.a0dt != 0.0;
  const int e = t / NPE, n = t - e * NPE;
  const bool own = e < ne;
  // the neighbours' v and q at this thread's face items, loaded before the first barrier
  constexpr int NFI = NE * NF * NFN, ROUNDS = (NFI + NT - 1) / NT;
  R vpre[ROUNDS], qpre[ROUNDS][DIM];
  int hasnb = 0;
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    const int it = t + r * NT;
    vpre[r] = R(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) qpre[r][d] = R(0);
    if (it < NFI) {
      const int j = it % NFN, f = (it / NFN) % NF, el = it / (NFN * NF);
      if (el < ne) {
        const int nb = a.nbr[(size_t)(e0 + el) * NF + f];
        if (nb >= 0) {
          const int node = sim_nbr_node<EL>(a, a.nbf[(size_t)(e0 + el) * NF + f], j);
          vpre[r] = R(v[(size_t)nb * NPE + node]);
#pragma unroll
          for (int d = 0; d < DIM; ++d) qpre[r][d] = R(q[((size_t)nb * DIM + d) * NPE + node]);
          hasnb |= 1 << r;
        }
      }
    }
  }
  R vn = R(0), qn[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) qn[d] = R(0);
  if (own) {
    vn = R(v[(size_t)(e0 + e) * NPE + n]);
#pragma unroll
    for (int d = 0; d < DIM; ++d) qn[d] = R(q[((size_t)(e0 + e) * DIM + d) * NPE + n]);
    Vs[e][n] = vn;
#pragma unroll
    for (int d = 0; d < DIM; ++d) Qs[e][d][n] = qn[d];
  }
  __syncthreads();
  // nodal fluxes; sJ fhat = tau sJ (v- - v+) + kappa/2 sJ (q- + q+).n + sJ beta.n v_upwind
  // at the face nodes (Dirichlet faces: v+ = 0, q+ = q-, no inflow)
  if (own) {
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      A s = CONV ? A(Ak[e][k][DIM] * vn) : A(0);
#pragma unroll
      for (int d = 0; d < DIM; ++d) s += Ak[e][k][d] * qn[d];
      Gk[e][k][n] = R(s);
    }
  }
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    const int it = t + r * NT;
    if (it >= NFI) break;
    const int j = it % NFN, f = (it / NFN) % NF, el = it / (NFN * NF);
    if (el >= ne) continue;
    const int node = EL::face_node(f, j);
    const R* fc = FC[el][f];
    const bool nb = (hasnb >> r) & 1;
    const R vm = Vs[el][node];
    A s = A(fc[DIM] * (vm - vpre[r]));
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const R qm = Qs[el][d][node];
      s += fc[d] * (qm + (nb ? qpre[r][d] : qm));
    }
    if (CONV) s += fc[DIM + 1] * (fc[DIM + 1] >= R(0) ? vm : vpre[r]);
    FF[el][f][j] = R(s);
  }
  __syncthreads();
  // face-mass moments of the fluxes; volume terms of the residual
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    const int it = t + r * NT;
    if (it >= NFI) break;
    const int j = it % NFN, f = (it / NFN) % NF, el = it / (NFN * NF);
    if (el >= ne) continue;
    const R* row = ops + O::MF + j * O::LDL;
    A s = A(0);
#pragma unroll
    for (int b = 0; b < NFN; ++b) s += row[b] * FF[el][f][b];
    FM[el][f][j] = R(s);
  }
  A r = A(0);
  if (own) {
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const R* row = ops + O::C + (k * NPE + n) * O::LDA;
#pragma unroll 8
      for (int m = 0; m < NPE; ++m) r -= row[m] * Gk[e][k][m];
    }
    if (tterm) {
      const R* row = ops + O::M + n * O::LDA;
      A h = A(0);
#pragma unroll 8
      for (int m = 0; m < NPE; ++m) h += row[m] * Vs[e][m];
      r += DJ[e] * R(h);
    }
  }
  __syncthreads();
  if (!own) return;
  for_node_faces<EL>(n, [&](int f, int j) { r += FM[e][f][j]; });
  ((double*)a.out)[(size_t)(e0 + e) * NPE + n] = (double)R(r);
}

template <class EL, bool CONV, class R, class QT>
cudaError_t launch_sim(const KArgs& a, void* qbuf, cudaStream_t s) {
  typedef SimShape<EL> S;
  constexpr size_t smem = SimOff<EL>::SIZE * sizeof(R);
  static const cudaError_t at1 =
      cudaFuncSetAttribute(k_sim_q<EL, R, QT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  static const cudaError_t at2 =
      cudaFuncSetAttribute(k_sim_r<EL, CONV, R, QT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (at1 != cudaSuccess) return at1;
  if (at2 != cudaSuccess) return at2;
  if (a.E <= 0) return cudaSuccess;
  const int grid = (a.E + S::NE - 1) / S::NE;
  KArgs b = a;
  b.out = qbuf;
  k_sim_q<EL, R, QT><<<grid, S::NT, smem, s>>>(b);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  b = a;
  b.q = qbuf;
  k_sim_r<EL, CONV, R, QT><<<grid, S::NT, smem, s>>>(b);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ldg
