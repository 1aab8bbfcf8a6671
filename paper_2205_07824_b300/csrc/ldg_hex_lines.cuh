// The nodal J.v of the linear models on affine hexahedra (the operator of ldg_linear.cuh)
// with one thread per node LINE instead of one per node.
//
// Thread (a, b) of an element owns three lines of its N1^3 nodes: the x-line
// (i1, i2) = (a, b), the y-line (i0, i2) = (a, b) and the z-line (i0, i1) = (a, b). The
// endpoints of these three lines are the element's face nodes with face index
// j = a + N1 b on all six faces (the face index of face 2k + s runs over the free axes in
// ascending order), so the thread that gathers a face node's neighbour value is the
// thread that needs it. Every 1-D contraction is done by the line's owner with the line
// in registers: N1 loads give N1 outputs, where one thread per node loads N1 values for
// one output. The 1-D operators (Dn, M1, C, L0, Lp) travel as a kernel parameter, so
// with the loops unrolled every coefficient is a constant-bank operand of its FMA and
// costs no load at all.
//
// q-stage (Eq. 1a): g_k = D_k v + L0(i_k) Delta_{2k} - Lp(i_k) Delta_{2k+1} on the
//   owner's k-line, then q_d = -sum_k Jinv[k][d] g_k per node.
// residual (Eq. 1b): with g_k = sum_d Ak[k][d] q_d + Ak[k][3] v per node,
//   R = -[M_z (M_y X + M_x Y) + M_x M_y Z],
//   X = C_x g0 - E_x Fhat_x - M_x h,  Y = C_y g1 - E_y Fhat_y,  Z = C_z g2 - E_z Fhat_z,
// h = a0/dt det J v (the BDF mass term) and E_k Fhat_k the flux sJ fhat of the two faces
// of axis k placed at the ends of the axis-k lines: the face mass sJ (M1 x M1) acts on
// the two free axes of the face, which the volume passes after C supply. So
//   phase 1: X on the x-lines, Y on the y-lines, Z on the z-lines (C, then the face fluxes
//            at the line's two ends, the thread's own six face nodes);
//   phase 2: X <- M_y X (y-lines), Y <- M_x Y (x-lines), Z <- M_x Z (x-lines);
//   phase 3: r = M_z (X + Y) on the z-line into registers, Z <- M_y Z (y-lines);
//   store: R = -(r + Z) on the z-line.
// Each phase updates its lines in place: a line is read and written by one thread only.
// Axis-aligned boxes take the trace form of ldg_linear.cuh in this layout
// (k_hex_qt, k_hex_rt below).
#pragma once
#include "ldg_linear.cuh"

namespace ldg {

template <int N1, class R> struct HexCoef {
  R dn[N1 * N1], m1[N1 * N1], c[N1 * N1], l0[N1], lp[N1];
  R cd[N1 * N1], cl0[N1], clp[N1];   // C Dn, C L0, C Lp (the trace form for boxes)
};

// Elements per CTA: up to 256 threads (FP32) or 128 (8-byte values), so that the
// static shared memory stays within 48 KB (34 KB at p = 4 either way).
template <int N1, class R> struct HexShape {
  static constexpr int NPE = N1 * N1 * N1, NL = N1 * N1, NF = 6;
  static constexpr int NE = (sizeof(R) == 4 ? 256 : 128) / NL > 0 ? (sizeof(R) == 4 ? 256 : 128) / NL : 1;
  static constexpr int NT = (NE * NL + 31) / 32 * 32;
  static constexpr int GEO = Geo<3>::size(NF);
};
// Resident CTAs asked of the register allocator. FP32 q-stage: eight (32 registers a
// thread, no spills), every warp slot for its gathers. FP32 residual: six (40 registers).
// Float pairs: five, which leaves 102 registers with 8-byte values, enough for the lines
// and the prefetched neighbour values without spills (measured on 48^3, p = 4: six CTAs
// spill and are 6% slower, four are 6% slower).
template <class R, bool QSTAGE> struct HexMinBlocks {
  static constexpr int value = sizeof(R) == 4 ? (QSTAGE ? 8 : 6) : 5;
};
// The trace-form residual of boxes (k_hex_rt) holds its line, the C and C Dn sums and the
// six face values in phase 1: five CTAs (48 registers in FP32, 96 in float pairs).
constexpr int kHexTraceMinBlocks = 5;

// the neighbour's local node of face node j on this element's face f
template <int N1> __device__ __forceinline__ int hex_nbr_node(const KArgs& a, int code, int j) {
  return lin_face_node<3, N1>(code & 7, a.perm[(code >> 3) * (N1 * N1) + j]);
}

// y[i] = sum_m A[i][m] x[m] (+ y[i] when ACC), A a parameter-space N1 x N1 matrix
template <int N1, class R, bool ACC> __device__ __forceinline__ void hex_apply(const R* A, const R* x, R* y) {
  typedef typename AccOf<R>::type Acc;
#pragma unroll
  for (int i = 0; i < N1; ++i) {
    Acc s = ACC ? Acc(y[i]) : Acc(0);
#pragma unroll
    for (int m = 0; m < N1; ++m) s += A[i * N1 + m] * x[m];
    y[i] = R(s);
  }
}

// ------------------------------------------------------------------ q-stage
template <int N1, class R, class QT>
__global__ void __launch_bounds__(HexShape<N1, R>::NT, (HexMinBlocks<R, true>::value)) k_hex_q(KArgs a, HexCoef<N1, R> P) {
  typedef HexShape<N1, R> S;
  typedef Geo<3> G;
  constexpr int NPE = S::NPE, NL = S::NL, NE = S::NE, NT = S::NT, GEO = S::GEO;
  typedef typename AccOf<R>::type A;
  if (a.skip && *a.skip) return;
  const int e0 = blockIdx.x * NE;
  const int ne = min(NE, a.E - e0);
  if (!cta_active(a, e0, ne)) return;
  __shared__ R Gs[NE][GEO];
  __shared__ R Vs[NE][NPE];
  __shared__ R Gk[3][NE][NPE];
  const int t = threadIdx.x;
  const int e = t / NL, l = t - e * NL, ia = l % N1, ib = l / N1;
  const bool own = e < ne;
  const double* v = (const double*)a.u;
  // the neighbours' values at this thread's six face nodes (face index ia + N1 ib),
  // loaded first so that their latency overlaps the element's own loads
  const int jf = ia + N1 * ib;
  R vnb[6];
  int hasnb = 0;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    vnb[f] = R(0);
    if (own) {
      const int nb = a.nbr[(size_t)(e0 + e) * 6 + f];
      if (nb >= 0) {
        vnb[f] = R(v[(size_t)nb * NPE + hex_nbr_node<N1>(a, a.nbf[(size_t)(e0 + e) * 6 + f], jf)]);
        hasnb |= 1 << f;
      }
    }
  }
  for (int i = t; i < ne * GEO; i += NT) Gs[i / GEO][i % GEO] = R(a.geo[(size_t)e0 * GEO + i]);
  for (int i = t; i < ne * NPE; i += NT) Vs[i / NPE][i % NPE] = R(v[(size_t)e0 * NPE + i]);
  __syncthreads();
  if (own) {
    // line k of this thread (one loop body for the three axes)
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
      const int base = k == 0 ? N1 * ia + NL * ib : (k == 1 ? ia + NL * ib : ia + N1 * ib);
      const int str = k == 0 ? 1 : (k == 1 ? N1 : NL);
      R x[N1], g[N1];
#pragma unroll
      for (int m = 0; m < N1; ++m) x[m] = Vs[e][base + m * str];
      // Delta = v- - vhat at the line's two ends (faces 2k and 2k + 1)
      R d0 = x[0], d1 = x[N1 - 1];
      const R vlo = k == 0 ? vnb[0] : (k == 1 ? vnb[2] : vnb[4]);
      const R vhi = k == 0 ? vnb[1] : (k == 1 ? vnb[3] : vnb[5]);
      if ((hasnb >> (2 * k)) & 1) d0 = (d0 - vlo) * R(0.5);
      if ((hasnb >> (2 * k + 1)) & 1) d1 = (d1 - vhi) * R(0.5);
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        A s = A(P.l0[i] * d0);
        s -= P.lp[i] * d1;
#pragma unroll
        for (int m = 0; m < N1; ++m) s += P.dn[i * N1 + m] * x[m];
        g[i] = R(s);
      }
#pragma unroll
      for (int i = 0; i < N1; ++i) Gk[k][e][base + i * str] = g[i];
    }
  }
  __syncthreads();
  // q_d = -sum_k Jinv[k][d] g_k, node by node (coalesced stores)
  QT* q = (QT*)a.out;
  for (int i = t; i < ne * NPE; i += NT) {
    const int el = i / NPE, n = i - el * NPE;
    const R g0 = Gk[0][el][n], g1 = Gk[1][el][n], g2 = Gk[2][el][n];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      A s = A(0);
      s -= Gs[el][G::JINV + d] * g0;
      s -= Gs[el][G::JINV + 3 + d] * g1;
      s -= Gs[el][G::JINV + 6 + d] * g2;
      q[((size_t)(e0 + el) * 3 + d) * NPE + n] = QT(R(s));
    }
  }
}

// ----------------------------------------------------------------- residual
template <int N1, bool CONV, class R, class QT>
__global__ void __launch_bounds__(HexShape<N1, R>::NT, (HexMinBlocks<R, false>::value)) k_hex_r(KArgs a, HexCoef<N1, R> P) {
  typedef HexShape<N1, R> S;
  typedef Geo<3> G;
  constexpr int NPE = S::NPE, NL = S::NL, NE = S::NE, NT = S::NT, GEO = S::GEO;
  typedef typename AccOf<R>::type A;
  if (a.skip && *a.skip) return;
  const int e0 = blockIdx.x * NE;
  const int ne = min(NE, a.E - e0);
  if (!cta_active(a, e0, ne)) return;
  __shared__ R Ak[NE][3][4];       // g_k = sum_d Ak[k][d] q_d + Ak[k][3] v
  __shared__ R FC[NE][6][5];       // per face: kappa/2 sJ n_d, tau sJ, sJ beta.n
  __shared__ R DJ[NE];             // a0/dt det J
  __shared__ R Gk[3][NE][NPE];     // g_k, then X, Y, Z in place
  __shared__ R Vs[NE][NPE];        // v
  __shared__ R Qs[NE][3][NPE];     // q
  const int t = threadIdx.x;
  const int e = t / NL, l = t - e * NL, ia = l % N1, ib = l / N1;
  const bool own = e < ne;
  const double* v = (const double*)a.u;
  const QT* q = (const QT*)a.q;
  // neighbours' v and q at this thread's six face nodes (the ends of its x-, y- and
  // z-lines, face index ia + N1 ib), loaded first
  const int jf = ia + N1 * ib;
  R vnb[6], qnb[6][3];
  int hasnb = 0;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    vnb[f] = R(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) qnb[f][d] = R(0);
    if (own) {
      const int nb = a.nbr[(size_t)(e0 + e) * 6 + f];
      if (nb >= 0) {
        const int node = hex_nbr_node<N1>(a, a.nbf[(size_t)(e0 + e) * 6 + f], jf);
        vnb[f] = R(v[(size_t)nb * NPE + node]);
#pragma unroll
        for (int d = 0; d < 3; ++d) qnb[f][d] = R(q[((size_t)nb * 3 + d) * NPE + node]);
        hasnb |= 1 << f;
      }
    }
  }
  for (int i = t; i < ne * 3; i += NT) {
    const int el = i / 3, k = i % 3;
    const double* g = a.geo + (size_t)(e0 + el) * GEO;
    const ModelParams mp = elem_mp(a, e0 + el);
    double bsum = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double jd = g[G::DETJ] * g[G::JINV + k * 3 + d];
      Ak[el][k][d] = R(mp.kappa * jd);
      bsum += jd * mp.beta[d];
    }
    Ak[el][k][3] = CONV ? R(bsum) : R(0);
  }
  for (int i = t; i < ne * 6; i += NT) {
    const int el = i / 6, f = i % 6;
    const double* g = a.geo + (size_t)(e0 + el) * GEO + G::FACE + f * 4;
    const ModelParams mp = elem_mp(a, e0 + el);
    const double sj = g[3];
    double bn = 0.0;
    for (int d = 0; d < 3; ++d) {
      FC[el][f][d] = R(0.5 * mp.kappa * sj * g[d]);
      bn += mp.beta[d] * g[d];
    }
    FC[el][f][3] = R(mp.tau * sj);
    FC[el][f][4] = CONV ? R(sj * bn) : R(0);
  }
  const bool tterm = a.a0dt != 0.0;
  for (int i = t; i < ne; i += NT) DJ[i] = R(a.a0dt * a.geo[(size_t)(e0 + i) * GEO + G::DETJ]);
  __syncthreads();
  // the part of sJ fhat at each of the six face nodes that does not depend on the own v:
  //   kappa/2 sJ q+.n - tau sJ v+ + (sJ beta.n v+ on inflow)
  // (Dirichlet faces: v+ = 0 and q+ = q-; the q- term joins in phase 1)
  R np[6];
  if (own) {
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const R* fc = FC[e][f];
      A s = A(0);
#pragma unroll
      for (int d = 0; d < 3; ++d) s += fc[d] * qnb[f][d];
      s -= fc[3] * vnb[f];
      if (CONV && !(fc[4] >= R(0))) s += fc[4] * vnb[f];
      np[f] = R(s);
    }
  }
  // nodal fluxes g_k and v (and q on general elements), node by node (coalesced loads)
  for (int i = t; i < ne * NPE; i += NT) {
    const int el = i / NPE, n = i - el * NPE;
    const R vn = R(v[(size_t)(e0 + el) * NPE + n]);
    R qn[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) qn[d] = R(q[((size_t)(e0 + el) * 3 + d) * NPE + n]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      A s = CONV ? A(Ak[el][k][3] * vn) : A(0);
#pragma unroll
      for (int d = 0; d < 3; ++d) s += Ak[el][k][d] * qn[d];
      Gk[k][el][n] = R(s);
    }
    Vs[el][n] = vn;
#pragma unroll
    for (int d = 0; d < 3; ++d) Qs[el][d][n] = qn[d];
  }
  __syncthreads();
  // ---- phase 1: C on the thread's k-line of g_k, then -sJ fhat at its two ends:
  //   sJ fhat = tau sJ (v- - v+) + kappa/2 sJ (q- + q+).n + sJ beta.n v_upwind
  // (Dirichlet faces: v+ = 0, q+ = q-, no inflow); X also takes -M_x h
  if (own) {
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
      const int base = k == 0 ? N1 * ia + NL * ib : (k == 1 ? ia + NL * ib : ia + N1 * ib);
      const int str = k == 0 ? 1 : (k == 1 ? N1 : NL);
      R x[N1], y[N1];
#pragma unroll
      for (int m = 0; m < N1; ++m) x[m] = Gk[k][e][base + m * str];
      hex_apply<N1, R, false>(P.c, x, y);
      if (k == 0 && tterm) {
#pragma unroll
        for (int m = 0; m < N1; ++m) x[m] = R(-(DJ[e] * Vs[e][base + m]));
        hex_apply<N1, R, true>(P.m1, x, y);
      }
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const int f = 2 * k + sd, node = base + sd * (N1 - 1) * str;
        const R* fc = FC[e][f];
        const R vm = Vs[e][node];
        A fs = A(fc[3] * vm);
        fs += k == 0 ? np[sd] : (k == 1 ? np[2 + sd] : np[4 + sd]);
        A qs = A(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) qs += fc[d] * Qs[e][d][node];
        const R qm = R(qs);
        fs += qm;
        fs += ((hasnb >> f) & 1) ? R(0) : qm;
        if (CONV) fs += fc[4] * (fc[4] >= R(0) ? vm : R(0));
        y[sd ? N1 - 1 : 0] -= R(fs);
      }
#pragma unroll
      for (int i = 0; i < N1; ++i) Gk[k][e][base + i * str] = y[i];
    }
  }
  __syncthreads();
  // ---- phase 2: X <- M_y X, Y <- M_x Y, Z <- M_x Z
  if (own) {
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
      const int base = k == 0 ? ia + NL * ib : N1 * ia + NL * ib;
      const int str = k == 0 ? N1 : 1;
      R x[N1], y[N1];
#pragma unroll
      for (int m = 0; m < N1; ++m) x[m] = Gk[k][e][base + m * str];
      hex_apply<N1, R, false>(P.m1, x, y);
#pragma unroll
      for (int i = 0; i < N1; ++i) Gk[k][e][base + i * str] = y[i];
    }
  }
  __syncthreads();
  // ---- phase 3: r = M_z (X + Y) on the z-line (ia, ib); Z <- M_y Z on the y-line
  const int bz = ia + N1 * ib;
  R r[N1];
  if (own) {
    R x[N1], y[N1];
#pragma unroll
    for (int m = 0; m < N1; ++m) x[m] = Gk[0][e][bz + NL * m] + Gk[1][e][bz + NL * m];
    hex_apply<N1, R, false>(P.m1, x, r);
    const int by = ia + NL * ib;
#pragma unroll
    for (int m = 0; m < N1; ++m) x[m] = Gk[2][e][by + N1 * m];
    hex_apply<N1, R, false>(P.m1, x, y);
#pragma unroll
    for (int i = 0; i < N1; ++i) Gk[2][e][by + N1 * i] = y[i];
  }
  __syncthreads();
  if (!own) return;
  double* out = (double*)a.out + (size_t)(e0 + e) * NPE + bz;
#pragma unroll
  for (int i = 0; i < N1; ++i) out[NL * i] = (double)(-(r[i] + Gk[2][e][bz + NL * i]));
}

// ---------------------------------------------- axis-aligned boxes: trace form
// The operator of k_lin_qt / k_lin_rt (ldg_linear.cuh) in the line layout. The q-stage
// forms q_k at the thread's six face nodes only, from its own three lines: the ends of
// the axis-k line are the nodes of faces 2k and 2k + 1, so rows 0 and p of D_k and the
// two trace jumps of that line give them. The residual applies
//   C_k g_k = b_k C v - a_k s_k (C Dn v + (C L0) Delta_{2k} - (C Lp) Delta_{2k+1})
// on the thread's axis-k line of v (no nodal flux loop), then the M1 passes of k_hex_r.
template <int N1, class R, class QT>
__global__ void __launch_bounds__(HexShape<N1, R>::NT, (HexMinBlocks<R, true>::value)) k_hex_qt(KArgs a, HexCoef<N1, R> P) {
  typedef HexShape<N1, R> S;
  typedef Geo<3> G;
  constexpr int NPE = S::NPE, NL = S::NL, NE = S::NE, NT = S::NT, GEO = S::GEO;
  typedef typename AccOf<R>::type A;
  if (a.skip && *a.skip) return;
  const int e0 = blockIdx.x * NE;
  const int ne = min(NE, a.E - e0);
  if (!cta_active(a, e0, ne)) return;
  __shared__ R SK[NE][3];          // -Jinv[k][k]
  __shared__ R Vs[NE][NPE];
  const int t = threadIdx.x;
  const int e = t / NL, l = t - e * NL, ia = l % N1, ib = l / N1;
  const bool own = e < ne;
  const double* v = (const double*)a.u;
  const int jf = ia + N1 * ib;
  R vnb[6];
  int hasnb = 0;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    vnb[f] = R(0);
    if (own) {
      const int nb = a.nbr[(size_t)(e0 + e) * 6 + f];
      if (nb >= 0) {
        vnb[f] = R(v[(size_t)nb * NPE + hex_nbr_node<N1>(a, a.nbf[(size_t)(e0 + e) * 6 + f], jf)]);
        hasnb |= 1 << f;
      }
    }
  }
  for (int i = t; i < ne * 3; i += NT) SK[i / 3][i % 3] = R(-a.geo[(size_t)(e0 + i / 3) * GEO + G::JINV + (i % 3) * 4]);
  for (int i = t; i < ne * NPE; i += NT) Vs[i / NPE][i % NPE] = R(v[(size_t)e0 * NPE + i]);
  __syncthreads();
  if (!own) return;
  QT* qt = (QT*)a.out + (size_t)(e0 + e) * 6 * NL + jf;
#pragma unroll 1
  for (int k = 0; k < 3; ++k) {
    const int base = k == 0 ? N1 * ia + NL * ib : (k == 1 ? ia + NL * ib : ia + N1 * ib);
    const int str = k == 0 ? 1 : (k == 1 ? N1 : NL);
    R x[N1];
#pragma unroll
    for (int m = 0; m < N1; ++m) x[m] = Vs[e][base + m * str];
    // Delta = v- - vhat at the line's two ends (faces 2k and 2k + 1)
    R d0 = x[0], d1 = x[N1 - 1];
    const R vlo = k == 0 ? vnb[0] : (k == 1 ? vnb[2] : vnb[4]);
    const R vhi = k == 0 ? vnb[1] : (k == 1 ? vnb[3] : vnb[5]);
    if ((hasnb >> (2 * k)) & 1) d0 = (d0 - vlo) * R(0.5);
    if ((hasnb >> (2 * k + 1)) & 1) d1 = (d1 - vhi) * R(0.5);
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      const int i = sd ? N1 - 1 : 0;
      A g = A(P.l0[i] * d0);
      g -= P.lp[i] * d1;
#pragma unroll
      for (int m = 0; m < N1; ++m) g += P.dn[i * N1 + m] * x[m];
      qt[(2 * k + sd) * NL] = QT(R(SK[e][k] * R(g)));
    }
  }
}

template <int N1, bool CONV, class R, class QT>
__global__ void __launch_bounds__(HexShape<N1, R>::NT, kHexTraceMinBlocks) k_hex_rt(KArgs a, HexCoef<N1, R> P) {
  typedef HexShape<N1, R> S;
  typedef Geo<3> G;
  constexpr int NPE = S::NPE, NL = S::NL, NE = S::NE, NT = S::NT, GEO = S::GEO;
  typedef typename AccOf<R>::type A;
  if (a.skip && *a.skip) return;
  const int e0 = blockIdx.x * NE;
  const int ne = min(NE, a.E - e0);
  if (!cta_active(a, e0, ne)) return;
  // FP32 applies C and C Dn to the line as constant-bank operands and scales the two sums
  // by b_k and a_k s_k; float pairs, whose products cost a dozen instructions each, build
  // W_k once per element in shared memory and apply that (measured: FP32 0.19 against
  // 0.26 ms, float pairs 0.62 against 0.74 ms for the residual on 48^3, p = 4)
  constexpr bool WS = !std::is_same<R, float>::value;
  __shared__ R AB[NE][3][2];       // a_k s_k, b_k
  __shared__ R W[WS ? NE : 1][3][N1 * N1];  // W_k = b_k C - a_k s_k (C Dn)
  __shared__ R WL[WS ? NE : 1][3][2][N1];   // -a_k s_k (C L0), +a_k s_k (C Lp)
  __shared__ R FC[NE][6][3];       // per face: kappa/2 sJ n_k, tau sJ, sJ beta.n
  __shared__ R DJ[NE];             // a0/dt det J
  __shared__ R Gk[3][NE][NPE];     // X, Y, Z in place
  __shared__ R Vs[NE][NPE];
  const int t = threadIdx.x;
  const int e = t / NL, l = t - e * NL, ia = l % N1, ib = l / N1;
  const bool own = e < ne;
  const double* v = (const double*)a.u;
  const QT* qt = (const QT*)a.q;
  // the own q_k and the neighbour's v and q_k at this thread's six face nodes
  const int jf = ia + N1 * ib;
  R vnb[6], qnb[6], qown[6];
  int hasnb = 0;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    vnb[f] = R(0);
    qnb[f] = R(0);
    qown[f] = R(0);
    if (own) {
      qown[f] = R(qt[((size_t)(e0 + e) * 6 + f) * NL + jf]);
      const int nb = a.nbr[(size_t)(e0 + e) * 6 + f];
      if (nb >= 0) {
        const int code = a.nbf[(size_t)(e0 + e) * 6 + f];
        const int jn = a.perm[(code >> 3) * NL + jf];
        vnb[f] = R(v[(size_t)nb * NPE + lin_face_node<3, N1>(code & 7, jn)]);
        qnb[f] = R(qt[((size_t)nb * 6 + (code & 7)) * NL + jn]);
        hasnb |= 1 << f;
      }
    }
  }
  for (int i = t; i < ne * 3; i += NT) {
    const int el = i / 3, k = i % 3;
    const double* g = a.geo + (size_t)(e0 + el) * GEO;
    const ModelParams mp = elem_mp(a, e0 + el);
    const double sk = g[G::JINV + k * 4], dj = g[G::DETJ];
    const double bk = k == 0 ? mp.beta[0] : (k == 1 ? mp.beta[1] : mp.beta[2]);
    AB[el][k][0] = R(mp.kappa * dj * sk * sk);
    AB[el][k][1] = CONV ? R(dj * sk * bk) : R(0);
  }
  for (int i = t; i < ne * 6; i += NT) {
    const int el = i / 6, f = i % 6, k = f >> 1;
    const double* g = a.geo + (size_t)(e0 + el) * GEO + G::FACE + f * 4;
    const ModelParams mp = elem_mp(a, e0 + el);
    const double bk = k == 0 ? mp.beta[0] : (k == 1 ? mp.beta[1] : mp.beta[2]);
    const double nk = k == 0 ? g[0] : (k == 1 ? g[1] : g[2]);
    FC[el][f][0] = R(0.5 * mp.kappa * g[3] * nk);
    FC[el][f][1] = R(mp.tau * g[3]);
    FC[el][f][2] = CONV ? R(g[3] * bk * nk) : R(0);
  }
  const bool tterm = a.a0dt != 0.0;
  for (int i = t; i < ne; i += NT) DJ[i] = R(a.a0dt * a.geo[(size_t)(e0 + i) * GEO + G::DETJ]);
  for (int i = t; i < ne * NPE; i += NT) Vs[i / NPE][i % NPE] = R(v[(size_t)e0 * NPE + i]);
  __syncthreads();
  // each element's W_k and lift coefficients (float pairs)
  if constexpr (WS) {
    for (int i = t; i < ne * 3 * N1 * N1; i += NT) {
      const int el = i / (3 * N1 * N1), k = (i / (N1 * N1)) % 3, c = i % (N1 * N1);
      const R as = AB[el][k][0], bk = AB[el][k][1];
      W[el][k][c] = bk * P.c[c] + (-(as * P.cd[c]));
      if (c < N1) {
        WL[el][k][0][c] = R(-(as * P.cl0[c]));
        WL[el][k][1][c] = R(as * P.clp[c]);
      }
    }
    __syncthreads();
  }
  // ---- phase 1: the axis-k line of v: W_k v + the lift of the trace jumps, then -sJ fhat
  // at its two ends (the part of the neighbour folded first):
  //   sJ fhat = tau sJ (v- - v+) + kappa/2 sJ (q- + q+)_k n_k + sJ beta.n v_upwind
  // (Dirichlet faces: v+ = 0, q+ = q-, no inflow); X also takes -M_x h
  if (own) {
    R np[6];
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const R* fc = FC[e][f];
      const bool nb = (hasnb >> f) & 1;
      A s = A(fc[0] * (qown[f] + (nb ? qnb[f] : qown[f])));
      s -= fc[1] * vnb[f];
      if (CONV && !(fc[2] >= R(0))) s += fc[2] * vnb[f];
      np[f] = R(s);
    }
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
      const int base = k == 0 ? N1 * ia + NL * ib : (k == 1 ? ia + NL * ib : ia + N1 * ib);
      const int str = k == 0 ? 1 : (k == 1 ? N1 : NL);
      R x[N1], y[N1];
#pragma unroll
      for (int m = 0; m < N1; ++m) x[m] = Vs[e][base + m * str];
      R d0 = x[0], d1 = x[N1 - 1];
      const R vlo = k == 0 ? vnb[0] : (k == 1 ? vnb[2] : vnb[4]);
      const R vhi = k == 0 ? vnb[1] : (k == 1 ? vnb[3] : vnb[5]);
      if ((hasnb >> (2 * k)) & 1) d0 = (d0 - vlo) * R(0.5);
      if ((hasnb >> (2 * k + 1)) & 1) d1 = (d1 - vhi) * R(0.5);
      if constexpr (WS) {
        const R* wk = W[e][k];
        const R* wl = WL[e][k][0];
#pragma unroll
        for (int i = 0; i < N1; ++i) {
          A u = A(wl[i] * d0);
          u += wl[N1 + i] * d1;
#pragma unroll
          for (int m = 0; m < N1; ++m) u += wk[i * N1 + m] * x[m];
          y[i] = R(u);
        }
      } else {
        const R as = AB[e][k][0], bk = AB[e][k][1];
#pragma unroll
        for (int i = 0; i < N1; ++i) {
          A u = A(0), w = A(P.cl0[i] * d0);
          w -= P.clp[i] * d1;
#pragma unroll
          for (int m = 0; m < N1; ++m) {
            u += P.c[i * N1 + m] * x[m];
            w += P.cd[i * N1 + m] * x[m];
          }
          y[i] = bk * R(u) + (-(as * R(w)));
        }
      }
      if (k == 0 && tterm) {
        R h[N1];
#pragma unroll
        for (int m = 0; m < N1; ++m) h[m] = R(-(DJ[e] * x[m]));
        hex_apply<N1, R, true>(P.m1, h, y);
      }
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const R* fc = FC[e][2 * k + sd];
        const R vm = sd ? x[N1 - 1] : x[0];
        A fs = A(fc[1] * vm);
        fs += k == 0 ? np[sd] : (k == 1 ? np[2 + sd] : np[4 + sd]);
        if (CONV) fs += fc[2] * (fc[2] >= R(0) ? vm : R(0));
        y[sd ? N1 - 1 : 0] -= R(fs);
      }
#pragma unroll
      for (int i = 0; i < N1; ++i) Gk[k][e][base + i * str] = y[i];
    }
  }
  __syncthreads();
  // ---- phase 2: X <- M_y X, Y <- M_x Y, Z <- M_x Z
  if (own) {
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
      const int base = k == 0 ? ia + NL * ib : N1 * ia + NL * ib;
      const int str = k == 0 ? N1 : 1;
      R x[N1], y[N1];
#pragma unroll
      for (int m = 0; m < N1; ++m) x[m] = Gk[k][e][base + m * str];
      hex_apply<N1, R, false>(P.m1, x, y);
#pragma unroll
      for (int i = 0; i < N1; ++i) Gk[k][e][base + i * str] = y[i];
    }
  }
  __syncthreads();
  // ---- phase 3: r = M_z (X + Y) on the z-line (ia, ib); Z <- M_y Z on the y-line
  const int bz = ia + N1 * ib;
  R r[N1];
  if (own) {
    R x[N1], y[N1];
#pragma unroll
    for (int m = 0; m < N1; ++m) x[m] = Gk[0][e][bz + NL * m] + Gk[1][e][bz + NL * m];
    hex_apply<N1, R, false>(P.m1, x, r);
    const int by = ia + NL * ib;
#pragma unroll
    for (int m = 0; m < N1; ++m) x[m] = Gk[2][e][by + N1 * m];
    hex_apply<N1, R, false>(P.m1, x, y);
#pragma unroll
    for (int i = 0; i < N1; ++i) Gk[2][e][by + N1 * i] = y[i];
  }
  __syncthreads();
  if (!own) return;
  double* out = (double*)a.out + (size_t)(e0 + e) * NPE + bz;
#pragma unroll
  for (int i = 0; i < N1; ++i) out[NL * i] = (double)(-(r[i] + Gk[2][e][bz + NL * i]));
}

// The 1-D operators of the blob (Dn, M1, C, L0, Lp; FP64) in the kernel's arithmetic.
template <int N1, class R> HexCoef<N1, R> hex_coef(const double* blob) {
  typedef LinOff<N1> O;
  HexCoef<N1, R> P;
  auto cv = [](double x) -> R {
    if constexpr (std::is_same<R, df>::value) {
      const float h = (float)x;
      return df(h, (float)(x - (double)h));
    } else {
      return R(x);
    }
  };
  for (int i = 0; i < N1 * N1; ++i) {
    P.dn[i] = cv(blob[O::DN + i]);
    P.m1[i] = cv(blob[O::M1 + i]);
    P.c[i] = cv(blob[O::C + i]);
  }
  for (int i = 0; i < N1; ++i) {
    P.l0[i] = cv(blob[O::L + i]);
    P.lp[i] = cv(blob[O::L + N1 + i]);
    P.cl0[i] = cv(blob[O::CL + i]);
    P.clp[i] = cv(blob[O::CL + N1 + i]);
  }
  for (int i = 0; i < N1 * N1; ++i) P.cd[i] = cv(blob[O::CD + i]);
  return P;
}

// Both stages of the hexahedral J.v: v -> q(v) in qbuf (QT), then J v.
template <int N1, bool CONV, class R, class QT, bool CART>
cudaError_t launch_hex(const KArgs& a, void* qbuf, cudaStream_t s) {
  typedef HexShape<N1, R> S;
  if (a.E <= 0) return cudaSuccess;
  if (!a.lops_host) return cudaErrorInvalidValue;
  const HexCoef<N1, R> P = hex_coef<N1, R>(a.lops_host);
  const int grid = (a.E + S::NE - 1) / S::NE;
  KArgs b = a;
  b.out = qbuf;
  if constexpr (CART) k_hex_qt<N1, R, QT><<<grid, S::NT, 0, s>>>(b, P);
  else k_hex_q<N1, R, QT><<<grid, S::NT, 0, s>>>(b, P);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  b = a;
  b.q = qbuf;
  if constexpr (CART) k_hex_rt<N1, CONV, R, QT><<<grid, S::NT, 0, s>>>(b, P);
  else k_hex_r<N1, CONV, R, QT><<<grid, S::NT, 0, s>>>(b, P);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ldg
