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
// CART (every element an axis-aligned box): the products with the zero entries of J^{-1}
// and of the face normals are left out, and only q along the face axis is gathered.
#pragma once
#include "ldg_linear.cuh"

namespace ldg {

template <int N1, class R> struct HexCoef {
  R dn[N1 * N1], m1[N1 * N1], c[N1 * N1], l0[N1], lp[N1];
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
template <int N1, class R, class QT, bool CART>
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
    if constexpr (CART) {
      q[((size_t)(e0 + el) * 3 + 0) * NPE + n] = QT(R(-(Gs[el][G::JINV] * g0)));
      q[((size_t)(e0 + el) * 3 + 1) * NPE + n] = QT(R(-(Gs[el][G::JINV + 4] * g1)));
      q[((size_t)(e0 + el) * 3 + 2) * NPE + n] = QT(R(-(Gs[el][G::JINV + 8] * g2)));
    } else {
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
}

// ----------------------------------------------------------------- residual
template <int N1, bool CONV, class R, class QT, bool CART>
__global__ void __launch_bounds__(HexShape<N1, R>::NT, (HexMinBlocks<R, false>::value)) k_hex_r(KArgs a, HexCoef<N1, R> P) {
  typedef HexShape<N1, R> S;
  typedef Geo<3> G;
  constexpr int NPE = S::NPE, NL = S::NL, NE = S::NE, NT = S::NT, GEO = S::GEO;
  constexpr int NQ = CART ? 1 : 3;   // components of q read at a face node
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
  __shared__ R Qs[CART ? 1 : NE][CART ? 1 : 3][CART ? 1 : NPE];   // q (general elements)
  const int t = threadIdx.x;
  const int e = t / NL, l = t - e * NL, ia = l % N1, ib = l / N1;
  const bool own = e < ne;
  const double* v = (const double*)a.u;
  const QT* q = (const QT*)a.q;
  // neighbours' v and q at this thread's six face nodes (the ends of its x-, y- and
  // z-lines, face index ia + N1 ib), loaded first; CART: also the own q along the face
  // axis at those nodes
  const int jf = ia + N1 * ib;
  R vnb[6], qnb[6][NQ], qown[6];
  int hasnb = 0;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    vnb[f] = R(0);
    qown[f] = R(0);
#pragma unroll
    for (int d = 0; d < NQ; ++d) qnb[f][d] = R(0);
    if (own) {
      if constexpr (CART) {
        const int node = lin_face_node<3, N1>(f, jf);
        qown[f] = R(q[((size_t)(e0 + e) * 3 + (f >> 1)) * NPE + node]);
      }
      const int nb = a.nbr[(size_t)(e0 + e) * 6 + f];
      if (nb >= 0) {
        const int node = hex_nbr_node<N1>(a, a.nbf[(size_t)(e0 + e) * 6 + f], jf);
        vnb[f] = R(v[(size_t)nb * NPE + node]);
#pragma unroll
        for (int d = 0; d < NQ; ++d)
          qnb[f][d] = R(q[((size_t)nb * 3 + (CART ? (f >> 1) : d)) * NPE + node]);
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
  //   kappa/2 sJ (q- + q+).n - tau sJ v+ + (sJ beta.n v+ on inflow)
  // (Dirichlet faces: v+ = 0 and q+ = q-; general elements: the q- term joins in phase 1)
  R np[6];
  if (own) {
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const R* fc = FC[e][f];
      const bool nb = (hasnb >> f) & 1;
      A s = A(0);
      if constexpr (CART) {
        s += fc[f >> 1] * (qown[f] + (nb ? qnb[f][0] : qown[f]));
      } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) s += fc[d] * qnb[f][d];
      }
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
      if constexpr (CART) {
        s += Ak[el][k][k] * qn[k];
      } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) s += Ak[el][k][d] * qn[d];
      }
      Gk[k][el][n] = R(s);
    }
    Vs[el][n] = vn;
    if constexpr (!CART) {
#pragma unroll
      for (int d = 0; d < 3; ++d) Qs[el][d][n] = qn[d];
    }
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
        if constexpr (!CART) {
          A qs = A(0);
#pragma unroll
          for (int d = 0; d < 3; ++d) qs += fc[d] * Qs[e][d][node];
          const R qm = R(qs);
          fs += qm;
          fs += ((hasnb >> f) & 1) ? R(0) : qm;
        }
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
  }
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
  k_hex_q<N1, R, QT, CART><<<grid, S::NT, 0, s>>>(b, P);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  b = a;
  b.q = qbuf;
  k_hex_r<N1, CONV, R, QT, CART><<<grid, S::NT, 0, s>>>(b, P);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ldg
