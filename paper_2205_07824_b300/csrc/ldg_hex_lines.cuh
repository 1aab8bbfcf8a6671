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
//   phase 1 (x-lines): T0 = C g0 - M h, T1 = M g1, T2 = M g2;
//   phase 2 (y-lines): U = M T0 + C T1, W = M T2;
//   phase 3 (z-lines): R = -(M U + C W) + the face moments of the line's nodes,
//   where h = a0/dt det J v (the BDF mass term). The face flux arrays sJ fhat are
//   contracted with M1 along their two free axes in the same phases, one face line per
//   thread (4 N1 lines a phase, so every thread of a warp does the same work).
// Each phase updates its lines in place: a line is read and written by one thread only.
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
// Resident CTAs asked of the register allocator: five, which leaves 51 registers a thread
// in FP32 and 102 with 8-byte values, enough for the lines and the prefetched neighbour
// values without spills (measured on 48^3, p = 4: six CTAs spill and are 12% slower in
// FP32, 6% in float pairs; four are 3% and 6% slower).
constexpr int kHexMinBlocks = 5;

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

// One of the 4 N1 face lines contracted with M1 in phase `ph` of the residual, in place
// in the element's face arrays FF[6][N1^2] (face index over the free axes, first fastest).
// Line fl: set fl / (2 N1), side (fl / N1) % 2, row or column fl % N1:
//   phase 1, along i0: rows of the y-faces (set 0) and of the z-faces (set 1);
//   phase 2, along i1: rows of the x-faces, columns of the z-faces;
//   phase 3, along i2: columns of the x-faces and of the y-faces.
// After the three phases each face array holds its moments sJ (M1 x M1) fhat.
template <int N1, class R> __device__ __forceinline__ void hex_face_line(const HexCoef<N1, R>& P, R (*FF)[N1 * N1],
                                                                        int ph, int fl) {
  const int set = fl / (2 * N1), side = (fl / N1) & 1, rc = fl % N1;
  int f, base, str;
  if (ph == 1) { f = (set ? 4 : 2) + side; base = N1 * rc; str = 1; }
  else if (ph == 2) { f = set ? 4 + side : side; base = set ? rc : N1 * rc; str = set ? N1 : 1; }
  else { f = (set ? 2 : 0) + side; base = rc; str = N1; }
  R* line = &FF[f][base];
  R x[N1], y[N1];
#pragma unroll
  for (int m = 0; m < N1; ++m) x[m] = line[m * str];
  hex_apply<N1, R, false>(P.m1, x, y);
#pragma unroll
  for (int i = 0; i < N1; ++i) line[i * str] = y[i];
}

// ------------------------------------------------------------------ q-stage
template <int N1, class R, class QT>
__global__ void __launch_bounds__(HexShape<N1, R>::NT, kHexMinBlocks) k_hex_q(KArgs a, HexCoef<N1, R> P) {
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
__global__ void __launch_bounds__(HexShape<N1, R>::NT, kHexMinBlocks) k_hex_r(KArgs a, HexCoef<N1, R> P) {
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
  __shared__ R Gk[3][NE][NPE];     // g_k, then the phase results in place
  __shared__ R Hs[NE][NPE];        // a0/dt det J v (time term)
  __shared__ R FF[NE][6][NL];      // own v at the face nodes, then sJ fhat, then its moments
  __shared__ R FQ[NE][6][NL];      // own kappa/2 sJ q.n at the face nodes
  const int t = threadIdx.x;
  const int e = t / NL, l = t - e * NL, ia = l % N1, ib = l / N1;
  const bool own = e < ne;
  const double* v = (const double*)a.u;
  const QT* q = (const QT*)a.q;
  // neighbours' v and q at this thread's six face nodes, loaded first
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
  // nodal fluxes g_k, the time term and the own face values, node by node (coalesced loads)
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
    if (tterm) Hs[el][n] = DJ[el] * vn;
    const int i0 = n % N1, i1 = (n / N1) % N1, i2 = n / NL;
    const int id[3] = {i0, i1, i2};
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int ax = f >> 1;
      if (id[ax] != ((f & 1) ? N1 - 1 : 0)) continue;
      const int j = lin_face_index<3, N1>(ax, id);
      A s = A(0);
#pragma unroll
      for (int d = 0; d < 3; ++d) s += FC[el][f][d] * qn[d];
      FF[el][f][j] = vn;
      FQ[el][f][j] = R(s);
    }
  }
  __syncthreads();
  // sJ fhat at this thread's six face nodes (in place of the own v)
  if (own) {
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const R* fc = FC[e][f];
      const R vm = FF[e][f][jf], qmn = FQ[e][f][jf], bs = fc[4];
      R fh;
      if ((hasnb >> f) & 1) {
        A qpn = A(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) qpn += fc[d] * qnb[f][d];
        fh = fc[3] * (vm - vnb[f]) + (qmn + R(qpn));
        if (CONV) fh += bs * (bs >= R(0) ? vm : vnb[f]);
      } else {
        fh = fc[3] * vm + R(2) * qmn;
        if (CONV && bs >= R(0)) fh += bs * vm;
      }
      FF[e][f][jf] = fh;
    }
  }
  __syncthreads();
  // ---- phases 1 and 2, one loop body (the face-line code once):
  //   phase 1: x-line (i1, i2) = (ia, ib): T0 = C g0 - M h, T1 = M g1, T2 = M g2;
  //   phase 2: y-line (i0, i2) = (ia, ib): U = M T0 + C T1, W = M T2;
  //   face lines along i0, then along i1
#pragma unroll 1
  for (int ph = 1; ph <= 2; ++ph) {
    if (own) {
      const int base = ph == 1 ? N1 * ia + NL * ib : ia + NL * ib;
      const int str = ph == 1 ? 1 : N1;
      R x[N1], y[N1];
      // field 0: C g0 (phase 1, with -M h when there is a time term) or M T0 + C T1 (phase 2)
#pragma unroll
      for (int i = 0; i < N1; ++i) y[i] = R(0);
      if (ph == 2 || tterm) {
        const R* src = ph == 1 ? Hs[e] : Gk[0][e];
#pragma unroll
        for (int m = 0; m < N1; ++m) x[m] = src[base + m * str];
        hex_apply<N1, R, false>(P.m1, x, y);
        if (ph == 1) {
#pragma unroll
          for (int i = 0; i < N1; ++i) y[i] = -y[i];
        }
      }
      const R* src = ph == 1 ? Gk[0][e] : Gk[1][e];
#pragma unroll
      for (int m = 0; m < N1; ++m) x[m] = src[base + m * str];
      hex_apply<N1, R, true>(P.c, x, y);
#pragma unroll
      for (int i = 0; i < N1; ++i) Gk[0][e][base + i * str] = y[i];
      // the fields that only take M: g1 and g2 (phase 1), T2 (phase 2)
#pragma unroll 1
      for (int k = ph == 1 ? 1 : 2; k < 3; ++k) {
#pragma unroll
        for (int m = 0; m < N1; ++m) x[m] = Gk[k][e][base + m * str];
        hex_apply<N1, R, false>(P.m1, x, y);
#pragma unroll
        for (int i = 0; i < N1; ++i) Gk[k][e][base + i * str] = y[i];
      }
      for (int fl = l; fl < 4 * N1; fl += NL) hex_face_line<N1, R>(P, FF[e], ph, fl);
    }
    __syncthreads();
  }
  // ---- phase 3: z-line (i0, i1) = (ia, ib) into registers; face lines along i2 (x- and
  // y-face columns), then the face moments on the line and the store
  const int bz = ia + N1 * ib;
  R r[N1];
  if (own) {
    R x0[N1], x1[N1];
#pragma unroll
    for (int m = 0; m < N1; ++m) {
      x0[m] = Gk[0][e][bz + NL * m];
      x1[m] = Gk[2][e][bz + NL * m];
    }
    hex_apply<N1, R, false>(P.m1, x0, r);
    hex_apply<N1, R, true>(P.c, x1, r);
    for (int fl = l; fl < 4 * N1; fl += NL) hex_face_line<N1, R>(P, FF[e], 3, fl);
  }
  __syncthreads();
  if (!own) return;
#pragma unroll
  for (int i = 0; i < N1; ++i) r[i] = -r[i];
  if (ia == 0 || ia == N1 - 1) {   // x-face moments at (ia, ib, i2)
    const R* fm = &FF[e][ia != 0][ib];
#pragma unroll
    for (int i = 0; i < N1; ++i) r[i] += fm[N1 * i];
  }
  if (ib == 0 || ib == N1 - 1) {   // y-face moments at (ia, ib, i2)
    const R* fm = &FF[e][2 + (ib != 0)][ia];
#pragma unroll
    for (int i = 0; i < N1; ++i) r[i] += fm[N1 * i];
  }
  // z-faces at the line's ends
  r[0] += FF[e][4][bz];
  r[N1 - 1] += FF[e][5][bz];
  double* out = (double*)a.out + (size_t)(e0 + e) * NPE + bz;
#pragma unroll
  for (int i = 0; i < N1; ++i) out[NL * i] = (double)r[i];
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
template <int N1, bool CONV, class R, class QT>
cudaError_t launch_hex(const KArgs& a, void* qbuf, cudaStream_t s) {
  typedef HexShape<N1, R> S;
  if (a.E <= 0) return cudaSuccess;
  if (!a.lops_host) return cudaErrorInvalidValue;
  const HexCoef<N1, R> P = hex_coef<N1, R>(a.lops_host);
  const int grid = (a.E + S::NE - 1) / S::NE;
  KArgs b = a;
  b.out = qbuf;
  k_hex_q<N1, R, QT><<<grid, S::NT, 0, s>>>(b, P);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  b = a;
  b.q = qbuf;
  k_hex_r<N1, CONV, R, QT><<<grid, S::NT, 0, s>>>(b, P);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ldg
