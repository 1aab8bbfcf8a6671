// Fused element-centric LDG stage kernels (Section 2.2, Eq. 1a-1b; Section 3.3).
//
// One CTA owns NE consecutive elements. Every stage is a loop of independent
// items over the CTA's threads, separated by __syncthreads, on data staged in
// shared memory. Each element evaluates both sides of its own faces (the
// neighbour's face-node values are read from global memory, normally an L2 hit),
// so no atomics are used and results are bitwise reproducible.
//
//   q-stage  : q_d = -d_d u_h + M^{-1} sum_f <(u- - uhat) n_d, phi>_f        (Eq. 1a)
//              (the weak form integrated by parts once; exact because the
//               quadrature integrates u d(phi) and the mass matrix exactly)
//   residual : R = -(f(u,q), grad phi) + <fhat.n, phi> - (s, phi) + M (a0 u + h)
//              with the BDF history h = (a1 u^n + a2 u^{n-1}) / dt          (Eq. 1b)
//
// MODE_R evaluates R(u); MODE_HOM the homogeneous linear part of a linear model
// (R(v) - R(0): no source, zero boundary data), which is its exact J.v; MODE_JV
// propagates dual numbers (u, v) through a nonlinear model and writes dR/du . v.
// A nonlinear model with q (Navier-Stokes) carries the dual pair (q(u), Q v) too:
// the q-stage is affine in u, so its derivative along v is the homogeneous q-stage
// Q v (zero boundary data), computed by the q-stage in MODE_HOM.
//
// Storage in HBM is always FP64. The compute type R is double (parity path) or
// float (the mixed-precision Krylov path): an FP32 instance converts its inputs
// on load, keeps operators, geometry and every intermediate in FP32, and widens
// its result on the store.
#pragma once
#include "ldg_device.cuh"

namespace ldg {

enum { MODE_R = 0, MODE_HOM = 1, MODE_JV = 2 };

// Tile shape of a kernel instance: the number of elements per CTA is the largest
// count whose shared-memory arrays fit the budget (bytes per CTA), at most NE_MAX.
// Smaller budgets give more, smaller CTAs per SM. Several tiles are compiled per
// (element, order, model) and the autotuner picks one per context.
template <int NEMAX, int BUDGET_R_, int BUDGET_Q_> struct Tile {
  static constexpr int NE_MAX = NEMAX, BUDGET_R = BUDGET_R_, BUDGET_Q = BUDGET_Q_;
};
typedef Tile<16, 100 * 1024, 96 * 1024> Tile0;   // default
typedef Tile<8, 48 * 1024, 48 * 1024> Tile1;
typedef Tile<32, 100 * 1024, 100 * 1024> Tile2;
typedef Tile<4, 24 * 1024, 24 * 1024> Tile3;
constexpr int N_TILES = 4;

struct KArgs {
  const void* u;              // [E][NCU][NPE]     state (R, JV) or direction (HOM)
  const void* v;              // [E][NCU][NPE]     direction (JV)
  const void* q;              // [E][NCU][DIM][NPE] q(u) (R, JV) or q(v) (HOM), models with q
  const void* dq;             // [E][NCU][DIM][NPE] Q v, the tangent of q (JV, nonlinear models with q)
  const void* hist;           // [E][NCU][NPE]     BDF history term, or null
  const double* radd;         // [E][NCU][NPE]     constant added to R in MODE_R (DIRK stage terms), or null
  void* out;                  // [E][NCU][NPE] residual / J.v, or [E][NCU][DIM][NPE] q
  const double* geo;          // [E][GEO] per-element affine geometry
  const double* cgeo;         // curved elements: [E][CGeo::SIZE] per-point metrics (FP64) ...
  const float* cgeof;         // ... and their FP32 copy
  const double* cx;           // curved: [E][CGeo::XSIZE] physical coordinates of volume and face points
  const double* minv;         // curved: [E][NPE][NPE] inverse element mass matrices (FP64) ...
  const float* minvf;         // ... and their FP32 copy
  const int* nbr;             // [E][NF] neighbour element; -1 data boundary face, -2 wall face
  const unsigned char* nbf;   // [E][NF] neighbour's local face | (orientation code << 3)
  const double* ops;          // reference operator blob (element traits), FP64
  const float* opsf;          // the same blob in FP32 (for FP32-compute instances)
  const unsigned char* perm;  // [n_orient][NFQ] face-point permutations
  const double* lops;         // 1-D operators of the nodal linear J.v kernels (ldg_linear.cuh), FP64 ...
  const float* lopsf;         // ... and FP32
  const double* lops_host;    // the same FP64 blob in host memory (launchers that pass the
                              // operators as a kernel parameter read it; kernels do not)
  float* q32_out;             // optional, MODE_R q-stage (FP64): FP32 copy of q(u) ...
  float* u32_out;             // ... and of u, read by the FP32 J.v of nonlinear models with q
  const int* skip;            // optional: the kernel returns at once when *skip != 0
  int blk_col;                // MODE_JV block extraction (models without q): -1 off; else the element's own tangent is
                              // unit vector blk_col, neighbours' tangents are zero, and column blk_col
                              // of each element's diagonal block dR_K/du_K is written to blk_out
  double* blk_out;            // [E][NLOC][NLOC] column-major blocks (NLOC = NCU * NPE)
  double a0dt;                // a0 / dt of the BDF scheme, 0 when steady
  double t;                   // time of the boundary data ...
  const double* t_dev;        // ... or, when set, read from device memory (graph replays)
  ModelParams mp;             // model parameters (all elements, unless inst is set)
  const int* inst;            // optional [E]: instance of each element (batched contexts) ...
  const ModelParams* mtab;    // ... indexing this per-instance parameter table
  const int* inst_skip;       // optional [n_inst]: a CTA whose elements all belong to instances
                              // with inst_skip != 0 returns at once (outputs left unchanged)
  int E;
};

// Model parameters of element e.
__device__ __forceinline__ ModelParams elem_mp(const KArgs& a, int e) { return a.inst ? a.mtab[a.inst[e]] : a.mp; }

// True when the CTA has at least one element of an instance that is not skipped
// (call from all threads; ne <= blockDim.x).
__device__ __forceinline__ bool cta_active(const KArgs& a, int e0, int ne) {
  if (!a.inst_skip) return true;
  const int act = (int)threadIdx.x < ne && !a.inst_skip[a.inst[e0 + threadIdx.x]];
  return __syncthreads_or(act) != 0;
}

// Per-element geometry record: Jinv[k][d] = d xi_k / d x_d, detJ, x(0), J[d][k] = d x_d / d xi_k,
// then for each face its unit outward normal and surface Jacobian.
template <int DIM> struct Geo {
  static constexpr int JINV = 0, DETJ = DIM * DIM, XM = DETJ + 1, JAC = XM + DIM, FACE = JAC + DIM * DIM;
  static constexpr int size(int nf) { return FACE + nf * (DIM + 1); }
};

// Per-element record of a curved element: at each volume point the metric
// w det J d xi_k / d x_d (k, d) and w det J; at each face point the outward unit
// normal and w sJ (reference face weight folded in). Physical coordinates of the
// volume and face points are a separate record (read only for data).
template <class EL> struct CGeo {
  static constexpr int DIM = EL::DIM, NV = DIM * DIM + 1, NFR = DIM + 1;
  static constexpr int VG = 0, FG = EL::NQV * NV, SIZE = FG + EL::NF * EL::NFQ * NFR;
  static constexpr int XV = 0, XF = EL::NQV * DIM, XSIZE = XF + EL::NF * EL::NFQ * DIM;
};
template <class EL> constexpr int geo_size() {
  if constexpr (EL::CURVED) return CGeo<EL>::SIZE;
  else return Geo<EL::DIM>::size(EL::NF);
}
// Geometry records in the kernel's compute precision.
template <class EL, class R> __device__ __forceinline__ const R* geo_src(const KArgs& a) {
  if constexpr (EL::CURVED) {
    if constexpr (sizeof(R) == 8) return (const R*)a.cgeo;
    else return (const R*)a.cgeof;
  } else {
    return nullptr;
  }
}

__host__ __device__ constexpr int al16(int b) { return (b + 15) & ~15; }

// Calls fn(f, j) for every face f that contains local node n, with j the node's
// index within that face. Written without dynamically indexed local arrays:
// nvcc 13.0 at -O3 mis-assigned the face ids of an earlier array-based form
// (correct at -G), so the enumeration is an unrolled loop of direct calls.
template <class EL, class F> __device__ __forceinline__ void for_node_faces(int n, F&& fn) {
  if constexpr (EL::TENSOR) {
    constexpr int N1 = EL::N1;
    const int i0 = n % N1, i1 = (n / N1) % N1, i2 = n / (N1 * N1);
    // axis 0: free axes (1, 2); axis 1: (0, 2); axis 2: (0, 1)
    if (i0 == 0) fn(0, i1 + N1 * i2);
    if (i0 == N1 - 1) fn(1, i1 + N1 * i2);
    if (i1 == 0) fn(2, i0 + N1 * i2);
    if (i1 == N1 - 1) fn(3, i0 + N1 * i2);
    if constexpr (EL::DIM == 3) {
      if (i2 == 0) fn(4, i0 + N1 * i1);
      if (i2 == N1 - 1) fn(5, i0 + N1 * i1);
    }
  } else if constexpr (EL::DIM == 2) {
    constexpr int P = EL::P;
    int j = 0, rem = n;
    while (rem > P - j) { rem -= P + 1 - j; ++j; }
    const int i = rem;
    if (j == 0) fn(0, i);
    if (i + j == P) fn(1, j);
    if (i == 0) fn(2, P - j);
  } else {
    // tetrahedron: node on face f when its barycentric coordinate l[f] is 0; its face
    // coordinates (a, b) are l[B], l[C] of the face's vertices (A, B, C)
    constexpr int P = EL::P;
    int l[4];
    EL::lattice(n, l);
    auto fidx = [](int a, int b) { return b * (P + 1) - b * (b - 1) / 2 + a; };
    if (l[0] == 0) fn(0, fidx(l[2], l[3]));
    if (l[1] == 0) fn(1, fidx(l[2], l[3]));
    if (l[2] == 0) fn(2, fidx(l[1], l[3]));
    if (l[3] == 0) fn(3, fidx(l[1], l[2]));
  }
}

// Neighbour traces: the neighbour's local node that carries face node j of this
// element's face, and the neighbour's face point that coincides with face point k.
// Elements with NODE_PERM permute the face nodes (the face points are then this
// element's own); the others permute the face points.
template <class EL> __device__ __forceinline__ int nbr_face_node(const KArgs& a, int nbf, int j) {
  if constexpr (EL::NODE_PERM) return EL::face_node(nbf & 7, a.perm[(nbf >> 3) * EL::NFN + j]);
  else return EL::face_node(nbf & 7, j);
}
template <class EL> __device__ __forceinline__ int nbr_face_point(const KArgs& a, int nbf, int k) {
  if constexpr (EL::NODE_PERM) return k;
  else return a.perm[(nbf >> 3) * EL::NFQ + k];
}

// Reference coordinates of face point k on face f.
template <class EL, class R> __device__ __forceinline__ void face_xi(const R* ops, int f, int k, R* xi) {
  if constexpr (EL::TENSOR) {
    const R* XQ = ops + EL::OXQ;
    const int ax = f >> 1;
    const R fix = (f & 1) ? R(1) : R(-1);
    if constexpr (EL::DIM == 2) {
      xi[ax] = fix;
      xi[1 - ax] = XQ[k];
    } else {
      // free axes in ascending order, the first one fastest
      const R s0 = XQ[k % EL::NQ], s1 = XQ[k / EL::NQ];
      if (ax == 0) { xi[0] = fix; xi[1] = s0; xi[2] = s1; }
      else if (ax == 1) { xi[0] = s0; xi[1] = fix; xi[2] = s1; }
      else { xi[0] = s0; xi[1] = s1; xi[2] = fix; }
    }
  } else if constexpr (EL::DIM == 2) {
    const R V[3][2] = {{R(-1), R(-1)}, {R(1), R(-1)}, {R(-1), R(1)}};
    const int a = f, b = (f + 1) % 3;
    const R s = ops[EL::OSF + k];
    xi[0] = R(0.5) * (R(1) - s) * V[a][0] + R(0.5) * (R(1) + s) * V[b][0];
    xi[1] = R(0.5) * (R(1) - s) * V[a][1] + R(0.5) * (R(1) + s) * V[b][1];
  } else {
    const R V[4][3] = {{R(-1), R(-1), R(-1)}, {R(1), R(-1), R(-1)}, {R(-1), R(1), R(-1)}, {R(-1), R(-1), R(1)}};
    int A, B, C;
    EL::face_verts(f, A, B, C);
    const R s = ops[EL::OSF + 2 * k], t = ops[EL::OSF + 2 * k + 1];
    for (int d = 0; d < 3; ++d)
      xi[d] = V[A][d] + R(0.5) * (R(1) + s) * (V[B][d] - V[A][d]) + R(0.5) * (R(1) + t) * (V[C][d] - V[A][d]);
  }
}
template <class EL, class R> __device__ __forceinline__ R face_w(const R* ops, int k) {
  if constexpr (EL::TENSOR) {
    const R* W = ops + EL::OW;
    return EL::DIM == 2 ? W[k] : W[k % EL::NQ] * W[k / EL::NQ];
  } else {
    return ops[EL::OWF + k];
  }
}
template <class EL, class R> __device__ __forceinline__ void vol_xi(const R* ops, int q, R* xi, R& w) {
  if constexpr (EL::TENSOR) {
    const R* XQ = ops + EL::OXQ;
    const R* W = ops + EL::OW;
    const int i0 = q % EL::NQ, i1 = (q / EL::NQ) % EL::NQ, i2 = q / (EL::NQ * EL::NQ);
    xi[0] = XQ[i0]; xi[1] = XQ[i1];
    w = W[i0] * W[i1];
    if constexpr (EL::DIM == 3) { xi[2] = XQ[i2]; w *= W[i2]; }
  } else {
    for (int d = 0; d < EL::DIM; ++d) xi[d] = ops[EL::OXQ + EL::DIM * q + d];
    w = ops[EL::OWV + q];
  }
}

template <int DIM, class R> __device__ __forceinline__ void phys_x(const R* g, const R* xi, double* x) {
  for (int d = 0; d < DIM; ++d) {
    double s = (double)g[Geo<DIM>::XM + d];
    for (int k = 0; k < DIM; ++k) s += (double)g[Geo<DIM>::JAC + d * DIM + k] * (double)xi[k];
    x[d] = s;
  }
}

// Outward unit normal (pointer to DIM values) and quadrature weight w sJ of face
// point k of face f; g is the element's geometry record.
template <class EL, class R>
__device__ __forceinline__ const R* face_frame(const R* g, const R* ops, int f, int k, R& w) {
  if constexpr (EL::CURVED) {
    const R* fr = g + CGeo<EL>::FG + (f * EL::NFQ + k) * CGeo<EL>::NFR;
    w = fr[EL::DIM];
    return fr;
  } else {
    const R* nrm = g + Geo<EL::DIM>::FACE + f * (EL::DIM + 1);
    w = face_w<EL>(ops, k) * nrm[EL::DIM];
    return nrm;
  }
}
// Physical coordinates of face point k of face f of element eg (global index).
template <class EL, class R>
__device__ __forceinline__ void face_phys(const KArgs& a, const R* g, const R* ops, int eg, int f, int k, double* x) {
  if constexpr (EL::CURVED) {
    const double* c = a.cx + (size_t)eg * CGeo<EL>::XSIZE + CGeo<EL>::XF + (f * EL::NFQ + k) * EL::DIM;
    for (int d = 0; d < EL::DIM; ++d) x[d] = c[d];
  } else {
    R xi[3];
    face_xi<EL>(ops, f, k, xi);
    phys_x<EL::DIM>(g, xi, x);
  }
}
// Physical coordinates of volume point q of element eg.
template <class EL, class R>
__device__ __forceinline__ void vol_phys(const KArgs& a, const R* g, const R* ops, int eg, int q, double* x) {
  if constexpr (EL::CURVED) {
    const double* c = a.cx + (size_t)eg * CGeo<EL>::XSIZE + CGeo<EL>::XV + q * EL::DIM;
    for (int d = 0; d < EL::DIM; ++d) x[d] = c[d];
  } else {
    R xi[3], w;
    vol_xi<EL>(ops, q, xi, w);
    phys_x<EL::DIM>(g, xi, x);
  }
}

// ---------------------------------------------- reference operators on batches
// face-node values [nb][NFN] -> face-point values [nb][NFQ]; tmp holds [nb][NQ*N1]
template <class EL, class T, class OT> __device__ __forceinline__ void face_trace(const T* in, T* out, T* tmp, const OT* ops, int nb) {
  if constexpr (EL::TENSOR) {
    const OT* B = ops + EL::OB;
    if constexpr (EL::DIM == 2) {
      contract<0, EL::N1, 1, 1, EL::NQ, false, false>(in, out, B, nb);
    } else {
      contract<0, EL::N1, EL::N1, 1, EL::NQ, false, false>(in, tmp, B, nb);
      __syncthreads();
      contract<1, EL::NQ, EL::N1, 1, EL::NQ, false, false>(tmp, out, B, nb);
    }
  } else {
    matvec<EL::NFQ, EL::NFN, false, false>(in, out, ops + EL::OBF, nb);
  }
}
// face-point values [nb][NFQ] -> face-node moments [nb][NFN] (transpose of face_trace)
template <class EL, class T, class OT> __device__ __forceinline__ void face_lift(const T* in, T* out, T* tmp, const OT* ops, int nb) {
  if constexpr (EL::TENSOR) {
    const OT* B = ops + EL::OB;
    if constexpr (EL::DIM == 2) {
      contract<0, EL::NQ, 1, 1, EL::N1, true, false>(in, out, B, nb);
    } else {
      contract<0, EL::NQ, EL::NQ, 1, EL::N1, true, false>(in, tmp, B, nb);
      __syncthreads();
      contract<1, EL::N1, EL::NQ, 1, EL::N1, true, false>(tmp, out, B, nb);
    }
  } else {
    matvec<EL::NFN, EL::NFQ, true, false>(in, out, ops + EL::OBF, nb);
  }
}
// nodal [nb][NPE] -> volume points [nb][NQV]; t1, t2 hold [nb][max(NQ,N1)^DIM]
template <class EL, class T, class OT> __device__ __forceinline__ void vol_interp(const T* in, T* out, T* t1, const OT* ops, int nb) {
  if constexpr (EL::TENSOR) {
    constexpr int N1 = EL::N1, NQ = EL::NQ;
    const OT* B = ops + EL::OB;
    if constexpr (EL::DIM == 2) {
      contract<0, N1, N1, 1, NQ, false, false>(in, t1, B, nb);
      __syncthreads();
      contract<1, NQ, N1, 1, NQ, false, false>(t1, out, B, nb);
    } else {
      contract<0, N1, N1, N1, NQ, false, false>(in, out, B, nb);
      __syncthreads();
      contract<1, NQ, N1, N1, NQ, false, false>(out, t1, B, nb);
      __syncthreads();
      contract<2, NQ, NQ, N1, NQ, false, false>(t1, out, B, nb);
    }
  } else {
    matvec<EL::NQV, EL::NPE, false, false>(in, out, ops + EL::OB, nb);
  }
}
// out[nb][NPE] (+)= sum over volume points of Op_k^T in_k: k < DIM uses the
// reference derivative along axis k, k == DIM the plain basis (both transposed).
template <class EL, bool ACC, class T, class OT>
__device__ __forceinline__ void vol_integrate(int k, const T* in, T* out, T* t1, T* t2, const OT* ops, int nb) {
  if constexpr (EL::TENSOR) {
    constexpr int N1 = EL::N1, NQ = EL::NQ;
    const OT* B = ops + EL::OB;
    const OT* D = ops + EL::OD;
    if constexpr (EL::DIM == 2) {
      contract<0, NQ, NQ, 1, N1, true, false>(in, t1, k == 0 ? D : B, nb);
      __syncthreads();
      contract<1, N1, NQ, 1, N1, true, ACC>(t1, out, k == 1 ? D : B, nb);
    } else {
      contract<0, NQ, NQ, NQ, N1, true, false>(in, t1, k == 0 ? D : B, nb);
      __syncthreads();
      contract<1, N1, NQ, NQ, N1, true, false>(t1, t2, k == 1 ? D : B, nb);
      __syncthreads();
      contract<2, N1, N1, NQ, N1, true, ACC>(t2, out, k == 2 ? D : B, nb);
    }
  } else {
    const OT* M = ops + (k == EL::DIM ? EL::OB : (k == 0 ? EL::ODR : (k == 1 ? EL::ODS : EL::ODT)));
    matvec<EL::NPE, EL::NQV, true, ACC>(in, out, M, nb);
  }
}
// reference derivative along axis k at the nodes (collocation): [nb][NPE] -> [nb][NPE]
template <class EL, class T, class OT> __device__ __forceinline__ void nodal_deriv(int k, const T* in, T* out, const OT* ops, int nb) {
  if constexpr (EL::TENSOR) {
    constexpr int N1 = EL::N1;
    const OT* Dn = ops + EL::ODN;
    if constexpr (EL::DIM == 2) {
      if (k == 0) contract<0, N1, N1, 1, N1, false, false>(in, out, Dn, nb);
      else contract<1, N1, N1, 1, N1, false, false>(in, out, Dn, nb);
    } else {
      if (k == 0) contract<0, N1, N1, N1, N1, false, false>(in, out, Dn, nb);
      else if (k == 1) contract<1, N1, N1, N1, N1, false, false>(in, out, Dn, nb);
      else contract<2, N1, N1, N1, N1, false, false>(in, out, Dn, nb);
    }
  } else {
    matvec<EL::NPE, EL::NPE, false, false>(in, out, ops + (k == 0 ? EL::ODNR : (k == 1 ? EL::ODNS : EL::ODNT)), nb);
  }
}
// reference mass inverse: [nb][NPE] -> [nb][NPE] (in is overwritten for tensor elements)
template <class EL, class T, class OT> __device__ __forceinline__ void mass_inv(T* in, T* out, const OT* ops, int nb) {
  if constexpr (EL::TENSOR) {
    constexpr int N1 = EL::N1;
    const OT* Mi = ops + EL::OMI;
    if constexpr (EL::DIM == 2) {
      contract<0, N1, N1, 1, N1, false, false>(in, out, Mi, nb);
      __syncthreads();
      contract<1, N1, N1, 1, N1, false, false>(out, in, Mi, nb);
      __syncthreads();
      for (int i = threadIdx.x; i < nb * EL::NPE; i += blockDim.x) out[i] = in[i];
    } else {
      contract<0, N1, N1, N1, N1, false, false>(in, out, Mi, nb);
      __syncthreads();
      contract<1, N1, N1, N1, N1, false, false>(out, in, Mi, nb);
      __syncthreads();
      contract<2, N1, N1, N1, N1, false, false>(in, out, Mi, nb);
    }
  } else {
    matvec<EL::NPE, EL::NPE, false, false>(in, out, ops + EL::OMI, nb);
  }
}

template <class EL> struct Sizes {
  static constexpr int M = (EL::TENSOR ? ipow(EL::NQ > EL::N1 ? EL::NQ : EL::N1, EL::DIM) : (EL::NQV > EL::NPE ? EL::NQV : EL::NPE));
  // face-trace temporary: only the 3-D sum factorisation needs one
  static constexpr int MF = (EL::TENSOR && EL::DIM == 3) ? EL::NQ * EL::N1 : 1;
};

template <class R> __device__ __forceinline__ const R* ops_of(const KArgs& a) {
  if constexpr (sizeof(R) == 8) return (const R*)a.ops;
  else return (const R*)a.opsf;
}

// ===================================================================== q-stage
template <class EL, class MD, class R, class TL> struct QLayout {
  static constexpr int DIM = EL::DIM, NCU = MD::NCU, NF = EL::NF;
  static constexpr int GEO = Geo<DIM>::size(NF);
  // bytes per element of each array
  static constexpr int B_GEO = al16(GEO * sizeof(R)), B_U = al16(NCU * EL::NPE * sizeof(R)),
                       B_LF = al16(NF * NCU * EL::NFN * sizeof(R));
  static constexpr int B_FN = al16(NF * NCU * EL::NFN * sizeof(R)), B_FT = al16(NF * NCU * Sizes<EL>::MF * sizeof(R)),
                       B_TR = al16(NF * NCU * EL::NFQ * sizeof(R));
  static constexpr int PHASE_F = 2 * B_FN + 2 * B_TR + 2 * B_FT;   // FNm, FNp, TRm, TRp, tmp
  static constexpr int B_V = al16(NCU * DIM * EL::NPE * sizeof(R));
  static constexpr int PHASE_V = 3 * B_V;                           // grad, b, scratch
  static constexpr int PER_ELEM = B_GEO + B_U + B_LF + (PHASE_F > PHASE_V ? PHASE_F : PHASE_V);
  static constexpr int NE_ = TL::BUDGET_Q / PER_ELEM;
  static constexpr int NE = NE_ < 1 ? 1 : (NE_ > TL::NE_MAX ? TL::NE_MAX : NE_);
  static constexpr int SMEM = NE * PER_ELEM;
};

// Storage of q written by a q-stage in arithmetic R and read by the residual stage: FP64
// for the FP64 kernels, FP32 for the FP32 ones (the Krylov J.v's scratch).
template <class R> using QOut = typename std::conditional<sizeof(R) == 4, float, double>::type;

template <class EL, class MD, int MODE, class R, class TL>
__global__ void __launch_bounds__(256) k_qstage(KArgs a) {
  typedef QLayout<EL, MD, R, TL> L;
  constexpr int DIM = EL::DIM, NCU = MD::NCU, NF = EL::NF, NPE = EL::NPE, NFN = EL::NFN, NFQ = EL::NFQ;
  constexpr int NE = L::NE, GEO = L::GEO;
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int e0 = blockIdx.x * NE;
  const int ne = min(NE, a.E - e0);
  if (!cta_active(a, e0, ne)) return;
  const R* OPS = ops_of<R>(a);
  R* Gs = (R*)smem;
  R* Us = (R*)(smem + NE * L::B_GEO);
  R* LF = (R*)(smem + NE * (L::B_GEO + L::B_U));
  unsigned char* arena = smem + NE * (L::B_GEO + L::B_U + L::B_LF);
  const double* u = (const double*)a.u;

  for (int i = threadIdx.x; i < ne * GEO; i += blockDim.x) Gs[i] = R(a.geo[(size_t)e0 * GEO + i]);
  for (int i = threadIdx.x; i < NE * NCU * NPE; i += blockDim.x) {
    const double x = i < ne * NCU * NPE ? u[(size_t)e0 * NCU * NPE + i] : 0.0;
    Us[i] = R(x);
    if (MODE == MODE_R && a.u32_out && i < ne * NCU * NPE) a.u32_out[(size_t)e0 * NCU * NPE + i] = (float)x;
  }
  __syncthreads();

  // ---- faces: traces of u on both sides, (u- - uhat) weighted, lifted to face nodes
  R* FNm = (R*)arena;
  R* FNp = (R*)(arena + NE * L::B_FN);
  R* TRm = (R*)(arena + NE * 2 * L::B_FN);
  R* TRp = (R*)(arena + NE * (2 * L::B_FN + L::B_TR));
  R* TMP = (R*)(arena + NE * (2 * L::B_FN + 2 * L::B_TR));
  for (int it = threadIdx.x; it < NE * NF * NCU * NFN; it += blockDim.x) {
    int j = it % NFN, c = (it / NFN) % NCU, f = (it / (NFN * NCU)) % NF, e = it / (NFN * NCU * NF);
    R vm = R(0), vp = R(0);
    if (e < ne) {
      vm = Us[(e * NCU + c) * NPE + EL::face_node(f, j)];
      int nb = a.nbr[(size_t)(e0 + e) * NF + f];
      if (nb >= 0) vp = R(u[((size_t)nb * NCU + c) * NPE + nbr_face_node<EL>(a, a.nbf[(size_t)(e0 + e) * NF + f], j)]);
    }
    FNm[it] = vm;
    FNp[it] = vp;
  }
  __syncthreads();
  face_trace<EL>(FNm, TRm, TMP, OPS, NE * NF * NCU);
  __syncthreads();
  face_trace<EL>(FNp, TRp, TMP, OPS, NE * NF * NCU);
  __syncthreads();
  for (int it = threadIdx.x; it < NE * NF * NFQ; it += blockDim.x) {
    int k = it % NFQ, f = (it / NFQ) % NF, e = it / (NFQ * NF);
    if (e >= ne) {
      for (int c = 0; c < NCU; ++c) TRm[((e * NF + f) * NCU + c) * NFQ + k] = R(0);
      continue;
    }
    const R* g = Gs + e * GEO;
    const R w = face_w<EL>(OPS, k) * g[Geo<DIM>::FACE + f * (DIM + 1) + DIM];
    int nb = a.nbr[(size_t)(e0 + e) * NF + f];
    double gb[4] = {0.0, 0.0, 0.0, 0.0};
    int kp = k;
    if (nb >= 0) {
      kp = nbr_face_point<EL>(a, a.nbf[(size_t)(e0 + e) * NF + f], k);
    } else if (MODE == MODE_R && nb == -1) {
      double x[3];
      face_phys<EL>(a, g, OPS, e0 + e, f, k, x);
      exact_state<DIM>(elem_mp(a, e0 + e), NCU, x, a.t_dev ? *a.t_dev : a.t, gb);
    }
    for (int c = 0; c < NCU; ++c) {
      int base = ((e * NF + f) * NCU + c) * NFQ;
      R um = TRm[base + k];
      // wall faces (gas models): the trace (rho-, 0, 0, (rho E)-), linear in u
      R uh = nb >= 0 ? (um + TRp[base + kp]) * R(0.5)
                     : (nb == -2 ? ((c == 0 || c == NCU - 1) ? um : R(0)) : R(gb[c]));
      // TRm is overwritten in place: only this thread reads entry (e,f,c,k)
      TRm[base + k] = (um - uh) * w;
    }
  }
  __syncthreads();
  face_lift<EL>(TRm, LF, TMP, OPS, NE * NF * NCU);
  __syncthreads();

  // ---- volume: q_d = -sum_k Jinv[k][d] D_k u + (1/detJ) M^{-1} sum_f n_d lift_f
  R* GR = (R*)arena;                          // [DIM][NE][NCU][NPE]
  R* BV = (R*)(arena + NE * L::B_V);          // [NE][NCU][DIM][NPE]
  R* SC = (R*)(arena + 2 * NE * L::B_V);
  for (int k = 0; k < DIM; ++k) nodal_deriv<EL>(k, Us, GR + k * NE * NCU * NPE, OPS, NE * NCU);
  for (int it = threadIdx.x; it < NE * NCU * DIM * NPE; it += blockDim.x) {
    int n = it % NPE, d = (it / NPE) % DIM, c = (it / (NPE * DIM)) % NCU, e = it / (NPE * DIM * NCU);
    R s = R(0);
    if (e < ne) {
      const R* g = Gs + e * GEO;
      for_node_faces<EL>(n, [&](int f, int j) {
        s += LF[((e * NF + f) * NCU + c) * NFN + j] * g[Geo<DIM>::FACE + f * (DIM + 1) + d];
      });
    }
    BV[it] = s;
  }
  __syncthreads();
  mass_inv<EL>(BV, SC, OPS, NE * NCU * DIM);
  __syncthreads();
  QOut<R>* qo = (QOut<R>*)a.out;
  for (int it = threadIdx.x; it < ne * NCU * DIM * NPE; it += blockDim.x) {
    int n = it % NPE, d = (it / NPE) % DIM, c = (it / (NPE * DIM)) % NCU, e = it / (NPE * DIM * NCU);
    const R* g = Gs + e * GEO;
    R s = SC[it] / g[Geo<DIM>::DETJ];
    for (int k = 0; k < DIM; ++k) s -= GR[(k * NE * NCU + e * NCU + c) * NPE + n] * g[Geo<DIM>::JINV + k * DIM + d];
    qo[(size_t)e0 * NCU * DIM * NPE + it] = (QOut<R>)s;
    if (MODE == MODE_R && a.q32_out) a.q32_out[(size_t)e0 * NCU * DIM * NPE + it] = (float)s;
  }
}

// ============================================================ curved q-stage
// Curved elements: the weak form of Eq. 1a with the element's own mass matrix,
//   (M_K q_d)_i = sum_q w det J u_h d_d phi_i - sum_f sum_k w sJ uhat n_d phi_i,
// the volume term by the transposed reference derivatives (sum-factorised on
// quadrilaterals) of the per-point
// metric times u_h, the face term by lifting -uhat n_d w per point, then q_d by the
// precomputed inverse M_K^{-1} (the strong form no longer equals it when the
// quadrature is inexact on curved elements).
template <class EL, class MD, class R, class TL> struct QLayoutC {
  static constexpr int DIM = EL::DIM, NCU = MD::NCU, NF = EL::NF, M = Sizes<EL>::M;
  static constexpr int GEO = CGeo<EL>::SIZE;
  static constexpr int B_GEO = al16(GEO * sizeof(R)), B_U = al16(NCU * EL::NPE * sizeof(R)),
                       B_LF = al16(NF * NCU * DIM * EL::NFN * sizeof(R));
  static constexpr int B_FN = al16(NF * NCU * EL::NFN * sizeof(R)), B_TR = al16(NF * NCU * EL::NFQ * sizeof(R)),
                       B_TD = al16(NF * NCU * DIM * EL::NFQ * sizeof(R)),
                       B_FT = al16(NF * NCU * DIM * Sizes<EL>::MF * sizeof(R));
  static constexpr int PHASE_F = 2 * B_FN + 2 * B_TR + B_TD + B_FT;
  static constexpr int B_Q = al16(NCU * M * sizeof(R)), B_RV = al16(NCU * EL::NPE * sizeof(R)),
                       B_BV = al16(NCU * DIM * EL::NPE * sizeof(R));
  static constexpr int PHASE_V = (1 + DIM + 2) * B_Q + B_RV + B_BV;   // u at points, DIM slabs, 2 temporaries
  static constexpr int PER_ELEM = B_GEO + B_U + B_LF + (PHASE_F > PHASE_V ? PHASE_F : PHASE_V);
  static constexpr int NE_ = TL::BUDGET_Q / PER_ELEM;
  static constexpr int NE = NE_ < 1 ? 1 : (NE_ > TL::NE_MAX ? TL::NE_MAX : NE_);
  static constexpr int SMEM = NE * PER_ELEM;
};

template <class EL, class MD, int MODE, class R, class TL>
__global__ void __launch_bounds__(256) k_qstage_curved(KArgs a) {
  typedef QLayoutC<EL, MD, R, TL> L;
  typedef CGeo<EL> CG;
  constexpr int DIM = EL::DIM, NCU = MD::NCU, NF = EL::NF, NPE = EL::NPE, NFN = EL::NFN, NFQ = EL::NFQ, NQV = EL::NQV;
  constexpr int NE = L::NE, GEO = L::GEO, M = Sizes<EL>::M;
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int e0 = blockIdx.x * NE;
  const int ne = min(NE, a.E - e0);
  if (!cta_active(a, e0, ne)) return;
  const R* OPS = ops_of<R>(a);
  const R* GSRC = geo_src<EL, R>(a);
  R* Gs = (R*)smem;
  R* Us = (R*)(smem + NE * L::B_GEO);
  R* LF = (R*)(smem + NE * (L::B_GEO + L::B_U));     // [NE][NF][NCU][DIM][NFN]
  unsigned char* arena = smem + NE * (L::B_GEO + L::B_U + L::B_LF);
  const double* u = (const double*)a.u;

  for (int i = threadIdx.x; i < ne * GEO; i += blockDim.x) Gs[i] = GSRC[(size_t)e0 * GEO + i];
  for (int i = threadIdx.x; i < NE * NCU * NPE; i += blockDim.x) {
    const double x = i < ne * NCU * NPE ? u[(size_t)e0 * NCU * NPE + i] : 0.0;
    Us[i] = R(x);
    if (MODE == MODE_R && a.u32_out && i < ne * NCU * NPE) a.u32_out[(size_t)e0 * NCU * NPE + i] = (float)x;
  }
  __syncthreads();

  // ---- faces: -uhat n_d w at every face point, lifted to the face nodes
  {
    R* FNm = (R*)arena;
    R* FNp = (R*)(arena + NE * L::B_FN);
    R* TRm = (R*)(arena + NE * 2 * L::B_FN);
    R* TRp = (R*)(arena + NE * (2 * L::B_FN + L::B_TR));
    R* TD = (R*)(arena + NE * (2 * L::B_FN + 2 * L::B_TR));
    R* TMP = (R*)(arena + NE * (2 * L::B_FN + 2 * L::B_TR + L::B_TD));
    for (int it = threadIdx.x; it < NE * NF * NCU * NFN; it += blockDim.x) {
      const int j = it % NFN, c = (it / NFN) % NCU, f = (it / (NFN * NCU)) % NF, e = it / (NFN * NCU * NF);
      R vm = R(0), vp = R(0);
      if (e < ne) {
        vm = Us[(e * NCU + c) * NPE + EL::face_node(f, j)];
        const int nb = a.nbr[(size_t)(e0 + e) * NF + f];
        if (nb >= 0) {
          const int nf = a.nbf[(size_t)(e0 + e) * NF + f] & 7;
          vp = R(u[((size_t)nb * NCU + c) * NPE + EL::face_node(nf, j)]);
        }
      }
      FNm[it] = vm;
      FNp[it] = vp;
    }
    __syncthreads();
    face_trace<EL>(FNm, TRm, TMP, OPS, NE * NF * NCU);
    __syncthreads();
    face_trace<EL>(FNp, TRp, TMP, OPS, NE * NF * NCU);
    __syncthreads();
    for (int it = threadIdx.x; it < NE * NF * NFQ; it += blockDim.x) {
      const int k = it % NFQ, f = (it / NFQ) % NF, e = it / (NFQ * NF);
      if (e >= ne) {
        for (int cd = 0; cd < NCU * DIM; ++cd) TD[((e * NF + f) * NCU * DIM + cd) * NFQ + k] = R(0);
        continue;
      }
      const R* g = Gs + e * GEO;
      R w;
      const R* nrm = face_frame<EL>(g, OPS, f, k, w);
      const int nb = a.nbr[(size_t)(e0 + e) * NF + f];
      double gb[4] = {0.0, 0.0, 0.0, 0.0};
      int kp = k;
      if (nb >= 0) {
        kp = a.perm[(a.nbf[(size_t)(e0 + e) * NF + f] >> 3) * NFQ + k];
      } else if (MODE == MODE_R && nb == -1) {
        double x[3];
        face_phys<EL>(a, g, OPS, e0 + e, f, k, x);
        exact_state<DIM>(elem_mp(a, e0 + e), NCU, x, a.t_dev ? *a.t_dev : a.t, gb);
      }
      for (int c = 0; c < NCU; ++c) {
        const int base = ((e * NF + f) * NCU + c) * NFQ;
        const R um = TRm[base + k];
        const R uh = nb >= 0 ? (um + TRp[base + kp]) * R(0.5)
                             : (nb == -2 ? ((c == 0 || c == NCU - 1) ? um : R(0)) : R(gb[c]));
        for (int d = 0; d < DIM; ++d) TD[(((e * NF + f) * NCU + c) * DIM + d) * NFQ + k] = -uh * nrm[d] * w;
      }
    }
    __syncthreads();
    face_lift<EL>(TD, LF, TMP, OPS, NE * NF * NCU * DIM);
    __syncthreads();
  }

  // ---- volume: sum_k D_k^T (metric_kd u_h) per d, plus the face moments; then M_K^{-1}
  R* UQ = (R*)arena;                                              // [NE][NCU][NQV]
  R* SL = (R*)(arena + NE * L::B_Q);                              // DIM slabs [NE][NCU][NQV]
  R* T1 = (R*)(arena + NE * (1 + DIM) * L::B_Q);
  R* T2 = (R*)(arena + NE * (2 + DIM) * L::B_Q);
  R* RV = (R*)(arena + NE * (3 + DIM) * L::B_Q);                  // [NE][NCU][NPE]
  R* BV = (R*)(arena + NE * ((3 + DIM) * L::B_Q + L::B_RV));      // [NE][NCU][DIM][NPE]
  constexpr int SLS = NE * L::B_Q / (int)sizeof(R);               // slab stride (elements)
  vol_interp<EL>(Us, UQ, T1, OPS, NE * NCU);
  __syncthreads();
  for (int d = 0; d < DIM; ++d) {
    for (int it = threadIdx.x; it < NE * NCU * NQV; it += blockDim.x) {
      const int q = it % NQV, e = it / (NQV * NCU);
      const R* g = Gs + e * GEO + CG::VG + q * CG::NV;
      for (int k = 0; k < DIM; ++k) SL[k * SLS + it] = e < ne ? g[k * DIM + d] * UQ[it] : R(0);
    }
    __syncthreads();
    vol_integrate<EL, false>(0, SL, RV, T1, T2, OPS, NE * NCU);
    __syncthreads();
    for (int k = 1; k < DIM; ++k) {
      vol_integrate<EL, true>(k, SL + k * SLS, RV, T1, T2, OPS, NE * NCU);
      __syncthreads();
    }
    for (int it = threadIdx.x; it < NE * NCU * NPE; it += blockDim.x) {
      const int n = it % NPE, c = (it / NPE) % NCU, e = it / (NPE * NCU);
      R sacc = RV[it];
      for_node_faces<EL>(n, [&](int f, int j) { sacc += LF[(((e * NF + f) * NCU + c) * DIM + d) * NFN + j]; });
      BV[((e * NCU + c) * DIM + d) * NPE + n] = sacc;
    }
    __syncthreads();
  }
  const R* MI;
  if constexpr (sizeof(R) == 8) MI = (const R*)a.minv;
  else MI = (const R*)a.minvf;
  QOut<R>* qo = (QOut<R>*)a.out;
  for (int it = threadIdx.x; it < ne * NCU * DIM * NPE; it += blockDim.x) {
    const int n = it % NPE, b = it / NPE, e = b / (NCU * DIM);
    const R* mi = MI + ((size_t)(e0 + e) * NPE + n) * NPE;
    const R* bv = BV + b * NPE;
    R sacc = R(0);
#pragma unroll 4
    for (int m = 0; m < NPE; ++m) sacc += mi[m] * bv[m];
    qo[(size_t)e0 * NCU * DIM * NPE + it] = (QOut<R>)sacc;
    if (MODE == MODE_R && a.q32_out) a.q32_out[(size_t)e0 * NCU * DIM * NPE + it] = (float)sacc;
  }
  (void)M;
}

// ==================================================================== residual
template <class EL, class MD, int MODE, class R, class TL> struct RLayout {
  typedef typename std::conditional<MODE == MODE_JV, Dual<R>, R>::type S;
  static constexpr int DIM = EL::DIM, NCU = MD::NCU, NF = EL::NF;
  static constexpr int NCV = NCU * (1 + (MD::HASQ ? DIM : 0));      // u and q fields
  static constexpr int GEO = geo_size<EL>();
  static constexpr int B_GEO = al16(GEO * sizeof(R)), B_X = al16(NCV * EL::NPE * sizeof(S)),
                       B_LF = al16(NF * NCU * EL::NFN * sizeof(R));
  // face phase
  static constexpr int B_FN = al16(NF * NCV * EL::NFN * sizeof(S)), B_FT = al16(NF * NCV * Sizes<EL>::MF * sizeof(S)),
                       B_TR = al16(NF * NCV * EL::NFQ * sizeof(S)), B_FH = al16(NF * NCU * EL::NFQ * sizeof(R));
  static constexpr int PHASE_F = 2 * B_FN + 2 * B_TR + B_FT + B_FH;
  // volume phase
  static constexpr int B_XQ = al16(NCV * Sizes<EL>::M * sizeof(S)), B_T1 = al16(NCV * Sizes<EL>::M * sizeof(S)),
                       B_H = MODE == MODE_R ? al16(NCU * Sizes<EL>::M * sizeof(R)) : 0,
                       B_G = al16(NCU * Sizes<EL>::M * sizeof(R));
  static constexpr int PHASE_V = B_XQ + B_T1 + 2 * B_H /*hist nodal + at points*/ + (DIM + 1) * B_G + 2 * B_G /*t1,t2*/ + B_G /*Rv*/;
  static constexpr int PER_ELEM = B_GEO + B_X + B_LF + (PHASE_F > PHASE_V ? PHASE_F : PHASE_V);
  static constexpr int NE_ = TL::BUDGET_R / PER_ELEM;
  static constexpr int NE = NE_ < 1 ? 1 : (NE_ > TL::NE_MAX ? TL::NE_MAX : NE_);
  static constexpr int SMEM = NE * PER_ELEM;
};

// Minimum resident CTAs per SM asked of the register allocator. For the FP32
// dual-number J.v of the Navier-Stokes model, whose register count otherwise leaves two
// 256-thread CTAs per SM: as many as the tile's shared-memory budget lets reside, at
// most 4 (64 registers; measured 9% faster than 3 on the 40,000-element cylinder, with
// about 100 bytes of spills per thread). 1 otherwise.
template <class MD, int MODE, class R, class TL> struct ResMinBlocks {
  static constexpr int BY_SMEM = (228 * 1024) / (TL::BUDGET_R + 1024);
  static constexpr int value =
      (MD::KIND == M_NS && MODE == MODE_JV && sizeof(R) == 4) ? (BY_SMEM < 1 ? 1 : (BY_SMEM > 4 ? 4 : BY_SMEM)) : 1;
};

template <class EL, class MD, int MODE, class R, class TL>
__global__ void __launch_bounds__(256, ResMinBlocks<MD, MODE, R, TL>::value) k_residual(KArgs a) {
  typedef RLayout<EL, MD, MODE, R, TL> L;
  typedef typename L::S S;
  constexpr int DIM = EL::DIM, NCU = MD::NCU, NF = EL::NF, NPE = EL::NPE, NFN = EL::NFN, NFQ = EL::NFQ, NQV = EL::NQV;
  constexpr int NE = L::NE, GEO = L::GEO, NCV = L::NCV;
  constexpr bool HASQ = MD::HASQ;
  static_assert(!(MODE == MODE_JV && HASQ && MD::LINEAR), "linear models take MODE_HOM for J.v");
  if (a.skip && *a.skip) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int e0 = blockIdx.x * NE;
  const int ne = min(NE, a.E - e0);
  if (!cta_active(a, e0, ne)) return;
  const R* OPS = ops_of<R>(a);
  __shared__ MPar<R> MPs[NE];   // per-element model parameters (padding elements: a.mp)
  for (int e = threadIdx.x; e < NE; e += blockDim.x) MPs[e] = mpar<R>(e < ne ? elem_mp(a, e0 + e) : a.mp);
  R* Gs = (R*)smem;
  S* X = (S*)(smem + NE * L::B_GEO);                       // [NE][NCV][NPE]
  R* LF = (R*)(smem + NE * (L::B_GEO + L::B_X));           // [NE][NF][NCU][NFN]
  unsigned char* arena = smem + NE * (L::B_GEO + L::B_X + L::B_LF);
  // FP32 instances read q scratch in FP32, and a nonlinear model's state too (its FP32
  // copy written by the FP64 q-stage of the residual)
  typedef typename std::conditional<(sizeof(R) == 4 && MODE == MODE_JV && HASQ), float, double>::type UIn;
  const UIn* u = (const UIn*)a.u;
  const double* v = (const double*)a.v;
  const QOut<R>* q = (const QOut<R>*)a.q;
  const QOut<R>* dq = (const QOut<R>*)a.dq;

  if constexpr (EL::CURVED) {
    const R* src = geo_src<EL, R>(a);
    for (int i = threadIdx.x; i < ne * GEO; i += blockDim.x) Gs[i] = src[(size_t)e0 * GEO + i];
  } else {
    for (int i = threadIdx.x; i < ne * GEO; i += blockDim.x) Gs[i] = R(a.geo[(size_t)e0 * GEO + i]);
  }
  for (int i = threadIdx.x; i < NE * NCV * NPE; i += blockDim.x) {
    int n = i % NPE, fld = (i / NPE) % NCV, e = i / (NPE * NCV);
    S val = S(R(0));
    if (e < ne) {
      if (fld < NCU) {
        size_t gi = ((size_t)(e0 + e) * NCU + fld) * NPE + n;
        if constexpr (MODE == MODE_JV)
          val = S(R(u[gi]), a.blk_col >= 0 ? R(fld * NPE + n == a.blk_col ? 1 : 0) : R(v[gi]));
        else val = S(R(u[gi]));
      } else if constexpr (HASQ) {
        const size_t gi = ((size_t)(e0 + e) * NCU * DIM + (fld - NCU)) * NPE + n;
        if constexpr (MODE == MODE_JV) val = S(R(q[gi]), R(dq[gi]));
        else val = S(R(q[gi]));
      }
    }
    X[i] = val;
  }
  __syncthreads();

  // ------------------------------------------------------------- face phase
  {
    S* FNm = (S*)arena;
    S* FNp = (S*)(arena + NE * L::B_FN);
    S* TRm = (S*)(arena + NE * 2 * L::B_FN);
    S* TRp = (S*)(arena + NE * (2 * L::B_FN + L::B_TR));
    S* TMP = (S*)(arena + NE * (2 * L::B_FN + 2 * L::B_TR));
    R* FH = (R*)(arena + NE * (2 * L::B_FN + 2 * L::B_TR + L::B_FT));
    for (int it = threadIdx.x; it < NE * NF * NCV * NFN; it += blockDim.x) {
      int j = it % NFN, fld = (it / NFN) % NCV, f = (it / (NFN * NCV)) % NF, e = it / (NFN * NCV * NF);
      S vm = S(R(0)), vp = S(R(0));
      if (e < ne) {
        vm = X[(e * NCV + fld) * NPE + EL::face_node(f, j)];
        int nb = a.nbr[(size_t)(e0 + e) * NF + f];
        if (nb >= 0) {
          const int nn = nbr_face_node<EL>(a, a.nbf[(size_t)(e0 + e) * NF + f], j);
          if (fld < NCU) {
            size_t gi = ((size_t)nb * NCU + fld) * NPE + nn;
            if constexpr (MODE == MODE_JV) vp = S(R(u[gi]), a.blk_col >= 0 ? R(0) : R(v[gi]));
            else vp = S(R(u[gi]));
          } else if constexpr (HASQ) {
            const size_t gi = ((size_t)nb * NCU * DIM + (fld - NCU)) * NPE + nn;
            if constexpr (MODE == MODE_JV) vp = S(R(q[gi]), R(dq[gi]));
            else vp = S(R(q[gi]));
          }
        }
      }
      FNm[it] = vm;
      FNp[it] = vp;
    }
    __syncthreads();
    face_trace<EL>(FNm, TRm, TMP, OPS, NE * NF * NCV);
    __syncthreads();
    face_trace<EL>(FNp, TRp, TMP, OPS, NE * NF * NCV);
    __syncthreads();
    for (int it = threadIdx.x; it < NE * NF * NFQ; it += blockDim.x) {
      int k = it % NFQ, f = (it / NFQ) % NF, e = it / (NFQ * NF);
      if (e >= ne) {
        for (int c = 0; c < NCU; ++c) FH[((e * NF + f) * NCU + c) * NFQ + k] = R(0);
        continue;
      }
      const R* g = Gs + e * GEO;
      R w;
      const R* nrm = face_frame<EL>(g, OPS, f, k, w);
      int nb = a.nbr[(size_t)(e0 + e) * NF + f];
      S um[NCU], qm[NCU * DIM + 1], fh[NCU];
      for (int fld = 0; fld < NCV; ++fld) {
        S val = TRm[((e * NF + f) * NCV + fld) * NFQ + k];
        if (fld < NCU) um[fld] = val; else qm[fld - NCU] = val;
      }
      if (nb >= 0) {
        const int kp = nbr_face_point<EL>(a, a.nbf[(size_t)(e0 + e) * NF + f], k);
        S up[NCU], qp[NCU * DIM + 1];
        for (int fld = 0; fld < NCV; ++fld) {
          S val = TRp[((e * NF + f) * NCV + fld) * NFQ + kp];
          if (fld < NCU) up[fld] = val; else qp[fld - NCU] = val;
        }
        MD::fhat(um, up, qm, qp, nrm, fh, MPs[e]);
      } else if (MD::NCU == 4 && nb == -2) {
        if constexpr (MD::NCU == 4) MD::fhat_wall(um, qm, nrm, fh, MPs[e]);
      } else {
        R gb[4] = {R(0), R(0), R(0), R(0)};
        if (MODE != MODE_HOM) {
          double x[3], gd[4] = {0.0, 0.0, 0.0, 0.0};
          face_phys<EL>(a, g, OPS, e0 + e, f, k, x);
          exact_state<DIM>(elem_mp(a, e0 + e), NCU, x, a.t_dev ? *a.t_dev : a.t, gd);
          for (int c = 0; c < 4; ++c) gb[c] = R(gd[c]);
        }
        MD::fhat_bnd(um, qm, gb, nrm, fh, MPs[e]);
      }
      for (int c = 0; c < NCU; ++c) FH[((e * NF + f) * NCU + c) * NFQ + k] = outp(fh[c]) * w;
    }
    __syncthreads();
    face_lift<EL>(FH, LF, (R*)TMP, OPS, NE * NF * NCU);
    __syncthreads();
  }

  // ----------------------------------------------------------- volume phase
  S* XQ = (S*)arena;                                                   // [NE][NCV][NQV]
  S* T1 = (S*)(arena + NE * L::B_XQ);
  R* HN = (R*)(arena + NE * (L::B_XQ + L::B_T1));                      // [NE][NCU][NPE]
  R* HQ = (R*)(arena + NE * (L::B_XQ + L::B_T1 + L::B_H));             // [NE][NCU][NQV]
  R* GK = (R*)(arena + NE * (L::B_XQ + L::B_T1 + 2 * L::B_H));         // [DIM+1][NE][NCU][NQV]
  R* R1 = GK + (DIM + 1) * NE * (L::B_G / sizeof(R));
  R* R2 = R1 + NE * (L::B_G / sizeof(R));
  R* RV = R2 + NE * (L::B_G / sizeof(R));                              // [NE][NCU][NPE]
  vol_interp<EL>(X, XQ, T1, OPS, NE * NCV);
  const bool hist = (MODE == MODE_R) && a.hist != nullptr;
  if (hist) {
    const double* h = (const double*)a.hist;
    for (int i = threadIdx.x; i < NE * NCU * NPE; i += blockDim.x)
      HN[i] = i < ne * NCU * NPE ? R(h[(size_t)e0 * NCU * NPE + i]) : R(0);
    __syncthreads();
    vol_interp<EL>(HN, HQ, (R*)T1, OPS, NE * NCU);
  }
  __syncthreads();
  const R a0dt = R(a.a0dt);
  for (int it = threadIdx.x; it < NE * NQV; it += blockDim.x) {
    int qp = it % NQV, e = it / NQV;
    S uq[NCU], qq[NCU * DIM + 1], f[NCU * DIM];
    for (int fld = 0; fld < NCV; ++fld) {
      S val = XQ[(e * NCV + fld) * NQV + qp];
      if (fld < NCU) uq[fld] = val; else qq[fld - NCU] = val;
    }
    const R* g = Gs + e * GEO;
    R wj;
    if constexpr (EL::CURVED) {
      wj = g[CGeo<EL>::VG + qp * CGeo<EL>::NV + DIM * DIM];
    } else {
      R xi[3], w;
      vol_xi<EL>(OPS, qp, xi, w);
      wj = w * g[Geo<DIM>::DETJ];
    }
    R src = R(0);
    if (MODE == MODE_R && e < ne && MD::SOURCE) {
      double x[3];
      vol_phys<EL>(a, g, OPS, e0 + e, qp, x);
      src = R(source_term<DIM>(elem_mp(a, e0 + e), MD::KIND == M_CONVDIFF, x));
    }
    MD::flux(uq, qq, f, MPs[e]);
    for (int c = 0; c < NCU; ++c) {
      for (int k = 0; k < DIM; ++k) {
        R s = R(0);
        if constexpr (EL::CURVED) {
          // the per-point metric already carries w det J
          for (int d = 0; d < DIM; ++d) s += outp(f[c * DIM + d]) * g[CGeo<EL>::VG + qp * CGeo<EL>::NV + k * DIM + d];
          GK[((k + 1) * NE * NCU + e * NCU + c) * NQV + qp] = (e < ne) ? -s : R(0);
        } else {
          for (int d = 0; d < DIM; ++d) s += outp(f[c * DIM + d]) * g[Geo<DIM>::JINV + k * DIM + d];
          GK[((k + 1) * NE * NCU + e * NCU + c) * NQV + qp] = (e < ne) ? -s * wj : R(0);
        }
      }
      R tt = outp(uq[c]) * a0dt;
      if (hist) tt += HQ[(e * NCU + c) * NQV + qp];
      GK[(e * NCU + c) * NQV + qp] = (e < ne) ? (tt - src) * wj : R(0);
    }
  }
  __syncthreads();
  // slab 0: time/source term with the plain basis; slabs 1..DIM: flux with derivative along k
  vol_integrate<EL, false>(DIM, GK, RV, R1, R2, OPS, NE * NCU);
  __syncthreads();
  for (int k = 0; k < DIM; ++k) {
    vol_integrate<EL, true>(k, GK + (k + 1) * NE * NCU * NQV, RV, R1, R2, OPS, NE * NCU);
    __syncthreads();
  }
  // ---- gather face moments and store
  double* out = (double*)a.out;
  for (int it = threadIdx.x; it < ne * NCU * NPE; it += blockDim.x) {
    int n = it % NPE, c = (it / NPE) % NCU, e = it / (NPE * NCU);
    R s = RV[it];
    for_node_faces<EL>(n, [&](int f, int j) { s += LF[((e * NF + f) * NCU + c) * NFN + j]; });
    if (MODE == MODE_JV && a.blk_col >= 0) {
      constexpr int NLOC = NCU * NPE;
      a.blk_out[((size_t)(e0 + e) * NLOC + a.blk_col) * NLOC + (it - e * NLOC)] = (double)s;
    } else if (MODE == MODE_R && a.radd) {
      const size_t gi = (size_t)e0 * NCU * NPE + it;
      out[gi] = (double)s + a.radd[gi];
    } else {
      out[(size_t)e0 * NCU * NPE + it] = (double)s;
    }
  }
}

// ============================================================ block columns
// Columns col0 .. col0 + KT - 1 of every element's diagonal block dR_K/du_K for a
// model without q (Euler): the same stages as k_residual in MODE_JV, with a dual
// number of KT tangents seeded with the unit columns on the element's own state and
// no tangent on its neighbours. The linear stages after the flux evaluation (face
// lift, volume integration) treat the KT tangents as KT extra components.
template <class EL, class MD, class R, class TL, int KT> struct BLayout {
  typedef DualK<R, KT> S;
  static constexpr int DIM = EL::DIM, NCU = MD::NCU, NF = EL::NF, NCO = NCU * KT;
  static constexpr int GEO = Geo<DIM>::size(NF);
  static constexpr int B_GEO = al16(GEO * sizeof(R)), B_X = al16(NCU * EL::NPE * sizeof(S)),
                       B_LF = al16(NF * NCO * EL::NFN * sizeof(R));
  static constexpr int B_FNM = al16(NF * NCU * EL::NFN * sizeof(S)), B_FNP = al16(NF * NCU * EL::NFN * sizeof(R)),
                       B_TRM = al16(NF * NCU * EL::NFQ * sizeof(S)), B_TRP = al16(NF * NCU * EL::NFQ * sizeof(R)),
                       B_FT = al16(NF * NCU * Sizes<EL>::MF * sizeof(S) > NF * NCO * Sizes<EL>::MF * sizeof(R)
                                       ? NF * NCU * Sizes<EL>::MF * sizeof(S)
                                       : NF * NCO * Sizes<EL>::MF * sizeof(R)),
                       B_FH = al16(NF * NCO * EL::NFQ * sizeof(R));
  static constexpr int PHASE_F = B_FNM + B_FNP + B_TRM + B_TRP + B_FT + B_FH;
  static constexpr int B_XQ = al16(NCU * Sizes<EL>::M * sizeof(S)), B_G = al16(NCO * Sizes<EL>::M * sizeof(R));
  static constexpr int PHASE_V = 2 * B_XQ + (DIM + 1) * B_G + 2 * B_G + B_G;
  static constexpr int PER_ELEM = B_GEO + B_X + B_LF + (PHASE_F > PHASE_V ? PHASE_F : PHASE_V);
  static constexpr int NE_ = TL::BUDGET_R / PER_ELEM;
  static constexpr int NE = NE_ < 1 ? 1 : (NE_ > TL::NE_MAX ? TL::NE_MAX : NE_);
  static constexpr int SMEM = NE * PER_ELEM;
};

template <class EL, class MD, class R, class TL, int KT>
__global__ void __launch_bounds__(256) k_block_columns(KArgs a, int col0) {
  typedef BLayout<EL, MD, R, TL, KT> L;
  typedef typename L::S S;
  constexpr int DIM = EL::DIM, NCU = MD::NCU, NF = EL::NF, NPE = EL::NPE, NFN = EL::NFN, NFQ = EL::NFQ, NQV = EL::NQV;
  constexpr int NE = L::NE, GEO = L::GEO, NCO = L::NCO, NLOC = NCU * NPE;
  static_assert(!MD::HASQ && !EL::CURVED, "block columns by dual numbers: affine models without q");
  extern __shared__ __align__(16) unsigned char smem[];
  const int e0 = blockIdx.x * NE;
  const int ne = min(NE, a.E - e0);
  if (!cta_active(a, e0, ne)) return;
  const R* OPS = ops_of<R>(a);
  __shared__ MPar<R> MPs[NE];
  for (int e = threadIdx.x; e < NE; e += blockDim.x) MPs[e] = mpar<R>(e < ne ? elem_mp(a, e0 + e) : a.mp);
  R* Gs = (R*)smem;
  S* X = (S*)(smem + NE * L::B_GEO);                        // [NE][NCU][NPE]
  R* LF = (R*)(smem + NE * (L::B_GEO + L::B_X));            // [NE][NF][NCO][NFN]
  unsigned char* arena = smem + NE * (L::B_GEO + L::B_X + L::B_LF);
  const double* u = (const double*)a.u;

  for (int i = threadIdx.x; i < ne * GEO; i += blockDim.x) Gs[i] = R(a.geo[(size_t)e0 * GEO + i]);
  for (int i = threadIdx.x; i < NE * NCU * NPE; i += blockDim.x) {
    const int loc = i % NLOC, e = i / NLOC;
    S val = S(R(0));
    if (e < ne) {
      val = S(R(u[(size_t)e0 * NLOC + i]));
#pragma unroll
      for (int t = 0; t < KT; ++t) val.d[t] = (loc == col0 + t) ? R(1) : R(0);
    }
    X[i] = val;
  }
  __syncthreads();

  // ------------------------------------------------------------- face phase
  {
    S* FNm = (S*)arena;
    R* FNp = (R*)(arena + NE * L::B_FNM);
    S* TRm = (S*)(arena + NE * (L::B_FNM + L::B_FNP));
    R* TRp = (R*)(arena + NE * (L::B_FNM + L::B_FNP + L::B_TRM));
    unsigned char* TMP = arena + NE * (L::B_FNM + L::B_FNP + L::B_TRM + L::B_TRP);
    R* FH = (R*)(arena + NE * (L::B_FNM + L::B_FNP + L::B_TRM + L::B_TRP + L::B_FT));
    for (int it = threadIdx.x; it < NE * NF * NCU * NFN; it += blockDim.x) {
      const int j = it % NFN, c = (it / NFN) % NCU, f = (it / (NFN * NCU)) % NF, e = it / (NFN * NCU * NF);
      S vm = S(R(0));
      R vp = R(0);
      if (e < ne) {
        vm = X[(e * NCU + c) * NPE + EL::face_node(f, j)];
        const int nb = a.nbr[(size_t)(e0 + e) * NF + f];
        if (nb >= 0) {
          const int nfc = a.nbf[(size_t)(e0 + e) * NF + f] & 7;
          vp = R(u[((size_t)nb * NCU + c) * NPE + EL::face_node(nfc, j)]);
        }
      }
      FNm[it] = vm;
      FNp[it] = vp;
    }
    __syncthreads();
    face_trace<EL>(FNm, TRm, (S*)TMP, OPS, NE * NF * NCU);
    __syncthreads();
    face_trace<EL>(FNp, TRp, (R*)TMP, OPS, NE * NF * NCU);
    __syncthreads();
    for (int it = threadIdx.x; it < NE * NF * NFQ; it += blockDim.x) {
      const int k = it % NFQ, f = (it / NFQ) % NF, e = it / (NFQ * NF);
      if (e >= ne) {
        for (int co = 0; co < NCO; ++co) FH[((e * NF + f) * NCO + co) * NFQ + k] = R(0);
        continue;
      }
      const R* g = Gs + e * GEO;
      const R* nrm = g + Geo<DIM>::FACE + f * (DIM + 1);
      const R w = face_w<EL>(OPS, k) * nrm[DIM];
      const int nb = a.nbr[(size_t)(e0 + e) * NF + f];
      S um[NCU], qm[1], fh[NCU];
      for (int c = 0; c < NCU; ++c) um[c] = TRm[((e * NF + f) * NCU + c) * NFQ + k];
      if (nb >= 0) {
        const int kp = a.perm[(a.nbf[(size_t)(e0 + e) * NF + f] >> 3) * NFQ + k];
        S up[NCU], qp[1];
        for (int c = 0; c < NCU; ++c) up[c] = S(TRp[((e * NF + f) * NCU + c) * NFQ + kp]);
        MD::fhat(um, up, qm, qp, nrm, fh, MPs[e]);
      } else if (nb == -2) {
        MD::fhat_wall(um, qm, nrm, fh, MPs[e]);
      } else {
        R gb[4] = {R(0), R(0), R(0), R(0)};
        R xi[3];
        double x[3], gd[4] = {0.0, 0.0, 0.0, 0.0};
        face_xi<EL>(OPS, f, k, xi);
        phys_x<DIM>(g, xi, x);
        exact_state<DIM>(elem_mp(a, e0 + e), NCU, x, a.t_dev ? *a.t_dev : a.t, gd);
        for (int c = 0; c < 4; ++c) gb[c] = R(gd[c]);
        MD::fhat_bnd(um, qm, gb, nrm, fh, MPs[e]);
      }
      for (int c = 0; c < NCU; ++c)
#pragma unroll
        for (int t = 0; t < KT; ++t) FH[((e * NF + f) * NCO + c * KT + t) * NFQ + k] = fh[c].d[t] * w;
    }
    __syncthreads();
    face_lift<EL>(FH, LF, (R*)TMP, OPS, NE * NF * NCO);
    __syncthreads();
  }

  // ----------------------------------------------------------- volume phase
  S* XQ = (S*)arena;                                                   // [NE][NCU][NQV]
  S* T1 = (S*)(arena + NE * L::B_XQ);
  R* GK = (R*)(arena + NE * 2 * L::B_XQ);                              // [DIM+1][NE][NCO][NQV]
  R* R1 = GK + (DIM + 1) * NE * (L::B_G / sizeof(R));
  R* R2 = R1 + NE * (L::B_G / sizeof(R));
  R* RV = R2 + NE * (L::B_G / sizeof(R));                              // [NE][NCO][NPE]
  vol_interp<EL>(X, XQ, T1, OPS, NE * NCU);
  __syncthreads();
  const R a0dt = R(a.a0dt);
  for (int it = threadIdx.x; it < NE * NQV; it += blockDim.x) {
    const int qp = it % NQV, e = it / NQV;
    S uq[NCU], qq[1], f[NCU * DIM];
    for (int c = 0; c < NCU; ++c) uq[c] = XQ[(e * NCU + c) * NQV + qp];
    R xi[3], w;
    vol_xi<EL>(OPS, qp, xi, w);
    const R* g = Gs + e * GEO;
    const R wj = w * g[Geo<DIM>::DETJ];
    MD::flux(uq, qq, f, MPs[e]);
    for (int c = 0; c < NCU; ++c)
#pragma unroll
      for (int t = 0; t < KT; ++t) {
        const int co = c * KT + t;
        for (int k = 0; k < DIM; ++k) {
          R sk = R(0);
          for (int d = 0; d < DIM; ++d) sk += f[c * DIM + d].d[t] * g[Geo<DIM>::JINV + k * DIM + d];
          GK[((k + 1) * NE * NCO + e * NCO + co) * NQV + qp] = (e < ne) ? -sk * wj : R(0);
        }
        GK[(e * NCO + co) * NQV + qp] = (e < ne) ? uq[c].d[t] * a0dt * wj : R(0);
      }
  }
  __syncthreads();
  vol_integrate<EL, false>(DIM, GK, RV, R1, R2, OPS, NE * NCO);
  __syncthreads();
  for (int k = 0; k < DIM; ++k) {
    vol_integrate<EL, true>(k, GK + (k + 1) * NE * NCO * NQV, RV, R1, R2, OPS, NE * NCO);
    __syncthreads();
  }
  // ---- gather face moments and store columns col0 + t of the blocks
  for (int it = threadIdx.x; it < ne * NCO * NPE; it += blockDim.x) {
    const int n = it % NPE, co = (it / NPE) % NCO, e = it / (NPE * NCO);
    const int c = co / KT, t = co - c * KT;
    if (col0 + t >= NLOC) continue;
    R sacc = RV[it];
    for_node_faces<EL>(n, [&](int f, int j) { sacc += LF[((e * NF + f) * NCO + co) * NFN + j]; });
    a.blk_out[((size_t)(e0 + e) * NLOC + col0 + t) * NLOC + c * NPE + n] = (double)sacc;
  }
}

}  // namespace ldg
