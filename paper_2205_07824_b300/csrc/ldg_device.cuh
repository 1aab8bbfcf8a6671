// Device building blocks of the LDG hot path (Section 2.2; Section 3.3):
// forward-mode dual numbers for the exact J.v, element traits with their
// reference operators (sum-factorised tensor elements, full-matrix triangles),
// and the pointwise model functions of the first-order system of Eq. 1a-1b.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ldg {

// ------------------------------------------------------------------ scalars
template <class R> struct Dual {
  R v, d;
  __host__ __device__ Dual() {}
  __host__ __device__ Dual(R a) : v(a), d(R(0)) {}
  __host__ __device__ Dual(R a, R b) : v(a), d(b) {}
};
template <class R> __device__ __forceinline__ Dual<R> operator+(Dual<R> a, Dual<R> b) { return Dual<R>(a.v + b.v, a.d + b.d); }
template <class R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a, Dual<R> b) { return Dual<R>(a.v - b.v, a.d - b.d); }
template <class R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a) { return Dual<R>(-a.v, -a.d); }
template <class R> __device__ __forceinline__ Dual<R> operator*(Dual<R> a, Dual<R> b) { return Dual<R>(a.v * b.v, a.d * b.v + a.v * b.d); }
template <class R> __device__ __forceinline__ Dual<R> operator/(Dual<R> a, Dual<R> b) {
  R inv = R(1) / b.v;
  R q = a.v * inv;
  return Dual<R>(q, (a.d - q * b.d) * inv);
}
template <class R> __device__ __forceinline__ Dual<R> operator+(Dual<R> a, R b) { return Dual<R>(a.v + b, a.d); }
template <class R> __device__ __forceinline__ Dual<R> operator+(R a, Dual<R> b) { return Dual<R>(a + b.v, b.d); }
template <class R> __device__ __forceinline__ Dual<R> operator-(Dual<R> a, R b) { return Dual<R>(a.v - b, a.d); }
template <class R> __device__ __forceinline__ Dual<R> operator-(R a, Dual<R> b) { return Dual<R>(a - b.v, -b.d); }
template <class R> __device__ __forceinline__ Dual<R> operator*(Dual<R> a, R b) { return Dual<R>(a.v * b, a.d * b); }
template <class R> __device__ __forceinline__ Dual<R> operator*(R a, Dual<R> b) { return Dual<R>(a * b.v, a * b.d); }
template <class R> __device__ __forceinline__ Dual<R> operator/(Dual<R> a, R b) { R i = R(1) / b; return Dual<R>(a.v * i, a.d * i); }
template <class R> __device__ __forceinline__ Dual<R> operator/(R a, Dual<R> b) {
  R i = R(1) / b.v;
  R q = a * i;
  return Dual<R>(q, -q * b.d * i);
}
template <class R> __device__ __forceinline__ Dual<R>& operator+=(Dual<R>& a, Dual<R> b) { a.v += b.v; a.d += b.d; return a; }
template <class R> __device__ __forceinline__ Dual<R>& operator-=(Dual<R>& a, Dual<R> b) { a.v -= b.v; a.d -= b.d; return a; }
__device__ __forceinline__ double dsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ float dsqrt(float a) { return sqrtf(a); }
// (the real part goes through the overloads above, so an FP32 instance stays in FP32)
template <class R> __device__ __forceinline__ Dual<R> dsqrt(Dual<R> a) {
  R s = dsqrt(a.v);
  return Dual<R>(s, a.d / (R(2) * s));
}

// Dual numbers with K tangents: the derivative along K directions in one evaluation
// (the element-diagonal block extraction seeds K unit columns at once).
template <class R, int K> struct DualK {
  R v, d[K];
  __host__ __device__ DualK() {}
  __host__ __device__ DualK(R a) : v(a) {
#pragma unroll
    for (int i = 0; i < K; ++i) d[i] = R(0);
  }
};
#define LDG_DK template <class R, int K> __device__ __forceinline__ DualK<R, K>
LDG_DK operator+(DualK<R, K> a, DualK<R, K> b) {
  a.v += b.v;
#pragma unroll
  for (int i = 0; i < K; ++i) a.d[i] += b.d[i];
  return a;
}
LDG_DK operator-(DualK<R, K> a, DualK<R, K> b) {
  a.v -= b.v;
#pragma unroll
  for (int i = 0; i < K; ++i) a.d[i] -= b.d[i];
  return a;
}
LDG_DK operator-(DualK<R, K> a) {
  a.v = -a.v;
#pragma unroll
  for (int i = 0; i < K; ++i) a.d[i] = -a.d[i];
  return a;
}
LDG_DK operator*(DualK<R, K> a, DualK<R, K> b) {
  DualK<R, K> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
LDG_DK operator/(DualK<R, K> a, DualK<R, K> b) {
  const R inv = R(1) / b.v;
  DualK<R, K> r;
  r.v = a.v * inv;
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * inv;
  return r;
}
LDG_DK operator+(DualK<R, K> a, R b) { a.v += b; return a; }
LDG_DK operator+(R a, DualK<R, K> b) { b.v += a; return b; }
LDG_DK operator-(DualK<R, K> a, R b) { a.v -= b; return a; }
LDG_DK operator-(R a, DualK<R, K> b) { return DualK<R, K>(a) - b; }
LDG_DK operator*(DualK<R, K> a, R b) {
  a.v *= b;
#pragma unroll
  for (int i = 0; i < K; ++i) a.d[i] *= b;
  return a;
}
LDG_DK operator*(R a, DualK<R, K> b) { return b * a; }
LDG_DK operator/(DualK<R, K> a, R b) { return a * (R(1) / b); }
LDG_DK operator/(R a, DualK<R, K> b) { return DualK<R, K>(a) / b; }
template <class R, int K> __device__ __forceinline__ DualK<R, K>& operator+=(DualK<R, K>& a, DualK<R, K> b) {
  a = a + b;
  return a;
}
template <class R, int K> __device__ __forceinline__ DualK<R, K>& operator-=(DualK<R, K>& a, DualK<R, K> b) {
  a = a - b;
  return a;
}
LDG_DK dsqrt(DualK<R, K> a) {
  DualK<R, K> r;
  r.v = dsqrt(a.v);
  const R h = R(1) / (R(2) * r.v);
#pragma unroll
  for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * h;
  return r;
}
#undef LDG_DK

template <class S> struct RealOf { typedef S type; };
template <class R> struct RealOf<Dual<R>> { typedef R type; };
template <class R, int K> struct RealOf<DualK<R, K>> { typedef R type; };

__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ float val(float x) { return x; }
template <class R> __device__ __forceinline__ R val(Dual<R> x) { return x.v; }
template <class R, int K> __device__ __forceinline__ R val(const DualK<R, K>& x) { return x.v; }
// The part of a scalar a kernel writes out: the tangent for dual numbers, else the value.
__device__ __forceinline__ double outp(double x) { return x; }
__device__ __forceinline__ float outp(float x) { return x; }
template <class R> __device__ __forceinline__ R outp(Dual<R> x) { return x.d; }

// |x| with d|x| = 0 at x = 0; max(a, b) takes a on a tie (the element's own side).
template <class S> __device__ __forceinline__ S sabs(S x) {
  auto r = val(x);
  return r > 0 ? x : (r < 0 ? -x : x * typename RealOf<S>::type(0));
}
template <class S> __device__ __forceinline__ S smax(S a, S b) { return val(a) >= val(b) ? a : b; }

constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// ----------------------------------------------------------------- models
enum { M_POISSON = 0, M_CONVDIFF = 1, M_EULER = 2, M_NS = 3 };
enum { C_ZERO = 0, C_SINSIN = 1, C_EXPSIN = 2, C_POLY2 = 3, C_LINEAR = 4, C_VORTEX = 5, C_CONST = 6,
       C_ROTATION = 7, C_CYLINDER = 8, C_REST = 9, C_CYLINDER_START = 10 };

// kappa: diffusivity, or the dynamic viscosity 1/Re of Navier-Stokes; tau: the
// LDG jump penalty; pr: the Prandtl number (Navier-Stokes)
struct ModelParams {
  double kappa, tau, beta[3], gamma, pr;
  int cas;
};

// Exact solution / boundary data and source of the manufactured and analytic cases.
template <int DIM>
__device__ void exact_state(const ModelParams& mp, int ncu, const double* x, double t, double* g) {
  const double PI = 3.141592653589793238462643;
  if (ncu == 4) {
    if (mp.cas == C_VORTEX) {
      // isentropic vortex of strength 5 centred at (5,5) + t (1,1) on the periodic [0,10]^2
      double dx = x[0] - 5.0 - t, dy = x[1] - 5.0 - t;
      dx -= 10.0 * floor(dx / 10.0 + 0.5);
      dy -= 10.0 * floor(dy / 10.0 + 0.5);
      double ex = exp(0.5 * (1.0 - dx * dx - dy * dy));
      double k = 5.0 / (2.0 * PI) * ex;
      double ux = 1.0 - k * dy, uy = 1.0 + k * dx;
      double gm = mp.gamma;
      double T = 1.0 - (gm - 1.0) * 25.0 / (8.0 * gm * PI * PI) * ex * ex;
      double rho = pow(T, 1.0 / (gm - 1.0));
      double p = pow(rho, gm);
      g[0] = rho; g[1] = rho * ux; g[2] = rho * uy;
      g[3] = p / (gm - 1.0) + 0.5 * rho * (ux * ux + uy * uy);
    } else if (mp.cas == C_ROTATION) {
      // rigid rotation v = (-y, x) / 2, density 1 + x / 10 + y / 20, internal energy 2:
      // zero strain rate and zero temperature gradient, so no viscous stress or heat flux
      const double rho = 1.0 + 0.1 * x[0] + 0.05 * x[1], ux = -0.5 * x[1], uy = 0.5 * x[0];
      g[0] = rho; g[1] = rho * ux; g[2] = rho * uy; g[3] = rho * (2.0 + 0.5 * (ux * ux + uy * uy));
    } else if (mp.cas == C_CYLINDER) {
      // cylinder free stream: rho = 1, v = (1, 0), Mach 0.2
      const double p = 1.0 / (mp.gamma * 0.04);
      g[0] = 1.0; g[1] = 1.0; g[2] = 0.0; g[3] = p / (mp.gamma - 1.0) + 0.5;
    } else if (mp.cas == C_CYLINDER_START) {
      // start of the cylinder flow: free stream with velocity tanh((r - 0.5) / 0.1)
      const double p = 1.0 / (mp.gamma * 0.04), r = sqrt(x[0] * x[0] + x[1] * x[1]);
      const double vx = tanh((r - 0.5) / 0.1);
      g[0] = 1.0; g[1] = vx; g[2] = 0.0; g[3] = p / (mp.gamma - 1.0) + 0.5 * vx * vx;
    } else if (mp.cas == C_REST) {
      g[0] = 1.0; g[1] = 0.0; g[2] = 0.0; g[3] = 1.0 / (mp.gamma - 1.0);
    } else {
      g[0] = 1.0; g[1] = 1.0; g[2] = 1.0; g[3] = 1.0 / (mp.gamma - 1.0) + 1.0;
    }
    return;
  }
  double u = 0.0;
  switch (mp.cas) {
    case C_SINSIN: { u = 1.0; for (int d = 0; d < DIM; ++d) u *= sin(PI * x[d]); break; }
    case C_EXPSIN: {
      double s = 0.0, pr = 1.0;
      for (int d = 0; d < DIM; ++d) { s += x[d]; pr *= x[d]; }
      u = exp(s) * sin(PI * pr);
      break;
    }
    case C_POLY2: {
      double X = x[0], Y = x[1];
      u = 1.0 + 0.5 * X - 0.3 * Y + 0.7 * X * Y - 0.4 * X * X + 0.2 * Y * Y;
      if (DIM == 3) { double Z = x[DIM - 1]; u += 0.25 * Z + 0.1 * X * Z - 0.35 * Z * Z; }
      break;
    }
    case C_LINEAR: {
      const double a[3] = {0.5, -0.3, 0.25};
      u = 1.0;
      for (int d = 0; d < DIM; ++d) u += a[d] * x[d];
      break;
    }
    default: u = 0.0;
  }
  g[0] = u;
}

// Gradient and Laplacian of the exact solution of the scalar cases.
template <int DIM>
__device__ void scalar_derivs(const ModelParams& mp, const double* x, double* grad, double& lap) {
  const double PI = 3.141592653589793238462643;
  grad[0] = grad[1] = grad[2] = 0.0;
  lap = 0.0;
  switch (mp.cas) {
    case C_SINSIN: {
      double sn[3], cs[3];
      for (int d = 0; d < DIM; ++d) { sn[d] = sin(PI * x[d]); cs[d] = cos(PI * x[d]); }
      double u = 1.0;
      for (int d = 0; d < DIM; ++d) u *= sn[d];
      for (int k = 0; k < DIM; ++k) {
        double g = PI * cs[k];
        for (int d = 0; d < DIM; ++d) if (d != k) g *= sn[d];
        grad[k] = g;
      }
      lap = -DIM * PI * PI * u;
      break;
    }
    case C_EXPSIN: {
      double s = 0.0, pr = 1.0;
      for (int d = 0; d < DIM; ++d) { s += x[d]; pr *= x[d]; }
      double E = exp(s), S = sin(PI * pr), C = cos(PI * pr);
      for (int k = 0; k < DIM; ++k) {
        double m = 1.0;
        for (int d = 0; d < DIM; ++d) if (d != k) m *= x[d];
        grad[k] = E * (S + PI * m * C);
        lap += E * (S + 2.0 * PI * m * C - PI * PI * m * m * S);
      }
      break;
    }
    case C_POLY2: {
      double X = x[0], Y = x[1];
      grad[0] = 0.5 + 0.7 * Y - 0.8 * X;
      grad[1] = -0.3 + 0.7 * X + 0.4 * Y;
      lap = -0.4;
      if (DIM == 3) {
        double Z = x[DIM - 1];
        grad[0] += 0.1 * Z;
        grad[DIM - 1] = 0.25 + 0.1 * X - 0.7 * Z;
        lap -= 0.7;
      }
      break;
    }
    case C_LINEAR: { grad[0] = 0.5; grad[1] = -0.3; if (DIM == 3) grad[DIM - 1] = 0.25; break; }
    default: break;
  }
}

// Source s of Eq. 1b such that div(beta u - kappa grad u) = s for the scalar cases.
template <int DIM>
__device__ double source_term(const ModelParams& mp, bool conv, const double* x) {
  double grad[3], lap;
  scalar_derivs<DIM>(mp, x, grad, lap);
  double bg = 0.0;
  if (conv) for (int d = 0; d < DIM; ++d) bg += mp.beta[d] * grad[d];
  return bg - mp.kappa * lap;
}

// Model parameters in the kernel's compute precision.
template <class R> struct MPar {
  R kappa, tau, beta[3], gamma, pr;
};
template <class R> __device__ __forceinline__ MPar<R> mpar(const ModelParams& mp) {
  MPar<R> r;
  r.kappa = R(mp.kappa); r.tau = R(mp.tau); r.gamma = R(mp.gamma); r.pr = R(mp.pr);
  for (int d = 0; d < 3; ++d) r.beta[d] = R(mp.beta[d]);
  return r;
}

// Scalar diffusion models: f = kappa q (Poisson) or beta u + kappa q (convection-diffusion).
template <int DIM, bool CONV> struct ScalarModel {
  static constexpr int NCU = 1;
  static constexpr bool HASQ = true;
  static constexpr bool LINEAR = true;
  static constexpr bool SOURCE = true;   // manufactured source s of Eq. 1b
  static constexpr int KIND = CONV ? M_CONVDIFF : M_POISSON;

  template <class S, class R> __device__ static void flux(const S* u, const S* q, S* f, const MPar<R>& mp) {
    for (int d = 0; d < DIM; ++d) {
      S v = q[d] * mp.kappa;
      if (CONV) v = v + u[0] * mp.beta[d];
      f[d] = v;
    }
  }
  // interior numerical flux: upwind convection, central diffusion plus tau jump
  template <class S, class R> __device__ static void fhat(const S* um, const S* up, const S* qm, const S* qp,
                                                          const R* n, S* fh, const MPar<R>& mp) {
    S acc = (um[0] - up[0]) * mp.tau;
    for (int d = 0; d < DIM; ++d) acc = acc + (qm[d] + qp[d]) * (R(0.5) * mp.kappa * n[d]);
    if (CONV) {
      R bn = R(0);
      for (int d = 0; d < DIM; ++d) bn += mp.beta[d] * n[d];
      acc = acc + (bn >= R(0) ? um[0] : up[0]) * bn;
    }
    fh[0] = acc;
  }
  // Dirichlet face: uhat = g; fhat = beta.n u_upwind + kappa q-.n + tau (u- - g)
  template <class S, class R> __device__ static void fhat_bnd(const S* um, const S* qm, const R* g, const R* n,
                                                              S* fh, const MPar<R>& mp) {
    S acc = (um[0] - g[0]) * mp.tau;
    for (int d = 0; d < DIM; ++d) acc = acc + qm[d] * (mp.kappa * n[d]);
    if (CONV) {
      R bn = R(0);
      for (int d = 0; d < DIM; ++d) bn += mp.beta[d] * n[d];
      acc = acc + (bn >= R(0) ? um[0] * bn : S(bn * g[0]));
    }
    fh[0] = acc;
  }
};

// 2-D compressible Euler with the local Lax-Friedrichs (Rusanov) flux.
struct EulerModel {
  static constexpr int NCU = 4;
  static constexpr bool HASQ = false;
  static constexpr bool LINEAR = false;
  static constexpr bool SOURCE = false;
  static constexpr int KIND = M_EULER;

  template <class S, class R> __device__ static void flux(const S* u, const S*, S* f, const MPar<R>& mp) {
    S ir = R(1) / u[0];
    S vx = u[1] * ir, vy = u[2] * ir;
    S p = (u[3] - (u[1] * vx + u[2] * vy) * R(0.5)) * (mp.gamma - R(1));
    S h = u[3] + p;
    f[0] = u[1];           f[1] = u[2];
    f[2] = u[1] * vx + p;  f[3] = u[1] * vy;
    f[4] = u[2] * vx;      f[5] = u[2] * vy + p;
    f[6] = h * vx;         f[7] = h * vy;
  }
  template <class S, class R> __device__ static S normal_flux(const S* u, const R* n, S* fn, const MPar<R>& mp) {
    S ir = R(1) / u[0];
    S vx = u[1] * ir, vy = u[2] * ir;
    S p = (u[3] - (u[1] * vx + u[2] * vy) * R(0.5)) * (mp.gamma - R(1));
    S vn = vx * n[0] + vy * n[1];
    fn[0] = u[0] * vn;
    fn[1] = u[1] * vn + p * n[0];
    fn[2] = u[2] * vn + p * n[1];
    fn[3] = (u[3] + p) * vn;
    S c = dsqrt(p * ir * mp.gamma);
    return sabs(vn) + c;
  }
  template <class S, class R> __device__ static void fhat(const S* um, const S* up, const S*, const S*,
                                                          const R* n, S* fh, const MPar<R>& mp) {
    S fm[4], fp[4];
    S lm = normal_flux(um, n, fm, mp);
    S lp = normal_flux(up, n, fp, mp);
    S lam = smax(lm, lp);
    for (int c = 0; c < 4; ++c) fh[c] = (fm[c] + fp[c]) * R(0.5) + lam * R(0.5) * (um[c] - up[c]);
  }
  // far field: Rusanov flux against the exact state
  template <class S, class R> __device__ static void fhat_bnd(const S* um, const S* qm, const R* g, const R* n,
                                                              S* fh, const MPar<R>& mp) {
    S up[4] = {S(g[0]), S(g[1]), S(g[2]), S(g[3])};
    fhat(um, up, qm, qm, n, fh, mp);
  }
  // solid wall: the physical flux of the wall state (rho-, 0, 0, (rho E)-), i.e. the
  // pressure (gamma - 1) (rho E)- on the momentum components only
  template <class S, class R> __device__ static void fhat_wall(const S* um, const S*, const R* n, S* fh,
                                                               const MPar<R>& mp) {
    const S p = um[3] * (mp.gamma - R(1));
    fh[0] = um[0] * R(0);
    fh[1] = p * n[0];
    fh[2] = p * n[1];
    fh[3] = um[3] * R(0);
  }
};

// 2-D compressible Navier-Stokes (Section 2.1): f = F(u) - F_v(u, grad u), the
// viscous flux taken from q = -grad u of Eq. 1a (LDG). Interior faces: the Euler
// Rusanov flux, minus the central average of F_v.n, plus the jump penalty
// tau (u- - u+); far-field faces: the same against the exact state with the
// one-sided F_v(u-, q-).n and tau (u- - g).
struct NSModel {
  static constexpr int NCU = 4;
  static constexpr bool HASQ = true;
  static constexpr bool LINEAR = false;
  static constexpr bool SOURCE = false;
  static constexpr int KIND = M_NS;

  // F_v[c * 2 + d] with grad u = -q: Stokes stress with bulk viscosity -2/3 mu and
  // Fourier heat flux mu gamma / Pr grad e, e = E / rho - |v|^2 / 2 the internal energy
  // (temperature in units of c_v); velocity and energy gradients by the chain rule.
  template <class S, class R> __device__ static void viscous(const S* u, const S* q, S* fv, const MPar<R>& mp) {
    const S ir = R(1) / u[0];
    const S vx = u[1] * ir, vy = u[2] * ir, E = u[3] * ir;
    const S vxx = (vx * q[0] - q[2]) * ir, vxy = (vx * q[1] - q[3]) * ir;   // d v_x / d x_d
    const S vyx = (vy * q[0] - q[4]) * ir, vyy = (vy * q[1] - q[5]) * ir;   // d v_y / d x_d
    const S dv = vxx + vyy;
    const S txx = (vxx * R(2) - dv * R(2.0 / 3.0)) * mp.kappa;
    const S tyy = (vyy * R(2) - dv * R(2.0 / 3.0)) * mp.kappa;
    const S txy = (vxy + vyx) * mp.kappa;
    const S ex = (E * q[0] - q[6]) * ir - (vx * vxx + vy * vyx);
    const S ey = (E * q[1] - q[7]) * ir - (vx * vxy + vy * vyy);
    const R kt = mp.kappa * mp.gamma / mp.pr;
    fv[0] = S(R(0)); fv[1] = S(R(0));
    fv[2] = txx;     fv[3] = txy;
    fv[4] = txy;     fv[5] = tyy;
    fv[6] = vx * txx + vy * txy + ex * kt;
    fv[7] = vx * txy + vy * tyy + ey * kt;
  }
  template <class S, class R> __device__ static void flux(const S* u, const S* q, S* f, const MPar<R>& mp) {
    S fv[8];
    EulerModel::flux(u, q, f, mp);
    viscous(u, q, fv, mp);
#pragma unroll
    for (int i = 0; i < 8; ++i) f[i] = f[i] - fv[i];
  }
  template <class S, class R> __device__ static void fhat(const S* um, const S* up, const S* qm, const S* qp,
                                                          const R* n, S* fh, const MPar<R>& mp) {
    S vm[8], vp[8];
    EulerModel::fhat(um, up, qm, qp, n, fh, mp);
    viscous(um, qm, vm, mp);
    viscous(up, qp, vp, mp);
#pragma unroll
    for (int c = 0; c < 4; ++c)
      fh[c] = fh[c] - ((vm[2 * c] + vp[2 * c]) * n[0] + (vm[2 * c + 1] + vp[2 * c + 1]) * n[1]) * R(0.5) +
              (um[c] - up[c]) * mp.tau;
  }
  template <class S, class R> __device__ static void fhat_bnd(const S* um, const S* qm, const R* g, const R* n,
                                                              S* fh, const MPar<R>& mp) {
    S vm[8];
    EulerModel::fhat_bnd(um, qm, g, n, fh, mp);
    viscous(um, qm, vm, mp);
#pragma unroll
    for (int c = 0; c < 4; ++c) fh[c] = fh[c] - (vm[2 * c] * n[0] + vm[2 * c + 1] * n[1]) + (um[c] - g[c]) * mp.tau;
  }
  // no-slip adiabatic wall: wall state ub = (rho-, 0, 0, (rho E)-); pressure flux,
  // minus the viscous momentum flux F_v(ub, q-).n (no energy flux: zero velocity and
  // zero heat flux), plus the penalty tau (u- - ub) on the momentum
  template <class S, class R> __device__ static void fhat_wall(const S* um, const S* qm, const R* n, S* fh,
                                                               const MPar<R>& mp) {
    const S z = um[0] * R(0);
    S ub[4] = {um[0], z, z, um[3]}, vb[8];
    EulerModel::fhat_wall(um, qm, n, fh, mp);
    viscous(ub, qm, vb, mp);
#pragma unroll
    for (int c = 1; c < 3; ++c) fh[c] = fh[c] - (vb[2 * c] * n[0] + vb[2 * c + 1] * n[1]) + um[c] * mp.tau;
  }
};

// -------------------------------------------------------- element traits
// Operator blob (row-major, one FP64 and one FP32 copy per context) shared by all elements:
//   tensor: B[NQ][N1], D[NQ][N1], W[NQ], XQ[NQ], Dn[N1][N1], Minv1[N1][N1], XN[N1]
//   triangle: B[NQV][NPE], Dr[NQV][NPE], Ds[NQV][NPE], WV[NQV], XQV[NQV][2],
//             Bf[NFQ][NFN], WF[NFQ], SF[NFQ], Dnr[NPE][NPE], Dns[NPE][NPE], Minv[NPE][NPE], XN[NPE][2]
template <int DIM_, int P_, int NQ_> struct TensorEl {
  static constexpr bool TENSOR = true;
  static constexpr bool CURVED = false;   // affine (parallelogram / parallelepiped) geometry
  static constexpr bool NODE_PERM = false;
  static constexpr int DIM = DIM_, P = P_, N1 = P_ + 1, NQ = NQ_;
  static constexpr int NPE = ipow(N1, DIM), NQV = ipow(NQ, DIM);
  static constexpr int NF = 2 * DIM, NFN = ipow(N1, DIM - 1), NFQ = ipow(NQ, DIM - 1);
  // blob offsets
  static constexpr int OB = 0, OD = OB + NQ * N1, OW = OD + NQ * N1, OXQ = OW + NQ, ODN = OXQ + NQ,
                       OMI = ODN + N1 * N1, OXN = OMI + N1 * N1, OPS = OXN + N1;
  // local node of face-node j on face f = 2*axis + side (free axes ascending, first fastest)
  __device__ static int face_node(int f, int j) {
    int ax = f >> 1, side = f & 1;
    int fix = side ? N1 - 1 : 0;
    int idx[3], m = 0, jj = j;
    for (int d = 0; d < DIM; ++d) {
      if (d == ax) idx[d] = fix;
      else { idx[d] = (m == 0) ? (jj % N1) : (jj / N1); ++m; }
    }
    int r = idx[0] + N1 * idx[1];
    if (DIM == 3) r += N1 * N1 * idx[2];
    return r;
  }
};

// Curved quadrilateral: the tensor element's reference operators with per-point
// geometry (the element map has its own degree; its metrics are sampled at the
// quadrature points on the host).
template <int P_, int NQ_> struct CurvedQuadEl : TensorEl<2, P_, NQ_> {
  static constexpr bool CURVED = true;
};

template <int P_, int NQ_> struct TriEl {
  static constexpr bool TENSOR = false;
  static constexpr bool CURVED = false;
  static constexpr bool NODE_PERM = false;   // neighbour traces matched by face-point permutation
  static constexpr int DIM = 2, P = P_, NQ = NQ_, N1 = P_ + 1;
  static constexpr int NPE = (P_ + 1) * (P_ + 2) / 2, NQV = NQ_ * NQ_;
  static constexpr int NF = 3, NFN = P_ + 1, NFQ = NQ_;
  static constexpr int OB = 0, ODR = OB + NQV * NPE, ODS = ODR + NQV * NPE, OWV = ODS + NQV * NPE,
                       OXQ = OWV + NQV, OBF = OXQ + 2 * NQV, OWF = OBF + NFQ * NFN, OSF = OWF + NFQ,
                       ODNR = OSF + NFQ, ODNS = ODNR + NPE * NPE, OMI = ODNS + NPE * NPE,
                       OXN = OMI + NPE * NPE, OPS = OXN + 2 * NPE;
  static constexpr int ODT = 0, ODNT = 0;    // (no third axis)
  // node (i, j), i + j <= P, numbered row by row: j (P+1) - j (j-1)/2 + i
  __device__ static int nidx(int i, int j) { return j * (P + 1) - j * (j - 1) / 2 + i; }
  // edge nodes in the direction of the edge: f0 v0->v1, f1 v1->v2, f2 v2->v0
  __device__ static int face_node(int f, int t) {
    if (f == 0) return nidx(t, 0);
    if (f == 1) return nidx(P - t, t);
    return nidx(0, P - t);
  }
};

// Curved triangle: the triangle's reference operators with per-point geometry (the
// element map has its own degree; its metrics are sampled at the collapsed Gauss
// points on the host).
template <int P_, int NQ_> struct CurvedTriEl : TriEl<P_, NQ_> {
  static constexpr bool CURVED = true;
};

// Tetrahedron with equispaced nodes (i, j, k), i + j + k <= P, numbered k outer, then
// j, then i; vertices V0 = (-1,-1,-1), V1 = (1,-1,-1), V2 = (-1,1,-1), V3 = (-1,-1,1);
// face f lies opposite vertex f, with vertices (A, B, C) = (1,2,3), (0,2,3), (0,1,3),
// (0,1,2) and face node (a, b) at V_A + a (V_B - V_A) / P + b (V_C - V_A) / P.
// Full-matrix reference operators; faces carry the collapsed Gauss rule in their own
// parameters, which is not symmetric, so a neighbour's trace is formed from its face
// nodes permuted into this element's face-node order (NODE_PERM).
template <int P_, int NQ_> struct TetEl {
  static constexpr bool TENSOR = false;
  static constexpr bool CURVED = false;
  static constexpr bool NODE_PERM = true;
  static constexpr int DIM = 3, P = P_, NQ = NQ_, N1 = P_ + 1;
  static constexpr int NPE = (P_ + 1) * (P_ + 2) * (P_ + 3) / 6, NQV = NQ_ * NQ_ * NQ_;
  static constexpr int NF = 4, NFN = (P_ + 1) * (P_ + 2) / 2, NFQ = NQ_ * NQ_;
  static constexpr int OB = 0, ODR = OB + NQV * NPE, ODS = ODR + NQV * NPE, ODT = ODS + NQV * NPE,
                       OWV = ODT + NQV * NPE, OXQ = OWV + NQV, OBF = OXQ + 3 * NQV, OWF = OBF + NFQ * NFN,
                       OSF = OWF + NFQ, ODNR = OSF + 2 * NFQ, ODNS = ODNR + NPE * NPE, ODNT = ODNS + NPE * NPE,
                       OMI = ODNT + NPE * NPE, OXN = OMI + NPE * NPE, OPS = OXN + 3 * NPE;
  // node (i, j, k): the layers below k hold sum_{k' < k} (P - k' + 1)(P - k' + 2) / 2 nodes
  __host__ __device__ static int nidx(int i, int j, int k) {
    int off = 0;
    for (int kk = 0; kk < k; ++kk) off += (P - kk + 1) * (P - kk + 2) / 2;
    const int q = P - k;
    return off + j * (q + 1) - j * (j - 1) / 2 + i;
  }
  // barycentric lattice coordinates of node n: l[0] = P - i - j - k, l[1..3] = (i, j, k)
  __host__ __device__ static void lattice(int n, int* l) {
    int k = 0, rem = n;
    while (rem >= (P - k + 1) * (P - k + 2) / 2) { rem -= (P - k + 1) * (P - k + 2) / 2; ++k; }
    const int q = P - k;
    int j = 0;
    while (rem > q - j) { rem -= q + 1 - j; ++j; }
    l[1] = rem; l[2] = j; l[3] = k; l[0] = P - rem - j - k;
  }
  __host__ __device__ static void face_verts(int f, int& A, int& B, int& C) {
    A = f == 0 ? 1 : 0;
    B = f <= 1 ? 2 : 1;
    C = f == 3 ? 2 : 3;
  }
  // local node of face-node jf = b (P + 1) - b (b - 1) / 2 + a on face f
  __host__ __device__ static int face_node(int f, int jf) {
    int b = 0, a = jf;
    while (a > P - b) { a -= P + 1 - b; ++b; }
    int A, B, C;
    face_verts(f, A, B, C);
    int l[4] = {0, 0, 0, 0};
    l[A] = P - a - b; l[B] = a; l[C] = b;
    return nidx(l[1], l[2], l[3]);
  }
};

// ---------------------------------------------------------- contractions
// out[b][o] = sum_i M(o, i) in[b][i] along axis AX of a tensor of extents E0 x E1 x E2
// (first fastest), with M(o, i) = Mat[o * NI + i] or, if TRANS, Mat[i * MOUT + o].
// Every output (line) is owned by one thread, so ACC (+=) is race-free. Both forms sum
// over i in the same order, so they give the same bits.
template <int AX, int E0, int E1, int E2, int MOUT, bool TRANS, bool ACC, class T, class TM>
__device__ __forceinline__ void contract(const T* __restrict__ in, T* __restrict__ out,
                                         const TM* __restrict__ Mat, int nbatch) {
  constexpr int O0 = AX == 0 ? MOUT : E0, O1 = AX == 1 ? MOUT : E1, O2 = AX == 2 ? MOUT : E2;
  constexpr int OSZ = O0 * O1 * O2, ISZ = E0 * E1 * E2;
  constexpr int NI = AX == 0 ? E0 : (AX == 1 ? E1 : E2);
  constexpr int STR = AX == 0 ? 1 : (AX == 1 ? E0 : E0 * E1);       // input stride along AX
  constexpr int OSTR = AX == 0 ? 1 : (AX == 1 ? O0 : O0 * O1);      // output stride along AX
  if constexpr (sizeof(TM) == 8 && MOUT * NI > 16) {
    // FP64 operators beyond 4 x 4: one thread per output point (the line form's
    // register-held operator measured slower here)
    const int total = nbatch * OSZ;
    for (int it = threadIdx.x; it < total; it += blockDim.x) {
      const int b = it / OSZ, r = it - b * OSZ;
      const int o0 = r % O0, o1 = (r / O0) % O1, o2 = r / (O0 * O1);
      const int oa = AX == 0 ? o0 : (AX == 1 ? o1 : o2);
      const T* src = in + b * ISZ + (AX == 0 ? o1 * E0 + o2 * E0 * E1 : (AX == 1 ? o0 + o2 * E0 * E1 : o0 + o1 * E0));
      T acc = ACC ? out[it] : T(0);
#pragma unroll
      for (int i = 0; i < NI; ++i) acc += src[i * STR] * (TRANS ? Mat[i * MOUT + oa] : Mat[oa * NI + i]);
      out[it] = acc;
    }
    return;
  }
  // one thread per line along AX: the line's NI inputs are loaded once, the MOUT x NI
  // operator is held in registers, and all MOUT outputs of the line are produced
  constexpr int LPB = ISZ / NI;                                      // lines per batch item
  TM m[MOUT][NI];
#pragma unroll
  for (int o = 0; o < MOUT; ++o)
#pragma unroll
    for (int i = 0; i < NI; ++i) m[o][i] = TRANS ? Mat[i * MOUT + o] : Mat[o * NI + i];
  const int total = nbatch * LPB;
  for (int it = threadIdx.x; it < total; it += blockDim.x) {
    const int b = it / LPB, r = it - b * LPB;
    // r enumerates the line's indices along the two other axes, the fastest first
    int ioff, ooff;
    if constexpr (AX == 0) {          // r = i1 + E1 i2
      ioff = r * E0;
      ooff = r * O0;
    } else if constexpr (AX == 1) {   // r = i0 + E0 i2
      const int i0 = r % E0, i2 = r / E0;
      ioff = i0 + i2 * E0 * E1;
      ooff = i0 + i2 * O0 * O1;
    } else {                          // r = i0 + E0 i1
      ioff = r;
      ooff = r;
    }
    const T* src = in + b * ISZ + ioff;
    T* dst = out + b * OSZ + ooff;
    T x[NI];
#pragma unroll
    for (int i = 0; i < NI; ++i) x[i] = src[i * STR];
#pragma unroll
    for (int o = 0; o < MOUT; ++o) {
      T acc = ACC ? dst[o * OSTR] : T(0);
#pragma unroll
      for (int i = 0; i < NI; ++i) acc += x[i] * m[o][i];
      dst[o * OSTR] = acc;
    }
  }
}

// out[b][o] = sum_i Mat[o][i] in[b][i] (full matrix, NO x NI), or transposed.
// The batch index runs fastest across the threads, so that a warp reads one (or a
// few) matrix entries per step, broadcast to its lanes, instead of up to 32 rows.
template <int NO, int NI, bool TRANS, bool ACC, class T, class TM>
__device__ __forceinline__ void matvec(const T* __restrict__ in, T* __restrict__ out,
                                       const TM* __restrict__ Mat, int nbatch) {
  const int total = nbatch * NO;
  for (int it = threadIdx.x; it < total; it += blockDim.x) {
    const int o = it / nbatch, b = it - o * nbatch, oi = b * NO + o;
    const T* src = in + b * NI;
    T acc = ACC ? out[oi] : T(0);
#pragma unroll 4
    for (int i = 0; i < NI; ++i) acc += src[i] * (TRANS ? Mat[i * NO + o] : Mat[o * NI + i]);
    out[oi] = acc;
  }
}

}  // namespace ldg
