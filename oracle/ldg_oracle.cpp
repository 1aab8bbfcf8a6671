// LDG oracle: a plain, slow, FP64 CPU implementation of the local discontinuous
// Galerkin discretisation of the first-order PDE system of Section 2.1 (Eq. 1a-1b)
// and of the matrix-free Newton-GMRES solve of Section 3.3.
//
// TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the benchmark's
// CPU-baseline leg load this library; the product path never does. It shares no
// code with the CUDA path. Every quantity is evaluated straight from its
// definition: basis functions are evaluated at each point from their formula,
// neighbour traces are found by mapping the physical quadrature point into the
// neighbour element, face normals come from the physical face vertices, and the
// element mass matrices are assembled and solved by dense LU. No sum
// factorisation, no tables shared between elements beyond the reference rules.
//
// Readings of the paper (it leaves numerical traces and fluxes to the user,
// Section 2.2):
//   q-stage (Eq. 1a, weak form on element K):
//     (q_d, phi)_K = (u_h, d_d phi)_K - <uhat n_d, phi>_dK
//   residual (Eq. 1b, weak form, steady part):
//     R_K = -(f(u_h,q_h), grad phi)_K + <fhat.n, phi>_dK - (s, phi)_K
//   time term (BDF1/BDF2) added as M (a0 u + a1 u^n + a2 u^{n-1}) / dt.
//   Interior traces: uhat = {u}; fhat.n = {f_c}.n + lambda/2 (u- - u+)
//     + kappa {q}.n + tau (u- - u+). lambda = |beta.n| (linear convection),
//     max(|v-.n|+c-, |v+.n|+c+) (Euler, local Lax-Friedrichs).
//   Dirichlet faces: uhat = g; fhat.n = beta.n u_up + kappa q-.n + tau (u- - g),
//     u_up = u- when beta.n >= 0 else g. Euler far field: Rusanov against the
//     exact state.
//   Navier-Stokes (2-D, conservative u = (rho, rho v, rho E), q = -grad u):
//     f = F(u) - Fv(u, grad u) with the Euler flux F, the Newtonian stress
//     tau_ij = mu (d_j v_i + d_i v_j) - 2/3 mu (div v) delta_ij, mu = 1/Re, and the
//     energy flux v.tau + (mu gamma / Pr) grad e (e = E - |v|^2 / 2, the internal
//     energy per unit mass); velocity and energy gradients follow from grad u by the
//     chain rule. Interior: Rusanov on F, central on Fv, penalty tau (u- - u+),
//     tau = 1/Re; far field: the same against the exact state, with Fv(u-, q-).
//   Non-differentiable points: d|x| at 0 is 0; max(a,b) with a == b is a.
//
// The residual is templated on the scalar type: double (R), Dual (exact
// forward-mode J.v, Section 3.3's AD option) and std::complex<double> (the
// complex-step Jacobian used as an independent pin of J.v).

#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <vector>

namespace {

typedef std::complex<double> cplx;

// ------------------------------------------------------------------ scalars
struct Dual {
  double v = 0.0, d = 0.0;
  Dual() {}
  Dual(double a) : v(a), d(0.0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
inline Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
inline Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
inline Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
inline Dual operator/(double a, Dual b) { return Dual(a / b.v, -a * b.d / (b.v * b.v)); }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}

inline double re(double x) { return x; }
inline double re(const Dual& x) { return x.v; }
inline double re(const cplx& x) { return x.real(); }

using std::sqrt;

// |x| with the convention d|x|/dx = 0 at x = 0 (branch on the real part).
template <class S> S absS(const S& x) {
  double r = re(x);
  if (r > 0) return x;
  if (r < 0) return -x;
  return x * 0.0;
}
// max(a, b); on a tie the first argument (the element's own side) is taken.
template <class S> S maxS(const S& a, const S& b) { return re(a) >= re(b) ? a : b; }

// ------------------------------------------------------- 1-D rules, Lagrange
// Legendre P_n and its first two derivatives by the three-term recurrence.
void legendre(int n, double x, double& P, double& dP, double& d2P) {
  double p0 = 1, p1 = x, dp0 = 0, dp1 = 1, ddp0 = 0, ddp1 = 0;
  if (n == 0) { P = 1; dP = 0; d2P = 0; return; }
  for (int k = 1; k < n; ++k) {
    double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    double dp2 = dp0 + (2 * k + 1) * p1;      // P'_{k+1} = P'_{k-1} + (2k+1) P_k
    double ddp2 = ddp0 + (2 * k + 1) * dp1;
    p0 = p1; p1 = p2; dp0 = dp1; dp1 = dp2; ddp0 = ddp1; ddp1 = ddp2;
  }
  P = p1; dP = dp1; d2P = ddp1;
}

// n-point Gauss-Legendre rule on [-1, 1].
void gauss_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0); w.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    double z = -std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP, d2P;
      legendre(n, z, P, dP, d2P);
      double dz = P / dP;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double P, dP, d2P;
    legendre(n, z, P, dP, d2P);
    x[i] = z;
    w[i] = 2.0 / ((1 - z * z) * dP * dP);
  }
}

// n1 Gauss-Lobatto-Legendre points: -1, the roots of P'_{n1-1}, +1.
void gll_points(int n1, std::vector<double>& x) {
  x.assign(n1, 0);
  int N = n1 - 1;
  x[0] = -1; x[N] = 1;
  for (int i = 1; i < N; ++i) {
    double z = -std::cos(M_PI * i / N);
    for (int it = 0; it < 100; ++it) {
      double P, dP, d2P;
      legendre(N, z, P, dP, d2P);
      double dz = dP / d2P;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
}

double lagrange(const std::vector<double>& X, int i, double x) {
  double v = 1;
  for (size_t j = 0; j < X.size(); ++j)
    if ((int)j != i) v *= (x - X[j]) / (X[i] - X[j]);
  return v;
}
double dlagrange(const std::vector<double>& X, int i, double x) {
  double s = 0;
  for (size_t m = 0; m < X.size(); ++m) {
    if ((int)m == i) continue;
    double t = 1.0 / (X[i] - X[m]);
    for (size_t j = 0; j < X.size(); ++j)
      if ((int)j != i && j != m) t *= (x - X[j]) / (X[i] - X[j]);
    s += t;
  }
  return s;
}

// Dense LU with partial pivoting (n x n, row-major), in place; piv receives row swaps.
bool lu_factor(std::vector<double>& A, int n, std::vector<int>& piv) {
  piv.assign(n, 0);
  for (int k = 0; k < n; ++k) {
    int pr = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > std::fabs(A[pr * n + k])) pr = i;
    piv[k] = pr;
    if (A[pr * n + k] == 0.0) return false;
    if (pr != k)
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[pr * n + j]);
    for (int i = k + 1; i < n; ++i) {
      A[i * n + k] /= A[k * n + k];
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= A[i * n + k] * A[k * n + j];
    }
  }
  return true;
}
template <class S>
void lu_solve(const std::vector<double>& LU, int n, const std::vector<int>& piv, S* b) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k) std::swap(b[k], b[piv[k]]);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) b[i] = b[i] - LU[i * n + j] * b[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) b[i] = b[i] - LU[i * n + j] * b[j];
    b[i] = b[i] / LU[i * n + i];
  }
}

// ------------------------------------------------------- reference elements
enum { TRI = 0, QUAD = 1, HEX = 2, TET = 3 };

struct Ref {
  int type, nd, p, npe, nv, nf, nq1, nfq;
  std::vector<double> gll;                       // tensor elements: 1-D nodes
  std::vector<std::array<double, 3>> node;       // reference node coordinates
  std::vector<std::array<int, 3>> mono;          // simplices: monomial exponents
  std::vector<double> coef;                      // simplices: phi_i = sum_m coef[m*npe+i] mono_m
  std::vector<std::array<double, 3>> qx;         // volume quadrature
  std::vector<double> qw;
  std::vector<std::array<double, 2>> fs;         // face quadrature (face parameter)
  std::vector<double> fw;
  std::vector<std::vector<int>> fverts;          // local vertices of each face
  std::vector<int> axisv;                        // vertex at the + end of each reference axis

  void init(int type_, int p_, int nq1_) {
    type = type_; p = p_; nq1 = nq1_;
    std::vector<double> gx, gw;
    gauss_rule(nq1, gx, gw);
    if (type == TRI) {
      nd = 2; nv = 3; nf = 3;
      npe = (p + 1) * (p + 2) / 2;
      for (int j = 0; j <= p; ++j)
        for (int i = 0; i + j <= p; ++i)
          node.push_back({-1.0 + 2.0 * i / p, -1.0 + 2.0 * j / p, 0.0});
      for (int a = 0; a <= p; ++a)
        for (int b = 0; a + b <= p; ++b) mono.push_back({a, b, 0});
      // phi_i is the unique degree-p polynomial with phi_i(node_j) = delta_ij:
      // coef = V^{-1}, V[j][m] = mono_m(node_j).
      std::vector<double> V(npe * npe);
      for (int j = 0; j < npe; ++j)
        for (int m = 0; m < npe; ++m)
          V[j * npe + m] = std::pow(node[j][0], mono[m][0]) * std::pow(node[j][1], mono[m][1]);   // 2-D
      std::vector<int> piv;
      lu_factor(V, npe, piv);
      coef.assign(npe * npe, 0.0);
      for (int i = 0; i < npe; ++i) {
        std::vector<double> e(npe, 0.0);
        e[i] = 1.0;
        lu_solve(V, npe, piv, e.data());
        for (int m = 0; m < npe; ++m) coef[m * npe + i] = e[m];
      }
      // collapsed (Duffy) Gauss rule on the reference triangle
      for (int jb = 0; jb < nq1; ++jb)
        for (int ia = 0; ia < nq1; ++ia) {
          double a = gx[ia], b = gx[jb];
          qx.push_back({(1 + a) * (1 - b) / 2 - 1, b, 0.0});
          qw.push_back(gw[ia] * gw[jb] * (1 - b) / 2);
        }
      for (int k = 0; k < nq1; ++k) { fs.push_back({gx[k], 0.0}); fw.push_back(gw[k]); }
      fverts = {{0, 1}, {1, 2}, {2, 0}};
      axisv = {1, 2};
    } else if (type == TET) {
      // reference tetrahedron with vertices (-1,-1,-1), (1,-1,-1), (-1,1,-1), (-1,-1,1)
      nd = 3; nv = 4; nf = 4;
      npe = (p + 1) * (p + 2) * (p + 3) / 6;
      for (int k = 0; k <= p; ++k)
        for (int j = 0; j + k <= p; ++j)
          for (int i = 0; i + j + k <= p; ++i)
            node.push_back({-1.0 + 2.0 * i / p, -1.0 + 2.0 * j / p, -1.0 + 2.0 * k / p});
      for (int a = 0; a <= p; ++a)
        for (int b = 0; a + b <= p; ++b)
          for (int c = 0; a + b + c <= p; ++c) mono.push_back({a, b, c});
      std::vector<double> V(npe * npe);
      for (int j = 0; j < npe; ++j)
        for (int m = 0; m < npe; ++m)
          V[j * npe + m] = std::pow(node[j][0], mono[m][0]) * std::pow(node[j][1], mono[m][1]) *
                           std::pow(node[j][2], mono[m][2]);
      std::vector<int> piv;
      lu_factor(V, npe, piv);
      coef.assign(npe * npe, 0.0);
      for (int i = 0; i < npe; ++i) {
        std::vector<double> e(npe, 0.0);
        e[i] = 1.0;
        lu_solve(V, npe, piv, e.data());
        for (int m = 0; m < npe; ++m) coef[m * npe + i] = e[m];
      }
      // collapsed (Duffy) Gauss rule: xi = (1+a)(1-b)(1-c)/4 - 1, eta = (1+b)(1-c)/2 - 1,
      // zeta = c, with Jacobian (1-b)(1-c)^2 / 8
      for (int kc = 0; kc < nq1; ++kc)
        for (int jb = 0; jb < nq1; ++jb)
          for (int ia = 0; ia < nq1; ++ia) {
            const double a = gx[ia], b = gx[jb], c = gx[kc];
            qx.push_back({(1 + a) * (1 - b) * (1 - c) / 4 - 1, (1 + b) * (1 - c) / 2 - 1, c});
            qw.push_back(gw[ia] * gw[jb] * gw[kc] * (1 - b) * (1 - c) * (1 - c) / 8);
          }
      // faces: the collapsed triangle rule in the face parameters (s, t) of the reference
      // triangle, face f opposite vertex f
      for (int jb = 0; jb < nq1; ++jb)
        for (int ia = 0; ia < nq1; ++ia) {
          const double a = gx[ia], b = gx[jb];
          fs.push_back({(1 + a) * (1 - b) / 2 - 1, b});
          fw.push_back(gw[ia] * gw[jb] * (1 - b) / 2);
        }
      fverts = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
      axisv = {1, 2, 3};
    } else {
      nd = (type == QUAD) ? 2 : 3;
      nv = 1 << nd; nf = 2 * nd;
      gll_points(p + 1, gll);
      int n1 = p + 1;
      npe = 1; for (int d = 0; d < nd; ++d) npe *= n1;
      for (int n = 0; n < npe; ++n) {
        int i = n % n1, j = (n / n1) % n1, k = n / (n1 * n1);
        node.push_back({gll[i], gll[j], nd == 3 ? gll[k] : 0.0});
      }
      int nqv = 1; for (int d = 0; d < nd; ++d) nqv *= nq1;
      for (int q = 0; q < nqv; ++q) {
        int i = q % nq1, j = (q / nq1) % nq1, k = q / (nq1 * nq1);
        qx.push_back({gx[i], gx[j], nd == 3 ? gx[k] : 0.0});
        qw.push_back(gw[i] * gw[j] * (nd == 3 ? gw[k] : 1.0));
      }
      if (nd == 2) {
        for (int k = 0; k < nq1; ++k) { fs.push_back({gx[k], 0.0}); fw.push_back(gw[k]); }
        // face f = 2*axis + side; vertices in lexicographic order
        fverts = {{0, 2}, {1, 3}, {0, 1}, {2, 3}};
        axisv = {1, 2};
      } else {
        for (int j = 0; j < nq1; ++j)
          for (int i = 0; i < nq1; ++i) { fs.push_back({gx[i], gx[j]}); fw.push_back(gw[i] * gw[j]); }
        fverts = {{0, 2, 4, 6}, {1, 3, 5, 7}, {0, 1, 4, 5}, {2, 3, 6, 7}, {0, 1, 2, 3}, {4, 5, 6, 7}};
        axisv = {1, 2, 4};
      }
    }
    nfq = (int)fs.size();
  }

  // Reference coordinates of face parameter s on face f.
  void face_xi(int f, const double* s, double* xi) const {
    if (type == TET) {
      static const double V[4][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
      const int A = fverts[f][0], B = fverts[f][1], C = fverts[f][2];
      for (int d = 0; d < 3; ++d)
        xi[d] = V[A][d] + 0.5 * (1 + s[0]) * (V[B][d] - V[A][d]) + 0.5 * (1 + s[1]) * (V[C][d] - V[A][d]);
      return;
    }
    if (type == TRI) {
      static const double V[3][2] = {{-1, -1}, {1, -1}, {-1, 1}};
      const int A = fverts[f][0], B = fverts[f][1];
      for (int d = 0; d < 2; ++d) xi[d] = 0.5 * (1 - s[0]) * V[A][d] + 0.5 * (1 + s[0]) * V[B][d];
      return;
    }
    int axis = f / 2, side = f % 2, m = 0;
    for (int d = 0; d < nd; ++d) {
      if (d == axis) xi[d] = side ? 1.0 : -1.0;
      else xi[d] = s[m++];
    }
  }

  // Basis values phi[i] and reference gradients dphi[i*nd + k] at reference point xi.
  void basis(const double* xi, double* phi, double* dphi) const {
    if (type == TET) {
      for (int i = 0; i < npe; ++i) { phi[i] = 0; dphi[3 * i] = 0; dphi[3 * i + 1] = 0; dphi[3 * i + 2] = 0; }
      for (int m = 0; m < npe; ++m) {
        const int a = mono[m][0], b = mono[m][1], c = mono[m][2];
        const double X = std::pow(xi[0], a), Y = std::pow(xi[1], b), Z = std::pow(xi[2], c);
        const double v = X * Y * Z;
        const double dx = a ? a * std::pow(xi[0], a - 1) * Y * Z : 0.0;
        const double dy = b ? b * X * std::pow(xi[1], b - 1) * Z : 0.0;
        const double dz = c ? c * X * Y * std::pow(xi[2], c - 1) : 0.0;
        for (int i = 0; i < npe; ++i) {
          const double cf = coef[m * npe + i];
          phi[i] += cf * v; dphi[3 * i] += cf * dx; dphi[3 * i + 1] += cf * dy; dphi[3 * i + 2] += cf * dz;
        }
      }
      return;
    }
    if (type == TRI) {
      for (int i = 0; i < npe; ++i) { phi[i] = 0; dphi[2 * i] = 0; dphi[2 * i + 1] = 0; }
      for (int m = 0; m < npe; ++m) {
        int a = mono[m][0], b = mono[m][1];
        double v = std::pow(xi[0], a) * std::pow(xi[1], b);
        double dx = a ? a * std::pow(xi[0], a - 1) * std::pow(xi[1], b) : 0.0;
        double dy = b ? b * std::pow(xi[0], a) * std::pow(xi[1], b - 1) : 0.0;
        for (int i = 0; i < npe; ++i) {
          double c = coef[m * npe + i];
          phi[i] += c * v; dphi[2 * i] += c * dx; dphi[2 * i + 1] += c * dy;
        }
      }
      return;
    }
    int n1 = p + 1;
    double L[3][16], dL[3][16];
    for (int d = 0; d < nd; ++d)
      for (int i = 0; i < n1; ++i) { L[d][i] = lagrange(gll, i, xi[d]); dL[d][i] = dlagrange(gll, i, xi[d]); }
    for (int n = 0; n < npe; ++n) {
      int id[3] = {n % n1, (n / n1) % n1, n / (n1 * n1)};
      double v = 1;
      for (int d = 0; d < nd; ++d) v *= L[d][id[d]];
      phi[n] = v;
      for (int k = 0; k < nd; ++k) {
        double g = 1;
        for (int d = 0; d < nd; ++d) g *= (d == k) ? dL[d][id[d]] : L[d][id[d]];
        dphi[n * nd + k] = g;
      }
    }
  }
};

// ------------------------------------------------------------------ models
enum { POISSON = 0, CONVDIFF = 1, EULER = 2, NS = 3 };
enum { CASE_ZERO = 0, CASE_SINSIN = 1, CASE_EXPSIN = 2, CASE_POLY2 = 3, CASE_LINEAR = 4,
       CASE_VORTEX = 5, CASE_CONST = 6, CASE_ROTATION = 7, CASE_CYLINDER = 8, CASE_REST = 9,
       CASE_CYLINDER_START = 10 };

struct Model {
  int kind, cas, nd, ncu;
  double kappa = 1, tau = 1, beta[3] = {0, 0, 0}, gamma = 1.4, pr = 0.72;   // NS: kappa = mu = 1/Re

  // exact solution u(x, t) for the manufactured / analytic cases
  void exact(const double* x, double t, double* u) const {
    if (kind == EULER || kind == NS) {
      if (cas == CASE_VORTEX) {
        // isentropic vortex: strength 5, centre (5,5), free stream rho = p = 1,
        // velocity (1,1), convected on the periodic square [0,10]^2.
        const double b = 5.0, L = 10.0;
        double dx = x[0] - 5.0 - t, dy = x[1] - 5.0 - t;
        dx -= L * std::floor(dx / L + 0.5);
        dy -= L * std::floor(dy / L + 0.5);
        double r2 = dx * dx + dy * dy;
        double e = std::exp(0.5 * (1 - r2));
        double vx = 1.0 - b / (2 * M_PI) * e * dy;
        double vy = 1.0 + b / (2 * M_PI) * e * dx;
        double T = 1.0 - (gamma - 1) * b * b / (8 * gamma * M_PI * M_PI) * e * e;
        double rho = std::pow(T, 1.0 / (gamma - 1));
        double pr = std::pow(rho, gamma);
        u[0] = rho; u[1] = rho * vx; u[2] = rho * vy;
        u[3] = pr / (gamma - 1) + 0.5 * rho * (vx * vx + vy * vy);
      } else if (cas == CASE_ROTATION) {
        // rigid rotation v = 0.5 (-y, x) with density 1 + 0.1 x + 0.05 y and uniform
        // internal energy e = 2: a cubic state with zero strain rate and zero grad e
        const double rho = 1.0 + 0.1 * x[0] + 0.05 * x[1], vx = -0.5 * x[1], vy = 0.5 * x[0];
        u[0] = rho; u[1] = rho * vx; u[2] = rho * vy; u[3] = rho * (2.0 + 0.5 * (vx * vx + vy * vy));
      } else if (cas == CASE_CYLINDER) {
        // free stream of the cylinder flow: rho = 1, v = (1, 0), Mach 0.2: p = 1 / (gamma 0.2^2)
        const double pr = 1.0 / (gamma * 0.04);
        u[0] = 1; u[1] = 1; u[2] = 0; u[3] = pr / (gamma - 1) + 0.5;
      } else if (cas == CASE_CYLINDER_START) {
        // start of the cylinder flow: the free stream with its velocity scaled by
        // tanh((r - 0.5) / 0.1), zero on the wall (pressure and density uniform)
        const double pr = 1.0 / (gamma * 0.04), r = std::sqrt(x[0] * x[0] + x[1] * x[1]);
        const double vx = std::tanh((r - 0.5) / 0.1);
        u[0] = 1; u[1] = vx; u[2] = 0; u[3] = pr / (gamma - 1) + 0.5 * vx * vx;
      } else if (cas == CASE_REST) {
        // gas at rest: rho = 1, v = 0, p = 1
        u[0] = 1; u[1] = 0; u[2] = 0; u[3] = 1.0 / (gamma - 1);
      } else {
        u[0] = 1; u[1] = 1; u[2] = 1; u[3] = 1.0 / (gamma - 1) + 1.0;
      }
      return;
    }
    double g[3];
    scalar_exact(x, u[0], g, nullptr);
  }
  // scalar cases: value, gradient and Laplacian
  void scalar_exact(const double* x, double& u, double* g, double* lap) const {
    double L = 0;
    for (int d = 0; d < 3; ++d) g[d] = 0;
    switch (cas) {
      case CASE_ZERO: u = 0; break;
      case CASE_SINSIN: {
        u = 1;
        for (int d = 0; d < nd; ++d) u *= std::sin(M_PI * x[d]);
        for (int k = 0; k < nd; ++k) {
          double v = M_PI * std::cos(M_PI * x[k]);
          for (int d = 0; d < nd; ++d) if (d != k) v *= std::sin(M_PI * x[d]);
          g[k] = v;
        }
        L = -nd * M_PI * M_PI * u;
        break;
      }
      case CASE_EXPSIN: {
        double s = 0, prod = 1;
        for (int d = 0; d < nd; ++d) { s += x[d]; prod *= x[d]; }
        double E = std::exp(s), S = std::sin(M_PI * prod), C = std::cos(M_PI * prod);
        u = E * S;
        for (int k = 0; k < nd; ++k) {
          double m = 1;
          for (int d = 0; d < nd; ++d) if (d != k) m *= x[d];
          g[k] = E * (S + M_PI * m * C);
          L += E * (S + 2 * M_PI * m * C - M_PI * M_PI * m * m * S);
        }
        break;
      }
      case CASE_POLY2: {
        // u = 1 + 0.5x - 0.3y + 0.25z + 0.7xy - 0.4x^2 + 0.2y^2 + 0.1xz - 0.35z^2
        double X = x[0], Y = x[1], Z = nd == 3 ? x[2] : 0.0;
        u = 1 + 0.5 * X - 0.3 * Y + 0.7 * X * Y - 0.4 * X * X + 0.2 * Y * Y;
        g[0] = 0.5 + 0.7 * Y - 0.8 * X;
        g[1] = -0.3 + 0.7 * X + 0.4 * Y;
        L = -0.8 + 0.4;
        if (nd == 3) {
          u += 0.25 * Z + 0.1 * X * Z - 0.35 * Z * Z;
          g[0] += 0.1 * Z;
          g[2] = 0.25 + 0.1 * X - 0.7 * Z;
          L += -0.7;
        }
        break;
      }
      case CASE_LINEAR: {
        const double a[3] = {0.5, -0.3, 0.25};
        u = 1;
        for (int d = 0; d < nd; ++d) { u += a[d] * x[d]; g[d] = a[d]; }
        break;
      }
      default: u = 0;
    }
    if (lap) *lap = L;
  }
  // source s(x) of Eq. 1b for the manufactured scalar cases: div f = s
  void source(const double* x, double* s) const {
    if (kind == EULER || kind == NS) { for (int c = 0; c < ncu; ++c) s[c] = 0; return; }
    double u, g[3], L;
    scalar_exact(x, u, g, &L);
    double bg = 0;
    if (kind == CONVDIFF) for (int d = 0; d < nd; ++d) bg += beta[d] * g[d];
    s[0] = bg - kappa * L;
  }

  // Euler flux F[c*2 + d](u)
  template <class S> void euler_flux(const S* u, S* f) const {
    S rho = u[0], vx = u[1] / rho, vy = u[2] / rho;
    S p = (gamma - 1) * (u[3] - 0.5 * (u[1] * vx + u[2] * vy));
    f[0] = u[1];          f[1] = u[2];
    f[2] = u[1] * vx + p; f[3] = u[1] * vy;
    f[4] = u[2] * vx;      f[5] = u[2] * vy + p;
    f[6] = (u[3] + p) * vx; f[7] = (u[3] + p) * vy;
  }

  // Navier-Stokes viscous flux Fv[c*2 + d](u, grad u) with grad u = -q
  template <class S> void viscous_flux(const S* u, const S* q, S* fv) const {
    const double mu = kappa;
    S rho = u[0], vx = u[1] / rho, vy = u[2] / rho, E = u[3] / rho;
    S g[4][2];
    for (int c = 0; c < 4; ++c)
      for (int d = 0; d < 2; ++d) g[c][d] = -q[c * 2 + d];
    // d v_i / d x_d = (d m_i / d x_d - v_i d rho / d x_d) / rho
    S vxx = (g[1][0] - vx * g[0][0]) / rho, vxy = (g[1][1] - vx * g[0][1]) / rho;
    S vyx = (g[2][0] - vy * g[0][0]) / rho, vyy = (g[2][1] - vy * g[0][1]) / rho;
    S dv = vxx + vyy;
    S txx = mu * (2.0 * vxx - (2.0 / 3.0) * dv);
    S tyy = mu * (2.0 * vyy - (2.0 / 3.0) * dv);
    S txy = mu * (vxy + vyx);
    // d e / d x_d = (d(rho E)/d x_d - E d rho / d x_d) / rho - v . d v / d x_d
    S ex = (g[3][0] - E * g[0][0]) / rho - (vx * vxx + vy * vyx);
    S ey = (g[3][1] - E * g[0][1]) / rho - (vx * vxy + vy * vyy);
    const double kt = mu * gamma / pr;
    fv[0] = 0.0; fv[1] = 0.0;
    fv[2] = txx; fv[3] = txy;
    fv[4] = txy; fv[5] = tyy;
    fv[6] = vx * txx + vy * txy + kt * ex;
    fv[7] = vx * txy + vy * tyy + kt * ey;
  }

  // physical flux f[c*nd + d](u, q): f = beta u + kappa q (q = -grad u), Euler, or
  // Navier-Stokes F(u) - Fv(u, grad u)
  template <class S> void flux(const S* u, const S* q, S* f) const {
    if (kind == EULER) { euler_flux(u, f); return; }
    if (kind == NS) {
      S fv[8];
      euler_flux(u, f);
      viscous_flux(u, q, fv);
      for (int i = 0; i < 8; ++i) f[i] = f[i] - fv[i];
      return;
    }
    for (int d = 0; d < nd; ++d) f[d] = kappa * q[d] + (kind == CONVDIFF ? beta[d] * u[0] : S(0.0));
  }

  // Euler normal wave speed |v.n| + c
  template <class S> S wave_speed(const S* u, const double* n) const {
    S rho = u[0], vx = u[1] / rho, vy = u[2] / rho;
    S pr = (gamma - 1) * (u[3] - 0.5 * (u[1] * vx + u[2] * vy));
    S c = sqrt(gamma * pr / rho);
    return absS(vx * n[0] + vy * n[1]) + c;
  }

  template <class S> void fhat_interior(const S* um, const S* up, const S* qm, const S* qp,
                                        const double* n, S* fh) const {
    if (kind == EULER || kind == NS) {
      S fm[8], fp[8];
      euler_flux(um, fm); euler_flux(up, fp);
      S lam = maxS(wave_speed(um, n), wave_speed(up, n));
      for (int c = 0; c < 4; ++c)
        fh[c] = 0.5 * ((fm[2 * c] + fp[2 * c]) * n[0] + (fm[2 * c + 1] + fp[2 * c + 1]) * n[1]) +
                0.5 * lam * (um[c] - up[c]);
      if (kind == NS) {
        S vm[8], vp[8];
        viscous_flux(um, qm, vm); viscous_flux(up, qp, vp);
        for (int c = 0; c < 4; ++c)
          fh[c] = fh[c] - 0.5 * ((vm[2 * c] + vp[2 * c]) * n[0] + (vm[2 * c + 1] + vp[2 * c + 1]) * n[1]) +
                  tau * (um[c] - up[c]);
      }
      return;
    }
    double bn = 0;
    if (kind == CONVDIFF) for (int d = 0; d < nd; ++d) bn += beta[d] * n[d];
    S qn = 0.0;
    for (int d = 0; d < nd; ++d) qn = qn + 0.5 * (qm[d] + qp[d]) * n[d];
    fh[0] = 0.5 * bn * (um[0] + up[0]) + 0.5 * std::fabs(bn) * (um[0] - up[0]) + kappa * qn +
            tau * (um[0] - up[0]);
  }

  // No-slip adiabatic wall (gas models): boundary state ub = (rho-, 0, 0, (rho E)-);
  // fhat.n = F(ub).n (pressure only) - F_v(ub, q-).n without its energy component
  // (zero velocity, zero heat flux) + tau (u- - ub) for Navier-Stokes.
  template <class S> void fhat_wall(const S* um, const S* qm, const double* n, S* fh) const {
    S ub[4] = {um[0], S(0.0), S(0.0), um[3]};
    S f[8];
    euler_flux(ub, f);
    for (int c = 0; c < 4; ++c) fh[c] = f[2 * c] * n[0] + f[2 * c + 1] * n[1];
    if (kind == NS) {
      S fv[8];
      viscous_flux(ub, qm, fv);
      for (int c = 0; c < 3; ++c) fh[c] = fh[c] - (fv[2 * c] * n[0] + fv[2 * c + 1] * n[1]) + tau * (um[c] - ub[c]);
    }
  }

  template <class S> void fhat_boundary(const S* um, const S* qm, const double* x, double t,
                                        const double* n, S* fh) const {
    double g[4];
    exact(x, t, g);
    if (kind == EULER || kind == NS) {
      S up[4] = {g[0], g[1], g[2], g[3]};
      S fm[8], fp[8];
      euler_flux(um, fm); euler_flux(up, fp);
      S lam = maxS(wave_speed(um, n), wave_speed(up, n));
      for (int c = 0; c < 4; ++c)
        fh[c] = 0.5 * ((fm[2 * c] + fp[2 * c]) * n[0] + (fm[2 * c + 1] + fp[2 * c + 1]) * n[1]) +
                0.5 * lam * (um[c] - up[c]);
      if (kind == NS) {
        S vm[8];
        viscous_flux(um, qm, vm);
        for (int c = 0; c < 4; ++c)
          fh[c] = fh[c] - (vm[2 * c] * n[0] + vm[2 * c + 1] * n[1]) + tau * (um[c] - up[c]);
      }
      return;
    }
    double bn = 0;
    if (kind == CONVDIFF) for (int d = 0; d < nd; ++d) bn += beta[d] * n[d];
    S qn = 0.0;
    for (int d = 0; d < nd; ++d) qn = qn + qm[d] * n[d];
    S conv = bn >= 0 ? bn * um[0] : S(bn * g[0]);
    fh[0] = conv + kappa * qn + tau * (um[0] - g[0]);
  }
};

// --------------------------------------------------------------- the problem
struct Face {
  int64_t nbr = -1;
  int nbr_face = -1;
  double shift[3] = {0, 0, 0};
  double n[3] = {0, 0, 0};
  double sJ = 0;
};

struct Problem {
  Ref ref, err;        // err: a richer rule for projections and errors
  Model model;
  int64_t E = 0;
  std::vector<double> v0, Ainv, Jinv, detJ;   // affine map x = v0 + A (xi+1)/2
  std::vector<double> A;
  std::vector<Face> faces;                    // [E][nf]
  int scheme = 0;                             // 0 steady, 1 BDF1, 2 BDF2
  double t = 0, dt = 1;
  std::vector<double> un, unm1;
  std::vector<double> radd;   // optional constant added to the residual ([E][ncu][npe])
  std::string msg;

  // Curved elements: x(xi) = sum_a xgeo[K][a] l_a(xi), the degree-pg Lagrange interpolant
  // through the equispaced reference points of degree pg: (pg+1)^2 on quadrilaterals
  // (first axis fastest), (pg+1)(pg+2)/2 on triangles (the node order of a degree-pg
  // triangle, whose basis gref evaluates).
  int pg = 0;
  std::vector<double> xgeo;           // [E][points][2]
  Ref gref;                           // curved triangles: the degree-pg triangle basis
  std::vector<unsigned char> bc;      // [E][nf]: 1 marks a wall face, 0 a data face
  bool curved() const { return pg > 0; }
  bool wall(int64_t K, int f) const {
    return !bc.empty() && bc[K * ref.nf + f] == 1 && (model.kind == EULER || model.kind == NS);
  }

  int nd() const { return ref.nd; }
  int ncu() const { return model.ncu; }
  int64_t nloc() const { return (int64_t)ref.npe * model.ncu; }
  int64_t ndof() const { return E * nloc(); }

  // 1-D Lagrange basis on the pg+1 equispaced points of [-1, 1] and its derivative
  void lagr(double t, double* l, double* dl) const {
    const int m = pg;
    for (int a = 0; a <= m; ++a) {
      const double ta = -1.0 + 2.0 * a / m;
      double den = 1, num = 1, der = 0;
      for (int b = 0; b <= m; ++b) {
        if (b == a) continue;
        const double tb = -1.0 + 2.0 * b / m;
        den *= ta - tb;
        // product rule: d/dt prod (t - t_b) = sum_c prod_{b != c} (t - t_b)
        der = der * (t - tb) + num;
        num *= t - tb;
      }
      l[a] = num / den;
      dl[a] = der / den;
    }
  }
  // curved map: x and J[d][k] = d x_d / d xi_k at xi
  void curved_map(int64_t K, const double* xi, double* x, double J[2][2]) const {
    if (ref.type == TRI) {
      const int np = gref.npe;
      std::vector<double> phi(np), dphi(2 * np);
      gref.basis(xi, phi.data(), dphi.data());
      x[0] = x[1] = 0;
      J[0][0] = J[0][1] = J[1][0] = J[1][1] = 0;
      for (int a = 0; a < np; ++a) {
        const double* X = &xgeo[((size_t)K * np + a) * 2];
        for (int d = 0; d < 2; ++d) {
          x[d] += X[d] * phi[a];
          J[d][0] += X[d] * dphi[2 * a];
          J[d][1] += X[d] * dphi[2 * a + 1];
        }
      }
      return;
    }
    double l0[16], d0[16], l1[16], d1[16];
    lagr(xi[0], l0, d0);
    lagr(xi[1], l1, d1);
    const int n1 = pg + 1;
    x[0] = x[1] = 0;
    J[0][0] = J[0][1] = J[1][0] = J[1][1] = 0;
    for (int b = 0; b < n1; ++b)
      for (int a = 0; a < n1; ++a) {
        const double* X = &xgeo[((size_t)K * n1 * n1 + a + n1 * b) * 2];
        for (int d = 0; d < 2; ++d) {
          x[d] += X[d] * l0[a] * l1[b];
          J[d][0] += X[d] * d0[a] * l1[b];
          J[d][1] += X[d] * l0[a] * d1[b];
        }
      }
  }

  void map(int64_t K, const double* xi, double* x) const {
    if (curved()) { double J[2][2]; curved_map(K, xi, x, J); return; }
    int d_ = nd();
    for (int d = 0; d < d_; ++d) {
      x[d] = v0[K * 3 + d];
      for (int k = 0; k < d_; ++k) x[d] += A[K * 9 + d * 3 + k] * 0.5 * (xi[k] + 1);
    }
  }
  // Ji[k*3 + d] = d xi_k / d x_d and det J at reference point xi
  void jac(int64_t K, const double* xi, double* Ji, double& det) const {
    if (!curved()) {
      for (int i = 0; i < 9; ++i) Ji[i] = Jinv[K * 9 + i];
      det = detJ[K];
      return;
    }
    double x[2], J[2][2];
    curved_map(K, xi, x, J);
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    for (int i = 0; i < 9; ++i) Ji[i] = 0;
    Ji[0] = J[1][1] / det; Ji[1] = -J[0][1] / det;
    Ji[3] = -J[1][0] / det; Ji[4] = J[0][0] / det;
  }
  // outward unit normal n and surface Jacobian sJ of face f at the reference point xi on it
  void face_frame(int64_t K, int f, const double* xi, double* n, double& sJ) const {
    if (!curved()) {
      const Face& F = faces[K * ref.nf + f];
      for (int d = 0; d < 3; ++d) n[d] = F.n[d];
      sJ = F.sJ;
      return;
    }
    if (ref.type == TRI) {
      // the face runs from its vertex A to B (counter-clockwise), parameter s in [-1, 1]:
      // tangent t = J d xi / ds, sJ = |t|, outward normal = t turned clockwise
      static const double V[3][2] = {{-1, -1}, {1, -1}, {-1, 1}};
      const int A = ref.fverts[f][0], B = ref.fverts[f][1];
      const double dxi[2] = {0.5 * (V[B][0] - V[A][0]), 0.5 * (V[B][1] - V[A][1])};
      double x[2], J[2][2];
      curved_map(K, xi, x, J);
      const double t0 = J[0][0] * dxi[0] + J[0][1] * dxi[1], t1 = J[1][0] * dxi[0] + J[1][1] * dxi[1];
      sJ = std::sqrt(t0 * t0 + t1 * t1);
      n[0] = t1 / sJ; n[1] = -t0 / sJ; n[2] = 0;
      return;
    }
    // n sJ = +-det J J^{-T} e_axis (Nanson), + on the face xi_axis = +1
    double Ji[9], det;
    jac(K, xi, Ji, det);
    const int ax = f / 2;
    const double sg = (f % 2) ? 1.0 : -1.0;
    double m[2] = {sg * det * Ji[ax * 3 + 0], sg * det * Ji[ax * 3 + 1]};
    sJ = std::sqrt(m[0] * m[0] + m[1] * m[1]);
    n[0] = m[0] / sJ; n[1] = m[1] / sJ; n[2] = 0;
  }
  void invmap(int64_t K, const double* x, double* xi) const {
    int d_ = nd();
    for (int k = 0; k < d_; ++k) {
      double s = 0;
      for (int d = 0; d < d_; ++d) s += Ainv[K * 9 + k * 3 + d] * (x[d] - v0[K * 3 + d]);
      xi[k] = 2 * s - 1;
    }
    if (!curved()) return;
    // Damped Newton iteration on x(xi) = x (step halved while the misfit grows), from
    // the corner-based affine guess, then from the reference centre and the face
    // centres; the first root found inside the reference element is taken.
    const bool tri = ref.type == TRI;
    const double sq[6][2] = {{xi[0], xi[1]}, {0, 0}, {-1, 0}, {1, 0}, {0, -1}, {0, 1}};
    const double tr[6][2] = {{xi[0], xi[1]}, {-1.0 / 3, -1.0 / 3}, {0, -1}, {0, 0}, {-1, 0}, {-0.5, -0.5}};
    const double (*starts)[2] = tri ? tr : sq;
    for (int st = 0; st < 6; ++st) {
      double z[2] = {starts[st][0], starts[st][1]};
      double y[2], J[2][2];
      curved_map(K, z, y, J);
      double res = std::hypot(y[0] - x[0], y[1] - x[1]);
      for (int it = 0; it < 100 && res > 0; ++it) {
        const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const double r0 = y[0] - x[0], r1 = y[1] - x[1];
        const double d0 = (J[1][1] * r0 - J[0][1] * r1) / det, d1 = (-J[1][0] * r0 + J[0][0] * r1) / det;
        double a = 1.0, zn[2], yn[2], Jn[2][2], rn = 0;
        for (int h = 0; h < 40; ++h, a *= 0.5) {
          zn[0] = z[0] - a * d0; zn[1] = z[1] - a * d1;
          curved_map(K, zn, yn, Jn);
          rn = std::hypot(yn[0] - x[0], yn[1] - x[1]);
          if (rn < res) break;
        }
        if (!(rn < res)) break;
        const double step = a * (std::fabs(d0) + std::fabs(d1));
        z[0] = zn[0]; z[1] = zn[1]; y[0] = yn[0]; y[1] = yn[1];
        J[0][0] = Jn[0][0]; J[0][1] = Jn[0][1]; J[1][0] = Jn[1][0]; J[1][1] = Jn[1][1];
        res = rn;
        if (step < 1e-15) break;
      }
      const bool inside = tri ? (z[0] >= -1 - 1e-9 && z[1] >= -1 - 1e-9 && z[0] + z[1] <= 1e-9)
                              : (std::fabs(z[0]) <= 1 + 1e-9 && std::fabs(z[1]) <= 1 + 1e-9);
      if (inside && res <= 1e-12 * (1 + std::fabs(x[0]) + std::fabs(x[1]))) {
        xi[0] = z[0]; xi[1] = z[1];
        return;
      }
    }
    xi[0] = xi[1] = std::nan("");   // no preimage: the mesh does not conform
  }
};

bool setup(Problem& P, int etype, int p, int nq1, int64_t E, const double* xyz, const int64_t* vid,
           int pg = 0, const double* xgeo = nullptr, const unsigned char* bc = nullptr) {
  P.ref.init(etype, p, nq1);
  P.err.init(etype, p, p + 3);
  P.E = E;
  if (pg > 0) {
    if ((etype != QUAD && etype != TRI) || !xgeo || pg > 15) {
      P.msg = "oracle: curved elements are quadrilaterals or triangles of degree <= 15";
      return false;
    }
    P.pg = pg;
    const size_t npts = etype == TRI ? (size_t)(pg + 1) * (pg + 2) / 2 : (size_t)(pg + 1) * (pg + 1);
    P.xgeo.assign(xgeo, xgeo + (size_t)E * npts * 2);
    if (etype == TRI) P.gref.init(TRI, pg, 2);
  }
  if (bc) P.bc.assign(bc, bc + (size_t)E * P.ref.nf);
  const int nd = P.ref.nd, nv = P.ref.nv, nf = P.ref.nf;
  P.v0.assign(E * 3, 0); P.A.assign(E * 9, 0); P.Ainv.assign(E * 9, 0);
  P.Jinv.assign(E * 9, 0); P.detJ.assign(E, 0);
  P.faces.assign(E * nf, Face());
  for (int64_t K = 0; K < E; ++K) {
    const double* X = xyz + K * nv * nd;
    for (int d = 0; d < nd; ++d) P.v0[K * 3 + d] = X[d];
    double M[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int k = 0; k < nd; ++k)
      for (int d = 0; d < nd; ++d) M[d][k] = X[P.ref.axisv[k] * nd + d] - X[d];
    // affine elements only: every vertex must be the affine image of its reference vertex
    if (etype != TRI && etype != TET && !P.curved())
      for (int v = 0; v < nv; ++v)
        for (int d = 0; d < nd; ++d) {
          double e = X[d];
          for (int k = 0; k < nd; ++k) if ((v >> k) & 1) e += M[d][k];
          if (std::fabs(e - X[v * nd + d]) > 1e-10 * (1 + std::fabs(e))) {
            P.msg = "oracle: element is not affine";
            return false;
          }
        }
    double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                 M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                 M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    if (!(det > 0) && !P.curved()) { P.msg = "oracle: element with non-positive orientation"; return false; }
    double inv[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        int i1 = (j + 1) % 3, i2 = (j + 2) % 3, j1 = (i + 1) % 3, j2 = (i + 2) % 3;
        inv[i][j] = (M[i1][j1] * M[i2][j2] - M[i1][j2] * M[i2][j1]) / det;
      }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        P.A[K * 9 + i * 3 + j] = M[i][j];
        P.Ainv[K * 9 + i * 3 + j] = inv[i][j];
        P.Jinv[K * 9 + i * 3 + j] = 2 * inv[i][j];   // d xi_i / d x_j
      }
    P.detJ[K] = det / std::pow(2.0, nd);
    // centroid of the element's vertices
    double cen[3] = {0, 0, 0};
    for (int v = 0; v < nv; ++v)
      for (int d = 0; d < nd; ++d) cen[d] += X[v * nd + d] / nv;
    for (int f = 0; f < nf; ++f) {
      Face& F = P.faces[K * nf + f];
      const std::vector<int>& fv = P.ref.fverts[f];
      double fc[3] = {0, 0, 0};
      for (int v : fv)
        for (int d = 0; d < nd; ++d) fc[d] += X[v * nd + d] / fv.size();
      double nn[3] = {0, 0, 0};
      if (nd == 2) {
        double tx = X[fv[1] * 2] - X[fv[0] * 2], ty = X[fv[1] * 2 + 1] - X[fv[0] * 2 + 1];
        double len = std::sqrt(tx * tx + ty * ty);
        F.sJ = len / 2;
        nn[0] = ty / len; nn[1] = -tx / len;
      } else {
        double e1[3], e2[3];
        for (int d = 0; d < 3; ++d) { e1[d] = X[fv[1] * 3 + d] - X[fv[0] * 3 + d]; e2[d] = X[fv[2] * 3 + d] - X[fv[0] * 3 + d]; }
        double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double a = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        F.sJ = a / 4;
        for (int d = 0; d < 3; ++d) nn[d] = c[d] / a;
      }
      double dot = 0;
      for (int d = 0; d < nd; ++d) dot += nn[d] * (fc[d] - cen[d]);
      if (dot < 0) for (int d = 0; d < nd; ++d) nn[d] = -nn[d];
      for (int d = 0; d < nd; ++d) F.n[d] = nn[d];
    }
  }
  // face neighbours: faces that share the same set of (topological) vertex ids
  std::map<std::array<int64_t, 4>, std::vector<std::pair<int64_t, int>>> byverts;
  for (int64_t K = 0; K < E; ++K)
    for (int f = 0; f < nf; ++f) {
      std::array<int64_t, 4> key = {-1, -1, -1, -1};
      const std::vector<int>& fv = P.ref.fverts[f];
      for (size_t i = 0; i < fv.size(); ++i) key[i] = vid[K * nv + fv[i]];
      std::sort(key.begin(), key.begin() + fv.size());
      byverts[key].push_back({K, f});
    }
  for (auto& kv : byverts) {
    if (kv.second.size() == 1) continue;
    if (kv.second.size() != 2) { P.msg = "oracle: non-manifold face"; return false; }
    for (int s = 0; s < 2; ++s) {
      int64_t K = kv.second[s].first; int f = kv.second[s].second;
      int64_t K2 = kv.second[1 - s].first; int f2 = kv.second[1 - s].second;
      Face& F = P.faces[K * nf + f];
      F.nbr = K2; F.nbr_face = f2;
      // periodic translation: centroid of this face minus centroid of the neighbour's face
      const std::vector<int>& fv = P.ref.fverts[f];
      const std::vector<int>& fv2 = P.ref.fverts[f2];
      for (int d = 0; d < nd; ++d) {
        double a = 0, b = 0;
        for (int v : fv) a += xyz[(K * nv + v) * nd + d] / fv.size();
        for (int v : fv2) b += xyz[(K2 * nv + v) * nd + d] / fv2.size();
        F.shift[d] = a - b;
      }
    }
  }
  if (P.curved()) {
    // the element maps must be positively oriented wherever they are evaluated
    std::vector<std::array<double, 3>> pts(P.ref.qx);
    pts.insert(pts.end(), P.err.qx.begin(), P.err.qx.end());
    pts.insert(pts.end(), P.ref.node.begin(), P.ref.node.end());
    for (int f = 0; f < nf; ++f)
      for (size_t k = 0; k < P.ref.fs.size(); ++k) {
        std::array<double, 3> xi = {0, 0, 0};
        P.ref.face_xi(f, P.ref.fs[k].data(), xi.data());
        pts.push_back(xi);
      }
    for (int64_t K = 0; K < E; ++K)
      for (const auto& xi : pts) {
        double Ji[9], det;
        P.jac(K, xi.data(), Ji, det);
        if (!(det > 0)) { P.msg = "oracle: curved element with non-positive Jacobian"; return false; }
      }
  }
  return true;
}

// ---------------------------------------------------------- LDG evaluation
// u_h on element K at reference point xi, all components.
template <class S>
void eval_u(const Problem& P, const S* u, int64_t K, const double* phi, S* out) {
  const int npe = P.ref.npe;
  for (int c = 0; c < P.ncu(); ++c) {
    S s = 0.0;
    for (int j = 0; j < npe; ++j) s = s + phi[j] * u[(K * P.ncu() + c) * npe + j];
    out[c] = s;
  }
}

// q-stage (Eq. 1a) on element K: q[c][d][i]
template <class S>
void q_stage(const Problem& P, const S* u, int64_t K, S* q) {
  const Ref& R = P.ref;
  const int npe = R.npe, nd = R.nd, ncu = P.ncu();
  std::vector<S> rhs(ncu * nd * npe, S(0.0));
  std::vector<double> M(npe * npe, 0.0), phi(npe), dphi(npe * nd), gphi(npe * nd);
  S uq[8];
  for (size_t qp = 0; qp < R.qx.size(); ++qp) {
    R.basis(R.qx[qp].data(), phi.data(), dphi.data());
    double Ji[9], dj;
    P.jac(K, R.qx[qp].data(), Ji, dj);
    double w = R.qw[qp] * dj;
    for (int i = 0; i < npe; ++i)
      for (int d = 0; d < nd; ++d) {
        double g = 0;
        for (int k = 0; k < nd; ++k) g += Ji[k * 3 + d] * dphi[i * nd + k];
        gphi[i * nd + d] = g;
      }
    eval_u(P, u, K, phi.data(), uq);
    for (int c = 0; c < ncu; ++c)
      for (int d = 0; d < nd; ++d)
        for (int i = 0; i < npe; ++i)
          rhs[(c * nd + d) * npe + i] = rhs[(c * nd + d) * npe + i] + w * uq[c] * gphi[i * nd + d];
    for (int i = 0; i < npe; ++i)
      for (int j = 0; j < npe; ++j) M[i * npe + j] += w * phi[i] * phi[j];
  }
  std::vector<double> phin(npe), dphin(npe * nd);
  for (int f = 0; f < R.nf; ++f) {
    const Face& F = P.faces[K * R.nf + f];
    for (int k = 0; k < R.nfq; ++k) {
      double xi[3], x[3], nrm[3], sJ;
      R.face_xi(f, R.fs[k].data(), xi);
      P.map(K, xi, x);
      P.face_frame(K, f, xi, nrm, sJ);
      R.basis(xi, phi.data(), dphi.data());
      double w = R.fw[k] * sJ;
      S um[8], uh[8];
      eval_u(P, u, K, phi.data(), um);
      if (F.nbr >= 0) {
        double xn[3], xin[3];
        for (int d = 0; d < nd; ++d) xn[d] = x[d] - F.shift[d];
        P.invmap(F.nbr, xn, xin);
        R.basis(xin, phin.data(), dphin.data());
        S up[8];
        eval_u(P, u, F.nbr, phin.data(), up);
        for (int c = 0; c < ncu; ++c) uh[c] = 0.5 * (um[c] + up[c]);
      } else if (P.wall(K, f)) {
        // no-slip adiabatic wall: trace (rho-, 0, 0, (rho E)-)
        uh[0] = um[0]; uh[1] = 0.0; uh[2] = 0.0; uh[3] = um[3];
      } else {
        double g[8];
        P.model.exact(x, P.t, g);
        for (int c = 0; c < ncu; ++c) uh[c] = g[c];
      }
      for (int c = 0; c < ncu; ++c)
        for (int d = 0; d < nd; ++d)
          for (int i = 0; i < npe; ++i)
            rhs[(c * nd + d) * npe + i] = rhs[(c * nd + d) * npe + i] - w * uh[c] * nrm[d] * phi[i];
    }
  }
  std::vector<int> piv;
  lu_factor(M, npe, piv);
  for (int cd = 0; cd < ncu * nd; ++cd) {
    lu_solve(M, npe, piv, &rhs[cd * npe]);
    for (int i = 0; i < npe; ++i) q[cd * npe + i] = rhs[cd * npe + i];
  }
}

// q_h on element K at reference point xi: out[c*nd + d]
template <class S>
void eval_q(const Problem& P, const S* qK, const double* phi, S* out) {
  const int npe = P.ref.npe, nd = P.ref.nd;
  for (int cd = 0; cd < P.ncu() * nd; ++cd) {
    S s = 0.0;
    for (int j = 0; j < npe; ++j) s = s + phi[j] * qK[cd * npe + j];
    out[cd] = s;
  }
}

// Residual (Eq. 1b plus the time term) on element K. qof(K) returns q of element K
// (nullptr for models without q).
template <class S, class QOF>
void residual_elem(const Problem& P, const S* u, int64_t K, QOF qof, S* r) {
  const Ref& R = P.ref;
  const Model& Mo = P.model;
  const int npe = R.npe, nd = R.nd, ncu = P.ncu();
  const bool hasq = Mo.kind != EULER;
  for (int i = 0; i < ncu * npe; ++i) r[i] = 0.0;
  std::vector<double> phi(npe), dphi(npe * nd), gphi(npe * nd), phin(npe), dphin(npe * nd);
  const S* qK = hasq ? qof(K) : nullptr;
  double a0 = 0, a1 = 0, a2 = 0;
  if (P.scheme == 1) { a0 = 1; a1 = -1; }
  if (P.scheme == 2) { a0 = 1.5; a1 = -2; a2 = 0.5; }
  for (size_t qp = 0; qp < R.qx.size(); ++qp) {
    R.basis(R.qx[qp].data(), phi.data(), dphi.data());
    double Ji[9], dj;
    P.jac(K, R.qx[qp].data(), Ji, dj);
    double w = R.qw[qp] * dj;
    for (int i = 0; i < npe; ++i)
      for (int d = 0; d < nd; ++d) {
        double g = 0;
        for (int k = 0; k < nd; ++k) g += Ji[k * 3 + d] * dphi[i * nd + k];
        gphi[i * nd + d] = g;
      }
    double xi[3] = {R.qx[qp][0], R.qx[qp][1], R.qx[qp][2]}, x[3];
    P.map(K, xi, x);
    S uq[8], qq[24], f[24];
    eval_u(P, u, K, phi.data(), uq);
    if (hasq) eval_q(P, qK, phi.data(), qq);
    Mo.flux(uq, qq, f);
    double s[8];
    Mo.source(x, s);
    for (int c = 0; c < ncu; ++c) {
      S tterm = 0.0;
      if (P.scheme) {
        double old = 0;
        for (int j = 0; j < npe; ++j)
          old += phi[j] * (a1 * P.un[(K * ncu + c) * npe + j] +
                           (P.scheme == 2 ? a2 * P.unm1[(K * ncu + c) * npe + j] : 0.0));
        tterm = (a0 * uq[c] + old) / P.dt;
      }
      for (int i = 0; i < npe; ++i) {
        S v = (tterm - s[c]) * phi[i];
        for (int d = 0; d < nd; ++d) v = v - f[c * nd + d] * gphi[i * nd + d];
        r[c * npe + i] = r[c * npe + i] + w * v;
      }
    }
  }
  for (int f = 0; f < R.nf; ++f) {
    const Face& F = P.faces[K * R.nf + f];
    for (int k = 0; k < R.nfq; ++k) {
      double xi[3], x[3], nrm[3], sJ;
      R.face_xi(f, R.fs[k].data(), xi);
      P.map(K, xi, x);
      P.face_frame(K, f, xi, nrm, sJ);
      R.basis(xi, phi.data(), dphi.data());
      double w = R.fw[k] * sJ;
      S um[8], qm[24], fh[8];
      eval_u(P, u, K, phi.data(), um);
      if (hasq) eval_q(P, qK, phi.data(), qm);
      if (F.nbr >= 0) {
        double xn[3], xin[3];
        for (int d = 0; d < nd; ++d) xn[d] = x[d] - F.shift[d];
        P.invmap(F.nbr, xn, xin);
        R.basis(xin, phin.data(), dphin.data());
        S up[8], qp[24];
        eval_u(P, u, F.nbr, phin.data(), up);
        if (hasq) eval_q(P, qof(F.nbr), phin.data(), qp);
        Mo.fhat_interior(um, up, qm, qp, nrm, fh);
      } else if (P.wall(K, f)) {
        Mo.fhat_wall(um, qm, nrm, fh);
      } else {
        Mo.fhat_boundary(um, qm, x, P.t, nrm, fh);
      }
      for (int c = 0; c < ncu; ++c)
        for (int i = 0; i < npe; ++i) r[c * npe + i] = r[c * npe + i] + w * fh[c] * phi[i];
    }
  }
  // a constant vector added to the residual (the earlier stages' terms of a DIRK stage)
  if (!P.radd.empty())
    for (int i = 0; i < ncu * npe; ++i) r[i] = r[i] + P.radd[K * ncu * npe + i];
}

// Full residual over all elements.
template <class S>
void residual_all(const Problem& P, const S* u, S* r) {
  const int64_t E = P.E;
  const int64_t nq = (int64_t)P.ncu() * P.nd() * P.ref.npe;
  std::vector<S> q;
  if (P.model.kind != EULER) {
    q.assign(E * nq, S(0.0));
    for (int64_t K = 0; K < E; ++K) q_stage(P, u, K, &q[K * nq]);
  }
  auto qof = [&](int64_t K) -> const S* { return q.empty() ? nullptr : &q[K * nq]; };
  for (int64_t K = 0; K < E; ++K) residual_elem(P, u, K, qof, r + K * P.nloc());
}

// Residual of a list of elements; q is formed only where it is needed.
template <class S>
void residual_some(const Problem& P, const S* u, int64_t ns, const int64_t* elems, S* r) {
  const int64_t nq = (int64_t)P.ncu() * P.nd() * P.ref.npe;
  std::map<int64_t, std::vector<S>> cache;
  auto qof = [&](int64_t K) -> const S* {
    if (P.model.kind == EULER) return nullptr;
    auto it = cache.find(K);
    if (it == cache.end()) {
      std::vector<S> q(nq, S(0.0));
      q_stage(P, u, K, q.data());
      it = cache.emplace(K, std::move(q)).first;
    }
    return it->second.data();
  };
  for (int64_t s = 0; s < ns; ++s) residual_elem(P, u, elems[s], qof, r + s * P.nloc());
}

// ------------------------------------------------------------ GMRES, Newton
double dot(const std::vector<double>& a, const std::vector<double>& b) {
  double s = 0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}

// Restarted GMRES(m) on A x = b from x = 0: modified Gram-Schmidt Arnoldi and
// Givens rotations; stops when the Givens residual estimate |g_{j+1}| <= rtol ||b||.
template <class MATVEC>
int gmres(int64_t n, MATVEC Av, const double* b, double* xout, int m, double rtol, int maxit,
          int* iters_out, std::vector<double>* hist) {
  std::vector<double> x(n, 0.0), r(b, b + n);
  double bn = std::sqrt(dot(r, r));
  int its = 0;
  if (hist) hist->push_back(bn);
  if (bn == 0) { std::fill(xout, xout + n, 0.0); *iters_out = 0; return 0; }
  double beta = bn;
  while (its < maxit) {
    std::vector<std::vector<double>> V(m + 1, std::vector<double>(n, 0.0));
    std::vector<double> H((m + 1) * m, 0.0), cs(m, 0), sn(m, 0), g(m + 1, 0.0);
    for (int64_t i = 0; i < n; ++i) V[0][i] = r[i] / beta;
    g[0] = beta;
    int j = 0;
    bool done = false;
    for (; j < m && its < maxit; ++j) {
      std::vector<double> w(n);
      Av(V[j].data(), w.data());
      ++its;
      for (int i = 0; i <= j; ++i) {
        double h = dot(w, V[i]);
        H[i * m + j] = h;
        for (int64_t k = 0; k < n; ++k) w[k] -= h * V[i][k];
      }
      double hn = std::sqrt(dot(w, w));
      H[(j + 1) * m + j] = hn;
      if (hn > 0) for (int64_t k = 0; k < n; ++k) V[j + 1][k] = w[k] / hn;
      for (int i = 0; i < j; ++i) {
        double a = H[i * m + j], c = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      double a = H[j * m + j], c = H[(j + 1) * m + j];
      double den = std::sqrt(a * a + c * c);
      cs[j] = a / den; sn[j] = c / den;
      H[j * m + j] = den; H[(j + 1) * m + j] = 0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      if (hist) hist->push_back(std::fabs(g[j + 1]));
      if (std::fabs(g[j + 1]) <= rtol * bn || hn == 0) { ++j; done = true; break; }
    }
    // back substitution for the j Krylov coefficients
    std::vector<double> y(j, 0.0);
    for (int i = j - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < j; ++k) s -= H[i * m + k] * y[k];
      y[i] = s / H[i * m + i];
    }
    for (int i = 0; i < j; ++i)
      for (int64_t k = 0; k < n; ++k) x[k] += y[i] * V[i][k];
    // true residual
    std::vector<double> ax(n);
    Av(x.data(), ax.data());
    for (int64_t k = 0; k < n; ++k) r[k] = b[k] - ax[k];
    beta = std::sqrt(dot(r, r));
    if (done || beta <= rtol * bn) break;
  }
  std::copy(x.begin(), x.end(), xout);
  *iters_out = its;
  return beta <= rtol * bn * 1.0001 ? 0 : 1;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

struct orc_stats {
  int newton_iters;
  int gmres_iters;
  int jv_calls;
  int residual_calls;
  double r0, rfinal;
};

void* orc_create_curved(int etype, int p, int nq1, int64_t E, const double* xyz, const int64_t* vid,
                        int model, int cas, int nmu, const double* mu, int pg, const double* xgeo,
                        const unsigned char* bc);

void* orc_create(int etype, int p, int nq1, int64_t E, const double* xyz, const int64_t* vid,
                 int model, int cas, int nmu, const double* mu) {
  return orc_create_curved(etype, p, nq1, E, xyz, vid, model, cas, nmu, mu, 0, nullptr, nullptr);
}

// pg > 0: curved quadrilaterals (map points xgeo [E][(pg+1)^2][2]) or triangles ([E][(pg+1)(pg+2)/2][2]); bc [E][nf]
// (optional) marks wall faces with 1.
void* orc_create_curved(int etype, int p, int nq1, int64_t E, const double* xyz, const int64_t* vid,
                        int model, int cas, int nmu, const double* mu, int pg, const double* xgeo,
                        const unsigned char* bc) {
  Problem* P = new Problem();
  P->model.kind = model;
  P->model.cas = cas;
  int nd = (etype == HEX || etype == TET) ? 3 : 2;
  P->model.nd = nd;
  P->model.ncu = (model == EULER || model == NS) ? 4 : 1;
  if (model == POISSON) { if (nmu > 0) P->model.kappa = mu[0]; if (nmu > 1) P->model.tau = mu[1]; }
  if (model == CONVDIFF) {
    if (nmu > 0) P->model.kappa = mu[0];
    if (nmu > 1) P->model.tau = mu[1];
    for (int d = 0; d < 3; ++d) if (nmu > 2 + d) P->model.beta[d] = mu[2 + d];
  }
  if (model == EULER && nmu > 0) P->model.gamma = mu[0];
  if (model == NS) {
    // mu = {gamma, Re, Pr, tau}; defaults 1.4, 100, 0.72 and tau = 1/Re
    const double re = nmu > 1 ? mu[1] : 100.0;
    if (nmu > 0) P->model.gamma = mu[0];
    P->model.kappa = 1.0 / re;
    if (nmu > 2) P->model.pr = mu[2];
    P->model.tau = nmu > 3 ? mu[3] : 1.0 / re;
  }
  if (!setup(*P, etype, p, nq1, E, xyz, vid, pg, xgeo, bc)) { delete P; return nullptr; }
  return P;
}

void orc_destroy(void* h) { delete (Problem*)h; }

int64_t orc_ndof(void* h) { return ((Problem*)h)->ndof(); }

void orc_set_time(void* h, int scheme, double t, double dt, const double* un, const double* unm1) {
  Problem* P = (Problem*)h;
  P->scheme = scheme; P->t = t; P->dt = dt;
  int64_t n = P->ndof();
  P->un.assign(n, 0.0); P->unm1.assign(n, 0.0);
  if (un) std::copy(un, un + n, P->un.begin());
  if (unm1) std::copy(unm1, unm1 + n, P->unm1.begin());
}

// radd (or null to clear): a constant vector added to every later residual
void orc_set_radd(void* h, const double* radd) {
  Problem* P = (Problem*)h;
  if (radd) P->radd.assign(radd, radd + P->ndof());
  else P->radd.clear();
}

void orc_residual(void* h, const double* u, double* r) {
  residual_all(*(Problem*)h, u, r);
}

void orc_jvp(void* h, const double* u, const double* v, double* jv) {
  Problem* P = (Problem*)h;
  int64_t n = P->ndof();
  std::vector<Dual> ud(n), rd(n);
  for (int64_t i = 0; i < n; ++i) ud[i] = Dual(u[i], v[i]);
  residual_all(*P, ud.data(), rd.data());
  for (int64_t i = 0; i < n; ++i) jv[i] = rd[i].d;
}

void orc_residual_some(void* h, const double* u, int64_t ns, const int64_t* elems, double* r) {
  residual_some(*(Problem*)h, u, ns, elems, r);
}

void orc_jvp_some(void* h, const double* u, const double* v, int64_t ns, const int64_t* elems,
                  double* jv) {
  Problem* P = (Problem*)h;
  // only the 2-ring of the sampled elements is read; converting the whole vector keeps it plain
  int64_t n = P->ndof(), nl = P->nloc();
  std::vector<Dual> ud(n), rd(ns * nl);
  for (int64_t i = 0; i < n; ++i) ud[i] = Dual(u[i], v[i]);
  residual_some(*P, ud.data(), ns, elems, rd.data());
  for (int64_t i = 0; i < ns * nl; ++i) jv[i] = rd[i].d;
}

// Residual evaluated on complex input (real part u, imaginary part ui): the complex step.
void orc_residual_complex(void* h, const double* u, const double* ui, double* rr, double* ri) {
  Problem* P = (Problem*)h;
  int64_t n = P->ndof();
  std::vector<cplx> uc(n), rc(n);
  for (int64_t i = 0; i < n; ++i) uc[i] = cplx(u[i], ui ? ui[i] : 0.0);
  residual_all(*P, uc.data(), rc.data());
  for (int64_t i = 0; i < n; ++i) { rr[i] = rc[i].real(); ri[i] = rc[i].imag(); }
}

// Dense Jacobian by the complex step: J[i][j] = Im R(u + i h e_j)_i / h, h = 1e-30.
void orc_jacobian_cs(void* h, const double* u, double* J) {
  Problem* P = (Problem*)h;
  int64_t n = P->ndof();
  const double hs = 1e-30;
  std::vector<cplx> uc(n), rc(n);
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < n; ++i) uc[i] = cplx(u[i], i == j ? hs : 0.0);
    residual_all(*P, uc.data(), rc.data());
    for (int64_t i = 0; i < n; ++i) J[i * n + j] = rc[i].imag() / hs;
  }
}

// q of every element (diffusion models): [E][ncu][nd][npe]
// Residual (Eq. 1b) of every element with q taken from the caller's array instead of
// the q-stage: the form an element-sharded evaluation needs, whose ghost elements carry
// q computed on another rank.
void orc_residual_with_q(void* h, const double* u, const double* q, double* r) {
  Problem* P = (Problem*)h;
  const int64_t nq = (int64_t)P->ncu() * P->nd() * P->ref.npe;
  auto qof = [&](int64_t K) -> const double* { return P->model.kind == EULER ? nullptr : q + K * nq; };
  for (int64_t K = 0; K < P->E; ++K) residual_elem(*P, u, K, qof, r + K * P->nloc());
}

void orc_q(void* h, const double* u, double* q) {
  Problem* P = (Problem*)h;
  int64_t nq = (int64_t)P->ncu() * P->nd() * P->ref.npe;
  for (int64_t K = 0; K < P->E; ++K) q_stage(*P, u, K, q + K * nq);
}

// L2 projection of the exact solution at time t onto the discrete space.
void orc_project(void* h, double t, double* u) {
  Problem* P = (Problem*)h;
  const Ref& R = P->ref;
  const Ref& Q = P->err;
  const int npe = R.npe, nd = R.nd, ncu = P->ncu();
  std::vector<double> phi(npe), dphi(npe * nd);
  for (int64_t K = 0; K < P->E; ++K) {
    std::vector<double> M(npe * npe, 0.0), b(ncu * npe, 0.0);
    for (size_t qp = 0; qp < Q.qx.size(); ++qp) {
      R.basis(Q.qx[qp].data(), phi.data(), dphi.data());
      double x[3], g[8], Ji[9], dj;
      P->jac(K, Q.qx[qp].data(), Ji, dj);
      const double w = Q.qw[qp] * dj;
      P->map(K, Q.qx[qp].data(), x);
      P->model.exact(x, t, g);
      for (int i = 0; i < npe; ++i) {
        for (int j = 0; j < npe; ++j) M[i * npe + j] += w * phi[i] * phi[j];
        for (int c = 0; c < ncu; ++c) b[c * npe + i] += w * g[c] * phi[i];
      }
    }
    std::vector<int> piv;
    lu_factor(M, npe, piv);
    for (int c = 0; c < ncu; ++c) {
      lu_solve(M, npe, piv, &b[c * npe]);
      for (int i = 0; i < npe; ++i) u[(K * ncu + c) * npe + i] = b[c * npe + i];
    }
  }
}

// Nodal interpolant of the exact solution (exact for polynomials of degree <= p).
void orc_interpolate(void* h, double t, double* u) {
  Problem* P = (Problem*)h;
  const int npe = P->ref.npe, ncu = P->ncu();
  for (int64_t K = 0; K < P->E; ++K)
    for (int i = 0; i < npe; ++i) {
      double x[3], g[8];
      P->map(K, P->ref.node[i].data(), x);
      P->model.exact(x, t, g);
      for (int c = 0; c < ncu; ++c) u[(K * ncu + c) * npe + i] = g[c];
    }
}

// Relative L2 errors of u_h and q_h (scalar manufactured cases; q from the q-stage).
void orc_l2_error(void* h, const double* u, double t, double* eu, double* eq) {
  Problem* P = (Problem*)h;
  const Ref& R = P->ref;
  const Ref& Q = P->err;
  const int npe = R.npe, nd = R.nd, ncu = P->ncu();
  const bool hasq = P->model.kind != EULER;
  int64_t nq = (int64_t)ncu * nd * npe;
  std::vector<double> qK(nq), phi(npe), dphi(npe * nd);
  double eu2 = 0, u2 = 0, eq2 = 0, q2 = 0;
  for (int64_t K = 0; K < P->E; ++K) {
    if (hasq) q_stage(*P, u, K, qK.data());
    for (size_t qp = 0; qp < Q.qx.size(); ++qp) {
      R.basis(Q.qx[qp].data(), phi.data(), dphi.data());
      double x[3], g[8], Ji[9], dj;
      P->jac(K, Q.qx[qp].data(), Ji, dj);
      const double w = Q.qw[qp] * dj;
      P->map(K, Q.qx[qp].data(), x);
      P->model.exact(x, t, g);
      double uh[8];
      eval_u(*P, u, K, phi.data(), uh);
      for (int c = 0; c < ncu; ++c) { eu2 += w * (uh[c] - g[c]) * (uh[c] - g[c]); u2 += w * g[c] * g[c]; }
      if (hasq) {
        double uu, gr[3], qh[3];
        P->model.scalar_exact(x, uu, gr, nullptr);
        eval_q(*P, qK.data(), phi.data(), qh);
        for (int d = 0; d < nd; ++d) {
          double qe = -gr[d];
          eq2 += w * (qh[d] - qe) * (qh[d] - qe);
          q2 += w * qe * qe;
        }
      }
    }
  }
  *eu = std::sqrt(eu2 / (u2 > 0 ? u2 : 1.0));
  *eq = hasq ? std::sqrt(eq2 / (q2 > 0 ? q2 : 1.0)) : 0.0;
}

// GMRES(m) on J(u) x = b with the exact forward-mode J.v.
int orc_gmres(void* h, const double* u, const double* b, double* x, int m, double rtol, int maxit,
              int* iters, double* hist, int hist_cap) {
  Problem* P = (Problem*)h;
  int64_t n = P->ndof();
  std::vector<double> hv;
  auto Av = [&](const double* v, double* out) { orc_jvp(h, u, v, out); };
  int rc = gmres(n, Av, b, x, m, rtol, maxit, iters, &hv);
  if (hist)
    for (int i = 0; i < hist_cap && i < (int)hv.size(); ++i) hist[i] = hv[i];
  return rc;
}

// Newton: u <- u - delta, J(u) delta = R(u), until ||R|| <= rtol ||R(u_0)||.
int orc_newton(void* h, double* u, int m, double newton_rtol, double gmres_rtol, int max_newton,
               int max_gmres, orc_stats* st) {
  Problem* P = (Problem*)h;
  int64_t n = P->ndof();
  std::vector<double> r(n), d(n);
  orc_residual(h, u, r.data());
  double r0 = std::sqrt(dot(r, r)), rn = r0;
  st->r0 = r0; st->newton_iters = 0; st->gmres_iters = 0; st->jv_calls = 0; st->residual_calls = 1;
  int k = 0;
  while (rn > newton_rtol * r0 && k < max_newton) {
    int its = 0;
    auto Av = [&](const double* v, double* out) { orc_jvp(h, u, v, out); st->jv_calls++; };
    gmres(n, Av, r.data(), d.data(), m, gmres_rtol, max_gmres, &its, nullptr);
    st->gmres_iters += its;
    for (int64_t i = 0; i < n; ++i) u[i] -= d[i];
    orc_residual(h, u, r.data());
    st->residual_calls++;
    rn = std::sqrt(dot(r, r));
    ++k;
  }
  st->newton_iters = k;
  st->rfinal = rn;
  return rn <= newton_rtol * r0 ? 0 : 1;
}

// Sizes of the reference element: npe, number of volume and face quadrature points.
void orc_sizes(void* h, int* npe, int* ncu, int* nd, int* nqv, int* nfq) {
  Problem* P = (Problem*)h;
  *npe = P->ref.npe; *ncu = P->ncu(); *nd = P->nd();
  *nqv = (int)P->ref.qx.size(); *nfq = P->ref.nfq;
}

// Face neighbour table [E][nf] (-1: boundary), for connectivity checks.
void orc_neighbours(void* h, int64_t* nbr) {
  Problem* P = (Problem*)h;
  for (size_t i = 0; i < P->faces.size(); ++i) nbr[i] = P->faces[i].nbr;
}

// Reference-element data for pinning tests: nodes [npe][3], quadrature points [nq][3] and weights.
void orc_ref_rules(void* h, double* nodes, double* qx, double* qw, double* fs, double* fw) {
  Problem* P = (Problem*)h;
  const Ref& R = P->ref;
  for (int i = 0; i < R.npe; ++i) for (int d = 0; d < 3; ++d) nodes[i * 3 + d] = R.node[i][d];
  for (size_t q = 0; q < R.qx.size(); ++q) {
    for (int d = 0; d < 3; ++d) qx[q * 3 + d] = R.qx[q][d];
    qw[q] = R.qw[q];
  }
  for (int q = 0; q < R.nfq; ++q) { fs[q * 2] = R.fs[q][0]; fs[q * 2 + 1] = R.fs[q][1]; fw[q] = R.fw[q]; }
}

// Basis values and reference gradients at m points xi [m][3]: phi [m][npe], dphi [m][npe][nd].
void orc_basis(void* h, int64_t m, const double* xi, double* phi, double* dphi) {
  Problem* P = (Problem*)h;
  const Ref& R = P->ref;
  for (int64_t k = 0; k < m; ++k) R.basis(xi + 3 * k, phi + k * R.npe, dphi + k * R.npe * R.nd);
}

// Element mass-matrix product M u (per element, per component).
void orc_mass(void* h, const double* u, double* Mu) {
  Problem* P = (Problem*)h;
  const Ref& R = P->ref;
  const int npe = R.npe, nd = R.nd, ncu = P->ncu();
  std::vector<double> phi(npe), dphi(npe * nd);
  for (int64_t i = 0; i < P->ndof(); ++i) Mu[i] = 0;
  for (int64_t K = 0; K < P->E; ++K)
    for (size_t qp = 0; qp < R.qx.size(); ++qp) {
      R.basis(R.qx[qp].data(), phi.data(), dphi.data());
      double Ji[9], dj, uq[8];
      P->jac(K, R.qx[qp].data(), Ji, dj);
      const double w = R.qw[qp] * dj;
      eval_u(*P, u, K, phi.data(), uq);
      for (int c = 0; c < ncu; ++c)
        for (int i = 0; i < npe; ++i) Mu[(K * ncu + c) * npe + i] += w * uq[c] * phi[i];
    }
}

const char* orc_version() { return "ldg-oracle 1"; }

}  // extern "C"
