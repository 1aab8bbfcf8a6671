// Host-side preparation of the LDG operator (see ldg_host.h).
//
// Reference elements follow the readings of Section 2.2 used throughout the
// library: tensor elements carry Gauss-Lobatto-Legendre nodes and Gauss-Legendre
// quadrature with nq points per direction; triangles carry equispaced nodes
// (Silvester's closed form of the Lagrange basis) and a collapsed Gauss rule.
#include "ldg_host.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <unordered_map>

namespace ldg {
namespace {

// Legendre P_n(x) and P_{n-1}(x) by the three-term recurrence.
void leg_pair(int n, double x, double& pn, double& pn1) {
  double a = 1.0, b = x;
  if (n == 0) { pn = 1.0; pn1 = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double c = ((2.0 * k - 1.0) * x * b - (k - 1.0) * a) / k;
    a = b; b = c;
  }
  pn = b; pn1 = a;
}

// Gauss-Legendre: Newton on P_n with P_n' = n (x P_n - P_{n-1}) / (x^2 - 1).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n); w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (4.0 * i + 3.0) / (4.0 * n + 2.0));
    double dp = 1.0;
    for (int it = 0; it < 60; ++it) {
      double pn, pn1;
      leg_pair(n, z, pn, pn1);
      dp = n * (z * pn - pn1) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) <= 1e-17) break;
    }
    double pn, pn1;
    leg_pair(n, z, pn, pn1);
    dp = n * (z * pn - pn1) / (z * z - 1.0);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Gauss-Lobatto-Legendre: endpoints and the zeros of P_N', by Newton with
// P_N'' from Legendre's equation (1 - x^2) P'' = 2 x P' - N (N + 1) P.
void gauss_lobatto(int n1, std::vector<double>& x) {
  int N = n1 - 1;
  x.assign(n1, 0.0);
  x[0] = -1.0; x[N] = 1.0;
  for (int i = 1; i < N; ++i) {
    double z = -std::cos(M_PI * i / N);
    for (int it = 0; it < 60; ++it) {
      double pn, pn1;
      leg_pair(N, z, pn, pn1);
      double d1 = N * (z * pn - pn1) / (z * z - 1.0);
      double d2 = (2.0 * z * d1 - N * (N + 1.0) * pn) / (1.0 - z * z);
      double dz = d1 / d2;
      z -= dz;
      if (std::fabs(dz) <= 1e-17) break;
    }
    x[i] = z;
  }
}

// Barycentric Lagrange interpolation on nodes X.
struct Bary {
  std::vector<double> X, lam;
  explicit Bary(const std::vector<double>& nodes) : X(nodes), lam(nodes.size(), 1.0) {
    for (size_t j = 0; j < X.size(); ++j)
      for (size_t m = 0; m < X.size(); ++m)
        if (m != j) lam[j] /= (X[j] - X[m]);
  }
  // values of all basis functions at x
  void values(double x, double* l) const {
    const size_t n = X.size();
    for (size_t j = 0; j < n; ++j)
      if (x == X[j]) { for (size_t m = 0; m < n; ++m) l[m] = (m == j) ? 1.0 : 0.0; return; }
    double den = 0.0;
    for (size_t j = 0; j < n; ++j) den += lam[j] / (x - X[j]);
    for (size_t j = 0; j < n; ++j) l[j] = lam[j] / (x - X[j]) / den;
  }
  // differentiation matrix at the nodes: Dn[i][j] = l_j'(X_i)
  std::vector<double> dmat() const {
    const size_t n = X.size();
    std::vector<double> D(n * n, 0.0);
    for (size_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (size_t j = 0; j < n; ++j) {
        if (j == i) continue;
        D[i * n + j] = (lam[j] / lam[i]) / (X[i] - X[j]);
        s += D[i * n + j];
      }
      D[i * n + i] = -s;
    }
    return D;
  }
};

bool invert(std::vector<double> A, int n, std::vector<double>& inv) {
  inv.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r) if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return false;
    for (int k = 0; k < n; ++k) { std::swap(A[c * n + k], A[piv * n + k]); std::swap(inv[c * n + k], inv[piv * n + k]); }
    double d = 1.0 / A[c * n + c];
    for (int k = 0; k < n; ++k) { A[c * n + k] *= d; inv[c * n + k] *= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = A[r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) { A[r * n + k] -= f * A[c * n + k]; inv[r * n + k] -= f * inv[c * n + k]; }
    }
  }
  return true;
}

// Silvester's product form of the equispaced Lagrange basis on the triangle:
// phi_{i,j,k} = R_k(l1) R_i(l2) R_j(l3), R_m(l) = prod_{a<m} (p l - a) / (a + 1),
// barycentric l1 = -(xi + eta)/2, l2 = (1 + xi)/2, l3 = (1 + eta)/2.
double silv(int m, int p, double l) {
  double r = 1.0;
  for (int a = 0; a < m; ++a) r *= (p * l - a) / (a + 1.0);
  return r;
}
double dsilv(int m, int p, double l) {
  double s = 0.0;
  for (int b = 0; b < m; ++b) {
    double t = p / (b + 1.0);
    for (int a = 0; a < m; ++a) if (a != b) t *= (p * l - a) / (a + 1.0);
    s += t;
  }
  return s;
}
void tri_basis(int p, double xi, double eta, double* phi, double* dr, double* ds) {
  double l1 = -(xi + eta) / 2.0, l2 = (1.0 + xi) / 2.0, l3 = (1.0 + eta) / 2.0;
  int n = 0;
  for (int j = 0; j <= p; ++j)
    for (int i = 0; i + j <= p; ++i, ++n) {
      int k = p - i - j;
      double a = silv(k, p, l1), b = silv(i, p, l2), c = silv(j, p, l3);
      double da = dsilv(k, p, l1), db = dsilv(i, p, l2), dc = dsilv(j, p, l3);
      phi[n] = a * b * c;
      // d l1/d xi = d l1/d eta = -1/2, d l2/d xi = 1/2, d l3/d eta = 1/2
      dr[n] = -0.5 * da * b * c + 0.5 * a * db * c;
      ds[n] = -0.5 * da * b * c + 0.5 * a * b * dc;
    }
}

// Silvester's form on the tetrahedron: phi_{i,j,k} = R_l(l0) R_i(l1) R_j(l2) R_k(l3),
// l = p - i - j - k, barycentric l1 = (1 + xi)/2, l2 = (1 + eta)/2, l3 = (1 + zeta)/2,
// l0 = -(1 + xi + eta + zeta)/2; nodes numbered k outer, then j, then i.
void tet_basis(int p, const double* x, double* phi, double* dr, double* ds, double* dt) {
  const double L[4] = {-(1.0 + x[0] + x[1] + x[2]) / 2.0, (1.0 + x[0]) / 2.0, (1.0 + x[1]) / 2.0,
                       (1.0 + x[2]) / 2.0};
  int n = 0;
  for (int k = 0; k <= p; ++k)
    for (int j = 0; j + k <= p; ++j)
      for (int i = 0; i + j + k <= p; ++i, ++n) {
        const int m[4] = {p - i - j - k, i, j, k};
        double v[4], dv[4];
        for (int a = 0; a < 4; ++a) { v[a] = silv(m[a], p, L[a]); dv[a] = dsilv(m[a], p, L[a]); }
        phi[n] = v[0] * v[1] * v[2] * v[3];
        // d l0 / d x_d = -1/2, d l_{d+1} / d x_d = 1/2
        const double g0 = dv[0] * v[1] * v[2] * v[3];
        dr[n] = 0.5 * (-g0 + v[0] * dv[1] * v[2] * v[3]);
        ds[n] = 0.5 * (-g0 + v[0] * v[1] * dv[2] * v[3]);
        dt[n] = 0.5 * (-g0 + v[0] * v[1] * v[2] * dv[3]);
      }
}

}  // namespace

bool build_ref_ops(int etype, int p, int nq, RefOps& R, std::string& err) {
  if (p < 1 || p > 8 || nq < 1 || nq > 10) { err = "unsupported order or quadrature"; return false; }
  R.etype = etype; R.p = p; R.nq = nq;
  std::vector<double> gx, gw;
  gauss_legendre(nq, gx, gw);
  R.blob.clear();
  auto put = [&](double v) { R.blob.push_back(v); };
  if (etype == E_TRI) {
    R.dim = 2; R.npe = (p + 1) * (p + 2) / 2; R.nqv = nq * nq; R.nf = 3; R.nfn = p + 1; R.nfq = nq;
    const int npe = R.npe, nqv = R.nqv;
    std::vector<double> qx(2 * nqv), qw(nqv);
    for (int b = 0; b < nq; ++b)
      for (int a = 0; a < nq; ++a) {
        int q = a + nq * b;
        qx[2 * q] = 0.5 * (1.0 + gx[a]) * (1.0 - gx[b]) - 1.0;
        qx[2 * q + 1] = gx[b];
        qw[q] = gw[a] * gw[b] * 0.5 * (1.0 - gx[b]);
      }
    std::vector<double> B(nqv * npe), Dr(nqv * npe), Ds(nqv * npe);
    for (int q = 0; q < nqv; ++q) tri_basis(p, qx[2 * q], qx[2 * q + 1], &B[q * npe], &Dr[q * npe], &Ds[q * npe]);
    std::vector<double> xn(2 * npe);
    {
      int n = 0;
      for (int j = 0; j <= p; ++j)
        for (int i = 0; i + j <= p; ++i, ++n) { xn[2 * n] = -1.0 + 2.0 * i / p; xn[2 * n + 1] = -1.0 + 2.0 * j / p; }
    }
    std::vector<double> Dnr(npe * npe), Dns(npe * npe), tmp(npe);
    for (int i = 0; i < npe; ++i) tri_basis(p, xn[2 * i], xn[2 * i + 1], tmp.data(), &Dnr[i * npe], &Dns[i * npe]);
    std::vector<double> M(npe * npe, 0.0), Mi;
    for (int q = 0; q < nqv; ++q)
      for (int i = 0; i < npe; ++i)
        for (int j = 0; j < npe; ++j) M[i * npe + j] += qw[q] * B[q * npe + i] * B[q * npe + j];
    if (!invert(M, npe, Mi)) { err = "singular reference mass matrix"; return false; }
    std::vector<double> en(p + 1);
    for (int t = 0; t <= p; ++t) en[t] = -1.0 + 2.0 * t / p;
    Bary eb(en);
    std::vector<double> Bf(nq * (p + 1));
    for (int k = 0; k < nq; ++k) eb.values(gx[k], &Bf[k * (p + 1)]);
    for (double v : B) put(v);
    for (double v : Dr) put(v);
    for (double v : Ds) put(v);
    for (double v : qw) put(v);
    for (double v : qx) put(v);
    for (double v : Bf) put(v);
    for (double v : gw) put(v);
    for (double v : gx) put(v);
    for (double v : Dnr) put(v);
    for (double v : Dns) put(v);
    for (double v : Mi) put(v);
    for (double v : xn) put(v);
    return true;
  }
  if (etype == E_TET) {
    R.dim = 3; R.npe = (p + 1) * (p + 2) * (p + 3) / 6; R.nqv = nq * nq * nq; R.nf = 4;
    R.nfn = (p + 1) * (p + 2) / 2; R.nfq = nq * nq;
    const int npe = R.npe, nqv = R.nqv, nfq = R.nfq, nfn = R.nfn;
    // collapsed Gauss rule: xi = (1+a)(1-b)(1-c)/4 - 1, eta = (1+b)(1-c)/2 - 1, zeta = c
    std::vector<double> qx(3 * nqv), qw(nqv);
    for (int c = 0; c < nq; ++c)
      for (int b = 0; b < nq; ++b)
        for (int a = 0; a < nq; ++a) {
          const int q = a + nq * (b + nq * c);
          const double A = gx[a], Bv = gx[b], Cv = gx[c];
          qx[3 * q] = (1.0 + A) * (1.0 - Bv) * (1.0 - Cv) / 4.0 - 1.0;
          qx[3 * q + 1] = (1.0 + Bv) * (1.0 - Cv) / 2.0 - 1.0;
          qx[3 * q + 2] = Cv;
          qw[q] = gw[a] * gw[b] * gw[c] * (1.0 - Bv) * (1.0 - Cv) * (1.0 - Cv) / 8.0;
        }
    std::vector<double> B(nqv * npe), Dr(nqv * npe), Ds(nqv * npe), Dt(nqv * npe);
    for (int q = 0; q < nqv; ++q) tet_basis(p, &qx[3 * q], &B[q * npe], &Dr[q * npe], &Ds[q * npe], &Dt[q * npe]);
    std::vector<double> xn(3 * npe);
    {
      int n = 0;
      for (int k = 0; k <= p; ++k)
        for (int j = 0; j + k <= p; ++j)
          for (int i = 0; i + j + k <= p; ++i, ++n) {
            xn[3 * n] = -1.0 + 2.0 * i / p; xn[3 * n + 1] = -1.0 + 2.0 * j / p; xn[3 * n + 2] = -1.0 + 2.0 * k / p;
          }
    }
    std::vector<double> Dnr(npe * npe), Dns(npe * npe), Dnt(npe * npe), tmp(npe);
    for (int i = 0; i < npe; ++i) tet_basis(p, &xn[3 * i], tmp.data(), &Dnr[i * npe], &Dns[i * npe], &Dnt[i * npe]);
    std::vector<double> M(npe * npe, 0.0), Mi;
    for (int q = 0; q < nqv; ++q)
      for (int i = 0; i < npe; ++i)
        for (int j = 0; j < npe; ++j) M[i * npe + j] += qw[q] * B[q * npe + i] * B[q * npe + j];
    if (!invert(M, npe, Mi)) { err = "singular reference mass matrix"; return false; }
    // faces: the collapsed rule on the reference triangle of the face parameters (s, t),
    // and the equispaced triangle basis in those parameters (face-node order b outer, a inner)
    std::vector<double> sf(2 * nfq), wf(nfq), Bf(nfq * nfn), d1(nfn), d2(nfn);
    for (int b = 0; b < nq; ++b)
      for (int a = 0; a < nq; ++a) {
        const int k = a + nq * b;
        sf[2 * k] = (1.0 + gx[a]) * (1.0 - gx[b]) / 2.0 - 1.0;
        sf[2 * k + 1] = gx[b];
        wf[k] = gw[a] * gw[b] * (1.0 - gx[b]) / 2.0;
        tri_basis(p, sf[2 * k], sf[2 * k + 1], &Bf[k * nfn], d1.data(), d2.data());
      }
    for (double v : B) put(v);
    for (double v : Dr) put(v);
    for (double v : Ds) put(v);
    for (double v : Dt) put(v);
    for (double v : qw) put(v);
    for (double v : qx) put(v);
    for (double v : Bf) put(v);
    for (double v : wf) put(v);
    for (double v : sf) put(v);
    for (double v : Dnr) put(v);
    for (double v : Dns) put(v);
    for (double v : Dnt) put(v);
    for (double v : Mi) put(v);
    for (double v : xn) put(v);
    return true;
  }
  if (etype != E_QUAD && etype != E_HEX) { err = "unknown element type"; return false; }
  R.dim = etype == E_QUAD ? 2 : 3;
  const int n1 = p + 1;
  R.npe = 1; R.nqv = 1; R.nfn = 1; R.nfq = 1;
  for (int d = 0; d < R.dim; ++d) { R.npe *= n1; R.nqv *= nq; }
  for (int d = 0; d < R.dim - 1; ++d) { R.nfn *= n1; R.nfq *= nq; }
  R.nf = 2 * R.dim;
  std::vector<double> xn;
  gauss_lobatto(n1, xn);
  Bary bl(xn);
  std::vector<double> Dn = bl.dmat();
  std::vector<double> B(nq * n1), D(nq * n1, 0.0);
  for (int q = 0; q < nq; ++q) bl.values(gx[q], &B[q * n1]);
  // l_j' is a polynomial of degree p: l_j'(x) = sum_i l_j'(X_i) l_i(x)
  for (int q = 0; q < nq; ++q)
    for (int j = 0; j < n1; ++j) {
      double s = 0.0;
      for (int i = 0; i < n1; ++i) s += Dn[i * n1 + j] * B[q * n1 + i];
      D[q * n1 + j] = s;
    }
  std::vector<double> M1(n1 * n1, 0.0), M1i;
  for (int q = 0; q < nq; ++q)
    for (int i = 0; i < n1; ++i)
      for (int j = 0; j < n1; ++j) M1[i * n1 + j] += gw[q] * B[q * n1 + i] * B[q * n1 + j];
  if (!invert(M1, n1, M1i)) { err = "singular 1-D mass matrix (nq < p + 1?)"; return false; }
  for (double v : B) put(v);
  for (double v : D) put(v);
  for (double v : gw) put(v);
  for (double v : gx) put(v);
  for (double v : Dn) put(v);
  for (double v : M1i) put(v);
  for (double v : xn) put(v);
  return true;
}

bool build_lin_ops(int p, std::vector<double>& blob, std::string& err) {
  if (p < 1 || p > 8) { err = "unsupported order"; return false; }
  const int n1 = p + 1;
  std::vector<double> xn, gx, gw;
  gauss_lobatto(n1, xn);
  gauss_legendre(n1, gx, gw);
  Bary bl(xn);
  std::vector<double> Dn = bl.dmat();
  std::vector<double> B(n1 * n1), D(n1 * n1, 0.0);
  for (int q = 0; q < n1; ++q) bl.values(gx[q], &B[q * n1]);
  for (int q = 0; q < n1; ++q)
    for (int j = 0; j < n1; ++j) {
      double s = 0.0;
      for (int i = 0; i < n1; ++i) s += Dn[i * n1 + j] * B[q * n1 + i];
      D[q * n1 + j] = s;
    }
  std::vector<double> M1(n1 * n1, 0.0), C(n1 * n1, 0.0), M1i;
  for (int q = 0; q < n1; ++q)
    for (int i = 0; i < n1; ++i)
      for (int j = 0; j < n1; ++j) {
        M1[i * n1 + j] += gw[q] * B[q * n1 + i] * B[q * n1 + j];
        C[i * n1 + j] += gw[q] * D[q * n1 + i] * B[q * n1 + j];
      }
  if (!invert(M1, n1, M1i)) { err = "singular 1-D mass matrix"; return false; }
  blob.clear();
  blob.insert(blob.end(), Dn.begin(), Dn.end());
  blob.insert(blob.end(), M1.begin(), M1.end());
  blob.insert(blob.end(), C.begin(), C.end());
  for (int i = 0; i < n1; ++i) blob.push_back(M1i[i * n1]);
  for (int i = 0; i < n1; ++i) blob.push_back(M1i[i * n1 + n1 - 1]);
  // products with C for the residual of axis-aligned boxes: C Dn, C L0, C Lp
  for (int i = 0; i < n1; ++i)
    for (int l = 0; l < n1; ++l) {
      double s = 0.0;
      for (int m = 0; m < n1; ++m) s += C[i * n1 + m] * Dn[m * n1 + l];
      blob.push_back(s);
    }
  for (int c = 0; c < 2; ++c)
    for (int i = 0; i < n1; ++i) {
      double s = 0.0;
      for (int m = 0; m < n1; ++m) s += C[i * n1 + m] * M1i[m * n1 + (c ? n1 - 1 : 0)];
      blob.push_back(s);
    }
  return true;
}

namespace {
int simplex_face_node(int etype, int p, int f, int j);
}  // namespace

int face_node_host(int etype, int p, int f, int j) {
  if (etype == E_QUAD || etype == E_HEX) {
    const int n1 = p + 1, ax = f >> 1, fix = (f & 1) ? p : 0;
    if (etype == E_QUAD) return ax == 0 ? fix + n1 * j : j + n1 * fix;
    const int a = j % n1, b = j / n1;
    if (ax == 0) return fix + n1 * (a + n1 * b);
    if (ax == 1) return a + n1 * (fix + n1 * b);
    return a + n1 * (b + n1 * fix);
  }
  return simplex_face_node(etype, p, f, j);
}

namespace {
// local node of face-node j on face f (numbering of tri_basis / tet_basis)
int simplex_face_node(int etype, int p, int f, int j) {
  auto tri_idx = [p](int i, int jj) { return jj * (p + 1) - jj * (jj - 1) / 2 + i; };
  if (etype == E_TRI) {
    if (f == 0) return tri_idx(j, 0);
    if (f == 1) return tri_idx(p - j, j);
    return tri_idx(0, p - j);
  }
  int b = 0, a = j;
  while (a > p - b) { a -= p + 1 - b; ++b; }
  const int A = f == 0 ? 1 : 0, B = f <= 1 ? 2 : 1, C = f == 3 ? 2 : 3;
  int l[4] = {0, 0, 0, 0};
  l[A] = p - a - b; l[B] = a; l[C] = b;
  int off = 0;
  for (int kk = 0; kk < l[3]; ++kk) off += (p - kk + 1) * (p - kk + 2) / 2;
  const int q = p - l[3];
  return off + l[2] * (q + 1) - l[2] * (l[2] - 1) / 2 + l[1];
}
}  // namespace

bool build_lin_simplex_ops(int etype, int p, std::vector<double>& blob, std::string& err) {
  if ((etype != E_TRI && etype != E_TET) || p < 1 || p > 6) { err = "unsupported simplex order"; return false; }
  const int dim = etype == E_TRI ? 2 : 3, nf = dim + 1;
  const int npe = etype == E_TRI ? (p + 1) * (p + 2) / 2 : (p + 1) * (p + 2) * (p + 3) / 6;
  const int nfn = etype == E_TRI ? p + 1 : (p + 1) * (p + 2) / 2;
  const int lda = npe | 1, ldl = nfn | 1;
  const int nq = p + 3;   // collapsed Gauss rule, exact beyond degree 2p
  std::vector<double> gx, gw;
  gauss_legendre(nq, gx, gw);
  // volume: M[i][j] = int phi_i phi_j, C_k[i][j] = int phi_j d_k phi_i
  std::vector<double> M((size_t)npe * npe, 0.0), C((size_t)dim * npe * npe, 0.0);
  std::vector<double> phi(npe), d0(npe), d1(npe), d2(npe);
  const int nqv = dim == 2 ? nq * nq : nq * nq * nq;
  for (int q = 0; q < nqv; ++q) {
    const int a = q % nq, b = (q / nq) % nq, c = q / (nq * nq);
    double w;
    if (dim == 2) {
      tri_basis(p, 0.5 * (1.0 + gx[a]) * (1.0 - gx[b]) - 1.0, gx[b], phi.data(), d0.data(), d1.data());
      w = gw[a] * gw[b] * 0.5 * (1.0 - gx[b]);
    } else {
      const double x[3] = {(1.0 + gx[a]) * (1.0 - gx[b]) * (1.0 - gx[c]) / 4.0 - 1.0,
                           (1.0 + gx[b]) * (1.0 - gx[c]) / 2.0 - 1.0, gx[c]};
      tet_basis(p, x, phi.data(), d0.data(), d1.data(), d2.data());
      w = gw[a] * gw[b] * gw[c] * (1.0 - gx[b]) * (1.0 - gx[c]) * (1.0 - gx[c]) / 8.0;
    }
    const double* dk[3] = {d0.data(), d1.data(), d2.data()};
    for (int i = 0; i < npe; ++i)
      for (int j = 0; j < npe; ++j) {
        M[(size_t)i * npe + j] += w * phi[i] * phi[j];
        for (int k = 0; k < dim; ++k) C[((size_t)k * npe + i) * npe + j] += w * phi[j] * dk[k][i];
      }
  }
  std::vector<double> Mi;
  if (!invert(M, npe, Mi)) { err = "singular reference mass matrix"; return false; }
  // nodal derivatives Dn_k[n][m] = d_k phi_m (x_n)
  std::vector<double> xn;
  {
    RefOps tmp;
    tmp.etype = etype; tmp.p = p; tmp.npe = npe; tmp.dim = dim;
    if (etype == E_TET) {
      // tet_basis numbering: k outer, then j, then i
      for (int k = 0; k <= p; ++k)
        for (int j = 0; j + k <= p; ++j)
          for (int i = 0; i + j + k <= p; ++i) {
            xn.push_back(-1.0 + 2.0 * i / p); xn.push_back(-1.0 + 2.0 * j / p); xn.push_back(-1.0 + 2.0 * k / p);
          }
    } else {
      for (int j = 0; j <= p; ++j)
        for (int i = 0; i + j <= p; ++i) { xn.push_back(-1.0 + 2.0 * i / p); xn.push_back(-1.0 + 2.0 * j / p); }
    }
  }
  std::vector<double> Dn((size_t)dim * npe * npe, 0.0);
  for (int n = 0; n < npe; ++n) {
    if (dim == 2) tri_basis(p, xn[2 * n], xn[2 * n + 1], phi.data(), d0.data(), d1.data());
    else tet_basis(p, &xn[3 * n], phi.data(), d0.data(), d1.data(), d2.data());
    const double* dk[3] = {d0.data(), d1.data(), d2.data()};
    for (int k = 0; k < dim; ++k)
      for (int m = 0; m < npe; ++m) Dn[((size_t)k * npe + n) * npe + m] = dk[k][m];
  }
  // face mass in the face parameters (the measure the geometry's sJ scales):
  // triangles: the equispaced Lagrange basis on s in [-1, 1]; tetrahedra: the triangle basis
  std::vector<double> MF((size_t)nfn * nfn, 0.0);
  if (dim == 2) {
    std::vector<double> en(p + 1), l(p + 1);
    for (int t = 0; t <= p; ++t) en[t] = -1.0 + 2.0 * t / p;
    Bary eb(en);
    for (int k = 0; k < nq; ++k) {
      eb.values(gx[k], l.data());
      for (int a = 0; a <= p; ++a)
        for (int b = 0; b <= p; ++b) MF[a * nfn + b] += gw[k] * l[a] * l[b];
    }
  } else {
    std::vector<double> fp(nfn), e1(nfn), e2(nfn);
    for (int b = 0; b < nq; ++b)
      for (int a = 0; a < nq; ++a) {
        tri_basis(p, (1.0 + gx[a]) * (1.0 - gx[b]) / 2.0 - 1.0, gx[b], fp.data(), e1.data(), e2.data());
        const double w = gw[a] * gw[b] * (1.0 - gx[b]) / 2.0;
        for (int i = 0; i < nfn; ++i)
          for (int j = 0; j < nfn; ++j) MF[(size_t)i * nfn + j] += w * fp[i] * fp[j];
      }
  }
  // lift of face f: M^{-1} E_f M_f
  std::vector<double> LIFT((size_t)nf * npe * nfn, 0.0);
  for (int f = 0; f < nf; ++f)
    for (int n = 0; n < npe; ++n)
      for (int j = 0; j < nfn; ++j) {
        double s = 0.0;
        for (int b = 0; b < nfn; ++b) s += Mi[(size_t)n * npe + simplex_face_node(etype, p, f, b)] * MF[(size_t)b * nfn + j];
        LIFT[((size_t)f * npe + n) * nfn + j] = s;
      }
  // padded layout: DN, C (dim x npe x lda), M (npe x lda), LIFT (nf x npe x ldl), MF (nfn x ldl)
  blob.assign((size_t)(2 * dim + 1) * npe * lda + (size_t)nf * npe * ldl + (size_t)nfn * ldl, 0.0);
  size_t o = 0;
  for (int k = 0; k < dim; ++k)
    for (int n = 0; n < npe; ++n)
      for (int m = 0; m < npe; ++m) blob[o + ((size_t)k * npe + n) * lda + m] = Dn[((size_t)k * npe + n) * npe + m];
  o += (size_t)dim * npe * lda;
  for (int k = 0; k < dim; ++k)
    for (int n = 0; n < npe; ++n)
      for (int m = 0; m < npe; ++m) blob[o + ((size_t)k * npe + n) * lda + m] = C[((size_t)k * npe + n) * npe + m];
  o += (size_t)dim * npe * lda;
  for (int n = 0; n < npe; ++n)
    for (int m = 0; m < npe; ++m) blob[o + (size_t)n * lda + m] = M[(size_t)n * npe + m];
  o += (size_t)npe * lda;
  for (int f = 0; f < nf; ++f)
    for (int n = 0; n < npe; ++n)
      for (int j = 0; j < nfn; ++j) blob[o + ((size_t)f * npe + n) * ldl + j] = LIFT[((size_t)f * npe + n) * nfn + j];
  o += (size_t)nf * npe * ldl;
  for (int i = 0; i < nfn; ++i)
    for (int j = 0; j < nfn; ++j) blob[o + (size_t)i * ldl + j] = MF[(size_t)i * nfn + j];
  return true;
}

bool build_err_rule(int etype, int p, int nqe, ErrRule& R, std::string& err) {
  if (p < 1 || p > 8 || nqe < 1 || nqe > 12) { err = "unsupported order for the error rule"; return false; }
  std::vector<double> gx, gw;
  gauss_legendre(nqe, gx, gw);
  int dim = (etype == E_QUAD || etype == E_TRI) ? 2 : 3;
  int npe;
  if (etype == E_TRI) npe = (p + 1) * (p + 2) / 2;
  else if (etype == E_TET) npe = (p + 1) * (p + 2) * (p + 3) / 6;
  else npe = dim == 2 ? (p + 1) * (p + 1) : (p + 1) * (p + 1) * (p + 1);
  int nqp = dim == 2 ? nqe * nqe : nqe * nqe * nqe;
  R.nqp = nqp;
  R.xi.assign((size_t)nqp * dim, 0.0);
  R.w.assign(nqp, 0.0);
  R.B.assign((size_t)nqp * npe, 0.0);
  // points and weights: tensor Gauss rules, collapsed (Duffy) on simplices
  for (int q = 0; q < nqp; ++q) {
    const int a = q % nqe, b = (q / nqe) % nqe, c = q / (nqe * nqe);
    double* x = &R.xi[(size_t)q * dim];
    if (etype == E_TRI) {
      x[0] = 0.5 * (1.0 + gx[a]) * (1.0 - gx[b]) - 1.0;
      x[1] = gx[b];
      R.w[q] = gw[a] * gw[b] * 0.5 * (1.0 - gx[b]);
    } else if (etype == E_TET) {
      x[0] = (1.0 + gx[a]) * (1.0 - gx[b]) * (1.0 - gx[c]) / 4.0 - 1.0;
      x[1] = (1.0 + gx[b]) * (1.0 - gx[c]) / 2.0 - 1.0;
      x[2] = gx[c];
      R.w[q] = gw[a] * gw[b] * gw[c] * (1.0 - gx[b]) * (1.0 - gx[c]) * (1.0 - gx[c]) / 8.0;
    } else {
      x[0] = gx[a]; x[1] = gx[b];
      R.w[q] = gw[a] * gw[b];
      if (dim == 3) { x[2] = gx[c]; R.w[q] *= gw[c]; }
    }
  }
  // basis values at the points
  std::vector<double> d1(npe), d2(npe), d3(npe);
  if (etype == E_TRI) {
    for (int q = 0; q < nqp; ++q) tri_basis(p, R.xi[2 * q], R.xi[2 * q + 1], &R.B[(size_t)q * npe], d1.data(), d2.data());
  } else if (etype == E_TET) {
    for (int q = 0; q < nqp; ++q) tet_basis(p, &R.xi[3 * q], &R.B[(size_t)q * npe], d1.data(), d2.data(), d3.data());
  } else {
    const int n1 = p + 1;
    std::vector<double> xn;
    gauss_lobatto(n1, xn);
    Bary bl(xn);
    std::vector<double> l(3 * n1);
    for (int q = 0; q < nqp; ++q) {
      for (int d = 0; d < dim; ++d) bl.values(R.xi[(size_t)q * dim + d], &l[d * n1]);
      for (int n = 0; n < npe; ++n) {
        const int id[3] = {n % n1, (n / n1) % n1, n / (n1 * n1)};
        double v = 1.0;
        for (int d = 0; d < dim; ++d) v *= l[d * n1 + id[d]];
        R.B[(size_t)q * npe + n] = v;
      }
    }
  }
  // projection operator P = Mref^{-1} B^T W
  std::vector<double> M((size_t)npe * npe, 0.0), Mi;
  for (int q = 0; q < nqp; ++q)
    for (int i = 0; i < npe; ++i)
      for (int j = 0; j < npe; ++j) M[(size_t)i * npe + j] += R.w[q] * R.B[(size_t)q * npe + i] * R.B[(size_t)q * npe + j];
  if (!invert(M, npe, Mi)) { err = "singular reference mass matrix"; return false; }
  R.P.assign((size_t)npe * nqp, 0.0);
  for (int i = 0; i < npe; ++i)
    for (int q = 0; q < nqp; ++q) {
      double s = 0.0;
      for (int j = 0; j < npe; ++j) s += Mi[(size_t)i * npe + j] * R.B[(size_t)q * npe + j];
      R.P[(size_t)i * nqp + q] = s * R.w[q];
    }
  return true;
}

void ref_nodes(const RefOps& R, std::vector<double>& out) {
  out.assign((size_t)R.npe * R.dim, 0.0);
  if (R.etype == E_TET) {
    const int nq = R.nq, npe = R.npe, nqv = R.nqv;
    const double* xn = R.blob.data() + 4 * (size_t)nqv * npe + nqv + 3 * nqv + (size_t)R.nfq * R.nfn + 3 * R.nfq +
                       4 * (size_t)npe * npe;
    (void)nq;
    for (int i = 0; i < 3 * npe; ++i) out[i] = xn[i];
    return;
  }
  if (R.etype == E_TRI) {
    int n = 0;
    for (int j = 0; j <= R.p; ++j)
      for (int i = 0; i + j <= R.p; ++i, ++n) { out[2 * n] = -1.0 + 2.0 * i / R.p; out[2 * n + 1] = -1.0 + 2.0 * j / R.p; }
    return;
  }
  const int n1 = R.p + 1;
  const double* xn = R.blob.data() + 2 * R.nq * n1 + 2 * R.nq + 2 * n1 * n1;
  for (int n = 0; n < R.npe; ++n) {
    int id[3] = {n % n1, (n / n1) % n1, n / (n1 * n1)};
    for (int d = 0; d < R.dim; ++d) out[n * R.dim + d] = xn[id[d]];
  }
}

void ref_face_point(const RefOps& R, int f, int k, double* xi) {
  std::vector<double> gx, gw;
  gauss_legendre(R.nq, gx, gw);
  if (R.etype == E_TET) {
    static const double V[4][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
    const int A = f == 0 ? 1 : 0, B = f <= 1 ? 2 : 1, C = f == 3 ? 2 : 3;
    const double s = (1.0 + gx[k % R.nq]) * (1.0 - gx[k / R.nq]) / 2.0 - 1.0, t = gx[k / R.nq];
    for (int d = 0; d < 3; ++d) xi[d] = V[A][d] + 0.5 * (1.0 + s) * (V[B][d] - V[A][d]) + 0.5 * (1.0 + t) * (V[C][d] - V[A][d]);
    return;
  }
  if (R.etype == E_TRI) {
    static const double V[3][2] = {{-1, -1}, {1, -1}, {-1, 1}};
    int a = f, b = (f + 1) % 3;
    double s = gx[k];
    for (int d = 0; d < 2; ++d) xi[d] = 0.5 * (1 - s) * V[a][d] + 0.5 * (1 + s) * V[b][d];
    return;
  }
  int ax = f >> 1, side = f & 1, m = 0;
  int kk[2] = {k % R.nq, k / R.nq};
  for (int d = 0; d < R.dim; ++d) xi[d] = (d == ax) ? (side ? 1.0 : -1.0) : gx[kk[m++]];
}

namespace {
// local vertex ids of each face, ordered so that vertex 0 -> 1 follows the face parameter
const std::vector<std::vector<int>>& face_vertices(int etype) {
  static const std::vector<std::vector<int>> tri = {{0, 1}, {1, 2}, {2, 0}};
  static const std::vector<std::vector<int>> quad = {{0, 2}, {1, 3}, {0, 1}, {2, 3}};
  static const std::vector<std::vector<int>> hex = {{0, 2, 4, 6}, {1, 3, 5, 7}, {0, 1, 4, 5},
                                                    {2, 3, 6, 7}, {0, 1, 2, 3}, {4, 5, 6, 7}};
  static const std::vector<std::vector<int>> tet = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
  return etype == E_TRI ? tri : (etype == E_QUAD ? quad : (etype == E_HEX ? hex : tet));
}
}  // namespace

namespace {
// 1-D Lagrange basis on the m+1 equispaced points of [-1, 1] and its derivative at t
void lagr_equi(int m, double t, double* l, double* dl) {
  for (int a = 0; a <= m; ++a) {
    const double ta = -1.0 + 2.0 * a / m;
    double den = 1.0, num = 1.0, der = 0.0;
    for (int b = 0; b <= m; ++b) {
      if (b == a) continue;
      const double tb = -1.0 + 2.0 * b / m;
      den *= ta - tb;
      der = der * (t - tb) + num;
      num *= t - tb;
    }
    l[a] = num / den;
    dl[a] = der / den;
  }
}
// map points per element: (pg+1)^2 on quadrilaterals, (pg+1)(pg+2)/2 on triangles
int curved_points(int etype, int pg) { return etype == E_TRI ? (pg + 1) * (pg + 2) / 2 : (pg + 1) * (pg + 1); }

// curved element map (quadrilateral or triangle): x and J[d][k] = d x_d / d xi_k at xi
void curved_point(int etype, int pg, const double* X, const double* xi, double* x, double J[2][2]) {
  if (etype == E_TRI) {
    // the degree-pg equispaced Lagrange basis of the triangle (tri_basis) at xi
    const int np = curved_points(E_TRI, pg);
    std::vector<double> phi(np), dr(np), ds(np);
    tri_basis(pg, xi[0], xi[1], phi.data(), dr.data(), ds.data());
    x[0] = x[1] = 0.0;
    J[0][0] = J[0][1] = J[1][0] = J[1][1] = 0.0;
    for (int a = 0; a < np; ++a)
      for (int d = 0; d < 2; ++d) {
        x[d] += X[a * 2 + d] * phi[a];
        J[d][0] += X[a * 2 + d] * dr[a];
        J[d][1] += X[a * 2 + d] * ds[a];
      }
    return;
  }
  double l0[16], d0[16], l1[16], d1[16];
  lagr_equi(pg, xi[0], l0, d0);
  lagr_equi(pg, xi[1], l1, d1);
  x[0] = x[1] = 0.0;
  J[0][0] = J[0][1] = J[1][0] = J[1][1] = 0.0;
  for (int b = 0; b <= pg; ++b)
    for (int a = 0; a <= pg; ++a) {
      const double* P = X + (a + (pg + 1) * b) * 2;
      for (int d = 0; d < 2; ++d) {
        x[d] += P[d] * l0[a] * l1[b];
        J[d][0] += P[d] * d0[a] * l1[b];
        J[d][1] += P[d] * l0[a] * d1[b];
      }
    }
}
}  // namespace

// Curved triangles: the same records at the collapsed Gauss points of the reference
// triangle; the face frame from the tangent t = J d xi / ds of face f (vertex f to f + 1,
// counter-clockwise): sJ = |t|, outward normal = t turned clockwise.
bool prepare_curved_tri(const RefOps& R, int64_t E, int pg, const double* xgeo, CurvedPrep& out, std::string& err) {
  const int npe = R.npe, nqv = R.nqv, nf = R.nf, nfq = R.nfq;
  std::vector<double> gx, gw;
  gauss_legendre(R.nq, gx, gw);
  const double* B = R.blob.data();                    // B[nqv][npe]
  const double* qw = B + 3 * (size_t)nqv * npe;       // reference weights
  const double* qx = qw + nqv;                        // [nqv][2] reference points
  out.rec = nqv * 5 + nf * nfq * 3;
  out.xrec = nqv * 2 + nf * nfq * 2;
  out.geo.assign((size_t)E * out.rec, 0.0);
  out.x.assign((size_t)E * out.xrec, 0.0);
  out.minv.assign((size_t)E * npe * npe, 0.0);
  out.xnode.assign((size_t)E * npe * 2, 0.0);
  std::vector<double> rn;
  ref_nodes(R, rn);
  const size_t mstride = (size_t)curved_points(E_TRI, pg) * 2;
  static const double V[3][2] = {{-1, -1}, {1, -1}, {-1, 1}};
  std::vector<double> M(npe * npe), Mi;
  for (int64_t e = 0; e < E; ++e) {
    const double* X = xgeo + e * mstride;
    double* g = &out.geo[(size_t)e * out.rec];
    double* xo = &out.x[(size_t)e * out.xrec];
    std::fill(M.begin(), M.end(), 0.0);
    for (int q = 0; q < nqv; ++q) {
      double x[2], J[2][2];
      curved_point(E_TRI, pg, X, &qx[2 * q], x, J);
      const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      if (!(det > 0.0)) { err = "curved element " + std::to_string(e) + " has a non-positive Jacobian"; return false; }
      const double w = qw[q] * det;
      g[q * 5 + 0] = qw[q] * J[1][1];
      g[q * 5 + 1] = -qw[q] * J[0][1];
      g[q * 5 + 2] = -qw[q] * J[1][0];
      g[q * 5 + 3] = qw[q] * J[0][0];
      g[q * 5 + 4] = w;
      xo[q * 2] = x[0];
      xo[q * 2 + 1] = x[1];
      for (int i = 0; i < npe; ++i)
        for (int j = 0; j < npe; ++j) M[i * npe + j] += w * B[q * npe + i] * B[q * npe + j];
    }
    for (int n = 0; n < npe; ++n) {
      double J[2][2];
      curved_point(E_TRI, pg, X, &rn[n * 2], &out.xnode[((size_t)e * npe + n) * 2], J);
    }
    if (!invert(M, npe, Mi)) { err = "singular element mass matrix"; return false; }
    std::copy(Mi.begin(), Mi.end(), out.minv.begin() + (size_t)e * npe * npe);
    for (int f = 0; f < nf; ++f) {
      const int a = f, b = (f + 1) % 3;
      const double dxi[2] = {0.5 * (V[b][0] - V[a][0]), 0.5 * (V[b][1] - V[a][1])};
      for (int k = 0; k < nfq; ++k) {
        double xi[3], x[2], J[2][2];
        ref_face_point(R, f, k, xi);
        curved_point(E_TRI, pg, X, xi, x, J);
        const double t0 = J[0][0] * dxi[0] + J[0][1] * dxi[1], t1 = J[1][0] * dxi[0] + J[1][1] * dxi[1];
        const double sj = std::sqrt(t0 * t0 + t1 * t1);
        double* fr = g + nqv * 5 + (f * nfq + k) * 3;
        fr[0] = t1 / sj;
        fr[1] = -t0 / sj;
        fr[2] = gw[k] * sj;
        xo[nqv * 2 + (f * nfq + k) * 2] = x[0];
        xo[nqv * 2 + (f * nfq + k) * 2 + 1] = x[1];
      }
    }
  }
  return true;
}

bool prepare_curved(const RefOps& R, int64_t E, int pg, const double* xgeo, CurvedPrep& out, std::string& err) {
  if ((R.etype != E_QUAD && R.etype != E_TRI) || pg < 1 || pg > 15 || !xgeo) {
    err = "curved elements are quadrilaterals or triangles with map degree 1..15";
    return false;
  }
  if (R.etype == E_TRI) return prepare_curved_tri(R, E, pg, xgeo, out, err);
  const int nq = R.nq, n1 = R.p + 1, npe = R.npe, nqv = R.nqv, nf = R.nf, nfq = R.nfq;
  std::vector<double> gx, gw;
  gauss_legendre(nq, gx, gw);
  const double* B = R.blob.data();   // B[nq][n1]
  out.rec = nqv * 5 + nf * nfq * 3;
  out.xrec = nqv * 2 + nf * nfq * 2;
  out.geo.assign((size_t)E * out.rec, 0.0);
  out.x.assign((size_t)E * out.xrec, 0.0);
  out.minv.assign((size_t)E * npe * npe, 0.0);
  out.xnode.assign((size_t)E * npe * 2, 0.0);
  std::vector<double> rn;
  ref_nodes(R, rn);
  const size_t mstride = (size_t)(pg + 1) * (pg + 1) * 2;
  std::vector<double> M(npe * npe), Mi;
  for (int64_t e = 0; e < E; ++e) {
    const double* X = xgeo + e * mstride;
    double* g = &out.geo[(size_t)e * out.rec];
    double* xo = &out.x[(size_t)e * out.xrec];
    std::fill(M.begin(), M.end(), 0.0);
    for (int q1 = 0; q1 < nq; ++q1)
      for (int q0 = 0; q0 < nq; ++q0) {
        const int q = q0 + nq * q1;
        const double xi[2] = {gx[q0], gx[q1]};
        double x[2], J[2][2];
        curved_point(E_QUAD, pg, X, xi, x, J);
        const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        if (!(det > 0.0)) { err = "curved element " + std::to_string(e) + " has a non-positive Jacobian"; return false; }
        const double w = gw[q0] * gw[q1] * det;
        // w det J (d xi_k / d x_d): the cofactors of J times the weight
        g[q * 5 + 0] = gw[q0] * gw[q1] * J[1][1];
        g[q * 5 + 1] = -gw[q0] * gw[q1] * J[0][1];
        g[q * 5 + 2] = -gw[q0] * gw[q1] * J[1][0];
        g[q * 5 + 3] = gw[q0] * gw[q1] * J[0][0];
        g[q * 5 + 4] = w;
        xo[q * 2] = x[0];
        xo[q * 2 + 1] = x[1];
        for (int i = 0; i < npe; ++i) {
          const double pi = B[q0 * n1 + i % n1] * B[q1 * n1 + i / n1];
          for (int j = 0; j < npe; ++j) M[i * npe + j] += w * pi * B[q0 * n1 + j % n1] * B[q1 * n1 + j / n1];
        }
      }
    for (int n = 0; n < npe; ++n) {
      double J[2][2];
      curved_point(E_QUAD, pg, X, &rn[n * 2], &out.xnode[((size_t)e * npe + n) * 2], J);
    }
    if (!invert(M, npe, Mi)) { err = "singular element mass matrix"; return false; }
    std::copy(Mi.begin(), Mi.end(), out.minv.begin() + (size_t)e * npe * npe);
    for (int f = 0; f < nf; ++f)
      for (int k = 0; k < nfq; ++k) {
        double xi[3], x[2], J[2][2];
        ref_face_point(R, f, k, xi);
        curved_point(E_QUAD, pg, X, xi, x, J);
        const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        if (!(det > 0.0)) { err = "curved element " + std::to_string(e) + " has a non-positive Jacobian"; return false; }
        // Nanson: n sJ = +-det J J^{-T} e_axis = +- (row `axis` of the cofactor matrix)
        const int ax = f >> 1;
        const double sg = (f & 1) ? 1.0 : -1.0;
        const double m0 = sg * (ax == 0 ? J[1][1] : -J[1][0]), m1 = sg * (ax == 0 ? -J[0][1] : J[0][0]);
        const double sj = std::sqrt(m0 * m0 + m1 * m1);
        double* fr = g + nqv * 5 + (f * nfq + k) * 3;
        fr[0] = m0 / sj;
        fr[1] = m1 / sj;
        fr[2] = gw[k] * sj;
        xo[nqv * 2 + (f * nfq + k) * 2] = x[0];
        xo[nqv * 2 + (f * nfq + k) * 2 + 1] = x[1];
      }
  }
  return true;
}

bool prepare_mesh(const RefOps& R, int64_t E, const double* xyz, const int64_t* vid, MeshPrep& out, std::string& err,
                  int pg, const double* xgeo) {
  const int dim = R.dim, nf = R.nf;
  const int nv = R.etype == E_TRI ? 3 : (R.etype == E_TET ? 4 : (1 << dim));
  const int GEO = dim * dim + 1 + dim + dim * dim + nf * (dim + 1);
  out.E = E;
  out.geo.assign((size_t)E * GEO, 0.0);
  out.nbr.assign((size_t)E * nf, -1);
  out.nbf.assign((size_t)E * nf, 0);
  const int axis_vert[3] = {1, 2, R.etype == E_TET ? 3 : 4};
  // Reference outward normals and the length factor |d xi / d s| of each face parameter.
  auto ref_normal = [&](int f, double* N, double& ds) {
    for (int d = 0; d < 3; ++d) N[d] = 0.0;
    ds = 1.0;
    if (R.etype == E_TRI) {
      if (f == 0) N[1] = -1.0;
      else if (f == 1) { N[0] = N[1] = 1.0 / std::sqrt(2.0); ds = std::sqrt(2.0); }
      else N[0] = -1.0;
    } else if (R.etype == E_TET) {
      // face f opposite vertex f; face 0 lies in xi + eta + zeta = -1, whose area is
      // sqrt(3) times that of the face parameters' reference triangle
      if (f == 0) { N[0] = N[1] = N[2] = 1.0 / std::sqrt(3.0); ds = std::sqrt(3.0); }
      else N[f - 1] = -1.0;
    } else {
      N[f >> 1] = (f & 1) ? 1.0 : -1.0;
    }
  };
  std::vector<double> J(9), Ji(9);
  for (int64_t e = 0; e < E; ++e) {
    const double* X = xyz + (size_t)e * nv * dim;
    // J[d][k] = (x_{axis vertex k} - x_0)_d / 2
    for (int d = 0; d < dim; ++d)
      for (int k = 0; k < dim; ++k) J[d * dim + k] = 0.5 * (X[axis_vert[k] * dim + d] - X[d]);
    if (R.etype != E_TRI && R.etype != E_TET && pg == 0) {
      for (int vtx = 0; vtx < nv; ++vtx)
        for (int d = 0; d < dim; ++d) {
          double pr = X[d];
          for (int k = 0; k < dim; ++k) if ((vtx >> k) & 1) pr += 2.0 * J[d * dim + k];
          if (std::fabs(pr - X[vtx * dim + d]) > 1e-10 * (1.0 + std::fabs(pr))) {
            err = "element " + std::to_string(e) + " is not affine (parallelogram/parallelepiped)";
            return false;
          }
        }
    }
    double det;
    if (dim == 2) {
      det = J[0] * J[3] - J[1] * J[2];
      Ji[0] = J[3] / det; Ji[1] = -J[1] / det; Ji[2] = -J[2] / det; Ji[3] = J[0] / det;
    } else {
      det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) + J[2] * (J[3] * J[7] - J[4] * J[6]);
      Ji[0] = (J[4] * J[8] - J[5] * J[7]) / det; Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det; Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det;
      Ji[3] = (J[5] * J[6] - J[3] * J[8]) / det; Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det; Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
      Ji[6] = (J[3] * J[7] - J[4] * J[6]) / det; Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det; Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
    }
    if (!(det > 0.0) && pg == 0) { err = "element " + std::to_string(e) + " has non-positive Jacobian"; return false; }
    double* g = &out.geo[(size_t)e * GEO];
    for (int i = 0; i < dim * dim; ++i) g[i] = Ji[i];
    g[dim * dim] = det;
    // x(xi) = x_0 + J (xi + 1)  =>  x(0) = x_0 + J 1
    for (int d = 0; d < dim; ++d) {
      double s = X[d];
      for (int k = 0; k < dim; ++k) s += J[d * dim + k];
      g[dim * dim + 1 + d] = s;
    }
    for (int i = 0; i < dim * dim; ++i) g[dim * dim + 1 + dim + i] = J[i];
    // Nanson: n dS = det J J^{-T} N dS_ref
    for (int f = 0; f < nf; ++f) {
      double N[3], ds;
      ref_normal(f, N, ds);
      double m[3] = {0, 0, 0}, len = 0.0;
      for (int d = 0; d < dim; ++d) {
        for (int k = 0; k < dim; ++k) m[d] += Ji[k * dim + d] * N[k];
        len += m[d] * m[d];
      }
      len = std::sqrt(len);
      double* fr = g + 2 * dim * dim + 1 + dim + f * (dim + 1);
      for (int d = 0; d < dim; ++d) fr[d] = m[d] / len;
      fr[dim] = det * len * ds;
    }
  }
  // connectivity by the sorted vertex ids of each face
  const auto& FV = face_vertices(R.etype);
  struct Key { int64_t v[4]; bool operator==(const Key& o) const { return v[0] == o.v[0] && v[1] == o.v[1] && v[2] == o.v[2] && v[3] == o.v[3]; } };
  struct KH { size_t operator()(const Key& k) const { size_t h = 1469598103934665603ull; for (int i = 0; i < 4; ++i) { h ^= (size_t)k.v[i] + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2); } return h; } };
  std::unordered_map<Key, int64_t, KH> open;
  open.reserve((size_t)E * nf);
  std::vector<int64_t> partner((size_t)E * nf, -1);
  for (int64_t e = 0; e < E; ++e)
    for (int f = 0; f < nf; ++f) {
      Key k = {{-1, -1, -1, -1}};
      for (size_t i = 0; i < FV[f].size(); ++i) k.v[i] = vid[e * nv + FV[f][i]];
      std::sort(k.v, k.v + FV[f].size());
      auto it = open.find(k);
      if (it == open.end()) open.emplace(k, e * nf + f);
      else {
        if (it->second < 0) { err = "a face is shared by more than two elements"; return false; }
        partner[e * nf + f] = it->second;
        partner[it->second] = e * nf + f;
        it->second = -2;
      }
    }
  // face-point coordinates and orientation permutations
  std::map<std::vector<unsigned char>, int> codes;
  // Matched positions: the face points, or for tetrahedra (whose face rule is not
  // symmetric) the face nodes, whose permutation the kernels apply to the neighbour's
  // face-node values.
  const bool tet = R.etype == E_TET;
  const int nmatch = tet ? R.nfn : R.nfq;
  std::vector<double> xs(nmatch * 3), xt(nmatch * 3);
  std::vector<double> fref((size_t)nf * nmatch * 3, 0.0);   // reference positions, computed once
  for (int f = 0; f < nf; ++f)
    for (int k = 0; k < nmatch; ++k) {
      double* xi = &fref[((size_t)f * nmatch + k) * 3];
      if (tet) {
        static const double V[4][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
        const int A = f == 0 ? 1 : 0, B = f <= 1 ? 2 : 1, C = f == 3 ? 2 : 3;
        int b = 0, a = k;
        while (a > R.p - b) { a -= R.p + 1 - b; ++b; }
        for (int d = 0; d < 3; ++d)
          xi[d] = V[A][d] + (double)a / R.p * (V[B][d] - V[A][d]) + (double)b / R.p * (V[C][d] - V[A][d]);
      } else {
        ref_face_point(R, f, k, xi);
      }
    }
  auto face_pts = [&](int64_t e, int f, double* P, const double* shift) {
    const double* g = &out.geo[(size_t)e * GEO];
    for (int k = 0; k < nmatch; ++k) {
      const double* xi = &fref[((size_t)f * nmatch + k) * 3];
      if (pg > 0) {
        double x[2], J[2][2];
        curved_point(R.etype, pg, xgeo + (size_t)e * curved_points(R.etype, pg) * 2, xi, x, J);
        for (int d = 0; d < 2; ++d) P[k * 3 + d] = x[d] + (shift ? shift[d] : 0.0);
        continue;
      }
      for (int d = 0; d < dim; ++d) {
        double s = g[dim * dim + 1 + d];
        for (int kk = 0; kk < dim; ++kk) s += g[dim * dim + 1 + dim + d * dim + kk] * xi[kk];
        P[k * 3 + d] = s + (shift ? shift[d] : 0.0);
      }
    }
  };
  int nb_faces = 0;
  for (int64_t e = 0; e < E; ++e) {
    const double* X = xyz + (size_t)e * nv * dim;
    for (int f = 0; f < nf; ++f) {
      int64_t pf = partner[e * nf + f];
      if (pf < 0) { ++nb_faces; continue; }
      int64_t e2 = pf / nf;
      int f2 = (int)(pf % nf);
      const double* X2 = xyz + (size_t)e2 * nv * dim;
      // periodic shift: centroid of this face minus centroid of the partner face
      double shift[3] = {0, 0, 0};
      for (int d = 0; d < dim; ++d) {
        double a = 0, b = 0;
        for (int vv : FV[f]) a += X[vv * dim + d];
        for (int vv : FV[f2]) b += X2[vv * dim + d];
        shift[d] = (a - b) / FV[f].size();
      }
      face_pts(e, f, xs.data(), nullptr);
      face_pts(e2, f2, xt.data(), shift);
      std::vector<unsigned char> pm(nmatch);
      double hscale = 0.0;
      for (int d = 0; d < dim; ++d) hscale = std::max(hscale, std::fabs(out.geo[(size_t)e * GEO + dim * dim + 1 + dim + d * dim]));
      for (int k = 0; k < nmatch; ++k) {
        int best = -1;
        double bd = 1e300;
        for (int k2 = 0; k2 < nmatch; ++k2) {
          double dd = 0;
          for (int d = 0; d < dim; ++d) dd += (xs[k * 3 + d] - xt[k2 * 3 + d]) * (xs[k * 3 + d] - xt[k2 * 3 + d]);
          if (dd < bd) { bd = dd; best = k2; }
        }
        if (std::sqrt(bd) > 1e-8 * (1.0 + hscale)) { err = "non-conforming face points"; return false; }
        pm[k] = (unsigned char)best;
      }
      auto it = codes.find(pm);
      int code;
      if (it == codes.end()) { code = (int)codes.size(); codes.emplace(pm, code); }
      else code = it->second;
      if (code > 31) { err = "too many face orientations"; return false; }
      out.nbr[e * nf + f] = (int)e2;
      out.nbf[e * nf + f] = (unsigned char)(f2 | (code << 3));
    }
  }
  out.n_orient = (int)codes.size();
  out.perm.assign((size_t)std::max(1, out.n_orient) * nmatch, 0);
  for (auto& kv : codes)
    for (int k = 0; k < nmatch; ++k) out.perm[kv.second * nmatch + k] = kv.first[k];
  out.n_boundary_faces = nb_faces;
  return true;
}

}  // namespace ldg
