// Host-side preparation of the LDG operator: reference-element operator blobs,
// affine geometry records and face connectivity (Section 2.2, Section 3.2).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace ldg {

enum { E_TRI = 0, E_QUAD = 1, E_HEX = 2, E_TET = 3 };

struct RefOps {
  int etype, p, nq, dim, npe, nqv, nf, nfn, nfq;
  std::vector<double> blob;   // layout of TensorEl / TriEl in ldg_device.cuh
};

// Builds the reference operator blob for (element type, p, quadrature points per direction).
bool build_ref_ops(int etype, int p, int nq, RefOps& out, std::string& err);

struct MeshPrep {
  int64_t E = 0;
  std::vector<double> geo;            // [E][GEO]
  std::vector<int> nbr;               // [E][NF], -1 boundary
  std::vector<unsigned char> nbf;     // [E][NF] neighbour face | orientation << 3
  std::vector<unsigned char> perm;    // [n_orient][NFQ]
  int n_orient = 0;
  int n_boundary_faces = 0;
};

// Geometry (Jacobians, normals, surface Jacobians by Nanson's formula) and face
// connectivity with face-point orientation permutations, from per-element vertex
// coordinates xyz [E][nv][dim] and topological vertex ids vid [E][nv]. With pg > 0
// the quadrilaterals are curved (map points xgeo, see prepare_curved): the affine
// record is then not checked, and face points are matched through the curved maps.
bool prepare_mesh(const RefOps& ref, int64_t E, const double* xyz, const int64_t* vid, MeshPrep& out,
                  std::string& err, int pg = 0, const double* xgeo = nullptr);

// Curved quadrilaterals: the element map is the degree-pg Lagrange interpolant of
// the map points xgeo [E][(pg+1)^2][2] at the equispaced reference points
// (-1 + 2a/pg, -1 + 2b/pg), a fastest. Sampled at the quadrature points:
struct CurvedPrep {
  int rec = 0, xrec = 0;
  std::vector<double> geo;    // [E][rec]: per volume point w det J d xi_k / d x_d (k, d) and w det J;
                              //           per face point the outward unit normal and w sJ
  std::vector<double> x;      // [E][xrec]: physical coordinates of the volume, then face points
  std::vector<double> minv;   // [E][npe][npe]: inverse element mass matrices
  std::vector<double> xnode;  // [E][npe][2]: physical coordinates of the element's nodes
};
bool prepare_curved(const RefOps& ref, int64_t E, int pg, const double* xgeo, CurvedPrep& out, std::string& err);

// A richer reference rule for L2 projections and errors: Gauss with nqe points per
// direction (collapsed on simplices). xi [nqp][dim] points, w [nqp] weights, B [nqp][npe]
// basis values, P = Mref^{-1} B^T W [npe][nqp] the reference L2 projection.
struct ErrRule {
  int nqp = 0;
  std::vector<double> xi, w, B, P;
};
bool build_err_rule(int etype, int p, int nqe, ErrRule& out, std::string& err);

// 1-D operators of the nodal linear J.v kernels for order p (Gauss-Lobatto basis l_i):
// Dn[i][j] = l_j'(x_i), M1[i][j] = int l_i l_j, C[i][j] = int l_i' l_j (Gauss rule of
// p + 1 points, exact), then columns 0 and p of M1^{-1}.
bool build_lin_ops(int p, std::vector<double>& blob, std::string& err);

// Dense reference operators of the nodal linear J.v kernels on triangles and
// tetrahedra (equispaced nodes), exact integrals, rows padded to odd lengths
// (lda = n_pe | 1, ldl = n_fn | 1): Dn_k[n][m] = d_k phi_m(x_n); C_k[i][j] =
// int phi_j d_k phi_i; M; LIFT_f = M^{-1} E_f M_f (face f's nodes); the face mass M_f
// in face-node order (the same on every face).
bool build_lin_simplex_ops(int etype, int p, std::vector<double>& blob, std::string& err);

// Local node of face-node j on face f (face-node numbering of the element kernels).
int face_node_host(int etype, int p, int f, int j);

// Reference coordinates of face point k of face f and of volume point q (for host-side projection).
void ref_face_point(const RefOps& ref, int f, int k, double* xi);
void ref_nodes(const RefOps& ref, std::vector<double>& xn);   // [npe][dim]

}  // namespace ldg
