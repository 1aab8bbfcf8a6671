// Host-side preparation of the LDG operator: reference-element operator blobs,
// affine geometry records and face connectivity (Section 2.2, Section 3.2).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace ldg {

enum { E_TRI = 0, E_QUAD = 1, E_HEX = 2 };

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
// coordinates xyz [E][nv][dim] and topological vertex ids vid [E][nv].
bool prepare_mesh(const RefOps& ref, int64_t E, const double* xyz, const int64_t* vid, MeshPrep& out,
                  std::string& err);

// Reference coordinates of face point k of face f and of volume point q (for host-side projection).
void ref_face_point(const RefOps& ref, int f, int k, double* xi);
void ref_nodes(const RefOps& ref, std::vector<double>& xn);   // [npe][dim]

}  // namespace ldg
