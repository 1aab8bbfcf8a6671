// Compiled instances of the nodal J.v kernels of the linear models: quadrilaterals
// p = 1..4 and hexahedra p = 1..6 (Poisson and convection-diffusion), FP64 arithmetic
// with an FP64 q scratch and FP32 arithmetic with an FP32 q scratch.
#include "ldg_launch.cuh"
#include "ldg_hex_lines.cuh"

namespace ldg {

// One thread per node (ldg_linear.cuh) for quadrilaterals and for FP64 hexahedra, one
// thread per line (ldg_hex_lines.cuh) for FP32 hexahedra. The FP64 J.v is bound by the
// FP64 pipe either way and the per-node form keeps it busier (48^3, p = 4: 3.39 ms against
// 3.49 ms); the FP32 J.v is bound by load-store instructions, which the line form cuts
// (0.61 ms against 0.37 ms).
// cart: every element is an axis-aligned box (the instances that skip the zero entries
// of J^{-1} and of the face normals).
template <int DIM, int N1, bool CONV> LinFn lin_pick(int prec, bool cart) {
  if (prec == 0) return cart ? &launch_lin<DIM, N1, CONV, double, double, true>
                             : &launch_lin<DIM, N1, CONV, double, double, false>;
  if constexpr (DIM == 3)
    return cart ? &launch_hex<N1, CONV, float, float, true> : &launch_hex<N1, CONV, float, float, false>;
  else return cart ? &launch_lin<DIM, N1, CONV, float, float, true> : &launch_lin<DIM, N1, CONV, float, float, false>;
}

template <int DIM, bool CONV> LinFn lin_by_p(int p, int prec, bool cart) {
  switch (p) {
    case 1: return lin_pick<DIM, 2, CONV>(prec, cart);
    case 2: return lin_pick<DIM, 3, CONV>(prec, cart);
    case 3: return lin_pick<DIM, 4, CONV>(prec, cart);
    case 4: return lin_pick<DIM, 5, CONV>(prec, cart);
    case 5: if constexpr (DIM == 3) return lin_pick<DIM, 6, CONV>(prec, cart); else return nullptr;
    case 6: if constexpr (DIM == 3) return lin_pick<DIM, 7, CONV>(prec, cart); else return nullptr;
    default: return nullptr;
  }
}

LinFn lin_launcher(int dim, int p, bool conv, int prec, bool cart) {
  if (prec != 0 && prec != 1) return nullptr;
  if (dim == 2) return conv ? lin_by_p<2, true>(p, prec, cart) : lin_by_p<2, false>(p, prec, cart);
  if (dim == 3) return conv ? lin_by_p<3, true>(p, prec, cart) : lin_by_p<3, false>(p, prec, cart);
  return nullptr;
}

}  // namespace ldg
