// Compiled instances of the nodal J.v kernels of the linear models: quadrilaterals
// p = 1..4 and hexahedra p = 1..6 (Poisson and convection-diffusion), FP64 arithmetic
// with an FP64 q scratch and FP32 arithmetic with an FP32 q scratch.
#include "ldg_launch.cuh"
#include "ldg_linear.cuh"

namespace ldg {

template <int DIM, int N1, bool CONV> LinFn lin_pick(int prec) {
  return prec == 0 ? &launch_lin<DIM, N1, CONV, double, double> : &launch_lin<DIM, N1, CONV, float, float>;
}

template <int DIM, bool CONV> LinFn lin_by_p(int p, int prec) {
  switch (p) {
    case 1: return lin_pick<DIM, 2, CONV>(prec);
    case 2: return lin_pick<DIM, 3, CONV>(prec);
    case 3: return lin_pick<DIM, 4, CONV>(prec);
    case 4: return lin_pick<DIM, 5, CONV>(prec);
    case 5: if constexpr (DIM == 3) return lin_pick<DIM, 6, CONV>(prec); else return nullptr;
    case 6: if constexpr (DIM == 3) return lin_pick<DIM, 7, CONV>(prec); else return nullptr;
    default: return nullptr;
  }
}

LinFn lin_launcher(int dim, int p, bool conv, int prec) {
  if (prec != 0 && prec != 1) return nullptr;
  if (dim == 2) return conv ? lin_by_p<2, true>(p, prec) : lin_by_p<2, false>(p, prec);
  if (dim == 3) return conv ? lin_by_p<3, true>(p, prec) : lin_by_p<3, false>(p, prec);
  return nullptr;
}

}  // namespace ldg
