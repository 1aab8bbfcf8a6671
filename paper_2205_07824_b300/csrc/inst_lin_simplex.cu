// Compiled instances of the nodal J.v kernels of the linear models on simplices:
// triangles p = 1..6 and tetrahedra p = 1..4 (Poisson and convection-diffusion), FP64
// arithmetic with an FP64 q scratch, FP32 arithmetic with an FP32 q scratch, and (hi, lo)
// float-pair arithmetic with a float-pair q scratch. The element traits' quadrature size
// does not enter these kernels.
#include "ldg_launch.cuh"
#include "ldg_linear.cuh"

namespace ldg {

template <class EL, bool CONV> LinFn sim_pick(int prec) {
  if (prec == 2) return &launch_sim<EL, CONV, df, df>;
  return prec == 0 ? &launch_sim<EL, CONV, double, double> : &launch_sim<EL, CONV, float, float>;
}

template <bool CONV> LinFn sim_by(int etype, int p, int prec) {
  if (etype == 0) {
    switch (p) {
      case 1: return sim_pick<TriEl<1, 3>, CONV>(prec);
      case 2: return sim_pick<TriEl<2, 4>, CONV>(prec);
      case 3: return sim_pick<TriEl<3, 5>, CONV>(prec);
      case 4: return sim_pick<TriEl<4, 6>, CONV>(prec);
      case 5: return sim_pick<TriEl<5, 7>, CONV>(prec);
      case 6: return sim_pick<TriEl<6, 8>, CONV>(prec);
      default: return nullptr;
    }
  }
  if (etype == 3) {
    switch (p) {
      case 1: return sim_pick<TetEl<1, 3>, CONV>(prec);
      case 2: return sim_pick<TetEl<2, 4>, CONV>(prec);
      case 3: return sim_pick<TetEl<3, 5>, CONV>(prec);
      case 4: return sim_pick<TetEl<4, 6>, CONV>(prec);
      default: return nullptr;
    }
  }
  return nullptr;
}

LinFn lin_simplex_launcher(int etype, int p, bool conv, int prec) {
  if (prec < 0 || prec > 2) return nullptr;
  return conv ? sim_by<true>(etype, p, prec) : sim_by<false>(etype, p, prec);
}

}  // namespace ldg
