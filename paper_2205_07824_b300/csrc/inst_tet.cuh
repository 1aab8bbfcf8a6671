// Tetrahedron instances: Poisson and convection-diffusion, p = 1..4, with p + 2
// collapsed Gauss points per direction.
#pragma once
#include "ldg_launch.cuh"
namespace ldg {
template <class TL> void register_tet_t(std::vector<KernelSet>& reg) {
  add_set<TetEl<1, 3>, ScalarModel<3, false>, TL>(reg, 3);
  add_set<TetEl<2, 4>, ScalarModel<3, false>, TL>(reg, 3);
  add_set<TetEl<3, 5>, ScalarModel<3, false>, TL>(reg, 3);
  add_set<TetEl<4, 6>, ScalarModel<3, false>, TL>(reg, 3);
  add_set<TetEl<1, 3>, ScalarModel<3, true>, TL>(reg, 3);
  add_set<TetEl<2, 4>, ScalarModel<3, true>, TL>(reg, 3);
  add_set<TetEl<3, 5>, ScalarModel<3, true>, TL>(reg, 3);
  add_set<TetEl<4, 6>, ScalarModel<3, true>, TL>(reg, 3);
}
}  // namespace ldg
