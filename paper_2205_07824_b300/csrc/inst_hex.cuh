// Hexahedron instances: linear models, p = 1..6 with p + 1 Gauss points per direction
// (Poisson p = 1, 2).
#pragma once
#include "ldg_launch.cuh"
namespace ldg {
template <class TL> void register_hex_t(std::vector<KernelSet>& reg) {
  add_set<TensorEl<3, 1, 2>, ScalarModel<3, false>, TL>(reg, 2);
  add_set<TensorEl<3, 2, 3>, ScalarModel<3, false>, TL>(reg, 2);
  add_set<TensorEl<3, 1, 2>, ScalarModel<3, true>, TL>(reg, 2);
  add_set<TensorEl<3, 2, 3>, ScalarModel<3, true>, TL>(reg, 2);
  add_set<TensorEl<3, 3, 4>, ScalarModel<3, true>, TL>(reg, 2);
  add_set<TensorEl<3, 4, 5>, ScalarModel<3, true>, TL>(reg, 2);
  add_set<TensorEl<3, 5, 6>, ScalarModel<3, true>, TL>(reg, 2);
  add_set<TensorEl<3, 6, 7>, ScalarModel<3, true>, TL>(reg, 2);
}
}  // namespace ldg
