// Quadrilateral instances: linear models with p + 1 Gauss points per direction
// (p = 1..4), Euler with p + 2 (p = 1..4).
#pragma once
#include "ldg_launch.cuh"
namespace ldg {
template <class TL> void register_quad_t(std::vector<KernelSet>& reg) {
  add_set<TensorEl<2, 1, 2>, ScalarModel<2, false>, TL>(reg, 1);
  add_set<TensorEl<2, 2, 3>, ScalarModel<2, false>, TL>(reg, 1);
  add_set<TensorEl<2, 3, 4>, ScalarModel<2, false>, TL>(reg, 1);
  add_set<TensorEl<2, 4, 5>, ScalarModel<2, false>, TL>(reg, 1);
  add_set<TensorEl<2, 1, 2>, ScalarModel<2, true>, TL>(reg, 1);
  add_set<TensorEl<2, 2, 3>, ScalarModel<2, true>, TL>(reg, 1);
  add_set<TensorEl<2, 3, 4>, ScalarModel<2, true>, TL>(reg, 1);
  add_set<TensorEl<2, 4, 5>, ScalarModel<2, true>, TL>(reg, 1);
  add_set<TensorEl<2, 1, 3>, EulerModel, TL>(reg, 1);
  add_set<TensorEl<2, 2, 4>, EulerModel, TL>(reg, 1);
  add_set<TensorEl<2, 3, 5>, EulerModel, TL>(reg, 1);
  add_set<TensorEl<2, 4, 6>, EulerModel, TL>(reg, 1);
}
}  // namespace ldg
