// Compiled hexahedron instances: linear models, p = 1..6 with p + 1 Gauss points per direction.
#include "ldg_launch.cuh"
namespace ldg {
void register_hex(std::vector<KernelSet>& reg) {
  add_set<TensorEl<3, 1, 2>, ScalarModel<3, false>>(reg, 2);
  add_set<TensorEl<3, 2, 3>, ScalarModel<3, false>>(reg, 2);
  add_set<TensorEl<3, 1, 2>, ScalarModel<3, true>>(reg, 2);
  add_set<TensorEl<3, 2, 3>, ScalarModel<3, true>>(reg, 2);
  add_set<TensorEl<3, 3, 4>, ScalarModel<3, true>>(reg, 2);
  add_set<TensorEl<3, 4, 5>, ScalarModel<3, true>>(reg, 2);
  add_set<TensorEl<3, 5, 6>, ScalarModel<3, true>>(reg, 2);
  add_set<TensorEl<3, 6, 7>, ScalarModel<3, true>>(reg, 2);
}
}  // namespace ldg
