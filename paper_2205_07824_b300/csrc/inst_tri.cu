// Compiled triangle instances: p = 1..3 with p + 2 collapsed Gauss points per direction.
#include "ldg_launch.cuh"
namespace ldg {
void register_tri(std::vector<KernelSet>& reg) {
  add_set<TriEl<1, 3>, ScalarModel<2, false>>(reg, 0);
  add_set<TriEl<2, 4>, ScalarModel<2, false>>(reg, 0);
  add_set<TriEl<3, 5>, ScalarModel<2, false>>(reg, 0);
  add_set<TriEl<1, 3>, ScalarModel<2, true>>(reg, 0);
  add_set<TriEl<2, 4>, ScalarModel<2, true>>(reg, 0);
  add_set<TriEl<3, 5>, ScalarModel<2, true>>(reg, 0);
}
}  // namespace ldg
