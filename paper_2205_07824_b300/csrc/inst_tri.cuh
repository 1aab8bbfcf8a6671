// Triangle instances: p = 1..6 with p + 2 collapsed Gauss points per direction.
#pragma once
#include "ldg_launch.cuh"
namespace ldg {
template <class TL> void register_tri_t(std::vector<KernelSet>& reg) {
  add_set<TriEl<1, 3>, ScalarModel<2, false>, TL>(reg, 0);
  add_set<TriEl<2, 4>, ScalarModel<2, false>, TL>(reg, 0);
  add_set<TriEl<3, 5>, ScalarModel<2, false>, TL>(reg, 0);
  add_set<TriEl<4, 6>, ScalarModel<2, false>, TL>(reg, 0);
  add_set<TriEl<5, 7>, ScalarModel<2, false>, TL>(reg, 0);
  add_set<TriEl<6, 8>, ScalarModel<2, false>, TL>(reg, 0);
  add_set<TriEl<1, 3>, ScalarModel<2, true>, TL>(reg, 0);
  add_set<TriEl<2, 4>, ScalarModel<2, true>, TL>(reg, 0);
  add_set<TriEl<3, 5>, ScalarModel<2, true>, TL>(reg, 0);
  add_set<TriEl<4, 6>, ScalarModel<2, true>, TL>(reg, 0);
  add_set<TriEl<5, 7>, ScalarModel<2, true>, TL>(reg, 0);
  add_set<TriEl<6, 8>, ScalarModel<2, true>, TL>(reg, 0);
}
}  // namespace ldg
