// Navier-Stokes instances: quadrilaterals, p = 1..4 with p + 2 Gauss points per
// direction (the viscous flux is a rational function of u and q, like Euler's).
#pragma once
#include "ldg_launch.cuh"
namespace ldg {
template <class TL> void register_ns_t(std::vector<KernelSet>& reg) {
  add_set<TensorEl<2, 1, 3>, NSModel, TL>(reg, 1);
  add_set<TensorEl<2, 2, 4>, NSModel, TL>(reg, 1);
  add_set<TensorEl<2, 3, 5>, NSModel, TL>(reg, 1);
  add_set<TensorEl<2, 4, 6>, NSModel, TL>(reg, 1);
}
}  // namespace ldg
