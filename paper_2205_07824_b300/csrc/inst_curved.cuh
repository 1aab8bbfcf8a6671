// Curved-element instances, p = 1..4. Quadrilaterals: Poisson and convection-diffusion
// with p + 1 Gauss points per direction, Euler and Navier-Stokes with p + 2. Triangles:
// Poisson and convection-diffusion with p + 2 collapsed Gauss points per direction.
#pragma once
#include "ldg_launch.cuh"
namespace ldg {
template <class TL> void register_curved_scalar_t(std::vector<KernelSet>& reg) {
  add_set<CurvedQuadEl<1, 2>, ScalarModel<2, false>, TL>(reg, 1);
  add_set<CurvedQuadEl<2, 3>, ScalarModel<2, false>, TL>(reg, 1);
  add_set<CurvedQuadEl<3, 4>, ScalarModel<2, false>, TL>(reg, 1);
  add_set<CurvedQuadEl<4, 5>, ScalarModel<2, false>, TL>(reg, 1);
  add_set<CurvedQuadEl<1, 2>, ScalarModel<2, true>, TL>(reg, 1);
  add_set<CurvedQuadEl<2, 3>, ScalarModel<2, true>, TL>(reg, 1);
  add_set<CurvedQuadEl<3, 4>, ScalarModel<2, true>, TL>(reg, 1);
  add_set<CurvedQuadEl<4, 5>, ScalarModel<2, true>, TL>(reg, 1);
}
template <class TL> void register_curved_gas_t(std::vector<KernelSet>& reg) {
  add_set<CurvedQuadEl<1, 3>, EulerModel, TL>(reg, 1);
  add_set<CurvedQuadEl<2, 4>, EulerModel, TL>(reg, 1);
  add_set<CurvedQuadEl<3, 5>, EulerModel, TL>(reg, 1);
  add_set<CurvedQuadEl<4, 6>, EulerModel, TL>(reg, 1);
  add_set<CurvedQuadEl<1, 3>, NSModel, TL>(reg, 1);
  add_set<CurvedQuadEl<2, 4>, NSModel, TL>(reg, 1);
  add_set<CurvedQuadEl<3, 5>, NSModel, TL>(reg, 1);
  add_set<CurvedQuadEl<4, 6>, NSModel, TL>(reg, 1);
}
template <class TL> void register_curved_tri_t(std::vector<KernelSet>& reg) {
  add_set<CurvedTriEl<1, 3>, ScalarModel<2, false>, TL>(reg, 0);
  add_set<CurvedTriEl<2, 4>, ScalarModel<2, false>, TL>(reg, 0);
  add_set<CurvedTriEl<3, 5>, ScalarModel<2, false>, TL>(reg, 0);
  add_set<CurvedTriEl<4, 6>, ScalarModel<2, false>, TL>(reg, 0);
  add_set<CurvedTriEl<1, 3>, ScalarModel<2, true>, TL>(reg, 0);
  add_set<CurvedTriEl<2, 4>, ScalarModel<2, true>, TL>(reg, 0);
  add_set<CurvedTriEl<3, 5>, ScalarModel<2, true>, TL>(reg, 0);
  add_set<CurvedTriEl<4, 6>, ScalarModel<2, true>, TL>(reg, 0);
}
}  // namespace ldg
