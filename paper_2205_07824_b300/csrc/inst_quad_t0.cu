// Compiled quad kernel instances with tile shape Tile0.
#include "inst_quad.cuh"
namespace ldg {
template void register_quad_t<Tile0>(std::vector<KernelSet>& reg);
}  // namespace ldg
