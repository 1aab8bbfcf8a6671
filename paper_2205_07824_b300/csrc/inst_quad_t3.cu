// Compiled quad kernel instances with tile shape Tile3.
#include "inst_quad.cuh"
namespace ldg {
template void register_quad_t<Tile3>(std::vector<KernelSet>& reg);
}  // namespace ldg
