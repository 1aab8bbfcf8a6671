// Compiled quad kernel instances with tile shape Tile2.
#include "inst_quad.cuh"
namespace ldg {
template void register_quad_t<Tile2>(std::vector<KernelSet>& reg);
}  // namespace ldg
