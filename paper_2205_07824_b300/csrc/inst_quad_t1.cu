// Compiled quad kernel instances with tile shape Tile1.
#include "inst_quad.cuh"
namespace ldg {
template void register_quad_t<Tile1>(std::vector<KernelSet>& reg);
}  // namespace ldg
