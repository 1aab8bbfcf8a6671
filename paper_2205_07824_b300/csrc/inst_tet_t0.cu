// Compiled tetrahedron kernel instances with tile shape Tile0.
#include "inst_tet.cuh"
namespace ldg {
template void register_tet_t<Tile0>(std::vector<KernelSet>& reg);
}  // namespace ldg
