// Compiled tetrahedron kernel instances with tile shape Tile1.
#include "inst_tet.cuh"
namespace ldg {
template void register_tet_t<Tile1>(std::vector<KernelSet>& reg);
}  // namespace ldg
