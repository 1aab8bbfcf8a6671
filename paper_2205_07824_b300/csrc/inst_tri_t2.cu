// Compiled tri kernel instances with tile shape Tile2.
#include "inst_tri.cuh"
namespace ldg {
template void register_tri_t<Tile2>(std::vector<KernelSet>& reg);
}  // namespace ldg
