// Compiled tri kernel instances with tile shape Tile3.
#include "inst_tri.cuh"
namespace ldg {
template void register_tri_t<Tile3>(std::vector<KernelSet>& reg);
}  // namespace ldg
