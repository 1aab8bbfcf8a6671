// Compiled tri kernel instances with tile shape Tile0.
#include "inst_tri.cuh"
namespace ldg {
template void register_tri_t<Tile0>(std::vector<KernelSet>& reg);
}  // namespace ldg
