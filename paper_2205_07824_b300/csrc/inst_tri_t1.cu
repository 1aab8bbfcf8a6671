// Compiled tri kernel instances with tile shape Tile1.
#include "inst_tri.cuh"
namespace ldg {
template void register_tri_t<Tile1>(std::vector<KernelSet>& reg);
}  // namespace ldg
