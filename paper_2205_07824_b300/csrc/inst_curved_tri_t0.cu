// Compiled curved-triangle kernel instances (scalar models) with tile shape Tile0.
#include "inst_curved.cuh"
namespace ldg {
template void register_curved_tri_t<Tile0>(std::vector<KernelSet>& reg);
}  // namespace ldg
