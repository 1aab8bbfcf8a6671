// Compiled hex kernel instances with tile shape Tile0.
#include "inst_hex.cuh"
namespace ldg {
template void register_hex_t<Tile0>(std::vector<KernelSet>& reg);
}  // namespace ldg
