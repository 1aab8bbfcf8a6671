// Compiled hex kernel instances with tile shape Tile2.
#include "inst_hex.cuh"
namespace ldg {
template void register_hex_t<Tile2>(std::vector<KernelSet>& reg);
}  // namespace ldg
