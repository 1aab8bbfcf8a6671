// Compiled hex kernel instances with tile shape Tile3.
#include "inst_hex.cuh"
namespace ldg {
template void register_hex_t<Tile3>(std::vector<KernelSet>& reg);
}  // namespace ldg
