// Compiled hex kernel instances with tile shape Tile1.
#include "inst_hex.cuh"
namespace ldg {
template void register_hex_t<Tile1>(std::vector<KernelSet>& reg);
}  // namespace ldg
