// Compiled Navier-Stokes kernel instances with tile shape Tile2.
#include "inst_ns.cuh"
namespace ldg {
template void register_ns_t<Tile2>(std::vector<KernelSet>& reg);
}  // namespace ldg
