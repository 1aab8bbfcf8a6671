// Compiled Navier-Stokes kernel instances with tile shape Tile0.
#include "inst_ns.cuh"
namespace ldg {
template void register_ns_t<Tile0>(std::vector<KernelSet>& reg);
}  // namespace ldg
