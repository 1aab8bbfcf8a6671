// Compiled Navier-Stokes kernel instances with tile shape Tile3.
#include "inst_ns.cuh"
namespace ldg {
template void register_ns_t<Tile3>(std::vector<KernelSet>& reg);
}  // namespace ldg
