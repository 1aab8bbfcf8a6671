// Compiled Navier-Stokes kernel instances with tile shape Tile1.
#include "inst_ns.cuh"
namespace ldg {
template void register_ns_t<Tile1>(std::vector<KernelSet>& reg);
}  // namespace ldg
