// Kernel instantiations for one (d, p) configuration.
#include "solve.cuh"
namespace hdg {
HDG_INSTANTIATE(3, 1)
HDG_INSTANTIATE_SOLVE(3, 1)
HDG_INSTANTIATE_MIXED(3, 1)
}  // namespace hdg
