// Kernel instantiations for one (d, p) configuration.
#include "solve.cuh"
namespace hdg {
HDG_INSTANTIATE(2, 3)
HDG_INSTANTIATE_SOLVE(2, 3)
HDG_INSTANTIATE_MIXED(2, 3)
}  // namespace hdg
