// Kernel instantiations for one group of (d, p) configurations.
#include "solve.cuh"
namespace hdg {
HDG_INSTANTIATE(2, 1)
HDG_INSTANTIATE_SOLVE(2, 1)
HDG_INSTANTIATE_MIXED(2, 1)
HDG_INSTANTIATE(2, 2)
HDG_INSTANTIATE_SOLVE(2, 2)
HDG_INSTANTIATE_MIXED(2, 2)
HDG_INSTANTIATE(2, 3)
HDG_INSTANTIATE_SOLVE(2, 3)
HDG_INSTANTIATE_MIXED(2, 3)
}  // namespace hdg
