// Kernel instantiations for one group of (d, p) configurations.
#include "kernels.cuh"
namespace hdg {
HDG_INSTANTIATE(2, 1)
HDG_INSTANTIATE(2, 2)
HDG_INSTANTIATE(2, 3)
}  // namespace hdg
