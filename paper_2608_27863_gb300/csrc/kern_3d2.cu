// Kernel instantiations for one group of (d, p) configurations.
#include "kernels.cuh"
namespace hdg {
HDG_INSTANTIATE(3, 2)
}  // namespace hdg
