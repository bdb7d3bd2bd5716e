// Host-side construction of TMA tensor maps (the driver's cuTensorMapEncodeTiled,
// reached through the runtime's driver entry point, so the library links only
// against cudart): 3-D FP64 tiles of row-major matrices batched over elements.
#pragma once

#include <cstdint>
#include <string>

#include <cuda.h>

namespace hdg {

// Map over the FP64 array base[z][y][x] (x fastest): extents d0 (x), d1 (y), d2 (z),
// strides s1 = bytes between consecutive y, s2 = bytes between consecutive z (both
// multiples of 16), box b0 x b1 x 1 elements (b0 * 8 a multiple of 16).  Loads
// outside the extents are zero-filled.  base must be 16-byte aligned.
int make_tmap_f64_3d(CUtensorMap* m, const void* base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t s1,
                     uint64_t s2, uint32_t b0, uint32_t b1, std::string& err);

}  // namespace hdg
