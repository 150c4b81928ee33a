// misa_tiles_f32_c.cu -- FP32 tile kernels (packed single-type and alloy gathers) of
// the shapes 8x8x12, 16x8x8; one of the units compiled in parallel.
#include "misa_tiles_impl.cuh"

namespace misa {

MISA_TILES_INSTANTIATE(float, 5)
MISA_TILES_INSTANTIATE(float, 6)

}  // namespace misa
