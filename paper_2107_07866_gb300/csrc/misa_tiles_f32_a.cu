// misa_tiles_f32_a.cu -- FP32 tile kernels (packed single-type and alloy gathers) of
// the shapes 8x8x8, 8x8x4, 8x4x4; one of the units compiled in parallel.
#include "misa_tiles_impl.cuh"

namespace misa {

MISA_TILES_INSTANTIATE(float, 0)
MISA_TILES_INSTANTIATE(float, 1)
MISA_TILES_INSTANTIATE(float, 2)

}  // namespace misa
