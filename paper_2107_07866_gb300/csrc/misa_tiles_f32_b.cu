// misa_tiles_f32_b.cu -- FP32 tile kernels (packed single-type and alloy gathers) of
// the shapes 16x8x4, 8x8x16; one of the units compiled in parallel.
#include "misa_tiles_impl.cuh"

namespace misa {

MISA_TILES_INSTANTIATE(float, 3)
MISA_TILES_INSTANTIATE(float, 4)

}  // namespace misa
