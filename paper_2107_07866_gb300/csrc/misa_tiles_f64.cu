// misa_tiles_f64.cu -- the FP64 tile kernels of every shape; one of the
// units compiled in parallel.
#include "misa_tiles_impl.cuh"

namespace misa {

MISA_TILES_INSTANTIATE(double, 0)
MISA_TILES_INSTANTIATE(double, 1)
MISA_TILES_INSTANTIATE(double, 2)
MISA_TILES_INSTANTIATE(double, 3)
MISA_TILES_INSTANTIATE(double, 4)
MISA_TILES_INSTANTIATE(double, 5)
MISA_TILES_INSTANTIATE(double, 6)

}  // namespace misa
