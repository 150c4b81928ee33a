// misa_tiles.cuh -- tile shapes of the gather passes and the launch
// interface of their kernels.  The kernels of each precision are
// instantiated in a translation unit of their own (misa_tiles_f32.cu,
// misa_tiles_f64.cu), compiled beside the host runtime (misa_api.cu).
#pragma once

#include <cuda_runtime.h>

#include "misa.h"
#include "misa_kernels.cuh"

namespace misa {

struct TileShape {
    int tx, ty, tz;
};
constexpr TileShape kTiles[] = {{8, 8, 8}, {8, 8, 4}, {8, 4, 4}, {16, 8, 4}, {8, 8, 16}, {8, 8, 12}, {16, 8, 8}};
constexpr int kNTiles = sizeof(kTiles) / sizeof(kTiles[0]);

// Shapes each precision's gathers are built for: FP64 runs one thread per
// site (2 tx ty tz <= 1024); FP32 runs two sites per thread folded in z
// (tz even, tx ty tz <= 1024); each parity fills whole warps.
constexpr bool tile_ok(int prec, const TileShape &t)
{
    const int cells = t.tx * t.ty * t.tz;
    if (prec == MISA_FP64) return 2 * cells <= 1024 && cells % 32 == 0;
    return t.tz % 2 == 0 && cells <= 1024 && (cells / 2) % 32 == 0;
}

// What the tile launches take from a handle.
struct TileLaunch {
    cudaStream_t st;
    size_t smem_density, smem_force;    // single-type passes
    size_t smem_alloy_d, smem_alloy_f;  // FP32 alloy passes (0: the shape's pass does not fit)
    int nsm;                            // SMs of the device
    int nsp;                            // species (> 1: the alloy passes run)
    bool dens_db;                       // FP32 density pass double-buffers its tiles
    bool dens_n3;                       // FP32 density pass with Newton's third law inside tiles
};

// Per shape K (an index into kTiles): dynamic shared-memory attributes of
// the density (force = false) or force kernels, and one density / force
// launch over the tiles of g on L.st (grid CTAs walk the tile list; the alloy
// force pass may run more CTAs per SM).  Instantiated for T = float in
// misa_tiles_f32_{a,b,c}.cu and for T = double in misa_tiles_f64.cu.
template <typename T, int K>
cudaError_t tile_attrs_k(bool force, const TileLaunch &L);
template <typename T, int K>
void tile_density_k(const TileLaunch &L, const GatherArgs<T> &g, int grid, bool energy);
template <typename T, int K>
void tile_force_k(const TileLaunch &L, const GatherArgs<T> &g, int grid, bool energy);

// the same with the shape chosen at run time (k built for T)
#define MISA_TILE_SWITCH(k, CALL)   \
    switch (k) {                    \
    case 0: return CALL(0);         \
    case 1: return CALL(1);         \
    case 2: return CALL(2);         \
    case 3: return CALL(3);         \
    case 4: return CALL(4);         \
    case 5: return CALL(5);         \
    default: return CALL(6);        \
    }

template <typename T>
inline cudaError_t tile_attrs(int k, bool force, const TileLaunch &L)
{
#define MISA_CALL(K) tile_attrs_k<T, K>(force, L)
    MISA_TILE_SWITCH(k, MISA_CALL)
#undef MISA_CALL
}

template <typename T>
inline void tile_density(int k, const TileLaunch &L, const GatherArgs<T> &g, int grid, bool energy)
{
#define MISA_CALL(K) tile_density_k<T, K>(L, g, grid, energy)
    MISA_TILE_SWITCH(k, MISA_CALL)
#undef MISA_CALL
}

template <typename T>
inline void tile_force(int k, const TileLaunch &L, const GatherArgs<T> &g, int grid, bool energy)
{
#define MISA_CALL(K) tile_force_k<T, K>(L, g, grid, energy)
    MISA_TILE_SWITCH(k, MISA_CALL)
#undef MISA_CALL
}

#undef MISA_TILE_SWITCH

}  // namespace misa
