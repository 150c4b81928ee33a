// misa_tiles_impl.cuh -- the tile kernels of every shape behind the launch
// interface of misa_tiles.cuh; included by the per-precision translation
// units, which instantiate it for their type.
#pragma once

#include "misa_alloy_packed.cuh"
#include "misa_newton3.cuh"
#include "misa_packed.cuh"
#include "misa_tiles.cuh"

namespace misa {

// one instantiation of the tile kernels per tile shape: FP32 the packed
// two-sites-per-thread gathers (single type or alloy), FP64 one thread per site
template <typename T, int TX, int TY, int TZ>
struct TileKernels {
    static constexpr bool kF32 = sizeof(T) == 4;
    static constexpr bool kBuilt = kF32 ? (TZ % 2 == 0 && TX * TY * TZ <= 1024) : (2 * TX * TY * TZ <= 1024);

    template <typename K>
    static cudaError_t smem(K kernel, size_t bytes)
    {
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    }

    static cudaError_t attrs_density(const TileLaunch &L)
    {
        cudaError_t e = cudaSuccess;
        if constexpr (!kBuilt) {
            return cudaErrorInvalidValue;
        } else if constexpr (kF32) {
            const size_t d = L.smem_density;
            if (L.dens_n3) {
                if (e == cudaSuccess) e = smem(k_density_n3<TX, TY, TZ, false, true>, d);
                if (e == cudaSuccess) e = smem(k_density_n3<TX, TY, TZ, true, true>, d);
                if (e == cudaSuccess) e = smem(k_density_n3<TX, TY, TZ, false, false>, d);
                if (e == cudaSuccess) e = smem(k_density_n3<TX, TY, TZ, true, false>, d);
            } else {
                if (e == cudaSuccess) e = smem(k_density_p<TX, TY, TZ, false, true>, d);
                if (e == cudaSuccess) e = smem(k_density_p<TX, TY, TZ, true, true>, d);
                if (e == cudaSuccess) e = smem(k_density_p<TX, TY, TZ, false, false>, d);
                if (e == cudaSuccess) e = smem(k_density_p<TX, TY, TZ, true, false>, d);
            }
            if (L.smem_alloy_d) {
                if (e == cudaSuccess) e = smem(k_density_pa<TX, TY, TZ, false>, L.smem_alloy_d);
                if (e == cudaSuccess) e = smem(k_density_pa<TX, TY, TZ, true>, L.smem_alloy_d);
            }
        } else {
            if (e == cudaSuccess) e = smem(k_density<T, TX, TY, TZ, false>, L.smem_density);
            if (e == cudaSuccess) e = smem(k_density<T, TX, TY, TZ, true>, L.smem_density);
        }
        return e;
    }

    static cudaError_t attrs_force(const TileLaunch &L)
    {
        cudaError_t e = cudaSuccess;
        if constexpr (!kBuilt) {
            return cudaErrorInvalidValue;
        } else if constexpr (kF32) {
            if (e == cudaSuccess) e = smem(k_force_p<TX, TY, TZ, false>, L.smem_force);
            if (e == cudaSuccess) e = smem(k_force_p<TX, TY, TZ, true>, L.smem_force);
            if (L.smem_alloy_f) {
                if (e == cudaSuccess) e = smem(k_force_pa<TX, TY, TZ, false>, L.smem_alloy_f);
                if (e == cudaSuccess) e = smem(k_force_pa<TX, TY, TZ, true>, L.smem_alloy_f);
            }
        } else {
            if (e == cudaSuccess) e = smem(k_force<T, TX, TY, TZ, false>, L.smem_force);
            if (e == cudaSuccess) e = smem(k_force<T, TX, TY, TZ, true>, L.smem_force);
        }
        return e;
    }

    static void density(const TileLaunch &L, const GatherArgs<T> &g, int grid, bool energy)
    {
        if constexpr (!kBuilt) {
            return;
        } else if constexpr (kF32) {
            constexpr int nt = TX * TY * TZ;
            if (L.nsp > 1) {  // alloys
                if (energy) k_density_pa<TX, TY, TZ, true><<<grid, nt, L.smem_alloy_d, L.st>>>(g);
                else k_density_pa<TX, TY, TZ, false><<<grid, nt, L.smem_alloy_d, L.st>>>(g);
                return;
            }
            const size_t b = L.smem_density;
            if (L.dens_n3) {
                if (L.dens_db) {
                    if (energy) k_density_n3<TX, TY, TZ, true, true><<<grid, nt, b, L.st>>>(g);
                    else k_density_n3<TX, TY, TZ, false, true><<<grid, nt, b, L.st>>>(g);
                } else {
                    if (energy) k_density_n3<TX, TY, TZ, true, false><<<grid, nt, b, L.st>>>(g);
                    else k_density_n3<TX, TY, TZ, false, false><<<grid, nt, b, L.st>>>(g);
                }
                return;
            }
            if (L.dens_db) {
                if (energy) k_density_p<TX, TY, TZ, true, true><<<grid, nt, b, L.st>>>(g);
                else k_density_p<TX, TY, TZ, false, true><<<grid, nt, b, L.st>>>(g);
            } else {
                if (energy) k_density_p<TX, TY, TZ, true, false><<<grid, nt, b, L.st>>>(g);
                else k_density_p<TX, TY, TZ, false, false><<<grid, nt, b, L.st>>>(g);
            }
        } else {
            constexpr int nt = 2 * TX * TY * TZ;
            if (energy) k_density<T, TX, TY, TZ, true><<<grid, nt, L.smem_density, L.st>>>(g);
            else k_density<T, TX, TY, TZ, false><<<grid, nt, L.smem_density, L.st>>>(g);
        }
    }

    static void force(const TileLaunch &L, const GatherArgs<T> &g, int grid, bool energy)
    {
        if constexpr (!kBuilt) {
            return;
        } else if constexpr (kF32) {
            constexpr int nt = TX * TY * TZ;
            if (L.nsp > 1) {  // alloys
                const int blocks = kForcePaBlocks<TX, TY, TZ>;
                const int g2 = g.ntiles < blocks * L.nsm ? g.ntiles : blocks * L.nsm;
                if (energy) k_force_pa<TX, TY, TZ, true><<<g2, nt, L.smem_alloy_f, L.st>>>(g);
                else k_force_pa<TX, TY, TZ, false><<<g2, nt, L.smem_alloy_f, L.st>>>(g);
                return;
            }
            if (energy) k_force_p<TX, TY, TZ, true><<<grid, nt, L.smem_force, L.st>>>(g);
            else k_force_p<TX, TY, TZ, false><<<grid, nt, L.smem_force, L.st>>>(g);
        } else {
            constexpr int nt = 2 * TX * TY * TZ;
            if (energy) k_force<T, TX, TY, TZ, true><<<grid, nt, L.smem_force, L.st>>>(g);
            else k_force<T, TX, TY, TZ, false><<<grid, nt, L.smem_force, L.st>>>(g);
        }
    }
};

static_assert(kNTiles == 7, "the tile dispatch covers seven shapes");

template <typename T, int K>
using TileK = TileKernels<T, kTiles[K].tx, kTiles[K].ty, kTiles[K].tz>;

template <typename T, int K>
cudaError_t tile_attrs_k(bool force, const TileLaunch &L)
{
    return force ? TileK<T, K>::attrs_force(L) : TileK<T, K>::attrs_density(L);
}

template <typename T, int K>
void tile_density_k(const TileLaunch &L, const GatherArgs<T> &g, int grid, bool energy)
{
    TileK<T, K>::density(L, g, grid, energy);
}

template <typename T, int K>
void tile_force_k(const TileLaunch &L, const GatherArgs<T> &g, int grid, bool energy)
{
    TileK<T, K>::force(L, g, grid, energy);
}

// explicit instantiation of shape K for type T (in the per-precision units)
#define MISA_TILES_INSTANTIATE(T, K)                                                                  \
    template cudaError_t tile_attrs_k<T, K>(bool, const TileLaunch &);                                \
    template void tile_density_k<T, K>(const TileLaunch &, const GatherArgs<T> &, int, bool);         \
    template void tile_force_k<T, K>(const TileLaunch &, const GatherArgs<T> &, int, bool);

}  // namespace misa
