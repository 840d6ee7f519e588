// jxf_flux_launch.cuh -- definitions of the face-sweep launchers declared in
// jxf_ops.cuh, and the macro that instantiates them for one (storage type,
// model, viscous half-width, scheme family) in a unit of its own.
#pragma once
#include "jxf_ops.cuh"

namespace jxf {

template <typename T, int MODEL, int NDIM, int VH, int RSV> void launch_flux(const Dev &P, int d, cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value) {  // axes y, z: staged in shared memory
        if (d > 0) {
            const dim3 grid((P.n[0] + kTileX - 1) / kTileX, (P.n[d] + kTileD - 1) / kTileD,
                            NDIM == 3 ? P.n[3 - d] : 1);
            if constexpr (NDIM > 1)
                if (d == 1) k_flux_td<T, MODEL, NDIM, 1, VH, RSV><<<grid, kFluxThreads, 0, s>>>(P);
            if constexpr (NDIM > 2)
                if (d == 2) k_flux_td<T, MODEL, NDIM, 2, VH, RSV><<<grid, kFluxThreads, 0, s>>>(P);
            return;
        }
    }
    long long nf = 1;
    for (int e = 0; e < 3; ++e) nf *= P.n[e] + (e == d ? 1 : 0);
    const unsigned g = grid_for(nf, kFluxThreads);
    if (d == 0) k_flux<T, MODEL, NDIM, 0, VH, RSV><<<g, kFluxThreads, 0, s>>>(P);
    if constexpr (NDIM > 1)
        if (d == 1) k_flux<T, MODEL, NDIM, 1, VH, RSV><<<g, kFluxThreads, 0, s>>>(P);
    if constexpr (NDIM > 2)
        if (d == 2) k_flux<T, MODEL, NDIM, 2, VH, RSV><<<g, kFluxThreads, 0, s>>>(P);
}

template <typename T, int MODEL, int NDIM, int VH, int RSV>
void launch_flux_update(const Dev &P, int epi, cudaStream_t s) {
    if constexpr (NDIM >= 2 && std::is_same<T, float>::value) {
        const dim3 grid = fused_grid(P, NDIM);
        k_flux_update<T, MODEL, NDIM, VH, RSV><<<grid, kFluxThreads, 0, s>>>(P, epi, kFusedRun);
    }
}

template <typename T, int MODEL, int NDIM, int VH, int RSV>
void launch_flux_batch(const Dev *devs, const Tile *tiles, int ntiles, unsigned *ticket, int d, int grid,
                       cudaStream_t s) {
    if (d == 0) k_flux_batch<T, MODEL, NDIM, 0, VH, RSV><<<grid, kFluxThreads, 0, s>>>(devs, tiles, ntiles, ticket);
    if constexpr (NDIM > 1)
        if (d == 1) k_flux_batch<T, MODEL, NDIM, 1, VH, RSV><<<grid, kFluxThreads, 0, s>>>(devs, tiles, ntiles, ticket);
    if constexpr (NDIM > 2)
        if (d == 2) k_flux_batch<T, MODEL, NDIM, 2, VH, RSV><<<grid, kFluxThreads, 0, s>>>(devs, tiles, ntiles, ticket);
}

}  // namespace jxf

#define JXF_INSTANTIATE_FLUX_NDIM(T, MODEL, NDIM, VH, RSV)                                                    \
    template void jxf::launch_flux<T, MODEL, NDIM, VH, RSV>(const jxf::Dev &, int, cudaStream_t);           \
    template void jxf::launch_flux_update<T, MODEL, NDIM, VH, RSV>(const jxf::Dev &, int, cudaStream_t);    \
    template void jxf::launch_flux_batch<T, MODEL, NDIM, VH, RSV>(const jxf::Dev *, const jxf::Tile *, int, \
                                                             unsigned *, int, int, cudaStream_t);
#define JXF_INSTANTIATE_FLUX(T, MODEL, VH, RSV)      \
    JXF_INSTANTIATE_FLUX_NDIM(T, MODEL, 1, VH, RSV) \
    JXF_INSTANTIATE_FLUX_NDIM(T, MODEL, 2, VH, RSV) \
    JXF_INSTANTIATE_FLUX_NDIM(T, MODEL, 3, VH, RSV)

// In the unit that builds the ops table: the viscous variants are compiled
// in their own units, not here.
#define JXF_EXTERN_FLUX_NDIM(T, MODEL, NDIM, VH, RSV)                                                          \
    extern template void jxf::launch_flux<T, MODEL, NDIM, VH, RSV>(const jxf::Dev &, int, cudaStream_t);      \
    extern template void jxf::launch_flux_update<T, MODEL, NDIM, VH, RSV>(const jxf::Dev &, int, cudaStream_t); \
    extern template void jxf::launch_flux_batch<T, MODEL, NDIM, VH, RSV>(const jxf::Dev *, const jxf::Tile *, \
                                                                    int, unsigned *, int, int, cudaStream_t);
#define JXF_EXTERN_FLUX(T, MODEL, VH, RSV)      \
    JXF_EXTERN_FLUX_NDIM(T, MODEL, 1, VH, RSV) \
    JXF_EXTERN_FLUX_NDIM(T, MODEL, 2, VH, RSV) \
    JXF_EXTERN_FLUX_NDIM(T, MODEL, 3, VH, RSV)
