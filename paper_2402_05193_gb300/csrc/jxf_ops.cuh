// jxf_ops.cuh -- launch table of one (storage type, model) instantiation.
#pragma once
#include "jxf_adjoint.cuh"
#include "jxf_batch.cuh"
#include "jxf_impl.cuh"

namespace jxf {

struct Ops {
    void (*flux)(const Dev &, int d, cudaStream_t);
    // the last axis's faces fused with the stage update (ndim >= 2)
    void (*flux_update)(const Dev &, int epi, cudaStream_t);
    void (*update)(const Dev &, int mode, int epi, cudaStream_t);
    void (*prim)(const Dev &, int epi, cudaStream_t);
    void (*from_prim)(const Dev &, const double *W64, cudaStream_t);
    void (*aux)(const Dev &, cudaStream_t);  // per-cell auxiliary pass (viscous gradient / THINC normal)
    // reverse mode (single-phase model only; null otherwise)
    void (*flux_vjp)(const Dev &, int d, cudaStream_t);  // every axis, then gather_vjp
    void (*gather_vjp)(const Dev &, cudaStream_t);
    void (*prim_vjp)(const Dev &, cudaStream_t);
    void (*axpbypcz)(void *out, long long n, double a, const void *x, double b, const void *y,
                     double c, const void *z, cudaStream_t);
    // batched persistent kernels (grid = persistent blocks)
    void (*flux_batch)(const Dev *devs, const Tile *tiles, int ntiles, unsigned *ticket, int d,
                       int vh, int teno, int grid, cudaStream_t);
    void (*update_batch)(const Dev *devs, const Tile *tiles, int ntiles, unsigned *ticket,
                         double *part, int epi, int grid, cudaStream_t);
    void (*aux_batch)(const Dev *devs, const Tile *tiles, int ntiles, unsigned *ticket, int grid,
                      cudaStream_t);
};

inline unsigned grid_for(long long n, int threads) {
    return (unsigned)((n + threads - 1) / threads);
}

// The fused last-axis sweep: cells per run along the last axis, and its
// grid (kFluxThreads columns per block by runs); one partial record per
// block.  Runs of 16 cells keep the extra face per run at 1/16 and give a
// 128^3 grid 1024 blocks.
#ifndef JXF_FUSED_RUN
#define JXF_FUSED_RUN 16
#endif
constexpr int kFusedRun = JXF_FUSED_RUN;  // overridable at build time for tuning sweeps
inline dim3 fused_grid(const Dev &P, int ndim) {
    const long long plane = (long long)P.n[0] * (ndim == 3 ? P.n[1] : 1);
    return dim3(grid_for(plane, kFluxThreads), (unsigned)((P.n[ndim - 1] + kFusedRun - 1) / kFusedRun));
}

// Face-sweep launchers, one instantiation per (storage type, model, ndim,
// viscous stencil half-width VH (0 = no viscous flux), scheme family RSV (0:
// WENO5, 2: TENO6-A)), compiled in their own units (jxf_flux_launch.cuh) so
// that each variant gets its own register allocation.
template <typename T, int MODEL, int NDIM, int VH, int RSV>
void launch_flux(const Dev &P, int d, cudaStream_t s);
template <typename T, int MODEL, int NDIM, int VH, int RSV>
void launch_flux_update(const Dev &P, int epi, cudaStream_t s);
template <typename T, int MODEL, int NDIM, int VH, int RSV>
void launch_flux_batch(const Dev *devs, const Tile *tiles, int ntiles, unsigned *ticket, int d, int grid,
                       cudaStream_t s);

template <typename T, int MODEL, int NDIM> struct Launch {
    template <int RSV> static void flux_rs(const Dev &P, int d, cudaStream_t s) {
        if constexpr (MODEL == JXF_SPM) {
            if (P.viscous) {
                if (P.visc_half == 1) return launch_flux<T, MODEL, NDIM, 1, RSV>(P, d, s);
                if (P.visc_half == 3) return launch_flux<T, MODEL, NDIM, 3, RSV>(P, d, s);
                return launch_flux<T, MODEL, NDIM, 2, RSV>(P, d, s);
            }
        }
        launch_flux<T, MODEL, NDIM, 0, RSV>(P, d, s);
    }
    static void flux(const Dev &P, int d, cudaStream_t s) {
        if (P.teno) flux_rs<2>(P, d, s);
        else flux_rs<0>(P, d, s);
    }
    template <int RSV> static void flux_update_rs(const Dev &P, int epi, cudaStream_t s) {
        if constexpr (MODEL == JXF_SPM) {
            if (P.viscous) {
                if (P.visc_half == 1) return launch_flux_update<T, MODEL, NDIM, 1, RSV>(P, epi, s);
                if (P.visc_half == 3) return launch_flux_update<T, MODEL, NDIM, 3, RSV>(P, epi, s);
                return launch_flux_update<T, MODEL, NDIM, 2, RSV>(P, epi, s);
            }
        }
        launch_flux_update<T, MODEL, NDIM, 0, RSV>(P, epi, s);
    }
    static void flux_update(const Dev &P, int epi, cudaStream_t s) {
        if (P.teno) flux_update_rs<2>(P, epi, s);
        else flux_update_rs<0>(P, epi, s);
    }
    static void update(const Dev &P, int mode, int epi, cudaStream_t s) {
        k_update<T, MODEL, NDIM><<<grid_for(P.ncell, kCellThreads), kCellThreads, 0, s>>>(P, mode, epi);
    }
    static void prim(const Dev &P, int epi, cudaStream_t s) {
        k_prim<T, MODEL, NDIM><<<grid_for(P.ncell, kCellThreads), kCellThreads, 0, s>>>(P, epi);
    }
    static void from_prim(const Dev &P, const double *W64, cudaStream_t s) {
        k_from_prim<T, MODEL, NDIM><<<grid_for(P.ncell, kCellThreads), kCellThreads, 0, s>>>(P, W64);
    }
    static void aux(const Dev &P, cudaStream_t s) {
        if constexpr (std::is_same<T, float>::value && MODEL == JXF_SPM && kAuxCells > 1) {
            // kAuxCells cells a thread with vector accesses, where rows hold a
            // multiple of kAuxCells cells and the arrays are aligned to the vector
            constexpr unsigned al = 4u * kAuxCells - 1u;
            if (P.n[0] % kAuxCells == 0 && P.vstride % kAuxCells == 0 && ((uintptr_t)P.W & al) == 0 &&
                ((uintptr_t)P.G & al) == 0) {
                k_aux_vec<NDIM><<<grid_for(P.ncell / kAuxCells, kCellThreads), kCellThreads, 0, s>>>(P);
                return;
            }
        }
        k_aux<T, MODEL, NDIM><<<grid_for(P.ncell, kCellThreads), kCellThreads, 0, s>>>(P);
    }
    static void aux_batch(const Dev *devs, const Tile *tiles, int ntiles, unsigned *ticket, int grid,
                          cudaStream_t s) {
        k_aux_batch<T, MODEL, NDIM><<<grid, kCellThreads, 0, s>>>(devs, tiles, ntiles, ticket);
    }
    static void flux_vjp(const Dev &P, int d, cudaStream_t s) {
        if constexpr (MODEL == JXF_SPM) {
            long long nf = 1;
            for (int e = 0; e < 3; ++e) nf *= P.n[e] + (e == d ? 1 : 0);
            const unsigned g = grid_for(nf, kFluxThreads);
            if (d == 0) k_flux_vjp<T, NDIM, 0><<<g, kFluxThreads, 0, s>>>(P);
            if constexpr (NDIM > 1)
                if (d == 1) k_flux_vjp<T, NDIM, 1><<<g, kFluxThreads, 0, s>>>(P);
            if constexpr (NDIM > 2)
                if (d == 2) k_flux_vjp<T, NDIM, 2><<<g, kFluxThreads, 0, s>>>(P);
        }
    }
    static void gather_vjp(const Dev &P, cudaStream_t s) {
        if constexpr (MODEL == JXF_SPM)
            k_gather_vjp<T, NDIM><<<grid_for(P.ncell, kCellThreads), kCellThreads, 0, s>>>(P);
    }
    static void prim_vjp(const Dev &P, cudaStream_t s) {
        if constexpr (MODEL == JXF_SPM)
            k_prim_vjp<T, NDIM><<<grid_for(P.ncell, kCellThreads), kCellThreads, 0, s>>>(P);
    }
    static void axpbypcz(void *out, long long n, double a, const void *x, double b, const void *y,
                         double c, const void *z, cudaStream_t s) {
        k_axpbypcz<T><<<grid_for(n, 256), 256, 0, s>>>(static_cast<T *>(out), n, a,
                                                        static_cast<const T *>(x), b,
                                                        static_cast<const T *>(y), c,
                                                        static_cast<const T *>(z));
    }
    template <int RSV>
    static void flux_batch_rs(const Dev *devs, const Tile *tiles, int ntiles, unsigned *ticket, int d,
                              int vh, int grid, cudaStream_t s) {
        if constexpr (MODEL == JXF_SPM) {
            if (vh == 1) return launch_flux_batch<T, MODEL, NDIM, 1, RSV>(devs, tiles, ntiles, ticket, d, grid, s);
            if (vh == 2) return launch_flux_batch<T, MODEL, NDIM, 2, RSV>(devs, tiles, ntiles, ticket, d, grid, s);
            if (vh == 3) return launch_flux_batch<T, MODEL, NDIM, 3, RSV>(devs, tiles, ntiles, ticket, d, grid, s);
        }
        launch_flux_batch<T, MODEL, NDIM, 0, RSV>(devs, tiles, ntiles, ticket, d, grid, s);
    }
    static void flux_batch(const Dev *devs, const Tile *tiles, int ntiles, unsigned *ticket, int d,
                           int vh, int teno, int grid, cudaStream_t s) {
        if (teno) flux_batch_rs<2>(devs, tiles, ntiles, ticket, d, vh, grid, s);
        else flux_batch_rs<0>(devs, tiles, ntiles, ticket, d, vh, grid, s);
    }
    static void update_batch(const Dev *devs, const Tile *tiles, int ntiles, unsigned *ticket,
                             double *part, int epi, int grid, cudaStream_t s) {
        k_update_batch<T, MODEL, NDIM><<<grid, kCellThreads, 0, s>>>(devs, tiles, ntiles, ticket, part, epi);
    }
    static constexpr Ops ops() {
        return Ops{flux, flux_update, update, prim, from_prim, aux, MODEL == JXF_SPM ? flux_vjp : nullptr,
                   MODEL == JXF_SPM ? gather_vjp : nullptr,
                   MODEL == JXF_SPM ? prim_vjp : nullptr, axpbypcz, flux_batch, update_batch,
                   aux_batch};
    }
};

// Defined in the instantiation units: tables for ndim = 1, 2, 3.
const Ops *ops_f64_spm(int ndim);
const Ops *ops_f64_dim(int ndim);
const Ops *ops_f32_spm(int ndim);
const Ops *ops_f32_dim(int ndim);

}  // namespace jxf

#define JXF_DEFINE_OPS(NAME, T, MODEL)                                          \
    namespace jxf {                                                             \
    const Ops *NAME(int ndim) {                                                 \
        static const Ops t1 = Launch<T, MODEL, 1>::ops();                       \
        static const Ops t2 = Launch<T, MODEL, 2>::ops();                       \
        static const Ops t3 = Launch<T, MODEL, 3>::ops();                       \
        return ndim == 1 ? &t1 : (ndim == 2 ? &t2 : (ndim == 3 ? &t3 : nullptr)); \
    }                                                                           \
    }
