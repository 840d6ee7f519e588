// jxf_batch.cuh -- batched form: many independent simulations of uneven
// grid sizes advanced together by persistent kernels.
//
// Every simulation keeps its own parameter block (Dev, one copy per RK stage
// so that the stage's buffer roles and coefficients are fixed), its own dt,
// t, sums and status.  The work of a stage is cut into tiles that never
// cross a simulation -- face tiles of a tunable length per sweep axis, cell
// tiles of one block -- and a persistent grid pulls tiles from a queue
// (one atomic ticket counter per launch, reset by the step's finalisation).
// A tile runs exactly the per-face / per-cell code of the single-grid
// kernels, so each simulation's result is that of its own single-grid run.
#pragma once
#include "jxf_impl.cuh"

namespace jxf {

struct Tile {
    int sim;          // simulation index
    int slot;         // reduction-partials slot (cell tiles)
    long long start;  // first face / cell of the tile within the simulation
    long long count;  // faces / cells in the tile
};

// Take the next tile of this launch's queue and broadcast its simulation's
// stage dt, the stage's c dt in the storage type and whether the
// simulation still steps (block-uniform; thread 0 does the double work).
template <typename T>
__device__ __forceinline__ int next_tile(unsigned *ticket, const Tile *__restrict__ tiles, int ntiles,
                                         const Dev *__restrict__ devs, double &dt, T &cdt, bool &go) {
    __shared__ int sh_t, sh_go;
    __shared__ double sh_dt;
    __shared__ T sh_cdt;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int t = (int)atomicAdd(ticket, 1u);
        sh_t = t;
        if (t < ntiles) {
            const Dev &P = devs[tiles[t].sim];
            const double d = *P.dtp;
            sh_dt = d;
            sh_cdt = T(P.cc * d);
            sh_go = !(P.skip_if_done && !(d > 0.0));
        }
    }
    __syncthreads();
    const int t = sh_t;
    if (t < ntiles) {
        dt = sh_dt;
        cdt = sh_cdt;
        go = sh_go != 0;
    }
    return t;
}

template <typename T, int MODEL, int NDIM, int d, int VH, int RSV>
__global__ void __launch_bounds__(kFluxThreads, SweepMinBlocks<T, RSV>::value)
    k_flux_batch(const Dev *__restrict__ devs, const Tile *__restrict__ tiles, int ntiles,
                 unsigned *ticket) {
    for (;;) {
        double dt = 0.0;
        T cdt;
        bool go = false;
        const int t = next_tile<T>(ticket, tiles, ntiles, devs, dt, cdt, go);
        if (t >= ntiles) return;
        if (!go) continue;
        const Tile tl = tiles[t];
        const Dev &P = devs[tl.sim];
        int m[3] = {P.n[0], P.n[1], P.n[2]};
        m[d] += 1;
        const long long nface = (long long)m[0] * m[1] * m[2];
        const long long end = tl.start + tl.count;
        for (long long b = tl.start; b < end; b += blockDim.x) {
            const long long g = b + threadIdx.x;
            bool il = false, fl = false;
            if (g < end) flux_face<T, MODEL, NDIM, d, VH, RSV>(P, dt, g, m, nface, il, fl);
            if (P.limiter) count_limited(P, il, fl);
        }
    }
}

// Cell tiles hold at most one block of cells; with epi the tile's partials
// go to its slot.
template <typename T, int MODEL, int NDIM>
__global__ void __launch_bounds__(kCellThreads, CellMinBlocks<T>::value)
    k_update_batch(const Dev *__restrict__ devs, const Tile *__restrict__ tiles, int ntiles,
                   unsigned *ticket, double *part, int epi) {
    using V = Vars<MODEL, NDIM>;
    constexpr int NV = V::NV;
    for (;;) {
        double dt = 0.0;
        T cdt = T(0);
        bool go = false;
        const int t = next_tile<T>(ticket, tiles, ntiles, devs, dt, cdt, go);
        if (t >= ntiles) return;
        if (!go) continue;
        const Tile tl = tiles[t];
        const Dev &P = devs[tl.sim];
        T smax = T(0), rmin = T(3e38), U[MAXV];
        bool bad = false;
#pragma unroll
        for (int v = 0; v < NV; ++v) U[v] = T(0);
        if (threadIdx.x < tl.count)
            update_cell<T, MODEL, NDIM>(P, cdt, tl.start + threadIdx.x, 1, U, smax, rmin, bad);
        if (epi) block_partials<T, NV>(P, smax, rmin, bad, U, part + (size_t)tl.slot * (3 + MAXV));
    }
}

// The per-cell auxiliary pass (viscous velocity gradient or THINC normal)
// of every simulation, cell tiles.
template <typename T, int MODEL, int NDIM>
__global__ void __launch_bounds__(kCellThreads, CellMinBlocks<T>::value)
    k_aux_batch(const Dev *__restrict__ devs, const Tile *__restrict__ tiles, int ntiles,
                unsigned *ticket) {
    for (;;) {
        double dt = 0.0;
        T cdt;
        bool go = false;
        const int t = next_tile<T>(ticket, tiles, ntiles, devs, dt, cdt, go);
        if (t >= ntiles) return;
        if (!go) continue;
        const Tile tl = tiles[t];
        const Dev &P = devs[tl.sim];
        if (threadIdx.x < tl.count) aux_cell<T, MODEL, NDIM>(P, tl.start + threadIdx.x);
    }
}

}  // namespace jxf
