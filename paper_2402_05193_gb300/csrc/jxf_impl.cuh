// jxf_impl.cuh -- device code of the GB300 finite-volume solver.
//
// Kernels (one RK stage = ndim face sweeps + one cell update):
//   k_flux<d>   one thread per face of axis d: gathers the 6-cell stencil of
//               primitives (boundary conditions resolved by index mapping),
//               WENO5 (Jiang-Shu or Z weights) or TENO6-A, component or
//               characteristic, THINC (five-equation model), interpolation
//               limiter, HLLC + upwinded face velocity, flux limiter,
//               central viscous flux of order 2/4/6; writes F = F^c - F^d
//               per face.
//   k_update    one thread per cell: divergence of the face fluxes and the
//               diffuse-interface source, RK3 stage combination (or the bare
//               right-hand side), primitives + temperature of the new state,
//               and in the last stage the CFL rate, minimum density,
//               conservation sums and admissibility, reduced per block.
//   k_aux       one thread per cell: cell-centred velocity gradient of the
//               new state (viscous) or the THINC interface normal.
//   k_finalize  one warp: deterministic reduction of the block partials
//               (first folded by k_reduce_partials on large grids), time
//               advance, next dt (CFL, viscous bound, t_end clip), status
//               word.
//   k_from_prim primitive (FP64) -> conservative state in storage precision.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "jxf.h"

namespace jxf {

constexpr int MAXV = 7;
constexpr int kFluxThreads = 128;
// minimum resident blocks of the face sweep per SM (register budget), per
// storage type; overridable at build time for tuning sweeps
#ifndef JXF_FLUX_MINB64
#define JXF_FLUX_MINB64 1
#endif
#ifndef JXF_FLUX_MINB32
#define JXF_FLUX_MINB32 8
#endif
template <typename T> struct FluxMinBlocks { static constexpr int value = JXF_FLUX_MINB32; };
template <> struct FluxMinBlocks<double> { static constexpr int value = JXF_FLUX_MINB64; };
// the same for the TENO6-A sweeps (scheme family RSV = 2), whose float
// evaluation carries both face values in packed registers
#ifndef JXF_TENO_MINB32
#define JXF_TENO_MINB32 5
#endif
template <typename T, int RSV> struct SweepMinBlocks { static constexpr int value = FluxMinBlocks<T>::value; };
template <> struct SweepMinBlocks<float, 2> { static constexpr int value = JXF_TENO_MINB32; };
constexpr int kCellThreads = 256;
// minimum resident blocks of the cell kernels (update, auxiliary pass) per
// SM, per storage type; overridable at build time for tuning sweeps
#ifndef JXF_CELL_MINB64
#define JXF_CELL_MINB64 1
#endif
#ifndef JXF_CELL_MINB32
#define JXF_CELL_MINB32 8
#endif
template <typename T> struct CellMinBlocks { static constexpr int value = JXF_CELL_MINB32; };
template <> struct CellMinBlocks<double> { static constexpr int value = JXF_CELL_MINB64; };

// device scalar slots (double)
enum {
    SC_T = 0,        // simulation time
    SC_DT = 1,       // dt of the next step (0: finished)
    SC_DT_LAST = 2,  // dt of the last step taken
    SC_RHS_DT = 3,   // dt argument of jxf_rhs
    SC_SMAX = 4,     // max CFL rate of the current state
    SC_RMIN = 5,     // min density of the current state
    SC_SUMS = 8,     // conservation sums (nv values)
    SC_N = 16
};

enum { ST_NONPHYSICAL = 1, ST_BAD_DT = 2, ST_BOUNDS = 4 };

// Division by an invariant integer via a multiplier (Granlund & Montgomery,
// "Division by invariant integers using multiplication", 1994): for
// 1 <= d < 2^31 with l = ceil(log2 d) and m = floor(2^32 (2^l - d)/d) + 1,
// n / d = (mulhi(m, n) + n) >> l for every 0 <= n < 2^31 (the sum stays
// below 2^32).  Replaces the runtime integer divisions of index decoding.
struct FastDiv {
    unsigned d = 1, m = 1;
    int l = 0;
    FastDiv() = default;
    explicit FastDiv(unsigned dd) : d(dd) {
        l = 0;
        while ((1ull << l) < dd) ++l;
        m = (unsigned)(((1ull << 32) * ((1ull << l) - dd)) / dd + 1ull);
    }
    __host__ __device__ __forceinline__ unsigned div(unsigned n) const {
#ifdef __CUDA_ARCH__
        return (__umulhi(m, n) + n) >> l;
#else
        return (unsigned)((((unsigned long long)m * n) >> 32) + n) >> l;
#endif
    }
};

// Scalar constants in the arithmetic type of the kernel using them (so that
// a float kernel never converts from double).
template <typename T> struct Cst {
    T inv_dx[3], vis_dn[3], vis_cd[3], fl_lam[3];
    T A1, A2, B1, B2, gamma0, pinf0, gm1_0, gpinf0;
    // B = gamma p_inf/(gamma - 1) as unevaluated pairs hi + lo (float kernels):
    // B1, B2 and dB = B1 - B2
    T B1h, B1l, B2h, B2l, dBh, dBl;
    // A = 1/(gamma-1) the same way: A1, A2 and dA = A1 - A2
    T A1h, A1l, A2h, A2l, dAh, dAl;
    T mu, lam_heat, R, inv_R;
    T eps_rho, eps_rhoc2, eps_alpha, one_m_eps_alpha, weno_eps, weno_eps4;
};

// Everything a kernel needs, passed by value.
struct Dev {
    int n[3];
    int bc[3][2];
    long long ncell;
    // distance between consecutive variables (and components) of the cell
    // arrays: ncell, or for a block of a decomposed grid the cells of its
    // halo-padded slab (the arrays then start at the first owned cell and
    // the halo planes lie before and after it)
    long long vstride;
    int skip_face0_count;  // limiter counters skip the faces at c = 0 of the last axis
    long long cell_lo, cell_hi;  // valid cell-array indices [cell_lo, cell_hi) (debug checks)
    FastDiv fd_cell[2];     // n[0], n[1]: cell index -> (x, y, z)
    FastDiv fd_face[3][2];  // per axis d: the face-array extents along x and y
    double inv_dx[3];
    double vol;
    // EOS: per fluid A = 1/(gamma-1), B = gamma pinf/(gamma-1); single-phase
    // shortcuts gm1 = gamma-1, gamma, pinf, gpinf = gamma pinf
    double A1, A2, B1, B2;
    double gamma0, pinf0, gm1_0, gpinf0;
    int stiff;  // p_inf != 0 somewhere: mixed precision recovers p in double
    double mu, lam_heat, R;
    double vis_dn[3], vis_cd[3];  // viscous stencil scales (face-normal, cell-centred derivative)
    // scheme
    int recon;   // JXF_WENO5JS_COMP (component) or JXF_WENO5JS_CHAR (characteristic)
    int weno_z;  // 0: Jiang-Shu weights, 1: WENO5-Z weights
    int teno;    // 1: TENO6-A instead of WENO5
    int viscous, limiter;
    int visc_half;  // viscous stencils: points per side (1, 2, 3 for order 2, 4, 6)
    int thinc;   // THINC volume-fraction reconstruction (five-equation model)
    double eps_rho, eps_rhoc2, eps_alpha, weno_eps;
    double cfl, fixed_dt, t_end, visc_dt_coef;
    double dx_min;     // smallest cell size (viscous time-step bound)
    double fl_lam[3];  // 2 D / dx_d: flux-limiter pseudo-time factor per dt
    // buffers (storage type unless noted)
    const void *W;      // primitives read by the flux sweeps
    const void *Ucell;  // conservative cell states read by the flux limiter
    const void *Tt;     // temperature read by the viscous flux
    void *F[3];         // face fluxes per axis, [v][face]
    void *UH[3];        // upwinded face velocity per axis (diffuse interface)
    const void *Un;     // U^n
    const void *Us;     // U^(s) (stage input)
    void *Uout;         // stage output (may alias Us or Un)
    void *Wout;         // primitives of the stage output
    void *Tout;         // temperature of the stage output
    void *G;            // per-cell auxiliary arrays: viscous, the cell-centred velocity
                        // gradient du_f/dx_e [f*ndim+e][cell]; THINC, |n_d| [d][cell]
                        // and psi [ndim][cell]
    void *dU;           // right-hand side output (rhs mode)
    double ca, cb, cc;  // Uout = ca Un + cb Us + cc dt R
    float ca32, cb32;   // the same in float
    int stage0;         // first stage: Uout = Us + cc dt R (no Un term)
    const double *dtp;  // dt read by the kernels
    int skip_if_done;   // return at once when *dtp == 0 (steps past t_end)
    double *scal;       // scalar slots
    double *part;       // per-block partials: [blk][2 + nv]
    int *status;
    unsigned long long *counters;  // [0] IL sides, [1] FL faces
    const void *Rbar;   // adjoint of the right-hand side (vjp)
    void *Sbar;         // stencil-slot adjoints of one axis's faces (vjp)
    void *Wbar;         // adjoint of the primitives (vjp, accumulated)
    void *Ubar;         // adjoint of the conservative state (vjp output)
    Cst<double> k64;
    Cst<float> k32;
};

template <typename T> __device__ __forceinline__ const Cst<T> &cst(const Dev &P);
template <> __device__ __forceinline__ const Cst<double> &cst<double>(const Dev &P) { return P.k64; }
template <> __device__ __forceinline__ const Cst<float> &cst<float>(const Dev &P) { return P.k32; }

// Copy the double-precision constants of P into both typed sets.
inline void fill_constants(Dev &P) {
    auto fill = [&](auto &k) {
        using T = typename std::remove_reference<decltype(k.A1)>::type;
        for (int e = 0; e < 3; ++e) {
            k.inv_dx[e] = T(P.inv_dx[e]);
            k.vis_dn[e] = T(P.vis_dn[e]);
            k.vis_cd[e] = T(P.vis_cd[e]);
            k.fl_lam[e] = T(P.fl_lam[e]);
        }
        k.A1 = T(P.A1); k.A2 = T(P.A2); k.B1 = T(P.B1); k.B2 = T(P.B2);
        k.B1h = T(P.B1); k.B1l = T(P.B1 - double(k.B1h));
        k.B2h = T(P.B2); k.B2l = T(P.B2 - double(k.B2h));
        k.dBh = T(P.B1 - P.B2); k.dBl = T((P.B1 - P.B2) - double(k.dBh));
        k.A1h = T(P.A1); k.A1l = T(P.A1 - double(k.A1h));
        k.A2h = T(P.A2); k.A2l = T(P.A2 - double(k.A2h));
        k.dAh = T(P.A1 - P.A2); k.dAl = T((P.A1 - P.A2) - double(k.dAh));
        k.gamma0 = T(P.gamma0); k.pinf0 = T(P.pinf0); k.gm1_0 = T(P.gm1_0); k.gpinf0 = T(P.gpinf0);
        k.mu = T(P.mu); k.lam_heat = T(P.lam_heat); k.R = T(P.R);
        k.inv_R = T(P.R > 0.0 ? 1.0 / P.R : 0.0);
        k.eps_rho = T(P.eps_rho); k.eps_rhoc2 = T(P.eps_rhoc2); k.eps_alpha = T(P.eps_alpha);
        k.one_m_eps_alpha = T(1.0 - P.eps_alpha);
        k.weno_eps = T(P.weno_eps);
        k.weno_eps4 = T(4.0 * P.weno_eps);
    };
    fill(P.k64);
    fill(P.k32);
}

template <int MODEL, int NDIM> struct Vars {
    static constexpr int NP = (MODEL == JXF_DIM) ? 2 : 1;
    static constexpr int IE = NP + NDIM;
    static constexpr int IA = (MODEL == JXF_DIM) ? IE + 1 : -1;
    static constexpr int NV = IE + 1 + ((MODEL == JXF_DIM) ? 1 : 0);
};

// ------------------------------------------------------------ helpers -----
template <typename T> __device__ __forceinline__ T dsqrt(T x);
template <> __device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }
// float: the special-function unit's approximation (PTX sqrt.approx.ftz.f32,
// about 1 ulp; float operands on this path are normal numbers)
template <> __device__ __forceinline__ float dsqrt<float>(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// Addition that is never fused with a neighbouring multiplication: results
// that must not depend on the kernel they are compiled into (the batched and
// single-grid kernels agree bitwise).
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
template <typename T> __device__ __forceinline__ T rsq(T x);  // 1/sqrt(x)
template <> __device__ __forceinline__ double rsq<double>(double x) { return rsqrt(x); }
template <> __device__ __forceinline__ float rsq<float>(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// Division.  Double: Newton-Raphson refinement of the hardware reciprocal
// estimate (PTX rcp.approx.ftz.f64): one step r <- r + r (1 - b r) squares
// the estimate's relative error, then q = a r is corrected once with the
// exact residual a - b q (both by fused multiply-add), which leaves q within
// about one ulp of a/b for normal operands -- 5 double instructions instead
// of the IEEE division sequence (checked against IEEE division by
// jxf_selftest_div).  Float: one special-function-unit reciprocal (PTX
// rcp.approx.ftz.f32, about 1 ulp) and a multiplication; all operands here
// are normal numbers far below 2^126 in magnitude.
__device__ __forceinline__ double fdiv(double a, double b) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(b));
    r = fma(r, fma(-b, r, 1.0), r);
    const double q = a * r;
    return fma(fma(-b, q, a), r, q);
}
__device__ __forceinline__ double rcp(double x) { return fdiv(1.0, x); }
__device__ __forceinline__ float rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float fdiv(float a, float b) { return a * rcp(b); }
template <typename T> __device__ __forceinline__ T tmin(T a, T b) { return b < a ? b : a; }
template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return b > a ? b : a; }

// Boundary conditions by index mapping (§3.1): periodic wrap, zero-gradient
// copy of the boundary cell, symmetry mirror (the velocity component of the
// mirrored axis changes sign: bit e of *mir flips).  A side shared with the
// neighbouring block of a decomposed grid (§4.3) maps to itself: its halo
// cells are stored next to the owned ones and filled by the exchange.
__device__ __forceinline__ int map_axis(int c, int n, int blo, int bhi, int &mir, int bit) {
    if (c < 0) {
        if (blo == JXF_BC_PERIODIC) return c + n;
        if (blo == JXF_BC_ZEROGRAD) return 0;
        if (blo == JXF_BC_NEIGHBOR) return c;
        mir ^= bit;
        return -1 - c;
    }
    if (c >= n) {
        if (bhi == JXF_BC_PERIODIC) return c - n;
        if (bhi == JXF_BC_ZEROGRAD) return n - 1;
        if (bhi == JXF_BC_NEIGHBOR) return c;
        mir ^= bit;
        return 2 * n - 1 - c;
    }
    return c;
}

// The stage's dt (device scalar, double) read once per block and shared:
// the float kernels then do no double arithmetic per thread.  Returns false
// when the step is to be skipped (past t_end).  All threads must call.
__device__ __forceinline__ bool block_dt(const Dev &P, double &dt) {
    __shared__ double s_dt;
    __shared__ int s_go;  // decided once per block: no double compare per thread
    __syncthreads();
    if (threadIdx.x == 0) {
        s_dt = *P.dtp;
        s_go = !(P.skip_if_done && !(s_dt > 0.0));
    }
    __syncthreads();
    dt = s_dt;
    return s_go != 0;
}

// Debug builds (-DJXF_DEBUG) check every computed cell and face index of the
// stencil and face loads against the arrays' extents, record a violation in
// the status word (ST_BOUNDS, reported by the next synchronising call) and
// clamp the index to the first entry so that no access leaves its array;
// release builds compile the checks away.
__device__ __forceinline__ int chk_cell(const Dev &P, long long idx) {
#ifdef JXF_DEBUG
    if (idx < P.cell_lo || idx >= P.cell_hi) {
        if (P.status) atomicOr(P.status, (int)ST_BOUNDS);
        return 0;
    }
#endif
    return (int)idx;
}
__device__ __forceinline__ int chk_face(const Dev &P, long long idx, long long nface) {
#ifdef JXF_DEBUG
    if (idx < 0 || idx >= nface) {
        if (P.status) atomicOr(P.status, (int)ST_BOUNDS);
        return 0;
    }
#else
    (void)P;
    (void)nface;
#endif
    return (int)idx;
}

// ---------------------------------------------------------------- EOS -----
// Stiffened-gas mixture (§2.4) in the form A = 1/(gamma-1),
// B = gamma p_inf/(gamma-1):  rho e = A p + B,  p = (rho e - B)/A,
// rho c^2 = gamma (p + p_inf) = p + (p + B)/A.
template <typename T, int MODEL> struct Eos {
    T A, B, invA;
    __device__ __forceinline__ Eos(const Dev &P, T a1) {
        const Cst<T> &C = cst<T>(P);
        if (MODEL == JXF_SPM) {
            A = C.A1;
            B = C.B1;
            invA = C.gm1_0;
        } else {
            const T a2 = T(1) - a1;
            A = a1 * C.A1 + a2 * C.A2;
            B = a1 * C.B1 + a2 * C.B2;
            invA = fdiv(T(1), A);
        }
    }
    __device__ __forceinline__ T rhoe_from_p(const Dev &P, T p) const {
        if (MODEL == JXF_SPM) return (p + cst<T>(P).gpinf0) * A;
        return A * p + B;
    }
    __device__ __forceinline__ T p_from_rhoe(const Dev &P, T rhoe) const {
        if (MODEL == JXF_SPM) return cst<T>(P).gm1_0 * rhoe - cst<T>(P).gpinf0;
        return (rhoe - B) * invA;
    }
    __device__ __forceinline__ T rc2_from_p(const Dev &P, T p) const {
        if (MODEL == JXF_SPM) return cst<T>(P).gamma0 * (p + cst<T>(P).pinf0);
        return p + (p + B) * invA;
    }
};

template <typename T, int MODEL, int NDIM>
__device__ __forceinline__ T density_of(const T *X) {
    if (MODEL == JXF_DIM) return X[0] + X[1];
    return X[0];
}
template <typename T, int MODEL, int NDIM>
__device__ __forceinline__ T alpha_of(const T *X) {
    if (MODEL == JXF_DIM) return X[Vars<MODEL, NDIM>::IA];
    return T(0);
}

// W -> U of one state; returns rho c^2 on the side.
template <typename T, int MODEL, int NDIM>
__device__ __forceinline__ void prim2cons(const Dev &P, const T *W, T *U, T &rc2) {
    using V = Vars<MODEL, NDIM>;
    const T rho = density_of<T, MODEL, NDIM>(W);
    Eos<T, MODEL> eos(P, alpha_of<T, MODEL, NDIM>(W));
#pragma unroll
    for (int k = 0; k < V::NP; ++k) U[k] = W[k];
    T uu = W[V::NP] * W[V::NP];
#pragma unroll
    for (int d = 1; d < NDIM; ++d) uu += W[V::NP + d] * W[V::NP + d];
#pragma unroll
    for (int d = 0; d < NDIM; ++d) U[V::NP + d] = rho * W[V::NP + d];
    const T rhoe = eos.rhoe_from_p(P, W[V::IE]);
    U[V::IE] = rhoe + T(0.5) * rho * uu;
    if (MODEL == JXF_DIM) U[V::IA] = W[V::IA];
    rc2 = eos.rc2_from_p(P, W[V::IE]);
}

// U -> W in precision C (C = double recovers the stiffened-gas pressure
// without the float cancellation of rho e - B).
template <typename C, typename T, int MODEL, int NDIM>
__device__ __forceinline__ void cons2prim(const Dev &P, const T *U, T *W, C &rho_o, C &p_o,
                                          C &rc2_o) {
    using V = Vars<MODEL, NDIM>;
    const C rho = (MODEL == JXF_DIM) ? C(U[0]) + C(U[1]) : C(U[0]);
    const C ir = rcp(rho);
    C uu = 0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        const C u = C(U[V::NP + d]) * ir;
        W[V::NP + d] = T(u);
        uu += C(U[V::NP + d]) * u;
    }
#pragma unroll
    for (int k = 0; k < V::NP; ++k) W[k] = U[k];
    Eos<C, MODEL> eos(P, (MODEL == JXF_DIM) ? C(U[V::IA]) : C(0));
    const C rhoe = C(U[V::IE]) - C(0.5) * uu;
    const C p = eos.p_from_rhoe(P, rhoe);
    W[V::IE] = T(p);
    if (MODEL == JXF_DIM) W[V::IA] = U[V::IA];
    rho_o = rho;
    p_o = p;
    rc2_o = eos.rc2_from_p(P, p);
}

// ------------------------------------------------------------ WENO5 -------
// Face values at x_{i+1/2} from the left and from the right, from the six
// cell averages x0..x5 = v_{i-2..i+3} (§3.2 step 3; Jiang-Shu candidates on
// the three 3-cell sub-stencils, smoothness indicators beta_k, linear
// weights d = (0.1, 0.6, 0.3)).  Everything is written in the undivided
// differences D_k = x_{k+1} - x_k and second differences A_k = D_{k+1} - D_k,
// scaled to avoid constant factors:
//   Q_k = 4 (beta_k + eps) = H_k^2 + 13/3 A^2 + 4 eps   (H_k = twice the
//         sub-stencil's one-sided combination),
//   E_k = 6 (p_k - centre)                               (candidate offsets),
//   value = centre + sum a_k E_k / (6 sum a_k),
// left value around x2 (H = 3D1 - D0, D1 + D2, D3 - 3D2; E = 5D1 - 2D0,
// D1 + 2D2, 4D2 - D3), right value the mirrored formula around x3 (two of
// its three second differences are the left value's).  A common factor of
// all Q_k leaves the normalised weights unchanged.  Weights: Jiang-Shu
// a_k = d_k/Q_k^2, or WENO5-Z (Borges et al. 2008) a_k = d_k (1 + tau/Q_k),
// tau = |Q_0 - Q_2| = 4 |beta_0 - beta_2|.  In double the three weight
// divisions fold into one (a_k scaled by prod_j Q_j^2 resp. prod_j Q_j); in
// float each weight keeps its own reciprocal so that large beta cannot
// overflow.
template <bool Z, typename T>
__device__ __forceinline__ T weno5_combine(T Q0, T Q1, T Q2, T E0, T E1, T E2, T centre) {
    T p0, p1, p2;  // weights without d_k
    if (sizeof(T) == 8) {
        if (Z) {
            const T tau = fabs(Q0 - Q2);
            p0 = (Q0 + tau) * (Q1 * Q2);
            p1 = (Q1 + tau) * (Q0 * Q2);
            p2 = (Q2 + tau) * (Q0 * Q1);
        } else {
            const T z0 = Q0 * Q0, z1 = Q1 * Q1, z2 = Q2 * Q2;
            p0 = z1 * z2;
            p1 = z0 * z2;
            p2 = z0 * z1;
        }
    } else {
        const T r0 = rcp(Q0), r1 = rcp(Q1), r2 = rcp(Q2);
        if (Z) {
            const T tau = fabs(Q0 - Q2);
            p0 = T(1) + tau * r0;
            p1 = T(1) + tau * r1;
            p2 = T(1) + tau * r2;
        } else {
            p0 = r0 * r0;
            p1 = r1 * r1;
            p2 = r2 * r2;
        }
    }
    const T num = T(0.1) * (p0 * E0) + T(0.6) * (p1 * E1) + T(0.3) * (p2 * E2);
    const T den = T(0.6) * p0 + T(3.6) * p1 + T(1.8) * p2;  // 6 sum d_k p_k
    return centre + fdiv(num, den);
}

// eps4 = 4 eps.
template <bool Z, typename T>
__device__ __forceinline__ void weno5_pair(const T (&x)[6], T eps4, T &vl, T &vr) {
    const T D0 = x[1] - x[0], D1 = x[2] - x[1], D2 = x[3] - x[2];
    const T D3 = x[4] - x[3], D4 = x[5] - x[4];
    const T A0 = D1 - D0, A1 = D2 - D1, A2 = D3 - D2, A3 = D4 - D3;
    const T k = T(13.0 / 3.0);
    const T C0 = (k * A0) * A0 + eps4, C1 = (k * A1) * A1 + eps4;
    const T C2 = (k * A2) * A2 + eps4, C3 = (k * A3) * A3 + eps4;
    {  // left value (centre x2): sub-stencils {i-2,i-1,i}, {i-1,i,i+1}, {i,i+1,i+2}
        const T H0 = T(3) * D1 - D0, H1 = D1 + D2, H2 = D3 - T(3) * D2;
        const T Q0 = H0 * H0 + C0, Q1 = H1 * H1 + C1, Q2 = H2 * H2 + C2;
        const T E0 = T(3) * D1 + (A0 + A0), E1 = T(2) * D2 + D1, E2 = T(4) * D2 - D3;
        vl = weno5_combine<Z>(Q0, Q1, Q2, E0, E1, E2, x[2]);
    }
    {  // right value (centre x3): mirrored sub-stencils {i+3,i+2,i+1},
       // {i+2,i+1,i}, {i+1,i,i-1}
        const T H0 = D4 - T(3) * D3, H1 = D2 + D3, H2 = T(3) * D2 - D1;
        const T Q0 = H0 * H0 + C3, Q1 = H1 * H1 + C2, Q2 = H2 * H2 + C1;
        const T E0 = T(-3) * D3 + (A3 + A3), E1 = T(-2) * D2 - D3, E2 = T(-4) * D2 + D1;
        vr = weno5_combine<Z>(Q0, Q1, Q2, E0, E1, E2, x[3]);
    }
}

// ------------------------------------------------- packed float WENO5 ----
// Two float lanes in one 64-bit register pair.  GB300's packed FP32
// instructions (add / sub / mul / fma on .f32x2) issue once for both lanes
// at the scalar per-lane rate, and the float face sweep is bound by
// instruction issue.  The right-biased value is the left-biased formula on
// the mirrored stencil, so lane a carries the left value's stencil x0..x4
// and lane b the mirrored x5..x1: one packed evaluation gives both values
// of a face (the reciprocals stay scalar, one per lane).
struct f2 {
    float2 v;
};
__device__ __forceinline__ f2 mk2(float a, float b) { return {make_float2(a, b)}; }
__device__ __forceinline__ f2 bc2(float a) { return {make_float2(a, a)}; }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return {__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 r;
    asm("{\n\t.reg .b64 ta, tb, td;\n\t"
        "mov.b64 ta, {%2, %3};\n\tmov.b64 tb, {%4, %5};\n\t"
        "sub.rn.f32x2 td, ta, tb;\n\tmov.b64 {%0, %1}, td;\n\t}"
        : "=f"(r.v.x), "=f"(r.v.y)
        : "f"(a.v.x), "f"(a.v.y), "f"(b.v.x), "f"(b.v.y));
    return r;
}
__device__ __forceinline__ f2 rcp2(f2 a) { return mk2(rcp(a.v.x), rcp(a.v.y)); }
__device__ __forceinline__ f2 abs2(f2 a) { return mk2(fabsf(a.v.x), fabsf(a.v.y)); }

// weno5_pair in float with the two sides in the lanes: P_k = (x_k, x_{5-k}),
// k = 0..4; the left formula of weno5_pair (centre P_2) on both lanes.
// One-sided combinations through the second differences where that saves
// an instruction (3 D1 - D0 = 2 D1 + A0, D3 - 3 D2 = A2 - 2 D2).
template <bool Z>
__device__ __forceinline__ void weno5_pair_f2(const float (&x)[6], float eps4, float &vl, float &vr) {
    const f2 P0 = mk2(x[0], x[5]), P1 = mk2(x[1], x[4]), P2 = mk2(x[2], x[3]);
    const f2 P3 = mk2(x[3], x[2]), P4 = mk2(x[4], x[1]);
    const f2 D0 = sub2(P1, P0), D1 = sub2(P2, P1), D2 = sub2(P3, P2), D3 = sub2(P4, P3);
    const f2 nD3 = sub2(P3, P4);
    const f2 A0 = sub2(D1, D0), A1 = sub2(D2, D1), A2 = sub2(D3, D2);
    const f2 k = bc2((float)(13.0 / 3.0)), e4 = bc2(eps4);
    const f2 H0 = fma2(bc2(2.f), D1, A0), H1 = add2(D1, D2), H2 = fma2(bc2(-2.f), D2, A2);
    const f2 Q0 = fma2(H0, H0, fma2(mul2(k, A0), A0, e4));
    const f2 Q1 = fma2(H1, H1, fma2(mul2(k, A1), A1, e4));
    const f2 Q2 = fma2(H2, H2, fma2(mul2(k, A2), A2, e4));
    const f2 E0 = fma2(bc2(3.f), D1, add2(A0, A0)), E1 = fma2(bc2(2.f), D2, D1);
    const f2 E2 = fma2(bc2(4.f), D2, nD3);
    const f2 r0 = rcp2(Q0), r1 = rcp2(Q1), r2 = rcp2(Q2);
    f2 p0, p1, p2;  // weights without d_k
    if (Z) {
        const f2 tau = abs2(sub2(Q0, Q2)), one = bc2(1.f);
        p0 = fma2(tau, r0, one);
        p1 = fma2(tau, r1, one);
        p2 = fma2(tau, r2, one);
    } else {
        p0 = mul2(r0, r0);
        p1 = mul2(r1, r1);
        p2 = mul2(r2, r2);
    }
    // d_k = (1, 6, 3) / 10; the common 1/10 cancels
    const f2 three = bc2(3.f), six = bc2(6.f);
    const f2 num = fma2(six, mul2(p1, E1), fma2(three, mul2(p2, E2), mul2(p0, E0)));
    const f2 den = fma2(six, p1, fma2(three, p2, p0));
    const f2 v = fma2(num, rcp2(mul2(six, den)), P2);
    vl = v.v.x;
    vr = v.v.y;
}

// One reconstruction of a face: packed in float, scalar in double.
template <bool Z, typename T>
__device__ __forceinline__ void weno5_face(const T (&x)[6], T eps4, T &vl, T &vr) {
    if constexpr (std::is_same<T, float>::value) weno5_pair_f2<Z>(x, eps4, vl, vr);
    else weno5_pair<Z>(x, eps4, vl, vr);
}

// ------------------------------------------------------------ TENO6-A -----
// Value at x_{i+1/2} from the left from v[0..5] = v_{i-2..i+3}: the TENO6-A
// scheme of the paper's single-phase runs (§3.2 step 3; Fu, Hu & Adams).
// Candidates q_k on S0 = {i-1,i,i+1}, S1 = {i,i+1,i+2}, S2 = {i-2,i-1,i},
// S3 = {i,..,i+3}; Jiang-Shu smoothness indicators beta_k and beta_6 of all
// six cells; tau6 = |beta_6 - (beta_0 + beta_2 + 4 beta_1)/6|; stencil k is
// kept iff gamma_k = (1 + tau6/(beta_k + 1e-30))^6 is at least C_T sum_j
// gamma_j, with the adaptive C_T = 10^-floor(10.5 - 3.5 (1 - g(m))),
// g(m) = (1-m)^4 (1+4m), m = 1 - min(1, eta/0.23) from the smoothest-pair
// measure eta of the cells i-1..i+2; the value is the kept candidates'
// combination with the renormalised linear weights d = (9, 6, 1, 4)/20.
// beta_6 is evaluated as a sum of squares of the degree-5 polynomial's
// derivative coefficients a_1..a_5 at the cell centre (an LDL^T form of the
// same quadratic form, free of the large cancelling coefficients of its
// expansion in the cell values).  The selection tests gamma_k < C_T sum_j
// gamma_j (in float with gamma_k / max_j gamma_j, tau/(beta_k + eps) capped
// at 1e30 so that neither overflows); C_T comes from comparing eta with three
// thresholds (in double by cross-multiplication, so eta is never divided
// out); in double the four gamma arguments share one division and the
// renormalisation takes one when a stencil is dropped.

// The adaptive cut-off C_T = 10^-floor(10.5 - 3.5 (1 - g(m))), g(m) =
// (1-m)^4 (1+4m), m = 1 - min(1, eta/C_r), C_r = 0.23, takes the four values
// 1e-7 .. 1e-10: floor(7 + 3.5 g) >= 7 + k exactly when g >= 2k/7, and g
// grows with the smoothness measure eta, so C_T follows from comparing eta
// with the three values eta_k = C_r (1 - m_k), g(m_k) = 2k/7 (bisection at
// compile time) -- no division for eta, no polynomial, no floor.
constexpr double teno_g(double m) { return (1.0 - m) * (1.0 - m) * (1.0 - m) * (1.0 - m) * (1.0 + 4.0 * m); }
constexpr double teno_eta_threshold(int k) {
    double lo = 0.0, hi = 1.0;  // g decreases on [0, 1]: the largest m with g(m) >= 2k/7
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (teno_g(mid) >= 2.0 * k / 7.0) lo = mid;
        else hi = mid;
    }
    return 0.23 * (1.0 - lo);
}
constexpr double kTenoEta1 = teno_eta_threshold(1), kTenoEta2 = teno_eta_threshold(2),
                 kTenoEta3 = teno_eta_threshold(3);
// C_T from the number k of thresholds eta reaches.
template <typename T> __device__ __forceinline__ T teno_cutoff(int k) {
    return k >= 3 ? T(1e-10) : (k == 2 ? T(1e-9) : (k == 1 ? T(1e-8) : T(1e-7)));
}

// The sharp selection of TENO6-A from the candidate values q, their
// smoothness indicators b, tau6 and the cut-off ct.
template <typename T>
__device__ __forceinline__ T teno6a_select(const T (&q)[4], const T (&b)[4], T tau, T ct) {
    // scale separation and sharp selection
    T gk[4], gs = T(0);
    if constexpr (sizeof(T) == 8) {  // the four reciprocals from one division
        const T e0 = b[0] + T(1e-30), e1 = b[1] + T(1e-30), e2 = b[2] + T(1e-30), e3 = b[3] + T(1e-30);
        const T p01 = e0 * e1, p23 = e2 * e3;
        const T r = rcp(p01 * p23);
        const T r01 = r * p23, r23 = r * p01;
        gk[0] = T(1) + tau * (r01 * e1);
        gk[1] = T(1) + tau * (r01 * e0);
        gk[2] = T(1) + tau * (r23 * e3);
        gk[3] = T(1) + tau * (r23 * e2);
    } else {
        // tau/(beta_k + 1e-30) of a flat sub-stencil (beta_k = 0) next to a
        // jump of dimensional data (tau ~ 1e10 for a 1e5 Pa step) exceeds the
        // float range: capped at 1e30, so that gamma_k / max gamma stays a
        // number (inf/inf would make every comparison below false and keep
        // all four stencils across the jump).  The cap changes a decision
        // only between two stencils that are both flat to below 1e-30 tau.
#pragma unroll
        for (int k = 0; k < 4; ++k) gk[k] = T(1) + tmin(tau * rcp(b[k] + T(1e-30)), T(1e30));
    }
    if constexpr (sizeof(T) == 8) {  // chi_k < C_T as gamma_k < C_T sum_j gamma_j
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const T a2 = gk[k] * gk[k];
            gk[k] = a2 * a2 * a2;
            gs += gk[k];
        }
    } else {  // relative to the largest: every ratio <= 1
        const T amax = tmax(tmax(gk[0], gk[1]), tmax(gk[2], gk[3]));
        const T ia = rcp(amax);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const T r = gk[k] * ia, r2 = r * r;
            gk[k] = r2 * r2 * r2;
            gs += gk[k];
        }
    }
    const T d[4] = {T(9.0 / 20.0), T(3.0 / 10.0), T(1.0 / 20.0), T(1.0 / 5.0)};
    const T cut = ct * gs;
    T num = T(0), den = T(0);
    int kept = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (!(gk[k] < cut)) {
            num += d[k] * q[k];
            den += d[k];
            ++kept;
        }
    }
    return kept == 4 ? num : fdiv(num, den);  // all four kept: the weights sum to 1
}

// e of the smoothness measure: 0.9 C_r xi^2 / (1 - 0.9 C_r), C_r = 0.23, xi = 1e-3
constexpr double kTenoE = 0.9 * 0.23 * 1e-6 / (1.0 - 0.9 * 0.23);

// The cut-off class of TENO6-A's smoothness measure eta of the stencil
// v[0..5] (how many of the three thresholds eta reaches): the smallest of
// the four ratios (|2 D+ D-| + e)/(D+^2 + D-^2 + e) at the cells v[1..4].
// The ratios are symmetric in the two differences, so the mirrored stencil
// of the face's other value has the same four ratios and the same class:
// computed once per face.  In double by cross-multiplication (the
// denominators are positive), so eta is never divided out; in float each
// ratio from its own fast reciprocal (the cross products of squared
// differences would overflow float for jumps above about 4e9).
template <typename T> __device__ __forceinline__ int teno6a_eta_class(const T (&v)[6]) {
    const T e = T(kTenoE);
    if constexpr (sizeof(T) == 8) {
        T en = T(1), ed = T(1);
#pragma unroll
        for (int j = 1; j <= 4; ++j) {
            const T dp = v[j + 1] - v[j], dm = v[j] - v[j - 1];
            const T n = fabs(T(2) * dp * dm) + e, dd = dp * dp + dm * dm + e;
            if (n * ed < en * dd) {
                en = n;
                ed = dd;
            }
        }
        return (en >= T(kTenoEta1) * ed) + (en >= T(kTenoEta2) * ed) + (en >= T(kTenoEta3) * ed);
    } else {
        T eta = T(1);
#pragma unroll
        for (int j = 1; j <= 4; ++j) {
            const T dp = v[j + 1] - v[j], dm = v[j] - v[j - 1];
            eta = tmin(eta, (fabs(T(2) * dp * dm) + e) * rcp(dp * dp + dm * dm + e));
        }
        return (eta >= T(kTenoEta1)) + (eta >= T(kTenoEta2)) + (eta >= T(kTenoEta3));
    }
}

template <typename T> __device__ __forceinline__ T teno6a_left(const T (&v)[6], int k) {
    const T vm2 = v[0], vm1 = v[1], v0 = v[2], vp1 = v[3], vp2 = v[4], vp3 = v[5];
    T q[4], b[4];
    q[0] = (-vm1 + T(5) * v0 + T(2) * vp1) * T(1.0 / 6.0);
    q[1] = (T(2) * v0 + T(5) * vp1 - vp2) * T(1.0 / 6.0);
    q[2] = (T(2) * vm2 - T(7) * vm1 + T(11) * v0) * T(1.0 / 6.0);
    q[3] = (T(3) * v0 + T(13) * vp1 - T(5) * vp2 + vp3) * T(1.0 / 12.0);
    {
        T a = vm1 - T(2) * v0 + vp1, c = vm1 - vp1;
        b[0] = T(13.0 / 12.0) * a * a + T(0.25) * c * c;
        a = v0 - T(2) * vp1 + vp2, c = T(3) * v0 - T(4) * vp1 + vp2;
        b[1] = T(13.0 / 12.0) * a * a + T(0.25) * c * c;
        a = vm2 - T(2) * vm1 + v0, c = vm2 - T(4) * vm1 + T(3) * v0;
        b[2] = T(13.0 / 12.0) * a * a + T(0.25) * c * c;
        const T e1 = T(-11) * v0 + T(18) * vp1 - T(9) * vp2 + T(2) * vp3;
        const T e2 = T(2) * v0 - T(5) * vp1 + T(4) * vp2 - vp3;
        const T e3 = -v0 + T(3) * vp1 - T(3) * vp2 + vp3;
        b[3] = T(1.0 / 36.0) * e1 * e1 + T(13.0 / 12.0) * e2 * e2 + T(781.0 / 720.0) * e3 * e3;
    }
    T b6;
    {
        const T a1 = (T(341) * vm2 - T(2785) * vm1 - T(2590) * v0 + T(6670) * vp1 - T(1895) * vp2 +
                      T(259) * vp3) * T(1.0 / 5760.0);
        const T a2 = (-vm2 + T(12) * vm1 - T(22) * v0 + T(12) * vp1 - vp2) * T(1.0 / 16.0);
        const T a3 = (T(-5) * vm2 - T(11) * vm1 + T(70) * v0 - T(94) * vp1 + T(47) * vp2 - T(7) * vp3) *
                     T(1.0 / 144.0);
        const T a4 = (vm2 - T(4) * vm1 + T(6) * v0 - T(4) * vp1 + vp2) * T(1.0 / 24.0);
        const T a5 = (-vm2 + T(5) * vm1 - T(10) * v0 + T(10) * vp1 - T(5) * vp2 + vp3) * T(1.0 / 120.0);
        const T s1 = a1 + T(0.25) * a3 + T(0.0625) * a5;
        const T s2 = a2 + T(63.0 / 130.0) * a4;
        const T s3 = a3 + T(8825.0 / 10934.0) * a5;
        b6 = s1 * s1 + T(13.0 / 3.0) * s2 * s2 + T(781.0 / 20.0) * s3 * s3 +
             T(1421461.0 / 2275.0) * a4 * a4 + T(21520059541.0 / 1377684.0) * a5 * a5;
    }
    const T tau = fabs(b6 - (b[0] + b[2] + T(4) * b[1]) * T(1.0 / 6.0));
    return teno6a_select(q, b, tau, teno_cutoff<T>(k));
}

// teno6a_left for both values of a face in float: lane a carries the stencil
// x0..x5, lane b the mirrored x5..x0, so candidates, indicators, tau6 and the
// smoothness measure are evaluated with packed instructions; the cut-off and
// the selection then run per lane.
__device__ __forceinline__ void teno6a_pair_f2(const float (&x)[6], float &vl, float &vr) {
    const f2 vm2 = mk2(x[0], x[5]), vm1 = mk2(x[1], x[4]), v0 = mk2(x[2], x[3]);
    const f2 vp1 = mk2(x[3], x[2]), vp2 = mk2(x[4], x[1]), vp3 = mk2(x[5], x[0]);
    f2 q[4], b[4];
    q[0] = mul2(sub2(fma2(bc2(5.f), v0, add2(vp1, vp1)), vm1), bc2((float)(1.0 / 6.0)));
    q[1] = mul2(sub2(fma2(bc2(5.f), vp1, add2(v0, v0)), vp2), bc2((float)(1.0 / 6.0)));
    q[2] = mul2(fma2(bc2(11.f), v0, fma2(bc2(-7.f), vm1, add2(vm2, vm2))), bc2((float)(1.0 / 6.0)));
    q[3] = mul2(add2(fma2(bc2(13.f), vp1, fma2(bc2(3.f), v0, vp3)), mul2(bc2(-5.f), vp2)),
                bc2((float)(1.0 / 12.0)));
    const f2 k13 = bc2((float)(13.0 / 12.0)), k4 = bc2(0.25f);
    {
        f2 a = fma2(bc2(-2.f), v0, add2(vm1, vp1)), c = sub2(vm1, vp1);
        b[0] = fma2(mul2(k13, a), a, mul2(mul2(k4, c), c));
        a = fma2(bc2(-2.f), vp1, add2(v0, vp2)), c = fma2(bc2(3.f), v0, fma2(bc2(-4.f), vp1, vp2));
        b[1] = fma2(mul2(k13, a), a, mul2(mul2(k4, c), c));
        a = fma2(bc2(-2.f), vm1, add2(vm2, v0)), c = fma2(bc2(3.f), v0, fma2(bc2(-4.f), vm1, vm2));
        b[2] = fma2(mul2(k13, a), a, mul2(mul2(k4, c), c));
        const f2 e1 = fma2(bc2(-11.f), v0, fma2(bc2(18.f), vp1, fma2(bc2(-9.f), vp2, add2(vp3, vp3))));
        const f2 e2 = sub2(fma2(bc2(2.f), v0, fma2(bc2(-5.f), vp1, mul2(bc2(4.f), vp2))), vp3);
        const f2 e3 = add2(sub2(fma2(bc2(3.f), vp1, mul2(bc2(-3.f), vp2)), v0), vp3);
        b[3] = fma2(mul2(bc2((float)(1.0 / 36.0)), e1), e1,
                    fma2(mul2(k13, e2), e2, mul2(mul2(bc2((float)(781.0 / 720.0)), e3), e3)));
    }
    f2 b6;
    {
        const f2 a1 = mul2(fma2(bc2(341.f), vm2, fma2(bc2(-2785.f), vm1, fma2(bc2(-2590.f), v0,
                          fma2(bc2(6670.f), vp1, fma2(bc2(-1895.f), vp2, mul2(bc2(259.f), vp3)))))),
                           bc2((float)(1.0 / 5760.0)));
        const f2 a2 = mul2(sub2(fma2(bc2(12.f), add2(vm1, vp1), mul2(bc2(-22.f), v0)), add2(vm2, vp2)),
                           bc2((float)(1.0 / 16.0)));
        const f2 a3 = mul2(fma2(bc2(-5.f), vm2, fma2(bc2(-11.f), vm1, fma2(bc2(70.f), v0,
                          fma2(bc2(-94.f), vp1, fma2(bc2(47.f), vp2, mul2(bc2(-7.f), vp3)))))),
                           bc2((float)(1.0 / 144.0)));
        const f2 a4 = mul2(fma2(bc2(-4.f), add2(vm1, vp1), fma2(bc2(6.f), v0, add2(vm2, vp2))),
                           bc2((float)(1.0 / 24.0)));
        const f2 a5 = mul2(add2(fma2(bc2(5.f), sub2(vm1, vp2), mul2(bc2(10.f), sub2(vp1, v0))), sub2(vp3, vm2)),
                           bc2((float)(1.0 / 120.0)));
        const f2 s1 = fma2(bc2(0.25f), a3, fma2(bc2(0.0625f), a5, a1));
        const f2 s2 = fma2(bc2((float)(63.0 / 130.0)), a4, a2);
        const f2 s3 = fma2(bc2((float)(8825.0 / 10934.0)), a5, a3);
        b6 = fma2(s1, s1, fma2(mul2(bc2((float)(13.0 / 3.0)), s2), s2,
                  fma2(mul2(bc2((float)(781.0 / 20.0)), s3), s3,
                       fma2(mul2(bc2((float)(1421461.0 / 2275.0)), a4), a4,
                            mul2(mul2(bc2((float)(21520059541.0 / 1377684.0)), a5), a5)))));
    }
    const f2 tau = abs2(sub2(b6, mul2(fma2(bc2(4.f), b[1], add2(b[0], b[2])), bc2((float)(1.0 / 6.0)))));
    const f2 P[6] = {vm2, vm1, v0, vp1, vp2, vp3};
    const f2 e = bc2((float)kTenoE), two = bc2(2.f);
    float etal = 1.f, etar = 1.f;
#pragma unroll
    for (int k = 1; k <= 4; ++k) {
        const f2 dp = sub2(P[k + 1], P[k]), dm = sub2(P[k], P[k - 1]);
        const f2 n = add2(abs2(mul2(mul2(two, dp), dm)), e);
        const f2 dd = fma2(dp, dp, fma2(dm, dm, e));
        const f2 r = mul2(n, rcp2(dd));
        etal = fminf(etal, r.v.x);
        etar = fminf(etar, r.v.y);
    }
    const float ql[4] = {q[0].v.x, q[1].v.x, q[2].v.x, q[3].v.x};
    const float qr[4] = {q[0].v.y, q[1].v.y, q[2].v.y, q[3].v.y};
    const float bl[4] = {b[0].v.x, b[1].v.x, b[2].v.x, b[3].v.x};
    const float br[4] = {b[0].v.y, b[1].v.y, b[2].v.y, b[3].v.y};
    const int kl = (etal >= float(kTenoEta1)) + (etal >= float(kTenoEta2)) + (etal >= float(kTenoEta3));
    const int kr = (etar >= float(kTenoEta1)) + (etar >= float(kTenoEta2)) + (etar >= float(kTenoEta3));
    vl = teno6a_select<float>(ql, bl, tau.v.x, teno_cutoff<float>(kl));
    vr = teno6a_select<float>(qr, br, tau.v.y, teno_cutoff<float>(kr));
}

// One reconstruction of a face: WENO5 (JS or Z weights) from x[0..4] and the
// mirrored x[5..1], or TENO6-A from x[0..5] and the mirrored x[5..0].
template <int RS, typename T>
__device__ __forceinline__ void recon_face(const T (&x)[6], T eps4, T &vl, T &vr) {
    if constexpr (RS == 2) {
        if constexpr (std::is_same<T, float>::value) {
            teno6a_pair_f2(x, vl, vr);
        } else {
            const T y[6] = {x[5], x[4], x[3], x[2], x[1], x[0]};
            const int k = teno6a_eta_class(x);  // shared by the mirrored stencil
            vl = teno6a_left(x, k);
            vr = teno6a_left(y, k);
        }
    } else {
        weno5_face<RS == 1>(x, eps4, vl, vr);
    }
}

// ------------------------------------------------------ reconstruction ----
// Face states of face i+1/2 from the stencil S[j] = W_{i-2+j}, j = 0..5.
// Characteristic mode (§3.2 steps 1-4, App. C.1): frozen state = mean of
// W_i and W_{i+1}; K^{-1} rows: acoustic (-/+ u_n/(2c) + p/(2 rho c^2)),
// entropy / partial densities (X_k - X_k_bar p/(rho c^2)), identity for the
// shear velocities and the volume fraction; back-projection with K.
// RS selects the scheme at compile time (0: WENO5-JS, 1: WENO5-Z, 2:
// TENO6-A); reconstruct() dispatches once per face on the run-time flags, so
// each scheme is scheduled as straight-line code.
template <typename T, int MODEL, int NDIM, int d, int RS>
__device__ __forceinline__ void reconstruct_w(const Dev &P, const T (&S)[6][MAXV], T *WL, T *WR) {
    using V = Vars<MODEL, NDIM>;
    constexpr int NV = V::NV, NP = V::NP, IE = V::IE;
    const T eps4 = cst<T>(P).weno_eps4;
    if (P.recon == JXF_WENO5JS_COMP) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const T x[6] = {S[0][v], S[1][v], S[2][v], S[3][v], S[4][v], S[5][v]};
            recon_face<RS>(x, eps4, WL[v], WR[v]);
        }
        return;
    }
    constexpr int in = NP + d;
    T Wb[MAXV];
#pragma unroll
    for (int v = 0; v < NV; ++v) Wb[v] = T(0.5) * (S[2][v] + S[3][v]);
    const T rho = density_of<T, MODEL, NDIM>(Wb);
    Eos<T, MODEL> eos(P, alpha_of<T, MODEL, NDIM>(Wb));
    const T rc2 = eos.rc2_from_p(P, Wb[IE]);
    // one reciprocal square root gives c, 1/c and 1/(rho c^2)
    const T t = rsq(rho * rc2);  // 1/(rho c)
    const T cb = rc2 * t;        // c
    const T rt = rho * t;        // 1/c
    const T irc2 = rt * t;       // 1/(rho c^2)
    const T h_c = T(0.5) * rt;
    const T h_rc2 = T(0.5) * irc2;
    T ent[2];
#pragma unroll
    for (int k = 0; k < NP; ++k) ent[k] = Wb[k] * irc2;

    T qL[MAXV], qR[MAXV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        T q[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            const T *w = S[j];
            T val;
            if (v < NP) val = w[v] - ent[v] * w[IE];
            else if (v == IE) val = h_c * w[in] + h_rc2 * w[IE];
            else if (v == in) val = -h_c * w[in] + h_rc2 * w[IE];
            else val = w[v];
            q[j] = val;
        }
        recon_face<RS>(q, eps4, qL[v], qR[v]);
    }
    T *outs[2] = {WL, WR};
    const T *qs[2] = {qL, qR};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        T *o = outs[s];
        const T *q = qs[s];
#pragma unroll
        for (int v = 0; v < NV; ++v) o[v] = q[v];
#pragma unroll
        for (int k = 0; k < NP; ++k) o[k] = Wb[k] * q[in] + q[k] + Wb[k] * q[IE];
        o[in] = cb * (q[IE] - q[in]);
        o[IE] = rc2 * (q[in] + q[IE]);
    }
}

// RSV: the kernel variant's scheme family -- 0: WENO5 (Jiang-Shu or Z
// weights, chosen per face from P.weno_z), 2: TENO6-A (its own kernels, so
// that its registers do not weigh on the WENO5 sweeps).
template <typename T, int MODEL, int NDIM, int d, int RSV>
__device__ __forceinline__ void reconstruct(const Dev &P, const T (&S)[6][MAXV], T *WL, T *WR) {
    if constexpr (RSV == 2) reconstruct_w<T, MODEL, NDIM, d, 2>(P, S, WL, WR);
    else if (P.weno_z) reconstruct_w<T, MODEL, NDIM, d, 1>(P, S, WL, WR);
    else reconstruct_w<T, MODEL, NDIM, d, 0>(P, S, WL, WR);
}

// ------------------------------------------------------------ limiters ----
// Interpolation limiter of one face side (§3.3 item 1): partial densities,
// volume fraction outside [eps_a, 1 - eps_a], rho c^2 -- any violation puts
// back the first-order (cell) state.  Returns 1 if switched.
template <typename T, int MODEL, int NDIM>
__device__ __forceinline__ int interp_limit(const Dev &P, T *Wf, const T *W1) {
    using V = Vars<MODEL, NDIM>;
    const Cst<T> &C = cst<T>(P);
    bool bad = false;
#pragma unroll
    for (int k = 0; k < V::NP; ++k) bad |= Wf[k] < C.eps_rho;
    if (MODEL == JXF_DIM) bad |= (Wf[V::IA] < C.eps_alpha) | (Wf[V::IA] > C.one_m_eps_alpha);
    if (!bad) {
        Eos<T, MODEL> eos(P, alpha_of<T, MODEL, NDIM>(Wf));
        bad = eos.rc2_from_p(P, Wf[V::IE]) < C.eps_rhoc2;
    }
    if (bad) {
#pragma unroll
        for (int v = 0; v < V::NV; ++v) Wf[v] = W1[v];
    }
    return bad ? 1 : 0;
}

// ---------------------------------------------------------------- HLLC ----
// HLLC flux and upwinded face velocity from primitive face states (§3.2
// step 6, App. C.2): Einfeldt s^L, s^R with sqrt(rho)-weighted averages,
// Batten s*; sign(s*) selects one branch, F^K + s^{-/+} (U^{*K} - U^K), and
// s* = 0 takes the mean of both.  The branch body exists once: its inputs
// are selected element-wise and it runs once (or twice at s* = 0).
template <typename T, int MODEL, int NDIM, int d>
__device__ __forceinline__ void hllc(const Dev &P, const T *WL, const T *WR, T *F, T &uh) {
    using V = Vars<MODEL, NDIM>;
    constexpr int NP = V::NP, IE = V::IE, NV = V::NV;
    constexpr int in = NP + d;
    const T rhoL = density_of<T, MODEL, NDIM>(WL), rhoR = density_of<T, MODEL, NDIM>(WR);
    const T uL = WL[in], uR = WR[in], pL = WL[IE], pR = WR[IE];
    Eos<T, MODEL> eL(P, alpha_of<T, MODEL, NDIM>(WL)), eR(P, alpha_of<T, MODEL, NDIM>(WR));
    // c = rho c^2 / (rho c) from one reciprocal square root per side; the
    // sqrt(rho)-weights sqrt(rho_K)/(sqrt(rho_L) + sqrt(rho_R)) from
    // r = sqrt(rho_R/rho_L): w_L = 1/(1 + r), w_R = r w_L
    const T rc2L = eL.rc2_from_p(P, pL), rc2R = eR.rc2_from_p(P, pR);
    const T cL = rc2L * rsq(rhoL * rc2L), cR = rc2R * rsq(rhoR * rc2R);
    const T c2L = cL * cL, c2R = cR * cR;
    const T r = rhoR * rsq(rhoL * rhoR);
    const T wL = rcp(T(1) + r), wR = r * wL;
    const T ubar = wL * uL + wR * uR;
    const T du = uR - uL;
    const T c2bar = wL * c2L + wR * c2R + T(0.5) * (wL * wR) * (du * du);
    const T cbar = dsqrt(c2bar);
    const T sL = tmin(ubar - cbar, uL - cL);
    const T sR = tmax(ubar + cbar, uR + cR);
    const T mL = rhoL * (sL - uL), mR = rhoR * (sR - uR);
    const T sstar = fdiv(pR - pL + mL * uL - mR * uR, mL - mR);
    const T sm = tmin(T(0), sL), sp = tmax(T(0), sR);
    const int first = sstar < T(0) ? 1 : 0;
    const int last = sstar > T(0) ? 0 : 1;
    const T wgt = first == last ? T(1) : T(0.5);
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = T(0);
    uh = T(0);
#pragma unroll 1
    for (int side = first; side <= last; ++side) {
        const bool R = side == 1;
        T W[MAXV];
#pragma unroll
        for (int v = 0; v < NV; ++v) W[v] = R ? WR[v] : WL[v];
        const T sK = R ? sR : sL, sPM = R ? sp : sm;
        T U[MAXV], rc2;
        prim2cons<T, MODEL, NDIM>(P, W, U, rc2);
        const T rho = R ? rhoR : rhoL;
        const T u = W[in], p = W[IE];
        const T su = sK - u;
        const T iD = rcp(sK - sstar);
        const T fac = su * iD;  // (s_K - u)/(s_K - s*); fac p/(s_K - u) = p iD
        T Us[MAXV];
#pragma unroll
        for (int k = 0; k < NP; ++k) Us[k] = fac * U[k];
#pragma unroll
        for (int e = 0; e < NDIM; ++e) Us[NP + e] = fac * (rho * W[NP + e]);
        Us[in] = fac * (rho * sstar);
        Us[IE] = fac * (U[IE] + (sstar - u) * (rho * sstar)) + (sstar - u) * (p * iD);
        if (MODEL == JXF_DIM) Us[V::IA] = fac * W[V::IA];
        T Fp[MAXV];
#pragma unroll
        for (int k = 0; k < NP; ++k) Fp[k] = U[k] * u;
#pragma unroll
        for (int e = 0; e < NDIM; ++e) Fp[NP + e] = U[NP + e] * u;
        Fp[in] += p;
        Fp[IE] = u * (U[IE] + p);
        if (MODEL == JXF_DIM) Fp[V::IA] = W[V::IA] * u;
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] += wgt * (Fp[v] + sPM * (Us[v] - U[v]));
        uh += wgt * (u + sPM * (fac - T(1)));
    }
}

// Flux-limiter test (§3.3 item 2) with the test states U_i - lam F and
// U_{i+1} + lam F (lam = 2 D dt/dx_d); the volume fraction also carries the
// face share of a1 div(u).  Returns true if the flux must fall back to first
// order.
template <typename T, int MODEL, int NDIM>
__device__ __forceinline__ bool flux_limit_violates(const Dev &P, T lam, const T *F, T uh,
                                                    const T *Ui, const T *Uj) {
    using V = Vars<MODEL, NDIM>;
    const Cst<T> &C = cst<T>(P);
    bool bad = false;
    const T *Uc[2] = {Ui, Uj};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const T sl = s == 0 ? -lam : lam;
        T Ts[MAXV];
#pragma unroll
        for (int v = 0; v < V::NV; ++v) Ts[v] = Uc[s][v] + sl * F[v];
        if (MODEL == JXF_DIM) Ts[V::IA] = Uc[s][V::IA] + sl * (F[V::IA] - Uc[s][V::IA] * uh);
#pragma unroll
        for (int k = 0; k < V::NP; ++k) bad |= Ts[k] < C.eps_rho;
        if (MODEL == JXF_DIM) bad |= (Ts[V::IA] < C.eps_alpha) | (Ts[V::IA] > C.one_m_eps_alpha);
        if (!bad) {
            T W[MAXV], rho, p, rc2;
            cons2prim<T, T, MODEL, NDIM>(P, Ts, W, rho, p, rc2);
            bad = rc2 < C.eps_rhoc2;
        }
    }
    return bad;
}

// ------------------------------------------------------------------ THINC --
// Interface capturing of the five-equation model (§3.2 step 4): in an
// interface cell (eps <= a1 <= 1 - eps, eps = 1e-4, and a1 monotone across
// the cell along the sweep axis) a1 follows 1/2 [1 + theta tanh(beta (xi +
// xc))] across the cell, theta = sign(a_{i+1} - a_{i-1}), beta = |n_d| + 0.01,
// xc fixed by the cell average.  With s = theta (2 a1 - 1),
// u = beta (1 + s), w = beta (1 - s), the profile's e^{2 beta (xi + xc)} is
//   xi = 1 (value from the left at the upper face): e^w expm1(u) / expm1(w)
//   xi = 0 (value from the right at the lower face): expm1(u) / (e^u expm1(w))
// and the face value e/(e+1) (theta = +1) or 1/(e+1) (theta = -1).  The
// partial densities follow with the cell's phase densities.
template <typename T> __device__ __forceinline__ T t_exp(T x);
template <> __device__ __forceinline__ double t_exp(double x) { return exp(x); }
template <> __device__ __forceinline__ float t_exp(float x) { return expf(x); }
template <typename T> __device__ __forceinline__ T t_expm1(T x);
template <> __device__ __forceinline__ double t_expm1(double x) { return expm1(x); }
template <> __device__ __forceinline__ float t_expm1(float x) { return expm1f(x); }
template <typename T> __device__ __forceinline__ T t_log(T x);
template <> __device__ __forceinline__ double t_log(double x) { return log(x); }
template <> __device__ __forceinline__ float t_log(float x) { return logf(x); }

// psi = a^0.1 / (a^0.1 + (1 - a)^0.1) of a1 clipped to [0, 1]: the smoothed
// volume fraction whose gradient gives the interface normal (§3.7),
// evaluated as 1 / (1 + ((1 - a)/a)^0.1) with one logarithm and one
// exponential (a = 0 gives 1/(1 + inf) = 0, a = 1 gives 1).
template <typename T> __device__ __forceinline__ T thinc_psi(T a1) {
    const T a = a1 < T(0) ? T(0) : (a1 > T(1) ? T(1) : a1);
    if (!(a > T(0))) return T(0);
    const T r = fdiv(T(1) - a, a);
    return rcp(T(1) + t_exp(T(0.1) * t_log(r)));
}

// One face side: cell volume fractions am, ac, ap along the axis, the cell's
// |n_d| and primitive state Wc; side 0 = the cell's upper face (WL of the
// face), side 1 = its lower face (WR).  Leaves Wf unchanged outside
// interface cells.
template <typename T, int MODEL, int NDIM>
__device__ __forceinline__ void thinc_side(T am, T ac, T ap, T nabs, int side, const T *Wc, T *Wf) {
    using V = Vars<MODEL, NDIM>;
    if (!(ac >= T(1e-4) && ac <= T(1) - T(1e-4))) return;
    if (!((ap - ac) * (ac - am) > T(0))) return;
    const bool up = ap > am;
    const T beta = nabs + T(0.01);
    const T s = up ? T(2) * ac - T(1) : T(1) - T(2) * ac;
    const T u = beta * (T(1) + s), w = beta * (T(1) - s);
    const T em = t_expm1(u);
    const T e = side == 0 ? fdiv(t_exp(w) * em, t_expm1(w)) : fdiv(em, t_exp(u) * t_expm1(w));
    const T a = up ? fdiv(e, e + T(1)) : rcp(e + T(1));
    Wf[0] = a * fdiv(Wc[0], ac);
    Wf[1] = (T(1) - a) * fdiv(Wc[1], T(1) - ac);
    Wf[V::IA] = a;
}

// |n_d| of cell i from central differences of psi (neighbours mapped through
// the boundary conditions): n = grad psi / |grad psi|, 0 where grad psi = 0.
template <typename T, int NDIM>
__device__ __forceinline__ void normal_cell(const Dev &P, long long i) {
    T *G = static_cast<T *>(P.G);
    const size_t nc = (size_t)P.vstride;
    const T *psi = G + (size_t)NDIM * nc;
    const unsigned iu = (unsigned)i;
    const unsigned qy = P.fd_cell[0].div(iu), qz = P.fd_cell[1].div(qy);
    const int c[3] = {(int)(iu - qy * (unsigned)P.n[0]), (int)(qy - qz * (unsigned)P.n[1]), (int)qz};
    T g[3], g2 = T(0);
#pragma unroll
    for (int e = 0; e < NDIM; ++e) {
        const int se = e == 0 ? 1 : (e == 1 ? P.n[0] : P.n[0] * P.n[1]);
        int mk = 0;
        const int cm = map_axis(c[e] - 1, P.n[e], P.bc[e][0], P.bc[e][1], mk, 1);
        const int cp = map_axis(c[e] + 1, P.n[e], P.bc[e][0], P.bc[e][1], mk, 1);
        const int b = (int)i - c[e] * se;
        g[e] = (__ldg(psi + chk_cell(P, b + cp * se)) - __ldg(psi + chk_cell(P, b + cm * se))) *
               (T(0.5) * cst<T>(P).inv_dx[e]);
        g2 += g[e] * g[e];
    }
    const T ig = g2 > T(0) ? rcp(dsqrt(g2)) : T(0);
#pragma unroll
    for (int e = 0; e < NDIM; ++e) (G + e * nc)[(int)i] = fabs(g[e]) * ig;
}

// ---------------------------------------------------------- viscous flux --
// Central stencils of order 2H (H points per side; §3.2 and App. A offer
// 2nd/4th/6th-order central differences for the dissipative terms), on the
// face's normal cells v[0..2H-1] = phi_{i+1-H..i+H}, or a cell's neighbours
// w[0..2H] = phi_{j-H..j+H} (scales 1/dx factors in vis_dn, vis_cd):
//   face-normal derivative: (v1 - v0) | (v0 - 27 v1 + 27 v2 - v3) |
//       (-9 v0 + 125 v1 - 2250 v2 + 2250 v3 - 125 v4 + 9 v5), times vis_dn
//   face value: (v0 + v1)/2 | (-v0 + 9 v1 + 9 v2 - v3)/16 |
//       (3 v0 - 25 v1 + 150 v2 + 150 v3 - 25 v4 + 3 v5)/256
//   cell-centred derivative: (w2 - w0) | (w0 - 8 w1 + 8 w3 - w4) |
//       (-w0 + 9 w1 - 45 w2 + 45 w4 - 9 w5 + w6), times vis_cd
template <int H, typename T> __device__ __forceinline__ T face_dn(const T *v) {
    if constexpr (H == 1) return v[1] - v[0];
    else if constexpr (H == 2) return (v[0] - v[3]) + T(27) * (v[2] - v[1]);
    else return T(9) * (v[5] - v[0]) + T(125) * (v[1] - v[4]) + T(2250) * (v[3] - v[2]);
}
template <int H, typename T> __device__ __forceinline__ T face_val(const T *v) {
    if constexpr (H == 1) return T(0.5) * (v[0] + v[1]);
    else if constexpr (H == 2) return T(9.0 / 16.0) * (v[1] + v[2]) - T(1.0 / 16.0) * (v[0] + v[3]);
    else
        return T(150.0 / 256.0) * (v[2] + v[3]) - T(25.0 / 256.0) * (v[1] + v[4]) +
               T(3.0 / 256.0) * (v[0] + v[5]);
}
template <int H, typename T> __device__ __forceinline__ T cell_dc(const T *w) {
    if constexpr (H == 1) return w[2] - w[0];
    else if constexpr (H == 2) return (w[0] - w[4]) + T(8) * (w[3] - w[1]);
    else return (w[6] - w[0]) + T(9) * (w[1] - w[5]) + T(45) * (w[4] - w[2]);
}

// Cell-centred velocity gradient of cell i (central, order 2H, neighbours
// boundary-mapped along e: a mirrored neighbour flips u_e), from the
// primitives W into G: the cross derivatives du_f/dx_e (f != e) in slot
// f*ndim+e, and in the diagonal slot d*ndim+d the part of div u a face of
// axis d needs from its tangential axes, D_d = sum_{e != d} du_e/dx_e.
// Computed once per cell and stage; the viscous face fluxes interpolate it.
template <typename T, int NDIM, int H>
__device__ __forceinline__ void grad_cell_h(const Dev &P, long long i) {
    const T *W = static_cast<const T *>(P.W);
    T *G = static_cast<T *>(P.G);
    const size_t nc = (size_t)P.vstride;
    const unsigned iu = (unsigned)i;
    const unsigned qy = P.fd_cell[0].div(iu), qz = P.fd_cell[1].div(qy);
    const int c[3] = {(int)(iu - qy * (unsigned)P.n[0]), (int)(qy - qz * (unsigned)P.n[1]), (int)qz};
    // cell indices stay below 2^31 (checked at creation): 32-bit index
    // arithmetic off warp-uniform field base pointers
    const int ic = (int)i;
    T diag[3];  // du_e/dx_e
#pragma unroll
    for (int e = 0; e < NDIM; ++e) {
        const int se = e == 0 ? 1 : (e == 1 ? P.n[0] : P.n[0] * P.n[1]);
        int nb[2 * H + 1];  // neighbour cell indices along e
        unsigned me = 0;
        if (c[e] >= H && c[e] < P.n[e] - H) {  // all neighbours inside: no mapping
#pragma unroll
            for (int k = 0; k <= 2 * H; ++k) nb[k] = chk_cell(P, ic + (k - H) * se);
        } else {
#pragma unroll
            for (int k = 0; k <= 2 * H; ++k) {
                int mk = 0;
                const int ck = map_axis(c[e] + k - H, P.n[e], P.bc[e][0], P.bc[e][1], mk, 1);
                nb[k] = chk_cell(P, ic + (ck - c[e]) * se);
                me |= (unsigned)mk << k;
            }
        }
#pragma unroll
        for (int f = 0; f < NDIM; ++f) {
            const T *Wf = W + (1 + f) * nc;
            T w[2 * H + 1];
#pragma unroll
            for (int k = 0; k <= 2 * H; ++k) {
                if (k == H) {
                    w[k] = T(0);  // the centre carries no weight
                    continue;
                }
                const T u = __ldg(Wf + nb[k]);
                w[k] = (f == e && ((me >> k) & 1u)) ? -u : u;
            }
            const T g = cell_dc<H>(w) * cst<T>(P).vis_cd[e];
            if (f == e) diag[e] = g;
            else (G + (f * NDIM + e) * nc)[ic] = g;
        }
    }
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        T sum = T(0);
#pragma unroll
        for (int e = 0; e < NDIM; ++e)
            if (e != d) sum = add_rn(sum, diag[e]);
        (G + (d * NDIM + d) * nc)[ic] = sum;
    }
}

template <typename T, int NDIM>
__device__ __forceinline__ void grad_cell(const Dev &P, long long i) {
    if (P.visc_half == 1) grad_cell_h<T, NDIM, 1>(P, i);
    else if (P.visc_half == 3) grad_cell_h<T, NDIM, 3>(P, i);
    else grad_cell_h<T, NDIM, 2>(P, i);
}

// The per-cell auxiliary pass after new primitives: the viscous velocity
// gradient (single phase) or the THINC interface normal (five-equation).
template <typename T, int MODEL, int NDIM> __device__ __forceinline__ void aux_cell(const Dev &P, long long i) {
    if constexpr (MODEL == JXF_SPM) grad_cell<T, NDIM>(P, i);
    else normal_cell<T, NDIM>(P, i);
}

template <typename T, int MODEL, int NDIM>
__global__ void __launch_bounds__(kCellThreads, CellMinBlocks<T>::value) k_aux(const Dev P) {
    double dt;
    if (!block_dt(P, dt)) return;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P.ncell) aux_cell<T, MODEL, NDIM>(P, i);
}

// The gradient pass of grad_cell_h for K = 2 or 4 consecutive cells
// x0..x0+K-1 of a row (float, n0 a multiple of K): each 8- or 16-byte load
// brings a neighbour's value for all K cells (the rows at the y / z offsets,
// and along x the cells x0-4..x0+K+3 in blocks of K), each 8- or 16-byte
// store writes one derivative of the K cells.  Neighbours outside the grid
// along x are mapped one by one; the arithmetic of each cell is that of
// grad_cell_h.
template <int K> struct VecF;
template <> struct VecF<2> {
    using type = float2;
    static __device__ __forceinline__ void put(float *p, const float *v) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    }
    static __device__ __forceinline__ void get(const float *p, float *v) {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        v[0] = t.x, v[1] = t.y;
    }
};
template <> struct VecF<4> {
    using type = float4;
    static __device__ __forceinline__ void put(float *p, const float *v) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
    static __device__ __forceinline__ void get(const float *p, float *v) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    }
};

template <int NDIM, int H, int K> __device__ __forceinline__ void grad_vec(const Dev &P, int q) {
    using VF = VecF<K>;
    const float *W = static_cast<const float *>(P.W);
    float *G = static_cast<float *>(P.G);
    const size_t nc = (size_t)P.vstride;
    const int i0 = K * q;
    const int n0 = P.n[0];
    const unsigned qy = P.fd_cell[0].div((unsigned)i0), qz = P.fd_cell[1].div(qy);
    const int c[3] = {i0 - (int)qy * n0, (int)(qy - qz * (unsigned)P.n[1]), (int)qz};
    float diag[3][K];
#pragma unroll
    for (int e = 0; e < NDIM; ++e) {
        const float sc = cst<float>(P).vis_cd[e];
        if (e == 0) {
#pragma unroll
            for (int f = 0; f < NDIM; ++f) {
                const float *Wf = W + (size_t)(1 + f) * nc;
                float v[K + 8];  // cells x0-4 .. x0+K+3 of the row
                VF::get(Wf + chk_cell(P, i0), v + 4);
                if (c[0] >= 4) {
#pragma unroll
                    for (int m = 0; m < 4; m += K) VF::get(Wf + chk_cell(P, i0 - 4 + m), v + m);
                } else {
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        int mk = 0;
                        const int xm = map_axis(c[0] - 4 + m, n0, P.bc[0][0], P.bc[0][1], mk, 1);
                        const float u = __ldg(Wf + chk_cell(P, i0 - c[0] + xm));
                        v[m] = (f == 0 && mk) ? -u : u;
                    }
                }
                if (c[0] + K + 4 <= n0) {
#pragma unroll
                    for (int m = 0; m < 4; m += K) VF::get(Wf + chk_cell(P, i0 + K + m), v + 4 + K + m);
                } else {
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        int mk = 0;
                        const int xm = map_axis(c[0] + K + m, n0, P.bc[0][0], P.bc[0][1], mk, 1);
                        const float u = __ldg(Wf + chk_cell(P, i0 - c[0] + xm));
                        v[4 + K + m] = (f == 0 && mk) ? -u : u;
                    }
                }
                float out[K];
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    float w[2 * H + 1];
#pragma unroll
                    for (int k = 0; k <= 2 * H; ++k) w[k] = k == H ? 0.f : v[4 + j + k - H];
                    out[j] = cell_dc<H>(w) * sc;
                }
                if (f == 0) {
#pragma unroll
                    for (int j = 0; j < K; ++j) diag[0][j] = out[j];
                } else {
                    VF::put(G + (size_t)(f * NDIM) * nc + i0, out);
                }
            }
        } else {
            const int se = e == 1 ? n0 : n0 * P.n[1];
            int off[2 * H + 1];
            unsigned me = 0;
#pragma unroll
            for (int k = 0; k <= 2 * H; ++k) {
                int mk = 0;
                const int ck = map_axis(c[e] + k - H, P.n[e], P.bc[e][0], P.bc[e][1], mk, 1);
                off[k] = (ck - c[e]) * se;
                me |= (unsigned)mk << k;
            }
#pragma unroll
            for (int f = 0; f < NDIM; ++f) {
                const float *Wf = W + (size_t)(1 + f) * nc;
                float r[2 * H + 1][K];
#pragma unroll
                for (int k = 0; k <= 2 * H; ++k)
                    if (k != H) VF::get(Wf + chk_cell(P, i0 + off[k]), r[k]);
                float out[K];
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    float w[2 * H + 1];
#pragma unroll
                    for (int k = 0; k <= 2 * H; ++k) {
                        if (k == H) {
                            w[k] = 0.f;
                            continue;
                        }
                        w[k] = (f == e && ((me >> k) & 1u)) ? -r[k][j] : r[k][j];
                    }
                    out[j] = cell_dc<H>(w) * sc;
                }
                if (f == e) {
#pragma unroll
                    for (int j = 0; j < K; ++j) diag[e][j] = out[j];
                } else {
                    VF::put(G + (size_t)(f * NDIM + e) * nc + i0, out);
                }
            }
        }
    }
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        float sum[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            sum[j] = 0.f;
#pragma unroll
            for (int e = 0; e < NDIM; ++e)
                if (e != d) sum[j] = add_rn(sum[j], diag[e][j]);
        }
        VF::put(G + (size_t)(d * NDIM + d) * nc + i0, sum);
    }
}

#ifndef JXF_AUX_CELLS
#define JXF_AUX_CELLS 4
#endif
constexpr int kAuxCells = JXF_AUX_CELLS;  // cells per thread of the float gradient pass (1: one-cell k_aux; 2; 4)
template <int NDIM>
__global__ void __launch_bounds__(kCellThreads, kAuxCells == 4 ? 4 : 6) k_aux_vec(const Dev P) {
    double dt;
    if (!block_dt(P, dt)) return;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= P.ncell / kAuxCells) return;
    if (P.visc_half == 1) grad_vec<NDIM, 1, kAuxCells>(P, (int)q);
    else if (P.visc_half == 3) grad_vec<NDIM, 3, kAuxCells>(P, (int)q);
    else grad_vec<NDIM, 2, kAuxCells>(P, (int)q);
}

// F^d on face i+1/2 of axis d (§2.1): tau_dk and the heat flux from the
// central stencils of order 2H above -- normal derivative and face value on
// the normal cells i+1-H..i+H, tangential derivative: the cell-centred
// derivative (k_aux) of those cells interpolated to the face.  Only du_d/dx_e
// and du_e/dx_e are needed along a tangential axis e.  S[0..5] are the face's
// stencil primitives (cells i-2..i+3, boundary-mapped along d, the mirrored
// normal velocity already flipped); src gives the temperature and the
// cell-centred derivatives of those cells.
template <typename T, int NDIM, int d, int H, typename Src>
__device__ __forceinline__ void viscous_flux(const Dev &P, const Src &src, const T (&S)[6][MAXV], T *Fd) {
    const Cst<T> &C = cst<T>(P);
    constexpr int j0 = 3 - H;  // first normal cell in the stencil
    T g[NDIM + 1][3];  // g[f][e]: d phi_f / d x_e at the face (phi = u_0.., T)
    T fu[NDIM];
#pragma unroll
    for (int f = 0; f <= NDIM; ++f) {
        T v[2 * H];
#pragma unroll
        for (int m = 0; m < 2 * H; ++m) v[m] = f < NDIM ? S[j0 + m][1 + f] : src.tt(j0 + m);
        g[f][d] = face_dn<H>(v) * C.vis_dn[d];
        if (f < NDIM) fu[f] = face_val<H>(v);
    }
    // tangential derivatives: the cell-centred cross derivatives du_d/dx_e and
    // the tangential divergence D_d of the normal cells, interpolated to the
    // face; a cell mirrored across the face's axis flips u_d (not D_d)
#pragma unroll
    for (int e = 0; e < NDIM; ++e) {
        if (e == d) continue;
        T gm[2 * H];
#pragma unroll
        for (int m = 0; m < 2 * H; ++m) gm[m] = src.gt(e, j0 + m);
        g[d][e] = face_val<H>(gm);
    }
    T div = g[d][d];
    if constexpr (NDIM > 1) {
        T gm[2 * H];
#pragma unroll
        for (int m = 0; m < 2 * H; ++m) gm[m] = src.gdiv(j0 + m);
        div += face_val<H>(gm);
    }
    const T mu = C.mu;
    T work = T(0);
    Fd[0] = T(0);
#pragma unroll
    for (int k = 0; k < NDIM; ++k) {
        T tau = mu * (g[d][k] + g[k][d]);
        if (k == d) tau -= T(2.0 / 3.0) * mu * div;
        Fd[1 + k] = tau;
        work += fu[k] * tau;
    }
    Fd[1 + NDIM] = work + C.lam_heat * g[NDIM][d];  // - q_d = + lambda dT/dx_d
}

// ------------------------------------------------------- stencil sources --
// Where the face code finds the values of its six stencil cells j = 0..5
// (cells i-2..i+3 along the face's axis d): the primitives w(j, v), the
// temperature tt(j), the cell-centred derivatives of the viscous flux
// (gt(e, j): du_d/dx_e, e != d; gdiv(j): D_d), the THINC normal |n_d| nd(j)
// and the conservative state of the face's two cells ucell(j, U), j = 2, 3.
// A cell mirrored across the face's axis carries u_d (and du_d/dx_e) with
// the opposite sign.
//
// The cell arrays in global memory, at the stencil's boundary-mapped cell
// indices idx with their mirror bits mir (MIR = false: no cell mirrored).
template <typename T, int MODEL, int NDIM, int d, bool MIR> struct GlobalStencil {
    using V = Vars<MODEL, NDIM>;
    const Dev &P;
    const int (&idx)[6];
    unsigned mir;
    __device__ __forceinline__ bool flipped(int j) const { return MIR && ((mir >> j) & 1u); }
    __device__ __forceinline__ T w(int j, int v) const {
        const T x = __ldg(static_cast<const T *>(P.W) + v * (size_t)P.vstride + idx[j]);
        return (v == V::NP + d && flipped(j)) ? -x : x;
    }
    __device__ __forceinline__ T tt(int j) const { return __ldg(static_cast<const T *>(P.Tt) + idx[j]); }
    __device__ __forceinline__ T gt(int e, int j) const {
        const T x = __ldg(static_cast<const T *>(P.G) + (size_t)(d * NDIM + e) * (size_t)P.vstride + idx[j]);
        return flipped(j) ? -x : x;
    }
    __device__ __forceinline__ T gdiv(int j) const {
        return __ldg(static_cast<const T *>(P.G) + (size_t)(d * NDIM + d) * (size_t)P.vstride + idx[j]);
    }
    __device__ __forceinline__ T nd(int j) const {
        return __ldg(static_cast<const T *>(P.G) + (size_t)d * (size_t)P.vstride + idx[j]);
    }
    __device__ __forceinline__ void ucell(int j, T *U) const {
        const T *Uc = static_cast<const T *>(P.Ucell);
#pragma unroll
        for (int v = 0; v < V::NV; ++v) U[v] = __ldg(Uc + v * (size_t)P.vstride + idx[j]);
        if (flipped(j)) U[V::NP + d] = -U[V::NP + d];
    }
};

// ------------------------------------------------------------ face sweep --
// The work of one face (stencil values from src): stencil
// gather, reconstruction, interpolation limiter, HLLC, flux limiter, viscous
// flux; returns F (and u_hllc).  Shared by the single-grid sweep, the fused
// last-axis sweep and the batched persistent sweep.
// VH: points per side of the viscous stencils (0: no viscous flux).
template <typename T, int MODEL, int NDIM, int d, int VH, int RSV, typename Src>
__device__ __forceinline__ void flux_face_eval(const Dev &P, double dt, const int (&c)[3], const Src &src, bool count,
                                               T (&F)[MAXV], T &uh, bool &il_hit, bool &fl_hit);

// The flux F (= F^c - F^d) and upwinded velocity uh of the face of axis d at
// face coordinates c (face c[d] lies between cells c[d]-1 and c[d]).
// count = false: the face is computed a second time (by a block that shares
// it) and stays out of the limiter counters.
template <typename T, int MODEL, int NDIM, int d, int VH, int RSV>
__device__ __forceinline__ void flux_face_at(const Dev &P, double dt, const int (&c)[3], bool count,
                                             T (&F)[MAXV], T &uh, bool &il_hit, bool &fl_hit) {
    // face c[d] lies between cells c[d]-1 (i) and c[d] (i+1).  Stencil
    // cells i-2..i+3 differ only along d: map that coordinate through
    // the boundary conditions once per cell (bit j of mir: mirrored).
    const int sd = d == 0 ? 1 : (d == 1 ? P.n[0] : P.n[0] * P.n[1]);
    const int base = ((c[2] * P.n[1] + c[1]) * P.n[0] + c[0]) - c[d] * sd;
    int idx[6];
    unsigned mir = 0;
    if (c[d] >= 3 && c[d] <= P.n[d] - 3) {  // whole stencil inside: no mapping
#pragma unroll
        for (int j = 0; j < 6; ++j) idx[j] = chk_cell(P, base + (c[d] + j - 3) * sd);
    } else {
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            int mj = 0;
            const int cj = map_axis(c[d] + j - 3, P.n[d], P.bc[d][0], P.bc[d][1], mj, 1);
            idx[j] = chk_cell(P, base + cj * sd);
            mir |= (unsigned)mj << j;
        }
    }
    // Float sweeps across y or z: the stencil's mirror pattern is constant
    // along a row of x-faces (so over a warp when the row length is a
    // multiple of 32); faces without mirrored cells take a copy of the face
    // code with the sign flips compiled out.
    if constexpr (d > 0 && std::is_same<T, float>::value) {
        if (mir == 0u) {
            const GlobalStencil<T, MODEL, NDIM, d, false> src{P, idx, 0u};
            flux_face_eval<T, MODEL, NDIM, d, VH, RSV>(P, dt, c, src, count, F, uh, il_hit, fl_hit);
            return;
        }
    }
    const GlobalStencil<T, MODEL, NDIM, d, true> src{P, idx, mir};
    flux_face_eval<T, MODEL, NDIM, d, VH, RSV>(P, dt, c, src, count, F, uh, il_hit, fl_hit);
}

// Face g of axis d (x-fastest index over the faces of axis d): its flux into
// the face arrays.
template <typename T, int MODEL, int NDIM, int d, int VH, int RSV>
__device__ __forceinline__ void flux_face(const Dev &P, double dt, long long g, const int (&m)[3],
                                          long long nface, bool &il_hit, bool &fl_hit) {
    const unsigned gu = (unsigned)g;
    const unsigned q0 = P.fd_face[d][0].div(gu);
    const unsigned q1 = P.fd_face[d][1].div(q0);
    const int c[3] = {(int)(gu - q0 * (unsigned)m[0]), (int)(q0 - q1 * (unsigned)m[1]), (int)q1};
    T F[MAXV], uh;
    flux_face_at<T, MODEL, NDIM, d, VH, RSV>(P, dt, c, true, F, uh, il_hit, fl_hit);
    constexpr int NV = Vars<MODEL, NDIM>::NV;
    T *Fo = static_cast<T *>(P.F[d]);
#pragma unroll
    for (int v = 0; v < NV; ++v) (Fo + v * nface)[(int)g] = F[v];  // g < 2^31 (checked at creation)
    if (MODEL == JXF_DIM) static_cast<T *>(P.UH[d])[(int)g] = uh;
}

template <typename T, int MODEL, int NDIM, int d, int VH, int RSV, typename Src>
__device__ __forceinline__ void flux_face_eval(const Dev &P, double dt, const int (&c)[3], const Src &src, bool count,
                                               T (&F)[MAXV], T &uh, bool &il_hit, bool &fl_hit) {
    using V = Vars<MODEL, NDIM>;
    constexpr int NV = V::NV;
    T S[6][MAXV];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
#pragma unroll
        for (int v = 0; v < NV; ++v) S[j][v] = src.w(j, v);
    }
    // dissipative flux first, while the stencil's velocities are at hand
    T Fd[MAXV];
    if constexpr (MODEL == JXF_SPM && VH > 0) viscous_flux<T, NDIM, d, VH>(P, src, S, Fd);
    T WL[MAXV], WR[MAXV];
    reconstruct<T, MODEL, NDIM, d, RSV>(P, S, WL, WR);
    if constexpr (MODEL == JXF_DIM) {
        if (P.thinc) {  // cell i's upper face value, cell i+1's lower face value
            constexpr int IA = V::IA;
            thinc_side<T, MODEL, NDIM>(S[1][IA], S[2][IA], S[3][IA], src.nd(2), 0, S[2], WL);
            thinc_side<T, MODEL, NDIM>(S[2][IA], S[3][IA], S[4][IA], src.nd(3), 1, S[3], WR);
        }
    }
    // the lowest face of a block whose lower side is shared with the block
    // below is that block's highest face too: only one of them counts it
    const bool counted = count && !(d == NDIM - 1 && c[d] == 0 && P.skip_face0_count);
    if (P.limiter) {
        int k = interp_limit<T, MODEL, NDIM>(P, WL, S[2]);
        k += interp_limit<T, MODEL, NDIM>(P, WR, S[3]);
        il_hit = counted && k != 0;
        if (k == 2 && counted) atomicAdd(P.counters, 1ull);  // count the extra side
    }
    // HLLC of the reconstructed states; the flux limiter may send the loop
    // round once more with the first-order states (one HLLC copy in code)
#pragma unroll 1
    for (int pass = 0;; ++pass) {
        hllc<T, MODEL, NDIM, d>(P, WL, WR, F, uh);
        if (pass > 0 || !P.limiter) break;
        T Ui[MAXV], Uj[MAXV];
        src.ucell(2, Ui);
        src.ucell(3, Uj);
        const T lam = T(cst<T>(P).fl_lam[d] * T(dt));
        if (!flux_limit_violates<T, MODEL, NDIM>(P, lam, F, uh, Ui, Uj)) break;
        fl_hit = counted;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            WL[v] = S[2][v];
            WR[v] = S[3][v];
        }
    }
    if constexpr (MODEL == JXF_SPM && VH > 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] -= Fd[v];
    }
}

// Limiter activity of a warp into the counters (all lanes must call).
__device__ __forceinline__ void count_limited(const Dev &P, bool il_hit, bool fl_hit) {
    const unsigned il = __popc(__ballot_sync(0xffffffffu, il_hit));
    const unsigned fl = __popc(__ballot_sync(0xffffffffu, fl_hit));
    if ((threadIdx.x & 31) == 0) {
        if (il) atomicAdd(P.counters, (unsigned long long)il);
        if (fl) atomicAdd(P.counters + 1, (unsigned long long)fl);
    }
}

template <typename T, int MODEL, int NDIM, int d, int VH, int RSV>
__global__ void __launch_bounds__(kFluxThreads, SweepMinBlocks<T, RSV>::value) k_flux(const Dev P) {
    double dt;
    if (!block_dt(P, dt)) return;
    int m[3] = {P.n[0], P.n[1], P.n[2]};
    m[d] += 1;
    const long long nface = (long long)m[0] * m[1] * m[2];
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool il_hit = false, fl_hit = false;
    if (g < nface) flux_face<T, MODEL, NDIM, d, VH, RSV>(P, dt, g, m, nface, il_hit, fl_hit);
    if (P.limiter) count_limited(P, il_hit, fl_hit);
}

// -------------------------------------------------- block reductions -----
// ---------------------------------------------------- shared-memory tiles --
// The float sweeps across y (and z outside the fused stage) stage the cells
// of a tile, with three halo cells on each side along the sweep axis, in
// shared memory once per launch: the boundary mapping and the mirror sign
// flips are applied while staging, and every face then reads its stencil at
// fixed offsets from one address (the face arithmetic is the same as from
// the global arrays, so are the results).  Measured on the 128^3 TGV: 57.5
// against 59.5 us per y sweep.  The x sweep (whole rows staged) and the
// fused last-axis sweep were slower staged and read the global arrays.  A staged cell holds its NA values side by side: the primitives,
// then (viscous single-phase) the temperature and the sweep axis's
// cell-centred derivatives du_d/dx_e (e != d, mirror-flipped) and D_d in slot
// NV + 1 + e, or (five-equation) the THINC normal |n_d| in slot NV.  NA is
// odd, so that consecutive cells fall in different shared-memory banks.
template <int MODEL, int NDIM, int VH> struct TileSlots {
    static constexpr int NV = Vars<MODEL, NDIM>::NV;
    static constexpr int NR = NV + (MODEL == JXF_SPM && VH > 0 ? 1 + NDIM : 0) + (MODEL == JXF_DIM ? 1 : 0);
    static constexpr int NA = NR | 1;
};

// Stage cell ci (mirrored across axis d's boundary if mir) into s.
template <typename T, int MODEL, int NDIM, int d, int VH>
__device__ __forceinline__ void stage_cell(const Dev &P, int ci, int mir, T *s) {
    using V = Vars<MODEL, NDIM>;
    constexpr int NV = V::NV;
    const size_t nc = (size_t)P.vstride;
    ci = chk_cell(P, ci);
    const T *W = static_cast<const T *>(P.W);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const T x = __ldg(W + v * nc + ci);
        s[v] = (mir && v == V::NP + d) ? -x : x;
    }
    if constexpr (MODEL == JXF_SPM && VH > 0) {
        s[NV] = __ldg(static_cast<const T *>(P.Tt) + ci);
        const T *G = static_cast<const T *>(P.G);
#pragma unroll
        for (int e = 0; e < NDIM; ++e) {
            const T x = __ldg(G + (size_t)(d * NDIM + e) * nc + ci);
            s[NV + 1 + e] = (mir && e != d) ? -x : x;
        }
    }
    if constexpr (MODEL == JXF_DIM) {
        if (P.thinc) s[NV] = __ldg(static_cast<const T *>(P.G) + (size_t)d * nc + ci);
    }
}

// Stencil source of a staged tile: s points at stencil cell 0 of the face,
// CS values apart from cell to cell.  The conservative states of the face's
// two cells (flux limiter) come from the global array.
template <typename T, int MODEL, int NDIM, int d, int VH, int CS> struct TileStencil {
    using V = Vars<MODEL, NDIM>;
    using Sl = TileSlots<MODEL, NDIM, VH>;
    const Dev &P;
    const T *s;
    const int (&c)[3];
    __device__ __forceinline__ T w(int j, int v) const { return s[j * CS + v]; }
    __device__ __forceinline__ T tt(int j) const { return s[j * CS + Sl::NV]; }
    __device__ __forceinline__ T gt(int e, int j) const { return s[j * CS + Sl::NV + 1 + e]; }
    __device__ __forceinline__ T gdiv(int j) const { return s[j * CS + Sl::NV + 1 + d]; }
    __device__ __forceinline__ T nd(int j) const { return s[j * CS + Sl::NV]; }
    __device__ __forceinline__ void ucell(int j, T *U) const {
        int mk = 0;
        const int cj = map_axis(c[d] - 3 + j, P.n[d], P.bc[d][0], P.bc[d][1], mk, 1);
        const int sd = d == 0 ? 1 : (d == 1 ? P.n[0] : P.n[0] * P.n[1]);
        const int i = chk_cell(P, ((c[2] * P.n[1] + c[1]) * P.n[0] + c[0]) + (cj - c[d]) * sd);
        const T *Uc = static_cast<const T *>(P.Ucell);
#pragma unroll
        for (int v = 0; v < V::NV; ++v) U[v] = __ldg(Uc + v * (size_t)P.vstride + i);
        if (mk) U[V::NP + d] = -U[V::NP + d];
    }
};

// Faces of axis d >= 1 (float): a block stages kTileX x-columns by
// kTileD + 6 cells along d (the remaining axis fixed: blockIdx.z) and
// computes the tile's faces d0 .. d0 + kTileD - 1 (the last tile along d also
// face n_d), warp w taking every fourth face row from w.
constexpr int kTileX = 32, kTileD = 16;
template <typename T, int MODEL, int NDIM, int d, int VH, int RSV>
__global__ void __launch_bounds__(kFluxThreads, SweepMinBlocks<T, RSV>::value) k_flux_td(const Dev P) {
    using Sl = TileSlots<MODEL, NDIM, VH>;
    constexpr int NV = Sl::NV, NA = Sl::NA, ROWS = kTileD + 6, WARPS = kFluxThreads / 32;
    __shared__ __align__(16) T sm[ROWS * kTileX * NA];
    double dt;
    if (!block_dt(P, dt)) return;
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int x = (int)blockIdx.x * kTileX + lane;
    const int d0 = (int)blockIdx.y * kTileD;
    const int o = (int)blockIdx.z;  // 3-D: the coordinate of the axis other than x and d
    const int nd = P.n[d];
    const bool xin = x < P.n[0];
    for (int k = wy; k < ROWS; k += WARPS) {
        int mir = 0;
        const int cd = map_axis(d0 - 3 + k, nd, P.bc[d][0], P.bc[d][1], mir, 1);
        if (xin) {
            int c[3] = {x, 0, 0};
            c[d] = cd;
            if (NDIM == 3) c[3 - d] = o;
            stage_cell<T, MODEL, NDIM, d, VH>(P, (c[2] * P.n[1] + c[1]) * P.n[0] + c[0], mir,
                                              sm + (k * kTileX + lane) * NA);
        }
    }
    __syncthreads();
    int m[3] = {P.n[0], P.n[1], P.n[2]};
    m[d] += 1;
    const long long nface = (long long)m[0] * m[1] * m[2];
    const int fend = min(d0 + kTileD, nd) + (d0 + kTileD >= nd ? 1 : 0);
    T *Fo = static_cast<T *>(P.F[d]);
    for (int f = d0 + wy; f < fend; f += WARPS) {  // warp-uniform
        bool il = false, fl = false;
        if (xin) {
            int c[3] = {x, 0, 0};
            c[d] = f;
            if (NDIM == 3) c[3 - d] = o;
            const TileStencil<T, MODEL, NDIM, d, VH, kTileX * NA> src{P, sm + ((f - d0) * kTileX + lane) * NA, c};
            T F[MAXV], uh;
            flux_face_eval<T, MODEL, NDIM, d, VH, RSV>(P, dt, c, src, true, F, uh, il, fl);
            const int g = chk_face(P, ((long long)c[2] * m[1] + c[1]) * m[0] + c[0], nface);
#pragma unroll
            for (int v = 0; v < NV; ++v) (Fo + v * nface)[g] = F[v];
            if (MODEL == JXF_DIM) static_cast<T *>(P.UH[d])[g] = uh;
        }
        if (P.limiter) count_limited(P, il, fl);
    }
}

template <typename T> __device__ __forceinline__ T shfl_down(T v, int o) {
    return __shfl_down_sync(0xffffffffu, v, o);
}
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_down(v, o);
    return v;
}
template <typename T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, shfl_down(v, o));
    return v;
}
template <typename T> __device__ __forceinline__ T warp_min(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, shfl_down(v, o));
    return v;
}

// Sum over a warp, returned in double on lane 0.  Double values add in
// double; float values add as compensated pairs (hi + lo, Knuth's TwoSum at
// every level) so that the warp sum keeps about 48 bits before it is handed
// to double -- the float path does no per-cell double arithmetic.
// Sum of per-thread compensated float pairs over a warp, in double on lane 0.
__device__ __forceinline__ double warp_sum_pairs_to_double(float hi, float lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_down_sync(0xffffffffu, hi, o), ol = __shfl_down_sync(0xffffffffu, lo, o);
        const float s = hi + oh;
        const float bb = s - hi;
        const float err = (hi - (s - bb)) + (oh - bb);
        lo = lo + ol + err;
        hi = s;
    }
    return (double)hi + (double)lo;
}
__device__ __forceinline__ double warp_sum_to_double(double v) { return warp_sum(v); }
__device__ __forceinline__ double warp_sum_to_double(float v) {
    float hi = v, lo = 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = shfl_down(hi, o), ol = shfl_down(lo, o);
        const float s = hi + oh;
        const float bb = s - hi;
        const float err = (hi - (s - bb)) + (oh - bb);
        lo = lo + ol + err;
        hi = s;
    }
    return (double)hi + (double)lo;
}

// Error-free transformations in float: a + b = s + e exactly (Knuth's
// TwoSum), and the rounding error of a product from one fused multiply-add.
__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// U -> W of a float state with p_inf != 0.  p = (rho e - B)/A with
// rho e = E - rho|u|^2/2 is a small difference of large numbers (water:
// B = gamma p_inf/(gamma-1) = 4.1e8, and up to 1e8 of kinetic energy at
// 500 m/s, against A p ~ 2e4).  The stored float state is exact input; the
// pressure is formed from it in compensated float arithmetic, so that it
// agrees with a double-precision evaluation of the same floats to a few
// float ulps of p: B is an unevaluated pair Bh + Bl (the mixture's
// B2 + a1 (B1 - B2) with an exact product error and an exact two-sum), the
// density and each velocity carry their rounding residuals (u = m/rho to
// about 2^-44 from one fused multiply-add residual), the kinetic energy is
// a pair (exact product errors, two-sums), E - Bh and the subtraction of
// the kinetic energy are two-sums, A = 1/(gamma-1) of the mixture is a pair
// like B, and the final division is corrected once by its residual.
// Velocities and the sound speed are plain float.
template <typename T, int MODEL, int NDIM>
__device__ __forceinline__ void cons2prim_stiff_float(const Dev &P, const T *U, T *W, T &rho_o, T &p_o,
                                                      T &rc2_o) {
    using V = Vars<MODEL, NDIM>;
    static_assert(sizeof(T) == 4, "float states only");
    T rh, rl = T(0);  // density as rh + rl
    if (MODEL == JXF_DIM) two_sum_f(U[0], U[1], rh, rl);
    else rh = U[0];
    const T ir = rcp(rh);
    T kh = T(0), kl = T(0);  // rho |u|^2 = kh + kl
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        const T m = U[V::NP + d];
        const T u0 = m * ir;
        // m - u0 rho exactly (to the small term u0 rl), then the correction
        const T r = __fsub_rn(__fmaf_rn(-u0, rh, m), u0 * rl);
        const T u1 = r * ir;
        W[V::NP + d] = u0;
        const T ph = __fmul_rn(m, u0);
        const T pe = __fmaf_rn(m, u0, -ph);
        T s, e;
        two_sum_f(kh, ph, s, e);
        kh = s;
        kl = __fadd_rn(kl, __fadd_rn(e, __fmaf_rn(m, u1, pe)));
    }
#pragma unroll
    for (int k = 0; k < V::NP; ++k) W[k] = U[k];
    const Cst<T> &C = cst<T>(P);
    T Ah, Al, Bh, Bl;  // A and B as pairs
    if (MODEL == JXF_DIM) {
        const T a1 = U[V::IA];
        T err;
        // A2 + a1 dA and B2 + a1 dB: the products' errors by fused multiply-add
        const T qh = __fmul_rn(a1, C.dAh);
        const T ql = __fmaf_rn(a1, C.dAl, __fmaf_rn(a1, C.dAh, -qh));
        two_sum_f(C.A2h, qh, Ah, err);
        Al = __fadd_rn(err, __fadd_rn(ql, C.A2l));
        const T ph = __fmul_rn(a1, C.dBh);
        const T pl = __fmaf_rn(a1, C.dBl, __fmaf_rn(a1, C.dBh, -ph));
        two_sum_f(C.B2h, ph, Bh, err);
        Bl = __fadd_rn(err, __fadd_rn(pl, C.B2l));
        W[V::IA] = a1;
    } else {
        Ah = C.A1h;
        Al = C.A1l;
        Bh = C.B1h;
        Bl = C.B1l;
    }
    const T invA = rcp(Ah);
    // rho e - B = (E - Bh) - rho|u|^2/2 - Bl with both large differences exact
    T s1, e1, s2, e2;
    two_sum_f(U[V::IE], -Bh, s1, e1);
    two_sum_f(s1, T(-0.5) * kh, s2, e2);
    const T lo = __fsub_rn(__fsub_rn(__fadd_rn(e1, e2), T(0.5) * kl), Bl);
    const T dif = __fadd_rn(s2, lo);
    // dif / (Ah + Al) with one residual correction
    const T p0 = dif * invA;
    const T p = __fmaf_rn(__fsub_rn(__fmaf_rn(-p0, Ah, dif), p0 * Al), invA, p0);
    W[V::IE] = p;
    rho_o = rh;
    p_o = p;
    rc2_o = p + (p + Bh) * invA;
}

// Per-block partials of the cell epilogue: [smax, rmin, bad, sums...] with
// the CFL maximum and the density minimum reduced in the storage type
// (exact) and the conservation sums in double (times the cell volume).
template <typename T, int NV, int NW = kCellThreads / 32>
__device__ __forceinline__ void block_partials(const Dev &P, T smax, T rmin, bool bad, const T *U,
                                               double *out) {
    __shared__ double sh[NW][3 + MAXV];  // NW >= blockDim.x / 32
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const T m = warp_max(smax), n = warp_min(rmin);
    const bool anybad = __any_sync(0xffffffffu, bad);
    double sums[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) sums[v] = warp_sum_to_double(U[v]);
    if (lane == 0) {
        sh[wid][0] = (double)m;
        sh[wid][1] = (double)n;
        sh[wid][2] = anybad ? 1.0 : 0.0;
#pragma unroll
        for (int v = 0; v < NV; ++v) sh[wid][3 + v] = sums[v];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        double a[3 + NV];
#pragma unroll
        for (int k = 0; k < 3 + NV; ++k) a[k] = sh[0][k];
        for (int w = 1; w < nw; ++w) {
            a[0] = fmax(a[0], sh[w][0]);
            a[1] = fmin(a[1], sh[w][1]);
            a[2] = fmax(a[2], sh[w][2]);
#pragma unroll
            for (int v = 0; v < NV; ++v) a[3 + v] += sh[w][3 + v];
        }
        double *o = out;
        o[0] = a[0];
        o[1] = a[1];
        o[2] = a[2];
#pragma unroll
        for (int v = 0; v < NV; ++v) o[3 + v] = a[3 + v] * P.vol;
    }
}

// Primitives (+ temperature) of one new cell state, and its CFL rate,
// density and admissibility for the epilogue.  Float storage recovers the
// stiffened-gas pressure in double (the cancellation of rho e - B); all else
// stays in the storage type.
template <typename T, int MODEL, int NDIM>
__device__ __forceinline__ void finish_cell(const Dev &P, long long i, const T *U, T &s_out,
                                            T &rho_out, bool &bad) {
    using V = Vars<MODEL, NDIM>;
    constexpr int NV = V::NV;
    T Wn[MAXV], rho, p, rc2;
    if constexpr (sizeof(T) == 4) {
        if (P.stiff) cons2prim_stiff_float<T, MODEL, NDIM>(P, U, Wn, rho, p, rc2);
        else cons2prim<T, T, MODEL, NDIM>(P, U, Wn, rho, p, rc2);
    } else {
        cons2prim<T, T, MODEL, NDIM>(P, U, Wn, rho, p, rc2);
    }
    T *Wo = static_cast<T *>(P.Wout);
    const size_t nc = (size_t)P.vstride;
    const int ic = (int)i;  // below 2^31 (checked at creation)
#pragma unroll
    for (int v = 0; v < NV; ++v) (Wo + v * nc)[ic] = Wn[v];
    // one reciprocal square root t = 1/(rho c): c = rho c^2 t, 1/rho = rho c^2 t^2
    const T t = rsq(rho * rc2);
    const T cs = rc2 * t;
    if (MODEL == JXF_SPM && P.viscous)
        static_cast<T *>(P.Tout)[ic] = p * (rc2 * t * t) * cst<T>(P).inv_R;  // T = p/(rho R)
    if constexpr (MODEL == JXF_DIM)
        if (P.thinc) (static_cast<T *>(P.G) + NDIM * nc)[ic] = thinc_psi(Wn[V::IA]);
    T s = T(0);
#pragma unroll
    for (int d = 0; d < NDIM; ++d) s += (fabs(Wn[V::NP + d]) + cs) * cst<T>(P).inv_dx[d];
    s_out = s;
    rho_out = rho;
    bool ok = (rho > T(0)) && (rc2 > T(0)) && isfinite(rho) && isfinite(p) && (s == s);
#pragma unroll
    for (int k = 0; k < V::NP; ++k) ok = ok && (U[k] > T(0));
    bad = !ok;
}

// --------------------------------------------------------------- k_update --
// The work of one cell i: divergence of the face fluxes (+ the a1 div(u)
// source), then mode 0: dU = R; mode 1: stage combination Uout = ca Un +
// cb Us + cc dt R and the new primitives, returning CFL rate, density and
// admissibility for the epilogue.  Shared by the single-grid and batched
// updates.
template <typename T, int MODEL, int NDIM>
__device__ __forceinline__ void update_cell(const Dev &P, T cdt, long long i, int mode, T *U,
                                            T &smax, T &rmin, bool &bad) {
    using V = Vars<MODEL, NDIM>;
    constexpr int NV = V::NV;
    const unsigned iu = (unsigned)i;
    const unsigned qy = P.fd_cell[0].div(iu), qz = P.fd_cell[1].div(qy);
    const int x = (int)(iu - qy * (unsigned)P.n[0]);
    const int y = (int)(qy - qz * (unsigned)P.n[1]);
    const int z = (int)qz;
    T R[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) R[v] = T(0);
    // cell and face indices stay below 2^31 (checked at creation): 32-bit
    // index arithmetic off warp-uniform field base pointers
    const size_t nc = (size_t)P.vstride;
    const int ic = (int)i;
    T a1 = T(0);
    if constexpr (MODEL == JXF_DIM) a1 = (static_cast<const T *>(P.Us) + V::IA * nc)[ic];
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        int m[3] = {P.n[0], P.n[1], P.n[2]};
        m[d] += 1;
        const size_t nface = (size_t)m[0] * m[1] * m[2];
        const int gm = chk_face(P, (z * m[1] + y) * m[0] + x, (long long)nface);
        const int gp = chk_face(P, gm + (d == 0 ? 1 : (d == 1 ? m[0] : m[0] * m[1])), (long long)nface);
        const T *F = static_cast<const T *>(P.F[d]);
        const T idx = cst<T>(P).inv_dx[d];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const T *Fv = F + v * nface;
            R[v] -= (__ldg(Fv + gp) - __ldg(Fv + gm)) * idx;
        }
        if (MODEL == JXF_DIM) {
            const T *UH = static_cast<const T *>(P.UH[d]);
            R[V::IA] += a1 * (__ldg(UH + gp) - __ldg(UH + gm)) * idx;
        }
    }
    if (mode == 0) {
        T *dU = static_cast<T *>(P.dU);
#pragma unroll
        for (int v = 0; v < NV; ++v) (dU + v * nc)[ic] = R[v];
        return;
    }
    const T *Un = static_cast<const T *>(P.Un);
    const T *Us = static_cast<const T *>(P.Us);
    T *Uo = static_cast<T *>(P.Uout);
    const bool first = P.stage0 != 0;  // stage 1: U1 = Un + dt R
    const T ca = first ? T(0) : (sizeof(T) == 8 ? T(P.ca) : T(P.ca32)), cb = sizeof(T) == 8 ? T(P.cb) : T(P.cb32);
    T un[MAXV], us[MAXV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {  // all loads before any store (Uout may alias)
        us[v] = (Us + v * nc)[ic];
        un[v] = first ? T(0) : (Un + v * nc)[ic];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        U[v] = first ? us[v] + cdt * R[v] : ca * un[v] + cb * us[v] + cdt * R[v];
        (Uo + v * nc)[ic] = U[v];
    }
    finish_cell<T, MODEL, NDIM>(P, i, U, smax, rmin, bad);
}

// c dt of the stage in the storage type, computed once per block.
template <typename T> __device__ __forceinline__ T block_cdt(const Dev &P, double dt) {
    __shared__ T s_c;
    if (threadIdx.x == 0) s_c = T(P.cc * dt);
    __syncthreads();
    return s_c;
}

template <typename T, int MODEL, int NDIM>
__global__ void __launch_bounds__(kCellThreads, CellMinBlocks<T>::value)
    k_update(const Dev P, const int mode, const int epi) {
    using V = Vars<MODEL, NDIM>;
    constexpr int NV = V::NV;
    double dt;
    if (!block_dt(P, dt)) return;
    const T cdt = block_cdt<T>(P, dt);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    T smax = T(0), rmin = T(3e38), U[MAXV];
    bool bad = false;
#pragma unroll
    for (int v = 0; v < NV; ++v) U[v] = T(0);
    if (i < P.ncell) update_cell<T, MODEL, NDIM>(P, cdt, i, mode, U, smax, rmin, bad);
    if (mode == 1 && epi)
        block_partials<T, NV>(P, smax, rmin, bad, U, P.part + (size_t)blockIdx.x * (3 + MAXV));
}

// ------------------------------------------- fused last-axis sweep ------
// The faces of the last axis d = NDIM-1 and the cell update of one RK stage
// in one kernel (float storage).  Each thread owns one column of cells along
// d (an x, or (x, y) in 3-D; a warp covers consecutive x) over a run of
// `run` cells, and marches up it: face c, then -- with the face below still
// in registers -- the update of cell c-1: the divergence of the other axes'
// face arrays and of the two faces along d, in the order of update_cell (so
// the result is bit for bit the unfused one), the RK stage combination, the
// new primitives and the epilogue.  The face array of axis d is never
// stored; a run computes one face more than it owns cells (the face it
// shares with the run above, counted there).  The stage reads W / Tt / Ucell
// and writes Wout / Tout / Uout, which must not alias them (the runs above
// and below still read the stencil cells).
template <typename T, int RSV> struct FusedMinBlocks { static constexpr int value = 7; };  // 72 registers
template <typename T> struct FusedMinBlocks<T, 2> { static constexpr int value = 4; };     // TENO6-A: 128

template <typename T, int MODEL, int NDIM, int VH, int RSV>
__global__ void __launch_bounds__(kFluxThreads, FusedMinBlocks<T, RSV>::value)
    k_flux_update(const Dev P, const int epi, const int run) {
    using V = Vars<MODEL, NDIM>;
    constexpr int NV = V::NV, d = NDIM - 1;
    __shared__ float s_hi[NV][kFluxThreads], s_lo[NV][kFluxThreads];  // conservation sums per thread
    double dt;
    if (!block_dt(P, dt)) return;
    const T cdt = block_cdt<T>(P, dt);
    const unsigned plane = NDIM == 3 ? (unsigned)(P.n[0] * P.n[1]) : (unsigned)P.n[0];
    const unsigned col = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = col < plane;
    const unsigned qy = P.fd_cell[0].div(col);
    int c[3] = {(int)(col - qy * (unsigned)P.n[0]), NDIM == 3 ? (int)qy : 0, 0};
    const int nd = P.n[d];
    const int d0 = (int)blockIdx.y * run, d1 = min(nd, d0 + run);
    const size_t nc = (size_t)P.vstride;
    const int sd = NDIM == 3 ? P.n[0] * P.n[1] : P.n[0];
    const int ic0 = (int)col;  // cell (x, y, 0)
    T smax = T(0), rmin = T(3e38);
    bool bad = false;
#pragma unroll
    for (int v = 0; v < NV; ++v) s_hi[v][threadIdx.x] = s_lo[v][threadIdx.x] = 0.f;
    T Fm[MAXV], uhm = T(0);
#pragma unroll
    for (int v = 0; v < NV; ++v) Fm[v] = T(0);
#pragma unroll 1
    for (int f = d0; f <= d1; ++f) {
        c[d] = f;
        T F[MAXV], uh = T(0);
        bool il = false, fl = false;
        if (active) flux_face_at<T, MODEL, NDIM, d, VH, RSV>(P, dt, c, f < d1 || d1 == nd, F, uh, il, fl);
        if (P.limiter) count_limited(P, il, fl);
        if (active && f > d0) {  // cell f-1 between the faces Fm (below) and F (above)
            const int z = f - 1;
            const int ic = chk_cell(P, ic0 + z * sd);
            const int x = c[0], y = NDIM == 3 ? c[1] : z, zz = NDIM == 3 ? z : 0;
            T R[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) R[v] = T(0);
            T a1 = T(0);
            if constexpr (MODEL == JXF_DIM) a1 = (static_cast<const T *>(P.Us) + V::IA * nc)[ic];
#pragma unroll
            for (int e = 0; e < NDIM; ++e) {
                const T idx = cst<T>(P).inv_dx[e];
                if (e < d) {
                    int m[3] = {P.n[0], P.n[1], P.n[2]};
                    m[e] += 1;
                    const size_t nface = (size_t)m[0] * m[1] * m[2];
                    const int gm = chk_face(P, (zz * m[1] + y) * m[0] + x, (long long)nface);
                    const int gp = chk_face(P, gm + (e == 0 ? 1 : m[0]), (long long)nface);
                    const T *Fe = static_cast<const T *>(P.F[e]);
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        const T *Fv = Fe + v * nface;
                        R[v] -= (__ldg(Fv + gp) - __ldg(Fv + gm)) * idx;
                    }
                    if (MODEL == JXF_DIM) {
                        const T *UH = static_cast<const T *>(P.UH[e]);
                        R[V::IA] += a1 * (__ldg(UH + gp) - __ldg(UH + gm)) * idx;
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < NV; ++v) R[v] -= (F[v] - Fm[v]) * idx;
                    if constexpr (MODEL == JXF_DIM) R[V::IA] += a1 * (uh - uhm) * idx;
                }
            }
            const T *Un = static_cast<const T *>(P.Un);
            const T *Us = static_cast<const T *>(P.Us);
            T *Uo = static_cast<T *>(P.Uout);
            const bool first = P.stage0 != 0;  // stage 1: U1 = Un + dt R
            const T ca = first ? T(0) : T(P.ca32), cb = T(P.cb32);
            T U[MAXV], un[MAXV], us[MAXV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                us[v] = (Us + v * nc)[ic];
                un[v] = first ? T(0) : (Un + v * nc)[ic];
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                U[v] = first ? us[v] + cdt * R[v] : ca * un[v] + cb * us[v] + cdt * R[v];
                (Uo + v * nc)[ic] = U[v];
            }
            T s1, r1;
            bool b1;
            finish_cell<T, MODEL, NDIM>(P, ic, U, s1, r1, b1);
            if (epi) {
                smax = tmax(smax, s1);
                rmin = tmin(rmin, r1);
                bad = bad || b1;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    float hs, e;
                    two_sum_f(s_hi[v][threadIdx.x], U[v], hs, e);
                    s_hi[v][threadIdx.x] = hs;
                    s_lo[v][threadIdx.x] = __fadd_rn(s_lo[v][threadIdx.x], e);
                }
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) Fm[v] = F[v];
        uhm = uh;
    }
    if (!epi) return;
    // per-block partials: [smax, rmin, bad, sums...] (sums times the cell volume)
    __shared__ double sh[kFluxThreads / 32][3 + MAXV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const T m = warp_max(smax), n = warp_min(rmin);
    const bool anybad = __any_sync(0xffffffffu, bad);
    double sums[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) sums[v] = warp_sum_pairs_to_double(s_hi[v][threadIdx.x], s_lo[v][threadIdx.x]);
    if (lane == 0) {
        sh[wid][0] = (double)m;
        sh[wid][1] = (double)n;
        sh[wid][2] = anybad ? 1.0 : 0.0;
#pragma unroll
        for (int v = 0; v < NV; ++v) sh[wid][3 + v] = sums[v];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a[3 + NV];
#pragma unroll
        for (int k = 0; k < 3 + NV; ++k) a[k] = sh[0][k];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            a[0] = fmax(a[0], sh[w][0]);
            a[1] = fmin(a[1], sh[w][1]);
            a[2] = fmax(a[2], sh[w][2]);
#pragma unroll
            for (int v = 0; v < NV; ++v) a[3 + v] += sh[w][3 + v];
        }
        double *o = P.part + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * (3 + MAXV);
        o[0] = a[0];
        o[1] = a[1];
        o[2] = a[2];
#pragma unroll
        for (int v = 0; v < NV; ++v) o[3 + v] = a[3 + v] * P.vol;
    }
}

// Primitives (+ temperature) of a conservative state, with the reduction
// epilogue (used after the state is set).
template <typename T, int MODEL, int NDIM>
__device__ __forceinline__ void prim_cell(const Dev &P, long long i, T *U, T &smax, T &rmin, bool &bad) {
    const T *Us = static_cast<const T *>(P.Us);
#pragma unroll
    for (int v = 0; v < Vars<MODEL, NDIM>::NV; ++v) U[v] = Us[v * P.vstride + i];
    finish_cell<T, MODEL, NDIM>(P, i, U, smax, rmin, bad);
}

template <typename T, int MODEL, int NDIM>
__global__ void __launch_bounds__(kCellThreads) k_prim(const Dev P, const int epi) {
    using V = Vars<MODEL, NDIM>;
    constexpr int NV = V::NV;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    T smax = T(0), rmin = T(3e38), U[MAXV];
    bool bad = false;
#pragma unroll
    for (int v = 0; v < NV; ++v) U[v] = T(0);
    if (i < P.ncell) prim_cell<T, MODEL, NDIM>(P, i, U, smax, rmin, bad);
    if (epi) block_partials<T, NV>(P, smax, rmin, bad, U, P.part + (size_t)blockIdx.x * (3 + MAXV));
}

// ------------------------------------------------------------- finalise ----
// Reduction of the partial records [begin, end) (max CFL rate, min density,
// admissibility flag, conservation sums) by one warp: strided records per
// lane (several in flight), then a shuffle tree -- a fixed order, so the
// result is deterministic.  One warp only: GB300's FP64 pipe does two
// operations per clock and SM, and a tree in every warp of a block costs
// more than the records themselves.  Valid in lane 0; all 32 lanes of the
// calling warp must call.
__device__ __forceinline__ void reduce_records(const double *part, int begin, int end, int nv,
                                               double (&a)[3 + MAXV]) {
    const int lane = threadIdx.x & 31;
    a[0] = -1e300;
    a[1] = 1e300;
    a[2] = 0.0;
#pragma unroll
    for (int v = 0; v < MAXV; ++v) a[3 + v] = 0.0;
#pragma unroll 4
    for (int b = begin + lane; b < end; b += 32) {
        const double *p = part + (size_t)b * (3 + MAXV);
        a[0] = fmax(a[0], p[0]);
        a[1] = fmin(a[1], p[1]);
        a[2] = fmax(a[2], p[2]);
#pragma unroll
        for (int v = 0; v < MAXV; ++v)
            if (v < nv) a[3 + v] += p[3 + v];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a[0] = fmax(a[0], __shfl_down_sync(0xffffffffu, a[0], o));
        a[1] = fmin(a[1], __shfl_down_sync(0xffffffffu, a[1], o));
        a[2] = fmax(a[2], __shfl_down_sync(0xffffffffu, a[2], o));
#pragma unroll
        for (int v = 0; v < MAXV; ++v)
            if (v < nv) a[3 + v] += __shfl_down_sync(0xffffffffu, a[3 + v], o);
    }
}

// First level of the reduction of many partial records (k_reduce_partials):
// GB300's FP64 rate per SM is low, so thousands of records are spread over
// kPartGroups blocks before the single-block finalisation.
constexpr int kPartGroups = 128;
constexpr int kPartThreads = 32;

// One block: deterministic reduction of npart per-block partials, then the
// time-step logic of §3.4: dt = CFL / max_cells sum_d (|u_d| + c)/dx_d,
// bounded by the viscous limit 3/14 rho_min dx_min^2/mu, or the fixed dt;
// clipped at t_end.  mode 0: partials -> diagnostics + dt; mode 1: the same
// after a step (advance t by the step's dt first); mode 2: re-clip dt from
// the stored diagnostics (after the time was set).
constexpr int kFinalThreads = 32;
__device__ __forceinline__ void finalize_block(const Dev &P, const double *part, int npart, int nv,
                                               int mode) {
    const int t = threadIdx.x;
    double *sc = P.scal;
    const double dt_cur = sc[SC_DT];
    if (mode == 1 && !(dt_cur > 0.0)) return;  // finished: the step did nothing
    double a[3 + MAXV];
    if (mode != 2 && t < 32) reduce_records(part, 0, npart, nv, a);
    if (t != 0) return;
    if (mode != 2) {
        sc[SC_SMAX] = a[0];
        sc[SC_RMIN] = a[1];
        for (int v = 0; v < nv; ++v) sc[SC_SUMS + v] = a[3 + v];
        if (a[2] > 0.0) *P.status |= ST_NONPHYSICAL;
    }
    if (mode == 1) {
        sc[SC_T] += dt_cur;
        sc[SC_DT_LAST] = dt_cur;
    }
    const double smax = sc[SC_SMAX], rmin = sc[SC_RMIN];
    double dt;
    if (P.fixed_dt > 0.0) {
        dt = P.fixed_dt;
    } else {
        dt = P.cfl / smax;
        if (P.viscous && P.mu > 0.0) {
            const double dtv = P.cfl * (3.0 / 14.0) * rmin * P.dx_min * P.dx_min / P.mu;
            dt = dtv < dt ? dtv : dt;
        }
    }
    if (P.t_end > 0.0) {
        const double rem = P.t_end - sc[SC_T];
        if (rem <= 1e-12 * P.t_end) dt = 0.0;
        else dt = rem < dt ? rem : dt;
    }
    if (!(dt >= 0.0) || isinf(dt)) {
        *P.status |= ST_BAD_DT;
        dt = 0.0;
    }
    sc[SC_DT] = dt;
}

// Primitive (double, host layout) -> conservative state in storage type.
template <typename T, int MODEL, int NDIM>
__global__ void __launch_bounds__(kCellThreads) k_from_prim(const Dev P, const double *__restrict__ W64) {
    using V = Vars<MODEL, NDIM>;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.ncell) return;
    double w[MAXV], u[MAXV], rc2;
#pragma unroll
    for (int v = 0; v < V::NV; ++v) w[v] = W64[v * P.ncell + i];
    prim2cons<double, MODEL, NDIM>(P, w, u, rc2);
    T *Uo = static_cast<T *>(P.Uout);
#pragma unroll
    for (int v = 0; v < V::NV; ++v) Uo[v * P.vstride + i] = T(u[v]);
}

}  // namespace jxf
