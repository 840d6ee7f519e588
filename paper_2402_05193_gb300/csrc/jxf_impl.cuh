// jxf_impl.cuh -- device code of the GB300 finite-volume solver.
//
// Kernels (one RK stage = ndim face sweeps + one cell update):
//   k_flux<d>   one thread per face of axis d: gathers the 6-cell stencil of
//               primitives (boundary conditions resolved by index mapping),
//               WENO5-JS (component or characteristic), interpolation
//               limiter, HLLC + upwinded face velocity, flux limiter,
//               4th-order viscous flux; writes F = F^c - F^d per face.
//   k_update    one thread per cell: divergence of the face fluxes and the
//               diffuse-interface source, RK3 stage combination (or the bare
//               right-hand side), primitives + temperature of the new state,
//               and in the last stage the CFL rate, minimum density,
//               conservation sums and admissibility, reduced per block.
//   k_finalize  one block: deterministic reduction of the block partials,
//               time advance, next dt (CFL, viscous bound, t_end clip),
//               status word.
//   k_from_prim primitive (FP64) -> conservative state in storage precision.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "jxf.h"

namespace jxf {

constexpr int MAXV = 7;
constexpr int kFluxThreads = 128;
constexpr int kCellThreads = 256;
constexpr int kFinalThreads = 512;

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

enum { ST_NONPHYSICAL = 1, ST_BAD_DT = 2 };

// Everything a kernel needs, passed by value.
struct Dev {
    int n[3];
    int bc[3][2];
    long long ncell;
    double inv_dx[3];
    double vol;
    // EOS: per fluid A = 1/(gamma-1), B = gamma pinf/(gamma-1); single-phase
    // shortcuts gm1 = gamma-1, gamma, pinf, gpinf = gamma pinf
    double A1, A2, B1, B2;
    double gamma0, pinf0, gm1_0, gpinf0;
    int stiff;  // p_inf != 0 somewhere: mixed precision recovers p in double
    double mu, lam_heat, R;
    double c24[3], c12[3];  // 1/(24 dx), 1/(12 dx)
    // scheme
    int recon, viscous, limiter;
    double eps_rho, eps_rhoc2, eps_alpha, weno_eps;
    double cfl, fixed_dt, t_end, visc_dt_coef;
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
    void *dU;           // right-hand side output (rhs mode)
    double ca, cb, cc;  // Uout = ca Un + cb Us + cc dt R
    const double *dtp;  // dt read by the kernels
    int skip_if_done;   // return at once when *dtp == 0 (steps past t_end)
    double *scal;       // scalar slots
    double *part;       // per-block partials: [blk][2 + nv]
    int *status;
    unsigned long long *counters;  // [0] IL sides, [1] FL faces
};

template <int MODEL, int NDIM> struct Vars {
    static constexpr int NP = (MODEL == JXF_DIM) ? 2 : 1;
    static constexpr int IE = NP + NDIM;
    static constexpr int IA = (MODEL == JXF_DIM) ? IE + 1 : -1;
    static constexpr int NV = IE + 1 + ((MODEL == JXF_DIM) ? 1 : 0);
};

// ------------------------------------------------------------ helpers -----
template <typename T> __device__ __forceinline__ T dsqrt(T x);
template <> __device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }
// correctly rounded reciprocal
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
template <typename T> __device__ __forceinline__ T tmin(T a, T b) { return b < a ? b : a; }
template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return b > a ? b : a; }

// Boundary conditions by index mapping (§3.1): periodic wrap, zero-gradient
// copy of the boundary cell, symmetry mirror (the velocity component of the
// mirrored axis changes sign: bit e of *mir flips).
__device__ __forceinline__ int map_axis(int c, int n, int blo, int bhi, int &mir, int bit) {
    if (c < 0) {
        if (blo == JXF_BC_PERIODIC) return c + n;
        if (blo == JXF_BC_ZEROGRAD) return 0;
        mir ^= bit;
        return -1 - c;
    }
    if (c >= n) {
        if (bhi == JXF_BC_PERIODIC) return c - n;
        if (bhi == JXF_BC_ZEROGRAD) return n - 1;
        mir ^= bit;
        return 2 * n - 1 - c;
    }
    return c;
}

template <int NDIM>
__device__ __forceinline__ long long cell_at(const Dev &P, int x, int y, int z, int &mir) {
    mir = 0;
    x = map_axis(x, P.n[0], P.bc[0][0], P.bc[0][1], mir, 1);
    if (NDIM > 1) y = map_axis(y, P.n[1], P.bc[1][0], P.bc[1][1], mir, 2);
    if (NDIM > 2) z = map_axis(z, P.n[2], P.bc[2][0], P.bc[2][1], mir, 4);
    return ((long long)z * P.n[1] + y) * P.n[0] + x;
}

// Load the primitive vector of a (possibly halo) cell.
template <typename T, int MODEL, int NDIM>
__device__ __forceinline__ void load_prim(const Dev &P, const T *__restrict__ W, int x, int y,
                                          int z, T *w) {
    using V = Vars<MODEL, NDIM>;
    int mir;
    const long long i = cell_at<NDIM>(P, x, y, z, mir);
#pragma unroll
    for (int v = 0; v < V::NV; ++v) w[v] = __ldg(W + v * P.ncell + i);
#pragma unroll
    for (int e = 0; e < NDIM; ++e)
        if (mir & (1 << e)) w[V::NP + e] = -w[V::NP + e];
}

// ---------------------------------------------------------------- EOS -----
// Stiffened-gas mixture (§2.4) in the form A = 1/(gamma-1),
// B = gamma p_inf/(gamma-1):  rho e = A p + B,  p = (rho e - B)/A,
// rho c^2 = gamma (p + p_inf) = p + (p + B)/A.
template <typename T, int MODEL> struct Eos {
    T A, B, invA;
    __device__ __forceinline__ Eos(const Dev &P, T a1) {
        if (MODEL == JXF_SPM) {
            A = T(P.A1);
            B = T(P.B1);
            invA = T(P.gm1_0);
        } else {
            const T a2 = T(1) - a1;
            A = a1 * T(P.A1) + a2 * T(P.A2);
            B = a1 * T(P.B1) + a2 * T(P.B2);
            invA = T(1) / A;
        }
    }
    __device__ __forceinline__ T rhoe_from_p(const Dev &P, T p) const {
        if (MODEL == JXF_SPM) return (p + T(P.gpinf0)) * A;
        return A * p + B;
    }
    __device__ __forceinline__ T p_from_rhoe(const Dev &P, T rhoe) const {
        if (MODEL == JXF_SPM) return T(P.gm1_0) * rhoe - T(P.gpinf0);
        return (rhoe - B) * invA;
    }
    __device__ __forceinline__ T rc2_from_p(const Dev &P, T p) const {
        if (MODEL == JXF_SPM) return T(P.gamma0) * (p + T(P.pinf0));
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
    const C ir = C(1) / rho;
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

// ------------------------------------------------------------ WENO5-JS ----
// Left-biased value at x_{i+1/2} from v_{i-2..i+2} (§3.2 step 3): Jiang-Shu
// candidates on S0, S1, S2, smoothness indicators, weights d_k/(eps+beta_k)^2
// normalised.  Double precision folds the three weight divisions into one
// (alpha_k q0^2 q1^2 q2^2); float keeps one reciprocal per weight so that
// large beta cannot overflow.
template <typename T>
__device__ __forceinline__ T weno5(T a, T b, T c, T d, T e, T eps) {
    const T p0 = (T(2) * a - T(7) * b + T(11) * c) * T(1.0 / 6.0);
    const T p1 = (-b + T(5) * c + T(2) * d) * T(1.0 / 6.0);
    const T p2 = (T(2) * c + T(5) * d - e) * T(1.0 / 6.0);
    const T s0a = a - T(2) * b + c, s0b = a - T(4) * b + T(3) * c;
    const T s1a = b - T(2) * c + d, s1b = b - d;
    const T s2a = c - T(2) * d + e, s2b = T(3) * c - T(4) * d + e;
    const T q0 = eps + T(13.0 / 12.0) * s0a * s0a + T(0.25) * s0b * s0b;
    const T q1 = eps + T(13.0 / 12.0) * s1a * s1a + T(0.25) * s1b * s1b;
    const T q2 = eps + T(13.0 / 12.0) * s2a * s2a + T(0.25) * s2b * s2b;
    T w0, w1, w2;
    if (sizeof(T) == 8) {
        const T z0 = q0 * q0, z1 = q1 * q1, z2 = q2 * q2;
        w0 = T(0.1) * (z1 * z2);
        w1 = T(0.6) * (z0 * z2);
        w2 = T(0.3) * (z0 * z1);
    } else {
        const T r0 = rcp(q0), r1 = rcp(q1), r2 = rcp(q2);
        w0 = T(0.1) * r0 * r0;
        w1 = T(0.6) * r1 * r1;
        w2 = T(0.3) * r2 * r2;
    }
    return (w0 * p0 + w1 * p1 + w2 * p2) / (w0 + w1 + w2);
}

// ------------------------------------------------------ reconstruction ----
// Face states of face i+1/2 from the stencil S[j] = W_{i-2+j}, j = 0..5.
// Characteristic mode (§3.2 steps 1-4, App. C.1): frozen state = mean of
// W_i and W_{i+1}; K^{-1} rows: acoustic (-/+ u_n/(2c) + p/(2 rho c^2)),
// entropy / partial densities (X_k - X_k_bar p/(rho c^2)), identity for the
// shear velocities and the volume fraction; back-projection with K.
template <typename T, int MODEL, int NDIM, int d>
__device__ __forceinline__ void reconstruct(const Dev &P, const T (&S)[6][MAXV], T *WL, T *WR) {
    using V = Vars<MODEL, NDIM>;
    constexpr int NV = V::NV, NP = V::NP, IE = V::IE;
    const T eps = T(P.weno_eps);
    if (P.recon == JXF_WENO5JS_COMP) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            WL[v] = weno5(S[0][v], S[1][v], S[2][v], S[3][v], S[4][v], eps);
            WR[v] = weno5(S[5][v], S[4][v], S[3][v], S[2][v], S[1][v], eps);
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
    const T irc2 = T(1) / rc2;
    const T cb = dsqrt(rc2 / rho);
    const T h_c = T(0.5) / cb;
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
        qL[v] = weno5(q[0], q[1], q[2], q[3], q[4], eps);
        qR[v] = weno5(q[5], q[4], q[3], q[2], q[1], eps);
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

// ------------------------------------------------------------ limiters ----
// Interpolation limiter of one face side (§3.3 item 1): partial densities,
// volume fraction outside [eps_a, 1 - eps_a], rho c^2 -- any violation puts
// back the first-order (cell) state.  Returns 1 if switched.
template <typename T, int MODEL, int NDIM>
__device__ __forceinline__ int interp_limit(const Dev &P, T *Wf, const T *W1) {
    using V = Vars<MODEL, NDIM>;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < V::NP; ++k) bad |= Wf[k] < T(P.eps_rho);
    if (MODEL == JXF_DIM)
        bad |= (Wf[V::IA] < T(P.eps_alpha)) | (Wf[V::IA] > T(1.0 - P.eps_alpha));
    if (!bad) {
        Eos<T, MODEL> eos(P, alpha_of<T, MODEL, NDIM>(Wf));
        bad = eos.rc2_from_p(P, Wf[V::IE]) < T(P.eps_rhoc2);
    }
    if (bad) {
#pragma unroll
        for (int v = 0; v < V::NV; ++v) Wf[v] = W1[v];
    }
    return bad ? 1 : 0;
}

// ---------------------------------------------------------------- HLLC ----
// One branch of the HLLC flux (§3.2 step 6): F^K + s^{-/+} (U^{*K} - U^K) and
// the matching upwinded normal velocity.
template <typename T, int MODEL, int NDIM, int d>
__device__ __forceinline__ void hllc_branch(const Dev &P, const T *W, T sK, T sPM, T sstar, T *F,
                                            T &uh) {
    using V = Vars<MODEL, NDIM>;
    constexpr int NP = V::NP, IE = V::IE;
    constexpr int in = NP + d;
    T U[MAXV], rc2;
    prim2cons<T, MODEL, NDIM>(P, W, U, rc2);
    const T rho = density_of<T, MODEL, NDIM>(W);
    const T u = W[in], p = W[IE];
    const T su = sK - u;
    const T fac = su / (sK - sstar);
    T Us[MAXV];
#pragma unroll
    for (int k = 0; k < NP; ++k) Us[k] = fac * U[k];
#pragma unroll
    for (int e = 0; e < NDIM; ++e) Us[NP + e] = fac * (rho * W[NP + e]);
    Us[in] = fac * (rho * sstar);
    Us[IE] = fac * (U[IE] + (sstar - u) * (rho * sstar + p / su));
    if (MODEL == JXF_DIM) Us[V::IA] = fac * W[V::IA];
    // physical flux
    T Fp[MAXV];
#pragma unroll
    for (int k = 0; k < NP; ++k) Fp[k] = U[k] * u;
#pragma unroll
    for (int e = 0; e < NDIM; ++e) Fp[NP + e] = U[NP + e] * u;
    Fp[in] += p;
    Fp[IE] = u * (U[IE] + p);
    if (MODEL == JXF_DIM) Fp[V::IA] = W[V::IA] * u;
#pragma unroll
    for (int v = 0; v < V::NV; ++v) F[v] = Fp[v] + sPM * (Us[v] - U[v]);
    uh = u + sPM * (fac - T(1));
}

// HLLC flux and upwinded face velocity from primitive face states (§3.2
// step 6, App. C.2): Einfeldt s^L, s^R with sqrt(rho)-weighted averages,
// Batten s*, sign(s*) selecting one branch (the mean of both at s* = 0).
template <typename T, int MODEL, int NDIM, int d>
__device__ __forceinline__ void hllc(const Dev &P, const T *WL, const T *WR, T *F, T &uh) {
    using V = Vars<MODEL, NDIM>;
    constexpr int NP = V::NP, IE = V::IE;
    constexpr int in = NP + d;
    const T rhoL = density_of<T, MODEL, NDIM>(WL), rhoR = density_of<T, MODEL, NDIM>(WR);
    const T uL = WL[in], uR = WR[in], pL = WL[IE], pR = WR[IE];
    Eos<T, MODEL> eL(P, alpha_of<T, MODEL, NDIM>(WL)), eR(P, alpha_of<T, MODEL, NDIM>(WR));
    const T c2L = eL.rc2_from_p(P, pL) / rhoL;
    const T c2R = eR.rc2_from_p(P, pR) / rhoR;
    const T cL = dsqrt(c2L), cR = dsqrt(c2R);
    const T srL = dsqrt(rhoL), srR = dsqrt(rhoR);
    const T is = T(1) / (srL + srR);
    const T ubar = (srL * uL + srR * uR) * is;
    const T du = uR - uL;
    const T c2bar = (srL * c2L + srR * c2R) * is + T(0.5) * (srL * srR) * (is * is) * (du * du);
    const T cbar = dsqrt(c2bar);
    const T sL = tmin(ubar - cbar, uL - cL);
    const T sR = tmax(ubar + cbar, uR + cR);
    const T mL = rhoL * (sL - uL), mR = rhoR * (sR - uR);
    const T sstar = (pR - pL + mL * uL - mR * uR) / (mL - mR);
    const T sm = tmin(T(0), sL), sp = tmax(T(0), sR);
    const bool left = !(sstar < T(0));
    hllc_branch<T, MODEL, NDIM, d>(P, left ? WL : WR, left ? sL : sR, left ? sm : sp, sstar, F, uh);
    if (sstar == T(0)) {  // sign(s*) = 0: mean of both branches
        T F2[MAXV], u2;
        hllc_branch<T, MODEL, NDIM, d>(P, WR, sR, sp, sstar, F2, u2);
#pragma unroll
        for (int v = 0; v < V::NV; ++v) F[v] = T(0.5) * F[v] + T(0.5) * F2[v];
        uh = T(0.5) * uh + T(0.5) * u2;
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
        for (int k = 0; k < V::NP; ++k) bad |= Ts[k] < T(P.eps_rho);
        if (MODEL == JXF_DIM)
            bad |= (Ts[V::IA] < T(P.eps_alpha)) | (Ts[V::IA] > T(1.0 - P.eps_alpha));
        if (!bad) {
            T W[MAXV], rho, p, rc2;
            cons2prim<T, T, MODEL, NDIM>(P, Ts, W, rho, p, rc2);
            bad = rc2 < T(P.eps_rhoc2);
        }
    }
    return bad;
}

// ---------------------------------------------------------- viscous flux --
// F^d on face i+1/2 of axis d (§2.1): tau_dk and the heat flux from
// 4th-order central stencils -- normal derivative (1,-27,27,-1)/(24 dx),
// face value (-1,9,9,-1)/16, tangential derivative (1,-8,8,-1)/(12 dy) at
// cells i-1..i+2 interpolated to the face.  Only du_d/dx_e and du_e/dx_e are
// needed along a tangential axis e.
template <typename T, int NDIM, int d>
__device__ __forceinline__ void viscous_flux(const Dev &P, int x, int y, int z, T *Fd) {
    const T *W = static_cast<const T *>(P.W);
    const T *Tt = static_cast<const T *>(P.Tt);
    int c[3] = {x, y, z};
    T g[NDIM + 1][3];  // g[f][e]: d phi_f / d x_e at the face (phi = u_0.., T)
    T fu[NDIM];
    // normal direction: cells i-1..i+2 = face coordinate - 2 .. + 1
#pragma unroll
    for (int f = 0; f <= NDIM; ++f) {
        T v[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            int q[3] = {c[0], c[1], c[2]};
            q[d] += m - 2;
            int mir;
            const long long i = cell_at<NDIM>(P, q[0], q[1], q[2], mir);
            if (f < NDIM) {
                T u = __ldg(W + (1 + f) * P.ncell + i);
                v[m] = (mir & (1 << f)) ? -u : u;
            } else {
                v[m] = __ldg(Tt + i);
            }
        }
        g[f][d] = (v[0] - T(27) * v[1] + T(27) * v[2] - v[3]) * T(P.c24[d]);
        if (f < NDIM) fu[f] = (-v[0] + T(9) * v[1] + T(9) * v[2] - v[3]) * T(1.0 / 16.0);
    }
#pragma unroll
    for (int e = 0; e < NDIM; ++e) {
        if (e == d) continue;
#pragma unroll
        for (int which = 0; which < 2; ++which) {
            const int f = which == 0 ? d : e;
            T gm[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                T s[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    int q[3] = {c[0], c[1], c[2]};
                    q[d] += m - 2;
                    q[e] += (k < 2) ? k - 2 : k - 1;  // -2, -1, +1, +2
                    int mir;
                    const long long i = cell_at<NDIM>(P, q[0], q[1], q[2], mir);
                    const T u = __ldg(W + (1 + f) * P.ncell + i);
                    s[k] = (mir & (1 << f)) ? -u : u;
                }
                gm[m] = (s[0] - T(8) * s[1] + T(8) * s[2] - s[3]) * T(P.c12[e]);
            }
            g[f][e] = (-gm[0] + T(9) * gm[1] + T(9) * gm[2] - gm[3]) * T(1.0 / 16.0);
        }
    }
    T div = g[0][0];
#pragma unroll
    for (int k = 1; k < NDIM; ++k) div += g[k][k];
    const T mu = T(P.mu);
    T work = T(0);
    Fd[0] = T(0);
#pragma unroll
    for (int k = 0; k < NDIM; ++k) {
        T tau = mu * (g[d][k] + g[k][d]);
        if (k == d) tau -= T(2.0 / 3.0) * mu * div;
        Fd[1 + k] = tau;
        work += fu[k] * tau;
    }
    Fd[1 + NDIM] = work + T(P.lam_heat) * g[NDIM][d];  // - q_d = + lambda dT/dx_d
}

// ---------------------------------------------------------------- k_flux --
template <typename T, int MODEL, int NDIM, int d>
__global__ void __launch_bounds__(kFluxThreads) k_flux(const Dev P) {
    using V = Vars<MODEL, NDIM>;
    constexpr int NV = V::NV;
    const double dt = *P.dtp;
    if (P.skip_if_done && !(dt > 0.0)) return;
    int m[3] = {P.n[0], P.n[1], P.n[2]};
    m[d] += 1;
    const long long nface = (long long)m[0] * m[1] * m[2];
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool il_hit = false, fl_hit = false;
    if (g < nface) {
        int c[3];
        c[0] = (int)(g % m[0]);
        const long long r = g / m[0];
        c[1] = (int)(r % m[1]);
        c[2] = (int)(r / m[1]);
        // face c[d] lies between cells c[d]-1 (i) and c[d] (i+1)
        const T *W = static_cast<const T *>(P.W);
        T S[6][MAXV];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            int q[3] = {c[0], c[1], c[2]};
            q[d] += j - 3;
            load_prim<T, MODEL, NDIM>(P, W, q[0], q[1], q[2], S[j]);
        }
        T WL[MAXV], WR[MAXV];
        reconstruct<T, MODEL, NDIM, d>(P, S, WL, WR);
        if (P.limiter) {
            int k = interp_limit<T, MODEL, NDIM>(P, WL, S[2]);
            k += interp_limit<T, MODEL, NDIM>(P, WR, S[3]);
            il_hit = k != 0;
            if (k == 2) atomicAdd(P.counters, 1ull);  // count the extra side
        }
        T F[MAXV], uh;
        hllc<T, MODEL, NDIM, d>(P, WL, WR, F, uh);
        if (P.limiter) {
            T Ui[MAXV], Uj[MAXV];
            const T *Uc = static_cast<const T *>(P.Ucell);
            int q[3] = {c[0], c[1], c[2]};
            q[d] -= 1;
            int mir;
            const long long ii = cell_at<NDIM>(P, q[0], q[1], q[2], mir);
            const int mi = mir;
            const long long jj = cell_at<NDIM>(P, c[0], c[1], c[2], mir);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                Ui[v] = __ldg(Uc + v * P.ncell + ii);
                Uj[v] = __ldg(Uc + v * P.ncell + jj);
            }
#pragma unroll
            for (int e = 0; e < NDIM; ++e) {
                if (mi & (1 << e)) Ui[V::NP + e] = -Ui[V::NP + e];
                if (mir & (1 << e)) Uj[V::NP + e] = -Uj[V::NP + e];
            }
            const T lam = T(P.fl_lam[d] * dt);
            if (flux_limit_violates<T, MODEL, NDIM>(P, lam, F, uh, Ui, Uj)) {
                hllc<T, MODEL, NDIM, d>(P, S[2], S[3], F, uh);
                fl_hit = true;
            }
        }
        if (MODEL == JXF_SPM && P.viscous) {
            T Fd[MAXV];
            viscous_flux<T, NDIM, d>(P, c[0], c[1], c[2], Fd);
#pragma unroll
            for (int v = 0; v < NV; ++v) F[v] -= Fd[v];
        }
        T *Fo = static_cast<T *>(P.F[d]);
#pragma unroll
        for (int v = 0; v < NV; ++v) Fo[v * nface + g] = F[v];
        if (MODEL == JXF_DIM) static_cast<T *>(P.UH[d])[g] = uh;
    }
    if (P.limiter) {
        const unsigned il = __popc(__ballot_sync(0xffffffffu, il_hit));
        const unsigned fl = __popc(__ballot_sync(0xffffffffu, fl_hit));
        if ((threadIdx.x & 31) == 0) {
            if (il) atomicAdd(P.counters, (unsigned long long)il);
            if (fl) atomicAdd(P.counters + 1, (unsigned long long)fl);
        }
    }
}

// -------------------------------------------------- block reductions -----
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Per-block partials of the cell epilogue: [smax, rmin, bad, sums...].
template <int NV>
__device__ __forceinline__ void block_partials(const Dev &P, double smax, double rmin, double bad,
                                               const double *sums) {
    __shared__ double sh[kCellThreads / 32][3 + MAXV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double vals[3 + NV];
    vals[0] = warp_max(smax);
    vals[1] = warp_min(rmin);
    vals[2] = warp_max(bad);
#pragma unroll
    for (int v = 0; v < NV; ++v) vals[3 + v] = warp_sum(sums[v]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 3 + NV; ++k) sh[wid][k] = vals[k];
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        double a[3 + NV];
#pragma unroll
        for (int k = 0; k < 3 + NV; ++k) a[k] = lane < nw ? sh[lane][k] : (k == 1 ? 1e300 : (k == 0 || k == 2 ? -1e300 : 0.0));
        a[0] = warp_max(a[0]);
        a[1] = warp_min(a[1]);
        a[2] = warp_max(a[2]);
#pragma unroll
        for (int v = 0; v < NV; ++v) a[3 + v] = warp_sum(a[3 + v]);
        if (lane == 0) {
            double *o = P.part + (size_t)blockIdx.x * (3 + MAXV);
#pragma unroll
            for (int k = 0; k < 3 + NV; ++k) o[k] = a[k];
        }
    }
}

// --------------------------------------------------------------- k_update --
// mode 0: dU = R(U) only.  mode 1: stage combination Uout = ca Un + cb Us +
// cc dt R, primitives of Uout; with epi = 1 also the reduction epilogue.
template <typename T, int MODEL, int NDIM>
__global__ void __launch_bounds__(kCellThreads) k_update(const Dev P, const int mode, const int epi) {
    using V = Vars<MODEL, NDIM>;
    constexpr int NV = V::NV;
    const double dt = *P.dtp;
    if (P.skip_if_done && !(dt > 0.0)) return;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double smax = -1e300, rmin = 1e300, bad = 0.0;
    double sums[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) sums[v] = 0.0;
    if (i < P.ncell) {
        const int x = (int)(i % P.n[0]);
        const long long r = i / P.n[0];
        const int y = (int)(r % P.n[1]);
        const int z = (int)(r / P.n[1]);
        T R[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) R[v] = T(0);
        T a1 = T(0);
        if (MODEL == JXF_DIM) a1 = static_cast<const T *>(P.Us)[V::IA * P.ncell + i];
#pragma unroll
        for (int d = 0; d < NDIM; ++d) {
            int m[3] = {P.n[0], P.n[1], P.n[2]};
            m[d] += 1;
            const long long nface = (long long)m[0] * m[1] * m[2];
            const long long gm = ((long long)z * m[1] + y) * m[0] + x;
            const long long gs = d == 0 ? 1 : (d == 1 ? (long long)m[0] : (long long)m[0] * m[1]);
            const T *F = static_cast<const T *>(P.F[d]);
            const T idx = T(P.inv_dx[d]);
#pragma unroll
            for (int v = 0; v < NV; ++v) R[v] -= (F[v * nface + gm + gs] - F[v * nface + gm]) * idx;
            if (MODEL == JXF_DIM) {
                const T *UH = static_cast<const T *>(P.UH[d]);
                R[V::IA] += a1 * (UH[gm + gs] - UH[gm]) * idx;
            }
        }
        if (mode == 0) {
            T *dU = static_cast<T *>(P.dU);
#pragma unroll
            for (int v = 0; v < NV; ++v) dU[v * P.ncell + i] = R[v];
        } else {
            const T *Un = static_cast<const T *>(P.Un);
            const T *Us = static_cast<const T *>(P.Us);
            T *Uo = static_cast<T *>(P.Uout);
            const T ca = T(P.ca), cb = T(P.cb), cdt = T(P.cc * dt);
            T U[MAXV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const T us = Us[v * P.ncell + i];
                U[v] = (P.ca != 0.0) ? ca * Un[v * P.ncell + i] + cb * us + cdt * R[v] : us + cdt * R[v];
                Uo[v * P.ncell + i] = U[v];
            }
            T Wn[MAXV];
            double rho, p, rc2;
            if (sizeof(T) == 4 && P.stiff) {
                cons2prim<double, T, MODEL, NDIM>(P, U, Wn, rho, p, rc2);
            } else {
                T rho_t, p_t, rc2_t;
                cons2prim<T, T, MODEL, NDIM>(P, U, Wn, rho_t, p_t, rc2_t);
                rho = rho_t;
                p = p_t;
                rc2 = rc2_t;
            }
            T *Wo = static_cast<T *>(P.Wout);
#pragma unroll
            for (int v = 0; v < NV; ++v) Wo[v * P.ncell + i] = Wn[v];
            if (MODEL == JXF_SPM && P.viscous)
                static_cast<T *>(P.Tout)[i] = T(p) / (T(rho) * T(P.R));
            if (epi) {
                const T cs = dsqrt(T(rc2) / T(rho));
                T s = T(0);
#pragma unroll
                for (int d = 0; d < NDIM; ++d) s += (fabs(Wn[V::NP + d]) + cs) * T(P.inv_dx[d]);
                smax = (double)s;
                rmin = rho;
                bool ok = (rho > 0.0) && (rc2 > 0.0) && isfinite(rho) && isfinite(p);
#pragma unroll
                for (int k = 0; k < V::NP; ++k) ok = ok && (U[k] > T(0));
                if (!ok || !(s == s)) bad = 1.0;
#pragma unroll
                for (int v = 0; v < NV; ++v) sums[v] = (double)U[v] * P.vol;
            }
        }
    }
    if (mode == 1 && epi) block_partials<NV>(P, smax, rmin, bad, sums);
}

// Primitives (+ temperature) of a conservative state, with the reduction
// epilogue (used after the state is set).
template <typename T, int MODEL, int NDIM>
__global__ void __launch_bounds__(kCellThreads) k_prim(const Dev P, const int epi) {
    using V = Vars<MODEL, NDIM>;
    constexpr int NV = V::NV;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double smax = -1e300, rmin = 1e300, bad = 0.0;
    double sums[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) sums[v] = 0.0;
    if (i < P.ncell) {
        const T *Us = static_cast<const T *>(P.Us);
        T U[MAXV], Wn[MAXV];
#pragma unroll
        for (int v = 0; v < NV; ++v) U[v] = Us[v * P.ncell + i];
        double rho, p, rc2;
        if (sizeof(T) == 4 && P.stiff) {
            cons2prim<double, T, MODEL, NDIM>(P, U, Wn, rho, p, rc2);
        } else {
            T rho_t, p_t, rc2_t;
            cons2prim<T, T, MODEL, NDIM>(P, U, Wn, rho_t, p_t, rc2_t);
            rho = rho_t;
            p = p_t;
            rc2 = rc2_t;
        }
        T *Wo = static_cast<T *>(P.Wout);
#pragma unroll
        for (int v = 0; v < NV; ++v) Wo[v * P.ncell + i] = Wn[v];
        if (MODEL == JXF_SPM && P.viscous)
            static_cast<T *>(P.Tout)[i] = T(p) / (T(rho) * T(P.R));
        if (epi) {
            const T cs = dsqrt(T(rc2) / T(rho));
            T s = T(0);
#pragma unroll
            for (int d = 0; d < NDIM; ++d) s += (fabs(Wn[V::NP + d]) + cs) * T(P.inv_dx[d]);
            smax = (double)s;
            rmin = rho;
            bool ok = (rho > 0.0) && (rc2 > 0.0) && isfinite(rho) && isfinite(p);
            if (!ok || !(s == s)) bad = 1.0;
#pragma unroll
            for (int v = 0; v < NV; ++v) sums[v] = (double)U[v] * P.vol;
        }
    }
    if (epi) block_partials<NV>(P, smax, rmin, bad, sums);
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
    for (int v = 0; v < V::NV; ++v) Uo[v * P.ncell + i] = T(u[v]);
}

}  // namespace jxf
