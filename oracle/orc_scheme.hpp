// orc_scheme.hpp -- the oracle's finite-volume scheme, templated on the scalar
// type (double for values, Dual for tangents, Counted for flop counts).
//
// Every routine follows one passage of the JAX-Fluids 2.0 paper (arXiv
// 2402.05193) and is written to be read against it: no blocking, fusion or
// reordering beyond what the paper states.  Where the paper is silent, the
// reading taken is stated at the routine.
//
// Test infrastructure only; shares nothing with the CUDA library.
#pragma once
#include <cstring>
#include <limits>
#include <type_traits>
#include <vector>

#include "orc.h"
#include "orc_types.hpp"

namespace orc {

constexpr int NVMAX = 7;
constexpr int NH = 3;  // halo width: WENO5 at face i+1/2 reads cells i-2..i+3

template <class T> constexpr bool kParallel = !std::is_same<T, Counted>::value;

// ------------------------------------------------------------------ layout --
// Variable order (§2.1, §2.3): single phase U = (rho, rho u_d, E),
// W = (rho, u_d, p); diffuse interface U = (a1 rho1, a2 rho2, rho u_d, E, a1),
// W = (a1 rho1, a2 rho2, u_d, p, a1).  Only the ndim active velocity
// components are carried.
struct Layout {
    int ndim, nv, np, ie, ia;
    int n[3], h[3], P[3];
    long ncell, npad;
    explicit Layout(const orc_config &c) {
        ndim = c.ndim;
        np = (c.model == ORC_DIM) ? 2 : 1;
        ie = np + ndim;
        ia = (c.model == ORC_DIM) ? ie + 1 : -1;
        nv = ie + 1 + (c.model == ORC_DIM ? 1 : 0);
        ncell = 1;
        npad = 1;
        for (int e = 0; e < 3; ++e) {
            n[e] = (e < ndim) ? c.n[e] : 1;
            h[e] = (e < ndim) ? NH : 0;
            P[e] = n[e] + 2 * h[e];
            ncell *= n[e];
            npad *= P[e];
        }
    }
    long cidx(int x, int y, int z) const { return ((long)z * n[1] + y) * n[0] + x; }
    long pidx(int x, int y, int z) const {
        return ((long)(z + h[2]) * P[1] + (y + h[1])) * P[0] + (x + h[0]);
    }
    long pstride(int e) const { return e == 0 ? 1 : (e == 1 ? P[0] : (long)P[0] * P[1]); }
};

// ---------------------------------------------------------------- EOS -------
template <class T> struct Mix { T gamma, pinf; };

// Mixture parameters of the stiffened gas (§2.4).  Single phase: the fluid's
// own (gamma, p_inf).  Diffuse interface: the isobaric closure
//   1/(gamma-1)            = a1/(g1-1) + (1-a1)/(g2-1)
//   gamma p_inf/(gamma-1)  = a1 g1 pinf1/(g1-1) + (1-a1) g2 pinf2/(g2-1).
template <class T> inline Mix<T> mixture(const orc_config &c, const T &a1) {
    if (c.model == ORC_SPM) return {T(c.gamma[0]), T(c.pinf[0])};
    const double g1 = c.gamma[0], g2 = c.gamma[1];
    const double k1 = g1 * c.pinf[0] / (g1 - 1.0), k2 = g2 * c.pinf[1] / (g2 - 1.0);
    T a2 = 1.0 - a1;
    T inv_gm1 = a1 / (g1 - 1.0) + a2 / (g2 - 1.0);
    T gpinf_gm1 = a1 * k1 + a2 * k2;
    T gamma = 1.0 + 1.0 / inv_gm1;
    T pinf = gpinf_gm1 / inv_gm1 / gamma;
    return {gamma, pinf};
}

template <class T> inline T density(const Layout &L, const T *X) {
    return L.np == 1 ? X[0] : X[0] + X[1];
}
template <class T> inline T alpha1(const Layout &L, const T *X) {
    return L.ia >= 0 ? X[L.ia] : T(0.0);
}

// U -> W (§2.1/§2.3 state vectors, §2.4 p = (gamma-1) rho e - gamma p_inf).
template <class T>
inline void cons2prim(const orc_config &c, const Layout &L, const T *U, T *W) {
    T rho = density(L, U);
    for (int k = 0; k < L.np; ++k) W[k] = U[k];
    for (int d = 0; d < L.ndim; ++d) W[L.np + d] = U[L.np + d] / rho;
    T uu = W[L.np] * W[L.np];
    for (int d = 1; d < L.ndim; ++d) uu = uu + W[L.np + d] * W[L.np + d];
    T rhoe = U[L.ie] - 0.5 * rho * uu;
    Mix<T> m = mixture(c, alpha1(L, U));
    W[L.ie] = (m.gamma - 1.0) * rhoe - m.gamma * m.pinf;
    if (L.ia >= 0) W[L.ia] = U[L.ia];
}

// W -> U, with rho e = (p + gamma p_inf)/(gamma - 1) from §2.4.
template <class T>
inline void prim2cons(const orc_config &c, const Layout &L, const T *W, T *U) {
    T rho = density(L, W);
    for (int k = 0; k < L.np; ++k) U[k] = W[k];
    for (int d = 0; d < L.ndim; ++d) U[L.np + d] = rho * W[L.np + d];
    T uu = W[L.np] * W[L.np];
    for (int d = 1; d < L.ndim; ++d) uu = uu + W[L.np + d] * W[L.np + d];
    Mix<T> m = mixture(c, alpha1(L, W));
    T rhoe = (W[L.ie] + m.gamma * m.pinf) / (m.gamma - 1.0);
    U[L.ie] = rhoe + 0.5 * rho * uu;
    if (L.ia >= 0) U[L.ia] = W[L.ia];
}

// rho c^2 = gamma (p + p_inf), the admissibility helper of §3.3.
template <class T> inline T rhoc2_of(const orc_config &c, const Layout &L, const T *W) {
    Mix<T> m = mixture(c, alpha1(L, W));
    return m.gamma * (W[L.ie] + m.pinf);
}

// ------------------------------------------------------------ WENO5 --------
// Candidate values and smoothness indicators for the value at x_{i+1/2} from
// the left, from the cell averages v_{i-2..i+2} (§3.2 step 3; Jiang & Shu
// candidate polynomials on S0={i-2,i-1,i}, S1={i-1,i,i+1}, S2={i,i+1,i+2},
// smoothness indicators beta_k).  The value from the right is the same
// function of the mirrored cells v_{i+3..i-1}.
template <class T>
inline void weno5_candidates(const T &vm2, const T &vm1, const T &v0, const T &vp1, const T &vp2,
                             T p[3], T b[3]) {
    p[0] = (2.0 * vm2 - 7.0 * vm1 + 11.0 * v0) / 6.0;
    p[1] = (-vm1 + 5.0 * v0 + 2.0 * vp1) / 6.0;
    p[2] = (2.0 * v0 + 5.0 * vp1 - vp2) / 6.0;
    T s0a = vm2 - 2.0 * vm1 + v0, s0b = vm2 - 4.0 * vm1 + 3.0 * v0;
    T s1a = vm1 - 2.0 * v0 + vp1, s1b = vm1 - vp1;
    T s2a = v0 - 2.0 * vp1 + vp2, s2b = 3.0 * v0 - 4.0 * vp1 + vp2;
    b[0] = (13.0 / 12.0) * s0a * s0a + 0.25 * s0b * s0b;
    b[1] = (13.0 / 12.0) * s1a * s1a + 0.25 * s1b * s1b;
    b[2] = (13.0 / 12.0) * s2a * s2a + 0.25 * s2b * s2b;
}

// Unnormalised nonlinear weights, linear weights d = (1/10, 6/10, 3/10).
// WENO5-JS (Jiang & Shu 1996): alpha_k = d_k / (eps + beta_k)^2.
// WENO5-Z (Borges, Carmona, Costa & Don 2008), the paper's default scheme:
// global indicator tau5 = |beta_0 - beta_2|,
// alpha_k = d_k (1 + tau5 / (beta_k + eps)).
template <class T> inline void weno5_alpha(const T b[3], double eps, int z, T a[3]) {
    const double d[3] = {0.1, 0.6, 0.3};
    if (z) {
        T tau = tabs(b[0] - b[2]);
        for (int k = 0; k < 3; ++k) a[k] = d[k] * (1.0 + tau / (b[k] + eps));
    } else {
        for (int k = 0; k < 3; ++k) {
            T e = eps + b[k];
            a[k] = d[k] / (e * e);
        }
    }
}

template <class T>
inline T weno5(const T &vm2, const T &vm1, const T &v0, const T &vp1, const T &vp2, double eps,
               int z) {
    T p[3], b[3], a[3];
    weno5_candidates(vm2, vm1, v0, vp1, vp2, p, b);
    weno5_alpha(b, eps, z, a);
    return (a[0] * p[0] + a[1] * p[1] + a[2] * p[2]) / (a[0] + a[1] + a[2]);
}

template <class T>
inline T weno5js(const T &vm2, const T &vm1, const T &v0, const T &vp1, const T &vp2,
                 double eps) {
    return weno5(vm2, vm1, v0, vp1, vp2, eps, 0);
}

// ----------------------------------------------------------- TENO6-A -------
// Value at x_{i+1/2} from the left from the six cell averages v[0..5] =
// v_{i-2..i+3}: the TENO6-A scheme the paper uses for single-phase flows
// (§3.2 step 3, candidate stencils of its stencil figure, S = {S0..S3} with
// r = {3, 3, 3, 4}; the formulas are those of Fu, Hu & Adams, which the paper
// cites without printing).  In order:
//  1. candidate values q_k at x_{i+1/2} of the polynomials that reproduce the
//     cell averages of S0 = {i-1,i,i+1}, S1 = {i,i+1,i+2}, S2 = {i-2,i-1,i},
//     S3 = {i,i+1,i+2,i+3};
//  2. smoothness indicators beta_k: the squared derivatives (orders 1 .. r-1,
//     scaled to unit spacing) of each candidate polynomial integrated over
//     cell i (the Jiang-Shu measure; S0-S2 give the WENO5 indicators);
//  3. tau6 = |beta_6 - (beta_0 + beta_2 + 4 beta_1)/6|, beta_6 the same
//     measure of the degree-5 polynomial of all six cells;
//  4. gamma_k = (C + tau6/(beta_k + eps))^q, C = 1, q = 6, eps = 1e-30;
//     chi_k = gamma_k / sum_j gamma_j;
//  5. delta_k = 0 where chi_k < C_T, else 1, with the adaptive cut-off:
//     eta_k = (|2 D_{k+1/2} D_{k-1/2}| + e) / (D_{k+1/2}^2 + D_{k-1/2}^2 + e),
//     D_{k+1/2} = v_{k+1} - v_k, e = 0.9 C_r xi^2 / (1 - 0.9 C_r), over the four
//     cells k = i-1 .. i+2 whose both differences lie in the stencil;
//     eta = min_k eta_k; m = 1 - min(1, eta / C_r); g = (1 - m)^4 (1 + 4 m);
//     b = alpha_1 - alpha_2 (1 - g); C_T = 10^-floor(b), with alpha_1 = 10.5,
//     alpha_2 = 3.5, C_r = 0.23, xi = 1e-3 (C_T runs from 1e-10 in smooth
//     regions to 1e-7 at discontinuities);
//  6. omega_k = d_k delta_k / sum_j d_j delta_j with d = (9/20, 3/10, 1/20, 1/5),
//     the weights that make sum d_k q_k the six-cell sixth-order value;
//  7. value = sum_k omega_k q_k.
// The value from the right is the same function of the mirrored cells
// v_{i+3..i-2}.
struct Teno6Parts {
    double q[4], beta[4], chi[4], ct, beta6;
    int delta[4];
};

template <class T> inline T teno6a(const T v[6], Teno6Parts *parts = nullptr) {
    const T &vm2 = v[0], &vm1 = v[1], &v0 = v[2], &vp1 = v[3], &vp2 = v[4], &vp3 = v[5];
    // 1. candidates
    T q[4];
    q[0] = (-vm1 + 5.0 * v0 + 2.0 * vp1) / 6.0;
    q[1] = (2.0 * v0 + 5.0 * vp1 - vp2) / 6.0;
    q[2] = (2.0 * vm2 - 7.0 * vm1 + 11.0 * v0) / 6.0;
    q[3] = (3.0 * v0 + 13.0 * vp1 - 5.0 * vp2 + vp3) / 12.0;
    // 2. smoothness indicators
    T b[4];
    {
        T a = vm1 - 2.0 * v0 + vp1, c = vm1 - vp1;
        b[0] = (13.0 / 12.0) * a * a + 0.25 * c * c;
        a = v0 - 2.0 * vp1 + vp2, c = 3.0 * v0 - 4.0 * vp1 + vp2;
        b[1] = (13.0 / 12.0) * a * a + 0.25 * c * c;
        a = vm2 - 2.0 * vm1 + v0, c = vm2 - 4.0 * vm1 + 3.0 * v0;
        b[2] = (13.0 / 12.0) * a * a + 0.25 * c * c;
        T e1 = -11.0 * v0 + 18.0 * vp1 - 9.0 * vp2 + 2.0 * vp3;
        T e2 = 2.0 * v0 - 5.0 * vp1 + 4.0 * vp2 - vp3;
        T e3 = -v0 + 3.0 * vp1 - 3.0 * vp2 + vp3;
        b[3] = (1.0 / 36.0) * e1 * e1 + (13.0 / 12.0) * e2 * e2 + (781.0 / 720.0) * e3 * e3;
    }
    // 3. the six-cell indicator, the quadratic form of step 2's integral for
    //    the degree-5 polynomial (common denominator 120960)
    const T b6 =
        (vm2 * (271779.0 * vm2 - 2380800.0 * vm1 + 4086352.0 * v0 - 3462252.0 * vp1 +
                1458762.0 * vp2 - 245620.0 * vp3) +
         vm1 * (5653317.0 * vm1 - 20427884.0 * v0 + 17905032.0 * vp1 - 7727988.0 * vp2 +
                1325006.0 * vp3) +
         v0 * (19510972.0 * v0 - 35817664.0 * vp1 + 15929912.0 * vp2 - 2792660.0 * vp3) +
         vp1 * (17195652.0 * vp1 - 15880404.0 * vp2 + 2863984.0 * vp3) +
         vp2 * (3824847.0 * vp2 - 1429976.0 * vp3) + vp3 * (139633.0 * vp3)) /
        120960.0;
    const T tau = tabs(b6 - (b[0] + b[2] + 4.0 * b[1]) / 6.0);
    // 4. scale separation
    T g[4], gs = T(0.0);
    for (int k = 0; k < 4; ++k) {
        const T a = 1.0 + tau / (b[k] + 1e-30);
        const T a2 = a * a;
        g[k] = a2 * a2 * a2;
        gs = gs + g[k];
    }
    T chi[4];
    for (int k = 0; k < 4; ++k) chi[k] = g[k] / gs;
    // 5. adaptive cut-off
    const double Cr = 0.23, xi = 1e-3, alpha1 = 10.5, alpha2 = 3.5;
    const double e = 0.9 * Cr * xi * xi / (1.0 - 0.9 * Cr);
    T eta = T(1e300);
    for (int k = 1; k <= 4; ++k) {  // cells i-1 .. i+2
        const T dp = v[k + 1] - v[k], dm = v[k] - v[k - 1];
        const T ek = (tabs(2.0 * dp * dm) + e) / (dp * dp + dm * dm + e);
        eta = tmin(eta, ek);
    }
    const T m = 1.0 - tmin(T(1.0), eta / Cr);
    const T om = 1.0 - m, om2 = om * om;
    const T gm = om2 * om2 * (1.0 + 4.0 * m);
    const T bb = alpha1 - alpha2 * (1.0 - gm);
    const int fl = (int)std::floor(val(bb));
    const double ct = std::pow(10.0, -fl);
    // 6-7. sharp selection, linear weights of the kept stencils
    const double d[4] = {9.0 / 20.0, 3.0 / 10.0, 1.0 / 20.0, 1.0 / 5.0};
    int delta[4];
    double dsum = 0.0;
    for (int k = 0; k < 4; ++k) {
        delta[k] = val(chi[k]) < ct ? 0 : 1;
        dsum += delta[k] * d[k];
    }
    T out = T(0.0);
    for (int k = 0; k < 4; ++k)
        if (delta[k]) out = out + (d[k] / dsum) * q[k];
    if (parts) {
        for (int k = 0; k < 4; ++k) {
            parts->q[k] = val(q[k]);
            parts->beta[k] = val(b[k]);
            parts->chi[k] = val(chi[k]);
            parts->delta[k] = delta[k];
        }
        parts->ct = ct;
        parts->beta6 = val(b6);
    }
    return out;
}

// One reconstructed value from the left: WENO5 (JS or Z weights) from
// v[0..4] or TENO6-A from v[0..5].
template <class T> inline T recon_left(const orc_config &c, const T v[6]) {
    if (c.teno) return teno6a(v);
    return weno5(v[0], v[1], v[2], v[3], v[4], c.weno_eps, c.weno_z);
}

// ---------------------------------------------------------- reconstruction --
// Component-wise: WENO5 (JS or Z weights) applied to each primitive variable
// (reading: the paper projects W in characteristic mode, so component mode
// reconstructs W).
template <class T>
inline void reconstruct_comp(const orc_config &c, const Layout &L, const T Ws[6][NVMAX], T *WL,
                             T *WR) {
    for (int v = 0; v < L.nv; ++v) {
        const T fwd[6] = {Ws[0][v], Ws[1][v], Ws[2][v], Ws[3][v], Ws[4][v], Ws[5][v]};
        const T bwd[6] = {Ws[5][v], Ws[4][v], Ws[3][v], Ws[2][v], Ws[1][v], Ws[0][v]};
        WL[v] = recon_left(c, fwd);
        WR[v] = recon_left(c, bwd);
    }
}

// Characteristic-wise (§3.2 steps 1-4, App. C.1): frozen state = arithmetic
// mean of W_i and W_{i+1}; project the six stencil cells with K^{-1}
// (the analytic inverse of the printed K, which the paper does not print),
// reconstruct every characteristic field, project back with K.
// Field slots: the u-c field sits in the normal-velocity slot, the u+c field
// in the pressure slot, the entropy/partial-density fields in the density
// slots, the shear and volume-fraction fields in their own slots.
template <class T>
inline void reconstruct_char(const orc_config &c, const Layout &L, int d, const T Ws[6][NVMAX],
                             T *WL, T *WR) {
    const int nv = L.nv, np = L.np, in = np + d, ie = L.ie;
    T Wb[NVMAX];
    for (int v = 0; v < nv; ++v) Wb[v] = 0.5 * (Ws[2][v] + Ws[3][v]);
    T rho = density(L, Wb);
    T rc2 = rhoc2_of(c, L, Wb);
    T cb = sqrt_(rc2 / rho);
    T h_c = 0.5 / cb;     // 1/(2c)
    T h_rc2 = 0.5 / rc2;  // 1/(2 rho c^2)
    T ent[2];             // entropy rows: (alpha_k rho_k)_bar / (rho c^2)
    for (int k = 0; k < np; ++k) ent[k] = Wb[k] / rc2;

    T Q[6][NVMAX];
    for (int j = 0; j < 6; ++j) {
        const T *w = Ws[j];
        for (int v = 0; v < nv; ++v) Q[j][v] = w[v];  // shear / alpha rows: identity
        for (int k = 0; k < np; ++k) Q[j][k] = w[k] - ent[k] * w[ie];
        Q[j][in] = -h_c * w[in] + h_rc2 * w[ie];
        Q[j][ie] = h_c * w[in] + h_rc2 * w[ie];
    }
    T qL[NVMAX], qR[NVMAX];
    for (int v = 0; v < nv; ++v) {
        const T fwd[6] = {Q[0][v], Q[1][v], Q[2][v], Q[3][v], Q[4][v], Q[5][v]};
        const T bwd[6] = {Q[5][v], Q[4][v], Q[3][v], Q[2][v], Q[1][v], Q[0][v]};
        qL[v] = recon_left(c, fwd);
        qR[v] = recon_left(c, bwd);
    }
    T *outs[2] = {WL, WR};
    T *qs[2] = {qL, qR};
    for (int s = 0; s < 2; ++s) {
        T *o = outs[s];
        const T *q = qs[s];
        for (int v = 0; v < nv; ++v) o[v] = q[v];
        for (int k = 0; k < np; ++k) o[k] = Wb[k] * q[in] + q[k] + Wb[k] * q[ie];
        o[in] = -cb * q[in] + cb * q[ie];
        o[ie] = rc2 * q[in] + rc2 * q[ie];
    }
}

// --------------------------------------------------------------- limiters --
// Interpolation limiter on one reconstructed face state (§3.3 item 1):
// successive checks -- partial densities (eps_rho), then (diffuse interface)
// the volume fraction outside [eps_a, 1-eps_a], then rho c^2 (eps_rhoc2) --
// each replacing the whole state by the first-order cell value on violation.
// Returns 1 if the side was switched.
template <class T>
inline int interp_limit(const orc_config &c, const Layout &L, T *Wf, const T *W1) {
    bool bad = false;
    for (int k = 0; k < L.np; ++k) bad = bad || val(Wf[k]) < c.eps_rho;
    if (!bad && L.ia >= 0)
        bad = val(Wf[L.ia]) < c.eps_alpha || val(Wf[L.ia]) > 1.0 - c.eps_alpha;
    if (!bad) bad = val(rhoc2_of(c, L, Wf)) < c.eps_rhoc2;
    if (!bad) return 0;
    for (int v = 0; v < L.nv; ++v) Wf[v] = W1[v];
    return 1;
}

// ------------------------------------------------------------------- HLLC --
// Physical convective flux along axis d (§2.1, §2.3).
template <class T>
inline void phys_flux(const Layout &L, int d, const T *W, const T *U, T *F) {
    const int in = L.np + d;
    T un = W[in], p = W[L.ie];
    for (int k = 0; k < L.np; ++k) F[k] = U[k] * un;
    for (int e = 0; e < L.ndim; ++e) F[L.np + e] = U[L.np + e] * un;
    F[in] = F[in] + p;
    F[L.ie] = un * (U[L.ie] + p);
    if (L.ia >= 0) F[L.ia] = W[L.ia] * un;
}

// HLLC flux and upwinded normal velocity (§3.2 step 6, App. C.2).
// Wave speeds: Einfeldt s^L, s^R with the Roe-type averages u_bar, c_bar
// (reading, Einfeldt 1988: sqrt(rho)-weighted mean velocity; c_bar^2 =
// sqrt(rho)-weighted mean of c^2 plus the velocity-jump term); Batten s*.
// sign(s*) = 0 at s* = 0 gives the mean of the two branches.
template <class T>
inline void hllc(const orc_config &c, const Layout &L, int d, const T *WL, const T *WR, T *F,
                 T &uh) {
    const int nv = L.nv, in = L.np + d, ie = L.ie;
    T UL[NVMAX], UR[NVMAX];
    prim2cons(c, L, WL, UL);
    prim2cons(c, L, WR, UR);
    T rhoL = density(L, WL), rhoR = density(L, WR);
    T uL = WL[in], uR = WR[in], pL = WL[ie], pR = WR[ie];
    T cL = sqrt_(rhoc2_of(c, L, WL) / rhoL);
    T cR = sqrt_(rhoc2_of(c, L, WR) / rhoR);

    T srL = sqrt_(rhoL), srR = sqrt_(rhoR);
    T ssum = srL + srR;
    T ubar = (srL * uL + srR * uR) / ssum;
    T du = uR - uL;
    T c2bar = (srL * cL * cL + srR * cR * cR) / ssum + 0.5 * srL * srR / (ssum * ssum) * du * du;
    T cbar = sqrt_(c2bar);
    T sL = tmin(ubar - cbar, uL - cL);
    T sR = tmax(ubar + cbar, uR + cR);
    T mL = rhoL * (sL - uL), mR = rhoR * (sR - uR);
    T sstar = (pR - pL + mL * uL - mR * uR) / (mL - mR);
    T sm = tmin(T(0.0), sL), sp = tmax(T(0.0), sR);

    const double sg = val(sstar) > 0.0 ? 1.0 : (val(sstar) < 0.0 ? -1.0 : 0.0);
    T FL[NVMAX], FR[NVMAX], Fb[2][NVMAX], ub[2];
    const T *Ws[2] = {WL, WR};
    const T *Us[2] = {UL, UR};
    const T sK[2] = {sL, sR}, sPM[2] = {sm, sp}, uK[2] = {uL, uR}, rK[2] = {rhoL, rhoR},
            pK[2] = {pL, pR};
    phys_flux(L, d, WL, UL, FL);
    phys_flux(L, d, WR, UR, FR);
    T *FK[2] = {FL, FR};
    for (int s = 0; s < 2; ++s) {
        if ((s == 0 && sg < 0.0) || (s == 1 && sg > 0.0)) continue;  // branch weight is zero
        const T *W = Ws[s];
        const T *U = Us[s];
        T fac = (sK[s] - uK[s]) / (sK[s] - sstar);
        T Us_[NVMAX];
        for (int k = 0; k < L.np; ++k) Us_[k] = fac * U[k];
        for (int e = 0; e < L.ndim; ++e) Us_[L.np + e] = fac * (rK[s] * W[L.np + e]);
        Us_[in] = fac * (rK[s] * sstar);
        Us_[ie] = fac * (U[ie] + (sstar - uK[s]) * (rK[s] * sstar + pK[s] / (sK[s] - uK[s])));
        if (L.ia >= 0) Us_[L.ia] = fac * W[L.ia];
        for (int v = 0; v < nv; ++v) Fb[s][v] = FK[s][v] + sPM[s] * (Us_[v] - U[v]);
        ub[s] = uK[s] + sPM[s] * (fac - 1.0);
    }
    if (sg > 0.0) {
        for (int v = 0; v < nv; ++v) F[v] = Fb[0][v];
        uh = ub[0];
    } else if (sg < 0.0) {
        for (int v = 0; v < nv; ++v) F[v] = Fb[1][v];
        uh = ub[1];
    } else {
        for (int v = 0; v < nv; ++v) F[v] = 0.5 * Fb[0][v] + 0.5 * Fb[1][v];
        uh = 0.5 * ub[0] + 0.5 * ub[1];
    }
}

// Pseudo-time factor of the flux limiter's test states of axis d (§3.3 item
// 2, reading after Hu, Adams & Shu 2013): lam = 2 D dt / dx_d with D the
// number of active axes.
inline double fl_lambda(const orc_config &c, const Layout &L, int d, double dt) {
    return 2.0 * L.ndim * dt / c.dx[d];
}

// Flux limiter test (§3.3 item 2).  Reading of the pseudo-time integration
// (after Hu, Adams & Shu 2013): with lam = 2 D dt/dx_d, the two test states
// of face i+1/2 are U_i - lam F and U_{i+1} + lam F; the volume-fraction
// component also carries the face's share of the a1 div(u) source,
// a1 -/+ lam (F_a - a1 u_hllc).  Loops: partial densities, volume fraction,
// rho c^2.  Returns true if the high-order flux must be replaced.
template <class T>
inline bool flux_limit_violates(const orc_config &c, const Layout &L, double lam, const T *F,
                                const T &uh, const T *Ui, const T *Uj) {
    T Ts[2][NVMAX];
    const T *Uc[2] = {Ui, Uj};
    const double sgn[2] = {-1.0, 1.0};
    for (int s = 0; s < 2; ++s) {
        for (int v = 0; v < L.nv; ++v) Ts[s][v] = Uc[s][v] + (sgn[s] * lam) * F[v];
        if (L.ia >= 0)
            Ts[s][L.ia] = Uc[s][L.ia] + (sgn[s] * lam) * (F[L.ia] - Uc[s][L.ia] * uh);
    }
    for (int s = 0; s < 2; ++s)
        for (int k = 0; k < L.np; ++k)
            if (val(Ts[s][k]) < c.eps_rho) return true;
    if (L.ia >= 0)
        for (int s = 0; s < 2; ++s)
            if (val(Ts[s][L.ia]) < c.eps_alpha || val(Ts[s][L.ia]) > 1.0 - c.eps_alpha)
                return true;
    for (int s = 0; s < 2; ++s) {
        T W[NVMAX];
        cons2prim(c, L, Ts[s], W);
        if (val(rhoc2_of(c, L, W)) < c.eps_rhoc2) return true;
    }
    return false;
}

// --------------------------------------------------------------- halos ------
// Halo fill of a padded array (§3.1, §4.3 order face -> edge -> vertex):
// axis by axis, each pass covering the halos already filled on the earlier
// axes.  Periodic wraps; zero-gradient copies the boundary cell; symmetry
// mirrors and flips the normal momentum.
template <class T>
void fill_halos(const orc_config &c, const Layout &L, std::vector<T> &A) {
    for (int d = 0; d < L.ndim; ++d) {
        int lo[3], hi[3];
        for (int e = 0; e < 3; ++e) {
            lo[e] = (e < d) ? -L.h[e] : 0;
            hi[e] = (e < d) ? L.n[e] + L.h[e] : L.n[e];
        }
        lo[d] = 0;
        hi[d] = 1;  // one pass per transverse position
        const long sd = L.pstride(d);
        const int N = L.n[d];
        for (int z = lo[2]; z < hi[2]; ++z)
            for (int y = lo[1]; y < hi[1]; ++y)
                for (int x = lo[0]; x < hi[0]; ++x) {
                    int q[3] = {x, y, z};
                    q[d] = 0;
                    const long base = L.pidx(q[0], q[1], q[2]);  // cell 0 along d
                    for (int side = 0; side < 2; ++side) {
                        const int bc = c.bc[d][side];
                        for (int k = 1; k <= NH; ++k) {
                            int dst = side == 0 ? -k : N - 1 + k;
                            int src;
                            if (bc == ORC_BC_PERIODIC) src = side == 0 ? N - k : k - 1;
                            else if (bc == ORC_BC_ZEROGRAD) src = side == 0 ? 0 : N - 1;
                            else src = side == 0 ? k - 1 : N - k;
                            for (int v = 0; v < L.nv; ++v) {
                                T s = A[v * L.npad + base + src * sd];
                                if (bc == ORC_BC_SYMMETRY && v == L.np + d) s = -s;
                                A[v * L.npad + base + dst * sd] = s;
                            }
                        }
                    }
                }
    }
}

// ------------------------------------------------------------------ THINC --
// Interface capturing for the five-equation model (§3.2 step 4, after Xiao
// et al. 2005/2011 and Garrick et al. 2017).  Used only in interface cells:
// eps <= a1_i <= 1 - eps (eps = 1e-4) and (a_{i+1} - a_i)(a_i - a_{i-1}) > 0
// along the reconstruction axis.  In such a cell a1 follows
//   a(xi) = 1/2 [1 + theta tanh(beta_i (xi + xc_i))],  xi = (x - x_{i-1/2})/dx,
// with beta_i = beta |n_d| + 0.01 (beta = 1), theta = sign(a_{i+1} - a_{i-1})
// (reading: the printed profile is the increasing case theta = +1), and xc_i
// (left blank in the paper; reading: fixed by the cell average) from
//   integral_0^1 a(xi) dxi = a_i
//   <=>  y = e^{2 beta xc} = (e^{beta(1+s)} - 1) / (e^{beta} e^{beta s} (e^{beta(1-s)} - 1)),
// s = theta (2 a_i - 1), evaluated with expm1 (no cancellation near
// |s| -> 1).  The face values are the profile at xi = 1 (from the left at
// x_{i+1/2}) and xi = 0 (from the right at x_{i-1/2}).
constexpr double THINC_EPS = 1e-4, THINC_BETA = 1.0;

template <class T> struct ThincFit {
    double theta;
    T beta, y;  // y = e^{2 beta xc}
};

template <class T>
inline bool thinc_fit(const T &am, const T &ac, const T &ap, const T &nabs, ThincFit<T> &f) {
    if (!(val(ac) >= THINC_EPS && val(ac) <= 1.0 - THINC_EPS)) return false;
    if (!(val(ap - ac) * val(ac - am) > 0.0)) return false;
    f.theta = val(ap) > val(am) ? 1.0 : -1.0;
    f.beta = THINC_BETA * nabs + 0.01;
    T s = f.theta * (2.0 * ac - 1.0);
    f.y = expm1_(f.beta * (1.0 + s)) / (exp_(f.beta) * exp_(f.beta * s) * expm1_(f.beta * (1.0 - s)));
    return true;
}

// Profile value at xi = 1 (side 0) or xi = 0 (side 1):
// e = e^{2 beta (xi + xc)}, a = e/(e + 1) for theta = +1, 1/(e + 1) for -1.
template <class T> inline T thinc_value(const ThincFit<T> &f, int side) {
    T e = side == 0 ? exp_(2.0 * f.beta) * f.y : f.y;
    return f.theta > 0.0 ? e / (e + 1.0) : 1.0 / (e + 1.0);
}

// psi = a^0.1 / (a^0.1 + (1 - a)^0.1) of a1 clipped to [0, 1] (reading: a
// slightly out-of-range a1 must not make the normal undefined).
template <class T> inline T thinc_psi(const T &a1) {
    T a = val(a1) < 0.0 ? T(0.0) : (val(a1) > 1.0 ? T(1.0) : a1);
    T b = 1.0 - a;
    T p = val(a) > 0.0 ? exp_(0.1 * log_(a)) : T(0.0);
    T q = val(b) > 0.0 ? exp_(0.1 * log_(b)) : T(0.0);
    return p / (p + q);
}

// |n_d| on every padded cell that has both neighbours along every axis
// (ghost cells included), from psi of the halo-filled primitives:
// n = grad psi/|grad psi| with (psi_{+e} - psi_{-e})/(2 dx_e); a zero gradient
// gives n = 0.
// flops_per_cell (Counted runs): psi per cell + normal per cell.
template <class T>
void thinc_normals(const orc_config &c, const Layout &L, const std::vector<T> &Wp,
                   std::vector<T> &nrm, double *flops_per_cell = nullptr) {
    const bool count = flops_per_cell && std::is_same<T, Counted>::value;
    long long t0 = count ? tally().total() : 0;
    std::vector<T> psi(L.npad);
    for (long p = 0; p < L.npad; ++p) psi[p] = thinc_psi(Wp[L.ia * L.npad + p]);
    long long t1 = count ? tally().total() : 0;
    long ncomp = 0;
    nrm.assign((size_t)L.ndim * L.npad, T(0.0));
    int lo[3], hi[3];
    for (int e = 0; e < 3; ++e) {
        lo[e] = -L.h[e] + (e < L.ndim ? 1 : 0);
        hi[e] = L.n[e] + L.h[e] - (e < L.ndim ? 1 : 0);
    }
    for (int z = lo[2]; z < hi[2]; ++z)
        for (int y = lo[1]; y < hi[1]; ++y)
            for (int x = lo[0]; x < hi[0]; ++x) {
                const long p = L.pidx(x, y, z);
                ++ncomp;
                T g[3];
                T g2 = T(0.0);
                for (int e = 0; e < L.ndim; ++e) {
                    const long se = L.pstride(e);
                    g[e] = (psi[p + se] - psi[p - se]) / (2.0 * c.dx[e]);
                    g2 = g2 + g[e] * g[e];
                }
                if (!(val(g2) > 0.0)) continue;
                T gn = sqrt_(g2);
                for (int e = 0; e < L.ndim; ++e) nrm[e * L.npad + p] = tabs(g[e]) / gn;
            }
    if (count) {
        const long long t2 = tally().total();
        *flops_per_cell = (double)(t1 - t0) / L.npad + (double)(t2 - t1) / ncomp;
    }
}

// Replace a1 and the partial densities of one reconstructed face side by the
// THINC values of cell p (padded index; neighbours p -/+ sd along the axis):
// (a_k rho_k) = a_k^THINC rho_k with the cell's phase densities rho_k
// (reading of the consistent adaptation of Garrick et al. 2017).
template <class T>
inline void thinc_side(const Layout &L, const std::vector<T> &Wp, const std::vector<T> &nrm, int d,
                       long p, long sd, int side, T *Wf) {
    const long np_ = L.npad;
    const T am = Wp[L.ia * np_ + p - sd], ac = Wp[L.ia * np_ + p], ap = Wp[L.ia * np_ + p + sd];
    ThincFit<T> f;
    if (!thinc_fit(am, ac, ap, nrm[d * np_ + p], f)) return;
    T a = thinc_value(f, side);
    Wf[0] = a * (Wp[p] / ac);
    Wf[1] = (1.0 - a) * (Wp[np_ + p] / (1.0 - ac));
    Wf[L.ia] = a;
}

// ---------------------------------------------------------- viscous flux --
// Dissipative flux on face i+1/2 along d (§2.1 Eqs. for F^d, tau, q), with
// central stencils of order 2, 4 or 6 (the paper offers 2nd/4th/6th-order
// central differences for the dissipative terms; reading of the stencils:
// the standard ones, written on the normal cells v = phi_{i+1-h..i+h}):
//   order 2: normal derivative (v_i+1 - v_i)/dx, face value (v_i + v_i+1)/2,
//            cell-centre derivative (phi_{j+1} - phi_{j-1})/(2 dy)
//   order 4: (v_{i-1} - 27 v_i + 27 v_{i+1} - v_{i+2})/(24 dx),
//            (-v_{i-1} + 9 v_i + 9 v_{i+1} - v_{i+2})/16,
//            (phi_{j-2} - 8 phi_{j-1} + 8 phi_{j+1} - phi_{j+2})/(12 dy)
//   order 6: (-9 v_{i-2} + 125 v_{i-1} - 2250 v_i + 2250 v_{i+1}
//             - 125 v_{i+2} + 9 v_{i+3})/(1920 dx),
//            (3 v_{i-2} - 25 v_{i-1} + 150 v_i + 150 v_{i+1} - 25 v_{i+2}
//             + 3 v_{i+3})/256,
//            (-phi_{j-3} + 9 phi_{j-2} - 45 phi_{j-1} + 45 phi_{j+1}
//             - 9 phi_{j+2} + phi_{j+3})/(60 dy);
// the tangential derivative is the cell-centre derivative at the normal
// cells interpolated to the face with the face-value weights.
// lambda = mu c_p / Pr with c_p = gamma R/(gamma-1) (the paper's printed
// lambda = Pr/(mu c_p) is dimensionally inconsistent).
inline int visc_half(const orc_config &c) { return c.visc_order == 2 ? 1 : (c.visc_order == 6 ? 3 : 2); }

// v[0..2h-1] = values at the normal cells i+1-h .. i+h
template <class T> inline T face_deriv(int h, const T *v, double dx) {
    if (h == 1) return (v[1] - v[0]) / dx;
    if (h == 2) return (v[0] - 27.0 * v[1] + 27.0 * v[2] - v[3]) / (24.0 * dx);
    return (-9.0 * v[0] + 125.0 * v[1] - 2250.0 * v[2] + 2250.0 * v[3] - 125.0 * v[4] + 9.0 * v[5]) /
           (1920.0 * dx);
}
template <class T> inline T face_value(int h, const T *v) {
    if (h == 1) return (v[0] + v[1]) / 2.0;
    if (h == 2) return (-v[0] + 9.0 * v[1] + 9.0 * v[2] - v[3]) / 16.0;
    return (3.0 * v[0] - 25.0 * v[1] + 150.0 * v[2] + 150.0 * v[3] - 25.0 * v[4] + 3.0 * v[5]) / 256.0;
}
// w[0..2h] = values at cells j-h .. j+h
template <class T> inline T cell_deriv(int h, const T *w, double dy) {
    if (h == 1) return (w[2] - w[0]) / (2.0 * dy);
    if (h == 2) return (w[0] - 8.0 * w[1] + 8.0 * w[3] - w[4]) / (12.0 * dy);
    return (-w[0] + 9.0 * w[1] - 45.0 * w[2] + 45.0 * w[4] - 9.0 * w[5] + w[6]) / (60.0 * dy);
}

template <class T>
void viscous_face(const orc_config &c, const Layout &L, int d, const std::vector<T> &Wp,
                  const std::vector<T> &Tp, long pface /* padded index of cell i+1 */, T *Fd) {
    const int nd = L.ndim, np = L.np;
    const long sd = L.pstride(d);
    const int nphi = nd + 1;  // u_0..u_{nd-1}, T
    const int h = visc_half(c);
    auto phi = [&](int f, long idx) -> T {
        return f < nd ? Wp[(np + f) * L.npad + idx] : Tp[idx];
    };
    // Gradients the fluxes use: every phi normal to the face; along a
    // tangential axis e only u_d (shear stress tau_de) and u_e (divergence).
    T grad[4][3], face_u[3];
    for (int f = 0; f < nphi; ++f) {
        T v[6];
        for (int m = 0; m < 2 * h; ++m) v[m] = phi(f, pface + (m - h) * sd);  // cells i+1-h..i+h
        grad[f][d] = face_deriv(h, v, c.dx[d]);
        if (f < nd) face_u[f] = face_value(h, v);
        for (int e = 0; e < nd; ++e) {
            if (e == d || (f != d && f != e)) continue;
            const long se = L.pstride(e);
            T g[6];
            for (int m = 0; m < 2 * h; ++m) {
                const long b = pface + (m - h) * sd;
                T w[7];
                for (int j = -h; j <= h; ++j) w[j + h] = phi(f, b + j * se);
                g[m] = cell_deriv(h, w, c.dx[e]);
            }
            grad[f][e] = face_value(h, g);
        }
    }
    T div = grad[0][0];
    for (int k = 1; k < nd; ++k) div = div + grad[k][k];
    const double mu = c.mu;
    const double cp = c.gamma[0] * c.R / (c.gamma[0] - 1.0);
    const double lambda = mu * cp / c.Pr;
    for (int v = 0; v < L.nv; ++v) Fd[v] = T(0.0);
    T work = T(0.0);
    for (int k = 0; k < nd; ++k) {
        T tau = mu * (grad[d][k] + grad[k][d]);
        if (k == d) tau = tau - (2.0 / 3.0 * mu) * div;
        Fd[np + k] = tau;
        work = (k == 0) ? face_u[k] * tau : work + face_u[k] * tau;
    }
    T q = -lambda * grad[nd][d];
    Fd[L.ie] = work - q;
}

// ---------------------------------------------------------------- RHS -------
struct PhaseSplit {  // flop tallies per phase (Counted runs only)
    long long axis[3] = {0, 0, 0};
    long long divergence = 0;
    double interface_normal = 0.0;  // THINC psi + normal, per cell
};

// R(U) of the semi-discrete form (§3.2):
//   dU/dt = -sum_d [(F^c - F^d)_{i+1/2} - (F^c - F^d)_{i-1/2}]/dx_d + S,
// with the diffuse-interface source a1 div(u) built from the HLLC-upwinded
// face velocities (§3.7).  Per face: reconstruct (component- or
// characteristic-wise), interpolation limiter, HLLC, flux limiter, viscous
// flux.  dt only enters the flux limiter.
template <class T>
void rhs_impl(const orc_config &c, const T *U, double dt, T *dU, orc_counts *cnt,
              PhaseSplit *split = nullptr) {
    const Layout L(c);
    const int nv = L.nv;
    std::vector<T> Up((size_t)nv * L.npad), Wp((size_t)nv * L.npad), Tp;
    for (int z = 0; z < L.n[2]; ++z)
        for (int y = 0; y < L.n[1]; ++y)
            for (int x = 0; x < L.n[0]; ++x)
                for (int v = 0; v < nv; ++v)
                    Up[v * L.npad + L.pidx(x, y, z)] = U[v * L.ncell + L.cidx(x, y, z)];
    fill_halos(c, L, Up);  // a1
    const bool visc = c.viscous && c.model == ORC_SPM;
    if (visc) Tp.assign(L.npad, T(0.0));
#pragma omp parallel for schedule(static) if (kParallel<T>)
    for (long p = 0; p < L.npad; ++p) {  // a2 on every padded cell
        T u[NVMAX], w[NVMAX];
        for (int v = 0; v < nv; ++v) u[v] = Up[v * L.npad + p];
        cons2prim(c, L, u, w);
        for (int v = 0; v < nv; ++v) Wp[v * L.npad + p] = w[v];
        if (visc) Tp[p] = w[L.ie] / (w[0] * c.R);  // T = p/(rho R)
    }

    const bool thinc = c.thinc && L.ia >= 0;
    std::vector<T> nrm;
    if (thinc) thinc_normals(c, L, Wp, nrm, split ? &split->interface_normal : nullptr);

    for (long i = 0; i < (long)nv * L.ncell; ++i) dU[i] = T(0.0);
    long long il = 0, fl = 0;
    for (int d = 0; d < L.ndim; ++d) {
        long long t0 = std::is_same<T, Counted>::value ? tally().total() : 0;
        int m[3] = {L.n[0], L.n[1], L.n[2]};
        m[d] += 1;  // faces along d
        const long nface = (long)m[0] * m[1] * m[2];
        std::vector<T> F((size_t)nv * nface), UH(L.ia >= 0 ? nface : 0);
        const long sd = L.pstride(d);
        const double lam = fl_lambda(c, L, d, dt);
#pragma omp parallel for schedule(static) reduction(+ : il, fl) if (kParallel<T>)
        for (long g = 0; g < nface; ++g) {
            int q[3] = {(int)(g % m[0]), (int)((g / m[0]) % m[1]), (int)(g / ((long)m[0] * m[1]))};
            // face q[d] lies between cells q[d]-1 (i) and q[d] (i+1)
            const long pR = L.pidx(q[0], q[1], q[2]);
            const long pL = pR - sd;
            T Ws[6][NVMAX];
            for (int j = 0; j < 6; ++j)
                for (int v = 0; v < nv; ++v) Ws[j][v] = Wp[v * L.npad + pL + (j - 2) * sd];
            T WL[NVMAX], WR[NVMAX];
            if (c.recon == ORC_CHAR) reconstruct_char(c, L, d, Ws, WL, WR);
            else reconstruct_comp(c, L, Ws, WL, WR);
            if (thinc) {
                thinc_side(L, Wp, nrm, d, pL, sd, 0, WL);  // cell i, value at its upper face
                thinc_side(L, Wp, nrm, d, pR, sd, 1, WR);  // cell i+1, value at its lower face
            }
            if (c.limiter) {
                il += interp_limit(c, L, WL, Ws[2]);
                il += interp_limit(c, L, WR, Ws[3]);
            }
            T Ff[NVMAX], uh;
            hllc(c, L, d, WL, WR, Ff, uh);
            if (c.limiter) {
                T Ui[NVMAX], Uj[NVMAX];
                for (int v = 0; v < nv; ++v) {
                    Ui[v] = Up[v * L.npad + pL];
                    Uj[v] = Up[v * L.npad + pR];
                }
                if (flux_limit_violates(c, L, lam, Ff, uh, Ui, Uj)) {
                    hllc(c, L, d, Ws[2], Ws[3], Ff, uh);  // first-order HLLC(U_i, U_{i+1})
                    fl += 1;
                }
            }
            if (visc) {
                T Fd[NVMAX];
                viscous_face(c, L, d, Wp, Tp, pR, Fd);
                for (int v = 0; v < nv; ++v) Ff[v] = Ff[v] - Fd[v];
            }
            for (int v = 0; v < nv; ++v) F[v * nface + g] = Ff[v];
            if (L.ia >= 0) UH[g] = uh;
        }
        long long t1 = std::is_same<T, Counted>::value ? tally().total() : 0;
        // divergence (and the a1 div(u) source) into dU
        const double dxd = c.dx[d];
        long fs = (d == 0) ? 1 : (d == 1 ? m[0] : (long)m[0] * m[1]);
#pragma omp parallel for schedule(static) if (kParallel<T>)
        for (long i = 0; i < L.ncell; ++i) {
            int q[3] = {(int)(i % L.n[0]), (int)((i / L.n[0]) % L.n[1]),
                        (int)(i / ((long)L.n[0] * L.n[1]))};
            const long gm = ((long)q[2] * m[1] + q[1]) * m[0] + q[0];  // face i-1/2
            const long gp = gm + fs;                                    // face i+1/2
            for (int v = 0; v < nv; ++v)
                dU[v * L.ncell + i] = dU[v * L.ncell + i] - (F[v * nface + gp] - F[v * nface + gm]) / dxd;
            if (L.ia >= 0)
                dU[L.ia * L.ncell + i] =
                    dU[L.ia * L.ncell + i] + U[L.ia * L.ncell + i] * (UH[gp] - UH[gm]) / dxd;
        }
        if (split) {
            long long t2 = tally().total();
            split->axis[d] += t1 - t0;
            split->divergence += t2 - t1;
        }
    }
    if (cnt) {
        cnt->il_sides += il;
        cnt->fl_faces += fl;
    }
}

// ------------------------------------------------------------ TVD-RK3 -------
// §3.4: U1 = Un + dt R(Un); U2 = 3/4 Un + 1/4 U1 + 1/4 dt R(U1);
//       U^{n+1} = 1/3 Un + 2/3 U2 + 2/3 dt R(U2), evaluated in printed order.
template <class T> void rk3_impl(const orc_config &c, T *U, double dt, orc_counts *cnt) {
    const Layout L(c);
    const long N = (long)L.nv * L.ncell;
    std::vector<T> Un(U, U + N), R(N), U1(N), U2(N);
    rhs_impl(c, Un.data(), dt, R.data(), cnt);
    for (long i = 0; i < N; ++i) U1[i] = Un[i] + dt * R[i];
    rhs_impl(c, U1.data(), dt, R.data(), cnt);
    for (long i = 0; i < N; ++i) U2[i] = 0.75 * Un[i] + 0.25 * U1[i] + (0.25 * dt) * R[i];
    rhs_impl(c, U2.data(), dt, R.data(), cnt);
    for (long i = 0; i < N; ++i)
        U[i] = (1.0 / 3.0) * Un[i] + (2.0 / 3.0) * U2[i] + (2.0 / 3.0 * dt) * R[i];
}

// ---------------------------------------------------------------- CFL -------
// Per-cell convective rate sum_d (|u_d| + c)/dx_d (§3.4; the paper defers the
// formula to Hoppe et al. 2022 -- reading).
template <class T> inline T cfl_rate(const orc_config &c, const Layout &L, const T *W) {
    T cs = sqrt_(rhoc2_of(c, L, W) / density(L, W));
    T s = (tabs(W[L.np]) + cs) / c.dx[0];
    for (int d = 1; d < L.ndim; ++d) s = s + (tabs(W[L.np + d]) + cs) / c.dx[d];
    return s;
}

// dt = CFL * min(1/max s, 3/14 min(rho) dx_min^2/mu [viscous]), or the fixed
// dt; then clipped to t_end - t.
inline double cfl_dt(const orc_config &c, const double *U, double t) {
    const Layout L(c);
    double smax = 0.0, rmin = std::numeric_limits<double>::infinity();
#pragma omp parallel for schedule(static) reduction(max : smax) reduction(min : rmin)
    for (long i = 0; i < L.ncell; ++i) {
        double u[NVMAX], w[NVMAX];
        for (int v = 0; v < L.nv; ++v) u[v] = U[v * L.ncell + i];
        cons2prim(c, L, u, w);
        double s = cfl_rate(c, L, w);
        smax = s > smax ? s : smax;
        double r = density(L, w);
        rmin = r < rmin ? r : rmin;
    }
    double dt;
    if (c.fixed_dt > 0.0) {
        dt = c.fixed_dt;
    } else {
        dt = c.cfl / smax;
        if (c.viscous && c.model == ORC_SPM && c.mu > 0.0) {
            double dxm = c.dx[0];
            for (int d = 1; d < L.ndim; ++d) dxm = c.dx[d] < dxm ? c.dx[d] : dxm;
            double dtv = c.cfl * (3.0 / 14.0) * rmin * dxm * dxm / c.mu;
            dt = dtv < dt ? dtv : dt;
        }
    }
    if (c.t_end > 0.0) {
        double rem = c.t_end - t;
        if (rem <= 1e-12 * c.t_end) return 0.0;
        dt = rem < dt ? rem : dt;
    }
    return dt;
}

}  // namespace orc
