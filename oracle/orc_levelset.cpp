// orc_levelset.cpp -- oracle of the level-set model's data-parallel parts
// (test infrastructure only; shares no code with the CUDA library).
//
// The level-set model of §3.5 and App. D on a uniform grid of cubic cells
// (2-D or 3-D):
//   * interface geometry (App. D): the level set interpolated to the cell
//     vertices, the face apertures of the positive phase, the interface
//     segment dGamma, the volume fraction alpha (pyramids from the cell
//     centre over the faces and the interface facet) and the interface
//     normal grad(phi)/|grad(phi)| from 4th-order central differences;
//   * level-set advection (Eq. levelset_advection, §3.5): R = -u . grad(phi)
//     with the 5th-order upstream-central derivative of each axis
//     (upstream side by the sign of u_d), integrated with TVD-RK3 (§3.4);
//   * reinitialisation (Eq. levelset_reinitialization, §3.5):
//     R = -sgn(phi0) (|grad(phi)| - 1), |grad(phi)| the Godunov Hamiltonian
//     of third-order WENO one-sided derivatives (Jiang & Peng), second-order
//     TVD Runge-Kutta in pseudo-time with dtau = 0.25 dx, cells whose
//     residual |R| is at most the threshold left unchanged;
//   * interface quantities (App. D, linearised two-material Riemann problem)
//     and the ghost-cell / interface-quantity extensions (§3.5);
//   * the cut-cell right-hand side of each phase (Eq. FVD_levelset) and the
//     conservative mixing (App. D);
//   * the two-phase time step chaining them (Alg. 2).
// Each function below states the reading it takes where the paper is
// silent.  Boundary conditions map indices as the flow solver does (a
// mirror copies the scalar).
#include <algorithm>
#include <cmath>
#include <vector>

#include "orc.h"
#include "orc_scheme.hpp"
#include "orc_types.hpp"

namespace orc {
namespace {

int map_index(int c, int n, int blo, int bhi) {
    if (c < 0) {
        if (blo == ORC_BC_PERIODIC) return ((c % n) + n) % n;
        if (blo == ORC_BC_ZEROGRAD) return 0;
        return -1 - c;  // symmetry mirror
    }
    if (c >= n) {
        if (bhi == ORC_BC_PERIODIC) return c % n;
        if (bhi == ORC_BC_ZEROGRAD) return n - 1;
        return 2 * n - 1 - c;
    }
    return c;
}

struct Grid {
    int ndim, n[3];
    double h;
    int bc[3][2];
    explicit Grid(const orc_config *c) : ndim(c->ndim), h(c->dx[0]) {
        for (int e = 0; e < 3; ++e) {
            n[e] = e < ndim ? c->n[e] : 1;
            bc[e][0] = c->bc[e][0];
            bc[e][1] = c->bc[e][1];
        }
    }
    long long ncell() const { return (long long)n[0] * n[1] * n[2]; }
    long long idx(int x, int y, int z) const { return ((long long)z * n[1] + y) * n[0] + x; }
    // value of a cell array at (possibly out-of-range) coordinates
    template <typename S> S at(const S *a, int x, int y, int z) const {
        const int c[3] = {x, y, z};
        int m[3];
        for (int e = 0; e < 3; ++e) m[e] = e < ndim ? map_index(c[e], n[e], bc[e][0], bc[e][1]) : 0;
        return a[idx(m[0], m[1], m[2])];
    }
    // the same along one axis from cell (x, y, z) moved by s along e
    template <typename S> S nb(const S *a, const int (&c)[3], int e, int s) const {
        int q[3] = {c[0], c[1], c[2]};
        q[e] += s;
        return at(a, q[0], q[1], q[2]);
    }
    long long nface(int d) const {
        long long f = 1;
        for (int e = 0; e < 3; ++e) f *= n[e] + (e == d ? 1 : 0);
        return f;
    }
};

// ---------------------------------------------------------------- geometry --
// Level set at the vertex with lower-corner cell (x, y, z) + 1/2 on every
// active axis: the mean of the 2^ndim cells sharing the vertex (linear
// interpolation to the vertex).
template <typename S> S vertex_phi(const Grid &g, const S *phi, int x, int y, int z) {
    S sum = S(0.0);
    const int nz = g.ndim == 3 ? 2 : 1, ny = g.ndim >= 2 ? 2 : 1;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < 2; ++i) sum = sum + g.at(phi, x + i, y + j, z + k);
    return sum / S((double)(2 * ny * nz));
}

// Fraction of an edge with phi > 0 from its end values (linear along the
// edge).
template <typename S> S edge_fraction(S a, S b) {
    const bool pa = val(a) > 0.0, pb = val(b) > 0.0;
    if (pa && pb) return S(1.0);
    if (!pa && !pb) return S(0.0);
    return pa ? a / (a - b) : b / (b - a);
}

// Fraction of a square face with phi > 0 from its corner values p[0..3]
// taken counter-clockwise: the region bounded by the face edges and straight
// segments between the edges' crossing points (phi linear along each edge).
// Two positive corners facing each other across the face (the saddle case)
// keep one triangle each, as the paper's aperture figure draws it; every
// other sign pattern gives one polygon, whose area is the shoelace sum.
template <typename S> S face_fraction(const S (&p)[4]) {
    int npos = 0;
    for (int k = 0; k < 4; ++k) npos += val(p[k]) > 0.0 ? 1 : 0;
    if (npos == 0) return S(0.0);
    if (npos == 4) return S(1.0);
    if (npos == 2 && (val(p[0]) > 0.0) == (val(p[2]) > 0.0)) {
        S area = S(0.0);
        for (int k = 0; k < 4; ++k) {
            if (!(val(p[k]) > 0.0)) continue;
            const S ta = p[k] / (p[k] - p[(k + 1) % 4]);  // along the edge to the next corner
            const S tb = p[k] / (p[k] - p[(k + 3) % 4]);  // along the edge to the previous corner
            area = area + S(0.5) * ta * tb;
        }
        return area;
    }
    static const double cx[4] = {0.0, 1.0, 1.0, 0.0}, cy[4] = {0.0, 0.0, 1.0, 1.0};
    S px[8], py[8];
    int m = 0;
    for (int k = 0; k < 4; ++k) {
        const int k1 = (k + 1) % 4;
        const bool pk = val(p[k]) > 0.0, pn = val(p[k1]) > 0.0;
        if (pk) {
            px[m] = S(cx[k]);
            py[m] = S(cy[k]);
            ++m;
        }
        if (pk != pn) {
            const S t = p[k] / (p[k] - p[k1]);
            px[m] = S(cx[k]) + t * S(cx[k1] - cx[k]);
            py[m] = S(cy[k]) + t * S(cy[k1] - cy[k]);
            ++m;
        }
    }
    S twice = S(0.0);
    for (int k = 0; k < m; ++k) {
        const int k1 = (k + 1) % m;
        twice = twice + (px[k] * py[k1] - px[k1] * py[k]);
    }
    return S(0.5) * twice;
}

// Aperture of face c (face c[d] between cells c[d]-1 and c[d]) of axis d.
template <typename S> S aperture(const Grid &g, const S *phi, int d, const int (&c)[3]) {
    // the vertex with lower-corner cell q has coordinates q + 1/2; the face's
    // vertices have q[d] = c[d] - 1 and q[e] in {c[e] - 1, c[e]} along the
    // face's axes
    if (g.ndim == 2) {
        const int e = 1 - d;
        int q[3] = {c[0], c[1], 0};
        q[d] = c[d] - 1;
        q[e] = c[e] - 1;
        const S a = vertex_phi(g, phi, q[0], q[1], q[2]);
        q[e] = c[e];
        const S b = vertex_phi(g, phi, q[0], q[1], q[2]);
        return edge_fraction(a, b);
    }
    const int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
    static const int o1[4] = {-1, 0, 0, -1}, o2[4] = {-1, -1, 0, 0};  // counter-clockwise in (e1, e2)
    S p[4];
    for (int k = 0; k < 4; ++k) {
        int q[3] = {c[0], c[1], c[2]};
        q[d] = c[d] - 1;
        q[e1] = c[e1] + o1[k];
        q[e2] = c[e2] + o2[k];
        p[k] = vertex_phi(g, phi, q[0], q[1], q[2]);
    }
    return face_fraction(p);
}

template <typename S>
void geometry(const Grid &g, const S *phi, S *apert, S *alpha, S *dgamma, S *normal) {
    const int nd = g.ndim;
    const double h = g.h;
    long long off[3] = {0, 0, 0};
    for (int d = 1; d < nd; ++d) off[d] = off[d - 1] + g.nface(d - 1);
    // apertures of every face of every axis
    for (int d = 0; d < nd; ++d) {
        int m[3] = {g.n[0], g.n[1], g.n[2]};
        m[d] += 1;
#pragma omp parallel for schedule(static) if (kParallel<S>)
        for (int z = 0; z < m[2]; ++z)
            for (int y = 0; y < m[1]; ++y)
                for (int x = 0; x < m[0]; ++x) {
                    const int c[3] = {x, y, z};
                    apert[off[d] + ((long long)z * m[1] + y) * m[0] + x] = aperture(g, phi, d, c);
                }
    }
    const double sface = nd == 3 ? h * h : h;   // face area (edge length in 2-D)
    const double vcell = nd == 3 ? h * h * h : h * h;
#pragma omp parallel for schedule(static) if (kParallel<S>)
    for (int z = 0; z < g.n[2]; ++z)
        for (int y = 0; y < g.n[1]; ++y)
            for (int x = 0; x < g.n[0]; ++x) {
                const long long i = g.idx(x, y, z);
                const int c[3] = {x, y, z};
                S am[3], ap[3];
                for (int d = 0; d < nd; ++d) {
                    int m[3] = {g.n[0], g.n[1], g.n[2]};
                    m[d] += 1;
                    int lo[3] = {x, y, z}, hi[3] = {x, y, z};
                    hi[d] += 1;
                    am[d] = apert[off[d] + ((long long)lo[2] * m[1] + lo[1]) * m[0] + lo[0]];
                    ap[d] = apert[off[d] + ((long long)hi[2] * m[1] + hi[1]) * m[0] + hi[0]];
                }
                // interface segment: |sum_d (A_{d+} - A_{d-}) S_d e_d| (App. D)
                S s2 = S(0.0);
                for (int d = 0; d < nd; ++d) {
                    const S t = (ap[d] - am[d]) * S(sface);
                    s2 = s2 + t * t;
                }
                const S dg = sqrt_(s2);
                dgamma[i] = dg;
                // volume fraction: pyramids (triangles in 2-D) from the cell
                // centre over the faces' positive parts (height h/2) and over
                // the interface facet (height phi at the centre), divided by
                // the cell volume; clipped to [0, 1]
                S vol = S(0.0);
                for (int d = 0; d < nd; ++d) vol = vol + (am[d] + ap[d]) * S(sface) * S(0.5 * h);
                vol = vol + dg * phi[i];
                S a = vol / S((double)nd * vcell);
                if (val(a) < 0.0) a = S(0.0);
                if (val(a) > 1.0) a = S(1.0);
                alpha[i] = a;
                // interface normal: 4th-order central gradient, normalised (0
                // where the gradient vanishes)
                S gr[3];
                S gg = S(0.0);
                for (int d = 0; d < nd; ++d) {
                    gr[d] = (g.nb(phi, c, d, -2) - S(8.0) * g.nb(phi, c, d, -1) + S(8.0) * g.nb(phi, c, d, 1) -
                             g.nb(phi, c, d, 2)) / S(12.0 * h);
                    gg = gg + gr[d] * gr[d];
                }
                const S gn = sqrt_(gg);
                for (int d = 0; d < nd; ++d)
                    normal[(long long)d * g.ncell() + i] = val(gn) > 0.0 ? gr[d] / gn : S(0.0);
            }
}

// --------------------------------------------------------------- advection --
// 5th-order upstream-central derivative of phi along d at cell c: the
// six-point stencil i-3..i+2 for u_d >= 0, its mirror i-2..i+3 for u_d < 0
// (coefficients (-2, 15, -60, 20, 30, -3)/60 and (3, -30, -20, 60, -15,
// 2)/60, the unique 6-point formulas exact for polynomials up to degree 5).
template <typename S> S houc5(const Grid &g, const S *phi, const int (&c)[3], int d, bool upwind_left) {
    if (upwind_left)
        return (S(-2.0) * g.nb(phi, c, d, -3) + S(15.0) * g.nb(phi, c, d, -2) - S(60.0) * g.nb(phi, c, d, -1) +
                S(20.0) * g.nb(phi, c, d, 0) + S(30.0) * g.nb(phi, c, d, 1) - S(3.0) * g.nb(phi, c, d, 2)) /
               S(60.0 * g.h);
    return (S(3.0) * g.nb(phi, c, d, -2) - S(30.0) * g.nb(phi, c, d, -1) - S(20.0) * g.nb(phi, c, d, 0) +
            S(60.0) * g.nb(phi, c, d, 1) - S(15.0) * g.nb(phi, c, d, 2) + S(2.0) * g.nb(phi, c, d, 3)) /
           S(60.0 * g.h);
}

// R_LSA = -u . grad(phi) (u: ndim arrays of cell velocities).
template <typename S> void advect_rhs(const Grid &g, const S *phi, const S *vel, S *rhs) {
    const long long nc = g.ncell();
#pragma omp parallel for schedule(static) if (kParallel<S>)
    for (int z = 0; z < g.n[2]; ++z)
        for (int y = 0; y < g.n[1]; ++y)
            for (int x = 0; x < g.n[0]; ++x) {
                const long long i = g.idx(x, y, z);
                const int c[3] = {x, y, z};
                S r = S(0.0);
                for (int d = 0; d < g.ndim; ++d) {
                    const S u = vel[(long long)d * nc + i];
                    r = r - u * houc5(g, phi, c, d, val(u) >= 0.0);
                }
                rhs[i] = r;
            }
}

// ---------------------------------------------------------- reinitialisation --
// Third-order WENO one-sided derivatives of phi along d at cell c (Jiang &
// Peng): from the backward differences v1, v2, v3 = D-phi at c-1, c, c+1
// the left-biased derivative combines (3 v2 - v1)/2 and (v2 + v3)/2 with
// the linear weights 1/3, 2/3 and the smoothness (v2 - v1)^2, (v3 - v2)^2;
// the right-biased one is the same formula on the mirrored differences.
template <typename S> S weno3_combine(S v1, S v2, S v3, double eps) {
    const S b0 = (v2 - v1) * (v2 - v1), b1 = (v3 - v2) * (v3 - v2);
    const S a0 = S(1.0 / 3.0) / ((S(eps) + b0) * (S(eps) + b0));
    const S a1 = S(2.0 / 3.0) / ((S(eps) + b1) * (S(eps) + b1));
    const S q0 = (S(3.0) * v2 - v1) / S(2.0), q1 = (v2 + v3) / S(2.0);
    return (a0 * q0 + a1 * q1) / (a0 + a1);
}
template <typename S> void weno3_hj(const Grid &g, const S *phi, const int (&c)[3], int d, S &dm, S &dp) {
    const S h = S(g.h);
    const S pm2 = g.nb(phi, c, d, -2), pm1 = g.nb(phi, c, d, -1), p0 = g.nb(phi, c, d, 0);
    const S pp1 = g.nb(phi, c, d, 1), pp2 = g.nb(phi, c, d, 2);
    dm = weno3_combine((pm1 - pm2) / h, (p0 - pm1) / h, (pp1 - p0) / h, 1e-6);
    dp = weno3_combine((pp2 - pp1) / h, (pp1 - p0) / h, (p0 - pm1) / h, 1e-6);
}

// R_reinit = -sgn(phi0) (|grad phi| - 1), |grad phi| from the Godunov
// Hamiltonian; 0 where |R| does not exceed the threshold.
template <typename S> void reinit_rhs(const Grid &g, const S *phi, const S *phi0, double thr, S *rhs) {
#pragma omp parallel for schedule(static) if (kParallel<S>)
    for (int z = 0; z < g.n[2]; ++z)
        for (int y = 0; y < g.n[1]; ++y)
            for (int x = 0; x < g.n[0]; ++x) {
                const long long i = g.idx(x, y, z);
                const int c[3] = {x, y, z};
                const double s = val(phi0[i]) > 0.0 ? 1.0 : (val(phi0[i]) < 0.0 ? -1.0 : 0.0);
                S h2 = S(0.0);
                for (int d = 0; d < g.ndim; ++d) {
                    S a, b;
                    weno3_hj(g, phi, c, d, a, b);
                    S t1, t2;
                    if (s > 0.0) {
                        t1 = val(a) > 0.0 ? a : S(0.0);  // max(a, 0)
                        t2 = val(b) < 0.0 ? b : S(0.0);  // min(b, 0)
                    } else {
                        t1 = val(a) < 0.0 ? a : S(0.0);  // min(a, 0)
                        t2 = val(b) > 0.0 ? b : S(0.0);  // max(b, 0)
                    }
                    const S q1 = t1 * t1, q2 = t2 * t2;
                    h2 = h2 + (val(q1) > val(q2) ? q1 : q2);
                }
                const S r = S(-s) * (sqrt_(h2) - S(1.0));
                rhs[i] = std::fabs(val(r)) > thr ? r : S(0.0);
            }
}

// ---------------------------------------------------------------- extension --
// One explicit Euler step (dtau) of dQ/dtau + a . grad Q = 0 for nq cell
// arrays q (each ncell long), first-order upwind per axis (backward
// difference where a_d > 0, forward where a_d < 0), with the advection
// velocity a = sdir(i) * n(i) (n: ndim cell arrays); cells with
// fixed(i) keep their values.
template <typename S>
void extend_step(const Grid &g, S *q, int nq, const S *n, const double *sdir, const unsigned char *fixed,
                 double dtau, std::vector<S> &tmp) {
    const long long nc = g.ncell();
    tmp.assign(q, q + (size_t)nq * nc);
#pragma omp parallel for schedule(static) if (kParallel<S>)
    for (int z = 0; z < g.n[2]; ++z)
        for (int y = 0; y < g.n[1]; ++y)
            for (int x = 0; x < g.n[0]; ++x) {
                const long long i = g.idx(x, y, z);
                if (fixed[i]) continue;
                const int c[3] = {x, y, z};
                for (int k = 0; k < nq; ++k) {
                    const S *qk = tmp.data() + (size_t)k * nc;
                    S r = S(0.0);
                    for (int d = 0; d < g.ndim; ++d) {
                        const S a = S(sdir[i]) * n[(long long)d * nc + i];
                        if (val(a) > 0.0) r = r + a * (qk[i] - g.nb(qk, c, d, -1)) / S(g.h);
                        else if (val(a) < 0.0) r = r + a * (g.nb(qk, c, d, 1) - qk[i]) / S(g.h);
                    }
                    q[(size_t)k * nc + i] = qk[i] - S(dtau) * r;
                }
            }
}

// Linearised two-material Riemann problem at the interface (App. D): with
// the acoustic impedances Z_p = rho_p c_p and the normal velocities
// un_p = u_p . n (n = grad phi/|grad phi| points into phase 1, the positive
// phase), u_Gamma = (Z1 un1 + Z2 un2 + p2 - p1)/(Z1 + Z2) (along n) and
// p_Gamma = (Z1 p2 + Z2 p1 + Z1 Z2 (un2 - un1))/(Z1 + Z2); no surface
// tension.
template <typename S> void interface_riemann(S Z1, S un1, S p1, S Z2, S un2, S p2, S &ug, S &pg) {
    const S zs = Z1 + Z2;
    ug = (Z1 * un1 + Z2 * un2 + p2 - p1) / zs;
    pg = (Z1 * p2 + Z2 * p1 + Z1 * Z2 * (un2 - un1)) / zs;
}

// ------------------------------------------------------- cut-cell right side --
// The right-hand side of phase p in every cell (Eq. FVD_levelset, inviscid,
// no surface tension) for the phase's primitive field W (extended into its
// ghost cells): the face fluxes F^p of the configured reconstruction and HLLC
// from W, weighted by the phase's apertures (A for phase 1 = phi > 0, 1 - A
// for phase 2), and the interface flux: the interface pressure pushes each
// phase along its inward normal (+n for phase 1, -n for phase 2, n pointing
// into phase 1) with the force p_G dGamma and the power p_G dGamma u_G,
// u_G = u_Gamma . n.  dU is d(alpha U)/dt of the phase.
void cut_rhs(const orc_config &c, const double *phi, const double *W, int phase, const double *ug,
             const double *pg, double *dU) {
    const Layout L(c);
    const int nv = L.nv, nd = L.ndim;
    const Grid g(&c);
    const long long nc = g.ncell();
    std::vector<double> ap(0), al(nc), dg(nc), nr((size_t)nd * nc);
    long long nfa = 0;
    for (int d = 0; d < nd; ++d) nfa += g.nface(d);
    ap.resize(nfa);
    geometry(g, phi, ap.data(), al.data(), dg.data(), nr.data());
    // the phase's primitives on the padded grid, halos by the boundary conditions
    std::vector<double> Wp((size_t)nv * L.npad);
    for (int z = 0; z < L.n[2]; ++z)
        for (int y = 0; y < L.n[1]; ++y)
            for (int x = 0; x < L.n[0]; ++x)
                for (int v = 0; v < nv; ++v) Wp[v * L.npad + L.pidx(x, y, z)] = W[v * L.ncell + L.cidx(x, y, z)];
    fill_halos(c, L, Wp);
    for (long long i = 0; i < (long long)nv * nc; ++i) dU[i] = 0.0;
    long long off = 0;
    for (int d = 0; d < nd; ++d) {
        int m[3] = {L.n[0], L.n[1], L.n[2]};
        m[d] += 1;
        const long nface = (long)m[0] * m[1] * m[2];
        std::vector<double> F((size_t)nv * nface);
        const long sd = L.pstride(d);
#pragma omp parallel for schedule(static)
        for (long f = 0; f < nface; ++f) {
            const int q[3] = {(int)(f % m[0]), (int)((f / m[0]) % m[1]), (int)(f / ((long)m[0] * m[1]))};
            const long pR = L.pidx(q[0], q[1], q[2]);
            const long pL = pR - sd;
            double Ws[6][NVMAX];
            for (int j = 0; j < 6; ++j)
                for (int v = 0; v < nv; ++v) Ws[j][v] = Wp[v * L.npad + pL + (j - 2) * sd];
            double WL[NVMAX], WR[NVMAX];
            if (c.recon == ORC_CHAR) reconstruct_char(c, L, d, Ws, WL, WR);
            else reconstruct_comp(c, L, Ws, WL, WR);
            double Ff[NVMAX], uh;
            hllc(c, L, d, WL, WR, Ff, uh);
            for (int v = 0; v < nv; ++v) F[v * nface + f] = Ff[v];
        }
        const double dxd = c.dx[d];
        const long fs = (d == 0) ? 1 : (d == 1 ? m[0] : (long)m[0] * m[1]);
        for (long i = 0; i < (long)nc; ++i) {
            const int q[3] = {(int)(i % L.n[0]), (int)((i / L.n[0]) % L.n[1]), (int)(i / ((long)L.n[0] * L.n[1]))};
            const long gm = ((long)q[2] * m[1] + q[1]) * m[0] + q[0];  // face i-1/2
            const long gp = gm + fs;                                   // face i+1/2
            double am = ap[off + gm], apx = ap[off + gp];
            if (phase == 2) {
                am = 1.0 - am;
                apx = 1.0 - apx;
            }
            for (int v = 0; v < nv; ++v)
                dU[v * nc + i] = dU[v * nc + i] - (apx * F[v * nface + gp] - am * F[v * nface + gm]) / dxd;
        }
        off += g.nface(d);
    }
    // interface flux (cut cells only: dGamma = 0 elsewhere)
    const double vol = nd == 3 ? c.dx[0] * c.dx[1] * c.dx[2] : c.dx[0] * c.dx[1];
    const double sp = phase == 1 ? 1.0 : -1.0;
    for (long long i = 0; i < nc; ++i) {
        if (!(dg[i] > 0.0)) continue;
        double un = 0.0;
        for (int d = 0; d < nd; ++d) un += ug[(long long)d * nc + i] * nr[(long long)d * nc + i];
        const double force = sp * pg[i] * dg[i] / vol;
        for (int d = 0; d < nd; ++d) dU[(1 + d) * nc + i] = dU[(1 + d) * nc + i] + force * nr[(long long)d * nc + i];
        dU[(1 + nd) * nc + i] = dU[(1 + nd) * nc + i] + force * un;
    }
}

// ------------------------------------------------------------------ mixing --
// Conservative mixing (App. D) of one phase's volume-weighted state aU (nv
// cell arrays of alpha U) after a stage, with the phase's volume fraction
// before (a0) and after (a1) the stage and its inward normal n^p (ndim cell
// arrays).  A cell mixes when it vanished (a1 = 0, a0 > 0), is new (a1 > 0,
// a0 = 0) or is small (a1 < amix).  Its targets are the neighbours one step
// along sign(n^p) on each axis, each pair of axes and all three (ndim = 2:
// x, y, xy); a target outside a non-periodic side gets no weight.  Weights
// beta_x = |n_x|^2 a_t, beta_xy = |n_x n_y| a_t, beta_xyz = |n_x n_y n_z|^(2/3)
// a_t (a_t the target's fraction after the stage), normalised to sum 1 (no
// mixing when they are all 0); the fluxes M_t = beta_t/(a beta_t + a_t)
// [(a_t U_t) a - (a U) a_t] from the states before mixing are added to the
// cell and taken from its targets.
void mix(const Grid &g, int nv, const double *a0, const double *a1, const double *np, double amix, double *aU) {
    const long long nc = g.ncell();
    const int nd = g.ndim;
    std::vector<double> star(aU, aU + (size_t)nv * nc);
    for (int z = 0; z < g.n[2]; ++z)
        for (int y = 0; y < g.n[1]; ++y)
            for (int x = 0; x < g.n[0]; ++x) {
                const long long i = g.idx(x, y, z);
                const bool mixing = (a1[i] == 0.0 && a0[i] > 0.0) || (a1[i] > 0.0 && a0[i] == 0.0) || a1[i] < amix;
                if (!mixing) continue;
                int sgn[3] = {0, 0, 0};
                double an[3] = {0.0, 0.0, 0.0};
                for (int d = 0; d < nd; ++d) {
                    const double nd_ = np[(long long)d * nc + i];
                    sgn[d] = nd_ > 0.0 ? 1 : (nd_ < 0.0 ? -1 : 0);
                    an[d] = std::fabs(nd_);
                }
                // the targets: every non-empty subset of the axes
                const int ntrg = nd == 3 ? 7 : 3;
                long long ti[7];
                double beta[7], at[7];
                double bsum = 0.0;
                for (int t = 0; t < ntrg; ++t) {
                    const int mask = t + 1;  // bit e: step along axis e
                    int q[3] = {x, y, z};
                    bool inside = true;
                    double w = 1.0;
                    int nbits = 0;
                    for (int e = 0; e < nd; ++e) {
                        if (!((mask >> e) & 1)) continue;
                        ++nbits;
                        if (sgn[e] == 0) inside = false;
                        q[e] += sgn[e];
                        if (q[e] < 0 || q[e] >= g.n[e]) {
                            if (g.bc[e][0] == ORC_BC_PERIODIC) q[e] = (q[e] + g.n[e]) % g.n[e];
                            else inside = false;
                        }
                        w *= an[e];
                    }
                    if (nbits == 1) w = w * w;                 // |n . e|^2
                    else if (nbits == 3) w = std::cbrt(w * w);  // |n_x n_y n_z|^(2/3)
                    ti[t] = inside ? g.idx(q[0], q[1], q[2]) : -1;
                    at[t] = inside ? a1[ti[t]] : 0.0;
                    beta[t] = inside ? w * at[t] : 0.0;
                    bsum += beta[t];
                }
                if (!(bsum > 0.0)) continue;
                for (int t = 0; t < ntrg; ++t) {
                    if (ti[t] < 0 || beta[t] == 0.0) continue;
                    const double b = beta[t] / bsum;
                    const double f = b / (a1[i] * b + at[t]);
                    for (int v = 0; v < nv; ++v) {
                        const double M = f * (star[(size_t)v * nc + ti[t]] * a1[i] - star[(size_t)v * nc + i] * at[t]);
                        aU[(size_t)v * nc + i] += M;
                        aU[(size_t)v * nc + ti[t]] -= M;
                    }
                }
            }
}

}  // namespace

// ------------------------------------------------------------- C interface --
// A cut cell holds an interface segment (Sec. 3.5): both phases have volume
// in it, or the interface runs along one of its faces (the cell on the side
// whose aperture drops to 0 there has alpha = 1 and dGamma = h^(ndim-1)).
static bool is_cut(double alpha, double dgamma) { return (alpha > 0.0 && alpha < 1.0) || dgamma > 0.0; }

static bool ls_ok(const orc_config *c) {
    if (c->ndim < 2 || c->ndim > 3) return false;
    for (int e = 1; e < c->ndim; ++e)
        if (c->dx[e] != c->dx[0]) return false;
    return true;
}

}  // namespace orc

using orc::Grid;

extern "C" {

long long orc_ls_nface(const orc_config *c) {
    if (!orc::ls_ok(c)) return -1;
    Grid g(c);
    long long s = 0;
    for (int d = 0; d < g.ndim; ++d) s += g.nface(d);
    return s;
}

int orc_ls_geometry(const orc_config *c, const double *phi, double *apert, double *alpha, double *dgamma,
                    double *normal) {
    if (!orc::ls_ok(c)) return -1;
    orc::geometry(Grid(c), phi, apert, alpha, dgamma, normal);
    return 0;
}

double orc_ls_face_fraction(const double *p4) {
    const double p[4] = {p4[0], p4[1], p4[2], p4[3]};
    return orc::face_fraction(p);
}

int orc_ls_rhs(const orc_config *c, const double *phi, const double *vel, double *rhs) {
    if (!orc::ls_ok(c)) return -1;
    orc::advect_rhs(Grid(c), phi, vel, rhs);
    return 0;
}

int orc_ls_advect(const orc_config *c, double *phi, const double *vel, double dt, int nsteps) {
    if (!orc::ls_ok(c)) return -1;
    Grid g(c);
    const long long n = g.ncell();
    std::vector<double> p0(n), r(n), p1(n);
    for (int step = 0; step < nsteps; ++step) {
        // TVD-RK3 (§3.4): p1 = p + dt R(p); p2 = 3/4 p + 1/4 (p1 + dt R(p1));
        // p^{n+1} = 1/3 p + 2/3 (p2 + dt R(p2))
        std::copy(phi, phi + n, p0.begin());
        orc::advect_rhs(g, phi, vel, r.data());
        for (long long i = 0; i < n; ++i) p1[i] = p0[i] + dt * r[i];
        orc::advect_rhs(g, p1.data(), vel, r.data());
        for (long long i = 0; i < n; ++i) p1[i] = 0.75 * p0[i] + 0.25 * (p1[i] + dt * r[i]);
        orc::advect_rhs(g, p1.data(), vel, r.data());
        for (long long i = 0; i < n; ++i) phi[i] = (1.0 / 3.0) * p0[i] + (2.0 / 3.0) * (p1[i] + dt * r[i]);
    }
    return 0;
}

int orc_ls_reinit_rhs(const orc_config *c, const double *phi, const double *phi0, double threshold,
                      double *rhs) {
    if (!orc::ls_ok(c)) return -1;
    orc::reinit_rhs(Grid(c), phi, phi0, threshold, rhs);
    return 0;
}

int orc_ls_reinit(const orc_config *c, double *phi, int steps, double threshold) {
    if (!orc::ls_ok(c)) return -1;
    Grid g(c);
    const long long n = g.ncell();
    const double dtau = 0.25 * g.h;
    std::vector<double> p0(phi, phi + n), pn(n), r(n), p1(n);
    for (int it = 0; it < steps; ++it) {
        // second-order TVD Runge-Kutta in pseudo-time: p1 = p + dtau R(p);
        // p^{n+1} = 1/2 p + 1/2 (p1 + dtau R(p1))
        std::copy(phi, phi + n, pn.begin());
        orc::reinit_rhs(g, phi, p0.data(), threshold, r.data());
        for (long long i = 0; i < n; ++i) p1[i] = pn[i] + dtau * r[i];
        orc::reinit_rhs(g, p1.data(), p0.data(), threshold, r.data());
        for (long long i = 0; i < n; ++i) phi[i] = 0.5 * pn[i] + 0.5 * (p1[i] + dtau * r[i]);
    }
    return 0;
}

int orc_ls_count_flops(const orc_config *c, const double *phi, const double *vel, double *out) {
    // out[0] geometry, out[1] one advection right-hand side, out[2] one
    // reinitialisation right-hand side (phi0 = phi), totals over the grid;
    // out[3], out[4] the flops of one advection RK3 stage combination and of
    // one reinitialisation RK2 stage combination per cell (the mean of the
    // stage forms)
    if (!orc::ls_ok(c)) return -1;
    using orc::Counted;
    Grid g(c);
    const long long n = g.ncell();
    std::vector<Counted> p(n), v((size_t)g.ndim * n), r(n), ap, al(n), dg(n), nr((size_t)g.ndim * n);
    for (long long i = 0; i < n; ++i) p[i] = Counted(phi[i]);
    for (long long i = 0; i < (long long)g.ndim * n; ++i) v[i] = Counted(vel[i]);
    long long nf = 0;
    for (int d = 0; d < g.ndim; ++d) nf += g.nface(d);
    ap.resize(nf);
    orc::FlopTally &t = orc::tally();
    t = orc::FlopTally();
    orc::geometry(g, p.data(), ap.data(), al.data(), dg.data(), nr.data());
    out[0] = (double)t.total();
    t = orc::FlopTally();
    orc::advect_rhs(g, p.data(), v.data(), r.data());
    out[1] = (double)t.total();
    t = orc::FlopTally();
    orc::reinit_rhs(g, p.data(), p.data(), 5e-2, r.data());
    out[2] = (double)t.total();
    // RK3 stages: p + dt r (2); 3/4 p + 1/4 (p1 + dt r) (5); 1/3 p + 2/3 (p2 + dt r) (5)
    out[3] = (2.0 + 5.0 + 5.0) / 3.0;
    // RK2 stages: p + dtau r (2); 1/2 p + 1/2 (p1 + dtau r) (5)
    out[4] = (2.0 + 5.0) / 2.0;
    return 0;
}

void orc_ls_interface_riemann(const double *in, double *ug, double *pg) {
    // in: Z1, un1, p1, Z2, un2, p2
    orc::interface_riemann(in[0], in[1], in[2], in[3], in[4], in[5], *ug, *pg);
}

int orc_ls_interface_quantities(const orc_config *c, const double *phi, const double *W1, const double *W2,
                                const double *gamma, const double *pinf, double *ug, double *pg) {
    // per cut cell (a cell holding an interface segment: 0 < alpha < 1 or
    // dGamma > 0, the latter where the interface runs along one of its
    // faces): the interface velocity (ndim arrays, u_Gamma n) and pressure
    // from the two phases' primitives (rho, u_d, p) at the cell; 0 in every
    // other cell
    if (!orc::ls_ok(c)) return -1;
    Grid g(c);
    const long long nc = g.ncell();
    const int nd = g.ndim;
    std::vector<double> ap((size_t)orc_ls_nface(c)), al(nc), dg(nc), nr((size_t)nd * nc);
    orc::geometry(g, phi, ap.data(), al.data(), dg.data(), nr.data());
    for (long long i = 0; i < nc; ++i) {
        for (int d = 0; d < nd; ++d) ug[(long long)d * nc + i] = 0.0;
        pg[i] = 0.0;
        if (!orc::is_cut(al[i], dg[i])) continue;
        double Z[2], un[2], p[2];
        const double *Wp[2] = {W1, W2};
        for (int k = 0; k < 2; ++k) {
            const double rho = Wp[k][i], pk = Wp[k][(long long)(1 + nd) * nc + i];
            double u = 0.0;
            for (int d = 0; d < nd; ++d) u += Wp[k][(long long)(1 + d) * nc + i] * nr[(long long)d * nc + i];
            Z[k] = rho * std::sqrt(gamma[k] * (pk + pinf[k]) / rho);  // rho c, c^2 = gamma (p + p_inf)/rho
            un[k] = u;
            p[k] = pk;
        }
        double u_g, p_g;
        orc::interface_riemann(Z[0], un[0], p[0], Z[1], un[1], p[1], u_g, p_g);
        for (int d = 0; d < nd; ++d) ug[(long long)d * nc + i] = u_g * nr[(long long)d * nc + i];
        pg[i] = p_g;
    }
    return 0;
}

int orc_ls_extend(const orc_config *c, const double *phi, double *q, int nq, int mode, int steps) {
    // mode 0 / 1: ghost cells of phase 1 / 2 (the primitives, Eq.
    // extension_prime): dW/dtau = n^p . grad W, i.e. advection with a =
    // -n^p (n^1 = n, n^2 = -n), in the cells where the phase has no volume
    // (alpha^p = 0); mode 2: interface quantities (Eq. extension_if),
    // dQ/dtau = -sgn(phi) n . grad Q, in every cell that is not a cut cell
    // (0 < alpha < 1 or dGamma > 0).
    // dtau = 0.25 h, explicit Euler, first-order upwind; n, alpha from
    // phi's geometry.
    if (!orc::ls_ok(c) || mode < 0 || mode > 2 || nq < 1) return -1;
    Grid g(c);
    const long long nc = g.ncell();
    const int nd = g.ndim;
    std::vector<double> ap((size_t)orc_ls_nface(c)), al(nc), dg(nc), nr((size_t)nd * nc), sdir(nc);
    std::vector<unsigned char> fixed(nc);
    orc::geometry(g, phi, ap.data(), al.data(), dg.data(), nr.data());
    for (long long i = 0; i < nc; ++i) {
        if (mode == 0) {
            sdir[i] = -1.0;
            fixed[i] = al[i] > 0.0;  // phase 1 present
        } else if (mode == 1) {
            sdir[i] = 1.0;
            fixed[i] = al[i] < 1.0;  // phase 2 present
        } else {
            sdir[i] = phi[i] > 0.0 ? 1.0 : (phi[i] < 0.0 ? -1.0 : 0.0);
            fixed[i] = orc::is_cut(al[i], dg[i]);
        }
    }
    std::vector<double> tmp;
    for (int it = 0; it < steps; ++it) orc::extend_step(g, q, nq, nr.data(), sdir.data(), fixed.data(), 0.25 * g.h, tmp);
    return 0;
}

int orc_ls_cut_rhs(const orc_config *c, const double *phi, const double *W, int phase, const double *ug,
                   const double *pg, double *dU) {
    if (!orc::ls_ok(c) || c->model != ORC_SPM || c->viscous || c->limiter || (phase != 1 && phase != 2)) return -1;
    orc::cut_rhs(*c, phi, W, phase, ug, pg, dU);
    return 0;
}

int orc_ls_mix(const orc_config *c, int nv, const double *a0, const double *a1, const double *np, double amix,
               double *aU) {
    if (!orc::ls_ok(c) || nv < 1) return -1;
    orc::mix(Grid(c), nv, a0, a1, np, amix, aU);
    return 0;
}

// ------------------------------------------------------- the level-set step --
// Interface quantities (App. D) of the cut cells from W1, W2 (rho, u_d, p)
// and the geometry (al, dg, nr), as orc_ls_interface_quantities computes
// them; 0 in every other cell.
static void ls_q(const orc_config *c1, const orc_config *c2, const Grid &g, const double *al, const double *dg,
                 const double *nr, const double *W1, const double *W2, double *ug, double *pg) {
    const long long nc = g.ncell();
    const int nd = g.ndim;
    const double gam[2] = {c1->gamma[0], c2->gamma[0]}, pin[2] = {c1->pinf[0], c2->pinf[0]};
    for (long long i = 0; i < nc; ++i) {
        for (int d = 0; d < nd; ++d) ug[(long long)d * nc + i] = 0.0;
        pg[i] = 0.0;
        if (!orc::is_cut(al[i], dg[i])) continue;
        double Z[2], un[2], p[2];
        const double *Wp[2] = {W1, W2};
        for (int k = 0; k < 2; ++k) {
            const double rho = Wp[k][i], pk = Wp[k][(long long)(1 + nd) * nc + i];
            double u = 0.0;
            for (int d = 0; d < nd; ++d) u += Wp[k][(long long)(1 + d) * nc + i] * nr[(long long)d * nc + i];
            Z[k] = rho * std::sqrt(gam[k] * (pk + pin[k]) / rho);
            un[k] = u;
            p[k] = pk;
        }
        double u_g, p_g;
        orc::interface_riemann(Z[0], un[0], p[0], Z[1], un[1], p[1], u_g, p_g);
        for (int d = 0; d < nd; ++d) ug[(long long)d * nc + i] = u_g * nr[(long long)d * nc + i];
        pg[i] = p_g;
    }
}

// steps extension steps (§3.5; modes 0, 1, 2 as orc_ls_extend) of nq
// arrays with the given geometry.
static void ls_ext(const Grid &g, const double *phi, const double *al, const double *dg, const double *nr, double *q,
                   int nq, int mode, int steps) {
    const long long nc = g.ncell();
    std::vector<double> sdir(nc);
    std::vector<unsigned char> fixed(nc);
    for (long long i = 0; i < nc; ++i) {
        if (mode == 0) {
            sdir[i] = -1.0;
            fixed[i] = al[i] > 0.0;
        } else if (mode == 1) {
            sdir[i] = 1.0;
            fixed[i] = al[i] < 1.0;
        } else {
            sdir[i] = phi[i] > 0.0 ? 1.0 : (phi[i] < 0.0 ? -1.0 : 0.0);
            fixed[i] = orc::is_cut(al[i], dg[i]);
        }
    }
    std::vector<double> tmp;
    for (int it = 0; it < steps; ++it) orc::extend_step(g, q, nq, nr, sdir.data(), fixed.data(), 0.25 * g.h, tmp);
}

// Primitives of a phase from its volume-weighted state (Alg. 2: W^p =
// cons2prim(alpha^p U^p / alpha^p)) in every cell holding it (ap_ > 0);
// the other cells keep W.
static void ls_prim(const orc_config *cp, const Grid &g, const double *ap_, const double *aU, double *W) {
    const orc::Layout L(*cp);
    const long long nc = g.ncell();
    const int nv = L.nv;
    for (long long i = 0; i < nc; ++i) {
        if (!(ap_[i] > 0.0)) continue;
        double u[orc::NVMAX], w[orc::NVMAX];
        for (int v = 0; v < nv; ++v) u[v] = aU[(long long)v * nc + i] / ap_[i];
        orc::cons2prim(*cp, L, u, w);
        for (int v = 0; v < nv; ++v) W[(long long)v * nc + i] = w[v];
    }
}

int orc_ls_init(const orc_config *c1, const orc_config *c2, const double *phi, const double *W1, const double *W2,
                double *aU1, double *aU2, double *ug, double *pg) {
    // from phi and the two phases' primitives (given in every cell): the
    // volume-weighted states alpha^p U(W^p) and the extended interface
    // quantities
    if (!orc::ls_ok(c1) || !orc::ls_ok(c2)) return -1;
    Grid g(c1);
    const long long nc = g.ncell();
    const int nd = g.ndim, nv = nd + 2;
    std::vector<double> ap((size_t)orc_ls_nface(c1)), al(nc), dg(nc), nr((size_t)nd * nc);
    orc::geometry(g, phi, ap.data(), al.data(), dg.data(), nr.data());
    const orc::Layout L1(*c1), L2(*c2);
    for (long long i = 0; i < nc; ++i) {
        double w[orc::NVMAX], u[orc::NVMAX];
        for (int v = 0; v < nv; ++v) w[v] = W1[(long long)v * nc + i];
        orc::prim2cons(*c1, L1, w, u);
        for (int v = 0; v < nv; ++v) aU1[(long long)v * nc + i] = al[i] * u[v];
        for (int v = 0; v < nv; ++v) w[v] = W2[(long long)v * nc + i];
        orc::prim2cons(*c2, L2, w, u);
        for (int v = 0; v < nv; ++v) aU2[(long long)v * nc + i] = (1.0 - al[i]) * u[v];
    }
    ls_q(c1, c2, g, al.data(), dg.data(), nr.data(), W1, W2, ug, pg);
    std::vector<double> q((size_t)(nd + 1) * nc);
    std::copy(ug, ug + (size_t)nd * nc, q.begin());
    std::copy(pg, pg + nc, q.begin() + (size_t)nd * nc);
    ls_ext(g, phi, al.data(), dg.data(), nr.data(), q.data(), nd + 1, 2, 20);
    std::copy(q.begin(), q.begin() + (size_t)nd * nc, ug);
    std::copy(q.begin() + (size_t)nd * nc, q.end(), pg);
    return 0;
}

int orc_ls_step(const orc_config *c1, const orc_config *c2, double dt, int nsteps, double amix, double *phi,
                double *aU1, double *aU2, double *W1, double *W2, double *ug, double *pg) {
    // nsteps TVD-RK3 steps of the level-set model (Alg. 2, inviscid, no
    // surface tension); each stage: the cut-cell right-hand sides of both
    // phases and the level-set advection with the interface velocity, the
    // stage combinations, the reinitialisation after the last stage, the
    // mixing of both phases against the new geometry, the primitives of the
    // cells holding each phase, their extension into the ghost cells, the
    // interface quantities and their extension
    if (!orc::ls_ok(c1) || !orc::ls_ok(c2)) return -1;
    Grid g(c1);
    const long long nc = g.ncell();
    const int nd = g.ndim, nv = nd + 2;
    const long long nf = orc_ls_nface(c1);
    std::vector<double> ap(nf), al0(nc), al1(nc), dg(nc), nr((size_t)nd * nc), nr2((size_t)nd * nc);
    std::vector<double> R1((size_t)nv * nc), R2((size_t)nv * nc), Rp(nc);
    std::vector<double> U1n((size_t)nv * nc), U2n((size_t)nv * nc), phin(nc), a0p(nc), a1p(nc);
    std::vector<double> q((size_t)(nd + 1) * nc);
    static const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0};
    for (int step = 0; step < nsteps; ++step) {
        std::copy(aU1, aU1 + (size_t)nv * nc, U1n.begin());
        std::copy(aU2, aU2 + (size_t)nv * nc, U2n.begin());
        std::copy(phi, phi + nc, phin.begin());
        for (int stage = 0; stage < 3; ++stage) {
            orc::geometry(g, phi, ap.data(), al0.data(), dg.data(), nr.data());
            orc::cut_rhs(*c1, phi, W1, 1, ug, pg, R1.data());
            orc::cut_rhs(*c2, phi, W2, 2, ug, pg, R2.data());
            orc::advect_rhs(g, phi, ug, Rp.data());
            for (long long k = 0; k < (long long)nv * nc; ++k) {
                if (stage == 0) {
                    aU1[k] = aU1[k] + dt * R1[k];
                    aU2[k] = aU2[k] + dt * R2[k];
                } else {
                    aU1[k] = ca[stage] * U1n[k] + cb[stage] * (aU1[k] + dt * R1[k]);
                    aU2[k] = ca[stage] * U2n[k] + cb[stage] * (aU2[k] + dt * R2[k]);
                }
            }
            for (long long i = 0; i < nc; ++i)
                phi[i] = stage == 0 ? phi[i] + dt * Rp[i] : ca[stage] * phin[i] + cb[stage] * (phi[i] + dt * Rp[i]);
            if (stage == 2) orc_ls_reinit(c1, phi, 10, 5e-2);
            orc::geometry(g, phi, ap.data(), al1.data(), dg.data(), nr.data());
            for (long long k = 0; k < (long long)nd * nc; ++k) nr2[k] = -nr[k];
            orc::mix(g, nv, al0.data(), al1.data(), nr.data(), amix, aU1);
            for (long long i = 0; i < nc; ++i) {
                a0p[i] = 1.0 - al0[i];
                a1p[i] = 1.0 - al1[i];
            }
            orc::mix(g, nv, a0p.data(), a1p.data(), nr2.data(), amix, aU2);
            ls_prim(c1, g, al1.data(), aU1, W1);
            ls_prim(c2, g, a1p.data(), aU2, W2);
            ls_ext(g, phi, al1.data(), dg.data(), nr.data(), W1, nv, 0, 10);
            ls_ext(g, phi, al1.data(), dg.data(), nr.data(), W2, nv, 1, 10);
            ls_q(c1, c2, g, al1.data(), dg.data(), nr.data(), W1, W2, ug, pg);
            std::copy(ug, ug + (size_t)nd * nc, q.begin());
            std::copy(pg, pg + nc, q.begin() + (size_t)nd * nc);
            ls_ext(g, phi, al1.data(), dg.data(), nr.data(), q.data(), nd + 1, 2, 20);
            std::copy(q.begin(), q.begin() + (size_t)nd * nc, ug);
            std::copy(q.begin() + (size_t)nd * nc, q.end(), pg);
        }
    }
    return 0;
}

void orc_ls_weno3_hj(const double *v5, double h, double *dm, double *dp) {
    // v5 = phi at i-2..i+2 along one axis (a 1-D helper for the unit pins)
    const double a = (v5[1] - v5[0]) / h, b = (v5[2] - v5[1]) / h, c3 = (v5[3] - v5[2]) / h,
                 d4 = (v5[4] - v5[3]) / h;
    *dm = orc::weno3_combine(a, b, c3, 1e-6);
    *dp = orc::weno3_combine(d4, c3, b, 1e-6);
}

}  // extern "C"
