// jxf_ls.cu -- the level-set model (§3.5, §3.6, App. D, Alg. 2), FP64, on
// device arrays of a grid of cubic cells (2-D or 3-D):
//   jxf_ls_geometry   apertures, interface segment, volume fraction, normal
//   jxf_ls_rhs        R = -u . grad(phi) (5th-order upstream-central)
//   jxf_ls_advect     TVD-RK3 steps of the level-set advection
//   jxf_ls_reinit     pseudo-time steps of the reinitialisation equation
//   jxf_ls_interface  interface velocity and pressure of the cut cells
//   jxf_ls_extend     ghost-cell and interface-quantity extension
//   jxf_ls_cut_rhs    cut-cell right-hand side of one phase
//   jxf_ls_mix        conservative mixing of one phase
//   jxf_ls_init, jxf_ls_step   the two-phase time step chaining them
// One thread per cell (x fastest, 256 a block) or per face; indices outside
// the grid map through the boundary conditions (a mirror copies the
// scalar).  Every kernel is bound by the FP64 pipe: compares, divisions and
// square roots are kept off it where an integer test or a reciprocal does.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "jxf.h"
#include "jxf_impl.cuh"  // fdiv; the face flux of the finite-volume scheme
#include "jxf_nvtx.cuh"
#include "jxf_setup.cuh"

namespace {

constexpr int kLsThreads = 256;

struct LsGrid {
    int ndim, n[3];
    int bc[3][2];
    double h, ih;  // cell size and its reciprocal
    long long ncell;
    long long stride[3];  // cell-index step of each axis
    long long foff[3];    // offset of axis d's face array in the concatenated apertures
};

__device__ __forceinline__ int ls_map(int c, int n, int blo, int bhi) {
    if (c < 0) {
        if (blo == JXF_BC_PERIODIC) return ((c % n) + n) % n;
        if (blo == JXF_BC_ZEROGRAD) return 0;
        return -1 - c;
    }
    if (c >= n) {
        if (bhi == JXF_BC_PERIODIC) return c % n;
        if (bhi == JXF_BC_ZEROGRAD) return n - 1;
        return 2 * n - 1 - c;
    }
    return c;
}

// phi at cell i moved by s along d (one boundary mapping)
__device__ __forceinline__ double ls_line(const LsGrid &g, const double *__restrict__ a, long long i, int cd, int d,
                                          int s) {
    const int m = ls_map(cd + s, g.n[d], g.bc[d][0], g.bc[d][1]);
    return __ldg(a + i + (long long)(m - cd) * g.stride[d]);
}

// cell coordinates of index i (32-bit arithmetic: ncell < 2^31)
__device__ __forceinline__ void ls_cell(const LsGrid &g, long long i, int (&c)[3]) {
    const unsigned u = (unsigned)i, n0 = (unsigned)g.n[0], n1 = (unsigned)g.n[1];
    const unsigned q = u / n0, r = q / n1;
    c[0] = (int)(u - q * n0);
    c[1] = (int)(q - r * n1);
    c[2] = (int)r;
}

// Sign tests and compares of doubles on their bit patterns (integer pipe;
// FP64 compares take slots of the narrow FP64 pipe), each equal to the
// FP64 compare for operands that are not NaN: x > 0, x < 0, and x > y for
// x, y >= 0 (non-negative doubles order as their bit patterns).
__device__ __forceinline__ bool ls_pos(double x) { return __double_as_longlong(x) > 0; }
__device__ __forceinline__ bool ls_neg(double x) {
    const long long b = __double_as_longlong(x);
    return b < 0 && (b << 1) != 0;
}
__device__ __forceinline__ bool ls_gt_nonneg(double x, double y) {
    return __double_as_longlong(x) > __double_as_longlong(y);
}

// ---------------------------------------------------------------- geometry --
// Fraction of an edge with phi > 0 (linear along the edge).
__device__ __forceinline__ double edge_fraction(double a, double b) {
    const bool pa = ls_pos(a), pb = ls_pos(b);
    if (pa && pb) return 1.0;
    if (!pa && !pb) return 0.0;
    return pa ? a / (a - b) : b / (b - a);
}

// Fraction of a square face with phi > 0 from its corner values
// (counter-clockwise from the face's lower corner): the polygon bounded by
// the face's edges and straight segments between the edges' zero crossings;
// two positive corners facing each other keep one triangle each.
__device__ double face_fraction(const double (&p)[4]) {
    int npos = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) npos += ls_pos(p[k]) ? 1 : 0;
    if (npos == 0) return 0.0;
    if (npos == 4) return 1.0;
    if (npos == 2 && ls_pos(p[0]) == ls_pos(p[2])) {
        double area = 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!ls_pos(p[k])) continue;
            const double ta = p[k] / (p[k] - p[(k + 1) & 3]);
            const double tb = p[k] / (p[k] - p[(k + 3) & 3]);
            area += 0.5 * ta * tb;
        }
        return area;
    }
    const double cx[4] = {0.0, 1.0, 1.0, 0.0}, cy[4] = {0.0, 0.0, 1.0, 1.0};
    double px[8], py[8];
    int m = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int k1 = (k + 1) & 3;
        const bool pk = ls_pos(p[k]), pn = ls_pos(p[k1]);
        if (pk) {
            px[m] = cx[k];
            py[m] = cy[k];
            ++m;
        }
        if (pk != pn) {
            const double t = p[k] / (p[k] - p[k1]);
            px[m] = cx[k] + t * (cx[k1] - cx[k]);
            py[m] = cy[k] + t * (cy[k1] - cy[k]);
            ++m;
        }
    }
    double twice = 0.0;
    for (int k = 0; k < m; ++k) {
        const int k1 = k + 1 == m ? 0 : k + 1;
        twice += px[k] * py[k1] - px[k1] * py[k];
    }
    return 0.5 * twice;
}

// Geometry of one cell: the level set at the 2^ndim vertices around each of
// its corners (the mean of the 2^ndim cells sharing the vertex, summed in a
// fixed order), the apertures of its 2 ndim faces, the interface segment
// and volume fraction (App. D) and the 4th-order normal.  The cell writes
// the apertures of its lower faces (and of its upper faces at the grid's
// upper end); both cells of a face compute the same value.
template <int NDIM>
__global__ void __launch_bounds__(kLsThreads) k_ls_geometry(const LsGrid g, const double *__restrict__ phi,
                                                             double *__restrict__ ap, double *__restrict__ alpha,
                                                             double *__restrict__ dgam, double *__restrict__ nrm) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.ncell) return;
    int c[3];
    ls_cell(g, i, c);
    const double h = g.h;
    double am[3], apx[3];  // apertures of the lower / upper face of each axis
    // mapped neighbour coordinates -1, 0, +1 of each axis
    long long ox[3], oy[3], oz[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        ox[k] = ls_map(c[0] + k - 1, g.n[0], g.bc[0][0], g.bc[0][1]);
        oy[k] = (long long)ls_map(c[1] + k - 1, g.n[1], g.bc[1][0], g.bc[1][1]) * g.n[0];
        oz[k] = NDIM == 3 ? (long long)ls_map(c[2] + k - 1, g.n[2], g.bc[2][0], g.bc[2][1]) * g.n[0] * g.n[1] : 0;
    }
    if constexpr (NDIM == 3) {
        double P[3][3][3];  // cells c + (x, y, z) - 1
#pragma unroll
        for (int z = 0; z < 3; ++z)
#pragma unroll
            for (int y = 0; y < 3; ++y)
#pragma unroll
                for (int x = 0; x < 3; ++x) P[z][y][x] = __ldg(phi + oz[z] + oy[y] + ox[x]);
        double V[2][2][2];  // vertex with lower-corner cell c + (a, b, e) - 1, as V[e][b][a]
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    double s = 0.0;
#pragma unroll
                    for (int k = 0; k < 2; ++k)
#pragma unroll
                        for (int j = 0; j < 2; ++j)
#pragma unroll
                            for (int ii = 0; ii < 2; ++ii) s = __dadd_rn(s, P[e + k][b + j][a + ii]);
                    V[e][b][a] = s / 8.0;
                }
        const int o1[4] = {0, 1, 1, 0}, o2[4] = {0, 0, 1, 1};  // counter-clockwise in (e1, e2)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                double p[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    int q[3];
                    q[d] = s;
                    q[e1] = o1[k];
                    q[e2] = o2[k];
                    p[k] = V[q[2]][q[1]][q[0]];
                }
                const double f = face_fraction(p);
                if (s == 0) am[d] = f;
                else apx[d] = f;
            }
        }
    } else {
        double P[3][3];
#pragma unroll
        for (int y = 0; y < 3; ++y)
#pragma unroll
            for (int x = 0; x < 3; ++x) P[y][x] = __ldg(phi + oy[y] + ox[x]);
        double V[2][2];  // V[b][a]
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                double s = 0.0;
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int ii = 0; ii < 2; ++ii) s = __dadd_rn(s, P[b + j][a + ii]);
                V[b][a] = s / 4.0;
            }
        am[0] = edge_fraction(V[0][0], V[1][0]);
        apx[0] = edge_fraction(V[0][1], V[1][1]);
        am[1] = edge_fraction(V[0][0], V[0][1]);
        apx[1] = edge_fraction(V[1][0], V[1][1]);
    }
    // apertures of the lower faces (and the upper ones at the grid's end)
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        int m[3] = {g.n[0], g.n[1], g.n[2]};
        m[d] += 1;
        const long long f = ((long long)c[2] * m[1] + c[1]) * m[0] + c[0];
        ap[g.foff[d] + f] = am[d];
        if (c[d] == g.n[d] - 1) ap[g.foff[d] + f + (d == 0 ? 1 : (d == 1 ? m[0] : (long long)m[0] * m[1]))] = apx[d];
    }
    const double sface = NDIM == 3 ? h * h : h, vcell = NDIM == 3 ? h * h * h : h * h;
    double s2 = 0.0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        const double t = (apx[d] - am[d]) * sface;
        s2 = __dadd_rn(s2, __dmul_rn(t, t));
    }
    const double dg = sqrt(s2);
    dgam[i] = dg;
    const double phic = __ldg(phi + i);
    double vol = 0.0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) vol = __dadd_rn(vol, __dmul_rn(__dmul_rn(__dadd_rn(am[d], apx[d]), sface), 0.5 * h));
    vol = __dadd_rn(vol, __dmul_rn(dg, phic));
    double a = vol / ((double)NDIM * vcell);
    a = ls_neg(a) ? 0.0 : (ls_gt_nonneg(a, 1.0) ? 1.0 : a);
    alpha[i] = a;
    double gr[3], gg = 0.0;
    const double k12 = g.ih * (1.0 / 12.0);
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        gr[d] = (ls_line(g, phi, i, c[d], d, -2) - 8.0 * ls_line(g, phi, i, c[d], d, -1) +
                 8.0 * ls_line(g, phi, i, c[d], d, 1) - ls_line(g, phi, i, c[d], d, 2)) *
                k12;
        gg += gr[d] * gr[d];
    }
    const double ign = ls_pos(gg) ? jxf::fdiv(1.0, sqrt(gg)) : 0.0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) nrm[(long long)d * g.ncell + i] = gr[d] * ign;
}

// --------------------------------------------------------------- advection --
// 5th-order upstream-central derivative along d: the stencil i-3..i+2 for
// u_d >= 0, its mirror i-2..i+3 otherwise.
__device__ __forceinline__ double houc5(const LsGrid &g, const double *__restrict__ p, const int (&c)[3],
                                        long long i, int d, bool left) {
    const double k = g.ih * (1.0 / 60.0);
    if (left)
        return (-2.0 * ls_line(g, p, i, c[d], d, -3) + 15.0 * ls_line(g, p, i, c[d], d, -2) -
                60.0 * ls_line(g, p, i, c[d], d, -1) + 20.0 * ls_line(g, p, i, c[d], d, 0) +
                30.0 * ls_line(g, p, i, c[d], d, 1) - 3.0 * ls_line(g, p, i, c[d], d, 2)) *
               k;
    return (3.0 * ls_line(g, p, i, c[d], d, -2) - 30.0 * ls_line(g, p, i, c[d], d, -1) -
            20.0 * ls_line(g, p, i, c[d], d, 0) + 60.0 * ls_line(g, p, i, c[d], d, 1) -
            15.0 * ls_line(g, p, i, c[d], d, 2) + 2.0 * ls_line(g, p, i, c[d], d, 3)) *
           k;
}

template <int NDIM>
__device__ __forceinline__ double advect_r(const LsGrid &g, const double *__restrict__ p,
                                           const double *__restrict__ vel, const int (&c)[3], long long i) {
    double r = 0.0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        const double u = __ldg(vel + (long long)d * g.ncell + i);
        r -= u * houc5(g, p, c, i, d, !ls_neg(u));
    }
    return r;
}

// R only (mode < 0), or one TVD-RK3 stage: out = ca pn + cb (ps + dt R(ps))
// (the first stage out = ps + dt R(ps)).  out may alias pn, not ps.
template <int NDIM>
__global__ void __launch_bounds__(kLsThreads) k_ls_advect(const LsGrid g, const double *__restrict__ ps,
                                                         const double *pn, const double *__restrict__ vel, double dt,
                                                         int mode, double ca, double cb, double *out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.ncell) return;
    int c[3];
    ls_cell(g, i, c);
    const double r = advect_r<NDIM>(g, ps, vel, c, i);
    if (mode < 0) out[i] = r;
    else if (mode == 0) out[i] = ps[i] + dt * r;
    else out[i] = ca * pn[i] + cb * (ps[i] + dt * r);
}

// ---------------------------------------------------------- reinitialisation --
// Third-order WENO combination of one-sided derivatives (Jiang & Peng):
// (3 v2 - v1)/2 and (v2 + v3)/2 with linear weights 1/3, 2/3 and the
// smoothness (v2 - v1)^2, (v3 - v2)^2, eps = 1e-6.  Here on the undivided
// differences (eps scaled by h^2, which leaves the weights unchanged), the
// weights d_k/(eps + beta_k)^2 normalised in one division:
// q1 + s1 (q0 - q1)/(s1 + 2 s0), s_k = (eps + beta_k)^2.
__device__ __forceinline__ double weno3(double v1, double v2, double v3, double eps) {
    const double e0 = eps + (v2 - v1) * (v2 - v1), e1 = eps + (v3 - v2) * (v3 - v2);
    const double s0 = e0 * e0, s1 = e1 * e1;
    const double q0 = 0.5 * (3.0 * v2 - v1), q1 = 0.5 * (v2 + v3);
    return q1 + jxf::fdiv(s1 * (q0 - q1), s1 + 2.0 * s0);
}

// R_reinit = -sgn(phi0) (|grad phi| - 1) with the Godunov Hamiltonian of the
// one-sided derivatives, 0 where |R| <= thr.
template <int NDIM>
__device__ __forceinline__ double reinit_r(const LsGrid &g, const double *__restrict__ p, double phi0, double thr,
                                           const int (&c)[3], long long i) {
    const bool spos = ls_pos(phi0);
    const double s = spos ? 1.0 : (ls_neg(phi0) ? -1.0 : 0.0);
    const double eps = 1e-6 * g.h * g.h;
    double h2 = 0.0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        const double pm2 = ls_line(g, p, i, c[d], d, -2), pm1 = ls_line(g, p, i, c[d], d, -1);
        const double p0 = __ldg(p + i);
        const double pp1 = ls_line(g, p, i, c[d], d, 1), pp2 = ls_line(g, p, i, c[d], d, 2);
        const double a = weno3(pm1 - pm2, p0 - pm1, pp1 - p0, eps) * g.ih;
        const double b = weno3(pp2 - pp1, pp1 - p0, p0 - pm1, eps) * g.ih;
        double t1, t2;
        if (spos) {
            t1 = ls_pos(a) ? a : 0.0;
            t2 = ls_neg(b) ? b : 0.0;
        } else {
            t1 = ls_neg(a) ? a : 0.0;
            t2 = ls_pos(b) ? b : 0.0;
        }
        const double q1 = t1 * t1, q2 = t2 * t2;
        h2 += ls_gt_nonneg(q1, q2) ? q1 : q2;
    }
    const double r = -s * (sqrt(h2) - 1.0);
    return ls_gt_nonneg(fabs(r), thr) ? r : 0.0;
}

// R only (mode < 0), or one second-order TVD Runge-Kutta stage in pseudo-time:
// mode 0: out = ps + dtau R(ps); mode 1: out = 1/2 pn + 1/2 (ps + dtau R(ps)).
// out may alias pn, not ps.
template <int NDIM>
__global__ void __launch_bounds__(kLsThreads) k_ls_reinit(const LsGrid g, const double *__restrict__ ps,
                                                         const double *pn, const double *__restrict__ p0, double thr,
                                                         double dtau, int mode, double *out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.ncell) return;
    int c[3];
    ls_cell(g, i, c);
    const double r = reinit_r<NDIM>(g, ps, __ldg(p0 + i), thr, c, i);
    if (mode < 0) out[i] = r;
    else if (mode == 0) out[i] = ps[i] + dtau * r;
    else out[i] = 0.5 * pn[i] + 0.5 * (ps[i] + dtau * r);
}

// ------------------------------------------------- interface quantities --
// A cut cell holds an interface segment (Sec. 3.5): both phases have volume
// in it, or the interface runs along one of its faces (alpha = 1 and
// dGamma > 0 on the side whose aperture drops to 0 there).
__device__ __forceinline__ bool ls_is_cut(double alpha, double dgamma) {
    return (ls_pos(alpha) && alpha < 1.0) || ls_pos(dgamma);
}

// The linearised two-material Riemann problem (App. D, no surface tension)
// in every cut cell: Z_p = rho_p c_p, un_p = u_p . n,
// u_Gamma = (Z1 un1 + Z2 un2 + p2 - p1)/(Z1 + Z2) along n, p_Gamma =
// (Z1 p2 + Z2 p1 + Z1 Z2 (un2 - un1))/(Z1 + Z2); 0 elsewhere.
template <int NDIM>
__global__ void __launch_bounds__(kLsThreads)
    k_ls_interface(const LsGrid g, const double *__restrict__ W1, const double *__restrict__ W2, double g1,
                   double pi1, double g2, double pi2, const double *__restrict__ alpha,
                   const double *__restrict__ dgamma, const double *__restrict__ nrm, double *__restrict__ ug,
                   double *__restrict__ pg) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.ncell) return;
    const long long nc = g.ncell;
    if (!ls_is_cut(__ldg(alpha + i), __ldg(dgamma + i))) {
#pragma unroll
        for (int d = 0; d < NDIM; ++d) ug[(long long)d * nc + i] = 0.0;
        pg[i] = 0.0;
        return;
    }
    double n[NDIM];
#pragma unroll
    for (int d = 0; d < NDIM; ++d) n[d] = __ldg(nrm + (long long)d * nc + i);
    double Z[2], un[2], p[2];
    const double *Wp[2] = {W1, W2};
    const double gm[2] = {g1, g2}, pim[2] = {pi1, pi2};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const double rho = __ldg(Wp[k] + i), pk = __ldg(Wp[k] + (long long)(1 + NDIM) * nc + i);
        double u = 0.0;
#pragma unroll
        for (int d = 0; d < NDIM; ++d) u += __ldg(Wp[k] + (long long)(1 + d) * nc + i) * n[d];
        Z[k] = rho * sqrt(gm[k] * (pk + pim[k]) / rho);
        un[k] = u;
        p[k] = pk;
    }
    const double zs = Z[0] + Z[1];
    const double u_g = (Z[0] * un[0] + Z[1] * un[1] + p[1] - p[0]) / zs;
    const double p_g = (Z[0] * p[1] + Z[1] * p[0] + Z[0] * Z[1] * (un[1] - un[0])) / zs;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) ug[(long long)d * nc + i] = u_g * n[d];
    pg[i] = p_g;
}

// ----------------------------------------------------------------- extension --
// One explicit Euler step (dtau) of dQ/dtau + a . grad Q = 0 on nq cell
// arrays, first-order upwind per axis, a = sdir n: with the upwind
// neighbour u_d of each axis (i - 1 where a_d > 0, i + 1 where a_d < 0) and
// w_d = (dtau/h) |a_d|, Q <- (1 - sum_d w_d) Q + sum_d w_d Q[u_d] (a convex
// combination, sum_d w_d <= sqrt(3)/4; no division on the device: dtau/h is
// an argument).  Mode 0 (ghost cells of phase 1): sdir = -1 where alpha =
// 0; mode 1 (phase 2): sdir = +1 where alpha = 1; mode 2 (interface
// quantities): sdir = sgn(phi) in every cell but the cut cells.  The other
// cells copy their values.  One launch serves one or two such extensions
// (modes ma and mb >= 0, each with its arrays): the ghost cells of both
// phases are one launch per pseudo-time step.  The upwind offsets and
// weights are found once per cell and extension (sign tests on the integer
// pipe), then applied to all nq arrays: four FP64 operations per value.
template <int NDIM>
__global__ void __launch_bounds__(kLsThreads, 4)
    k_ls_extend(const LsGrid g, const double *__restrict__ phi, const double *__restrict__ alpha,
                const double *__restrict__ dgamma, const double *__restrict__ nrm, int ma, int mb, int nq,
                double cfl, const double *__restrict__ qa_in, double *__restrict__ qa_out,
                const double *__restrict__ qb_in, double *__restrict__ qb_out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.ncell) return;
    const long long nc = g.ncell;
    const double al = __ldg(alpha + i);
    int c[3] = {-1, 0, 0};  // found on first use
    for (int job = 0; job < 2; ++job) {
        const int mode = job ? mb : ma;
        if (mode < 0) break;
        const double *qin = job ? qb_in : qa_in;
        double *qout = job ? qb_out : qa_out;
        // alpha in [0, 1]: alpha < 1 as a bit-pattern compare with 1.0
        const bool a_pos = ls_pos(al), a_lt1 = __double_as_longlong(al) < 0x3FF0000000000000LL;
        int sdir;
        bool fixed;
        if (mode == 0) {
            sdir = -1;
            fixed = a_pos;
        } else if (mode == 1) {
            sdir = 1;
            fixed = a_lt1;
        } else {
            const double ph = __ldg(phi + i);
            sdir = ls_pos(ph) ? 1 : (ls_neg(ph) ? -1 : 0);
            fixed = (a_pos && a_lt1) || ls_pos(__ldg(dgamma + i));
        }
        if (fixed) {
            for (int k = 0; k < nq; ++k) qout[(long long)k * nc + i] = __ldg(qin + (long long)k * nc + i);
            continue;
        }
        if (c[0] < 0) ls_cell(g, i, c);
        long long off[NDIM];  // upwind neighbour minus i (0 where a_d = 0)
        double w[NDIM];       // (dtau/h) |a_d|
        double wsum = 0.0;
#pragma unroll
        for (int d = 0; d < NDIM; ++d) {
            const double n = __ldg(nrm + (long long)d * nc + i);
            const int sn = ls_pos(n) ? 1 : (ls_neg(n) ? -1 : 0);
            const int s = -sdir * sn;  // step to the upwind neighbour: against the sign of a_d = sdir n_d
            off[d] = s ? (long long)(ls_map(c[d] + s, g.n[d], g.bc[d][0], g.bc[d][1]) - c[d]) * g.stride[d] : 0;
            w[d] = s ? cfl * fabs(n) : 0.0;
            wsum += w[d];
        }
        const double w0 = 1.0 - wsum;
        for (int k = 0; k < nq; ++k) {
            const double *q = qin + (long long)k * nc + i;
            double r = w0 * __ldg(q);
#pragma unroll
            for (int d = 0; d < NDIM; ++d) r = fma(w[d], __ldg(q + off[d]), r);
            qout[(long long)k * nc + i] = r;
        }
    }
}

// ------------------------------------------------------- cut-cell right side --
// Face fluxes of one phase: the scheme's face flux (reconstruction and HLLC
// of jxf_impl.cuh, single-phase model, no limiter, inviscid; RSV 0: WENO5,
// 2: TENO6-A) from the phase's primitives P.W, one thread per face of axis
// d, into F (nv arrays of the axis's faces).  A face the phase does not wet (its aperture A,
// resp. 1 - A for phase 2, is 0) carries no flux of the phase: F = 0 there,
// without evaluating it (the right-hand side weighs it by 0 either way).
template <int NDIM, int d, int RSV>
__global__ void __launch_bounds__(jxf::kFluxThreads)
    k_ls_cut_faces(const jxf::Dev P, const double *__restrict__ apd, int phase, double *__restrict__ F) {
    using V = jxf::Vars<JXF_SPM, NDIM>;
    int m[3] = {P.n[0], P.n[1], P.n[2]};
    m[d] += 1;
    const long long nface = (long long)m[0] * m[1] * m[2];
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nface) return;
    const double A = __ldg(apd + g);
    if (phase == 1 ? !(A > 0.0) : !(A < 1.0)) {
#pragma unroll
        for (int v = 0; v < V::NV; ++v) F[v * nface + g] = 0.0;
        return;
    }
    const unsigned gu = (unsigned)g;
    const unsigned q0 = P.fd_face[d][0].div(gu), q1 = P.fd_face[d][1].div(q0);
    const int c[3] = {(int)(gu - q0 * (unsigned)m[0]), (int)(q0 - q1 * (unsigned)m[1]), (int)q1};
    double Fv[jxf::MAXV], uh;
    bool il = false, fl = false;
    jxf::flux_face_at<double, JXF_SPM, NDIM, d, 0, RSV>(P, 0.0, c, false, Fv, uh, il, fl);
#pragma unroll
    for (int v = 0; v < V::NV; ++v) F[v * nface + g] = Fv[v];
}

// d(alpha U)/dt of phase 1 (phi > 0) or 2 in every cell: the face fluxes
// weighted by the phase's apertures (A resp. 1 - A), then the interface
// pressure force and power along the phase's inward normal (+n resp. -n):
// sp pg dGamma / V (n, u_Gamma . n).
template <int NDIM>
__global__ void __launch_bounds__(kLsThreads)
    k_ls_cut_update(const LsGrid g, const double *__restrict__ F, const double *__restrict__ ap,
                    const double *__restrict__ dgam, const double *__restrict__ nrm, const double *__restrict__ ug,
                    const double *__restrict__ pg, int phase, double *__restrict__ dU) {
    constexpr int NV = NDIM + 2;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.ncell) return;
    const long long nc = g.ncell;
    int c[3];
    ls_cell(g, i, c);
    double R[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) R[v] = 0.0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        int m[3] = {g.n[0], g.n[1], g.n[2]};
        m[d] += 1;
        const long long nface = (long long)m[0] * m[1] * m[2];
        const long long gm = ((long long)c[2] * m[1] + c[1]) * m[0] + c[0];
        const long long gp = gm + (d == 0 ? 1 : (d == 1 ? m[0] : (long long)m[0] * m[1]));
        double am = __ldg(ap + g.foff[d] + gm), apx = __ldg(ap + g.foff[d] + gp);
        if (phase == 2) {
            am = 1.0 - am;
            apx = 1.0 - apx;
        }
        const double *Fd = F + (long long)NV * g.foff[d];
#pragma unroll
        for (int v = 0; v < NV; ++v)
            R[v] = R[v] - (apx * __ldg(Fd + v * nface + gp) - am * __ldg(Fd + v * nface + gm)) * g.ih;
    }
    const double dg = __ldg(dgam + i);
    if (dg > 0.0) {
        const double ivol = NDIM == 3 ? g.ih * g.ih * g.ih : g.ih * g.ih;
        double n[NDIM], un = 0.0;
#pragma unroll
        for (int d = 0; d < NDIM; ++d) {
            n[d] = __ldg(nrm + (long long)d * nc + i);
            un += __ldg(ug + (long long)d * nc + i) * n[d];
        }
        const double force = (phase == 1 ? 1.0 : -1.0) * __ldg(pg + i) * dg * ivol;
#pragma unroll
        for (int d = 0; d < NDIM; ++d) R[1 + d] = R[1 + d] + force * n[d];
        R[1 + NDIM] = R[1 + NDIM] + force * un;
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) dU[v * nc + i] = R[v];
}

// ------------------------------------------------------------------ mixing --
// Conservative mixing (App. D) of one phase's volume-weighted state, as a
// gather in two passes (no atomics: the result does not depend on the
// order threads run in).  Pass 1: every cell that vanished (a1 = 0 < a0),
// is new (a0 = 0 < a1) or is small (a1 < amix) computes the fluxes to its
// targets -- the neighbours one step along sign(n^p) on each axis, pair of
// axes and all three -- with the weights |n_e|^2 a_t, |n_e n_f| a_t,
// |n_x n_y n_z|^(2/3) a_t normalised to 1 (a target outside a non-periodic
// side weighs 0): M_t = beta_t/(a beta_t + a_t) [(a_t U_t) a - (a U) a_t],
// stored as M[t][v][cell], and a code byte per cell: 0 for a cell without
// fluxes (M is then neither written nor read), else 0x80 | the signs of
// n^p (2 bits per axis, sign + 1).  Pass 2, in place: every cell adds its
// own fluxes and subtracts those its neighbours aimed at it (it reads aU
// only at itself, so no other thread sees the update).
__device__ __forceinline__ bool ls_mixing(double a0, double a1, double amix) {
    return (a1 == 0.0 && a0 > 0.0) || (a1 > 0.0 && a0 == 0.0) || a1 < amix;
}

// Target t (subset mask t + 1 of the axes) of cell c along the signs sg:
// false when it lies outside a non-periodic side (or a sign is 0).
__device__ __forceinline__ bool ls_target(const LsGrid &g, const int (&c)[3], const int (&sg)[3], int t, int (&q)[3]) {
    q[0] = c[0], q[1] = c[1], q[2] = c[2];
    const int mask = t + 1;
    for (int e = 0; e < g.ndim; ++e) {
        if (!((mask >> e) & 1)) continue;
        if (sg[e] == 0) return false;
        q[e] += sg[e];
        if (q[e] < 0 || q[e] >= g.n[e]) {
            if (g.bc[e][0] != JXF_BC_PERIODIC) return false;
            q[e] = (q[e] + g.n[e]) % g.n[e];
        }
    }
    return true;
}

template <int NDIM>
__global__ void __launch_bounds__(kLsThreads)
    k_ls_mix_flux(const LsGrid g, int nv, const double *__restrict__ a0, const double *__restrict__ a1,
                  const double *__restrict__ np, double amix, const double *__restrict__ aU, double *__restrict__ M,
                  unsigned char *__restrict__ code) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.ncell) return;
    const long long nc = g.ncell;
    constexpr int ntrg = NDIM == 3 ? 7 : 3;
    const double ai = __ldg(a1 + i);
    code[i] = 0;
    if (!ls_mixing(__ldg(a0 + i), ai, amix)) return;
    int c[3];
    ls_cell(g, i, c);
    int sg[3] = {0, 0, 0};
    double an[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
        const double nd = __ldg(np + (long long)d * nc + i);
        sg[d] = nd > 0.0 ? 1 : (nd < 0.0 ? -1 : 0);
        an[d] = fabs(nd);
    }
    long long ti[7];
    double beta[7], at[7], bsum = 0.0;
#pragma unroll
    for (int t = 0; t < ntrg; ++t) {
        int q[3];
        const bool in = ls_target(g, c, sg, t, q);
        const int mask = t + 1;
        double w = 1.0;
        int nbits = 0;
#pragma unroll
        for (int e = 0; e < NDIM; ++e)
            if ((mask >> e) & 1) {
                ++nbits;
                w *= an[e];
            }
        if (nbits == 1) w = w * w;
        else if (nbits == 3) w = cbrt(w * w);
        ti[t] = in ? ((long long)q[2] * g.n[1] + q[1]) * g.n[0] + q[0] : -1;
        at[t] = in ? __ldg(a1 + ti[t]) : 0.0;
        beta[t] = in ? w * at[t] : 0.0;
        bsum += beta[t];
    }
    if (!(bsum > 0.0)) return;
#pragma unroll
    for (int t = 0; t < ntrg; ++t) {
        if (ti[t] < 0 || beta[t] == 0.0) {
            for (int v = 0; v < nv; ++v) M[((long long)t * nv + v) * nc + i] = 0.0;
            continue;
        }
        const double b = beta[t] / bsum;
        const double f = b / (ai * b + at[t]);
        for (int v = 0; v < nv; ++v)
            M[((long long)t * nv + v) * nc + i] =
                f * (__ldg(aU + (long long)v * nc + ti[t]) * ai - __ldg(aU + (long long)v * nc + i) * at[t]);
    }
    code[i] = (unsigned char)(0x80 | (sg[0] + 1) | ((sg[1] + 1) << 2) | ((sg[2] + 1) << 4));
}

__global__ void __launch_bounds__(kLsThreads)
    k_ls_mix_apply(const LsGrid g, int nv, const double *__restrict__ M, const unsigned char *__restrict__ code,
                   double *__restrict__ aU) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.ncell) return;
    const long long nc = g.ncell;
    const int ntrg = g.ndim == 3 ? 7 : 3;
    int c[3];
    ls_cell(g, i, c);
    // first the neighbours whose fluxes land here: bit j of hit for the
    // offset o = (j % 3, j / 3 % 3, j / 9) - 1 (k = c - o), with its cell
    // index and target recomputed when the fluxes are gathered
    unsigned hit = 0;
    // fluxes aimed at this cell by its neighbours k = c - o (o one step along
    // some axes): k's target t lands here when its step is o
    const int nz = g.ndim == 3 ? 1 : 0;
    for (int oz = -nz; oz <= nz; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                if (ox == 0 && oy == 0 && oz == 0) continue;
                const int o[3] = {ox, oy, oz};
                int k[3];
                bool in = true;
                for (int e = 0; e < 3; ++e) {
                    k[e] = c[e] - o[e];
                    if (e >= g.ndim) continue;
                    if (k[e] < 0 || k[e] >= g.n[e]) {
                        if (g.bc[e][0] != JXF_BC_PERIODIC) in = false;
                        else k[e] = (k[e] + g.n[e]) % g.n[e];
                    }
                }
                if (!in) continue;
                const long long ki = ((long long)k[2] * g.n[1] + k[1]) * g.n[0] + k[0];
                const int ck = __ldg(code + ki);
                if (!ck) continue;
                int sg[3];
                for (int d = 0; d < 3; ++d) sg[d] = ((ck >> (2 * d)) & 3) - 1;
                // the subset of axes k steps along to reach this cell
                int mask = 0;
                bool match = true;
                for (int e = 0; e < g.ndim; ++e) {
                    if (o[e] == 0) continue;
                    if (sg[e] != o[e]) match = false;
                    mask |= 1 << e;
                }
                if (!match) continue;
                hit |= 1u << ((oz + 1) * 9 + (oy + 1) * 3 + (ox + 1));
            }
    const bool own = code[i] != 0;
    if (!own && !hit) return;
    for (int v = 0; v < nv; ++v) {
        double r = aU[(long long)v * nc + i];
        if (own)
            for (int t = 0; t < ntrg; ++t) r += __ldg(M + ((long long)t * nv + v) * nc + i);
        for (unsigned m = hit; m; m &= m - 1) {
            const int j = __ffs(m) - 1;
            const int o[3] = {j % 3 - 1, j / 3 % 3 - 1, j / 9 - 1};
            int k[3], mask = 0;
            for (int e = 0; e < 3; ++e) {
                k[e] = c[e] - o[e];
                if (e < g.ndim && (k[e] < 0 || k[e] >= g.n[e])) k[e] = (k[e] + g.n[e]) % g.n[e];  // periodic
                if (o[e] != 0) mask |= 1 << e;
            }
            const long long ki = ((long long)k[2] * g.n[1] + k[1]) * g.n[0] + k[0];
            r -= __ldg(M + ((long long)(mask - 1) * nv + v) * nc + ki);
        }
        aU[(long long)v * nc + i] = r;
    }
}

// ----------------------------------------------------------- the time step --
// Volume-weighted conservative states of both phases from their primitives
// (rho, u_d, p, given in every cell): aU1 = alpha U(W1), aU2 = (1 - alpha)
// U(W2), each phase's stiffened gas in its Dev.
template <int NDIM>
__global__ void __launch_bounds__(kLsThreads)
    k_ls_cons(const jxf::Dev P1, const jxf::Dev P2, long long nc, const double *__restrict__ alpha,
              const double *__restrict__ W1, const double *__restrict__ W2, double *__restrict__ aU1,
              double *__restrict__ aU2) {
    constexpr int NV = NDIM + 2;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const double a = __ldg(alpha + i);
    double w[NV], u[NV], rc2;
#pragma unroll
    for (int v = 0; v < NV; ++v) w[v] = __ldg(W1 + v * nc + i);
    jxf::prim2cons<double, JXF_SPM, NDIM>(P1, w, u, rc2);
#pragma unroll
    for (int v = 0; v < NV; ++v) aU1[v * nc + i] = a * u[v];
#pragma unroll
    for (int v = 0; v < NV; ++v) w[v] = __ldg(W2 + v * nc + i);
    jxf::prim2cons<double, JXF_SPM, NDIM>(P2, w, u, rc2);
#pragma unroll
    for (int v = 0; v < NV; ++v) aU2[v * nc + i] = (1.0 - a) * u[v];
}

// One TVD-RK3 stage of both phases' volume-weighted states (n values each):
// U <- U + dt R in the first stage, else U <- ca Un + cb (U + dt R).
__global__ void __launch_bounds__(kLsThreads)
    k_ls_stage(long long n, int first, double ca, double cb, double dt, const double *__restrict__ U1n,
               const double *__restrict__ R1, double *__restrict__ U1, const double *__restrict__ U2n,
               const double *__restrict__ R2, double *__restrict__ U2) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    if (first) {
        U1[k] = U1[k] + dt * __ldg(R1 + k);
        U2[k] = U2[k] + dt * __ldg(R2 + k);
    } else {
        U1[k] = ca * __ldg(U1n + k) + cb * (U1[k] + dt * __ldg(R1 + k));
        U2[k] = ca * __ldg(U2n + k) + cb * (U2[k] + dt * __ldg(R2 + k));
    }
}

// Phase 2's fractions before and after a stage and its inward normal:
// 1 - a0, 1 - a1, -n.
template <int NDIM>
__global__ void __launch_bounds__(kLsThreads)
    k_ls_phase2(long long nc, const double *__restrict__ a0, const double *__restrict__ a1,
                const double *__restrict__ nrm, double *__restrict__ b0, double *__restrict__ b1,
                double *__restrict__ n2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    b0[i] = 1.0 - __ldg(a0 + i);
    b1[i] = 1.0 - __ldg(a1 + i);
#pragma unroll
    for (int d = 0; d < NDIM; ++d) n2[d * nc + i] = -__ldg(nrm + d * nc + i);
}

// Primitives of the cells holding a phase (fraction ap > 0) from its
// volume-weighted state: W = cons2prim(aU / ap); the other cells keep W.
template <int NDIM>
__global__ void __launch_bounds__(kLsThreads)
    k_ls_prim(const jxf::Dev P, long long nc, const double *__restrict__ ap, const double *__restrict__ aU,
              double *__restrict__ W) {
    constexpr int NV = NDIM + 2;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const double a = __ldg(ap + i);
    if (!(a > 0.0)) return;
    double u[NV], w[NV], rho, p, rc2;
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = __ldg(aU + v * nc + i) / a;
    jxf::cons2prim<double, double, JXF_SPM, NDIM>(P, u, w, rho, p, rc2);
#pragma unroll
    for (int v = 0; v < NV; ++v) W[v * nc + i] = w[v];
}

// ------------------------------------------------------------------- host --
jxf_status ls_grid(const jxf_grid *grid, LsGrid &g) {
    if (!grid || grid->ndim < 2 || grid->ndim > 3) return JXF_ERR_ARG;
    g.ndim = grid->ndim;
    long long nc = 1;
    for (int e = 0; e < 3; ++e) {
        g.n[e] = e < g.ndim ? grid->n[e] : 1;
        if (g.n[e] < 1) return JXF_ERR_ARG;
        for (int s = 0; s < 2; ++s) {
            g.bc[e][s] = grid->bc[e][s];
            if (e < g.ndim && (g.bc[e][s] < JXF_BC_PERIODIC || g.bc[e][s] > JXF_BC_SYMMETRY)) return JXF_ERR_ARG;
        }
        if (e < g.ndim && (grid->bc[e][0] == JXF_BC_PERIODIC) != (grid->bc[e][1] == JXF_BC_PERIODIC))
            return JXF_ERR_ARG;
        nc *= g.n[e];
    }
    g.h = (grid->hi[0] - grid->lo[0]) / g.n[0];
    if (!(g.h > 0.0)) return JXF_ERR_ARG;
    g.ih = 1.0 / g.h;
    g.stride[0] = 1;
    g.stride[1] = g.n[0];
    g.stride[2] = (long long)g.n[0] * g.n[1];
    for (int e = 1; e < g.ndim; ++e) {
        const double he = (grid->hi[e] - grid->lo[e]) / g.n[e];
        if (std::fabs(he - g.h) > 1e-12 * g.h) return JXF_ERR_ARG;  // cubic cells only (§3.5)
    }
    // the boundary mapping reaches 3 cells past an end (one reflection)
    for (int e = 0; e < g.ndim; ++e)
        if (g.n[e] < 3) return JXF_ERR_ARG;
    if (nc >= (1ll << 31)) return JXF_ERR_ARG;
    g.ncell = nc;
    long long off = 0;
    for (int d = 0; d < 3; ++d) {
        g.foff[d] = off;
        if (d < g.ndim) {
            long long f = 1;
            for (int e = 0; e < 3; ++e) f *= g.n[e] + (e == d ? 1 : 0);
            off += f;
        }
    }
    return JXF_OK;
}

unsigned ls_blocks(const LsGrid &g) { return (unsigned)((g.ncell + kLsThreads - 1) / kLsThreads); }

void advect_launch(const LsGrid &g, const double *ps, const double *pn, const double *vel, double dt, int mode,
                   double ca, double cb, double *out, cudaStream_t s) {
    if (g.ndim == 3) k_ls_advect<3><<<ls_blocks(g), kLsThreads, 0, s>>>(g, ps, pn, vel, dt, mode, ca, cb, out);
    else k_ls_advect<2><<<ls_blocks(g), kLsThreads, 0, s>>>(g, ps, pn, vel, dt, mode, ca, cb, out);
}

void reinit_launch(const LsGrid &g, const double *ps, const double *pn, const double *p0, double thr, double dtau,
                   int mode, double *out, cudaStream_t s) {
    if (g.ndim == 3) k_ls_reinit<3><<<ls_blocks(g), kLsThreads, 0, s>>>(g, ps, pn, p0, thr, dtau, mode, out);
    else k_ls_reinit<2><<<ls_blocks(g), kLsThreads, 0, s>>>(g, ps, pn, p0, thr, dtau, mode, out);
}

jxf_status ls_launched() {
    return cudaPeekAtLastError() == cudaSuccess ? JXF_OK : (cudaGetLastError(), JXF_ERR_CUDA);
}

unsigned ls_blocks_n(long long n) { return (unsigned)((n + kLsThreads - 1) / kLsThreads); }

template <int RSV>
void ls_cut_faces_rsv(int ndim, int d, unsigned blocks, cudaStream_t s, const jxf::Dev &P, const double *A,
                      int phase, double *F) {
    if (ndim == 3) {
        if (d == 0) k_ls_cut_faces<3, 0, RSV><<<blocks, jxf::kFluxThreads, 0, s>>>(P, A, phase, F);
        if (d == 1) k_ls_cut_faces<3, 1, RSV><<<blocks, jxf::kFluxThreads, 0, s>>>(P, A, phase, F);
        if (d == 2) k_ls_cut_faces<3, 2, RSV><<<blocks, jxf::kFluxThreads, 0, s>>>(P, A, phase, F);
    } else {
        if (d == 0) k_ls_cut_faces<2, 0, RSV><<<blocks, jxf::kFluxThreads, 0, s>>>(P, A, phase, F);
        if (d == 1) k_ls_cut_faces<2, 1, RSV><<<blocks, jxf::kFluxThreads, 0, s>>>(P, A, phase, F);
    }
}

// The face-flux launch of axis d for the scheme family (WENO5 or TENO6-A).
void ls_cut_faces_launch(int ndim, int d, bool teno, unsigned blocks, cudaStream_t s, const jxf::Dev &P,
                         const double *A, int phase, double *F) {
    if (teno) ls_cut_faces_rsv<2>(ndim, d, blocks, s, P, A, phase, F);
    else ls_cut_faces_rsv<0>(ndim, d, blocks, s, P, A, phase, F);
}

// steps pseudo-time steps of one extension (mode ma of the nq arrays qa) or
// two at once (mode mb >= 0 of qb as well), ping-ponging through scratch
// (nq ncell doubles per extension); the results end in qa (and qb).
jxf_status ls_extend_launch(const LsGrid &g, const double *phi, const double *alpha, const double *dgamma,
                            const double *normal, int ma, double *qa, int mb, double *qb, int nq, int steps,
                            double *scratch, cudaStream_t s) {
    const double cfl = 0.25;  // dtau / h, dtau = 0.25 h
    const long long nb = (long long)nq * g.ncell;
    double *a0 = qa, *a1 = scratch, *b0 = qb, *b1 = mb >= 0 ? scratch + nb : nullptr;
    for (int k = 0; k < steps; ++k) {
        if (g.ndim == 3)
            k_ls_extend<3><<<ls_blocks(g), kLsThreads, 0, s>>>(g, phi, alpha, dgamma, normal, ma, mb, nq, cfl, a0, a1,
                                                              b0, b1);
        else
            k_ls_extend<2><<<ls_blocks(g), kLsThreads, 0, s>>>(g, phi, alpha, dgamma, normal, ma, mb, nq, cfl, a0, a1,
                                                              b0, b1);
        std::swap(a0, a1);
        std::swap(b0, b1);
    }
    if (a0 != qa && cudaMemcpyAsync(qa, a0, (size_t)nb * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return JXF_ERR_CUDA;
    if (mb >= 0 && b0 != qb &&
        cudaMemcpyAsync(qb, b0, (size_t)nb * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return JXF_ERR_CUDA;
    return ls_launched();
}

// Work buffer of the time step, in doubles (see jxf_ls_step_work).
struct LsWork {
    double *ap, *al0, *al1, *dg, *nr, *n2, *b0, *b1, *phin, *phit, *R1, *R2, *U1n, *U2n, *scr;
    long long total;
};

LsWork ls_work(const LsGrid &g, long long nface, double *base) {
    const long long nc = g.ncell;
    const int nd = g.ndim, nv = nd + 2, ntrg = nd == 3 ? 7 : 3;
    LsWork w{};
    long long off = 0;
    auto take = [&](long long n) {
        double *p = base ? base + off : nullptr;
        off += (n + 31) / 32 * 32;  // 256-byte aligned pieces
        return p;
    };
    w.ap = take(nface);
    w.al0 = take(nc);
    w.al1 = take(nc);
    w.dg = take(nc);
    w.nr = take((long long)nd * nc);
    w.n2 = take((long long)nd * nc);
    w.b0 = take(nc);
    w.b1 = take(nc);
    w.phin = take(nc);
    w.phit = take(nc);
    w.R1 = take((long long)nv * nc);
    w.R2 = take((long long)nv * nc);
    w.U1n = take((long long)nv * nc);
    w.U2n = take((long long)nv * nc);
    // shared by the calls of one stage, one at a time: the face fluxes of the
    // cut-cell right-hand side, the mixing fluxes, the extension and
    // reinitialisation ping-pong buffers
    w.scr = take(std::max((long long)nv * nface, (long long)(ntrg + 1) * nv * nc));
    w.total = off;
    return w;
}

// The arguments of jxf_ls_init / jxf_ls_step: both phases single-phase
// stiffened gases on the same grid, the FP64 inviscid scheme without limiter.
jxf_status ls_step_args(const jxf_grid *grid, const jxf_eos *eos1, const jxf_eos *eos2, const jxf_scheme *scheme,
                        LsGrid &g, jxf::Dev &P1, jxf::Dev &P2) {
    long long ncell = 0;
    if (ls_grid(grid, g) != JXF_OK || !eos1 || !eos2 || !scheme) return JXF_ERR_ARG;
    if (eos1->model != JXF_SPM || eos2->model != JXF_SPM) return JXF_ERR_UNSUPPORTED;
    if (jxf::validate_setup(grid, eos1, scheme, &ncell, false) != JXF_OK ||
        jxf::validate_setup(grid, eos2, scheme, &ncell, false) != JXF_OK)
        return JXF_ERR_ARG;
    if (eos1->model != JXF_SPM || eos2->model != JXF_SPM || scheme->precision != JXF_FP64 || scheme->viscous ||
        scheme->limiter || scheme->recon > JXF_TENO6A_CHAR)
        return JXF_ERR_UNSUPPORTED;
    jxf::fill_dev(grid, eos1, scheme, ncell, P1);
    jxf::fill_dev(grid, eos2, scheme, ncell, P2);
    return JXF_OK;
}

// Interface quantities from W1, W2 and the geometry (al, dg, nr) and their
// extension (20 steps): qg = (u_Gamma n_d ..., p_Gamma).
jxf_status ls_interface_ext(const jxf_grid *grid, const LsGrid &g, const jxf_eos *eos1, const jxf_eos *eos2,
                            const double *phi, const double *W1, const double *W2, const double *al,
                            const double *dg, const double *nr, double *qg, double *scr, cudaStream_t s) {
    const double gam[2] = {eos1->gamma[0], eos2->gamma[0]}, pin[2] = {eos1->pinf[0], eos2->pinf[0]};
    jxf_status st = jxf_ls_interface(grid, W1, W2, gam, pin, al, dg, nr, qg, qg + (long long)g.ndim * g.ncell,
                                     (jxf_stream)s);
    if (st != JXF_OK) return st;
    return jxf_ls_extend(grid, phi, al, dg, nr, qg, g.ndim + 1, 2, 20, scr, (jxf_stream)s);
}

}  // namespace

extern "C" {

long long jxf_ls_nface(const jxf_grid *grid) {
    LsGrid g;
    if (ls_grid(grid, g) != JXF_OK) return -1;
    long long s = 0;
    for (int d = 0; d < g.ndim; ++d) {
        long long f = 1;
        for (int e = 0; e < 3; ++e) f *= g.n[e] + (e == d ? 1 : 0);
        s += f;
    }
    return s;
}

jxf_status jxf_ls_geometry(const jxf_grid *grid, const double *phi, double *apert, double *alpha, double *dgamma,
                           double *normal, jxf_stream stream) {
    JXF_RANGE("jxf_ls_geometry");
    LsGrid g;
    if (ls_grid(grid, g) != JXF_OK || !phi || !apert || !alpha || !dgamma || !normal) return JXF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (g.ndim == 3) k_ls_geometry<3><<<ls_blocks(g), kLsThreads, 0, s>>>(g, phi, apert, alpha, dgamma, normal);
    else k_ls_geometry<2><<<ls_blocks(g), kLsThreads, 0, s>>>(g, phi, apert, alpha, dgamma, normal);
    return ls_launched();
}

jxf_status jxf_ls_rhs(const jxf_grid *grid, const double *phi, const double *vel, double *rhs, jxf_stream stream) {
    JXF_RANGE("jxf_ls_rhs");
    LsGrid g;
    if (ls_grid(grid, g) != JXF_OK || !phi || !vel || !rhs || rhs == phi) return JXF_ERR_ARG;
    advect_launch(g, phi, phi, vel, 0.0, -1, 0.0, 0.0, rhs, (cudaStream_t)stream);
    return ls_launched();
}

jxf_status jxf_ls_advect(const jxf_grid *grid, double *phi, const double *vel, double dt, int nsteps,
                         double *scratch, jxf_stream stream) {
    JXF_RANGE("jxf_ls_advect");
    LsGrid g;
    if (ls_grid(grid, g) != JXF_OK || !phi || !vel || !scratch || nsteps < 0 || !std::isfinite(dt))
        return JXF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    double *p1 = scratch, *p2 = scratch + g.ncell;
    for (int k = 0; k < nsteps; ++k) {
        // TVD-RK3 (§3.4): p1 = p + dt R(p); p2 = 3/4 p + 1/4 (p1 + dt R(p1));
        // p <- 1/3 p + 2/3 (p2 + dt R(p2))
        advect_launch(g, phi, phi, vel, dt, 0, 0.0, 1.0, p1, s);
        advect_launch(g, p1, phi, vel, dt, 1, 0.75, 0.25, p2, s);
        advect_launch(g, p2, phi, vel, dt, 1, 1.0 / 3.0, 2.0 / 3.0, phi, s);
    }
    return ls_launched();
}

jxf_status jxf_ls_reinit_rhs(const jxf_grid *grid, const double *phi, const double *phi0, double threshold,
                             double *rhs, jxf_stream stream) {
    JXF_RANGE("jxf_ls_reinit_rhs");
    LsGrid g;
    if (ls_grid(grid, g) != JXF_OK || !phi || !phi0 || !rhs || rhs == phi || !(threshold >= 0.0))
        return JXF_ERR_ARG;
    reinit_launch(g, phi, phi, phi0, threshold, 0.0, -1, rhs, (cudaStream_t)stream);
    return ls_launched();
}

jxf_status jxf_ls_interface(const jxf_grid *grid, const double *W1, const double *W2, const double *gamma,
                            const double *pinf, const double *alpha, const double *dgamma, const double *normal,
                            double *ug, double *pg, jxf_stream stream) {
    JXF_RANGE("jxf_ls_interface");
    LsGrid g;
    if (ls_grid(grid, g) != JXF_OK || !W1 || !W2 || !gamma || !pinf || !alpha || !dgamma || !normal || !ug || !pg)
        return JXF_ERR_ARG;
    for (int k = 0; k < 2; ++k)
        if (!(gamma[k] > 1.0) || !(pinf[k] >= 0.0)) return JXF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (g.ndim == 3)
        k_ls_interface<3><<<ls_blocks(g), kLsThreads, 0, s>>>(g, W1, W2, gamma[0], pinf[0], gamma[1], pinf[1], alpha,
                                                             dgamma, normal, ug, pg);
    else
        k_ls_interface<2><<<ls_blocks(g), kLsThreads, 0, s>>>(g, W1, W2, gamma[0], pinf[0], gamma[1], pinf[1], alpha,
                                                             dgamma, normal, ug, pg);
    return ls_launched();
}

jxf_status jxf_ls_extend(const jxf_grid *grid, const double *phi, const double *alpha, const double *dgamma,
                         const double *normal, double *q, int nq, int mode, int steps, double *scratch,
                         jxf_stream stream) {
    JXF_RANGE("jxf_ls_extend");
    LsGrid g;
    if (ls_grid(grid, g) != JXF_OK || !phi || !alpha || !dgamma || !normal || !q || !scratch || nq < 1 || mode < 0 ||
        mode > 2 || steps < 0)
        return JXF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    return ls_extend_launch(g, phi, alpha, dgamma, normal, mode, q, -1, nullptr, nq, steps, scratch, s);
}

jxf_status jxf_ls_cut_rhs(const jxf_grid *grid, const jxf_eos *eos, const jxf_scheme *scheme, const double *apert,
                          const double *dgamma, const double *normal, const double *W, int phase, const double *ug,
                          const double *pg, double *dU, double *scratch, jxf_stream stream) {
    JXF_RANGE("jxf_ls_cut_rhs");
    LsGrid g;
    long long ncell = 0;
    if (ls_grid(grid, g) != JXF_OK || !eos || !scheme || !apert || !dgamma || !normal || !W || !ug || !pg || !dU ||
        !scratch || (phase != 1 && phase != 2))
        return JXF_ERR_ARG;
    if (jxf::validate_setup(grid, eos, scheme, &ncell, false) != JXF_OK) return JXF_ERR_ARG;
    if (eos->model != JXF_SPM || scheme->precision != JXF_FP64 || scheme->viscous || scheme->limiter ||
        scheme->recon > JXF_TENO6A_CHAR)
        return JXF_ERR_UNSUPPORTED;
    jxf::Dev P;
    jxf::fill_dev(grid, eos, scheme, ncell, P);
    P.W = const_cast<double *>(W);
    cudaStream_t s = (cudaStream_t)stream;
    const int nv = g.ndim + 2;
    for (int d = 0; d < g.ndim; ++d) {
        long long nf = 1;
        for (int e = 0; e < 3; ++e) nf *= g.n[e] + (e == d ? 1 : 0);
        const unsigned blocks = (unsigned)((nf + jxf::kFluxThreads - 1) / jxf::kFluxThreads);
        double *F = scratch + (long long)nv * g.foff[d];
        const double *A = apert + g.foff[d];
        ls_cut_faces_launch(g.ndim, d, P.teno != 0, blocks, s, P, A, phase, F);
    }
    if (g.ndim == 3)
        k_ls_cut_update<3><<<ls_blocks(g), kLsThreads, 0, s>>>(g, scratch, apert, dgamma, normal, ug, pg, phase, dU);
    else k_ls_cut_update<2><<<ls_blocks(g), kLsThreads, 0, s>>>(g, scratch, apert, dgamma, normal, ug, pg, phase, dU);
    return ls_launched();
}

jxf_status jxf_ls_mix(const jxf_grid *grid, int nv, const double *a0, const double *a1, const double *np,
                      double amix, double *aU, double *scratch, jxf_stream stream) {
    JXF_RANGE("jxf_ls_mix");
    LsGrid g;
    if (ls_grid(grid, g) != JXF_OK || nv < 1 || nv > 8 || !a0 || !a1 || !np || !aU || !scratch || !(amix >= 0.0))
        return JXF_ERR_ARG;
    for (int e = 0; e < g.ndim; ++e)  // mixing reaches one cell across a side
        if (g.bc[e][0] == JXF_BC_PERIODIC && g.n[e] < 3) return JXF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int ntrg = g.ndim == 3 ? 7 : 3;
    double *M = scratch;
    unsigned char *code = reinterpret_cast<unsigned char *>(scratch + (long long)ntrg * nv * g.ncell);
    if (g.ndim == 3) k_ls_mix_flux<3><<<ls_blocks(g), kLsThreads, 0, s>>>(g, nv, a0, a1, np, amix, aU, M, code);
    else k_ls_mix_flux<2><<<ls_blocks(g), kLsThreads, 0, s>>>(g, nv, a0, a1, np, amix, aU, M, code);
    k_ls_mix_apply<<<ls_blocks(g), kLsThreads, 0, s>>>(g, nv, M, code, aU);
    return ls_launched();
}

long long jxf_ls_step_work(const jxf_grid *grid) {
    LsGrid g;
    if (ls_grid(grid, g) != JXF_OK) return -1;
    return ls_work(g, jxf_ls_nface(grid), nullptr).total;
}

jxf_status jxf_ls_init(const jxf_grid *grid, const jxf_eos *eos1, const jxf_eos *eos2, const jxf_scheme *scheme,
                       const double *phi, const double *W1, const double *W2, double *aU1, double *aU2, double *qg,
                       double *work, jxf_stream stream) {
    JXF_RANGE("jxf_ls_init");
    LsGrid g;
    jxf::Dev P1, P2;
    jxf_status st = ls_step_args(grid, eos1, eos2, scheme, g, P1, P2);
    if (st != JXF_OK) return st;
    if (!phi || !W1 || !W2 || !aU1 || !aU2 || !qg || !work) return JXF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const LsWork w = ls_work(g, jxf_ls_nface(grid), work);
    if ((st = jxf_ls_geometry(grid, phi, w.ap, w.al0, w.dg, w.nr, stream)) != JXF_OK) return st;
    if (g.ndim == 3) k_ls_cons<3><<<ls_blocks(g), kLsThreads, 0, s>>>(P1, P2, g.ncell, w.al0, W1, W2, aU1, aU2);
    else k_ls_cons<2><<<ls_blocks(g), kLsThreads, 0, s>>>(P1, P2, g.ncell, w.al0, W1, W2, aU1, aU2);
    if ((st = ls_launched()) != JXF_OK) return st;
    return ls_interface_ext(grid, g, eos1, eos2, phi, W1, W2, w.al0, w.dg, w.nr, qg, w.scr, s);
}

jxf_status jxf_ls_step(const jxf_grid *grid, const jxf_eos *eos1, const jxf_eos *eos2, const jxf_scheme *scheme,
                       double dt, int nsteps, double amix, double *phi, double *aU1, double *aU2, double *W1,
                       double *W2, double *qg, double *work, jxf_stream stream) {
    JXF_RANGE("jxf_ls_step");
    LsGrid g;
    jxf::Dev P1, P2;
    jxf_status st = ls_step_args(grid, eos1, eos2, scheme, g, P1, P2);
    if (st != JXF_OK) return st;
    if (!phi || !aU1 || !aU2 || !W1 || !W2 || !qg || !work || nsteps < 0 || !std::isfinite(dt) ||
        !(amix >= 0.0))
        return JXF_ERR_ARG;
    if (nsteps == 0) return JXF_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const long long nc = g.ncell;
    const int nd = g.ndim, nv = nd + 2;
    const size_t ubytes = (size_t)nv * nc * sizeof(double), pbytes = (size_t)nc * sizeof(double);
    const LsWork w = ls_work(g, jxf_ls_nface(grid), work);
    double *al0 = w.al0, *al1 = w.al1;
    const double *ug = qg, *pg = qg + (long long)nd * nc;
    static const double ca[3] = {0.0, 0.75, 1.0 / 3.0}, cb[3] = {1.0, 0.25, 2.0 / 3.0};
#define LS_TRY(x)                          \
    do {                                   \
        if ((st = (x)) != JXF_OK) return st; \
    } while (0)
    // the geometry of phi on entry; afterwards each stage leaves the
    // geometry of its result in (ap, al1, dg, nr), which the next stage
    // starts from
    LS_TRY(jxf_ls_geometry(grid, phi, w.ap, al0, w.dg, w.nr, stream));
    for (int step = 0; step < nsteps; ++step) {
        if (cudaMemcpyAsync(w.U1n, aU1, ubytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(w.U2n, aU2, ubytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(w.phin, phi, pbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return JXF_ERR_CUDA;
        for (int stage = 0; stage < 3; ++stage) {
            // right-hand sides of both phases and the level set's stage
            LS_TRY(jxf_ls_cut_rhs(grid, eos1, scheme, w.ap, w.dg, w.nr, W1, 1, ug, pg, w.R1, w.scr, stream));
            LS_TRY(jxf_ls_cut_rhs(grid, eos2, scheme, w.ap, w.dg, w.nr, W2, 2, ug, pg, w.R2, w.scr, stream));
            advect_launch(g, phi, w.phin, ug, dt, stage == 0 ? 0 : 1, ca[stage], cb[stage], w.phit, s);
            k_ls_stage<<<ls_blocks_n((long long)nv * nc), kLsThreads, 0, s>>>(
                (long long)nv * nc, stage == 0, ca[stage], cb[stage], dt, w.U1n, w.R1, aU1, w.U2n, w.R2, aU2);
            LS_TRY(ls_launched());
            if (cudaMemcpyAsync(phi, w.phit, pbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                return JXF_ERR_CUDA;
            if (stage == 2) LS_TRY(jxf_ls_reinit(grid, phi, 10, 5e-2, w.scr, stream));
            // the new geometry, mixing against it, the phases' primitives and
            // ghost cells, the interface quantities
            LS_TRY(jxf_ls_geometry(grid, phi, w.ap, al1, w.dg, w.nr, stream));
            if (nd == 3) k_ls_phase2<3><<<ls_blocks(g), kLsThreads, 0, s>>>(nc, al0, al1, w.nr, w.b0, w.b1, w.n2);
            else k_ls_phase2<2><<<ls_blocks(g), kLsThreads, 0, s>>>(nc, al0, al1, w.nr, w.b0, w.b1, w.n2);
            LS_TRY(jxf_ls_mix(grid, nv, al0, al1, w.nr, amix, aU1, w.scr, stream));
            LS_TRY(jxf_ls_mix(grid, nv, w.b0, w.b1, w.n2, amix, aU2, w.scr, stream));
            if (nd == 3) {
                k_ls_prim<3><<<ls_blocks(g), kLsThreads, 0, s>>>(P1, nc, al1, aU1, W1);
                k_ls_prim<3><<<ls_blocks(g), kLsThreads, 0, s>>>(P2, nc, w.b1, aU2, W2);
            } else {
                k_ls_prim<2><<<ls_blocks(g), kLsThreads, 0, s>>>(P1, nc, al1, aU1, W1);
                k_ls_prim<2><<<ls_blocks(g), kLsThreads, 0, s>>>(P2, nc, w.b1, aU2, W2);
            }
            LS_TRY(ls_launched());
            LS_TRY(ls_extend_launch(g, phi, al1, w.dg, w.nr, 0, W1, 1, W2, nv, 10, w.scr, s));
            LS_TRY(ls_interface_ext(grid, g, eos1, eos2, phi, W1, W2, al1, w.dg, w.nr, qg, w.scr, s));
            std::swap(al0, al1);
        }
    }
#undef LS_TRY
    return JXF_OK;
}

jxf_status jxf_ls_reinit(const jxf_grid *grid, double *phi, int steps, double threshold, double *scratch,
                         jxf_stream stream) {
    JXF_RANGE("jxf_ls_reinit");
    LsGrid g;
    if (ls_grid(grid, g) != JXF_OK || !phi || !scratch || steps < 0 || !(threshold >= 0.0)) return JXF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    double *p0 = scratch, *p1 = scratch + g.ncell;
    if (steps == 0) return JXF_OK;
    if (cudaMemcpyAsync(p0, phi, (size_t)g.ncell * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return JXF_ERR_CUDA;
    const double dtau = 0.25 * g.h;
    for (int k = 0; k < steps; ++k) {
        // second-order TVD Runge-Kutta: p1 = p + dtau R(p); p <- 1/2 p + 1/2 (p1 + dtau R(p1))
        reinit_launch(g, phi, phi, p0, threshold, dtau, 0, p1, s);
        reinit_launch(g, p1, phi, p0, threshold, dtau, 1, phi, s);
    }
    return ls_launched();
}

}  // extern "C"
