// jxf_setup.cuh -- host-side validation of (grid, eos, scheme) and the
// kernel parameter block they define; shared by the single-grid handle and
// the batch.
#pragma once
#include <cmath>
#include <cstring>

#include "jxf.h"
#include "jxf_impl.cuh"

namespace jxf {

// Per-cell auxiliary arrays of a stage, written after the primitives: the
// viscous velocity gradient du_f/dx_e (ndim^2 arrays) or, with THINC, the
// interface-normal components |n_d| (ndim arrays) and psi (one array).
inline int aux_arrays(int ndim, const jxf_eos *eos, const jxf_scheme *scheme) {
    if (scheme->viscous && eos->model == JXF_SPM) return ndim * ndim;
    if (scheme->thinc && eos->model == JXF_DIM) return ndim + 1;
    return 0;
}

// Checks the structs (see include/jxf.h); *ncell_out receives the cell count.
// need_time_step = false leaves out the CFL / fixed-dt requirement (a bare
// right-hand side takes no time step of its own).
inline jxf_status validate_setup(const jxf_grid *grid, const jxf_eos *eos, const jxf_scheme *scheme,
                                 long long *ncell_out, bool need_time_step = true) {
    if (!grid || !eos || !scheme) return JXF_ERR_ARG;
    if (grid->ndim < 1 || grid->ndim > 3) return JXF_ERR_ARG;
    if (eos->model != JXF_SPM && eos->model != JXF_DIM) return JXF_ERR_ARG;
    if (scheme->recon < JXF_WENO5JS_COMP || scheme->recon > JXF_TENO6A_CHAR) return JXF_ERR_ARG;
    if (scheme->precision != JXF_FP64 && scheme->precision != JXF_MIXED32) return JXF_ERR_ARG;
    long long ncell = 1;
    for (int e = 0; e < 3; ++e) {
        const int n = grid->n[e];
        if (e >= grid->ndim) {
            if (n != 1) return JXF_ERR_ARG;
            continue;
        }
        if (n < 1 || !(grid->hi[e] > grid->lo[e])) return JXF_ERR_ARG;
        for (int s = 0; s < 2; ++s) {
            const int b = grid->bc[e][s];
            if (b != JXF_BC_PERIODIC && b != JXF_BC_ZEROGRAD && b != JXF_BC_SYMMETRY) return JXF_ERR_ARG;
            if (b != JXF_BC_ZEROGRAD && n < 3) return JXF_ERR_ARG;
        }
        if ((grid->bc[e][0] == JXF_BC_PERIODIC) != (grid->bc[e][1] == JXF_BC_PERIODIC)) return JXF_ERR_ARG;
        ncell *= n;
    }
    // 32-bit cell and face indices (face arrays have one more plane per axis)
    for (int d = 0; d < grid->ndim; ++d)
        if (ncell / grid->n[d] * (grid->n[d] + 1ll) >= (1ll << 31)) return JXF_ERR_ARG;
    for (int k = 0; k < (eos->model == JXF_DIM ? 2 : 1); ++k)
        if (!(eos->gamma[k] > 1.0) || !(eos->pinf[k] >= 0.0)) return JXF_ERR_ARG;
    if (scheme->viscous && eos->model != JXF_SPM) return JXF_ERR_UNSUPPORTED;
    if (scheme->thinc != 0 && scheme->thinc != 1) return JXF_ERR_ARG;
    if (scheme->visc_order != 0 && scheme->visc_order != 2 && scheme->visc_order != 4 &&
        scheme->visc_order != 6)
        return JXF_ERR_ARG;
    if (scheme->thinc && eos->model != JXF_DIM) return JXF_ERR_UNSUPPORTED;
    if (scheme->viscous && (!(eos->mu >= 0.0) || !(eos->Pr > 0.0) || !(eos->R > 0.0))) return JXF_ERR_ARG;
    if (need_time_step && !(scheme->cfl > 0.0) && !(scheme->fixed_dt > 0.0)) return JXF_ERR_ARG;
    *ncell_out = ncell;
    return JXF_OK;
}

// The grid, material and scheme constants of the kernel parameter block
// (buffers and scalar slots are left null).
inline void fill_dev(const jxf_grid *grid, const jxf_eos *eos, const jxf_scheme *scheme,
                     long long ncell, Dev &P) {
    std::memset(&P, 0, sizeof(P));
    double vol = 1.0;
    for (int e = 0; e < 3; ++e) {
        P.n[e] = e < grid->ndim ? grid->n[e] : 1;
        P.bc[e][0] = grid->bc[e][0];
        P.bc[e][1] = grid->bc[e][1];
        if (e < grid->ndim) {
            const double dx = (grid->hi[e] - grid->lo[e]) / grid->n[e];
            P.inv_dx[e] = 1.0 / dx;
            // viscous stencils (order 2 / 4 / 6): scale of the face-normal
            // derivative and of the cell-centred derivative
            const int ord = scheme->visc_order ? scheme->visc_order : 4;
            P.vis_dn[e] = 1.0 / ((ord == 2 ? 1.0 : (ord == 4 ? 24.0 : 1920.0)) * dx);
            P.vis_cd[e] = 1.0 / ((ord == 2 ? 2.0 : (ord == 4 ? 12.0 : 60.0)) * dx);
            P.fl_lam[e] = 2.0 * grid->ndim / dx;
            vol *= dx;
        }
    }
    P.ncell = ncell;
    P.vstride = ncell;
    P.cell_lo = 0;
    P.cell_hi = ncell;
    P.vol = vol;
    P.fd_cell[0] = FastDiv((unsigned)P.n[0]);
    P.fd_cell[1] = FastDiv((unsigned)P.n[1]);
    for (int d = 0; d < 3; ++d) {
        P.fd_face[d][0] = FastDiv((unsigned)(P.n[0] + (d == 0 ? 1 : 0)));
        P.fd_face[d][1] = FastDiv((unsigned)(P.n[1] + (d == 1 ? 1 : 0)));
    }
    P.dx_min = 1e300;
    for (int e = 0; e < grid->ndim; ++e) P.dx_min = fmin(P.dx_min, 1.0 / P.inv_dx[e]);
    const double g1 = eos->gamma[0], g2 = eos->model == JXF_DIM ? eos->gamma[1] : g1;
    const double p1 = eos->pinf[0], p2 = eos->model == JXF_DIM ? eos->pinf[1] : p1;
    P.A1 = 1.0 / (g1 - 1.0);
    P.A2 = 1.0 / (g2 - 1.0);
    P.B1 = g1 * p1 / (g1 - 1.0);
    P.B2 = g2 * p2 / (g2 - 1.0);
    P.gamma0 = g1;
    P.pinf0 = p1;
    P.gm1_0 = g1 - 1.0;
    P.gpinf0 = g1 * p1;
    P.stiff = (p1 != 0.0 || p2 != 0.0) ? 1 : 0;
    P.mu = eos->mu;
    P.R = eos->R;
    P.lam_heat = eos->model == JXF_SPM && scheme->viscous ? eos->mu * (g1 * eos->R / (g1 - 1.0)) / eos->Pr : 0.0;
    P.recon = scheme->recon & 1;  // JXF_WENO5JS_COMP / _CHAR: component / characteristic
    P.weno_z = (scheme->recon >> 1) == 1;
    P.teno = (scheme->recon >> 1) == 2;
    P.viscous = scheme->viscous ? 1 : 0;
    P.visc_half = scheme->visc_order == 2 ? 1 : (scheme->visc_order == 6 ? 3 : 2);
    P.thinc = scheme->thinc && eos->model == JXF_DIM ? 1 : 0;
    P.limiter = scheme->limiter ? 1 : 0;
    const bool f64 = scheme->precision == JXF_FP64;
    P.eps_rho = scheme->eps_rho > 0.0 ? scheme->eps_rho : (f64 ? 1e-12 : 1e-10);
    P.eps_rhoc2 = scheme->eps_rhoc2 > 0.0 ? scheme->eps_rhoc2 : (f64 ? 1e-10 : 1e-8);
    P.eps_alpha = scheme->eps_alpha > 0.0 ? scheme->eps_alpha : (f64 ? 1e-12 : 1e-10);
    P.weno_eps = scheme->weno_eps > 0.0 ? scheme->weno_eps : 1e-6;
    P.cfl = scheme->cfl;
    P.fixed_dt = scheme->fixed_dt;
    P.t_end = scheme->t_end;
    fill_constants(P);
}

}  // namespace jxf
