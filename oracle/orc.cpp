// orc.cpp -- C entry points of the CPU oracle (test infrastructure only).
// Instantiates the templated scheme of orc_scheme.hpp for values (double),
// forward tangents (Dual) and flop counting (Counted).
#include <cstring>
#include <vector>

#include "orc.h"
#include "orc_scheme.hpp"

namespace orc {
FlopTally &tally() {
    static FlopTally t;
    return t;
}
}  // namespace orc

using namespace orc;

extern "C" {

int orc_nvar(const orc_config *c) { return Layout(*c).nv; }

void orc_prim_to_cons(const orc_config *c, const double *W, double *U) {
    const Layout L(*c);
    for (long i = 0; i < L.ncell; ++i) {
        double w[NVMAX], u[NVMAX];
        for (int v = 0; v < L.nv; ++v) w[v] = W[v * L.ncell + i];
        prim2cons(*c, L, w, u);
        for (int v = 0; v < L.nv; ++v) U[v * L.ncell + i] = u[v];
    }
}

void orc_cons_to_prim(const orc_config *c, const double *U, double *W) {
    const Layout L(*c);
    for (long i = 0; i < L.ncell; ++i) {
        double w[NVMAX], u[NVMAX];
        for (int v = 0; v < L.nv; ++v) u[v] = U[v * L.ncell + i];
        cons2prim(*c, L, u, w);
        for (int v = 0; v < L.nv; ++v) W[v * L.ncell + i] = w[v];
    }
}

void orc_rhs(const orc_config *c, const double *U, double dt, double *dU, orc_counts *counts) {
    rhs_impl<double>(*c, U, dt, dU, counts);
}

double orc_dt(const orc_config *c, const double *U, double t) { return cfl_dt(*c, U, t); }

void orc_rk3(const orc_config *c, double *U, double dt, orc_counts *counts) {
    rk3_impl<double>(*c, U, dt, counts);
}

int orc_run(const orc_config *c, double *U, int nsteps, double *t, double *dt_last,
            orc_counts *counts) {
    int taken = 0;
    for (int s = 0; s < nsteps; ++s) {
        double dt = cfl_dt(*c, U, *t);
        if (!(dt > 0.0)) break;
        rk3_impl<double>(*c, U, dt, counts);
        *t += dt;
        if (dt_last) *dt_last = dt;
        ++taken;
    }
    return taken;
}

void orc_sums(const orc_config *c, const double *U, double *sums) {
    const Layout L(*c);
    double vol = c->dx[0];
    for (int d = 1; d < L.ndim; ++d) vol *= c->dx[d];
    for (int v = 0; v < L.nv; ++v) {
        double s = 0.0;
        for (long i = 0; i < L.ncell; ++i) s += U[v * L.ncell + i] * vol;
        sums[v] = s;
    }
}

void orc_rhs_tangent(const orc_config *c, const double *U, const double *Ud, double dt,
                     double *R, double *Rd) {
    const Layout L(*c);
    const long N = (long)L.nv * L.ncell;
    std::vector<Dual> u(N), r(N);
    for (long i = 0; i < N; ++i) u[i] = Dual(U[i], Ud[i]);
    rhs_impl<Dual>(*c, u.data(), dt, r.data(), nullptr);
    for (long i = 0; i < N; ++i) {
        R[i] = r[i].v;
        Rd[i] = r[i].d;
    }
}

void orc_run_tangent(const orc_config *c, double *U, double *Ud, int nsteps, double dt) {
    const Layout L(*c);
    const long N = (long)L.nv * L.ncell;
    std::vector<Dual> u(N);
    for (long i = 0; i < N; ++i) u[i] = Dual(U[i], Ud[i]);
    for (int s = 0; s < nsteps; ++s) rk3_impl<Dual>(*c, u.data(), dt, nullptr);
    for (long i = 0; i < N; ++i) {
        U[i] = u[i].v;
        Ud[i] = u[i].d;
    }
}

void orc_count_flops(const orc_config *c, const double *U, double dt, double *out) {
    const Layout L(*c);
    const long N = (long)L.nv * L.ncell;
    std::vector<Counted> u(N), r(N);
    for (long i = 0; i < N; ++i) u[i] = Counted(U[i]);
    FlopTally &t = tally();
    t = FlopTally();
    PhaseSplit split;
    rhs_impl<Counted>(*c, u.data(), dt, r.data(), nullptr, &split);
    const long long rhs_div = t.div, rhs_sqrt = t.sqrt;
    for (int d = 0; d < 3; ++d) out[d] = (double)split.axis[d];
    out[3] = (double)split.divergence;
    out[9] = split.interface_normal * L.ncell;

    t = FlopTally();
    for (long i = 0; i < L.ncell; ++i) {
        Counted uc[NVMAX], wc[NVMAX];
        for (int v = 0; v < L.nv; ++v) uc[v] = u[v * L.ncell + i];
        cons2prim(*c, L, uc, wc);
    }
    out[4] = (double)t.total();
    const long long c2p_div = t.div, c2p_sqrt = t.sqrt;

    // RK stage combinations: stage 1, 2 and 3 forms, averaged
    t = FlopTally();
    for (long i = 0; i < N; ++i) {
        Counted a = u[i] + dt * r[i];
        Counted b = 0.75 * u[i] + 0.25 * a + (0.25 * dt) * r[i];
        Counted e = (1.0 / 3.0) * u[i] + (2.0 / 3.0) * b + (2.0 / 3.0 * dt) * r[i];
        (void)e;
    }
    out[5] = (double)t.total() / 3.0;

    // per-cell CFL rate on primitives computed outside the tally
    t = FlopTally();
    for (long i = 0; i < L.ncell; ++i) {
        double ud[NVMAX], wd[NVMAX];
        Counted wc[NVMAX];
        for (int v = 0; v < L.nv; ++v) ud[v] = U[v * L.ncell + i];
        cons2prim(*c, L, ud, wd);
        for (int v = 0; v < L.nv; ++v) wc[v] = Counted(wd[v]);
        (void)cfl_rate(*c, L, wc);
    }
    out[6] = (double)t.total();
    out[7] = (double)(rhs_div + c2p_div);
    out[8] = (double)(rhs_sqrt + c2p_sqrt);
    t = FlopTally();
}

double orc_weno5js(const double *v, double eps) {
    return weno5js(v[0], v[1], v[2], v[3], v[4], eps);
}

double orc_weno5z(const double *v, double eps) { return weno5(v[0], v[1], v[2], v[3], v[4], eps, 1); }

void orc_weno5_weights(const double *v, double eps, int z, double *omega) {
    double p[3], b[3], a[3];
    weno5_candidates(v[0], v[1], v[2], v[3], v[4], p, b);
    weno5_alpha(b, eps, z, a);
    for (int k = 0; k < 3; ++k) omega[k] = a[k] / (a[0] + a[1] + a[2]);
}

void orc_reconstruct(const orc_config *c, int d, const double *Ws, double *WL, double *WR) {
    const Layout L(*c);
    double S[6][NVMAX];
    for (int j = 0; j < 6; ++j)
        for (int v = 0; v < L.nv; ++v) S[j][v] = Ws[j * L.nv + v];
    if (c->recon == ORC_CHAR) reconstruct_char(*c, L, d, S, WL, WR);
    else reconstruct_comp(*c, L, S, WL, WR);
}

double orc_teno6a(const double *v, double *parts) {
    Teno6Parts pt;
    const double out = teno6a(v, &pt);
    if (parts) {
        for (int k = 0; k < 4; ++k) {
            parts[k] = pt.q[k];
            parts[4 + k] = pt.beta[k];
            parts[8 + k] = pt.chi[k];
            parts[12 + k] = pt.delta[k];
        }
        parts[16] = pt.ct;
        parts[17] = pt.beta6;
    }
    return out;
}

int orc_thinc_fit(double am, double ac, double ap, double nabs, double *theta, double *beta,
                  double *xc) {
    ThincFit<double> f;
    if (!thinc_fit(am, ac, ap, nabs, f)) return 0;
    *theta = f.theta;
    *beta = f.beta;
    *xc = std::log(f.y) / (2.0 * f.beta);
    return 1;
}

int orc_thinc_face(double am, double ac, double ap, double nabs, int side, double *out) {
    ThincFit<double> f;
    if (!thinc_fit(am, ac, ap, nabs, f)) return 0;
    *out = thinc_value(f, side);
    return 1;
}

void orc_thinc_normals(const orc_config *c, const double *W, double *out) {
    const Layout L(*c);
    std::vector<double> Wp((size_t)L.nv * L.npad, 0.0), nrm;
    for (int z = 0; z < L.n[2]; ++z)
        for (int y = 0; y < L.n[1]; ++y)
            for (int x = 0; x < L.n[0]; ++x)
                for (int v = 0; v < L.nv; ++v)
                    Wp[v * L.npad + L.pidx(x, y, z)] = W[v * L.ncell + L.cidx(x, y, z)];
    fill_halos(*c, L, Wp);
    thinc_normals(*c, L, Wp, nrm);
    for (int d = 0; d < L.ndim; ++d)
        for (int z = 0; z < L.n[2]; ++z)
            for (int y = 0; y < L.n[1]; ++y)
                for (int x = 0; x < L.n[0]; ++x)
                    out[d * L.ncell + L.cidx(x, y, z)] = nrm[d * L.npad + L.pidx(x, y, z)];
}

int orc_interp_limit(const orc_config *c, double *Wf, const double *W1) {
    const Layout L(*c);
    return interp_limit(*c, L, Wf, W1);
}

int orc_flux_limit_test(const orc_config *c, int d, double dt, const double *F, double uh,
                        const double *Ui, const double *Uj) {
    const Layout L(*c);
    return flux_limit_violates(*c, L, fl_lambda(*c, L, d, dt), F, uh, Ui, Uj) ? 1 : 0;
}

void orc_hllc(const orc_config *c, int d, const double *WL, const double *WR, double *F,
              double *uh) {
    const Layout L(*c);
    hllc(*c, L, d, WL, WR, F, *uh);
}

}  // extern "C"
