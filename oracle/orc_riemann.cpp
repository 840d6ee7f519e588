// orc_riemann.cpp -- exact solution of the 1-D Riemann problem between two
// stiffened gases (test infrastructure only).
//
// This is the reference solution of the paper's shock-tube verifications
// (§5.3: air-helium and air-water tubes compared with an exact Riemann
// solver).  Method: the classical pressure-function iteration for the star
// pressure (Newton on f_L(p) + f_R(p) + u_R - u_L = 0), with each side's
// stiffened gas reduced to an ideal gas in the shifted pressure P = p + p_inf,
// then sampling of the self-similar wave pattern.
#include <cmath>

#include "orc.h"

namespace {

struct Side {
    double g, pinf, rho, u, p;
    double P() const { return p + pinf; }  // shifted pressure
    double c() const { return std::sqrt(g * P() / rho); }
};

// Pressure function of one side and its derivative at star pressure p:
// shock (Rankine-Hugoniot) if the shifted star pressure exceeds the side's,
// rarefaction (isentropic) otherwise.
void pfun(const Side &s, double p, double &f, double &df) {
    const double Ps = p + s.pinf, Pk = s.P();
    if (Ps > Pk) {
        const double A = 2.0 / ((s.g + 1.0) * s.rho);
        const double B = (s.g - 1.0) / (s.g + 1.0) * Pk;
        const double q = std::sqrt(A / (Ps + B));
        f = (Ps - Pk) * q;
        df = q * (1.0 - 0.5 * (Ps - Pk) / (Ps + B));
    } else {
        const double ck = s.c();
        const double r = Ps / Pk;
        f = 2.0 * ck / (s.g - 1.0) * (std::pow(r, (s.g - 1.0) / (2.0 * s.g)) - 1.0);
        df = 1.0 / (s.rho * ck) * std::pow(r, -(s.g + 1.0) / (2.0 * s.g));
    }
}

// Density behind the wave on one side at star pressure p.
double star_density(const Side &s, double p) {
    const double Ps = p + s.pinf, Pk = s.P();
    const double r = Ps / Pk;
    if (Ps > Pk) {
        const double m = (s.g - 1.0) / (s.g + 1.0);
        return s.rho * (r + m) / (m * r + 1.0);
    }
    return s.rho * std::pow(r, 1.0 / s.g);
}

// Sample the left side (sign = +1) or the mirrored right side (sign = -1).
void sample_side(const Side &s, double sign, double ps, double us, double xi, double &rho,
                 double &u, double &p) {
    // mirror the right side onto the left-side formulas: u -> -u, xi -> -xi
    const double uk = sign * s.u, usm = sign * us, x = sign * xi;
    const double Ps = ps + s.pinf, Pk = s.P(), ck = s.c(), g = s.g;
    if (Ps > Pk) {
        const double S = uk - ck * std::sqrt((g + 1.0) / (2.0 * g) * Ps / Pk + (g - 1.0) / (2.0 * g));
        if (x <= S) {
            rho = s.rho; u = uk; p = s.p;
        } else {
            rho = star_density(s, ps); u = usm; p = ps;
        }
    } else {
        const double head = uk - ck;
        const double cstar = ck * std::pow(Ps / Pk, (g - 1.0) / (2.0 * g));
        const double tail = usm - cstar;
        if (x <= head) {
            rho = s.rho; u = uk; p = s.p;
        } else if (x > tail) {
            rho = star_density(s, ps); u = usm; p = ps;
        } else {  // inside the fan
            const double cf = 2.0 / (g + 1.0) * (ck + 0.5 * (g - 1.0) * (uk - x));
            u = 2.0 / (g + 1.0) * (ck + 0.5 * (g - 1.0) * uk + x);
            rho = s.rho * std::pow(cf / ck, 2.0 / (g - 1.0));
            p = Pk * std::pow(cf / ck, 2.0 * g / (g - 1.0)) - s.pinf;
        }
    }
    u = sign * u;
}

}  // namespace

extern "C" int orc_exact_riemann(double gL, double pinfL, double rhoL, double uL, double pL,
                                 double gR, double pinfR, double rhoR, double uR, double pR,
                                 const double *xi, int nxi, double *rho, double *u, double *p,
                                 int *mat, double *star) {
    const Side L{gL, pinfL, rhoL, uL, pL}, R{gR, pinfR, rhoR, uR, pR};
    // admissible star pressures keep both shifted pressures positive
    const double pmin = -(pinfL < pinfR ? pinfL : pinfR);
    double ps = 0.5 * (pL + pR);
    int it = 0;
    for (; it < 200; ++it) {
        double fl, dfl, fr, dfr;
        pfun(L, ps, fl, dfl);
        pfun(R, ps, fr, dfr);
        const double g = fl + fr + (uR - uL);
        double pn = ps - g / (dfl + dfr);
        if (pn <= pmin) pn = 0.5 * (ps + pmin);
        const double change = std::fabs(pn - ps) / (0.5 * std::fabs(pn + ps) + 1e-300);
        ps = pn;
        if (change < 1e-15) break;
    }
    if (it >= 200 || !std::isfinite(ps)) return -1;
    double fl, dfl, fr, dfr;
    pfun(L, ps, fl, dfl);
    pfun(R, ps, fr, dfr);
    const double us = 0.5 * (uL + uR) + 0.5 * (fr - fl);
    if (star) {
        star[0] = ps;
        star[1] = us;
        star[2] = star_density(L, ps);
        star[3] = star_density(R, ps);
    }
    for (int k = 0; k < nxi; ++k) {
        if (xi[k] <= us) {
            sample_side(L, 1.0, ps, us, xi[k], rho[k], u[k], p[k]);
            if (mat) mat[k] = 0;
        } else {
            sample_side(R, -1.0, ps, us, xi[k], rho[k], u[k], p[k]);
            if (mat) mat[k] = 1;
        }
    }
    return it + 1;
}
