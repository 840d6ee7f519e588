/*
 * orc.h -- C interface of the CPU oracle (test infrastructure only).
 *
 * The oracle is a plain, slow FP64 implementation of the JAX-Fluids 2.0
 * finite-volume scheme on a uniform Cartesian grid (Bezgin, Buhendwa, Adams,
 * arXiv 2402.05193): WENO5 reconstruction with Jiang-Shu (JS) or Borges (Z)
 * weights (component- or characteristic-wise, §3.2 steps 1-4 and App. C.1),
 * HLLC flux (§3.2 step 6,
 * App. C.2), interpolation and flux limiters (§3.3), 4th-order central
 * viscous and heat fluxes (§2.1, §3.2), the five-equation diffuse-interface
 * model with the stiffened-gas mixture EOS (§2.3, §2.4, §3.7), TVD-RK3 and a
 * CFL time step (§3.4); and the level-set model's data-parallel parts
 * (§3.5, App. D): interface geometry, level-set advection and
 * reinitialisation.
 *
 * It exists to check the CUDA library against: only the tests, the smoke
 * entry point and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code with the CUDA path.
 *
 * State arrays are structure-of-arrays over the interior cells only:
 * A[v][z][y][x], x fastest, nv = ndim + 2 (single phase: rho, rho*u_d, E) or
 * ndim + 4 (diffuse interface: a1*rho1, a2*rho2, rho*u_d, E, a1).
 * Primitive arrays use the same layout with (rho, u_d, p) resp.
 * (a1*rho1, a2*rho2, u_d, p, a1).
 */
#ifndef ORC_H
#define ORC_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_SPM = 0, ORC_DIM = 1 };
enum { ORC_COMP = 0, ORC_CHAR = 1 };
enum { ORC_BC_PERIODIC = 0, ORC_BC_ZEROGRAD = 1, ORC_BC_SYMMETRY = 2 };

typedef struct {
    int ndim;            /* 1, 2 or 3 active axes (x first) */
    int n[3];            /* interior cells per axis; 1 for inactive axes */
    double dx[3];        /* uniform cell size per axis */
    int bc[3][2];        /* ORC_BC_* at the low / high side of each axis */
    int model;           /* ORC_SPM or ORC_DIM */
    double gamma[2];     /* stiffened-gas gamma of fluid 1 (and fluid 2) */
    double pinf[2];      /* stiffened-gas background pressure */
    double mu, Pr, R;    /* constant viscosity, Prandtl number, gas constant */
    int recon;           /* ORC_COMP (primitive variables) or ORC_CHAR */
    int viscous;         /* 1: add the dissipative fluxes (single phase only) */
    int limiter;         /* 1: interpolation + flux limiter */
    double cfl;          /* CFL number */
    double fixed_dt;     /* > 0: use this time step instead of the CFL one */
    double t_end;        /* > 0: clip the last step to end exactly here */
    double eps_rho, eps_rhoc2, eps_alpha; /* limiter tolerances */
    double weno_eps;     /* epsilon of the WENO5 weights */
    int weno_z;          /* 0: WENO5-JS weights (Jiang & Shu), 1: WENO5-Z (Borges et al.) */
    int thinc;           /* 1: THINC interface reconstruction of a1 (five-equation model) */
    int visc_order;      /* 2, 4 or 6: order of the central dissipative stencils (0 = 4) */
    int teno;            /* 1: TENO6-A reconstruction instead of WENO5 */
} orc_config;

/* counters of limiter activity, accumulated by the calls that take them */
typedef struct {
    long long il_sides;  /* reconstructed face sides switched to first order */
    long long fl_faces;  /* faces whose flux was switched to first order */
} orc_counts;

int orc_nvar(const orc_config *c);

/* Primitive <-> conservative conversion (§2.1, §2.3, §2.4). */
void orc_prim_to_cons(const orc_config *c, const double *W, double *U);
void orc_cons_to_prim(const orc_config *c, const double *U, double *W);

/* Right-hand side R(U) of the semi-discrete form (§3.2).  dt only enters the
 * flux limiter's pseudo-time test states (§3.3). */
void orc_rhs(const orc_config *c, const double *U, double dt, double *dU,
             orc_counts *counts);

/* CFL time step from U, clipped to t_end - t (§3.4). Returns 0 when t has
 * reached t_end. */
double orc_dt(const orc_config *c, const double *U, double t);

/* One TVD-RK3 step with the given dt (§3.4), in place. */
void orc_rk3(const orc_config *c, double *U, double dt, orc_counts *counts);

/* nsteps TVD-RK3 steps, each with the CFL (or fixed) time step computed from
 * U^n and clipped at t_end.  Updates *t; returns the number of steps taken;
 * *dt_last receives the last step's dt. */
int orc_run(const orc_config *c, double *U, int nsteps, double *t,
            double *dt_last, orc_counts *counts);

/* Sum over cells of U_v * cell volume, per variable (FP64, serial). */
void orc_sums(const orc_config *c, const double *U, double *sums);

/* Forward tangent of R and of nsteps fixed-dt RK3 steps (dual numbers):
 * given U and a direction dU0, returns U(n) and its directional derivative.
 * Limiter switches and min/max/sign are differentiated along the branch
 * taken. */
void orc_rhs_tangent(const orc_config *c, const double *U, const double *Ud,
                     double dt, double *R, double *Rd);
void orc_run_tangent(const orc_config *c, double *U, double *Ud, int nsteps,
                     double dt);

/* Flop count on the given state (add/sub/mul/div/sqrt and exp/expm1/log = 1
 * each; negation, comparisons, min/max/abs = 0), every entry a total over the
 * whole grid: out[0..2] = face fluxes along x, y, z of one right-hand side
 * (reconstruct, THINC, limiters, HLLC, viscous), out[3] = divergence and
 * source, out[4] = conservative->primitive over the interior cells,
 * out[5] = one RK stage combination (mean of the three stage forms),
 * out[6] = the per-cell CFL rates, out[7] = divisions and out[8] = square
 * roots within out[0..4], out[9] = the THINC interface-normal pass (psi and
 * the normal of every cell). */
void orc_count_flops(const orc_config *c, const double *U, double dt,
                     double *out);

/* Single-face building blocks, exposed for unit pins:
 * WENO5-JS value at x_{i+1/2} from v[0..4] = v_{i-2..i+2} (§3.2 step 3);
 * reconstruction of the left/right face states of axis d from the six
 * primitive stencil cells Ws[j*nv + v], j = 0..5 <-> cells i-2..i+3, in the
 * configured (component or characteristic) mode (§3.2 steps 1-4);
 * HLLC flux F[nv] and upwinded normal velocity from two primitive face
 * states (§3.2 step 6, App. C.2). */
double orc_weno5js(const double *v, double eps);
/* WENO5-Z value from the left at x_{i+1/2} from v[0..4] = v_{i-2..i+2}, and
 * the normalised nonlinear weights omega[0..2] of either weight family
 * (z = 0: Jiang-Shu, z = 1: Borges et al.) for the same stencil. */
double orc_weno5z(const double *v, double eps);
/* TENO6-A value at x_{i+1/2} from the left from v_{i-2..i+3} (six values);
 * parts (18 values, may be null): candidates q_0..3, smoothness indicators
 * beta_0..3, scale-separation weights chi_0..3, stencil flags delta_0..3,
 * cut-off C_T, the six-cell indicator beta_6. */
double orc_teno6a(const double *v, double *parts);
void orc_weno5_weights(const double *v, double eps, int z, double *omega);

/* THINC (§3.2 step 4, five-equation model).  For the cell with volume
 * fractions am, ac, ap (neighbours along the reconstruction axis) and
 * interface-normal component |n_d| = nabs: returns 1 if it is an interface
 * cell and then the fitted profile a(xi) = 1/2 [1 + theta tanh(beta (xi + xc))],
 * xi in [0, 1] across the cell (theta, beta, xc), else 0.  orc_thinc_face
 * gives the profile's value at xi = 1 (side 0, the value from the left at
 * the cell's upper face) or xi = 0 (side 1). */
int orc_thinc_fit(double am, double ac, double ap, double nabs, double *theta, double *beta,
                  double *xc);
int orc_thinc_face(double am, double ac, double ap, double nabs, int side, double *out);
/* |n_d| of every interior cell (out[d][cell], d < ndim) from the primitive
 * state W: n = grad psi / |grad psi|, psi = a1^0.1/(a1^0.1 + (1-a1)^0.1),
 * second-order central differences with the boundary conditions. */
void orc_thinc_normals(const orc_config *c, const double *W, double *out);
void orc_reconstruct(const orc_config *c, int d, const double *Ws, double *WL,
                     double *WR);
/* Interpolation limiter of one reconstructed face side (§3.3): the
 * primitive face state Wf[nv] is replaced by the first-order cell state
 * W1[nv] when a partial density is below eps_rho, the volume fraction lies
 * outside [eps_alpha, 1 - eps_alpha] or rho c^2 is below eps_rhoc2; returns
 * 1 then, else 0 with Wf unchanged. */
int orc_interp_limit(const orc_config *c, double *Wf, const double *W1);
/* Flux-limiter test of a face of axis d (§3.3): the test states of the
 * conservative cell states Ui, Uj (nv each) on either side under the face
 * flux F[nv], the upwinded face velocity uh and the step's dt (the same
 * pseudo-time factor the right-hand side uses); returns 1 if the flux must
 * fall back to first order. */
int orc_flux_limit_test(const orc_config *c, int d, double dt, const double *F, double uh,
                        const double *Ui, const double *Uj);
void orc_hllc(const orc_config *c, int d, const double *WL, const double *WR,
              double *F, double *uh);

/* Exact solution of the 1-D Riemann problem between two stiffened gases
 * (left: gL, pinfL, rhoL, uL, pL; right likewise), sampled at the similarity
 * coordinates xi[k] = (x - x0) / t.  Outputs rho, u, p and the material
 * (0 left, 1 right) at each sample; star[0..3] = p*, u*, rho*_L, rho*_R.
 * Returns the number of Newton iterations, or -1 on failure. */
int orc_exact_riemann(double gL, double pinfL, double rhoL, double uL,
                      double pL, double gR, double pinfR, double rhoR,
                      double uR, double pR, const double *xi, int nxi,
                      double *rho, double *u, double *p, int *mat,
                      double *star);

/* ---- Level-set model (§3.5, App. D): its data-parallel parts on a grid of
 * cubic cells (ndim 2 or 3, dx equal on every axis; the functions return -1
 * otherwise).  phi is a cell array like one state variable.  Apertures are
 * the positive phase's face fractions, one face array per axis (axis d has
 * n_d + 1 faces along d, x fastest), concatenated in axis order
 * (orc_ls_nface values); alpha and dGamma are cell arrays; the normal is
 * ndim cell arrays.  The level set is advected with a cell velocity field
 * vel (ndim cell arrays). */
long long orc_ls_nface(const orc_config *c);
int orc_ls_geometry(const orc_config *c, const double *phi, double *apert, double *alpha,
                    double *dgamma, double *normal);
/* fraction of a unit square face with phi > 0 from its corner values
 * (counter-clockwise) -- the building block of the 3-D apertures */
double orc_ls_face_fraction(const double *p4);
/* R_LSA = -u . grad(phi), 5th-order upstream-central derivatives */
int orc_ls_rhs(const orc_config *c, const double *phi, const double *vel, double *rhs);
/* nsteps TVD-RK3 steps of the level-set advection with time step dt */
int orc_ls_advect(const orc_config *c, double *phi, const double *vel, double dt, int nsteps);
/* R_reinit = -sgn(phi0) (|grad phi| - 1) (Godunov Hamiltonian of third-order
 * WENO one-sided derivatives), 0 where |R| <= threshold */
int orc_ls_reinit_rhs(const orc_config *c, const double *phi, const double *phi0, double threshold,
                      double *rhs);
/* steps pseudo-time steps of reinitialisation (second-order TVD Runge-Kutta,
 * dtau = 0.25 dx), phi0 = phi on entry */
int orc_ls_reinit(const orc_config *c, double *phi, int steps, double threshold);
/* flop counts (the counting scalar of orc_count_flops): out[0] geometry,
 * out[1] one advection right-hand side, out[2] one reinitialisation
 * right-hand side (phi0 = phi), each a total over the grid; out[3], out[4]
 * per cell: one advection RK3 and one reinitialisation RK2 stage
 * combination (the mean over the stages) */
int orc_ls_count_flops(const orc_config *c, const double *phi, const double *vel, double *out);
/* Linearised two-material interface Riemann problem (App. D, no surface
 * tension): in = Z1, un1, p1, Z2, un2, p2 (acoustic impedances rho c, normal
 * velocities u_p . n with n = grad phi/|grad phi| pointing into phase 1,
 * pressures); *ug = the interface's normal velocity, *pg its pressure. */
void orc_ls_interface_riemann(const double *in, double *ug, double *pg);
/* The interface velocity (ndim cell arrays, u_Gamma n) and pressure in every
 * cut cell (0 < alpha < 1; 0 elsewhere) from the primitives W1, W2 (rho,
 * u_d, p; 2 + ndim cell arrays each) of phases 1 (phi > 0) and 2 at the
 * cell, stiffened gas gamma[p], pinf[p]. */
int orc_ls_interface_quantities(const orc_config *c, const double *phi, const double *W1, const double *W2,
                                const double *gamma, const double *pinf, double *ug, double *pg);
/* steps explicit Euler steps (dtau = 0.25 h) of the extension equations
 * (§3.5), first-order upwind, on nq cell arrays q in place: mode 0 / 1 the
 * ghost cells of phase 1 / 2 (Eq. extension_prime: the cells without volume
 * of the phase take values carried along -n^p), mode 2 the interface
 * quantities (Eq. extension_if: every cell but the cut cells, carried away
 * from the interface on both sides). */
int orc_ls_extend(const orc_config *c, const double *phi, double *q, int nq, int mode, int steps);
/* Cut-cell right-hand side of phase 1 (phi > 0) or 2 (Eq. FVD_levelset,
 * inviscid, no surface tension), d(alpha U)/dt in every cell: the face
 * fluxes of the configured reconstruction and HLLC from the phase's
 * primitives W (extended into its ghost cells; single-phase model, the
 * phase's stiffened gas in gamma[0], pinf[0], no limiter) weighted by the
 * phase's apertures (A, resp. 1 - A), plus the interface flux: the interface
 * pressure pg pushes the phase along its inward normal (+n for phase 1, -n
 * for phase 2) with force pg dGamma and power pg dGamma (ug . n) (ug: ndim
 * cell arrays, the interface velocity vector). */
int orc_ls_cut_rhs(const orc_config *c, const double *phi, const double *W, int phase, const double *ug,
                   const double *pg, double *dU);
/* Conservative mixing (App. D) of one phase's volume-weighted state aU (nv
 * cell arrays, in place) after a stage: a0 / a1 its volume fraction before /
 * after the stage, np its inward normal (ndim cell arrays).  Cells that
 * vanished, are new or are below amix move the fluxes M_t = beta_t/(a
 * beta_t + a_t) [(a_t U_t) a - (a U) a_t] to / from their targets (the
 * neighbours along sign(np) on each axis, pair of axes and all three),
 * beta from the normal and the targets' fractions, normalised; all fluxes
 * from the states before mixing. */
int orc_ls_mix(const orc_config *c, int nv, const double *a0, const double *a1, const double *np, double amix,
               double *aU);
/* The level-set model's time step (Alg. 2, inviscid, no surface tension)
 * for two phases on one grid: c1, c2 the single-phase configurations of
 * phase 1 (phi > 0) and phase 2 (the same grid and scheme, each its own
 * stiffened gas in gamma[0], pinf[0]).  orc_ls_init forms the
 * volume-weighted states aU1, aU2 (2 + ndim cell arrays each) from phi and
 * the phases' primitives W1, W2 given in every cell, and the interface
 * quantities ug (ndim cell arrays, u_Gamma n) and pg, extended.
 * orc_ls_step takes nsteps TVD-RK3 steps of size dt in place: per stage the
 * cut-cell right-hand sides of both phases and the level-set advection with
 * ug, the stage combinations, after the last stage 10 reinitialisation
 * steps, the mixing of both phases (threshold amix) against the new
 * geometry, the primitives of the cells holding each phase, their extension
 * into the ghost cells (10 steps), the interface quantities and their
 * extension (20 steps). */
int orc_ls_init(const orc_config *c1, const orc_config *c2, const double *phi, const double *W1, const double *W2,
                double *aU1, double *aU2, double *ug, double *pg);
int orc_ls_step(const orc_config *c1, const orc_config *c2, double dt, int nsteps, double amix, double *phi,
                double *aU1, double *aU2, double *W1, double *W2, double *ug, double *pg);
/* third-order WENO one-sided derivatives at the middle of v5 = phi_{i-2..i+2}
 * (cell size h): dm from the left, dp from the right */
void orc_ls_weno3_hj(const double *v5, double h, double *dm, double *dp);

#ifdef __cplusplus
}
#endif
#endif
