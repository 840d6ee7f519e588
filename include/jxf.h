/*
 * jxf.h -- C interface of the GB300 (sm_103a) compressible-flow library.
 *
 * The library advances the compressible Euler / Navier-Stokes equations on a
 * uniform Cartesian grid with the finite-volume scheme of JAX-Fluids 2.0
 * (Bezgin, Buhendwa, Adams, arXiv 2402.05193):
 *   U^{n+1} = I(U^n, R(U^n), dt)                                  (§3.4)
 * where R is the semi-discrete right-hand side of §3.2 (WENO5 reconstruction
 * with Jiang-Shu or WENO5-Z weights, component- or characteristic-wise, THINC
 * for the volume fraction, HLLC flux, central viscous and heat fluxes of
 * order 2, 4 or 6, conservative divergence, the diffuse-interface
 * volume-fraction source of §3.7), limited by the interpolation and flux
 * limiters of §3.3, for the single-phase model (§2.1) or the five-equation
 * diffuse-interface model (§2.3) with the stiffened-gas mixture EOS (§2.4),
 * and I is TVD-RK3 with a CFL time step (§3.4).
 *
 * Every computation runs in this library's CUDA kernels on the device that
 * was current when the handle was created.
 *
 * Data layout.  A state is structure-of-arrays over the interior cells:
 *   A[v][z][y][x], x fastest, no halo cells,
 * with nv = ndim + 2 variables for a single phase,
 *   U = (rho, rho u_1..rho u_ndim, E),  W = (rho, u_1..u_ndim, p),
 * or nv = ndim + 4 for the diffuse-interface model,
 *   U = (a1 rho1, a2 rho2, rho u_1..rho u_ndim, E, a1),
 *   W = (a1 rho1, a2 rho2, u_1..u_ndim, p, a1).
 * Conservative states passed to or from the library use the storage type of
 * the handle: double for JXF_FP64, float for JXF_MIXED32.
 *
 * Pointers.  Unless stated otherwise a state pointer may be host memory
 * (pageable or pinned) or device memory of the handle's device; the library
 * only borrows it for the duration of the call on the given stream, and
 * copies through cudaMemcpyAsync (so a pageable host buffer makes the call
 * synchronous with respect to the host).
 *
 * Errors.  Every call returns a jxf_status; nothing throws across this
 * interface.  Arguments are checked before any work is queued.  Failures of
 * queued device work (a CUDA error, a non-admissible state after a step, a
 * non-finite or non-positive time step) are reported by the next call that
 * synchronises: jxf_step with t_out != NULL, jxf_get_state, jxf_stats.
 * jxf_last_error() gives a message for the last failure on a handle.
 * A handle is not thread-safe: use it from one host thread and one stream at
 * a time.
 */
#ifndef JXF_H
#define JXF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct jxf_ctx *jxf_handle;
typedef struct CUstream_st *jxf_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    JXF_OK = 0,
    JXF_ERR_ARG = 1,          /* invalid argument (nothing was queued) */
    JXF_ERR_CUDA = 2,         /* a CUDA runtime call or kernel failed */
    JXF_ERR_OOM = 3,          /* device allocation failed */
    JXF_ERR_NONPHYSICAL = 4,  /* non-admissible state or non-finite dt after a step */
    JXF_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
    JXF_ERR_UNSUPPORTED = 6,  /* combination of options not implemented */
    JXF_ERR_BOUNDS = 7        /* a stencil or face index left its array: reported only by
                                 a library built with -DJXF_DEBUG (every such index is
                                 checked and clamped; release builds do not check) */
} jxf_status;

enum { JXF_BC_PERIODIC = 0, JXF_BC_ZEROGRAD = 1, JXF_BC_SYMMETRY = 2 };
/* Internal to the blocks of a decomposed grid (set by jxf_create_block, not
 * accepted by jxf_create): a block side shared with its neighbouring block,
 * whose halo cells are filled by the halo exchange. */
enum { JXF_BC_NEIGHBOR = 3 };
enum { JXF_SPM = 0, JXF_DIM = 1 };
/* reconstruction: WENO5 with Jiang-Shu (JS) or Borges et al. (Z) weights, or
 * TENO6-A (Fu et al.), on primitive variables (COMP) or in characteristic
 * space (CHAR) */
enum {
    JXF_WENO5JS_COMP = 0,
    JXF_WENO5JS_CHAR = 1,
    JXF_WENO5Z_COMP = 2,
    JXF_WENO5Z_CHAR = 3,
    JXF_TENO6A_COMP = 4,
    JXF_TENO6A_CHAR = 5
};
enum { JXF_FP64 = 0, JXF_MIXED32 = 1 };

/* Uniform Cartesian grid (§3.1).  Active axes are x (ndim >= 1), y (>= 2),
 * z (3); n[e] cells on [lo[e], hi[e]] along axis e; inactive axes must have
 * n = 1.  bc[e][0|1] is the condition at the low|high side of axis e:
 * periodic, zero-gradient, or symmetry (mirror with the normal velocity
 * reversed).  Periodic and symmetry axes need n >= 3. */
typedef struct {
    int ndim;
    int n[3];
    double lo[3], hi[3];
    int bc[3][2];
} jxf_grid;

/* Material model (§2.1-§2.5).  model = JXF_SPM uses gamma[0], pinf[0];
 * JXF_DIM mixes fluids 1 and 2 with the isobaric closure of §2.4.  The
 * dissipative fluxes (single phase only) use constant viscosity mu, Prandtl
 * number Pr and gas constant R (T = p/(rho R), lambda = mu c_p/Pr). */
typedef struct {
    int model;
    double gamma[2], pinf[2];
    double mu, Pr, R;
} jxf_eos;

/* Numerical scheme.  recon: WENO5 on primitive variables or in
 * characteristic space (§3.2), with the Jiang-Shu weights
 * alpha_k = d_k/(eps+beta_k)^2 or the WENO5-Z weights of Borges et al.,
 * alpha_k = d_k (1 + |beta_0 - beta_2|/(beta_k + eps)) (the paper's default
 * scheme), or TENO6-A on the six-cell stencil (the paper's single-phase
 * scheme: four candidate stencils, scale separation with the six-cell
 * smoothness indicator, sharp stencil selection with an adaptive cut-off,
 * renormalised linear weights of the sixth-order stencil; weno_eps unused;
 * no reverse mode); viscous: add the 4th-order central viscous and
 * heat fluxes; limiter: interpolation + flux limiter (§3.3); precision:
 * JXF_FP64, or JXF_MIXED32 (float storage and bulk arithmetic; double for the
 * time step, the conservation sums and, with p_inf != 0, the pressure
 * recovered from the conservative state).  cfl: CFL number; fixed_dt > 0
 * replaces the CFL step; t_end > 0 clips the last step to end there.
 * eps_rho, eps_rhoc2, eps_alpha <= 0 select the paper's tolerances for the
 * precision (1e-12, 1e-10, 1e-12 in FP64; 1e-10, 1e-8, 1e-10 in FP32);
 * weno_eps <= 0 selects 1e-6.  thinc: THINC reconstruction of the volume
 * fraction in interface cells (five-equation model only, §3.2 step 4): a
 * tanh profile fitted to the cell average with steepness |n_d| + 0.01 along
 * axis d (n the normal from the smoothed volume fraction of §3.7), partial
 * densities scaled consistently; JXF_ERR_UNSUPPORTED with the single-phase
 * model.  visc_order: 2, 4 or 6, the order of the central stencils of the
 * viscous and heat fluxes (§3.2, App. A: 2nd/4th/6th-order central); 0
 * selects 4. */
typedef struct {
    int recon;
    int viscous;
    int limiter;
    int precision;
    double cfl, fixed_dt, t_end;
    double eps_rho, eps_rhoc2, eps_alpha;
    double weno_eps;
    int thinc;
    int visc_order;
} jxf_scheme;

/* Create a solver for one grid on the current device; allocates all device
 * buffers (state, stage state, primitives, face fluxes, reductions).  The
 * state is zero until set.  *out receives the handle (NULL on failure). */
jxf_status jxf_create(const jxf_grid *grid, const jxf_eos *eos, const jxf_scheme *scheme,
                      jxf_handle *out);

/* Free every buffer of the handle (synchronises the device first). */
jxf_status jxf_destroy(jxf_handle h);

/* Number of variables per cell and number of cells. */
int jxf_nvar(jxf_handle h);
long long jxf_ncell(jxf_handle h);

/* Copy a conservative state U (storage type, nv * ncell values) into the
 * solver, derive its primitives and the CFL time step for the next step.
 * The simulation time is left unchanged (see jxf_set_time); the device
 * status word is cleared, then set again if the new state is not
 * admissible (reported by the next synchronising call). */
jxf_status jxf_set_state(jxf_handle h, const void *U, jxf_stream stream);

/* Same from a primitive state W given in double precision (host or device);
 * the conversion W -> U runs on the device (§2.1, §2.3, §2.4). */
jxf_status jxf_set_primitive(jxf_handle h, const double *W, jxf_stream stream);

/* Copy the current conservative state out (storage type). */
jxf_status jxf_get_state(jxf_handle h, void *U, jxf_stream stream);

/* Copy the current primitive state out (storage type). */
jxf_status jxf_get_primitive(jxf_handle h, void *W, jxf_stream stream);

/* Set / read the simulation time; setting it recomputes the clipped dt. */
jxf_status jxf_set_time(jxf_handle h, double t, jxf_stream stream);

/* dU = R(U) for the given conservative state (storage type), without
 * touching the solver's own state.  dt enters only the flux limiter's
 * pseudo-time test states (§3.3). */
jxf_status jxf_rhs(jxf_handle h, const void *U, void *dU, double dt, jxf_stream stream);

/* Advance n full TVD-RK3 steps (§3.4), each with the CFL (or fixed) time
 * step of its own U^n, clipped at t_end (steps after t_end do nothing).  The
 * steps run as one captured CUDA graph replayed n times on the stream.  If
 * t_out != NULL the call synchronises the stream, checks the device status
 * and stores the simulation time; otherwise it returns after queuing. */
jxf_status jxf_step(jxf_handle h, int n, double *t_out, jxf_stream stream);

/* Reverse mode (the differentiable solver of §6, with dt held fixed):
 * vector-Jacobian products of the right-hand side and of one TVD-RK3 step,
 * for the single-phase model with WENO5 reconstruction, without viscous
 * fluxes or limiters (other combinations, TENO6-A among them, return
 * JXF_ERR_UNSUPPORTED).  Every branch -- the min/max of
 * the wave speeds, sign(s*), the WENO weights -- is differentiated along the
 * branch the forward evaluation takes.  The solver's own state is not
 * touched; arrays are in the storage type (host or device pointers).
 *
 * jxf_rhs_vjp: U_bar = (dR/dU)^T R_bar at the state U (dt unused: no limiter).
 * jxf_step_vjp: U_bar_n = (dU^{n+1}/dU^n)^T U_bar_np1 for one RK3 step of
 * size dt from U_n (the stage states are recomputed from U_n). */
jxf_status jxf_rhs_vjp(jxf_handle h, const void *U, const void *R_bar, void *U_bar, double dt,
                       jxf_stream stream);
jxf_status jxf_step_vjp(jxf_handle h, const void *U_n, double dt, const void *U_bar_np1,
                        void *U_bar_n, jxf_stream stream);

/* Diagnostics of the current state (synchronises the last stream used):
 * sums[v] = sum over cells of U_v * cell volume in double (nv values; may be
 * NULL), *dt_last = dt of the last step taken, limited[0|1] = interpolation-
 * limited face sides | flux-limited faces accumulated since creation. */
jxf_status jxf_stats(jxf_handle h, double *sums, double *dt_last, long long *limited);

/* ----------------------------------------------------- decomposed grid --
 * One grid split into equal blocks along its last active axis (slabs), one
 * block per handle, each block on its own device or several on one device:
 * the homogeneous domain decomposition of §4.2 with the per-stage halo
 * update of §4.3 and Alg. 1.  A block stores its cells with three halo
 * planes on each side of the split axis; a face stencil that crosses a block
 * side reads them as it would read its own cells.  Along the split axis the
 * stencils of this library reach three cells (WENO5 / TENO6-A, the viscous
 * normal stencils) or a cell-centred quantity of a neighbouring cell
 * (velocity gradient, THINC normal): so face halos suffice -- no edge or
 * vertex halos -- when the cell-centred velocity gradient (viscous) and
 * interface normal (THINC) are exchanged after they are computed, instead of
 * recomputing them in the halo.
 *
 * The caller drives a step in phases and moves the halos and the reduction
 * record between them (same process: jxf_block_exchange and
 * jxf_block_allreduce; across processes: any transport, e.g. NCCL
 * point-to-point and all-reduce, on the regions jxf_block_halo and
 * jxf_block_record describe):
 *
 *   after jxf_set_state / jxf_set_primitive on every block (primitives only):
 *     exchange JXF_HALO_STATE; JXF_PHASE_AUX; exchange JXF_HALO_AUX;
 *     JXF_PHASE_REDUCE; all-reduce the records; JXF_PHASE_FINISH(0)
 *   one TVD-RK3 step: for stage s = 0, 1, 2:
 *     JXF_PHASE_STAGE(s); exchange JXF_HALO_STATE; JXF_PHASE_AUX;
 *     exchange JXF_HALO_AUX
 *   then JXF_PHASE_REDUCE; all-reduce the records; JXF_PHASE_FINISH(1).
 *
 * All blocks then hold the same time and dt, and their owned cells equal
 * the corresponding cells of a single-grid run (bit for bit: the same
 * arithmetic on the same values). */
typedef struct {
    int lo[3];      /* global index of the block's first cell per axis */
    int n[3];       /* cells of the block per axis (the grid's n except on the split axis) */
    int nbr[3][2];  /* 1: that side of the split axis faces another block (or the block
                       itself across a periodic boundary); 0 elsewhere */
} jxf_block;

/* A block of the grid `grid` (the whole grid's extents and conditions).  Only
 * the last active axis may be split: along it 0 <= lo, n >= 3, lo + n <= the
 * grid's n, and a side with nbr = 0 must be on the grid's boundary (then its
 * condition applies); a side with nbr = 1 on the grid's boundary needs a
 * periodic grid.  Cell size and all constants are those of the whole grid.
 * jxf_set_state / jxf_set_primitive / jxf_get_state / jxf_get_primitive /
 * jxf_stats take the block's owned cells (layout as above with n = block n);
 * jxf_step, jxf_rhs, jxf_set_time and the reverse mode return
 * JXF_ERR_UNSUPPORTED for a block (it steps through the phases below). */
jxf_status jxf_create_block(const jxf_grid *grid, const jxf_eos *eos, const jxf_scheme *scheme,
                            const jxf_block *block, jxf_handle *out);

enum { JXF_PHASE_STAGE = 0, JXF_PHASE_AUX = 1, JXF_PHASE_REDUCE = 2, JXF_PHASE_FINISH = 3 };
/* Queue one phase on the stream:
 * JXF_PHASE_STAGE, arg = s in {0, 1, 2}: face sweeps and cell update of RK
 *   stage s (the update of stage 2 also writes the reduction partials);
 * JXF_PHASE_AUX: the per-cell auxiliary pass of the current primitives
 *   (velocity gradient or THINC normal; nothing for schemes without one);
 * JXF_PHASE_REDUCE: fold the partials of the last update (or of the state
 *   just set) into the block's record;
 * JXF_PHASE_FINISH, arg = 0 after a new state, 1 after a step: diagnostics,
 *   time advance and the next dt (§3.4) from the block's record, which the
 *   caller has replaced by the reduction over all blocks. */
jxf_status jxf_block_phase(jxf_handle h, int phase, int arg, jxf_stream stream);

enum { JXF_HALO_STATE = 0, JXF_HALO_AUX = 1 };
/* Number of halo regions of a kind for this block (the same for every block
 * of a grid): JXF_HALO_STATE covers the primitives, the temperature
 * (viscous), the conservative state the next stage reads (limiters) and the
 * smoothed volume fraction (THINC); JXF_HALO_AUX the velocity gradient
 * (viscous) or the interface normal (THINC). */
int jxf_block_halo_count(jxf_handle h, int kind);
/* Region `index` of a kind on `side` (0 = low, 1 = high end of the split
 * axis): recv = 0 the three owned planes next to that side (what the
 * neighbour there needs), recv = 1 the three halo planes beyond it (what
 * that neighbour fills).  A region is a 2-D array in the block's device
 * memory: *height rows (one per variable or component) of *width bytes (the
 * three planes, contiguous, in increasing order along the axis), *pitch
 * bytes apart.  So the high-side send region of block k is copied row by row
 * into the low-side receive region of block k + 1, and the low-side send
 * region of block k + 1 into the high-side receive region of block k. */
jxf_status jxf_block_halo(jxf_handle h, int kind, int index, int side, int recv, void **ptr,
                          size_t *pitch, size_t *width, int *height);
/* Same-process exchange of one kind between the block `lo_blk` and the block
 * `hi_blk` above it (hi_blk may equal lo_blk or lie on another device):
 * lo_blk's high-side regions into hi_blk's low-side halo and hi_blk's
 * low-side regions into lo_blk's high-side halo, queued on the stream (the
 * caller orders it after both blocks' producing phases). */
jxf_status jxf_block_exchange(jxf_handle lo_blk, jxf_handle hi_blk, int kind, jxf_stream stream);

/* The block's reduction record in its device memory: JXF_RECORD_LEN doubles
 * [max CFL rate, min density, non-admissible flag (0/1), conservation sums
 * (nv values), unused]; the reduction over blocks takes the maximum of
 * entries 0 and 2, the minimum of entry 1 and the sum of the sums. */
#define JXF_RECORD_LEN 10
jxf_status jxf_block_record(jxf_handle h, double **record);
/* Same-process reduction of the records of n blocks (any devices) in a fixed
 * order, written back to every block's record; queued on the stream. */
jxf_status jxf_block_allreduce(const jxf_handle *blocks, int n, jxf_stream stream);

/* ------------------------------------------------------------------ batch --
 * Many independent simulations of uneven grid sizes (same dimension, one
 * material model and scheme) advanced together: every step of every
 * simulation runs in persistent kernels that pull tiles (face runs of a
 * tunable length, cell blocks) from a queue, each simulation with its own
 * CFL time step, time and diagnostics; n steps are captured as one CUDA graph
 * and replayed with a single launch.  Results equal each simulation's own
 * single-grid run.  The handle owns one arena of device memory for all
 * simulations. */
typedef struct jxf_batch_ctx *jxf_batch;

/* grids: nsim entries (sizes may differ, ndim must agree). */
jxf_status jxf_batch_create(int nsim, const jxf_grid *grids, const jxf_eos *eos,
                            const jxf_scheme *scheme, jxf_batch *out);
jxf_status jxf_batch_destroy(jxf_batch b);
int jxf_batch_nsim(jxf_batch b);
/* Per-simulation state in / out (as jxf_set_primitive / jxf_set_state /
 * jxf_get_state, for simulation sim). */
jxf_status jxf_batch_set_primitive(jxf_batch b, int sim, const double *W, jxf_stream stream);
jxf_status jxf_batch_set_state(jxf_batch b, int sim, const void *U, jxf_stream stream);
jxf_status jxf_batch_set_time(jxf_batch b, int sim, double t, jxf_stream stream);
jxf_status jxf_batch_get_state(jxf_batch b, int sim, void *U, jxf_stream stream);
/* Tile shape of the face sweeps: tile_faces (a multiple of 128) faces per
 * tile, persistent grid of blocks_per_sm blocks per SM (0: one block per
 * tile).  Picked by the autotuner (paper_2402_05193_gb300.autotune). */
jxf_status jxf_batch_set_tiling(jxf_batch b, int tile_faces, int blocks_per_sm);
/* n RK3 steps of every simulation (queued on the stream, one graph launch). */
jxf_status jxf_batch_step(jxf_batch b, int n, jxf_stream stream);
/* Simulation sim's time, conservation sums (nv values, may be NULL), last dt,
 * and the batch-wide limiter counters; synchronises the last stream used and
 * reports a non-admissible state of that simulation as JXF_ERR_NONPHYSICAL. */
jxf_status jxf_batch_stats(jxf_batch b, int sim, double *t, double *sums, double *dt_last,
                           long long *limited);
const char *jxf_batch_last_error(jxf_batch b);

/* Profiling: advance n steps exactly as jxf_step does, but launch the kernels
 * without a graph, with CUDA events on the stream around each kind, and
 * accumulate per kind k: ms[k] += device time, launches[k] += kernels
 * launched, for k = 0, 1, 2: face sweeps along x, y, z; 3: cell update (and
 * the auxiliary pass after it, where the scheme has one); 4: step
 * finalisation (its one or two kernels).  5 entries each, caller-owned host
 * arrays.  Synchronises the stream after every step; returns the status of
 * the device check. */
jxf_status jxf_step_profiled(jxf_handle h, int n, float *ms, int *launches, jxf_stream stream);

/* Host-side fault injection (tests of the failure paths): the k-th device
 * allocation made by handle creation or by a call's first use of its
 * scratch after this call (k = 0: the next one) fails as if the device were
 * out of memory -- the call returns JXF_ERR_OOM after freeing what it had
 * allocated; k < 0 disarms.  One shot; process-wide. */
void jxf_fail_allocation_after(int k);

/* Right-hand side without any device allocation -- an addition of this
 * library; the paper has no counterpart.
 *
 * dU = R(U) exactly as jxf_rhs computes it, for callers that cannot allocate
 * device memory: code running while another runtime has reserved (nearly)
 * all of the GPU's memory for its own pool, code that must not trigger the
 * implicit device-wide synchronisation of cudaFree, and loops that forbid
 * allocation after start-up.  No handle is created: grid, eos and scheme are
 * the structs jxf_create takes, U and dU are device pointers of the current
 * device (storage type of scheme->precision, layout as everywhere above), and
 * the call queues its kernels on the stream and returns.
 *
 * The intermediate arrays (primitives, temperature, velocity gradients, face
 * fluxes) live in one
 * fixed device array of JXF_STATIC_SCRATCH_BYTES inside the library, which
 * every GPU that loads the library keeps until the process exits.  A grid
 * whose intermediates do not fit (they take about 170 bytes per cell in
 * FP64, 240 with viscous fluxes, half that in FP32: roughly 1e5 cells, e.g.
 * 46^3 single-phase or 300^2 diffuse-interface in FP64) is rejected with
 * JXF_ERR_ARG and a message saying how many bytes it needs.  All calls share the array and it keeps the last
 * call's contents: calls whose kernels overlap on the same GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * The first call on each device looks up the array's device address (with
 * that device current); make that first call before any stream capture.
 * The address is kept for the life of the process: after cudaDeviceReset
 * (or any other teardown of the device's primary context) it is stale, and
 * calls on that device are not supported.  The structs are checked as
 * jxf_create checks them, except that no CFL number or fixed dt is needed.
 * msg (may be NULL) receives a message of at most msg_len bytes on failure.
 * Nothing is allocated on the device: no cudaMalloc, cudaFree or allocating
 * library routine is called. */
#define JXF_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)
jxf_status jxf_rhs_static(const jxf_grid *grid, const jxf_eos *eos, const jxf_scheme *scheme,
                          const void *U, void *dU, double dt, jxf_stream stream, char *msg,
                          size_t msg_len);

/* Test hook: q[k] = a[k] / b[k], k < n, computed on the current device with
 * the double-precision division the kernels use (a Newton-Raphson refinement
 * of the hardware reciprocal estimate, within about one ulp of IEEE
 * division for normal operands).  a, b, q: device pointers; synchronous. */
jxf_status jxf_selftest_div(const double *a, const double *b, double *q, long long n);

/* Measurement probe: fused multiply-add throughput of the plain ALUs of the
 * current device in JXF_FP64 or JXF_MIXED32 (float) arithmetic -- eight
 * independent FMA chains per thread on a grid that fills every SM, timed
 * with CUDA events; *tflops receives 2 x FMAs / time in TFLOP/s.
 * Synchronous; the denominator check of the benchmark's ALU roofline. */
jxf_status jxf_peak_probe(int precision, double *tflops);

/* Message describing the last failure on h (static string if h is NULL). */
const char *jxf_last_error(jxf_handle h);

/* ------------------------------------------------------------- level set --
 * The level-set model's data-parallel parts (§3.5 and App. D), FP64, on a
 * 2-D or 3-D grid of cubic cells (hi - lo over n equal on every active axis,
 * at least 3 cells per axis; bc as above without JXF_BC_NEIGHBOR: a mirror
 * copies the level set).  Every array is a device array of the cells (x
 * fastest) unless stated; calls are asynchronous on the stream and return
 * JXF_ERR_ARG (nothing queued) for an invalid grid or argument, JXF_ERR_CUDA
 * if a launch fails.  The library allocates nothing here; the caller owns
 * every buffer.
 *
 * The positive phase is phi > 0.  Its face apertures (App. D) come from phi
 * interpolated to the cell vertices (the mean of the 2^ndim cells around
 * each vertex): phi is taken linear along each face edge, the positive part
 * of a face is bounded by its edges and straight segments between the edges'
 * zero crossings, and a face whose two positive corners face each other
 * keeps one triangle per corner.  The interface segment is
 * dGamma = |sum_d (A_{d+} - A_{d-}) S_d e_d| (S_d the face area) and the
 * volume fraction the pyramids from the cell centre over the faces' positive
 * parts and the interface facet, (sum_f A_f S_f h/2 + dGamma phi) / (ndim
 * h^ndim), clipped to [0, 1]; the normal is grad(phi)/|grad(phi)| from
 * 4th-order central differences (0 where the gradient vanishes). */

/* Number of apertures: sum over the active axes d of the faces of axis d,
 * (n_d + 1) prod_{e != d} n_e; -1 for an invalid grid. */
long long jxf_ls_nface(const jxf_grid *grid);

/* Geometry of every cell from phi: apert[jxf_ls_nface] (the face arrays of
 * axes 0, 1(, 2) one after the other, each x fastest with n_d + 1 faces
 * along its axis), alpha[ncell], dgamma[ncell], normal[ndim][ncell]. */
jxf_status jxf_ls_geometry(const jxf_grid *grid, const double *phi, double *apert, double *alpha,
                           double *dgamma, double *normal, jxf_stream stream);

/* Right-hand side of the level-set advection (Eq. levelset_advection):
 * rhs = -u . grad(phi), each derivative the 5th-order upstream-central
 * formula of its axis (stencil i-3..i+2 for u_d >= 0, its mirror else).
 * vel: ndim cell arrays; rhs must not alias phi. */
jxf_status jxf_ls_rhs(const jxf_grid *grid, const double *phi, const double *vel, double *rhs,
                      jxf_stream stream);

/* nsteps TVD-RK3 steps (§3.4) of the advection with time step dt, phi
 * updated in place; scratch: 2 ncell doubles. */
jxf_status jxf_ls_advect(const jxf_grid *grid, double *phi, const double *vel, double dt, int nsteps,
                         double *scratch, jxf_stream stream);

/* Right-hand side of the reinitialisation equation (Eq.
 * levelset_reinitialization): rhs = -sgn(phi0) (|grad phi| - 1), |grad phi|
 * the Godunov Hamiltonian of third-order WENO one-sided derivatives (Jiang &
 * Peng; eps = 1e-6), sgn the sharp sign (0 at phi0 = 0), and rhs = 0 where
 * |rhs| <= threshold (the paper's 5e-2).  rhs must not alias phi. */
jxf_status jxf_ls_reinit_rhs(const jxf_grid *grid, const double *phi, const double *phi0, double threshold,
                             double *rhs, jxf_stream stream);

/* steps pseudo-time steps of the reinitialisation (second-order TVD
 * Runge-Kutta, dtau = 0.25 h; the paper takes 10), phi0 = phi on entry, phi
 * updated in place; scratch: 2 ncell doubles. */
jxf_status jxf_ls_reinit(const jxf_grid *grid, double *phi, int steps, double threshold, double *scratch,
                         jxf_stream stream);

/* Interface quantities (App. D): in every cut cell -- a cell holding an
 * interface segment (Sec. 3.5): 0 < alpha < 1, or dGamma > 0 where the
 * interface runs along one of its faces -- the
 * linearised two-material Riemann problem between the primitives W1 (phase
 * 1, phi > 0) and W2 (phase 2) of the cell -- 2 + ndim cell arrays each
 * (rho, u_d, p), stiffened gas gamma[p] > 1, pinf[p] >= 0 (host arrays of
 * two): Z_p = rho_p c_p, un_p = u_p . n, u_Gamma = (Z1 un1 + Z2 un2 + p2 -
 * p1)/(Z1 + Z2), p_Gamma = (Z1 p2 + Z2 p1 + Z1 Z2 (un2 - un1))/(Z1 + Z2)
 * (no surface tension).  ug[ndim][ncell] = u_Gamma n, pg[ncell]; 0 outside
 * the cut cells.  alpha, dgamma and normal are jxf_ls_geometry's outputs. */
jxf_status jxf_ls_interface(const jxf_grid *grid, const double *W1, const double *W2, const double *gamma,
                            const double *pinf, const double *alpha, const double *dgamma, const double *normal,
                            double *ug, double *pg, jxf_stream stream);

/* steps explicit Euler steps (dtau = 0.25 h) of the extension equations of
 * §3.5 on nq cell arrays q (in place), first-order upwind along the advection
 * velocity a = sdir n (normal from jxf_ls_geometry): mode 0 / 1 extend phase
 * 1's / phase 2's primitives into its ghost cells (Eq. extension_prime:
 * sdir = -1 in the cells with alpha = 0 / sdir = +1 in those with alpha = 1;
 * the paper takes 10 steps); mode 2 extends interface quantities from the
 * cut cells to both sides (Eq. extension_if: sdir = sgn(phi) in every cell
 * but the cut cells, as jxf_ls_interface defines them; 20 steps).  The
 * other cells keep their values.  alpha, dgamma, normal: jxf_ls_geometry's
 * outputs for phi.  scratch: nq ncell doubles. */
jxf_status jxf_ls_extend(const jxf_grid *grid, const double *phi, const double *alpha, const double *dgamma,
                         const double *normal, double *q, int nq, int mode, int steps, double *scratch,
                         jxf_stream stream);

/* Cut-cell right-hand side of phase 1 (phi > 0) or 2 (Eq. FVD_levelset,
 * inviscid, no surface tension): dU = d(alpha U)/dt of the phase in every
 * cell (2 + ndim cell arrays: rho, rho u_d, E).  The face fluxes are the
 * single-grid scheme's (reconstruction and HLLC of scheme->recon: WENO5-JS,
 * WENO5-Z or TENO6-A, component or characteristic) from the phase's
 * primitives W (rho, u_d,
 * p; extended into its ghost cells, e.g. by jxf_ls_extend), weighted by the
 * phase's apertures (A, resp. 1 - A); the interface pressure pg pushes the
 * phase along its inward normal (+n, resp. -n) with the force pg dGamma and
 * the power pg dGamma (ug . n) per cell volume (ug: ndim cell arrays, the
 * interface velocity vector).  The sign is the one that keeps a flat
 * interface in pressure equilibrium at rest.  apert, dgamma, normal:
 * jxf_ls_geometry's outputs.  eos: JXF_SPM with the phase's stiffened gas in
 * gamma[0], pinf[0]; scheme: JXF_FP64, no viscous flux, no limiter
 * (JXF_ERR_UNSUPPORTED otherwise).  scratch: (2 + ndim) jxf_ls_nface
 * doubles (the face fluxes). */
jxf_status jxf_ls_cut_rhs(const jxf_grid *grid, const jxf_eos *eos, const jxf_scheme *scheme, const double *apert,
                          const double *dgamma, const double *normal, const double *W, int phase,
                          const double *ug, const double *pg, double *dU, double *scratch, jxf_stream stream);

/* Conservative mixing (App. D) of one phase's volume-weighted state aU (nv
 * <= 8 cell arrays of alpha U, in place) after a stage: a0 / a1 the phase's
 * volume fraction before / after the stage, np its inward normal (ndim cell
 * arrays: +n for phase 1, -n for phase 2).  A cell that vanished (a1 = 0 <
 * a0), is new (a0 = 0 < a1) or is small (a1 < amix) mixes with its targets,
 * the neighbours one step along sign(np) on each axis, each pair of axes
 * and all three (3, resp. 7 in 3-D; a target outside a non-periodic side
 * weighs 0): weights |n_e|^2 a_t, |n_e n_f| a_t, |n_x n_y n_z|^(2/3) a_t
 * normalised to 1, fluxes M_t = beta_t/(a beta_t + a_t) [(a_t U_t) a -
 * (a U) a_t] from the states before mixing, added to the cell and taken from
 * the target.  Computed as a gather (the result does not depend on thread
 * order).  scratch: (ntargets + 1) nv ncell doubles. */
jxf_status jxf_ls_mix(const jxf_grid *grid, int nv, const double *a0, const double *a1, const double *np,
                      double amix, double *aU, double *scratch, jxf_stream stream);

/* The level-set model's time step (Alg. 2, inviscid, no surface tension)
 * for two phases on one grid: phase 1 (phi > 0) with eos1, phase 2 with
 * eos2 (both JXF_SPM, stiffened gas in gamma[0], pinf[0]); scheme: FP64,
 * inviscid, no limiter, any reconstruction.  The state, all device cell
 * arrays in the layout above: phi; aU1, aU2 (2 + ndim arrays each: the
 * volume-weighted conservative states alpha^p U^p); W1, W2 (2 + ndim
 * arrays each: rho, u_d, p of each phase, extended into its ghost cells);
 * qg (ndim + 1 arrays: the interface velocity u_Gamma n component by
 * component, then p_Gamma, extended from the cut cells).  work: device
 * buffer of jxf_ls_step_work(grid) doubles (-1: invalid grid), overwritten.
 *
 * jxf_ls_init fills aU1, aU2 and qg from phi and the primitives W1, W2
 * given in every cell.  jxf_ls_step advances the state by nsteps TVD-RK3
 * steps of size dt, in place; per stage: the cut-cell right-hand sides of
 * both phases (jxf_ls_cut_rhs) and the level set's advection with u_Gamma n
 * (HOUC5), the stage combinations, after the last stage 10
 * reinitialisation steps (threshold 5e-2), the new geometry, the mixing of
 * both phases (jxf_ls_mix, threshold amix; the paper's 0.6) against it, the
 * primitives of every cell holding a phase, their extension into the ghost
 * cells (10 steps, modes 0 and 1), the interface quantities of the cut
 * cells and their extension (20 steps).  Everything is queued on stream;
 * JXF_ERR_UNSUPPORTED for another model or scheme. */
long long jxf_ls_step_work(const jxf_grid *grid);
jxf_status jxf_ls_init(const jxf_grid *grid, const jxf_eos *eos1, const jxf_eos *eos2, const jxf_scheme *scheme,
                       const double *phi, const double *W1, const double *W2, double *aU1, double *aU2, double *qg,
                       double *work, jxf_stream stream);
jxf_status jxf_ls_step(const jxf_grid *grid, const jxf_eos *eos1, const jxf_eos *eos2, const jxf_scheme *scheme,
                       double dt, int nsteps, double amix, double *phi, double *aU1, double *aU2, double *W1,
                       double *W2, double *qg, double *work, jxf_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* JXF_H */
