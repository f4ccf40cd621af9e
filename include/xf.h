/* xf.h -- C-ABI of the B300 (sm_103a) multicomponent RHS / SSP-RK3 library.
 *
 * The library advances the multicomponent compressible Navier-Stokes system of
 * arXiv 2403.05910 (XFluids), Sec. II.A Eq. 1-7, on a uniform structured grid,
 * in FP64, on one GPU. One right-hand-side evaluation L(U) (Eq. 13) consists of
 *   - primitive recovery with the Newton temperature solve of Eq. 21;
 *   - per direction, characteristic-space reconstruction (Eq. 14-15: WENO5-JS,
 *     WENO-CU6 or WENO7-JS) with local Lax-Friedrichs splitting, the
 *     multicomponent eigensystem at a Roe-averaged face state, and the partial
 *     eigensystem reconstruction (PER, Sec. III.D.3: one eigenvalue, one left
 *     row and one right column per field), optionally blended with the local
 *     Lax-Friedrichs flux to keep partial densities positive (Eq. 17-20);
 *   - 4th-order central viscous and species-diffusion fluxes (Eq. 3-6, Eq. 22,
 *     Eq. 29 transport fits, a constant Lewis number or the mixture-averaged
 *     diffusivities of Eq. 25-26);
 *   - the conservative flux difference (Eq. 13) and the SSP-RK3 stages (Eq. 16).
 * On top: the reverse mode (vector-Jacobian products) of the RHS and of a
 * step (the step's stage states recomputed, or taken from a taped step), a
 * step of a host-resident state with the copies overlapped with the compute,
 * and a batched form that advances many 2D grids in one persistent kernel
 * per stage.
 *
 * Conventions (all entry points):
 *   - FP64 throughout. Field arrays are structure-of-arrays [n_v][nz][ny][nx]
 *     (i fastest), interior cells only, n_v = dim + 2 + (N - 1) rows:
 *     conserved  U = (rho, rho u_1..rho u_dim, E, rho Y_1..rho Y_{N-1});
 *     primitive  P = (rho, u_1..u_dim, p, Y_1..Y_{N-1});  Y_N = 1 - sum.
 *     All quantities are dimensionless (rho/rho_ref, u/a_ref, p/(rho_ref a_ref^2),
 *     x/L_ref); temperatures are in kelvin.
 *   - Ownership: the caller owns every pointer it passes and may free it when
 *     the call returns (copies are enqueued on `stream`; keep host memory alive
 *     and unmodified until the stream reaches that point). The handle owns its
 *     internal device buffers (state, stage state, temperatures, per-cell
 *     primitives, face fluxes, time step, status word).
 *   - Pointers marked "host or device" may point to either (copies use
 *     unified addressing); all others must be device pointers.
 *   - Asynchrony: every call enqueues work on `stream` (a cudaStream_t, NULL =
 *     the legacy default stream) and returns without synchronising, except
 *     xf_get_status.
 *   - Errors: argument errors return XF_ERR_ARG immediately and enqueue
 *     nothing; CUDA launch/copy failures return XF_ERR_CUDA (xf_last_error
 *     gives the message). Physical faults detected on the device (NaN, rho <= 0,
 *     p <= 0, T <= 0, a non-converged Newton solve, a non-positive face sound
 *     speed) are OR-ed into a device status word and reported by xf_get_status;
 *     device code never traps.
 */
#ifndef XF_H
#define XF_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define XF_MAX_SPECIES 5

typedef enum {
  XF_OK = 0,
  XF_ERR_ARG = 1,     /* invalid argument; nothing was enqueued */
  XF_ERR_CUDA = 2,    /* a CUDA call failed (see xf_last_error) */
  XF_ERR_NONPHYS = 3, /* device saw NaN/inf, rho <= 0, p <= 0 or T <= 0 */
  XF_ERR_NEWTON = 4,  /* the temperature Newton solve did not converge */
  XF_ERR_EIGEN = 5,   /* a face sound speed squared was <= 0 */
  XF_ERR_TIMEOUT = 6, /* a bounded device wait gave up */
  XF_ERR_OOM = 7      /* device allocation failed */
} xf_status;

/* bits of the device status word (xf_get_status) */
#define XF_FLAG_NONPHYS 1u
#define XF_FLAG_NEWTON 2u
#define XF_FLAG_EIGEN 4u
#define XF_FLAG_TIMEOUT 8u

/* boundary conditions, per axis and side (applied to 3 ghost layers) */
#define XF_BC_TRANSMISSIVE 0 /* zero-gradient copy of the boundary cell */
#define XF_BC_PERIODIC 1     /* both sides of an axis must be periodic */
#define XF_BC_SYMMETRIC 2    /* mirror; the normal momentum changes sign */

/* Uniform cell-centred grid. dim in {1,2,3}; n[a] >= 3 (>= 4 with WENO7) for active axes
 * (n[a] is ignored for a >= dim); [lo, hi] is the dimensionless extent. */
typedef struct xf_grid {
  int dim;
  int64_t n[3];
  double lo[3], hi[3];
  int bc[3][2];
} xf_grid;

/* Species tables (copied at xf_create; host pointers), N = 2..XF_MAX_SPECIES.
 *  W[N]             molar masses, kg/mol (Eq. 7)
 *  T_lo, T_hi       range of the c_p polynomials, K
 *  cp_coef[N][5]    c_p,s/R_s = sum_j cp_coef[s][j] tau^j, tau = (T-T_lo)/(T_hi-T_lo),
 *                   held at its end value outside [T_lo, T_hi]
 *  h_off[N]         h_s/R_s at T_lo, K (enthalpy continues linearly outside)
 *  mu_coef[N][4]    ln mu_s [Pa s]   = sum_n mu_coef[s][n] (ln T)^n   (Eq. 29)
 *  kappa_coef[N][4] ln kappa_s [W/(m K)] likewise
 *  lewis            constant Lewis number: D_s = kappa/(rho c_p Le) for all s
 *                   (xf_opts.diffusion = 0)
 *  a_ref2, rho_ref, L_ref  reference scales (m^2/s^2, kg/m^3, m)
 *  dbin_coef[N][N][4]  ln(p D_st [Pa m^2/s]) = sum_n dbin_coef[s][t][n] (ln T)^n,
 *                   the binary diffusion coefficients of Eq. 25 in the fit form
 *                   of Eq. 29 (entries s != t are used; the caller keeps them
 *                   symmetric); required with xf_opts.diffusion = 1, else may
 *                   be NULL */
typedef struct xf_thermo {
  int n_species;
  const double *W;
  double T_lo, T_hi;
  const double *cp_coef;
  const double *h_off;
  const double *mu_coef;
  const double *kappa_coef;
  double lewis;
  double a_ref2, rho_ref, L_ref;
  const double *dbin_coef;
} xf_thermo;

/* Numerical options. weno selects the reconstruction REC of Eq. 15: 5 for
 * WENO5-JS (ref. 35), 6 for WENO-CU6 (ref. 34: linear weights (1,9,9,1)/20,
 * C = 20, q = 1, tau = beta_6 - (beta_0 + beta_2 + 4 beta_1)/6), 7 for
 * WENO7-JS (ref. 36: linear weights (1,12,18,4)/35; 8-cell stencil, 4 ghost
 * layers, so every axis needs n >= 4, else n >= 3); split must be
 * 0 (LLF); viscous switches the viscous + diffusion fluxes; convective switches
 * the inviscid fluxes (off only for testing the viscous operator);
 * newton_max/newton_rtol bound the Newton solve (stop when |dT| <= rtol T);
 * weno_eps is the absolute epsilon of the reconstructions. diffusion selects
 * the species diffusivities of Eq. 6: 0 for D_s = kappa/(rho c_p Le) for every
 * species, 1 for the mixture-averaged D_sm of Eq. 26 from the binary D_st of
 * Eq. 25 (xf_thermo.dbin_coef), with the mole fractions regularised as
 * X~_t = (max(X_t, 0) + 1e-12) / sum so that a pure species keeps a finite
 * D_sm. The adjoint entry points support every option; the batched form
 * too, with one reconstruction (weno) shared by all its instances.
 * positivity switches the positivity-preserving flux blend of Eq. 17-20 inside
 * RK stages: F* = (1 - theta) F_LF + theta F_hat per face, with the local LF
 * flux of Eq. 19 (alpha = max(|u_d| + c) of the two cells) and the smallest
 * theta in [0, 1] that keeps every partial density rho Y_s of the one-sided
 * states U_i - 2 lam F*, U_{i+1} + 2 lam F* (Eq. 18, lam = dim dt/dx_d) at or
 * above min(pos_eps, its LF value). xf_rhs (no dt) never blends, nor does
 * xf_rhs_adjoint; xf_step_rk3_adjoint and its taped form reverse the blend of
 * every stage. */
typedef struct xf_opts {
  double cfl;
  int weno;
  int split;
  int viscous;
  int convective;
  int newton_max;
  double newton_rtol;
  double weno_eps;
  int positivity;
  double pos_eps;
  int diffusion;
} xf_opts;

typedef struct xf_handle xf_handle;

/* Allocate a solver for one grid (Eq. 1-2 on that grid). Returns XF_ERR_ARG on
 * a bad grid/table/option, XF_ERR_OOM if device memory runs out. */
xf_status xf_create(const xf_grid *grid, const xf_thermo *thermo,
                    const xf_opts *opts, xf_handle **out);
void xf_destroy(xf_handle *h);

int xf_nv(const xf_handle *h);        /* n_v */
int64_t xf_cells(const xf_handle *h); /* interior cells */

/* Load the state from conserved U [n_v][cells] (host or device); T_guess
 * [cells] (host or device, nullable: 300 K) seeds the Newton warm start. */
xf_status xf_set_state(xf_handle *h, const double *U, const double *T_guess,
                       void *stream);
/* Load the state from primitives P [n_v][cells] (host or device) with the
 * ideal-gas EOS (Eq. 7): T = p/(rho R), E = rho (e(T, Y) + |u|^2/2). */
xf_status xf_set_primitive(xf_handle *h, const double *P, void *stream);
/* Copy the state out: U [n_v][cells] and/or T [cells] (host or device,
 * nullable). */
xf_status xf_get_state(xf_handle *h, double *U, double *T, void *stream);

/* dUdt = L(U) (Eq. 13) for device arrays U, dUdt [n_v][cells]. The handle's
 * state is untouched; its temperature warm start is refreshed from U. */
xf_status xf_rhs(xf_handle *h, const double *U, double *dUdt, void *stream);

/* Time step of the current state (reading of the CFL condition of Eq. 17):
 * dt = CFL / max_cells sum_d (|u_d| + c)/dx_d and, when viscous, also
 * <= CFL dx_min^2 / (2 dim max(4 mu/(3 rho), kappa/(rho c_v), D)).
 * Written to dt_dev (device). */
xf_status xf_compute_dt(xf_handle *h, double *dt_dev, void *stream);

/* One SSP-RK3 step (Eq. 16) of the handle's state. dt > 0: that step; dt <= 0:
 * the CFL step of U^n computed on the device. dt_dev_out (device, nullable)
 * receives the step used. No host synchronisation. */
xf_status xf_step_rk3(xf_handle *h, double dt, double *dt_dev_out, void *stream);
/* One xf_step_rk3 of a state that lives in host memory: U_in [n_v][cells] and
 * T_in [cells] (the Newton warm start, nullable: 300 K) are loaded as by
 * xf_set_state, the step is taken (same dt rule, dt_dev_out as above) and
 * U^{n+1} and the warm start it leaves are written to U_out and T_out
 * (nullable) as by xf_get_state; results are bitwise those three calls'.
 * U_out may equal U_in. The copies run on a copy stream of the handle,
 * overlapped with the compute in up to 8 slabs of planes of the slowest axis
 * (dim - 1; slabs of >= 16 planes and >= 2^18 cells, else one; from 4 slabs
 * on the first and the last are a quarter of the others, since their upload
 * and read-back are the copies no compute hides): stage 1
 * recovers each slab's primitives as soon as its upload lands, and stage 3
 * sends each slab's U^{n+1} out as soon as its faces and update are done.
 * Pointers: host or device; overlap needs page-locked host memory. The call
 * returns after enqueueing; `stream` reaches its end once every copy is done,
 * and the host buffers must stay valid until then. */
xf_status xf_step_rk3_host(xf_handle *h, const double *U_in, const double *T_in,
                           double *U_out, double *T_out, double dt, double *dt_dev_out,
                           void *stream);
/* nsteps steps of xf_step_rk3 (same dt rule, no dt output), replayed from a
 * CUDA graph of one step that the handle captures on first use (one per
 * temperature-buffer parity and step size; recaptured when dt changes), so
 * that small grids are not bound by launch overhead. Results are bitwise
 * those of nsteps xf_step_rk3 calls. With profiling on, the steps are plain
 * launches. nsteps >= 0. */
xf_status xf_step_rk3_n(xf_handle *h, int nsteps, double dt, void *stream);

/* ---- Adjoint (vector-Jacobian products). All arrays are device
 * arrays [n_v][cells]; results ACCUMULATE into the bar arrays (gradient
 * convention). Non-smooth points follow fixed conventions: the LLF maximum
 * passes its adjoint to the first maximal stencil cell, d|x|/dx = 0 at 0.
 *
 * U_bar += (dL/dU)^T dUdt_bar at the state U (Eq. 13-15, 3-6 reversed, the
 * Newton temperature of Eq. 21 through the implicit-function theorem). The
 * handle's state is untouched. Allocates the adjoint buffers on first use. */
xf_status xf_rhs_adjoint(xf_handle *h, const double *U, const double *dUdt_bar,
                         double *U_bar, void *stream);
/* Reverse of one fixed-dt SSP-RK3 step (Eq. 16) taken from the handle's
 * current state U^n: on entry U_bar holds dJ/dU^{n+1}, on return dJ/dU^n.
 * Recomputes the two intermediate stage states itself; dt > 0 (the adjoint
 * assumes the frozen time step). On its first call it allocates two more
 * per-cell field blocks (the fields of U^n and U1, kept between the forward
 * and reverse passes); the temperature warm start is left at that of U2. */
xf_status xf_step_rk3_adjoint(xf_handle *h, double dt, double *U_bar, void *stream);
/* Taped form of the pair above, for reverse passes that replay the forward
 * steps anyway (checkpointed segments): xf_step_rk3_tape is one fixed-dt
 * step (dt > 0; results bitwise those of xf_step_rk3) that also leaves its two
 * intermediate SSP-RK3 stage states of Eq. 16, U1 = U^n + dt L(U^n) and
 * U2 = 3/4 U^n + 1/4 (U1 + dt L(U1)), in U1 and U2 (device [n_v][cells],
 * caller-owned, distinct from each other). xf_step_rk3_adjoint_tape is
 * xf_step_rk3_adjoint from the handle's state U^n (and its temperature warm
 * start, as the tape step began from them) with those stage states given
 * instead of recomputed (same dt, U1/U2 as the tape step wrote them; not
 * checked): only the per-cell fields of U^n, U1 and U2 are recomputed, in
 * that order, so every Newton solve starts where the forward step's did and
 * the reverse sees bitwise the fields the forward faces saw (which matters
 * where a discrete choice, such as the blend's binding partial density, rests
 * on round-off). Same U_bar convention, the same two extra field blocks as
 * xf_step_rk3_adjoint, the warm start left at that of U2; results equal
 * xf_step_rk3_adjoint's up to the order of its atomic adds. */
xf_status xf_step_rk3_tape(xf_handle *h, double dt, double *U1, double *U2, void *stream);
xf_status xf_step_rk3_adjoint_tape(xf_handle *h, double dt, const double *U1, const double *U2,
                                   double *U_bar, void *stream);
/* The taped pair above with a flux tape, for handles with the positivity-
 * preserving blend (Eq. 17-20), whose reverse needs every face's unblended
 * convective flux F_hat (Eq. 15) to reverse theta. xf_step_rk3_tape_flux is
 * xf_step_rk3_tape that also writes F_hat of its three stages into Fhat
 * (device, caller-owned, xf_tape_flux_len(h) doubles: stage by stage,
 * direction by direction, each direction [n_v][faces] in the order of the
 * face fluxes, faces i fastest); xf_step_rk3_adjoint_tape_flux is
 * xf_step_rk3_adjoint_tape reading F_hat from that tape instead of
 * recomputing it (same dt, U1, U2 and Fhat as the tape step wrote them; not
 * checked). Without the blend the tape is written and not read. Results equal
 * those of the pair above up to the order of the atomic adds. XF_ERR_ARG for
 * null or non-device buffers, U1 == U2 or dt <= 0. xf_tape_flux_len returns
 * -1 for a null handle. */
int64_t xf_tape_flux_len(const xf_handle *h);
xf_status xf_step_rk3_tape_flux(xf_handle *h, double dt, double *U1, double *U2, double *Fhat,
                                void *stream);
xf_status xf_step_rk3_adjoint_tape_flux(xf_handle *h, double dt, const double *U1,
                                        const double *U2, const double *Fhat, double *U_bar,
                                        void *stream);
/* Mixing measure J = sum_cells Y_s (1 - Y_s) dV of species `species` (0-based)
 * for the state U: J_dev (device, one double) = J, U_bar = dJ/dU (overwritten). */
xf_status xf_objective_mixing(xf_handle *h, const double *U, int species,
                              double *J_dev, double *U_bar, void *stream);
/* Reverse of xf_set_primitive's EOS conversion at primitives P:
 * P_bar = (dU/dP)^T U_bar (overwritten). */
xf_status xf_set_primitive_adjoint(xf_handle *h, const double *P, const double *U_bar,
                                   double *P_bar, void *stream);

/* Synchronise `stream` and return the OR of device status bits since the last
 * xf_clear_status; the return value maps the lowest set bit to an xf_status. */
xf_status xf_get_status(xf_handle *h, uint32_t *flags, void *stream);
xf_status xf_clear_status(xf_handle *h, void *stream);

/* Per-kernel tracing. While enabled, every kernel the handle launches is
 * bracketed by two CUDA events on its stream (no synchronisation). Reading
 * synchronises on the recorded events, returns the summed milliseconds and
 * launch counts per kernel class (arrays of XF_PROF_SLOTS) and resets them. */
#define XF_PROF_SLOTS 10
#define XF_PROF_PRIM 0   /* primitive recovery + transport (+ CFL reduction) */
#define XF_PROF_DT 1     /* time-step finalisation */
#define XF_PROF_GRAD 2   /* nodal velocity derivatives */
#define XF_PROF_FACE_X 3 /* face fluxes, x (y = 4, z = 5) */
#define XF_PROF_UPDATE 6 /* conservative difference + RK3 combination */
#define XF_PROF_FACE_ADJ 7 /* face-flux adjoints (all directions) */
#define XF_PROF_PRIM_ADJ 8 /* primitive-recovery adjoint */
xf_status xf_profile_enable(xf_handle *h, int on);
xf_status xf_profile_read(xf_handle *h, double *ms, int64_t *launches);

/* FP64 FMA throughput of the current device (eight independent fma chains
 * per thread, `blocks_per_sm` blocks of 256 threads per SM, `iters` steps),
 * in TFLOP/s counting an FMA as two flops. Synchronises the device. Used to
 * state the measured FP64 ceiling beside the nominal one. */
xf_status xf_probe_fp64(int64_t iters, int blocks_per_sm, double *tflops);
/* The reciprocal the kernels use in place of division (Newton-Raphson
 * refinement of the hardware approximation; tooling, no counterpart in the
 * paper): y[i] = that reciprocal of x[i] and ref[i] = the correctly rounded
 * 1.0 / x[i], for device arrays of n doubles. Enqueued on `stream`. */
xf_status xf_probe_rcp(const double *x, double *y, double *ref, int64_t n, void *stream);
/* The exponential the primitive recovery uses for the transport fits
 * (Tang's table-driven method; tooling, no counterpart in the paper):
 * y[i] = that exp of x[i] and ref[i] = CUDA's exp(x[i]), for device arrays
 * of n doubles. Enqueued on `stream`. XF_ERR_ARG for null or non-device
 * arrays or n < 0. */
xf_status xf_probe_exp(const double *x, double *y, double *ref, int64_t n, void *stream);
/* The logarithm the primitive recovery uses for the transport fits' ln T
 * (Tang's table-driven method; tooling, no counterpart in the paper):
 * y[i] = that log of x[i] and ref[i] = CUDA's log(x[i]), for device arrays
 * of n doubles. Enqueued on `stream`. XF_ERR_ARG for null or non-device
 * arrays or n < 0. */
xf_status xf_probe_log(const double *x, double *y, double *ref, int64_t n, void *stream);

/* ---- Batched form: many independent 2D instances (uneven grids, N = 2..5)
 * advanced together. Each RK stage is ONE persistent cooperative kernel that
 * runs every phase of the stage (primitive recovery with per-instance CFL
 * reduction, per-instance dt, nodal gradients, x and y face fluxes, update)
 * for all instances, with a grid barrier between phases; a step is replayed
 * from a CUDA graph (captured per temperature-buffer parity and dt). Every cell
 * and face uses the same device code as xf_step_rk3, so each instance's result
 * is bitwise identical to a single-grid handle stepped alone.
 * The grid barrier is bounded: a block that waits past its limit sets
 * XF_FLAG_TIMEOUT in the batch status and the kernel still finishes. */
typedef struct xf_batch xf_batch;
/* grids/thermos/opts: arrays of n (host); every grid must be 2D and every
 * opts[i].weno the same (XF_ERR_ARG otherwise). */
xf_status xf_batch_create(int n, const xf_grid *grids, const xf_thermo *thermos,
                          const xf_opts *opts, xf_batch **out);
void xf_batch_destroy(xf_batch *b);
int xf_batch_size(const xf_batch *b);
/* 1 while steps replay from a CUDA graph; 0 if capture was unavailable and
 * steps are launched directly (same kernels, same results). */
int xf_batch_uses_graph(const xf_batch *b);
/* per instance i: like xf_set_primitive / xf_set_state / xf_get_state */
xf_status xf_batch_set_primitive(xf_batch *b, int i, const double *P, void *stream);
xf_status xf_batch_set_state(xf_batch *b, int i, const double *U,
                             const double *T_guess, void *stream);
xf_status xf_batch_get_state(xf_batch *b, int i, double *U, double *T, void *stream);
/* One SSP-RK3 step of every instance: dt > 0 for all, dt <= 0 each its own
 * CFL step. No host synchronisation. */
xf_status xf_batch_step_rk3(xf_batch *b, double dt, void *stream);
/* Autotuner: times `steps` CFL steps for every candidate launch shape (block
 * size 128/256, face tiles from 256x1 to 8x32 faces), keeps the fastest and
 * returns its index; ms_out (nullable, xf_batch_num_candidates() entries)
 * receives each candidate's ms per step. Restores every instance's state
 * afterwards; synchronises. */
xf_status xf_batch_autotune(xf_batch *b, int steps, int *choice, float *ms_out,
                            void *stream);
int xf_batch_num_candidates(void);
/* Select candidate `choice` (< 0: keep the current one) and report its shape. */
xf_status xf_batch_config(xf_batch *b, int choice, int *block_threads,
                          int *tile_w, int *tile_h);
/* Synchronise and return the status bits of instance i (i = -1: all, plus the
 * batch's barrier-timeout bit). */
xf_status xf_batch_get_status(xf_batch *b, int i, uint32_t *flags, void *stream);
/* Runs one bounded grid barrier that expects `extra_arrivals` more blocks than
 * the grid has, with the given limit in SM clock cycles, and returns the status
 * bits it produced: XF_FLAG_TIMEOUT when the wait ran out (extra_arrivals > 0),
 * 0 otherwise. Synchronises the device. Checks the timeout path without
 * faulting or hanging the GPU. */
xf_status xf_barrier_probe(int64_t timeout_cycles, int extra_arrivals, uint32_t *flags);

/* Allocation-free RHS. The paper has no counterpart: this entry point exists
 * for callers that may not allocate device memory -- for example a host that
 * hands all device memory to its own pool or caching allocator and forbids
 * other cudaMalloc calls, or a latency-critical loop where an allocation would
 * synchronise the device. It computes dUdt = L(U) exactly like xf_rhs, but
 * without a handle: its scratch (a device copy of the solver parameters,
 * padded per-cell fields, face fluxes, temperature warm start, status word)
 * is one fixed array in the library's
 * device memory, xf_rhs_static_capacity_bytes() bytes (32 MiB) per GPU, held
 * by every GPU that loads the library until the process exits. It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *   grid, thermo, opts: as for xf_create (host structs).
 *   U [n_v][cells], dUdt [n_v][cells]: device arrays owned by the caller.
 *   T_guess [cells]: device array seeding the Newton warm start (nullable:
 *     300 K); it is read, not updated.
 *   flags_out: host pointer (nullable). When given, the call synchronises
 *     `stream` and stores the device status bits (XF_FLAG_*) of this call.
 * Returns XF_ERR_ARG, with the required and available sizes in
 * xf_last_error(), when the grid's scratch exceeds the capacity (about
 * 3.5e4 cells in 3D with 5 species, 8e4 cells in 2D with 3 species); also
 * XF_ERR_ARG, with xf_last_error() naming the cause, for null or non-device
 * U / dUdt / T_guess and for invalid grid, thermo or options.
 * The array is part of the library's device image: it is placed in device
 * memory when the library's kernels are loaded on a device (at the latest on
 * the first call), not by any call.
 * The first call on each device looks up the array's device address (with
 * that device current) and caches it; make that first call before any stream
 * capture. Every call on a device shares the one array and leaves its contents
 * behind (the status word and accumulators are cleared at the start of each
 * call): calls that overlap on the GPU -- on different streams or from
 * different threads -- race and must not be issued. */
xf_status xf_rhs_static(const xf_grid *grid, const xf_thermo *thermo,
                        const xf_opts *opts, const double *U,
                        const double *T_guess, double *dUdt,
                        uint32_t *flags_out, void *stream);
int64_t xf_rhs_static_capacity_bytes(void);

const char *xf_status_str(xf_status s);
const char *xf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
