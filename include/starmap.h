/*
 * starmap.h -- C ABI of the GB300 StaRMAP stepper.
 *
 * The library advances the 2D spherical-harmonics P_N system (and the slab
 * P_N system) with the staggered-grid scheme of Seibold & Frank, "StaRMAP --
 * A Second Order Staggered Grid Method for Spherical Harmonics Moment
 * Equations of Radiative Transfer" (arXiv:1211.2205):
 *
 *   d_t u + Mx d_x u + My d_y u + C u = q              (section 4, eq. hyperbolic_balance_law)
 *
 * with the moments stored on four mutually staggered grids G11, G21, G12, G22
 * (section 4.1, eqs. grid11 and staggered_grids), half-grid central
 * differences (eq. central_differences), exact integration of the decay
 * over each sub-step (eq. sub_step_solution) and the Strang composition
 * S = S^o_1/2 o S^e_1/2 o S^e_1/2 o S^o_1/2 (eq. solution_operator_full_step).
 *
 * Conventions used by every entry point
 * -------------------------------------
 * - All functions return an int status: STARMAP_OK (0) or a negative
 *   STARMAP_E_* code.  Nothing aborts, traps or exits; the message of the last
 *   failure of a handle is available from starmap_last_error().
 * - Components j = 0 .. starmap_num_moments()-1 follow the paper's real
 *   ordering R_0^0, R_1^1, I_1^1, R_2^2, I_2^2, R_2^0, R_3^3, ... (section 3,
 *   eq. transformation); for the slab system component j is psi_j.
 * - Grids are numbered 0 = G11, 1 = G21, 2 = G12, 3 = G22.  Grid g has
 *   nx_g x ny_g points (section 5.2): nx_g = n_x for G11/G12 and
 *   n_x + 1 - p_x for G21/G22, where p_x = 1 for periodic and 0 for
 *   extrapolation boundaries (eq. periodicity_flags); likewise in y.
 *   Point (i, k) of grid g lies at (x0_g + i*dx, y0_g + k*dy), see
 *   starmap_grid_info().
 * - Every host array that holds a field on a grid is dense, row-major with
 *   x fastest: element (i, k) at index k*nx_g + i.  Host arrays are always
 *   double precision; they are copied in or out (the caller keeps ownership).
 * - Device memory belongs to the library.  Pointers returned by
 *   starmap_device_ptr() are borrowed and stay valid until starmap_destroy().
 * - All work is queued on the handle's CUDA stream (the caller's stream if
 *   one was given in the config).  Entry points that return host data
 *   synchronise that stream.
 */
#ifndef STARMAP_H
#define STARMAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define STARMAP_OK            0
#define STARMAP_E_ARG        -1   /* invalid argument, size or index          */
#define STARMAP_E_CFL        -2   /* time step beyond the stability bound     */
#define STARMAP_E_NOMEM      -3   /* device or host allocation failed         */
#define STARMAP_E_CUDA       -4   /* a CUDA runtime call failed               */
#define STARMAP_E_NONFINITE  -5   /* NaN or Inf found in the state            */
#define STARMAP_E_TIMEOUT    -6   /* a bounded device wait gave up            */
#define STARMAP_E_STATE      -7   /* call not valid in the handle's state     */
#define STARMAP_E_UNSUPPORTED -8  /* configuration not supported by a kernel  */
#define STARMAP_E_GROWTH     -9   /* health check: the L2 norm grew past its bound */

/* ------------------------------------------------------------------ enums */
#define STARMAP_PERIODIC       0  /* p = 1 in eq. periodicity_flags */
#define STARMAP_EXTRAPOLATION  1  /* p = 0: ghost copies, section 4.2 */

#define STARMAP_PN2D  0           /* 2D real P_N system, section 3 */
#define STARMAP_SLAB  1           /* slab P_N system, eq. PN_slab (My = 0, ny = 1 allowed) */

#define STARMAP_FP64  0
#define STARMAP_FP32  1

/* Step schedules.  LITERAL: every step is odd half, even pair, odd half
 * (eq. solution_operator_full_step; the even pair is applied as one fused
 * pass, algebraically identical to two half-steps with frozen odd data).
 * MERGED: for time-independent material and sources the odd halves of
 * consecutive steps are merged into one full odd pass (section 5.8 remark),
 * O_1/2 (E O)^(n-1) E O_1/2 inside one starmap_step(n) call. */
#define STARMAP_SCHEDULE_LITERAL 0
#define STARMAP_SCHEDULE_MERGED  1
/* FUSED: the merged schedule with each inner (E O) pair run as one
 * temporally fused launch: per tile, the full even update and then the full
 * odd update from the new even values (on chip and in L2), so the inner
 * steps read and write the state once instead of moving it three times;
 * results equal MERGED bit for bit.  Needs the tiled kernel (FP32, 2D,
 * no closure) and a second copy of the state on the device; the step's
 * inner pairs run two at a time (an odd count runs one of them unfused).
 * E_UNSUPPORTED where the order's tables leave no room in shared memory. */
#define STARMAP_SCHEDULE_FUSED   2

/* Kernel selection for the half-step passes. */
#define STARMAP_KERNEL_AUTO    0  /* tiled kernel where supported (FP32 2D P_N, N <= 63),
                                     else gather */
#define STARMAP_KERNEL_GATHER  1  /* one thread per point, CSR loop over moments */
#define STARMAP_KERNEL_TILED   2  /* TMA-staged tiles, moments streamed by order (FP32, 2D P_N,
                                     N <= 63); tile height chosen by N, and 5-row tiles at
                                     one CTA per SM where the tables of the 10-row tiles
                                     leave no room for their ring (N >= 56 or so); up to
                                     2^36 values per staggered grid */
#define STARMAP_KERNEL_TILED_TALL  3  /* tiled, 64 x 10 tiles, one CTA per SM (E_UNSUPPORTED where
                                         their tables do not fit, N >= 56 or so) */
#define STARMAP_KERNEL_TILED_SHORT 4  /* tiled, 64 x 5 tiles, two CTAs per SM */

/* Closure of the moment hierarchy.  NONE: the P_N truncation of section 3
 * (moments of order N+1 are zero).  MLP8: not in the paper (its outlook,
 * section 7, names closures that add information at the highest order):
 * only with the 2D system and N = 7.  The handle then holds the P_8 system
 * (45 components; 36..44 are the order-8 moments R_8^8, I_8^8, R_8^6, I_8^6,
 * R_8^4, I_8^4, R_8^2, I_8^2, R_8^0).  The even passes leave the order-8
 * components alone; before every odd half-step a per-cell network (set by
 * starmap_set_closure) predicts them from the local moments of order <= 7,
 * so the order-7 rows see the P_8 couplings times the prediction instead of
 * zero.  The network runs before every odd pass: with the literal schedule
 * before each odd half-step (two evaluations per step), with the merged
 * schedule once per merged odd pass (the second odd half of a step and the
 * first of the next share one prediction; n + 1 evaluations per
 * starmap_step(h, n)).  dt defaults to the P_8 bound
 * cn * min(dx, dy) / lambda_max(Mx of P_8). */
#define STARMAP_CLOSURE_NONE 0
#define STARMAP_CLOSURE_MLP8 1

typedef struct starmap_s starmap_t;

typedef struct {
    int    system;      /* STARMAP_PN2D or STARMAP_SLAB                         */
    int    N;           /* moment order, 1 <= N <= 63                           */
    double ax[4];       /* domain xmin, xmax, ymin, ymax (par.ax, section 5.1)  */
    int    n[2];        /* cells n_x, n_y (par.n)                               */
    int    bc[2];       /* STARMAP_PERIODIC / STARMAP_EXTRAPOLATION per axis    */
    double cn;          /* CFL number: dt = cn * min(dx, dy) / lambda_max(Mx)   */
    double dt;          /* if > 0: use this time step instead of cn             */
    int    precision;   /* STARMAP_FP64 or STARMAP_FP32                         */
    int    schedule;    /* STARMAP_SCHEDULE_*                                   */
    int    kernel;      /* STARMAP_KERNEL_*                                     */
    void*  cuda_stream; /* cudaStream_t to queue work on, or NULL for the
                           library's own stream                               */
    int    closure;     /* STARMAP_CLOSURE_*                                    */
} starmap_config;

/* Fill *cfg with defaults: 2D P_N, N = 1, [0,1]^2, 16x16 periodic, cn = 0.5,
 * FP64, literal schedule, auto kernel, library stream, no closure. */
void starmap_config_default(starmap_config* cfg);

/* ----------------------------------------------------------- host math
 * Pure host functions (no GPU needed).  Moment matrices of section 3: the
 * complex P_N matrices read off eq. Pncomplex with the recursion
 * coefficients a..f, transformed by S (eq. transformation), or the slab
 * matrix of eq. PN_slab.  ncomp = (N+1)(N+2)/2 (2D) or N+1 (slab).
 *   Mx, My : caller arrays of ncomp*ncomp doubles, row-major (may be NULL)
 *   grid   : caller array of ncomp ints, grid number 0..3 per component
 *            (index sets I11, I21, I12, I22 of eq. matrix_conditions,
 *            placed as in section 5.3) (may be NULL)
 *   order  : caller array of ncomp ints, moment order l (may be NULL)
 *   lambda_max : largest |eigenvalue| of Mx (section 5.3) (may be NULL)
 * Returns STARMAP_E_ARG for N out of range or a too small ncomp_capacity. */
int starmap_host_matrices(int system, int N, int ncomp_capacity,
                          double* Mx, double* My, int* grid, int* order,
                          double* lambda_max);

/* Moments of a unit beam: the real spherical harmonic of every component
 * of the 2D system (section 3: orthonormal, without the Condon-Shortley
 * phase, so that R_1^1 ~ Omega_x and I_1^1 ~ Omega_y; R_l^m ~ sqrt2 N_l^m
 * P_l^m(mu) cos(m phi), I_l^m ~ sqrt2 N_l^m P_l^m(mu) sin(m phi), R_l^0 ~
 * N_l^0 P_l(mu)) at the direction Omega = (sqrt(1-mu^2) cos phi,
 * sqrt(1-mu^2) sin phi, mu), in the component order of starmap_host_matrices.
 * A source q(x, Omega) = qbar(x) delta(Omega - Omega_0) (the beam of
 * section 6) has the moments qbar(x) * out[j].  out holds count >= ncomp
 * doubles.  Host function.  Errors: E_ARG (slab system, N out of range,
 * |mu| > 1, short out). */
int starmap_direction_moments(int system, int N, double mu, double phi, double* out, size_t count);

/* The tiled kernel's schedule of one pass, built on the host exactly as
 * the stepper builds it (no GPU needed; for tests and inspection).  The
 * pass updates the components of order parity `parity` (1: the odd pass
 * of eq. solution_operator_full_step, 0: the even pair) from half-grid
 * differences of the other parity, streaming the inputs by order
 * (section 5.5, with the reach of Lemma 2).  frozen_top: the order-N
 * components are not updated (a closure sets them).  Outputs, each may be
 * NULL, filled up to its capacity (counts always reports the full sizes):
 *   stages : 4 ints per pipeline stage, global component indices of the
 *            stage's input R, input I, finalised output R and output I
 *            (-1 where absent), in consumer order;
 *   coef   : 16 floats per streamed input: for the four targets in reach
 *            (order l'-1 with q'-1 and q', order l'+1 with q' and q'+1) the
 *            coefficient -Mx[target][input]/dx of the input's own kind, then
 *            -My[target][input]/dy of the other kind, each value twice (one
 *            per point of an f32x2 pair); zero where a target is absent;
 *   fin    : per finalising event, the component finalised (-1: no I part);
 *   counts : {stages, streamed inputs, finalising events}.
 * Errors: E_ARG (N outside 1..63, parity not 0/1), E_UNSUPPORTED (a
 * placement the kernel does not cover). */
int starmap_tiled_schedule(int N, int parity, int frozen_top, double dx, double dy,
                           int* stages, size_t stage_capacity, float* coef, size_t coef_capacity,
                           int* fin, size_t fin_capacity, long* counts);

/* E(c) = (exp(c) - 1)/c, section 5.6 (series for |c| <= 2e-4), applied to
 * count values in place.  Host function, for tests. */
int starmap_host_expm1div(double* c, size_t count);

/* ------------------------------------------------------------ lifetime */
/* Create a stepper: builds the matrices, grid assignment and time step on
 * the host, allocates the state on the current CUDA device and zeroes it.
 * Material defaults to vacuum (sigma_a = sigma_s0 = 0), no source.
 * Errors: E_ARG (bad sizes, N, boundary, precision), E_CFL (cn beyond
 * 1/sqrt(2) in 2D or 1 in slab, or dt beyond that bound), E_UNSUPPORTED
 * (kernel choice not available for the configuration), E_NOMEM, E_CUDA.
 * On failure *out is NULL. */
int  starmap_create(const starmap_config* cfg, starmap_t** out);
void starmap_destroy(starmap_t* h);
const char* starmap_last_error(const starmap_t* h);

/* ------------------------------------------------------------ queries */
int    starmap_num_moments(const starmap_t* h);
double starmap_dt(const starmap_t* h);
double starmap_time(const starmap_t* h);
long   starmap_steps_done(const starmap_t* h);
/* Kernel actually used for the passes (STARMAP_KERNEL_GATHER, _TILED_TALL or
 * _TILED_SHORT). */
int    starmap_kernel(const starmap_t* h);
/* Component j: order l, index m (>= 0), is_imag (1 for I_l^m), grid 0..3,
 * and the size nx x ny of its grid.  Any output pointer may be NULL. */
int starmap_moment_info(const starmap_t* h, int j, int* l, int* m, int* is_imag,
                        int* grid, int* nx, int* ny);
/* Grid g: size and the coordinates of its point (0, 0); point (i, k) is at
 * (x0 + i*dx, y0 + k*dy).  eq. grid11 / staggered_grids. */
int starmap_grid_info(const starmap_t* h, int g, int* nx, int* ny,
                      double* x0, double* y0, double* dx, double* dy);

/* ----------------------------------------------------------- problem data
 * Material of section 5.7, sampled by the caller at the points of grid g
 * (nx_g*ny_g doubles each).  The decay of component j is Sigma_a for l = 0
 * and Sigma_a + Sigma_s0 - Sigma_sl for l >= 1 (section 2).  Calling this
 * for all four grids defines the medium; grids never set stay vacuum.  The
 * coefficients exp(-c dt/2) and dt/2 E(-c dt/2) are formed on the host in
 * FP64 and uploaded.  For time-dependent media call it again (at t + dt/2)
 * before each starmap_step(h, 1) with the literal schedule. */
int starmap_set_material(starmap_t* h, int g, const double* sigma_a,
                         const double* sigma_s0, size_t count);
/* Anisotropic scattering: Sigma_sl = Sigma_s0 * factor[l] for 1 <= l <= N
 * (e.g. Henyey-Greenstein g^l).  factor has N+1 entries (factor[0] unused).
 * NULL restores isotropic scattering (Sigma_sl = 0 for l >= 1).  Takes
 * effect at the next starmap_set_material() call. */
int starmap_set_scattering_factors(starmap_t* h, const double* factor, int count);
/* Source of component j (par.source / par.source_ind), sampled on the grid
 * of j; count = nx*ny of that grid.  NULL clears it. */
int starmap_set_source(starmap_t* h, int j, const double* q, size_t count);
/* Time-dependent material and sources (section 5.7): each step freezes
 * them at its midpoint t + dt/2.  With a callback set, starmap_step (and
 * starmap_advance_to) asks it before every step for sigma_a and sigma_s0 on
 * each of the four grids and for the source of every listed component at
 * t + dt/2, uploads them (starmap_set_material / starmap_set_source: the
 * decay coefficients are formed in FP64 on the host), and runs that step as
 * O_1/2 E E O_1/2 (the literal schedule, whatever the handle's schedule).
 * fn(user, field, t, g, x, y, count, out) fills out[i] with the value of
 * `field` at time t at the points (x[i], y[i]) of grid g, for
 *   field = STARMAP_FIELD_SIGMA_A, STARMAP_FIELD_SIGMA_S0, or
 *   STARMAP_FIELD_SOURCE + j: the source of component j (g is j's grid);
 * it returns 0, or nonzero to stop the step (the call then returns E_ARG
 * with the state of the steps done so far).  source_comps lists the
 * n_sources components with a source; sources of other components are
 * removed.  The handle keeps fn, user and the list until the next call;
 * fn = NULL turns the time dependence off (material and sources stay as
 * last set).  fn runs on the calling thread inside the stepping call.  With
 * the health check on, it checks after every such step.  Costs a host
 * evaluation and an upload per step: a correctness path, not a fast one. */
#define STARMAP_FIELD_SIGMA_A   0
#define STARMAP_FIELD_SIGMA_S0  1
#define STARMAP_FIELD_SOURCE    2
typedef int (*starmap_field_fn)(void* user, int field, double t, int g, const double* x,
                                const double* y, size_t count, double* out);
int starmap_set_time_dependence(starmap_t* h, starmap_field_fn fn, void* user,
                                const int* source_comps, int n_sources);
/* Set component j (initial condition, par.ic); count = nx*ny of its grid. */
int starmap_set_moment(starmap_t* h, int j, const double* u, size_t count);
/* Zero every component (and its boundary copies) on the device and reset
 * time and step count to 0; material and sources are kept.  Use before
 * setting a new initial condition with starmap_set_moment. */
int starmap_clear(starmap_t* h);
/* Set the time t (for starmap_time / advance_to bookkeeping). */
int starmap_set_time(starmap_t* h, double t);

/* ------------------------------------------------------------ stepping */
/* Advance nsteps full time steps (eq. solution_operator_full_step) with the
 * configured schedule.  Asynchronous on the handle's stream. */
int starmap_step(starmap_t* h, long nsteps);
/* Periodic health check of the stepping (failure detection; the paper has
 * no counterpart).  With every > 0, starmap_step and starmap_advance_to run
 * their steps in spans of at most `every` steps; after each span the state
 * is reduced in FP64 (the reduction of starmap_diagnostics, one host
 * synchronisation per span) and the span fails if
 *   - any value is NaN or Inf (STARMAP_E_NONFINITE), or
 *   - the discrete L2 norm (eq. discrete_L2_norm) exceeds
 *     growth * (l2_start + t_span * q_l2) (STARMAP_E_GROWTH),
 *     l2_start the norm at the span's start, t_span the span's time and
 *     q_l2 the discrete L2 norm of the sources.  The exact solution obeys
 *     this bound with growth = 1 (absorption and scattering do not increase
 *     the norm, a source adds at most t_span * q_l2); the scheme keeps its
 *     norm to a small fraction (section 6.2), so growth = 1.05 only fires
 *     on a run that diverges, such as a closure network feeding energy in.
 * On failure the state, time and step count go back to the end of the last
 * span that passed (or the start of the call), kept in a device copy of the
 * state that exists while the check is on; the call then returns the
 * error, and starmap_health reports where it happened.  Spans make the
 * merged schedule's odd halves split at their ends (equal up to rounding)
 * and, with the closure, add one network evaluation per span.
 * every = 0 turns the check off and frees the copy.  E_ARG for every < 0
 * or growth < 1. */
int starmap_set_health_check(starmap_t* h, long every, double growth);
/* State of the health check: steps done at the last span that passed, the
 * L2 norm there, and the L2 norm found at the failed span's end (NaN if
 * none failed).  Any output may be NULL. */
int starmap_health(const starmap_t* h, long* good_steps, double* l2_good, double* l2_failed);
/* The health check's decision on its own (host only; for tests and for
 * callers doing their own checks): STARMAP_E_NONFINITE if nonfinite > 0 or
 * a norm is not finite, STARMAP_E_GROWTH if l2_end > growth * (l2_start +
 * t_span * q_l2), else STARMAP_OK. */
int starmap_health_verdict(double l2_start, double l2_end, double t_span, double q_l2, double growth,
                           long nonfinite);
/* Run one pass of the step: parity 1 updates the odd components (grids
 * G21, G12) from the even ones, parity 0 the even components (G11, G22) from
 * the odd ones; which = 0 applies the half-step coefficients (tau = dt/2),
 * which = 1 the full-step ones (tau = dt: the fused even pair, or two merged
 * odd halves).  Time and step count are not advanced.  For profiling and for
 * callers composing their own schedule of eq. solution_operator_full_step.
 * With the fused schedule, parity 2 (which = 1) runs two fused inner steps
 * E_dt O_dt E_dt O_dt (two launches and their boundary refreshes). */
int starmap_pass(starmap_t* h, int parity, int which);
/* Step until t_out lies in (t, t + dt] and keep the solution of the last
 * two time levels; starmap_output() then returns the linear interpolation
 * (1 - lambda) u(t) + lambda u(t + dt), lambda = (t_out - t)/dt
 * (section 5.8).  E_ARG if t_out < current time. */
int starmap_advance_to(starmap_t* h, double t_out);
int starmap_output(starmap_t* h, int j, double* out, size_t count);

/* ------------------------------------------------------------ read-out */
/* Copy component j (nx*ny doubles of its grid) to the host. */
int starmap_moments(starmap_t* h, int j, double* out, size_t count);
/* Copy the nx x ny sub-rectangle of component j whose first point is
 * (i0, k0) of its grid to the host (nx*ny doubles, x fastest).  E_ARG if the
 * rectangle leaves the grid. */
int starmap_moments_window(starmap_t* h, int j, int i0, int k0, int nx, int ny,
                           double* out, size_t count);
/* FP64 device reductions (precision policy: FP64 only for these):
 * mass = dx dy sum R_0^0 over G11, l2 = sqrt(dx dy sum_j sum u_j^2)
 * (discrete L2 norm, eq. discrete_L2_norm), nonfinite = count of NaN/Inf
 * values.  Any output may be NULL.  Returns E_NONFINITE if nonfinite > 0. */
int starmap_diagnostics(starmap_t* h, double* mass, double* l2, long* nonfinite);
/* Allocation-free FP64 diagnostics over caller-owned device data.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory where they need the reduction (GPU memory
 * budgeted once at start-up, plug-ins running inside another framework's
 * callbacks, real-time loops where cudaMalloc and its implicit
 * synchronisation are not allowed).  It computes what starmap_diagnostics
 * computes, for ncomp components of one grid: out_device[0] = cell * sum of
 * component 0, out_device[1] = sqrt(cell * sum of squares of all values),
 * out_device[2] = number of NaN/Inf values (as a double).  Element (x, y) of
 * component k is data[origin + k*comp_stride + y*pitch + x] (elements of
 * type double for STARMAP_FP64, float for STARMAP_FP32); data and
 * out_device are device pointers owned by the caller.  Work is queued on
 * `stream` (NULL = legacy default stream); the call does not synchronise.
 *
 * Scratch: the per-block partial sums live in a library-wide array of
 * STARMAP_NOALLOC_MAX_BLOCKS x 3 doubles that every GPU loading the library
 * keeps until process exit; nothing is allocated or freed.  The first call
 * on a device looks up that array's device address (make that first call
 * before any stream capture); a call that finds a different current context
 * on that device than the lookup saw (after cudaDeviceReset, for instance)
 * looks it up again.  All calls share the array: calls whose work
 * overlaps on the GPU race and give wrong results; serialise them (one
 * stream, or events).  Every partial a call reads is written by the same
 * call, so no clearing is needed between calls.
 * Errors: E_ARG for null pointers, bad layout (pitch < nx, comp_stride <
 * pitch*ny, origin < 0), more than STARMAP_NOALLOC_MAX_ROWS rows (ncomp*ny),
 * more than STARMAP_NOALLOC_MAX_ROW_LENGTH points per row or a pitch above
 * STARMAP_NOALLOC_MAX_PITCH elements; E_CUDA if a launch or the address
 * lookup fails. */
#define STARMAP_NOALLOC_MAX_BLOCKS      1024
#define STARMAP_NOALLOC_MAX_ROWS        (1L << 26)
#define STARMAP_NOALLOC_MAX_ROW_LENGTH  (1L << 24)
#define STARMAP_NOALLOC_MAX_PITCH       (1L << 31)
int starmap_diagnostics_noalloc(const void* data, int precision, int ncomp, int nx, int ny,
                                long pitch, long comp_stride, long origin, double cell,
                                double* out_device, void* stream);
/* Rows of a grid for halo exchanges (a spatial split of the domain over
 * several GPUs; the paper has no counterpart).  pack copies rows
 * [y0, y0 + rows) of every component of grid g (in its local order) to buf,
 * laid out [component][row][x] with nx_g values per row in the run's
 * precision; unpack copies such a buffer into those rows (and marks the
 * boundary copies for refresh before the next pass).  bytes must equal
 * K_g * rows * nx_g * element size.  buf may be host or device memory
 * (any address the CUDA runtime can copy from); the copy is asynchronous on
 * the handle's stream (synchronise before reusing a host buffer).  E_ARG if
 * the rows leave the grid or the size does not match. */
int starmap_pack_rows(starmap_t* h, int g, int y0, int rows, void* buf, size_t bytes);
int starmap_unpack_rows(starmap_t* h, int g, int y0, int rows, const void* buf, size_t bytes);
/* Device pointer of component j (borrowed), with its row pitch in elements
 * and the offset of point (0,0) in elements.  Element (i, k) is at
 * ptr[offset + k*pitch + i]; indices -1 and nx_g / ny_g hold boundary
 * copies.  Element type is double (FP64) or float (FP32). */
int starmap_device_ptr(starmap_t* h, int j, void** ptr, long* pitch, long* offset);

/* ------------------------------------------------------ checkpointing */
/* Size in bytes of a state snapshot: all components in the run's precision
 * plus time and step count.  get/set copy that snapshot to/from a host
 * buffer of at least that size. */
size_t starmap_state_bytes(const starmap_t* h);
int starmap_get_state(starmap_t* h, void* buf, size_t bytes);
int starmap_set_state(starmap_t* h, const void* buf, size_t bytes);

/* Wait for all queued work of the handle. */
int starmap_sync(starmap_t* h);

/* Failure-detection self-test (no counterpart in the paper).  Runs one CTA
 * that waits, with the same bounded wait the pass kernels use (2 s limit),
 * for an mbarrier phase that nothing completes, and one that runs the
 * network kernels' three waits (2 s each): the closure kernel's and the
 * forward / training kernels' waits on an mbarrier phase that nothing
 * completes, and the wait for a TMEM slot of a pool with every slot held.
 * Each wait must give up, raise the error flag and return; the call then
 * returns STARMAP_E_TIMEOUT (the expected outcome; the CUDA context stays
 * usable).  STARMAP_E_STATE if a wait did not give up, STARMAP_E_CUDA if a
 * kernel could not run.  Synchronous (legacy default stream), about 8 s. */
int starmap_selftest_bounded_wait(void);

/* Host-side fault injection for tests (no counterpart in the paper): the
 * n-th device allocation the library makes from now on (in any handle,
 * network or batch of the process) fails as if the device were out of
 * memory, once; n = 0 disables it.  The failing call returns its error
 * status (E_NOMEM or E_CUDA) and must leave the process usable.  E_ARG for
 * n < 0.  Not thread-safe against concurrent creation calls. */
int starmap_debug_fail_allocation(int n);

/* ------------------------------------------------------ learned closure
 * Not in the paper.  The network maps 38 inputs to the 9 order-8 moments:
 *   inputs  x = (u_0 .. u_35) / s, log(1 + sigma_a), log(1 + sigma_s0), the
 *           36 moments of order <= 7 averaged to a cell centre from their
 *           own grid (two neighbours on G21 / G12, four on G22) and divided
 *           by their RMS s over the 36 values (x = 0 and s = 0 where all
 *           36 vanish); sigma from grid G11's material
 *           (starmap_set_material(h, 0, ...));
 *   network h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = W3 h2 + b3
 *           (128 hidden units per layer; BF16 operands, FP32 accumulation);
 *   output  s * y = (R_8^8, I_8^8, R_8^6, I_8^6, R_8^4, I_8^4, R_8^2,
 *           I_8^2, R_8^0) at the cell centre.  R_8^m are stored at the cell
 *           centres (G11), I_8^m at each G22 point as the mean of its four
 *           surrounding cells (boundary cells wrapped when periodic, the
 *           nearest boundary cell for extrapolation).
 * Parameters are one FP32 vector of STARMAP_MLP_PARAMS values: W1[128][38],
 * b1[128], W2[128][128], b2[128], W3[9][128], b3[9] (row-major [out][in]). */
#define STARMAP_MLP_INPUTS   38
#define STARMAP_MLP_HIDDEN   128
#define STARMAP_MLP_OUTPUTS  9
#define STARMAP_MLP_PARAMS   22665

/* Set the closure network of a STARMAP_CLOSURE_MLP8 handle from host FP32
 * parameters (count = STARMAP_MLP_PARAMS; copied, rounded to BF16 on the
 * device).  Stepping such a handle before this call returns E_STATE.
 * E_STATE also for a handle without closure. */
int starmap_set_closure(starmap_t* h, const float* params, size_t count);

/* Training samples of the current state, on the device: for each cell
 * m = iy*n_x + ix (M = n_x*n_y cells) the 38 network inputs X[m][38], the
 * scale s[m], and, if targets is not NULL, the 9 order-8 moments averaged
 * to the cell centre and divided by s[m] (0 where s[m] = 0), targets[m][9]
 * (the network's regression target).  X, scale, targets are caller-owned device pointers of M*38,
 * M and M*9 floats; count must equal M.  Needs the 2D system with N >= 7
 * (N >= 8 or the closure for targets).  Asynchronous on the handle's
 * stream. */
int starmap_closure_samples(starmap_t* h, float* X, float* scale, float* targets, size_t count);

/* Tensor-core path of the network's inference: MMA_SYNC (warp-level
 * mma.sync, BF16 -> FP32, activations in registers) or TCGEN05 (5th-gen
 * tensor cores: tcgen05.mma from shared-memory operands into a TMEM
 * accumulator).  Same arithmetic per element up to the FP32 summation
 * order.  Default for the stepper: TCGEN05; for starmap_mlp_forward:
 * MMA_SYNC.  Training always uses the mma.sync kernels. */
#define STARMAP_MLP_ENGINE_MMA_SYNC 0
#define STARMAP_MLP_ENGINE_TCGEN05  1
int starmap_set_closure_engine(starmap_t* h, int engine);

/* Network object for inference and training on the device.  All X, Y, T,
 * grad, loss and idx pointers are caller-owned device pointers; work is
 * queued on the object's stream (cuda_stream, or a library stream if NULL)
 * and does not synchronise unless stated. */
typedef struct starmap_mlp_s starmap_mlp_t;
/* Create from host FP32 parameters (count = STARMAP_MLP_PARAMS). */
int  starmap_mlp_create(const float* params, size_t count, void* cuda_stream, starmap_mlp_t** out);
void starmap_mlp_destroy(starmap_mlp_t* net);
const char* starmap_mlp_last_error(const starmap_mlp_t* net);
/* Copy the FP32 master parameters to / from the host (synchronises).
 * set_params also resets the optimiser state. */
int starmap_mlp_get_params(starmap_mlp_t* net, float* params, size_t count);
int starmap_mlp_set_params(starmap_mlp_t* net, const float* params, size_t count);
/* Y[m][9] = network(X[m][38]) for m < M. */
int starmap_mlp_forward(starmap_mlp_t* net, const float* X, size_t M, float* Y);
/* Mean squared error L = sum_{b,o} (y_bo - T_bo)^2 / (9 B) over the B
 * samples idx[0..B) (idx NULL: samples 0..B-1) and its gradient: grad gets
 * STARMAP_MLP_PARAMS floats in the parameter layout, loss one float (may be
 * NULL).  Deterministic: per-tile partial sums reduced in a fixed order. */
int starmap_mlp_loss_grad(starmap_mlp_t* net, const float* X, const float* T, const int32_t* idx,
                          size_t B, float* grad, float* loss);
/* One Adam step (Kingma & Ba 2015; beta1 = 0.9, beta2 = 0.999, eps = 1e-8,
 * bias-corrected) on the gradient of the minibatch idx[0..B) with learning
 * rate lr; loss (device, may be NULL) gets the minibatch loss before the
 * step. */
int starmap_mlp_train_step(starmap_mlp_t* net, const float* X, const float* T, const int32_t* idx,
                           size_t B, float lr, float* loss);
/* Training-input noise (not in the paper; a regulariser of the closure's
 * training): Xn[m][c] = X[m][c] + sigma * g for c < cols, Xn[m][c] = X[m][c]
 * for cols <= c < 38, over M rows of 38 floats.  g is a standard normal
 * drawn from a counter-based stream (the SplitMix64 finaliser of
 * seed * 0x9e3779b97f4a7c15 + the element's index, Box-Muller), so the same
 * seed gives the same noise.  X and Xn are caller-owned device pointers
 * (distinct or equal); queued on the network's stream.  E_ARG for cols
 * outside [0, 38] or a negative or non-finite sigma. */
int starmap_mlp_perturb_inputs(starmap_mlp_t* net, const float* X, float* Xn, size_t M, int cols, float sigma,
                               unsigned long long seed);
/* Sample order for a training epoch (not in the paper): out[i] =
 * index[perm(i)] for i < count (index NULL: out[i] = perm(i)), where perm is
 * a pseudo-random permutation of [0, count) determined by seed (a four-round
 * Feistel network on the smallest even number of bits covering count,
 * restricted to [0, count) by cycle walking), so the order is drawn on the
 * device with no host work and the same seed gives the same order.  index
 * (count int32, may be NULL) and out (count int32) are caller-owned device
 * pointers, distinct; queued on the network's stream.  E_ARG for a NULL out
 * or count >= 2^31. */
int starmap_mlp_shuffle(starmap_mlp_t* net, const int32_t* index, size_t count, unsigned long long seed,
                        int32_t* out);
/* ------------------------------------------------------------- batches
 * Not in the paper: many independent problems advanced together.  A batch
 * holds `count` FP32 2D P_N instances (any grid size, N up to the order at
 * which the tiled kernel's tables still fit in shared memory -- about 50 --, without
 * closure), each a full handle with its own state, material and sources.
 * starmap_batch_step advances every instance by nsteps of its own dt with
 * one CUDA graph launch: per pass, one persistent kernel walks the tiles of
 * all instances with each instance's own tables (work units of all
 * instances dealt to the CTAs by load: strips of consecutive tiles in y
 * for short tiles, single tiles for long ones), then one kernel refreshes
 * the boundary copies of every instance; the pass sequence of a step count
 * is captured once and replayed.  The
 * schedule is cfgs[0].schedule for all; cfgs[0].cuda_stream (if not NULL)
 * must be a non-default stream (graphs are captured on it).  Tile shape:
 * cfgs[0].kernel = STARMAP_KERNEL_TILED_TALL or _TILED_SHORT forces 64 x 10
 * or 64 x 5 tiles; anything else runs the autotuner, which builds the batch
 * with both, times four steps of each on the fresh all-zero state (left
 * zero; time and step counters are reset) and keeps the faster -- creation
 * then takes both builds and needs twice the state memory meanwhile.
 * Errors: E_UNSUPPORTED for an FP64, slab or closure instance, else as
 * starmap_create (the message names the instance). */
typedef struct starmap_batch_s starmap_batch_t;
int  starmap_batch_create(const starmap_config* cfgs, int count, starmap_batch_t** out);
void starmap_batch_destroy(starmap_batch_t* b);
const char* starmap_batch_last_error(const starmap_batch_t* b);
int  starmap_batch_count(const starmap_batch_t* b);
/* Handle of instance i (borrowed; valid until starmap_batch_destroy) for
 * the problem-data, read-out and diagnostics entry points.  Stepping an
 * instance alone with starmap_step is allowed.  NULL if i is out of range. */
starmap_t* starmap_batch_instance(starmap_batch_t* b, int i);
/* Rows of the tiles the batch uses (10 or 5) and the autotuner's ms per
 * step for each (-1 where it did not time them).  Outputs may be NULL. */
int  starmap_batch_tile_rows(const starmap_batch_t* b, double* ms_tall, double* ms_short);
/* The autotuner's choice: tile rows (10 or 5), stages per strip of short
 * tiles (96, 192 or 384), and whether it came from the tuning cache (1) or
 * from timing (0).  The autotuner (kernel AUTO) builds the batch with each
 * tile height, plans its work units with each strip length, times four
 * steps of every candidate and keeps the fastest; it caches the choice in a
 * text file keyed by the device and every instance's system, order, cells,
 * boundaries and schedule, so a later batch of the same shapes skips the
 * timing.  The file is $STARMAP_TUNE_CACHE, else
 * $HOME/.cache/starmap/batch_tune.txt; STARMAP_TUNE_CACHE=off disables it.
 * A file that cannot be read or written only means no cache. */
int  starmap_batch_tuning(const starmap_batch_t* b, int* tile_rows, int* strip_stages, int* from_cache);
/* Kernel launches of one starmap_batch_step(b, nsteps) (inside its graph). */
long starmap_batch_launches(const starmap_batch_t* b, long nsteps);
int  starmap_batch_step(starmap_batch_t* b, long nsteps);
/* Wait for the batch's stream; reports a bounded-wait failure of any
 * instance (E_TIMEOUT). */
int  starmap_batch_sync(starmap_batch_t* b);

/* The work-unit plan starmap_batch_create uses, computed on the host (no
 * GPU; for tests and inspection).  Instance i has tiles_x[i] x tiles_y[i]
 * tiles of cost[i] pipeline stages each; slots = CTAs the persistent grid
 * may hold.  items gets 4 ints per item (instance, first tile, tile count,
 * tile stride: the item covers tiles first + k * stride, k < count, tile t
 * at column t mod tiles_x, row t / tiles_x); off gets grid + 1 ints (CTA c
 * runs items off[c] .. off[c + 1] - 1); counts = {grid, items}.  Outputs
 * may be NULL and are filled up to their capacities.  E_ARG for count or
 * slots < 1 or a shape with no tiles. */
int starmap_batch_plan(const int* tiles_x, const int* tiles_y, const int* cost, int count, int slots,
                       int* items, size_t item_capacity, int* off, size_t off_capacity, long* counts);

/* Engine (STARMAP_MLP_ENGINE_*) of starmap_mlp_forward and of the loss and
 * gradient of starmap_mlp_loss_grad / starmap_mlp_train_step: MMA_SYNC
 * (mma.sync tiles, the default) or TCGEN05 (tcgen05.mma with TMEM
 * accumulators; the backward contractions read the activations MN-major).
 * Both give the same gradients up to FP32 summation order.  E_ARG for an
 * unknown engine. */
int  starmap_mlp_set_engine(starmap_mlp_t* net, int engine);
/* Number of Adam steps taken since creation or the last set_params. */
long starmap_mlp_steps(const starmap_mlp_t* net);
int  starmap_mlp_sync(starmap_mlp_t* net);

#ifdef __cplusplus
}
#endif
#endif /* STARMAP_H */
