/*
 * oecdg.h -- C-ABI of the GB300 (sm_103a) FP64 implementation of the
 * oscillation-eliminating central DG (OECDG) forward time step of
 * Peng, Wu, Yuan, arXiv:2503.12473.
 *
 * Scope of the CUDA path:
 *   - 2D: the tensor space Q^k or the total-degree space P^k, k = 1, 2 or 3,
 *     linear advection, Burgers (f = g = u^2/2) and the compressible Euler
 *     equations.  Q^2 with advection or Euler and forward Euler, SSP-RK2 or
 *     SSP-RK3 runs on the tiled, sum-factorised kernels (the measured hot
 *     path); every other 2D configuration, RK4 included, on the
 *     degree-generic kernels;
 *   - 1D: P^k with k = 1, 2 or 3, linear advection, Burgers (f = u^2/2) and
 *     the 1D Euler equations;
 *   - time stepping: forward Euler, SSP-RK2, SSP-RK3 or the classical
 *     four-stage RK4 (written in Shu-Osher form, used for Table 2);
 * with periodic, transmissive or (Euler) reflective boundaries, set per side.
 *
 * Conventions shared by every entry point
 *   - Every call returns a cdg_status; nothing throws, aborts or exits.
 *     cdg_last_error(ctx) returns a static text for the last failure.
 *   - State arrays are FP64 DEVICE pointers owned by the caller, with
 *     cdg_state_numel() elements laid out as
 *         u[mesh][field][mode][j][i]     (i fastest),
 *     mesh 0 = primal mesh T_h^C, mesh 1 = dual mesh T_h^D (the primal mesh
 *     shifted by (+hx/2, +hy/2); dual cell (i,j) is centred on primal vertex
 *     (i+1, j+1)); field = conserved variable (Euler 2D: rho, rho u, rho v, E;
 *     1D: rho, rho v, E; advection: u); mode = Legendre mode (a,b) of the
 *     unnormalised Legendre polynomials P_a(xi) P_b(eta): Q^k at index
 *     b*(k+1) + a, P^k ordered by total degree a+b and then by decreasing a
 *     ((0,0), (1,0), (0,1), (2,0), (1,1), (0,2), ...); 1D: a = 0..k.  j is
 *     absent (ny = 1) in 1D.  Both meshes' planes have nxs x nys cells: nx x ny,
 *     plus one column (row) where the low x (y) side is a reflective wall.  The
 *     dual mesh keeps its cell centred on that wall in the extra slot (i = nx,
 *     resp. j = ny); the primal mesh leaves the slot unused (it is neither read
 *     nor written; cdg_project_ic sets it to 0).  The dual cell centred on a
 *     high-side wall is its ordinary last cell.
 *   - All calls are asynchronous on the context's stream unless stated.
 *   - tau and tau_max live in device memory owned by the context, so that a
 *     sequence of cdg_step_async calls can be captured in a CUDA graph.
 *   - Scratch memory (two state-sized buffers, four with RK4, and reduction
 *     partials) is owned by the context and allocated in cdg_init_mesh.
 */
#ifndef OECDG_H
#define OECDG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CDG_OK = 0,
  CDG_EINVAL = 1,        /* invalid argument (null pointer, bad size, bad enum) */
  CDG_ENOMEM = 2,        /* device allocation failed */
  CDG_ECUDA = 3,         /* a CUDA runtime call failed */
  CDG_ENONPHYSICAL = 4,  /* a cell average with rho <= 0 or p <= 0 was met */
  CDG_ETIMEOUT = 5,      /* a bounded device wait gave up */
  CDG_EUNSUPPORTED = 6   /* the configuration is outside the CUDA path's scope */
} cdg_status;

enum { CDG_ADVECTION = 0, CDG_BURGERS = 1, CDG_EULER = 2 };
enum { CDG_BASIS_Q = 0, CDG_BASIS_P = 1 };
enum { CDG_PERIODIC = 0, CDG_TRANSMISSIVE = 1, CDG_REFLECTIVE = 2 };
enum { CDG_RK_EULER1 = 1, CDG_RK_SSP2 = 2, CDG_RK_SSP3 = 3, CDG_RK_RK4 = 4 };

/* Problem description (Section 2.1 meshes and spaces; Section 4 time stepping). */
typedef struct {
  int dim;       /* 1 or 2 */
  int nx, ny;    /* primal cells per direction (ny is ignored when dim = 1) */
  int k;         /* polynomial degree: 1..3 */
  int basis;     /* CDG_BASIS_Q or CDG_BASIS_P (1D: P^k = Q^k, either accepted) */
  int system;    /* CDG_ADVECTION, CDG_BURGERS or CDG_EULER */
  int bc[4];     /* boundary condition of each side: x-low, x-high, y-low, y-high
                    (1D: the first two).  CDG_PERIODIC (on both sides of a
                    direction or on neither), CDG_TRANSMISSIVE (outflow: the
                    ghost cell is a copy of the nearest cell), CDG_REFLECTIVE
                    (a wall, Euler only: the restriction of the mirror-extended
                    problem -- the state beyond the wall is the mirror image
                    with the normal momentum negated; sigma and avg are those
                    of the mirror-extended domain) */
  int oe;        /* 1: apply the OE step F_tau after every RK stage */
  int rk;        /* CDG_RK_EULER1, _SSP2, _SSP3 or _RK4 */
  double ax, bx, ay, by; /* domain [ax,bx] x [ay,by] */
  double gamma;          /* ratio of specific heats (Euler) */
  double adv_x, adv_y;   /* advection velocity */
  double cfl;            /* C_CFL of the time step, Section 4 */
} cdg_mesh_desc;

typedef struct cdg_ctx cdg_ctx;

/* Create a context for the mesh pair of Section 2.1 (primal + dual), bound to
 * `stream` (a cudaStream_t; NULL = the legacy default stream), on the current
 * device.  Allocates the geometry constants and the scratch buffers.
 * Contexts whose four sides are all periodic or all transmissive run the Q^2
 * configurations on the tiled kernels; any other combination (and every
 * reflective wall) runs on the degree-generic kernels.
 * Errors: CDG_EINVAL (null pointers, sizes < 2, bad enums, a periodic side
 * without its periodic partner, a reflective wall for a system other than
 * Euler), CDG_EUNSUPPORTED (k outside 1..3), CDG_ENOMEM, CDG_ECUDA.  On error
 * *out is NULL. */
cdg_status cdg_init_mesh(const cdg_mesh_desc* desc, void* stream, cdg_ctx** out);

/* Release a context (synchronises its stream first).  NULL is accepted. */
cdg_status cdg_free(cdg_ctx* ctx);

/* Static text describing the last error of `ctx` ("" if none; NULL ctx ok). */
const char* cdg_last_error(const cdg_ctx* ctx);

/* Number of FP64 elements of a state array (2 meshes x fields x modes x
 * nxs x nys cells, the padded layout above). */
cdg_status cdg_state_numel(const cdg_ctx* ctx, size_t* numel);

/* Sampling points of the projection-based initialisation (Section 3.3): on
 * every stored cell of both meshes (the padded layout; an unused primal slot
 * gets valid points whose values are ignored), (k+1) x (k+1) (1D: k + 1) Gauss
 * points on each of its 4 (1D: 2) sub-cells, layout [mesh][j][i][sy][sx][qy][qx]
 * of (x, y) pairs (1D: [mesh][i][sx][qx] of x).  The outer half of a
 * wall-centred dual cell lies beyond the wall: its points are folded back to
 * their mirror images inside, and cdg_project_ic negates the normal momentum
 * sampled there.  With d_xy == NULL only *npts is set; otherwise d_xy is a
 * device array of npts * dim doubles. */
cdg_status cdg_quad_points(cdg_ctx* ctx, double* d_xy, size_t* npts);

/* L^2 projection of sampled initial data onto both meshes (the projection-
 * based initialisation of Section 3.3) with the composite Gauss rule of
 * cdg_quad_points.  d_vals: device [npts][fields] conserved values at the
 * points; d_u: device state (output). */
cdg_status cdg_project_ic(cdg_ctx* ctx, const double* d_vals, double* d_u);

/* Semi-discrete right-hand side of the CDG method, Eq. (equcdg) (1D Eq.
 * (eq:1D_H), 2D Eq. (eq:2D_H)): d_L = M^{-1} H(u, .) on both meshes, with the
 * dissipation coefficient 1/tau_max.  d_L must not alias d_u. */
cdg_status cdg_rhs(cdg_ctx* ctx, const double* d_u, double tau_max, double* d_L);

/* Time step of Section 4 (2D: tau_max = C_CFL / (beta_x/h_x + beta_y/h_y);
 * 1D: C_CFL h / beta) from the maximum wave speed over the cell averages of
 * both meshes; tau = tau_max, clipped so that t + tau does not pass T_end
 * (T_end <= 0: no end time).  Stores (tau, tau_max) in the context's device
 * memory.  A non-physical cell average sets the context's status flag. */
cdg_status cdg_compute_dt(cdg_ctx* ctx, const double* d_u, double t, double T_end);

/* Set (tau, tau_max) directly (host values). */
cdg_status cdg_set_dt(cdg_ctx* ctx, double tau, double tau_max);

/* Read (tau, tau_max) back to the host; synchronises the stream. */
cdg_status cdg_get_dt(cdg_ctx* ctx, double* tau, double* tau_max);

/* One RK stage of Eq. (eq:RKCDG) without the OE step, with the context's tau
 * and tau_max, in the Shu-Osher form of the context's method:
 *   forward Euler   l = 0:        d_out = d_ul + tau L(d_ul)
 *   SSP-RK2/SSP-RK3 l >= 1:       d_out = c_l d_un + (1 - c_l)(d_ul + tau L(d_ul)),
 *                                 c = (0, 1/2) resp. (0, 3/4, 1/3)
 *   RK4             l = 0, 1, 2:  d_out = d_un + a_l tau L(d_ul), a = (1/2, 1/2, 1)
 *                                 (l = 0: d_un is d_ul and is not read)
 * RK4's last stage combines four states: use cdg_rk_combine for it (l = 3 is
 * CDG_EINVAL here).  d_out must not alias d_ul or d_un. */
cdg_status cdg_rk_stage(cdg_ctx* ctx, int l, const double* d_un, const double* d_ul, double* d_out);

/* A general Shu-Osher stage (Eq. (eq:RKCDG) with any explicit RK method):
 *     d_out = sum_{m < n} coef[m] d_terms[m] + ct tau L(d_ul),
 * n in 1..4, d_terms a HOST array of n device state pointers, coef a host
 * array of n doubles.  Classical RK4's last stage is n = 4 with terms
 * (u^n, u^(1), u^(2), u^(3)), coef (-1/3, 1/3, 2/3, 1/3), ct = 1/6 and
 * d_ul = u^(3).  On the tiled 2D Q^2 path only the two-state form (n = 2,
 * d_terms[1] == d_ul, coef[1] == ct, or n = 1, d_terms[0] == d_ul,
 * coef[0] == ct == 1) runs; other forms return CDG_EUNSUPPORTED there.  d_out must not alias d_ul or
 * any term. */
cdg_status cdg_rk_combine(cdg_ctx* ctx, const double* d_ul, int n, const double* const* d_terms, const double* coef,
                          double ct, double* d_out);

/* The OE step u_sigma = F_tau u_h (Eq. (OEstep2D), solved exactly): sigma_K
 * and avg per mesh and field (sigma = the max over every cell's Gauss points
 * of |u - avg|, taken as 0 when it is at most 2^-40 of the field's largest
 * |u| there: a field constant up to rounding, whose delta is then 0 as for an
 * exactly constant one), the damping coefficients delta_K^m (m = 0..k)
 * from the traces of u^C - u^D on the half-faces of every cell, the wave speed
 * beta_{e,K} at the cell average, and the exponential decay of every mode of
 * total degree >= 1.  tau from the context.  d_usig must not alias d_uh.
 * A non-physical cell average sets the context's status flag. */
cdg_status cdg_oe_damp(cdg_ctx* ctx, const double* d_uh, double* d_usig);

/* The damping coefficients alone, for inspection: d_delta [2][nys][nxs][k+1]
 * (the padded layout), d_sigma [2][fields] (either may be NULL). */
cdg_status cdg_oe_coefficients(cdg_ctx* ctx, const double* d_uh, double* d_delta, double* d_sigma);

/* nsteps full time steps of Eq. (eq:RKCDG) in place on d_u, starting at time t
 * (tau recomputed at the start of every step, clipped at T_end > 0; steps
 * after T_end is reached are skipped on the device with tau = 0).  Uses the
 * context's scratch.  Synchronises at the end and returns CDG_ENONPHYSICAL if
 * the status flag was set. */
cdg_status cdg_step(cdg_ctx* ctx, double* d_u, double t, double T_end, int nsteps);

/* As cdg_step, but without the final synchronisation and status check, so
 * that it can be captured in a CUDA graph; the time advanced so far is kept on
 * the device (cdg_get_time). */
cdg_status cdg_step_async(cdg_ctx* ctx, double* d_u, double t, double T_end, int nsteps);

/* As cdg_step_async, for many small steps: the kernels of one step (Eq.
 * (eq:RKCDG), the same launches as cdg_step_async) are captured once into a
 * CUDA graph on the context's stream, and the graph is replayed nsteps times,
 * one graph launch per step instead of one launch per kernel.  tau, tau_max
 * and t stay on the device, so replays need no host work; steps after T_end
 * is reached are skipped on the device as in cdg_step.  The graph is bound to
 * d_u and T_end: a call with another d_u or T_end captures a new one (after a
 * stream synchronisation).  Needs a context created with its own stream
 * (CDG_EINVAL with the legacy default stream).  Kernel timing
 * (cdg_profile_begin) does not see replayed steps.  Asynchronous; check the
 * status with cdg_check_status. */
cdg_status cdg_step_graph(cdg_ctx* ctx, double* d_u, double t, double T_end, int nsteps);

/* As cdg_step_async, for 1D meshes (whose steps are far too small to fill the
 * GPU, so that a step is bound by the latency of its launches): all nsteps
 * steps of Eq. (eq:RKCDG) -- the wave speed and tau, and every stage's CDG
 * right-hand side, RK combination, sigma and OE step -- run in ONE cooperative
 * launch whose blocks meet at grid-wide barriers between those phases.  Same
 * per-cell code and fixed-order reductions as cdg_step: the results are equal
 * bit for bit.  Every barrier wait is bounded (cdg_set_wait; 5 s by default);
 * a wait that runs out makes every block leave the kernel and sets the status
 * that cdg_check_status reports as CDG_ETIMEOUT (d_u is then partly advanced).
 * The first call allocates a small scratch (one double per block of the grid
 * and the barrier counter) in the context.  Asynchronous; not for use inside a
 * stream capture (the first call allocates).  Errors: CDG_EINVAL,
 * CDG_EUNSUPPORTED (2D contexts), CDG_ENOMEM, CDG_ECUDA. */
cdg_status cdg_step_persistent(cdg_ctx* ctx, double* d_u, double t, double T_end, int nsteps);

/* Bounded wait of the grid barriers of cdg_step_persistent: a block that has
 * waited limit_s seconds (0 < limit_s <= 3600) at one barrier gives up (status
 * CDG_ETIMEOUT).  withheld >= 0 is a test hook: every barrier then waits for
 * that many more arrivals than there are blocks, which never come, so that a
 * test can make the wait run out on purpose (0 for normal use). */
cdg_status cdg_set_wait(cdg_ctx* ctx, double limit_s, int withheld);

/* Device time after the last cdg_step / cdg_step_async; synchronises. */
cdg_status cdg_get_time(cdg_ctx* ctx, double* t);

/* Adjoint of one time step (not in the paper; the forward step is Eq.
 * (eq:RKCDG) with SSP-RK3 and the OE step after every stage):
 *     d_lam = (d u^{n+1} / d u^n)^T d_lam_next,
 * with tau = tau_max computed from u^n as in cdg_step (no end time).  The
 * derivative follows every path the forward step takes: the CDG right-hand
 * side (Euler flux Jacobians at the quadrature points, the dissipation term and
 * 1/tau_max), the RK combination, the OE step (the exponential scaling, the
 * damping coefficients through the half-face traces of u^C - u^D, the
 * cell-average wave speeds beta, sigma through its extremal Gauss point and the
 * domain average, and tau), and tau through the cell with the largest wave
 * speed.  At non-differentiable points it takes sign(0) = 0, zero for the
 * gradient of sqrt at a zero sum, and the lowest index for ties of max / argmax.
 * The three stages are recomputed from d_un.  d_un, d_lam_next: device states
 * (inputs); d_lam: device state (output, must not alias d_un; may alias
 * d_lam_next); d_gtau: NULL or 2 device doubles receiving the adjoints of tau
 * and tau_max of the step.  2D periodic Q^2 advection or Euler with SSP-RK3
 * only, i.e. the tiled path (CDG_EUNSUPPORTED otherwise); with oe = 0 the
 * OE paths are left out as in the forward step.  The first call allocates the
 * adjoint scratch (12 state-sized buffers) in the context.  Asynchronous. */
cdg_status cdg_step_adjoint(cdg_ctx* ctx, const double* d_un, const double* d_lam_next, double* d_lam,
                            double* d_gtau);

/* Recorded variant for gradients over many steps: cdg_step_record advances
 * d_u by one step (as cdg_step_async, no end time) and stores in d_rec what
 * the adjoint of that step needs -- u^n, the three stages' u_h and the first
 * two stages' u_sigma, (tau, tau_max), and per cell and stage the OE step's
 * damping coefficients with the field that gives each of them and that field's
 * face sums: cdg_record_numel() doubles (6 states + 2 + 3 x 24 x cells).
 * cdg_step_adjoint_recorded then runs the backward pass without recomputing
 * the stages: d_lam = (du^{n+1}/du^n)^T d_lam_next, as cdg_step_adjoint.  Same
 * scope and scratch as cdg_step_adjoint. */
cdg_status cdg_record_numel(const cdg_ctx* ctx, size_t* numel);
cdg_status cdg_step_record(cdg_ctx* ctx, double* d_u, double* d_rec);
cdg_status cdg_step_adjoint_recorded(cdg_ctx* ctx, const double* d_rec, const double* d_lam_next, double* d_lam,
                                     double* d_gtau);

/* Read and clear the device status flag (synchronises): CDG_OK,
 * CDG_ETIMEOUT (a grid barrier of cdg_step_persistent ran out of time) or
 * CDG_ENONPHYSICAL. */
cdg_status cdg_check_status(cdg_ctx* ctx);

/* Optional per-kernel timing: between cdg_profile_begin and cdg_profile_end,
 * every stage kernel (CDG RHS + RK combine) and every OE kernel launched by the
 * context is bracketed by CUDA events on the context's stream (at most
 * max_launches of each).  cdg_profile_end synchronises and returns the summed
 * event durations (ms) and the launch counts of the two kernel classes (any
 * pointer may be NULL).  Not for use inside a CUDA graph capture. */
cdg_status cdg_profile_begin(cdg_ctx* ctx, int max_launches);
cdg_status cdg_profile_end(cdg_ctx* ctx, double* ms_stage, long long* n_stage, double* ms_oe, long long* n_oe);

/* The OE step of cdg_oe_damp for callers that cannot allocate device memory.
 *
 * Some callers cannot call cudaMalloc: code embedded in a host application
 * whose memory manager owns the whole device heap (a direct allocation would
 * be refused or fragment it), or a latency-critical path that must not
 * allocate, nor wait on an allocation, once it is running.  This entry point
 * needs no context and allocates nothing.  Its scratch (sigma partials, sigma
 * and avg, tau and a status word) is a 1 MiB array compiled into the library's
 * device image, so every GPU that loads the library holds it until the process
 * exits.  The paper has no counterpart: this is an interface for such callers,
 * not a step of the method.
 *
 * desc:   mesh description, same rules as cdg_init_mesh within the scope below.
 * d_uh:   device state to damp (input, caller-owned); d_usig: device state
 *         (output, caller-owned, must not alias d_uh); both cdg_state_numel()
 *         doubles in the layout above.
 * tau:    damping time (>= 0), as the context's tau in cdg_oe_damp.
 * stream: a cudaStream_t (NULL = the legacy default stream); asynchronous.
 * Limit:  the partials need 2 * ceil(cells per mesh / 256) * fields * 3
 *         doubles of the 131,008 available: at most 1,397,248 cells per mesh
 *         with 4 fields (2D Euler; 1024 x 1024 fits), 1,863,168 with 3 (1D
 *         Euler), 5,589,504 with 1 (advection).  Larger meshes return
 *         CDG_EINVAL without launching anything.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  The address is kept for the life of the process, so do
 * not use this entry point on a device after cudaDeviceReset (or any other
 * teardown of its primary context) in the same process.  Every call shares the one array and overwrites or clears
 * what it uses, so calls that overlap on the GPU (two streams, or two host
 * threads) race: the caller must order them.  Non-physical cell averages are
 * not reported by this entry point (their wave speed is taken as 0).
 * Errors: CDG_EINVAL (bad pointers or sizes, aliasing, tau < 0, mesh beyond the
 * limit), CDG_EUNSUPPORTED (k != 2, basis P in 2D, or Burgers: this entry
 * point covers 2D Q^2 and 1D P^2 advection and Euler only), CDG_ECUDA. */
cdg_status cdg_oe_damp_noalloc(const cdg_mesh_desc* desc, const double* d_uh, double tau, double* d_usig,
                               void* stream);

/* Number of kernels launched by the context so far (host-side counter). */
cdg_status cdg_launch_count(const cdg_ctx* ctx, long long* count);

/* The FP64 reciprocal (op CDG_MATH_RCP) and square root (op CDG_MATH_SQRT)
 * that the kernels use in their hot loops (1/rho of the Euler flux, the
 * norms in the damping coefficients of Eq. (OEstep2D)), applied elementwise:
 * d_y[i] = op(d_x[i]), i < n, so that they can be checked against correctly
 * rounded results.  Not a step of the method.  The reciprocal is within 1 ulp
 * for 2^-1022 <= |x| <= 2^1022, either sign (point densities can be negative
 * in discontinuous runs), and odd: rcp(-x) = -rcp(x); the square root within
 * 1 ulp for 2^-1022 <= x <= 2^1022.  Outside those ranges (zero, subnormal,
 * infinite, NaN, or a negative square-root argument) the results are not
 * specified (the reciprocal gives NaN for zero and subnormal |x|).  d_x, d_y:
 * device arrays of n
 * doubles (caller-owned; they may alias).  stream: a cudaStream_t (NULL =
 * the legacy default stream); asynchronous.  n = 0 launches nothing.
 * Errors: CDG_EINVAL (null pointers with n > 0, bad op), CDG_ECUDA. */
enum { CDG_MATH_RCP = 0, CDG_MATH_SQRT = 1 };
cdg_status cdg_math_eval(int op, const double* d_x, size_t n, double* d_y, void* stream);

/* ------------------------------------------------------------- batches ---
 * Many independent 2D Euler Q^2 problems of uneven mesh sizes advanced together.
 * Not in the paper: each instance is exactly the single-mesh scheme above
 * (Eq. (eq:RKCDG) with SSP-RK3 and the OE step), with its own sigma, wave speed,
 * tau and time.  Two ways to run the steps, with bitwise-equal results:
 *   - per-phase launches: every phase of a step is one launch over the tiles
 *     of all instances (11 launches per step whatever the number of
 *     instances), optionally captured in a CUDA graph;
 *   - persistent: ONE cooperative launch runs all nsteps steps; its blocks
 *     loop over the same tiles phase by phase and meet at grid-wide barriers.
 *     Every barrier wait is bounded (cdg_batch_set_wait; 5 s by default): a
 *     wait that runs out sets the batch's status to CDG_ETIMEOUT and every
 *     block leaves the kernel, so nothing hangs.  The launch can also be
 *     captured in a CUDA graph. */
typedef struct cdg_batch cdg_batch;

/* Create a batch of n instances (descs[q]: dim 2, k 2, basis Q, system Euler,
 * rk SSP-RK3, oe 1; the same boundary condition for all), bound to `stream`
 * (NULL: the batch creates and owns a non-blocking stream; graph capture needs
 * a stream other than the legacy default).  Allocates per instance two scratch
 * states and the reduction slots.  Errors: CDG_EINVAL, CDG_EUNSUPPORTED,
 * CDG_ENOMEM, CDG_ECUDA. */
cdg_status cdg_init_batch(const cdg_mesh_desc* descs, int n, void* stream, cdg_batch** out);

/* Release a batch (synchronises its stream).  NULL is accepted. */
cdg_status cdg_batch_free(cdg_batch* batch);

/* Static text describing the batch's last error. */
const char* cdg_batch_last_error(const cdg_batch* batch);

/* nsteps SSP-RK3 steps of every instance, in place on the caller's device
 * states d_us[0..n-1] (a host array of n device pointers, each with the
 * single-mesh layout of its instance).  The instance table is re-uploaded
 * (synchronously) only when the pointers change.  flags:
 *   0                                         per-phase launches;
 *   CDG_BATCH_GRAPH                           per-phase launches of nsteps steps
 *                                             captured once in a CUDA graph;
 *   CDG_BATCH_PERSISTENT                      one persistent cooperative launch
 *                                             for all nsteps steps;
 *   CDG_BATCH_PERSISTENT | CDG_BATCH_GRAPH    that launch captured in a graph.
 * A graph is re-captured when nsteps, flags, the pointers or the batch's
 * settings change.  Asynchronous; check the outcome (CDG_ENONPHYSICAL,
 * CDG_ETIMEOUT) with cdg_batch_check_status.  Errors: CDG_EINVAL (bad
 * pointers, nsteps < 0, flags outside 0..3), CDG_ECUDA (a launch failed, for
 * example a persistent grid that does not fit the device). */
enum { CDG_BATCH_GRAPH = 1, CDG_BATCH_PERSISTENT = 2 };
cdg_status cdg_batch_step(cdg_batch* batch, double* const* d_us, int nsteps, int flags);

/* Bounded wait of the persistent kernel's grid barriers: a block that has
 * waited limit_s seconds (0 < limit_s <= 3600) at one barrier gives up and the
 * batch's status becomes CDG_ETIMEOUT.  withheld >= 0 is a test hook: every
 * barrier then waits for that many more arrivals than there are blocks, which
 * never come, so that a test can make the wait run out on purpose (0 for
 * normal use).  Synchronises the batch's stream. */
cdg_status cdg_batch_set_wait(cdg_batch* batch, double limit_s, int withheld);

/* Persistent grid: blocks_per_sm blocks on every SM (0 = as many as fit the
 * register and shared-memory budget of the kernel for the current tile
 * height; more than fit is clamped).  Synchronises the batch's stream. */
cdg_status cdg_batch_set_grid(cdg_batch* batch, int blocks_per_sm);

/* The persistent grid in use: blocks per SM and the total block count. */
cdg_status cdg_batch_grid(const cdg_batch* batch, int* blocks_per_sm, int* grid);

/* Read and clear the batch's status flag (synchronises): CDG_OK,
 * CDG_ETIMEOUT (a persistent grid barrier ran out of time; the instances' states
 * are then partly advanced and must be restored by the caller) or
 * CDG_ENONPHYSICAL. */
cdg_status cdg_batch_check_status(cdg_batch* batch);

/* Time of every instance (t[0..n-1], host); synchronises. */
cdg_status cdg_batch_get_time(cdg_batch* batch, double* t);

/* Kernels launched by the batch so far (graph launches count their kernels). */
cdg_status cdg_batch_launch_count(const cdg_batch* batch, long long* count);

/* Set the tile height (2, 4 or 8 rows of 32 cells per block); synchronises. */
cdg_status cdg_batch_set_rows(cdg_batch* batch, int rows);

/* Tile height (rows of 32 cells per block: 2, 4 or 8) currently in use. */
cdg_status cdg_batch_rows(const cdg_batch* batch, int* rows);

/* Pick the tile height (2, 4 or 8 rows of 32 cells per block) and the
 * persistent grid (blocks per SM, 1 up to what fits for that height) for this
 * batch: look them up in the JSON cache file `cache_path` (keyed by a
 * signature of the mesh sizes; NULL: no cache; value rows * 100 + blocks per
 * SM), or time the persistent kernel on one first stage of every instance for
 * each candidate (it reads the states d_us and writes only scratch) and store
 * the fastest.  Resets the instances' time to 0.  *rows_out (nullable)
 * receives the tile height; cdg_batch_grid reports the grid.  Errors as
 * cdg_batch_step, and CDG_ETIMEOUT if a timed run's barrier ran out. */
cdg_status cdg_batch_autotune(cdg_batch* batch, double* const* d_us, const char* cache_path, int* rows_out);

#ifdef __cplusplus
}
#endif

#endif /* OECDG_H */
