/*
 * claw.h -- C ABI of the GB300 wave-propagation library.
 *
 * The library advances hyperbolic conservation laws with the dimensionally
 * split, second-order finite-volume wave-propagation step of CUDACLAW
 * (arXiv 1805.08846, Sec. 3, Eq. LW-update):
 *   x sweep  Q^n -> Q*,  y sweep  Q* -> Q** (, z sweep -> Q^{n+1}),
 * each sweep solving a Riemann problem at every interface (waves W^p,
 * speeds s^p), forming the fluctuations A-dQ / A+dQ, limiting the waves
 * (minmod or MC) into the correction flux F~ and applying the conservative
 * update.  The step size follows the CFL condition (Eq. CFL-condition):
 * the largest |s^p| / dx_d of a step decides whether the step is kept
 * (Courant number <= cfl_max) or redone, and sets the next step to
 * cfl_desired / max_d(max|s^p| / dx_d)  (Sec. 4.1, time-step adjustment).
 *
 * PDE systems (Sec. 3, Eq. acoustics and Eq. SW):
 *   CLAW_ACOUSTICS      p_t + K div u = 0, rho u_t + grad p = 0, constant
 *                       rho, K; 2D (m = 3: p,u,v) or 3D (m = 4: p,u,v,w);
 *                       mwaves = 2.
 *   CLAW_ACOUSTICS_VAR  the same with per-cell rho, K (claw_set_aux).
 *   CLAW_SHALLOW_WATER  2D shallow water, m = 3 (h, hu, hv), mwaves = 3,
 *                       Roe solver with the Harten-Hyman entropy fix.
 *   CLAW_SHALLOW_WATER_BATHY  2D shallow water over a bottom elevation B
 *                       (claw_set_bathymetry; flat B = 0 until set): the
 *                       source -g h grad B enters the Riemann problem as
 *                       f-waves of f(Q_r) - f(Q_l) - (0, -g h_bar dB, 0) on
 *                       the Roe eigenvectors (Sec. 3's Clawpack base adds
 *                       source terms to the hyperbolic part), so a lake at
 *                       rest stays exactly at rest; no entropy fix, h > 0.
 *   CLAW_SHALLOW_WATER_DRY  the same over B with wetting and drying: a cell
 *                       with h <= claw_params.dry_tol is dry (h = 0 allowed).
 *                       Each interface reconstructs the depths hydrostatically
 *                       against max(B_l, B_r) and solves the flat problem by
 *                       HLLE (Einfeldt's speeds, dry-bed front speed u -/+ 2c);
 *                       no second-order correction at the shoreline.  Mass is
 *                       conserved, a lake at rest (also around an emerged
 *                       island) stays exactly at rest, h stays >= 0.  The paper
 *                       is silent on dry states: this is the library's reading
 *                       of Sec. 3's source terms for them.
 *
 * Conventions for every call:
 *   - State arrays crossing the boundary are FP64, structure of arrays,
 *     q[f][z][y][x] with x fastest, interior cells only (no ghosts),
 *     m * nx * ny * nz doubles.  on_device = 0: a host pointer (pinned or
 *     pageable); on_device = 1: a CUDA device pointer of the current device.
 *     The caller keeps ownership; no pointer is retained after a call returns.
 *   - The solver owns all of its device memory (state versions, material
 *     arrays, control block) and a CUDA stream (the caller's, or its own
 *     non-blocking one when the caller passes NULL).  Calls are asynchronous
 *     on that stream except where a call says it synchronises.
 *   - Every call returns a claw_status.  Faults found on the device (a
 *     non-finite state, h <= 0, repeated CFL rejections, a timed-out wait)
 *     are latched and returned by the next synchronising call.  No call
 *     aborts the process and none waits without bound.
 *   - claw_last_error() returns a thread-local message for the last failure.
 *   - Precision: claw_params.precision = 64 keeps state and arithmetic in
 *     FP64; 32 keeps the state and the Riemann / limiter / update arithmetic
 *     in FP32, with the time step, simulated time and conservation sums in
 *     FP64 in both cases.
 */
#ifndef CLAW_H
#define CLAW_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct claw_solver claw_solver;   /* opaque; owns all device memory */

typedef enum {
    CLAW_OK = 0,
    CLAW_EINVAL = 1,     /* bad argument; nothing was changed */
    CLAW_ENOMEM = 2,     /* device or pinned host allocation failed */
    CLAW_ECUDA = 3,      /* a CUDA runtime call failed (message in claw_last_error) */
    CLAW_ECFL = 4,       /* more than max_retries consecutive CFL rejections */
    CLAW_ENONPHYS = 5,   /* NaN / Inf in the state, or h <= 0 (shallow water; h < 0 with
                            wetting and drying) */
    CLAW_ETIMEOUT = 6,   /* a bounded device-side wait gave up */
    CLAW_EBOUNDS = 7     /* a size or index outside the supported range */
} claw_status;

typedef enum { CLAW_BC_PERIODIC = 0, CLAW_BC_EXTRAP = 1, CLAW_BC_WALL = 2 } claw_bc;
typedef enum {
    CLAW_ACOUSTICS = 0,
    CLAW_ACOUSTICS_VAR = 1,
    CLAW_SHALLOW_WATER = 2,
    CLAW_SHALLOW_WATER_BATHY = 3,
    CLAW_SHALLOW_WATER_DRY = 4
} claw_system;
/* Second-order correction of Sec. 3 Eq. LW-update: NONE applies it
 * unlimited (Lax-Wendroff), MINMOD / MC limit each wave against its upwind
 * neighbour; FIRST_ORDER drops it (Godunov's first-order upwind method: the
 * Riemann solution and fluctuation update alone, the part of the sweep Sec.
 * 7.1 measures as its "Riemann solver" kernels). */
typedef enum {
    CLAW_LIM_NONE = 0,
    CLAW_LIM_MINMOD = 1,
    CLAW_LIM_MC = 2,
    CLAW_LIM_FIRST_ORDER = 3
} claw_limiter;

/* Grid of one problem: ndim = 2 or 3; n[d] interior cells (>= 2 in each
 * used direction; n[2] is ignored in 2D); dx[d] > 0 cell widths. */
typedef struct { int ndim; int n[3]; double dx[3]; } claw_grid;

/* Sweep order of a step.  GODUNOV: x(dt) y(dt) [z(dt)], Sec. 3 Eq.
 * LW-update as the paper runs it.  STRANG: x(dt/2) y(dt) x(dt/2) in 2D,
 * x(dt/2) y(dt/2) z(dt) y(dt/2) x(dt/2) in 3D, the second-order splitting
 * of the same Clawpack base.  UNSPLIT (2D acoustics and shallow water, not
 * CLAW_SHALLOW_WATER_BATHY or _DRY; CLAW_EINVAL otherwise): no splitting -- every
 * Riemann problem of the step is solved from Q^n and each cell is updated
 * once from its x and y fluctuations and corrections, with transverse
 * solvers carrying the fluctuations (modified by the corrections) across
 * the neighbouring transverse interfaces (the unsplit form of Eq.
 * LW-update in the same Clawpack base).  In every case a step's Courant
 * number is dt * max_d(m_d / dx_d), m_d the largest speed along d in the
 * step. */
typedef enum { CLAW_SPLIT_GODUNOV = 0, CLAW_SPLIT_STRANG = 1, CLAW_SPLIT_UNSPLIT = 2 } claw_splitting;

/* rho, K: constant acoustics coefficients (also the initial per-cell values
 * of CLAW_ACOUSTICS_VAR); g: gravity; cfl_desired: Courant number the next
 * step aims at; cfl_max: a step above it is redone; dt_max: cap on dt;
 * precision: 32 or 64; max_retries: consecutive rejections before
 * CLAW_ECFL (<= 0 selects 8); splitting: a claw_splitting; dry_tol
 * (CLAW_SHALLOW_WATER_DRY, >= 0): a cell with h <= dry_tol is dry (in FP32
 * at least every depth below the smallest normal float, 1.2e-38).  Keep it
 * well above rounding (e.g. 1e-3 of the depth scale): with dry_tol near 0 a
 * draining film can round below zero, which stops the run with
 * CLAW_ENONPHYS. */
typedef struct {
    double rho, K, g;
    double cfl_desired, cfl_max, dt_max;
    int precision;
    int max_retries;
    int splitting;
    double dry_tol;
} claw_params;

/* Ghost cells, two per side, filled inside each sweep from the state it is
 * about to read (Sec. 4.1 boundary stage): bc[2d] is the low side of
 * direction d, bc[2d+1] the high side.  PERIODIC wraps; EXTRAP copies the
 * edge cell; WALL mirrors the two edge cells and negates the normal
 * velocity / momentum.  Material coefficients follow the same index rule. */

/* ---------------------------------------------------------------- single grid */

/* Create a solver for one grid of cell averages Q_{i,j} of Sec. 3 (the
 * finite-volume unknowns of Eq. conslaw) and the pipeline of Sec. 4.1
 * around it.  (m, mwaves) must match the system:
 * (3,2) 2D acoustics, (4,2) 3D acoustics, (3,3) shallow water (2D only);
 * otherwise CLAW_EINVAL.  cuda_stream: a cudaStream_t (e.g. a torch stream)
 * or NULL.  The state starts at zero (h = 1 for shallow water), t = 0. */
claw_status claw_create(const claw_grid* grid, int m, int mwaves, claw_system system,
                        claw_limiter limiter, const claw_bc bc[6], const claw_params* params,
                        void* cuda_stream, claw_solver** out);

/* Release every resource of the solver created for Sec. 4.1's pipeline
 * (synchronises its stream).  NULL is a no-op. */
void claw_destroy(claw_solver* s);

/* Copy a new state of cell averages in (Sec. 3; FP64 SoA, see conventions:
 * the double-precision interface of Sec. 6 in front of a solver that may
 * compute in single precision) and set the next step from a speeds-only
 * Riemann pass over it, dt = cfl_desired / max_d(m_d / dx_d) (Eq.
 * CFL-condition). */
claw_status claw_set_q(claw_solver* s, const double* q_soa, int on_device);

/* Copy the current cell averages out (Sec. 3; FP64 SoA, the solution read
 * back at any step as in Sec. 6).  Synchronises; returns any latched device
 * fault. */
claw_status claw_get_q(claw_solver* s, double* q_soa, int on_device);

/* Per-cell rho and K of Eq. acoustics with coefficients (Sec. 3; nx*ny*nz
 * doubles each, x fastest) for CLAW_ACOUSTICS_VAR; impedance Z = rho c and c = sqrt(K / rho) are formed
 * once per cell, in FP64.  CLAW_EINVAL for other systems or rho, K <= 0 is
 * not checked (the caller guarantees positivity). */
claw_status claw_set_aux(claw_solver* s, const double* rho, const double* K, int on_device);

/* Bottom elevation B per cell of the shallow-water source term (Sec. 3:
 * source terms added to Eq. SW; nx*ny doubles, x fastest) for
 * CLAW_SHALLOW_WATER_BATHY and CLAW_SHALLOW_WATER_DRY, stored in the state's
 * precision.  The bathymetry system's wave speeds do not depend on B, so dt
 * is unchanged; with wetting and drying they do (the reconstruction), and
 * the next step is set again from a speeds-only pass.  CLAW_EINVAL for other
 * systems.  Synchronises. */
claw_status claw_set_bathymetry(claw_solver* s, const double* B, int on_device);

/* One accepted step of Eq. LW-update.  dt > 0: exactly that step, always
 * kept (no CFL control); dt <= 0: the CFL rule of Eq. CFL-condition and
 * Sec. 4.1 (revert and redo on a violation).  *cfl_out (may be
 * NULL) receives the Courant number of the kept step.  Synchronises. */
claw_status claw_step(claw_solver* s, double dt, double* cfl_out);

/* Advance to t_final (>= current t, else CLAW_EINVAL) under the CFL rule
 * (Eq. CFL-condition, Sec. 4.1 time-step adjustment; Sec. 6 evolves a
 * problem this way);
 * the last step is shortened to land on t_final exactly.  cfl_target > 0
 * replaces cfl_desired.  *nsteps_out (may be NULL) gets the accepted steps.
 * Runs as CUDA graphs of several steps with the step control on the device.
 * Synchronises. */
claw_status claw_advance(claw_solver* s, double t_final, double cfl_target, int* nsteps_out);

/* Take nsteps accepted steps of Eq. LW-update under the CFL rule (Eq.
 * CFL-condition; rejected attempts are redone, Sec. 4.1, and not counted),
 * as CUDA graphs.  Synchronises. */
claw_status claw_run_steps(claw_solver* s, int nsteps);

/* max_d (max|s^p| / dx_d) of the current state, in FP64: the fastest wave
 * speed of Eq. CFL-condition, from the speed reduction of Sec. 4.1.
 * Synchronises. */
claw_status claw_max_speed(claw_solver* s, double* smax_over_dx);

/* Simulated time, next step (Eq. CFL-condition, Sec. 4.1 time-step
 * adjustment), accepted steps.  Synchronises. */
claw_status claw_get_time(claw_solver* s, double* t, double* dt, long* nsteps);

/* Restore the clock (checkpoint / resume).  dt <= 0 recomputes the next
 * step from the current state by Eq. CFL-condition (Sec. 4.1). */
claw_status claw_set_time(claw_solver* s, double t, double dt, long nsteps);

/* Sum of each field over the interior cells (m doubles), accumulated in
 * FP64 in a fixed order (deterministic): the totals the conservation form of
 * Sec. 3 (Eq. conslaw, Eq. LW-update in flux-difference form) keeps
 * constant up to boundary fluxes.  Synchronises. */
claw_status claw_conservation_sums(claw_solver* s, double* sums);

/* Attempts rejected and redone so far (Sec. 4.1: a step that violates Eq.
 * CFL-condition is reverted).  Synchronises. */
claw_status claw_get_rejections(claw_solver* s, long* nrej);

/* nsteps steps of exactly dt > 0, all kept (no CFL decision), replayed as
 * CUDA graphs like claw_run_steps; *cfl_peak (may be NULL) receives the
 * largest Courant number dt * max_d(m_d / dx_d) among them, so a caller that
 * decides the step size itself -- e.g. over several solvers holding pieces
 * of one grid (Sec. 8: independent subproblems advanced for several steps)
 * -- can check the CFL condition (Eq. CFL-condition) afterwards.  For an
 * ensemble, the largest over the instances.  Synchronises. */
claw_status claw_run_fixed_steps(claw_solver* s, int nsteps, double dt, double* cfl_peak);

/* Rows [y0, y0 + nrows) of every field of a single 2D grid (Sec. 8: the
 * independent subproblems of a multi-GPU run exchange these), FP64,
 * structure of arrays (m, nrows, nx), x fastest: copied out of (get) or
 * into (set) the current state.  The pieces of a grid split along y
 * exchange their boundary rows this way.  on_device as for claw_set_q.
 * claw_set_rows leaves the next step size as it is (claw_max_speed gives the
 * speeds of the new state); it is asynchronous for a device buffer, which
 * must stay valid until the solver's stream reaches the copy.  claw_get_rows
 * synchronises.  CLAW_EINVAL for an ensemble or a 3D grid, CLAW_EBOUNDS for
 * rows outside [0, ny). */
claw_status claw_get_rows(claw_solver* s, int y0, int nrows, double* out, int on_device);
claw_status claw_set_rows(claw_solver* s, int y0, int nrows, const double* rows, int on_device);

/* Keep a copy of the current state (every field's kept version, in the
 * state's precision, in device memory the solver allocates on the first call:
 * one state version) and of the clock and step control; claw_rollback
 * returns to it, bitwise -- state, t, next dt, step counts.  A caller that
 * takes a period of fixed steps and may have to redo it (the CFL condition
 * checked afterwards, Eq. CFL-condition) keeps the period's start this way
 * without a round trip through FP64.  claw_rollback without a checkpoint:
 * CLAW_EINVAL.  Both synchronise. */
claw_status claw_checkpoint(claw_solver* s);
claw_status claw_rollback(claw_solver* s);

/* Thread-local text of the last failure ("" if none).  Error reporting of
 * this library; the paper has no counterpart. */
const char* claw_last_error(void);

/* ---------------------------------------------------------------- ensembles */

/* B >= 1 independent problems of one system and limiter, each with its own
 * grid (all of the same ndim), time, step size and CFL control (Eq.
 * CFL-condition per instance), advanced together: one launch per sweep
 * covers the tiles of every instance, the way Sec. 5.1's independent blocks
 * each advance their own subdomain.  m and mwaves follow from the system;
 * bc[6] (per face, as for claw_create) applies to every instance. */
claw_status claw_ensemble_create(int B, const claw_grid* grids, claw_system system,
                                 claw_limiter limiter, const claw_bc bc[6],
                                 const claw_params* params, void* cuda_stream,
                                 claw_solver** out);
/* Instance i's cell averages in and out (Sec. 3; as claw_set_q / claw_get_q,
 * i in [0, B), else CLAW_EINVAL), its material coefficients (Eq. acoustics
 * with coefficients, as claw_set_aux) and its bottom elevation (Sec. 3
 * source terms, as claw_set_bathymetry). */
claw_status claw_ensemble_set_q(claw_solver* s, int i, const double* q, int on_device);
claw_status claw_ensemble_get_q(claw_solver* s, int i, double* q, int on_device);
claw_status claw_ensemble_set_aux(claw_solver* s, int i, const double* rho, const double* K,
                                  int on_device);
claw_status claw_ensemble_set_bathymetry(claw_solver* s, int i, const double* B, int on_device);
/* nsteps accepted steps of Eq. LW-update for every instance, each under its
 * own CFL rule (Eq. CFL-condition, Sec. 4.1).  Synchronises. */
claw_status claw_ensemble_run_steps(claw_solver* s, int nsteps);
/* Instance i's clock as claw_get_time (Sec. 4.1 time-step adjustment);
 * synchronises.  claw_ensemble_size: B (0 for NULL), the number of
 * independent problems of Sec. 5.1's kind this solver advances. */
claw_status claw_ensemble_get_time(claw_solver* s, int i, double* t, double* dt, long* nsteps);
int         claw_ensemble_size(const claw_solver* s);

/* ---------------------------------------------------------------- no allocation */

/* The CFL speed pass of claw_max_speed over a caller-owned state, without
 * creating a solver and without allocating anything.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * (cudaMalloc, cudaFree or any allocating library routine) -- for example a
 * host framework that owns every byte of device memory through its own
 * pool, or a latency-critical loop where an allocation could synchronise
 * the device -- but already hold the state on the GPU.
 *
 *   q        FP64 device array, SoA q[f][z][y][x], interior cells, m fields
 *            (m = 3 for 2D acoustics and shallow water, 4 for 3D acoustics)
 *   rho, K   FP64 device arrays of nx*ny*nz cells for CLAW_ACOUSTICS_VAR,
 *            else ignored (may be NULL); params->rho, K, g give the constants
 *   out      device pointer to one double: max_d (max|s^p| / dx_d), computed
 *            in FP64 like claw_max_speed of a precision-64 solver; NaN if a
 *            speed is not finite
 *   cuda_stream  stream both kernels run on (NULL = legacy default stream)
 *
 * Scratch: a fixed 384 KiB array in the library's device memory (one
 * partial maximum per 128 lines per direction) that every GPU loading the
 * library holds until the process exits.  Grids with more than 2,097,152
 * lines in some direction are rejected with CLAW_EBOUNDS.  All calls on one
 * device share that device's copy of the array, and it keeps the last call's
 * contents; calls that overlap on the same device (different streams) race
 * on it, so serialise them there.  Calls on different devices use different
 * copies and do not interfere.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  Asynchronous on cuda_stream: *out
 * is valid once the stream reaches it.  Errors: CLAW_EINVAL for bad
 * arguments, CLAW_EBOUNDS for oversized grids, CLAW_ECUDA if the lookup or a
 * launch fails (message in claw_last_error()). */
claw_status claw_max_speed_noalloc(const claw_grid* grid, claw_system system,
                                   const claw_bc bc[6], const claw_params* params,
                                   const double* q, const double* rho, const double* K,
                                   double* out, void* cuda_stream);

/* ---------------------------------------------------------------- measurement */

/* Take nsteps accepted steps like claw_run_steps inside one CUDA graph whose
 * kernels are bracketed by CUDA events (the per-kernel times Sec. 7.1's
 * roofline analysis works from), and report the average duration of
 * one launch of each kernel kind: kernel_ms[d] for the d-sweep (d < ndim;
 * with Strang splitting the sum over the step's d sweeps; with
 * CLAW_SPLIT_UNSPLIT kernel_ms[0] is the unsplit update and kernel_ms[1] is
 * 0), kernel_ms[3] for the step-control kernel; *total_ms for the whole graph.
 * *launches receives the number of kernels launched.  Synchronises. */
claw_status claw_profile_steps(claw_solver* s, int nsteps, double kernel_ms[4],
                               double* total_ms, long* launches);

/* Fused multiply-add throughput of this GPU (flop/s, 2 per FMA) in FP32 or
 * FP64, measured with independent FMA chains on every SM -- the arithmetic
 * roof the sweeps are compared with (Sec. 7.1 measures the same "achievable
 * roof").  Synchronises cuda_stream (NULL = legacy default stream). */
claw_status claw_probe_fma(int precision, double* flops_per_s, void* cuda_stream);

/* Tuning knobs (the autotuner drives these; Sec. 5.2: the tile shape of each
 * direction's kernel needs careful tuning): cells per line segment of one
 * thread in direction d (>= 4, rounded up to a multiple of 8).  With
 * CLAW_SPLIT_UNSPLIT the direction-1 length is also the rows per strip tile
 * of the unsplit update (a warp marches 28 columns down that many rows).
 * Rebuilds the tile lists. */
claw_status claw_set_segment(claw_solver* s, int d, int seg_len);

/* Order in which a direction's persistent sweep takes its tiles: the most
 * cells first (longest processing time first: balances uneven instances), or
 * the tile list's own order (instance, then line groups, then segments along
 * the lines). */
typedef enum { CLAW_ORDER_LARGEST_FIRST = 0, CLAW_ORDER_LIST = 1 } claw_tile_order;

/* Tile shape of direction d's sweep (Sec. 5.2: the block shape of each
 * direction's kernel needs careful tuning): lines per tile (the kernel
 * offers its full width and, except the two-line x sweep, half of it: 128
 * or 64 lines; 0 keeps the current one), cells per line segment (>= 4,
 * rounded up to whole 8-cell chunks; 0 keeps it) and the tile order (a
 * claw_tile_order, -1 keeps it).  The result of a step does not depend on
 * the shape beyond rounding (the first cells of a segment take separately
 * compiled code).  Rebuilds the tile lists.  CLAW_EINVAL for an unoffered
 * width. */
claw_status claw_set_tile_shape(claw_solver* s, int d, int lines, int seg_len, int order);
claw_status claw_get_tile_shape(claw_solver* s, int d, int* lines, int* seg_len, int* order);

/* Autotuner (the tuning of tile shapes Sec. 5.2 calls for): for every direction, time trial_steps steps (CUDA events around
 * each sweep) twice with each candidate segment length and keep the fastest
 * (with CLAW_SPLIT_UNSPLIT: the rows per strip tile, timed on the unsplit
 * kernel, from fixed lengths 16..256).  The
 * candidates are fixed lengths plus, for w = 1..4, the shortest length whose
 * tiles fit in w waves of the CTAs the GPU holds at once; a second pass
 * tries the lengths that split the longest line into equal whole chunks
 * within a factor 1.5 of the first pass's best; this for each tile width
 * the direction offers, then the tile order at the best shape;
 * seg_out[d] (may be NULL) receives the segment length
 * (claw_get_tile_shape gives the whole shape).  The state, clock and step
 * counters are restored afterwards, so the solution is unchanged.
 * Synchronises. */
claw_status claw_autotune(claw_solver* s, int trial_steps, int seg_out[3]);

#ifdef __cplusplus
}
#endif
#endif /* CLAW_H */
