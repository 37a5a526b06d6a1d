/*
 * CPU oracle for the dimension-split finite-volume wave-propagation step of
 * CUDACLAW (Sec. 3, Eq. LW-update, Eq. CFL-condition; Sec. 4.1 pipeline).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA path: only
 * the tests, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or constant with the CUDA library and
 * neither side includes the other.  It is plain, slow and written to be read
 * against the paper: FP64 everywhere, one line of cells at a time, full
 * temporaries (waves W[I][p][c], speeds s[I][p], limited waves, correction
 * fluxes) and no fusion.  Build it with -O2 -ffp-contract=off so no multiply
 * is fused into an add.
 *
 * Formulas the paper leaves to its textbook reference (the acoustic and
 * shallow-water Riemann solvers, the Harten-Hyman entropy fix, the minmod and
 * MC limiters, the ghost-cell rules) are the standard ones; each function
 * states the one it implements.
 *
 * Conventions:
 *   state q: structure of arrays, q[f][z][y][x], interior cells only,
 *            x fastest; ncell = nx*ny*nz (nz = 1 in 2D).
 *   interface I of a line lies between cells I-1 and I.
 *   reduced state along direction d: component 0 = p (acoustics) or h (shallow
 *   water), 1 = the velocity / momentum normal to the sweep, 2 = the
 *   transverse momentum (shallow water only).
 */
#ifndef ORC_H
#define ORC_H

#ifdef __cplusplus
extern "C" {
#endif

/* ORC_SHALLOW_WATER_BATHY: shallow water over a bottom elevation B per
 * cell, in the f-wave form (the returned "waves" are f-waves Z_p, and the
 * correction term uses sign(s_p) instead of |s_p|).  ORC_SHALLOW_WATER_DRY:
 * shallow water over B with wetting and drying (cells with h <= dry_tol are
 * dry), HLLE waves; see orc_rp_shallow_water_dry. */
enum { ORC_ACOUSTICS = 0, ORC_ACOUSTICS_VAR = 1, ORC_SHALLOW_WATER = 2, ORC_SHALLOW_WATER_BATHY = 3,
       ORC_SHALLOW_WATER_DRY = 4 };
/* ORC_LIM_NONE: unlimited second-order correction (Lax-Wendroff);
 * ORC_LIM_FIRST_ORDER: no correction at all (Godunov's first-order upwind
 * method: the Riemann solution and the fluctuation update alone). */
enum { ORC_LIM_NONE = 0, ORC_LIM_MINMOD = 1, ORC_LIM_MC = 2, ORC_LIM_FIRST_ORDER = 3 };
enum { ORC_BC_PERIODIC = 0, ORC_BC_EXTRAP = 1, ORC_BC_WALL = 2 };
/* Sweep order of a step (the splittings of Eq. LW-update's Clawpack base,
 * Sec. 3): GODUNOV x(dt) y(dt) [z(dt)]; STRANG x(dt/2) y(dt) x(dt/2) in 2D,
 * x(dt/2) y(dt/2) z(dt) y(dt/2) x(dt/2) in 3D; UNSPLIT one update from the x
 * and y Riemann problems of Q^n with transverse waves (2D; orc_unsplit.c). */
enum { ORC_SPLIT_GODUNOV = 0, ORC_SPLIT_STRANG = 1, ORC_SPLIT_UNSPLIT = 2 };

typedef struct {
    int ndim;              /* 2 or 3 */
    int n[3];              /* interior cells per direction; n[2] = 1 in 2D */
    double dx[3];          /* cell widths */
    int system;            /* ORC_ACOUSTICS, ORC_ACOUSTICS_VAR, ORC_SHALLOW_WATER */
    int limiter;           /* ORC_LIM_* */
    int bc[6];             /* x-lo, x-hi, y-lo, y-hi, z-lo, z-hi: ORC_BC_* */
    double rho, K;         /* constant acoustics coefficients */
    double g;              /* gravity (shallow water) */
    double cfl_desired;    /* target Courant number for the next step */
    double cfl_max;        /* a step whose Courant number exceeds this is redone */
    double dt_max;         /* cap on the step when every speed is zero */
    int max_retries;       /* consecutive rejections before giving up */
    const double *rho_cell;/* per-cell rho, K (ORC_ACOUSTICS_VAR), else NULL */
    const double *K_cell;
    int splitting;         /* ORC_SPLIT_* */
    const double *B_cell;  /* bottom elevation per cell (ORC_SHALLOW_WATER_BATHY / _DRY), else NULL */
    double dry_tol;        /* ORC_SHALLOW_WATER_DRY: a cell with h <= dry_tol is dry */
} orc_problem;

/* Number of state fields m and waves mwaves for a problem. */
int orc_m(const orc_problem *P);
int orc_mwaves(const orc_problem *P);

/* Riemann solvers at one interface, on reduced states (see above).
 * Outputs: W[p][c] (waves), s[p] (speeds), amdq[c] = A-dQ, apdq[c] = A+dQ. */
void orc_rp_acoustics(const double *ql, const double *qr,
                      double rho_l, double K_l, double rho_r, double K_r,
                      double W[3][3], double s[3], double amdq[3], double apdq[3]);
void orc_rp_shallow_water(const double *ql, const double *qr, double g,
                          double W[3][3], double s[3], double amdq[3], double apdq[3]);
/* f-waves W[p][c] = Z_p of the bathymetry system (see orc_shallow_water.c). */
void orc_rp_shallow_water_bathy(const double *ql, const double *qr, double B_l, double B_r,
                                double g, double W[3][3], double s[3], double amdq[3],
                                double apdq[3]);

/* HLLE waves of the wet/dry bathymetry system (see orc_shallow_water.c);
 * zero waves (but not fluctuations) at an interface with a dry side. */
void orc_rp_shallow_water_dry(const double *ql, const double *qr, double B_l, double B_r,
                              double g, double dry_tol, double W[3][3], double s[3],
                              double amdq[3], double apdq[3]);

/* Wave limiter function phi(theta), minmod or MC; ORC_LIM_NONE gives 1. */
double orc_phi(int limiter, double theta);

/* One directional sweep (one half of Eq. LW-update) over lines
 * [line_lo, line_hi) of direction d, qin -> qout, with nu = dt / dx[d].
 * Fields the sweep does not change are copied.  Ghost cells come from qin by
 * the boundary rules.  Returns the largest |s^p| over the interfaces bounding
 * the interior cells of those lines.  line_hi < 0 means all lines. */
double orc_sweep(const orc_problem *P, int d, const double *qin, double *qout,
                 double dt, long line_lo, long line_hi);

/* Transverse solvers of the unsplit update (see orc_unsplit.c): split the
 * reduced fluctuation a (p or h, normal, transverse component) of a cell
 * into the parts crossing its lower (bm) and upper (bp) transverse
 * interfaces. */
void orc_tr_acoustics(const double *a, double rho_d, double K_d, double rho_c, double K_c,
                      double rho_u, double K_u, double bm[3], double bp[3]);
void orc_tr_shallow_water(const double *a, const double *qd, const double *qc,
                          const double *qu, double g, double bm[3], double bp[3]);

/* One unsplit step qin -> qout with dt (2D acoustics or shallow water);
 * m_d[0], m_d[1] receive the largest |s| along x and y.  Returns 0, or -1
 * for a problem it does not cover. */
int orc_unsplit_step(const orc_problem *P, const double *qin, double *qout, double dt,
                     double m_d[3]);

/* Largest |s^p| along direction d from a Riemann pass over q (no update). */
double orc_max_speed_dir(const orc_problem *P, int d, const double *q);

/* Number of independent lines of direction d. */
long orc_nlines(const orc_problem *P, int d);

/* Sweeps of one step: direction and fraction of dt of each, in order;
 * returns their number. */
int orc_sequence(const orc_problem *P, int dirs[5], double frac[5]);

/* Time stepping with the CFL rule (Eq. CFL-condition; Sec. 4.1 revert-and-redo).
 * m_d is the largest speed over every sweep along d in the step; the
 * Courant number of a step is dt * max_d(m_d / dx_d) for either splitting.
 *   mode 0: take nsteps accepted steps;  mode 1: advance to t_final.
 *   *dt <= 0 on entry: start from dt = cfl_desired / max_d(m_d / dx_d) of q.
 *   fixed_dt > 0: every step uses fixed_dt and is accepted (no CFL control).
 * On return q holds the new state, *t, *dt (the next step), *nacc, *nrej
 * are updated.  Returns 0, -1 after max_retries consecutive rejections, or
 * -2 for an unsplit step on a problem it does not cover. */
int orc_run(const orc_problem *P, double *q, int mode, long nsteps, double t_final,
            double fixed_dt, double *t, double *dt, long *nacc, long *nrej,
            double *cfl_last);

/* Threads the sweeps use. */
int orc_threads(void);

#ifdef __cplusplus
}
#endif
#endif
