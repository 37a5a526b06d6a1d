/*
 * Oracle (test infrastructure only): boundary ghost cells, wave limiter,
 * one directional sweep of the split update, and the CFL time-step control.
 *
 * Sec. 3 Eq. LW-update: along direction d, with nu = dt / dx_d,
 *     Q_i <- Q_i - nu (A+dQ_{i-1/2} + A-dQ_{i+1/2}) - nu (F_{i+1/2} - F_{i-1/2}),
 *     F_{i-1/2} = 1/2 sum_p |s_p| (1 - nu |s_p|) W~_p,
 * where W~_p is the wave limited against the same family's wave at the
 * upwind interface (Sec. 3, the wave limiter).  Without the second term
 * (W~ = 0) this is Godunov's first-order upwind method: the Riemann solution
 * and its fluctuation update alone, the part of the sweep the paper isolates
 * as its "Riemann solver" kernels (Sec. 7.1).  The x sweep maps Q^n to Q*,
 * the y sweep Q* to Q** (and z in 3D); every step runs x, y(, z) in order.
 * The CFL rule (Eq. CFL-condition, Sec. 4.1): a step taken with dt is kept
 * when dt * max_d(m_d / dx_d) <= cfl_max, else redone with the new estimate;
 * the next dt is cfl_desired / max_d(m_d / dx_d).
 *
 * Ghost cells (two per side; the paper's BC stage, Sec. 4.1):
 *   periodic: ghost -1 = cell N-1, ghost -2 = cell N-2, ghost N = cell 0, N+1 = cell 1;
 *   extrap:   every ghost copies the nearest interior cell;
 *   wall:     ghost -1 = cell 0, ghost -2 = cell 1 (and mirrored at the top),
 *             with the normal velocity / momentum negated.
 * Material coefficients in the ghosts follow the same index rule, unsigned.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "orc.h"

static int is_sw(const orc_problem *P)
{
    return P->system == ORC_SHALLOW_WATER || P->system == ORC_SHALLOW_WATER_BATHY ||
           P->system == ORC_SHALLOW_WATER_DRY;
}

/* Systems whose Riemann solver returns f-waves over a bottom elevation. */
static int has_bed(const orc_problem *P)
{
    return P->system == ORC_SHALLOW_WATER_BATHY || P->system == ORC_SHALLOW_WATER_DRY;
}

int orc_m(const orc_problem *P)
{
    if (is_sw(P)) return 3;
    return P->ndim + 1;
}

int orc_mwaves(const orc_problem *P)
{
    return is_sw(P) ? 3 : 2;
}

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Components of the reduced state along d, as field indices. */
static int nq_of(const orc_problem *P)
{
    return is_sw(P) ? 3 : 2;
}

static int field_of(const orc_problem *P, int d, int c)
{
    if (c == 0) return 0;
    if (c == 1) return 1 + d;             /* normal velocity or momentum */
    return 2 - d;                          /* shallow water transverse momentum (2D) */
}

long orc_nlines(const orc_problem *P, int d)
{
    long ncell = (long)P->n[0] * P->n[1] * P->n[2];
    return ncell / P->n[d];
}

/* Flat index of cell i of line `line` along direction d. */
static long cell_index(const orc_problem *P, int d, long line, int i)
{
    long nx = P->n[0], ny = P->n[1];
    long x, y, z;
    if (d == 0) {
        y = line % ny; z = line / ny; x = i;
    } else if (d == 1) {
        x = line % nx; z = line / nx; y = i;
    } else {
        x = line % nx; y = line / nx; z = i;
    }
    return (z * ny + y) * nx + x;
}

/* Interior cell that ghost / interior position i stands for, and the sign of
 * the normal component there. */
static int source_cell(const orc_problem *P, int d, int i, double *sign)
{
    int N = P->n[d];
    *sign = 1.0;
    if (i >= 0 && i < N) return i;
    int lo = i < 0;
    int kind = P->bc[2 * d + (lo ? 0 : 1)];
    if (kind == ORC_BC_PERIODIC) {
        return lo ? i + N : i - N;
    }
    if (kind == ORC_BC_EXTRAP) {
        return lo ? 0 : N - 1;
    }
    /* wall */
    *sign = -1.0;
    return lo ? -1 - i : 2 * N - 1 - i;
}

double orc_phi(int limiter, double theta)
{
    if (limiter == ORC_LIM_MINMOD) {
        double a = theta < 1.0 ? theta : 1.0;
        return a > 0.0 ? a : 0.0;
    }
    if (limiter == ORC_LIM_FIRST_ORDER) return 0.0;
    if (limiter == ORC_LIM_MC) {
        double a = 0.5 * (1.0 + theta);
        if (2.0 < a) a = 2.0;
        if (2.0 * theta < a) a = 2.0 * theta;
        return a > 0.0 ? a : 0.0;
    }
    return 1.0;
}

static void riemann(const orc_problem *P, const double *ql, const double *qr,
                    double rho_l, double K_l, double rho_r, double K_r, double B_l, double B_r,
                    double W[3][3], double s[3], double amdq[3], double apdq[3])
{
    if (P->system == ORC_SHALLOW_WATER)
        orc_rp_shallow_water(ql, qr, P->g, W, s, amdq, apdq);
    else if (P->system == ORC_SHALLOW_WATER_BATHY)
        orc_rp_shallow_water_bathy(ql, qr, B_l, B_r, P->g, W, s, amdq, apdq);
    else if (P->system == ORC_SHALLOW_WATER_DRY)
        orc_rp_shallow_water_dry(ql, qr, B_l, B_r, P->g, P->dry_tol, W, s, amdq, apdq);
    else
        orc_rp_acoustics(ql, qr, rho_l, K_l, rho_r, K_r, W, s, amdq, apdq);
}

/* Per-thread work arrays for one line of N cells (+ 2 ghosts each side). */
typedef struct {
    double (*q)[3];        /* cells -2..N+1 at index i+2 */
    double *rho, *K;       /* same indexing */
    double *B;             /* bottom elevation, same indexing */
    double (*W)[3][3];     /* interfaces -1..N+1 at index I+1 */
    double (*s)[3];
    double (*amdq)[3];
    double (*apdq)[3];
    double (*Wt)[3][3];    /* limited waves */
    double (*F)[3];        /* correction flux */
    double (*qnew)[3];     /* cells 0..N-1 */
} line_work;

static void work_alloc(line_work *w, int N)
{
    w->q = malloc(sizeof(double[3]) * (N + 4));
    w->rho = malloc(sizeof(double) * (N + 4));
    w->K = malloc(sizeof(double) * (N + 4));
    w->B = malloc(sizeof(double) * (N + 4));
    w->W = malloc(sizeof(double[3][3]) * (N + 3));
    w->s = malloc(sizeof(double[3]) * (N + 3));
    w->amdq = malloc(sizeof(double[3]) * (N + 3));
    w->apdq = malloc(sizeof(double[3]) * (N + 3));
    w->Wt = malloc(sizeof(double[3][3]) * (N + 3));
    w->F = malloc(sizeof(double[3]) * (N + 3));
    w->qnew = malloc(sizeof(double[3]) * N);
}

static void work_free(line_work *w)
{
    free(w->q); free(w->rho); free(w->K); free(w->B); free(w->W); free(w->s);
    free(w->amdq); free(w->apdq); free(w->Wt); free(w->F); free(w->qnew);
}

/* Fill the line's cells -2..N+1 (reduced state and coefficients). */
static void gather_line(const orc_problem *P, int d, long line, const double *qin,
                        line_work *w)
{
    int N = P->n[d];
    long ncell = (long)P->n[0] * P->n[1] * P->n[2];
    int nq = nq_of(P);
    for (int i = -2; i < N + 2; ++i) {
        double sign;
        int j = source_cell(P, d, i, &sign);
        long idx = cell_index(P, d, line, j);
        for (int c = 0; c < nq; ++c) {
            double v = qin[(long)field_of(P, d, c) * ncell + idx];
            w->q[i + 2][c] = (c == 1) ? sign * v : v;
        }
        w->B[i + 2] = has_bed(P) ? P->B_cell[idx] : 0.0;
        if (P->system == ORC_ACOUSTICS_VAR) {
            w->rho[i + 2] = P->rho_cell[idx];
            w->K[i + 2] = P->K_cell[idx];
        } else {
            w->rho[i + 2] = P->rho;
            w->K[i + 2] = P->K;
        }
    }
}

/* The split update along one line; returns max |s| over interfaces 0..N. */
static double update_line(const orc_problem *P, int d, double nu, line_work *w)
{
    int N = P->n[d];
    int nq = nq_of(P);
    int nw = orc_mwaves(P);

    /* 1. Riemann problems at interfaces I = -1..N+1 (between cells I-1, I). */
    for (int I = -1; I <= N + 1; ++I) {
        int L = I - 1 + 2, R = I + 2;   /* array positions of cells I-1, I */
        riemann(P, w->q[L], w->q[R], w->rho[L], w->K[L], w->rho[R], w->K[R], w->B[L], w->B[R],
                w->W[I + 1], w->s[I + 1], w->amdq[I + 1], w->apdq[I + 1]);
    }

    /* 2. Limiter at interfaces I = 0..N: compare each wave with the same
     *    family's wave at the upwind interface (I-1 if s > 0, else I+1).
     *    The first-order method has no correction: W~ = 0, so F = 0. */
    for (int I = 0; I <= N; ++I) {
        if (P->limiter == ORC_LIM_FIRST_ORDER) {
            for (int p = 0; p < nw; ++p)
                for (int c = 0; c < nq; ++c) w->Wt[I + 1][p][c] = 0.0;
            continue;
        }
        for (int p = 0; p < nw; ++p) {
            const double *Wi = w->W[I + 1][p];
            int J = w->s[I + 1][p] > 0.0 ? I - 1 : I + 1;
            const double *Wj = w->W[J + 1][p];
            double dot_ii = 0.0, dot_ji = 0.0;
            for (int c = 0; c < nq; ++c) {
                dot_ii += Wi[c] * Wi[c];
                dot_ji += Wj[c] * Wi[c];
            }
            double phi = 0.0;
            if (dot_ii != 0.0) phi = orc_phi(P->limiter, dot_ji / dot_ii);
            for (int c = 0; c < nq; ++c) w->Wt[I + 1][p][c] = phi * Wi[c];
        }
    }

    /* 3. Correction flux F_I = 1/2 sum_p |s_p| (1 - nu |s_p|) W~_p; for
     *    f-waves Z_p = s_p W_p the factor |s_p| becomes sign(s_p). */
    int fwave = P->system == ORC_SHALLOW_WATER_BATHY;
    for (int I = 0; I <= N; ++I) {
        for (int c = 0; c < nq; ++c) {
            double acc = 0.0;
            for (int p = 0; p < nw; ++p) {
                double sp = w->s[I + 1][p];
                double as = fabs(sp);
                double k = fwave ? (sp > 0.0 ? 1.0 : (sp < 0.0 ? -1.0 : 0.0)) : as;
                acc += k * (1.0 - nu * as) * w->Wt[I + 1][p][c];
            }
            w->F[I + 1][c] = 0.5 * acc;
        }
    }

    /* 4. Conservative update of cells 0..N-1. */
    for (int i = 0; i < N; ++i) {
        for (int c = 0; c < nq; ++c) {
            double first = w->apdq[i + 1][c] + w->amdq[i + 2][c];
            double second = w->F[i + 2][c] - w->F[i + 1][c];
            w->qnew[i][c] = w->q[i + 2][c] - nu * first - nu * second;
        }
    }

    /* 5. Largest speed over the interfaces that bound interior cells. */
    double m = 0.0;
    for (int I = 0; I <= N; ++I)
        for (int p = 0; p < nw; ++p) {
            double as = fabs(w->s[I + 1][p]);
            if (as > m) m = as;
        }
    return m;
}

double orc_sweep(const orc_problem *P, int d, const double *qin, double *qout,
                 double dt, long line_lo, long line_hi)
{
    long ncell = (long)P->n[0] * P->n[1] * P->n[2];
    int m = orc_m(P);
    int nq = nq_of(P);
    int N = P->n[d];
    double nu = dt / P->dx[d];
    long nlines = orc_nlines(P, d);
    if (line_hi < 0 || line_hi > nlines) line_hi = nlines;
    if (line_lo < 0) line_lo = 0;

    if (qout != qin) {
        if (line_lo == 0 && line_hi == nlines) {
            memcpy(qout, qin, sizeof(double) * (size_t)m * (size_t)ncell);
        } else {
            /* copy only the cells of the selected lines */
            for (long line = line_lo; line < line_hi; ++line)
                for (int i = 0; i < N; ++i) {
                    long idx = cell_index(P, d, line, i);
                    for (int f = 0; f < m; ++f) qout[f * ncell + idx] = qin[f * ncell + idx];
                }
        }
    }

    double mmax = 0.0;
#pragma omp parallel reduction(max : mmax)
    {
        line_work w;
        work_alloc(&w, N);
#pragma omp for schedule(static)
        for (long line = line_lo; line < line_hi; ++line) {
            gather_line(P, d, line, qin, &w);
            double ml = update_line(P, d, nu, &w);
            if (ml > mmax) mmax = ml;
            for (int i = 0; i < N; ++i) {
                long idx = cell_index(P, d, line, i);
                for (int c = 0; c < nq; ++c)
                    qout[(long)field_of(P, d, c) * ncell + idx] = w.qnew[i][c];
            }
        }
        work_free(&w);
    }
    return mmax;
}

double orc_max_speed_dir(const orc_problem *P, int d, const double *q)
{
    int N = P->n[d];
    int nw = orc_mwaves(P);
    long nlines = orc_nlines(P, d);
    double mmax = 0.0;
#pragma omp parallel reduction(max : mmax)
    {
        line_work w;
        work_alloc(&w, N);
#pragma omp for schedule(static)
        for (long line = 0; line < nlines; ++line) {
            gather_line(P, d, line, q, &w);
            for (int I = 0; I <= N; ++I) {
                double W[3][3], s[3], amdq[3], apdq[3];
                int L = I + 1, R = I + 2;
                riemann(P, w.q[L], w.q[R], w.rho[L], w.K[L], w.rho[R], w.K[R], w.B[L], w.B[R],
                        W, s, amdq, apdq);
                for (int p = 0; p < nw; ++p)
                    if (fabs(s[p]) > mmax) mmax = fabs(s[p]);
            }
        }
        work_free(&w);
    }
    return mmax;
}

/* max_d (m_d / dx_d), the quantity the CFL condition bounds. */
static double speed_over_dx(const orc_problem *P, const double *m_d)
{
    double M = 0.0;
    for (int d = 0; d < P->ndim; ++d) {
        double v = m_d[d] / P->dx[d];
        if (v > M) M = v;
    }
    return M;
}

static double next_dt(const orc_problem *P, double M)
{
    double dt = M > 0.0 ? P->cfl_desired / M : P->dt_max;
    return dt < P->dt_max ? dt : P->dt_max;
}

int orc_sequence(const orc_problem *P, int dirs[5], double frac[5])
{
    int n = 0;
    if (P->splitting == ORC_SPLIT_STRANG) {
        /* half steps outside-in, the last direction a full step */
        for (int d = 0; d < P->ndim - 1; ++d) { dirs[n] = d; frac[n] = 0.5; ++n; }
        dirs[n] = P->ndim - 1; frac[n] = 1.0; ++n;
        for (int d = P->ndim - 2; d >= 0; --d) { dirs[n] = d; frac[n] = 0.5; ++n; }
    } else {
        for (int d = 0; d < P->ndim; ++d) { dirs[n] = d; frac[n] = 1.0; ++n; }
    }
    return n;
}

int orc_run(const orc_problem *P, double *q, int mode, long nsteps, double t_final,
            double fixed_dt, double *t, double *dt, long *nacc, long *nrej,
            double *cfl_last)
{
    long ncell = (long)P->n[0] * P->n[1] * P->n[2];
    size_t bytes = sizeof(double) * (size_t)orc_m(P) * (size_t)ncell;
    double *a = malloc(bytes), *b = malloc(bytes);
    int status = 0;

    if (fixed_dt <= 0.0 && *dt <= 0.0) {
        double m_d[3] = {0.0, 0.0, 0.0};
        for (int d = 0; d < P->ndim; ++d) m_d[d] = orc_max_speed_dir(P, d, q);
        *dt = next_dt(P, speed_over_dx(P, m_d));
    }

    long taken = 0;
    int streak = 0;
    for (;;) {
        if (mode == 0 && taken >= nsteps) break;
        if (mode == 1 && *t >= t_final) break;

        double dt_try = fixed_dt > 0.0 ? fixed_dt : *dt;
        int last = 0;
        if (mode == 1 && dt_try >= t_final - *t) {
            dt_try = t_final - *t;
            last = 1;
        }

        /* x, y (, z) sweeps in order: q -> a -> b (-> a) */
        double m_d[3] = {0.0, 0.0, 0.0};
        const double *src = q;
        double *dst = a;
        for (int d = 0; d < 3; ++d) m_d[d] = 0.0;
        if (P->splitting == ORC_SPLIT_UNSPLIT) {
            if (orc_unsplit_step(P, q, a, dt_try, m_d) != 0) { status = -2; break; }
            src = a;
        } else {
            int dirs[5];
            double frac[5];
            int nsw = orc_sequence(P, dirs, frac);
            for (int k = 0; k < nsw; ++k) {
                double m = orc_sweep(P, dirs[k], src, dst, frac[k] * dt_try, 0, -1);
                if (m > m_d[dirs[k]]) m_d[dirs[k]] = m;
                src = dst;
                dst = (dst == a) ? b : a;
            }
        }
        double M = speed_over_dx(P, m_d);
        double cfl = dt_try * M;
        if (cfl_last) *cfl_last = cfl;

        if (fixed_dt <= 0.0 && cfl > P->cfl_max) {
            *nrej += 1;
            *dt = next_dt(P, M);
            if (++streak > P->max_retries) { status = -1; break; }
            continue;
        }
        streak = 0;
        memcpy(q, src, bytes);
        *t = last ? t_final : *t + dt_try;
        *nacc += 1;
        taken += 1;
        if (fixed_dt <= 0.0) *dt = next_dt(P, M);
    }
    free(a);
    free(b);
    return status;
}
