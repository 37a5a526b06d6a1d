/*
 * Oracle (test infrastructure only): the unsplit two-dimensional form of the
 * wave-propagation update (Sec. 3 Eq. LW-update without dimensional
 * splitting; the Clawpack base offers both), with transverse propagation of
 * the fluctuations and of the second-order corrections.
 *
 * Every Riemann problem of a step is taken from Q^n.  Along x, at interface
 * i-1/2 of row j (cells i-1, i): waves W_p, speeds s_p, A-dQ, A+dQ, and the
 * correction cq = sum_p |s_p| (1 - nu_x |s_p|) W~_p (W~ limited as in the
 * split sweep), so F_{i-1/2,j} = cq / 2.  The fluctuations, modified by the
 * correction (A-dQ + cq enters cell i-1, A+dQ - cq enters cell i), are split
 * by a transverse solver along y into a down-going part B-(.) and an
 * up-going part B+(.), which change the y-direction fluxes of the cell they
 * entered:
 *   G_{k,j-1/2} -= (nu_x / 2) B-(.),   G_{k,j+1/2} -= (nu_x / 2) B+(.),
 * k the cell's column.  Along y the roles of x and y swap.  The update is
 *   Q_ij <- Q_ij - nu_x (A+dQ_{i-1/2,j} + A-dQ_{i+1/2,j}) - nu_x (F_{i+1/2,j} - F_{i-1/2,j})
 *               - nu_y (B+dQ_{i,j-1/2} + B-dQ_{i,j+1/2}) - nu_y (G_{i,j+1/2} - G_{i,j-1/2}).
 *
 * Transverse solvers (x sweep; a y sweep uses the same with u, v swapped),
 * on a fluctuation a in the reduced state of the sweep:
 *   acoustics: the down-going part uses the interface between the cell below
 *     (Z_d, c_d) and the cell (Z_c):  al = (-a_p + Z_c a_t) / (Z_d + Z_c),
 *     B-(a) = -c_d al (-Z_d, 0, 1);  the up-going part the interface to the
 *     cell above (Z_u, c_u): ar = (a_p + Z_c a_t) / (Z_c + Z_u),
 *     B+(a) = c_u ar (Z_u, 0, 1)   (components: p, normal, transverse velocity).
 *   shallow water: Roe averages with the cell below (for B-) or above (for
 *     B+), transverse eigenvectors (1, u~, v~ -+ c~), (0, 1, 0) with speeds
 *     v~ -+ c~, v~; strengths a1 = ((v~ + c~) a_0 - a_2) / 2c~,
 *     a2 = a_1 - u~ a_0, a3 = (a_2 - (v~ - c~) a_0) / 2c~;
 *     B-(a) = sum min(speed, 0) a_p r_p, B+(a) = sum max(speed, 0) a_p r_p.
 * Ghost cells: two layers; a corner ghost maps its x and y indices by their
 * own boundary rules (the maps act on different coordinates and commute).
 * 2D only; acoustics (constant or per-cell coefficients) and shallow water.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "orc.h"

void orc_tr_acoustics(const double *a, double rho_d, double K_d, double rho_c, double K_c,
                      double rho_u, double K_u, double bm[3], double bp[3])
{
    double c_d = sqrt(K_d / rho_d), c_c = sqrt(K_c / rho_c), c_u = sqrt(K_u / rho_u);
    double Z_d = rho_d * c_d, Z_c = rho_c * c_c, Z_u = rho_u * c_u;
    double al = (-a[0] + Z_c * a[2]) / (Z_d + Z_c);
    double ar = (a[0] + Z_c * a[2]) / (Z_c + Z_u);
    bm[0] = -c_d * al * (-Z_d);
    bm[1] = 0.0;
    bm[2] = -c_d * al;
    bp[0] = c_u * ar * Z_u;
    bp[1] = 0.0;
    bp[2] = c_u * ar;
}

/* One half of the shallow-water transverse split: the Roe averages of the
 * cell and its neighbour n, then the part with speeds of the given sign. */
static void tr_sw_half(const double *a, const double *qn, const double *qc, double g,
                       int upward, double out[3])
{
    double h_n = qn[0], h_c = qc[0];
    double sn = sqrt(h_n), sc = sqrt(h_c);
    double ut = (sn * (qn[1] / h_n) + sc * (qc[1] / h_c)) / (sn + sc);   /* along the sweep */
    double vt = (sn * (qn[2] / h_n) + sc * (qc[2] / h_c)) / (sn + sc);   /* transverse */
    double ct = sqrt(g * 0.5 * (h_n + h_c));
    double a1 = ((vt + ct) * a[0] - a[2]) / (2.0 * ct);
    double a2 = a[1] - ut * a[0];
    double a3 = (a[2] - (vt - ct) * a[0]) / (2.0 * ct);
    double lam[3] = {vt - ct, vt, vt + ct};
    double r[3][3] = {{1.0, ut, vt - ct}, {0.0, 1.0, 0.0}, {1.0, ut, vt + ct}};
    double al[3] = {a1, a2, a3};
    for (int c = 0; c < 3; ++c) out[c] = 0.0;
    for (int p = 0; p < 3; ++p) {
        double l = upward ? (lam[p] > 0.0 ? lam[p] : 0.0) : (lam[p] < 0.0 ? lam[p] : 0.0);
        for (int c = 0; c < 3; ++c) out[c] += l * al[p] * r[p][c];
    }
}

void orc_tr_shallow_water(const double *a, const double *qd, const double *qc,
                          const double *qu, double g, double bm[3], double bp[3])
{
    tr_sw_half(a, qd, qc, g, 0, bm);
    tr_sw_half(a, qu, qc, g, 1, bp);
}

/* Padded 2D arrays: cell (i, j), i in [-2, nx+1], j in [-2, ny+1]. */
typedef struct {
    int nx, ny;
    double *q;       /* [(j+2)(nx+4) + (i+2)][3] */
    double *rho, *K;
} padded;

static long pidx(const padded *u, int i, int j) { return (long)(j + 2) * (u->nx + 4) + (i + 2); }

static int map_index(const orc_problem *P, int d, int k, double *sign)
{
    int N = P->n[d];
    *sign = 1.0;
    if (k >= 0 && k < N) return k;
    int lo = k < 0;
    int kind = P->bc[2 * d + (lo ? 0 : 1)];
    if (kind == ORC_BC_PERIODIC) return lo ? k + N : k - N;
    if (kind == ORC_BC_EXTRAP) return lo ? 0 : N - 1;
    *sign = -1.0;
    return lo ? -1 - k : 2 * N - 1 - k;
}

static void fill_padded(const orc_problem *P, const double *q, padded *u)
{
    int nx = P->n[0], ny = P->n[1];
    long ncell = (long)nx * ny;
    for (int j = -2; j < ny + 2; ++j)
        for (int i = -2; i < nx + 2; ++i) {
            double sx, sy;
            int si = map_index(P, 0, i, &sx);
            int sj = map_index(P, 1, j, &sy);
            long src = (long)sj * nx + si;
            long k = pidx(u, i, j);
            u->q[3 * k + 0] = q[src];
            u->q[3 * k + 1] = sx * q[ncell + src];
            u->q[3 * k + 2] = sy * q[2 * ncell + src];
            if (P->system == ORC_ACOUSTICS_VAR) {
                u->rho[k] = P->rho_cell[src];
                u->K[k] = P->K_cell[src];
            } else {
                u->rho[k] = P->rho;
                u->K[k] = P->K;
            }
        }
}

/* Reduced state of cell (i, j) for a sweep along d: (p, u_n, u_t) or
 * (h, h u_n, h u_t). */
static void reduced(const padded *u, int i, int j, int d, double r[3])
{
    const double *c = u->q + 3 * pidx(u, i, j);
    r[0] = c[0];
    r[1] = d == 0 ? c[1] : c[2];
    r[2] = d == 0 ? c[2] : c[1];
}

/* A reduced vector of a sweep along d back in field order. */
static void to_fields(int d, const double r[3], double f[3])
{
    f[0] = r[0];
    f[1] = d == 0 ? r[1] : r[2];
    f[2] = d == 0 ? r[2] : r[1];
}

static void normal_rp(const orc_problem *P, const padded *u, int d, int il, int jl, int ir, int jr,
                      double W[3][3], double s[3], double am[3], double ap[3])
{
    double ql[3], qr[3];
    reduced(u, il, jl, d, ql);
    reduced(u, ir, jr, d, qr);
    if (P->system == ORC_SHALLOW_WATER) {
        orc_rp_shallow_water(ql, qr, P->g, W, s, am, ap);
    } else {
        long kl = pidx(u, il, jl), kr = pidx(u, ir, jr);
        orc_rp_acoustics(ql, qr, u->rho[kl], u->K[kl], u->rho[kr], u->K[kr], W, s, am, ap);
        /* the third (transverse) component of every acoustic wave is zero */
        s[2] = 0.0;
        for (int c = 0; c < 3; ++c) W[2][c] = 0.0;
    }
}

/* Transverse split of a reduced fluctuation a of a sweep along d entering
 * cell (i, j): the neighbours are the cells before and after it along the
 * other direction. */
static void transverse(const orc_problem *P, const padded *u, int d, int i, int j,
                       const double a[3], double bm[3], double bp[3])
{
    int di = d == 0 ? 0 : 1, dj = d == 0 ? 1 : 0;
    if (P->system == ORC_SHALLOW_WATER) {
        double qd[3], qc[3], qu[3];
        reduced(u, i - di, j - dj, d, qd);
        reduced(u, i, j, d, qc);
        reduced(u, i + di, j + dj, d, qu);
        orc_tr_shallow_water(a, qd, qc, qu, P->g, bm, bp);
    } else {
        long kd = pidx(u, i - di, j - dj), kc = pidx(u, i, j), ku = pidx(u, i + di, j + dj);
        orc_tr_acoustics(a, u->rho[kd], u->K[kd], u->rho[kc], u->K[kc], u->rho[ku], u->K[ku],
                         bm, bp);
    }
}

int orc_unsplit_step(const orc_problem *P, const double *qin, double *qout, double dt,
                     double m_d[3])
{
    if (P->ndim != 2 || P->system == ORC_SHALLOW_WATER_BATHY || P->system == ORC_SHALLOW_WATER_DRY)
        return -1;
    int nx = P->n[0], ny = P->n[1];
    long ncell = (long)nx * ny;
    int nw = orc_mwaves(P);
    double nu[2] = {dt / P->dx[0], dt / P->dx[1]};
    padded u;
    u.nx = nx;
    u.ny = ny;
    long np = (long)(nx + 4) * (ny + 4);
    u.q = malloc(sizeof(double) * 3 * np);
    u.rho = malloc(sizeof(double) * np);
    u.K = malloc(sizeof(double) * np);
    fill_padded(P, qin, &u);

    /* Fluxes in field order on every interface of the padded grid:
     * F[(j+2)(nx+4) + (I+2)] at x-interface I of row j (I, j in the padded
     * range), G likewise at y-interface J of column i; fluctuation sums
     * dQ per interior cell. */
    double *F = calloc(3 * np, sizeof(double));
    double *G = calloc(3 * np, sizeof(double));
    double *fl = calloc(3 * 2 * np, sizeof(double));   /* [d][cell]: A+dQ in + A-dQ in */

    for (int d = 0; d < 2; ++d) {
        /* lines along d: rows (d = 0) or columns (d = 1), including the first
         * ghost line on each side (their transverse parts reach the grid) */
        int nlines = d == 0 ? ny : nx, N = d == 0 ? nx : ny;
        double *flux_d = d == 0 ? F : G;        /* correction of this direction */
        double *flux_t = d == 0 ? G : F;        /* the transverse direction's */
        double (*W)[3][3] = malloc(sizeof(double[3][3]) * (N + 3));
        double (*s)[3] = malloc(sizeof(double[3]) * (N + 3));
        double (*am)[3] = malloc(sizeof(double[3]) * (N + 3));
        double (*ap)[3] = malloc(sizeof(double[3]) * (N + 3));
        double m = 0.0;
        for (int L = -1; L <= nlines; ++L) {
            /* interfaces I = -1 .. N+1 between cells I-1 and I along the line */
            for (int I = -1; I <= N + 1; ++I) {
                int il = d == 0 ? I - 1 : L, jl = d == 0 ? L : I - 1;
                int ir = d == 0 ? I : L, jr = d == 0 ? L : I;
                normal_rp(P, &u, d, il, jl, ir, jr, W[I + 1], s[I + 1], am[I + 1], ap[I + 1]);
            }
            int interior = L >= 0 && L < nlines;
            for (int I = 0; I <= N; ++I) {
                double cq[3] = {0.0, 0.0, 0.0};
                for (int p = 0; p < nw; ++p) {
                    const double *Wi = W[I + 1][p];
                    int J = s[I + 1][p] > 0.0 ? I - 1 : I + 1;
                    const double *Wj = W[J + 1][p];
                    double dii = 0.0, dji = 0.0;
                    for (int c = 0; c < 3; ++c) {
                        dii += Wi[c] * Wi[c];
                        dji += Wj[c] * Wi[c];
                    }
                    double phi = 0.0;
                    if (dii != 0.0) phi = orc_phi(P->limiter, dji / dii);
                    double as = fabs(s[I + 1][p]);
                    for (int c = 0; c < 3; ++c) cq[c] += as * (1.0 - nu[d] * as) * (phi * Wi[c]);
                    if (interior && as > m) m = as;
                }
                /* cells on the two sides of interface I along the line */
                int il = d == 0 ? I - 1 : L, jl = d == 0 ? L : I - 1;
                int ir = d == 0 ? I : L, jr = d == 0 ? L : I;
                double f[3], half[3];
                for (int c = 0; c < 3; ++c) half[c] = 0.5 * cq[c];
                to_fields(d, half, f);
                long kI = d == 0 ? pidx(&u, I, L) : pidx(&u, L, I);
                for (int c = 0; c < 3; ++c) flux_d[3 * kI + c] += f[c];
                /* the fluctuations enter their cells (interior lines only) */
                if (interior) {
                    double fa[3], fb[3];
                    to_fields(d, am[I + 1], fa);
                    to_fields(d, ap[I + 1], fb);
                    if (I - 1 >= 0) for (int c = 0; c < 3; ++c) fl[3 * (d * np + pidx(&u, il, jl)) + c] += fa[c];
                    if (I < N) for (int c = 0; c < 3; ++c) fl[3 * (d * np + pidx(&u, ir, jr)) + c] += fb[c];
                }
                /* transverse parts of the modified fluctuations */
                double amod[3], apmod[3], bm[3], bp[3], fm[3], fp[3];
                for (int c = 0; c < 3; ++c) {
                    amod[c] = am[I + 1][c] + cq[c];
                    apmod[c] = ap[I + 1][c] - cq[c];
                }
                int side_i[2] = {il, ir}, side_j[2] = {jl, jr};
                const double *mod[2] = {amod, apmod};
                for (int sd = 0; sd < 2; ++sd) {
                    transverse(P, &u, d, side_i[sd], side_j[sd], mod[sd], bm, bp);
                    to_fields(d, bm, fm);
                    to_fields(d, bp, fp);
                    /* transverse interfaces below / above the cell:
                     * index of the interface before the cell = the cell's own index */
                    int ci = side_i[sd], cj = side_j[sd];
                    long kb = pidx(&u, ci, cj);
                    long ka = d == 0 ? pidx(&u, ci, cj + 1) : pidx(&u, ci + 1, cj);
                    for (int c = 0; c < 3; ++c) {
                        flux_t[3 * kb + c] -= 0.5 * nu[d] * fm[c];
                        flux_t[3 * ka + c] -= 0.5 * nu[d] * fp[c];
                    }
                }
            }
        }
        m_d[d] = m;
        free(W); free(s); free(am); free(ap);
    }

    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            long k = pidx(&u, i, j);
            long kxr = pidx(&u, i + 1, j), kyr = pidx(&u, i, j + 1);
            for (int c = 0; c < 3; ++c) {
                double first_x = fl[3 * k + c];
                double second_x = F[3 * kxr + c] - F[3 * k + c];
                double first_y = fl[3 * (np + k) + c];
                double second_y = G[3 * kyr + c] - G[3 * k + c];
                qout[c * ncell + (long)j * nx + i] =
                    u.q[3 * k + c] - nu[0] * first_x - nu[0] * second_x - nu[1] * first_y - nu[1] * second_y;
            }
        }
    free(F); free(G); free(fl);
    free(u.q); free(u.rho); free(u.K);
    return 0;
}
