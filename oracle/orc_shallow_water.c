/*
 * Oracle (test infrastructure only): Roe Riemann solver for the 2D shallow
 * water equations, Sec. 3 Eq. SW, with the Harten-Hyman entropy fix.
 *
 * Reduced state along a direction: q = (h, h u_n, h u_t).  Flux along that
 * direction: f(q) = (h u_n, h u_n^2 + g h^2 / 2, h u_n u_t).
 *
 * Roe averages:  h_bar = (h_l + h_r) / 2,
 *                u_hat = (sqrt(h_l) u_l + sqrt(h_r) u_r) / (sqrt(h_l) + sqrt(h_r)),
 *                v_hat likewise for the transverse velocity,
 *                c_hat = sqrt(g h_bar).
 * Speeds s = (u_hat - c_hat, u_hat, u_hat + c_hat); eigenvectors
 * r1 = (1, u_hat - c_hat, v_hat), r2 = (0, 0, 1), r3 = (1, u_hat + c_hat, v_hat);
 * strengths from dq = sum_p alpha_p r_p.
 *
 * Fluctuations: A-dQ = sum min(s_p,0) W_p, A+dQ = sum max(s_p,0) W_p, except
 * for a transonic rarefaction in the 1- or 3-family, which Harten-Hyman splits:
 *   1-wave: lam_l = u_l - sqrt(g h_l), middle state q_m = Q_l + W1,
 *           lam_m = u_m - sqrt(g h_m); if lam_l < 0 < lam_m then with
 *           beta = (lam_m - s1) / (lam_m - lam_l)
 *           A-dQ gets beta lam_l W1 and A+dQ gets (1 - beta) lam_m W1.
 *   3-wave: q_m = Q_r - W3, lam_m = u_m + sqrt(g h_m), lam_r = u_r + sqrt(g h_r);
 *           if lam_m < 0 < lam_r then beta = (lam_r - s3) / (lam_r - lam_m),
 *           A-dQ gets beta lam_m W3 and A+dQ gets (1 - beta) lam_r W3.
 * The shear (2-) wave is never fixed.  Either way A-dQ + A+dQ = sum s_p W_p.
 */
#include <math.h>
#include "orc.h"

void orc_rp_shallow_water(const double *ql, const double *qr, double g,
                          double W[3][3], double s[3], double amdq[3], double apdq[3])
{
    double h_l = ql[0], h_r = qr[0];
    double u_l = ql[1] / h_l, u_r = qr[1] / h_r;
    double v_l = ql[2] / h_l, v_r = qr[2] / h_r;
    double sqh_l = sqrt(h_l), sqh_r = sqrt(h_r);

    double h_bar = 0.5 * (h_l + h_r);
    double u_hat = (sqh_l * u_l + sqh_r * u_r) / (sqh_l + sqh_r);
    double v_hat = (sqh_l * v_l + sqh_r * v_r) / (sqh_l + sqh_r);
    double c_hat = sqrt(g * h_bar);

    double d0 = qr[0] - ql[0];
    double d1 = qr[1] - ql[1];
    double d2 = qr[2] - ql[2];

    double alpha1 = ((u_hat + c_hat) * d0 - d1) / (2.0 * c_hat);
    double alpha2 = d2 - v_hat * d0;
    double alpha3 = (d1 - (u_hat - c_hat) * d0) / (2.0 * c_hat);

    s[0] = u_hat - c_hat;
    s[1] = u_hat;
    s[2] = u_hat + c_hat;

    W[0][0] = alpha1;
    W[0][1] = alpha1 * (u_hat - c_hat);
    W[0][2] = alpha1 * v_hat;

    W[1][0] = 0.0;
    W[1][1] = 0.0;
    W[1][2] = alpha2;

    W[2][0] = alpha3;
    W[2][1] = alpha3 * (u_hat + c_hat);
    W[2][2] = alpha3 * v_hat;

    for (int c = 0; c < 3; ++c) {
        amdq[c] = 0.0;
        apdq[c] = 0.0;
    }

    /* 1-wave */
    {
        double lam_l = u_l - sqrt(g * h_l);
        double h_m = h_l + W[0][0];
        double hu_m = ql[1] + W[0][1];
        double lam_m = hu_m / h_m - sqrt(g * h_m);
        if (lam_l < 0.0 && 0.0 < lam_m) {
            double beta = (lam_m - s[0]) / (lam_m - lam_l);
            for (int c = 0; c < 3; ++c) {
                amdq[c] += beta * lam_l * W[0][c];
                apdq[c] += (1.0 - beta) * lam_m * W[0][c];
            }
        } else {
            for (int c = 0; c < 3; ++c) {
                if (s[0] < 0.0) amdq[c] += s[0] * W[0][c];
                else            apdq[c] += s[0] * W[0][c];
            }
        }
    }
    /* 2-wave (shear) */
    for (int c = 0; c < 3; ++c) {
        if (s[1] < 0.0) amdq[c] += s[1] * W[1][c];
        else            apdq[c] += s[1] * W[1][c];
    }
    /* 3-wave */
    {
        double lam_r = u_r + sqrt(g * h_r);
        double h_m = h_r - W[2][0];
        double hu_m = qr[1] - W[2][1];
        double lam_m = hu_m / h_m + sqrt(g * h_m);
        if (lam_m < 0.0 && 0.0 < lam_r) {
            double beta = (lam_r - s[2]) / (lam_r - lam_m);
            for (int c = 0; c < 3; ++c) {
                amdq[c] += beta * lam_m * W[2][c];
                apdq[c] += (1.0 - beta) * lam_r * W[2][c];
            }
        } else {
            for (int c = 0; c < 3; ++c) {
                if (s[2] < 0.0) amdq[c] += s[2] * W[2][c];
                else            apdq[c] += s[2] * W[2][c];
            }
        }
    }
}

/*
 * Shallow water over bathymetry B(x) (bottom elevation), the source term
 * (0, -g h B_x, -g h B_y) of Sec. 3's Clawpack base (source terms are added
 * to the hyperbolic part there) folded into the Riemann problem as f-waves,
 * the well-balanced form of the wave-propagation method:
 *
 *   psi  = (0, -g h_bar (B_r - B_l), 0)              source across the interface
 *   delta = f(Q_r) - f(Q_l) - psi = sum_p Z_p,        Z_p = beta_p r_p
 * with the Roe speeds and eigenvectors above.  The momentum component uses
 * g (h_r^2 - h_l^2) / 2 = g h_bar (h_r - h_l):
 *   delta_0 = (hu)_r - (hu)_l
 *   delta_1 = (hu u)_r - (hu u)_l + g h_bar ((h_r - h_l) + (B_r - B_l))
 *   delta_2 = (hu v)_r - (hu v)_l
 * so a lake at rest (u = v = 0, h + B constant) gives delta = 0 exactly.
 *   beta_1 = ((u_hat + c_hat) delta_0 - delta_1) / (2 c_hat)
 *   beta_2 = delta_2 - v_hat delta_0
 *   beta_3 = (delta_1 - (u_hat - c_hat) delta_0) / (2 c_hat)
 * Fluctuations: A-dQ = sum of Z_p with s_p < 0, A+dQ = sum of the others.
 * No entropy fix.  Returns the f-waves in W.
 */
void orc_rp_shallow_water_bathy(const double *ql, const double *qr, double B_l, double B_r,
                                double g, double W[3][3], double s[3], double amdq[3],
                                double apdq[3])
{
    double h_l = ql[0], h_r = qr[0];
    double u_l = ql[1] / h_l, u_r = qr[1] / h_r;
    double v_l = ql[2] / h_l, v_r = qr[2] / h_r;
    double sqh_l = sqrt(h_l), sqh_r = sqrt(h_r);

    double h_bar = 0.5 * (h_l + h_r);
    double u_hat = (sqh_l * u_l + sqh_r * u_r) / (sqh_l + sqh_r);
    double v_hat = (sqh_l * v_l + sqh_r * v_r) / (sqh_l + sqh_r);
    double c_hat = sqrt(g * h_bar);

    double delta0 = qr[1] - ql[1];
    double delta1 = (qr[1] * u_r - ql[1] * u_l) + g * h_bar * ((h_r - h_l) + (B_r - B_l));
    double delta2 = qr[1] * v_r - ql[1] * v_l;

    double beta1 = ((u_hat + c_hat) * delta0 - delta1) / (2.0 * c_hat);
    double beta2 = delta2 - v_hat * delta0;
    double beta3 = (delta1 - (u_hat - c_hat) * delta0) / (2.0 * c_hat);

    s[0] = u_hat - c_hat;
    s[1] = u_hat;
    s[2] = u_hat + c_hat;

    W[0][0] = beta1;
    W[0][1] = beta1 * (u_hat - c_hat);
    W[0][2] = beta1 * v_hat;
    W[1][0] = 0.0;
    W[1][1] = 0.0;
    W[1][2] = beta2;
    W[2][0] = beta3;
    W[2][1] = beta3 * (u_hat + c_hat);
    W[2][2] = beta3 * v_hat;

    for (int c = 0; c < 3; ++c) {
        amdq[c] = 0.0;
        apdq[c] = 0.0;
        for (int p = 0; p < 3; ++p) {
            if (s[p] < 0.0) amdq[c] += W[p][c];
            else            apdq[c] += W[p][c];
        }
    }
}

/*
 * Shallow water over bathymetry with wetting and drying.  The paper adds
 * source terms to the hyperbolic part (Sec. 3) and is silent on dry states;
 * this is the reading the library implements, written out plainly: the
 * hydrostatic reconstruction of Audusse, Bouchut, Bristeau, Klein and
 * Perthame (2004) around the HLLE solver (Harten-Lax-van Leer with
 * Einfeldt's speeds), in fluctuation form.
 *
 * A cell is dry when h <= dry_tol; its velocities count as zero.  At the
 * interface between cells l and r, with B* = max(B_l, B_r):
 *   reconstructed depths  h_l* = h_l + B_l - B*,  h_r* = h_r + B_r - B*,
 *                         each set to 0 when <= dry_tol (a dry side),
 *   reconstructed states  q_l* = h_l* (1, u_l, v_l),  q_r* = h_r* (1, u_r, v_r)
 * (a bed step higher than the other side's surface leaves no water on that
 * side: the interface acts as a wall, and at a lake at rest h_l* = h_r*).
 * The flat-bottom problem between q_l* and q_r* is solved by HLLE: a dry
 * side has zero gravity speed; with the Roe averages of the reconstructed states (h_bar = (h_l* +
 * h_r*)/2, sqrt(h*)-weighted u_hat, c_hat = sqrt(g h_bar)) the speeds are
 *   s1 = min(lam_l^-, u_hat - c_hat),  s3 = max(lam_r^+, u_hat + c_hat),
 *   lam_l^- = u_l - c_l* (l wet) or u_r - 2 c_r* (l dry),
 *   lam_r^+ = u_r + c_r* (r wet) or u_l + 2 c_l* (r dry),  c* = sqrt(g h*),
 * (u -/+ 2c is the front of a rarefaction into a dry bed), s2 = u_hat, and
 * the two waves split the jump so that W1 + W3 = q_r* - q_l* and
 * s1 W1 + s3 W3 = f(q_r*) - f(q_l*), f(q) = (hu, hu u + g h^2/2, hu v):
 *   W1 = (s3 dq* - df*) / (s3 - s1),  W3 = (df* - s1 dq*) / (s3 - s1),
 * with a zero middle (shear) wave; a-dq* = sum of s_p W_p over s_p < 0,
 * a+dq* = the others.  Both reconstructed sides dry: no waves, speeds 0.
 * The fluctuations of the cells themselves add what the reconstruction took
 * away (the hydrostatic pressure terms of the reconstruction cancel exactly):
 *   A-dQ = a-dq* + (h_l* - h_l) (u_l, u_l^2, u_l v_l),
 *   A+dQ = a+dq* + (h_r - h_r*) (u_r, u_r^2, u_r v_r),
 * so the mass fluxes telescope (mass is conserved), a lake at rest gives
 * zero, and the first-order update keeps h >= 0 under the CFL condition.
 *
 * The waves returned for the limiter and the second-order correction are W_p,
 * except where a reconstructed side is dry: there they are zero and the
 * correction is dropped (first order at the shoreline).  Speeds are
 * returned in every case (they enter the CFL maximum).
 */
void orc_rp_shallow_water_dry(const double *ql, const double *qr, double B_l, double B_r,
                              double g, double dry_tol, double W[3][3], double s[3],
                              double amdq[3], double apdq[3])
{
    for (int p = 0; p < 3; ++p) {
        s[p] = 0.0;
        amdq[p] = 0.0;
        apdq[p] = 0.0;
        for (int c = 0; c < 3; ++c) W[p][c] = 0.0;
    }
    double h_l = ql[0], h_r = qr[0];
    double u_l = h_l > dry_tol ? ql[1] / h_l : 0.0, v_l = h_l > dry_tol ? ql[2] / h_l : 0.0;
    double u_r = h_r > dry_tol ? qr[1] / h_r : 0.0, v_r = h_r > dry_tol ? qr[2] / h_r : 0.0;

    /* hydrostatic reconstruction; a reconstructed depth <= dry_tol is a dry
     * side and counts as no water at all */
    double Bs = B_l > B_r ? B_l : B_r;
    double hl = h_l + B_l - Bs, hr = h_r + B_r - Bs;
    if (!(hl > dry_tol)) hl = 0.0;
    if (!(hr > dry_tol)) hr = 0.0;

    /* what the reconstruction removed from each cell's flux */
    double cut_l[3] = {u_l, u_l * u_l, u_l * v_l}, cut_r[3] = {u_r, u_r * u_r, u_r * v_r};
    for (int c = 0; c < 3; ++c) {
        amdq[c] = (hl - h_l) * cut_l[c];
        apdq[c] = (h_r - hr) * cut_r[c];
    }

    int wet_l = hl > 0.0, wet_r = hr > 0.0;
    if (!wet_l && !wet_r) return;

    double sqh_l = wet_l ? sqrt(hl) : 0.0, sqh_r = wet_r ? sqrt(hr) : 0.0;
    double c_l = wet_l ? sqrt(g * hl) : 0.0, c_r = wet_r ? sqrt(g * hr) : 0.0;
    double h_bar = 0.5 * (hl + hr);
    double u_hat = (sqh_l * u_l + sqh_r * u_r) / (sqh_l + sqh_r);
    double c_hat = sqrt(g * h_bar);
    double lam_lm = wet_l ? u_l - c_l : u_r - 2.0 * c_r;
    double lam_rp = wet_r ? u_r + c_r : u_l + 2.0 * c_l;
    double s1 = u_hat - c_hat < lam_lm ? u_hat - c_hat : lam_lm;
    double s3 = u_hat + c_hat > lam_rp ? u_hat + c_hat : lam_rp;

    /* reconstructed states (a dry side is all zero) and their fluxes */
    double qsl[3] = {hl, hl * u_l, hl * v_l};
    double qsr[3] = {hr, hr * u_r, hr * v_r};
    double fl[3] = {qsl[1], qsl[1] * u_l + 0.5 * g * hl * hl, qsl[1] * v_l};
    double fr[3] = {qsr[1], qsr[1] * u_r + 0.5 * g * hr * hr, qsr[1] * v_r};

    s[0] = s1;
    s[1] = u_hat;
    s[2] = s3;
    for (int c = 0; c < 3; ++c) {
        double dq = qsr[c] - qsl[c], df = fr[c] - fl[c];
        W[0][c] = (s3 * dq - df) / (s3 - s1);
        W[2][c] = (df - s1 * dq) / (s3 - s1);
    }
    for (int c = 0; c < 3; ++c)
        for (int p = 0; p < 3; ++p) {
            if (s[p] < 0.0) amdq[c] += s[p] * W[p][c];
            else            apdq[c] += s[p] * W[p][c];
        }

    /* first order at the shoreline: no waves for the correction */
    if (!wet_l || !wet_r)
        for (int p = 0; p < 3; ++p)
            for (int c = 0; c < 3; ++c) W[p][c] = 0.0;
}
