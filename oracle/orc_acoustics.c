/*
 * Oracle (test infrastructure only): Riemann solver for linear acoustics,
 * Sec. 3 Eq. acoustics, with the coefficients written out:
 *     p_t + K div(u) = 0,     rho u_t + grad p = 0.
 * Along one direction the normal part is q = (p, u_n) with
 *     A = [[0, K], [1/rho, 0]],  eigenvalues -c, +c,  c = sqrt(K/rho),
 *     eigenvectors r1 = (-Z, 1), r2 = (Z, 1),  Z = rho c (impedance).
 * For cells with different (rho, K) the left-going wave uses the left cell's
 * (Z, c) and the right-going wave the right cell's (the textbook solver for
 * heterogeneous media); with equal cells it is the constant-coefficient one.
 * The transverse velocity is carried by no wave.
 */
#include <math.h>
#include "orc.h"

void orc_rp_acoustics(const double *ql, const double *qr,
                      double rho_l, double K_l, double rho_r, double K_r,
                      double W[3][3], double s[3], double amdq[3], double apdq[3])
{
    double c_l = sqrt(K_l / rho_l);
    double c_r = sqrt(K_r / rho_r);
    double Z_l = rho_l * c_l;
    double Z_r = rho_r * c_r;

    double dp = qr[0] - ql[0];
    double du = qr[1] - ql[1];

    /* Strengths: dq = alpha1 (-Z_l, 1) + alpha2 (Z_r, 1). */
    double alpha1 = (-dp + Z_r * du) / (Z_l + Z_r);
    double alpha2 = (dp + Z_l * du) / (Z_l + Z_r);

    W[0][0] = -alpha1 * Z_l;
    W[0][1] = alpha1;
    W[0][2] = 0.0;
    s[0] = -c_l;

    W[1][0] = alpha2 * Z_r;
    W[1][1] = alpha2;
    W[1][2] = 0.0;
    s[1] = c_r;

    /* A-dQ = sum_p min(s_p, 0) W_p ;  A+dQ = sum_p max(s_p, 0) W_p */
    for (int c = 0; c < 3; ++c) {
        amdq[c] = 0.0;
        apdq[c] = 0.0;
        for (int p = 0; p < 2; ++p) {
            double sm = s[p] < 0.0 ? s[p] : 0.0;
            double sp = s[p] > 0.0 ? s[p] : 0.0;
            amdq[c] += sm * W[p][c];
            apdq[c] += sp * W[p][c];
        }
    }
}
