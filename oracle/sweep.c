/*
 * sweep.c -- oracle: high-order multigroup transport sweep and its QD factors.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  FP64, single threaded.
 *
 * Follows:
 *   eq. rt / rt-bc   multigroup RT equation  (1/c) dI_g/dt + mu dI_g/dx + sigma_E,g I_g
 *                    = sigma_B,g B_g, inflow I_g^+ at x=0 (mu>0), I_g^- at x=X (mu<0);
 *   Sec. 5           implicit Euler in time (opacities and emission at the new level),
 *                    simple corner balance in space (1D slab: two corners per cell,
 *                    the cell-centre value is the corner average, the cell-edge
 *                    values are upwinded corner values);
 *   eq. f_g, c_g     the QD factor f_g = int mu^2 I / int I and the boundary factors
 *                    C_g^- (x=0, mu<0 half range), C_g^+ (x=X, mu>0 half range).
 * With sigma_t = sigma_E,g + 1/(c dt) and corner sources S = e_g + I^{j-1}/(c dt),
 * for mu > 0 in a cell of width h with inflow psi_in:
 *   (|mu|/2 + sigma_t h/2) psi_L + (|mu|/2) psi_R = (h/2) S_L + |mu| psi_in
 *  -(|mu|/2) psi_L + (|mu|/2 + sigma_t h/2) psi_R = (h/2) S_R,      outflow psi_R;
 * mu < 0 mirrors it (inflow enters the right corner, outflow psi_L).
 * Readings (paper silent): cell moments use the cell average (psi_L+psi_R)/2; the
 * face factors at x=0 and x=X use the face intensities (inflow from the boundary
 * condition, outflow from the sweep); zero denominators give the isotropic values
 * f = 1/3, C^- = -1/2, C^+ = +1/2.
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

#define IIDX(m, i, c, g) ((((size_t)(m) * nx + (i)) * 2 + (c)) * G + (g))

void orc_sweep(int nx, const double *h, int M, const double *mu, const double *w,
               int G, const double *sigE, const double *emis, double inv_cdt,
               const double *I_old, const double *Iin_left, const double *Iin_right,
               double *I_new, double *f, double *fb0, double *fbX, double *C0, double *CX)
{
    /* groups are independent: with OpenMP each thread sweeps whole groups with its own
     * scratch, in the same order as one thread (the results do not depend on the count) */
#pragma omp parallel
    {
    double *A0 = (double *)calloc((size_t)nx, sizeof(double));   /* sum_m w psi_bar      */
    double *A2 = (double *)calloc((size_t)nx, sizeof(double));   /* sum_m w mu^2 psi_bar */
    double *out = (double *)malloc(sizeof(double) * M);         /* outflow face values  */

#pragma omp for schedule(static)
    for (int g = 0; g < G; ++g) {
        for (int i = 0; i < nx; ++i) { A0[i] = 0.0; A2[i] = 0.0; }
        for (int m = 0; m < M; ++m) {
            double am = fabs(mu[m]);
            double b = 0.5 * am;
            if (mu[m] > 0.0) {
                double psi_in = Iin_left[g];
                for (int i = 0; i < nx; ++i) {
                    double sigt = sigE[(size_t)g * nx + i] + inv_cdt;
                    double a = b + 0.5 * sigt * h[i];
                    double SL = emis[(size_t)g * nx + i] + inv_cdt * I_old[IIDX(m, i, 0, g)];
                    double SR = emis[(size_t)g * nx + i] + inv_cdt * I_old[IIDX(m, i, 1, g)];
                    double rL = 0.5 * h[i] * SL + am * psi_in;
                    double rR = 0.5 * h[i] * SR;
                    double det = a * a + b * b;
                    double psiL = (a * rL - b * rR) / det;
                    double psiR = (a * rR + b * rL) / det;
                    I_new[IIDX(m, i, 0, g)] = psiL;
                    I_new[IIDX(m, i, 1, g)] = psiR;
                    double pbar = 0.5 * (psiL + psiR);
                    A0[i] += w[m] * pbar;
                    A2[i] += w[m] * mu[m] * mu[m] * pbar;
                    psi_in = psiR;
                }
                out[m] = psi_in;   /* leaves through x = X */
            } else {
                double psi_in = Iin_right[g];
                for (int i = nx - 1; i >= 0; --i) {
                    double sigt = sigE[(size_t)g * nx + i] + inv_cdt;
                    double a = b + 0.5 * sigt * h[i];
                    double SL = emis[(size_t)g * nx + i] + inv_cdt * I_old[IIDX(m, i, 0, g)];
                    double SR = emis[(size_t)g * nx + i] + inv_cdt * I_old[IIDX(m, i, 1, g)];
                    double rR = 0.5 * h[i] * SR + am * psi_in;
                    double rL = 0.5 * h[i] * SL;
                    double det = a * a + b * b;
                    double psiR = (a * rR - b * rL) / det;
                    double psiL = (a * rL + b * rR) / det;
                    I_new[IIDX(m, i, 0, g)] = psiL;
                    I_new[IIDX(m, i, 1, g)] = psiR;
                    double pbar = 0.5 * (psiL + psiR);
                    A0[i] += w[m] * pbar;
                    A2[i] += w[m] * mu[m] * mu[m] * pbar;
                    psi_in = psiL;
                }
                out[m] = psi_in;   /* leaves through x = 0 */
            }
        }
        for (int i = 0; i < nx; ++i)
            f[(size_t)g * nx + i] = (A0[i] != 0.0) ? A2[i] / A0[i] : 1.0 / 3.0;

        /* face intensities at x = 0: inflow for mu>0, outflow for mu<0 */
        double s0 = 0.0, s2 = 0.0, hm0 = 0.0, hm1 = 0.0;
        for (int m = 0; m < M; ++m) {
            double psi = (mu[m] > 0.0) ? Iin_left[g] : out[m];
            s0 += w[m] * psi;
            s2 += w[m] * mu[m] * mu[m] * psi;
            if (mu[m] < 0.0) { hm0 += w[m] * psi; hm1 += w[m] * mu[m] * psi; }
        }
        fb0[g] = (s0 != 0.0) ? s2 / s0 : 1.0 / 3.0;
        C0[g] = (hm0 != 0.0) ? hm1 / hm0 : -0.5;

        /* face intensities at x = X: outflow for mu>0, inflow for mu<0 */
        s0 = s2 = hm0 = hm1 = 0.0;
        for (int m = 0; m < M; ++m) {
            double psi = (mu[m] > 0.0) ? out[m] : Iin_right[g];
            s0 += w[m] * psi;
            s2 += w[m] * mu[m] * mu[m] * psi;
            if (mu[m] > 0.0) { hm0 += w[m] * psi; hm1 += w[m] * mu[m] * psi; }
        }
        fbX[g] = (s0 != 0.0) ? s2 / s0 : 1.0 / 3.0;
        CX[g] = (hm0 != 0.0) ? hm1 / hm0 : 0.5;
    }
    free(A0);
    free(A2);
    free(out);
    }
}
