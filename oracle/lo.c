/*
 * lo.c -- oracle: low-order QD systems, restriction between frequency grids, and the
 * grey LOQD + material energy balance Newton step.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  FP64, single threaded.
 *
 * One "level" (the fine grid, a coarse grid gamma, or the grey grid) is described by
 *   cell  : phi (f or f-bar), sig (sigma_E or its average), emis (sum of sigma_B B),
 *           Eold (E at t^{j-1})
 *   face  : sigR, etaR (eta-hat, multiplies E on the right of the face),
 *           etaL (eta-check, multiplies E on the left), Fold (F at t^{j-1})
 *   bound : phib0/phibX (factor at the boundary faces), C0 = C^- (x=0), CX = C^+ (x=X),
 *           Ein0, Fin0 (inflow moments at x=0), EinX, FinX (inflow moments at x=X).
 *
 * Discretisation (Sec. 5, eqs. mloqd-d and mloqd-d-gamma):
 *   balance over cell i:
 *     (dx_i/dt)(E_i - Eold_i) + F_{i+1/2} - F_{i-1/2} + dx_i a_i E_i = dx_i s_i,
 *     with a = c sig and s = 2 emis on the group levels;
 *   first moment over [x_i, x_{i+1}] (interior face):
 *     (dx_f/(c dt))(F - Fold) + c (phiR E_{i+1} - phiL E_i) + sigR dx_f F = 0,
 *     phiR = phi_{i+1} + etaR, phiL = phi_i + etaL, dx_f = (dx_i + dx_{i+1})/2.
 * Readings (paper silent or garbled):
 *   - the balance source carries the factor 2 of eq. mloqd-1 (its absence in the
 *     discrete balance is read as a typo), and dx_j there is dx_i;
 *   - at x=0 and x=X the first-moment equation is taken over the half cell next to
 *     the boundary (width dx/2) with the boundary-face factor, and the face energy is
 *     eliminated with the boundary condition eq. mloqd-bcs:
 *     F = c C (E_face - Ein) + Fin;
 *   - sigma_R on a boundary half face is the cell value.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

/* The two conditioning readings (|F| floor of the Rosseland weights, secant cut-off of the
 * Newton step between grey solves built on different grids), adjustable by
 * orc_set_readings so that a test can show that the converged state does not depend on
 * them. */
static double orc_flux_floor = 1e-6;
double orc_secant_cut = 1e-7;

void orc_set_readings(double flux_floor, double secant_cut)
{
    orc_flux_floor = flux_floor;
    orc_secant_cut = secant_cut;
}

/* Thomas algorithm (Gaussian elimination without pivoting for a tridiagonal matrix). */
void orc_tridiag(int n, const double *lo, const double *di, const double *up,
                 const double *rhs, double *x)
{
    double *cp = (double *)malloc(sizeof(double) * n);
    double *dp = (double *)malloc(sizeof(double) * n);
    cp[0] = up[0] / di[0];
    dp[0] = rhs[0] / di[0];
    for (int i = 1; i < n; ++i) {
        double m = di[i] - lo[i] * cp[i - 1];
        cp[i] = up[i] / m;
        dp[i] = (rhs[i] - lo[i] * dp[i - 1]) / m;
    }
    x[n - 1] = dp[n - 1];
    for (int i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
    free(cp);
    free(dp);
}

/* Face Rosseland opacity (Sec. 5): dx-weighted mean of the two cells at interior
 * faces, the cell value at the two boundary half faces.  Layout [G][nx+1]. */
void orc_fine_face_sigR(int nx, const double *h, int G, const double *sigR_cell,
                        double *sigR_face)
{
    for (int g = 0; g < G; ++g) {
        const double *sc = sigR_cell + (size_t)g * nx;
        double *sf = sigR_face + (size_t)g * (nx + 1);
        sf[0] = sc[0];
        sf[nx] = sc[nx - 1];
        for (int f = 1; f < nx; ++f)
            sf[f] = (sc[f - 1] * h[f - 1] + sc[f] * h[f]) / (h[f - 1] + h[f]);
    }
}

/* One low-order system (one group of one level): eliminate F face by face, solve the
 * tridiagonal system for the cell energies, then recover F and the boundary-face
 * energies.  Face f: F_f = GD_f + PL_f E_{f-1} - PR_f E_f (boundary faces lose the
 * term of the eliminated face energy). */
void orc_lo_solve(int nx, const double *h, double dt,
                  const double *a, const double *s, const double *Eold,
                  const double *phi, const double *sigR, const double *etaR,
                  const double *etaL, const double *Fold,
                  double phib0, double phibX, double C0, double CX,
                  double Ein0, double Fin0, double EinX, double FinX,
                  double *E, double *F, double *Eb0, double *EbX)
{
    const double c = orc_c();
    const double icdt = 1.0 / (c * dt);
    double *PL = (double *)malloc(sizeof(double) * (nx + 1));
    double *PR = (double *)malloc(sizeof(double) * (nx + 1));
    double *GD = (double *)malloc(sizeof(double) * (nx + 1));
    double *lo = (double *)malloc(sizeof(double) * nx);
    double *di = (double *)malloc(sizeof(double) * nx);
    double *up = (double *)malloc(sizeof(double) * nx);
    double *rh = (double *)malloc(sizeof(double) * nx);

    for (int f = 0; f <= nx; ++f) {
        double dx, phiL, phiR;
        double eR = etaR ? etaR[f] : 0.0, eL = etaL ? etaL[f] : 0.0;
        if (f == 0) {
            dx = 0.5 * h[0];
            phiL = phib0 + eL;
            phiR = phi[0] + eR;
        } else if (f == nx) {
            dx = 0.5 * h[nx - 1];
            phiL = phi[nx - 1] + eL;
            phiR = phibX + eR;
        } else {
            dx = 0.5 * (h[f - 1] + h[f]);
            phiL = phi[f - 1] + eL;
            phiR = phi[f] + eR;
        }
        double D = dx * (icdt + sigR[f]);
        double Gf = dx * Fold[f] * icdt;
        if (f == 0) {            /* E_face = Ein0 + (F - Fin0)/(c C0) */
            D -= phiL / C0;
            Gf += c * phiL * Ein0 - phiL * Fin0 / C0;
        } else if (f == nx) {    /* E_face = EinX + (F - FinX)/(c CX) */
            D += phiR / CX;
            Gf += -c * phiR * EinX + phiR * FinX / CX;
        }
        PL[f] = c * phiL / D;
        PR[f] = c * phiR / D;
        GD[f] = Gf / D;
    }
    for (int i = 0; i < nx; ++i) {
        di[i] = h[i] / dt + h[i] * a[i] + PL[i + 1] + PR[i];
        up[i] = (i < nx - 1) ? -PR[i + 1] : 0.0;
        lo[i] = (i > 0) ? -PL[i] : 0.0;
        rh[i] = h[i] * s[i] + h[i] * Eold[i] / dt - GD[i + 1] + GD[i];
    }
    orc_tridiag(nx, lo, di, up, rh, E);
    F[0] = GD[0] - PR[0] * E[0];
    for (int f = 1; f < nx; ++f) F[f] = GD[f] + PL[f] * E[f - 1] - PR[f] * E[f];
    F[nx] = GD[nx] + PL[nx] * E[nx - 1];
    *Eb0 = Ein0 + (F[0] - Fin0) / (c * C0);
    *EbX = EinX + (F[nx] - FinX) / (c * CX);
    free(PL); free(PR); free(GD); free(lo); free(di); free(up); free(rh);
}

/* weighted mean sum(v w)/sum(w) over the members of one coarse group; an all-zero
 * weight set falls back to the arithmetic mean (reading: paper silent). */
static double wmean(int n_from, const int *map, int P, const double *v, size_t sv,
                    const double *wt, size_t sw, int absw)
{
    double num = 0.0, den = 0.0, sum = 0.0;
    int cnt = 0;
    for (int p = 0; p < n_from; ++p) {
        if (map[p] != P) continue;
        double ww = wt[(size_t)p * sw];
        if (absw) ww = fabs(ww);
        num += v[(size_t)p * sv] * ww;
        den += ww;
        sum += v[(size_t)p * sv];
        ++cnt;
    }
    return (den != 0.0) ? num / den : sum / cnt;
}

/* Restriction of a level (n_from groups, coefficients + solution) onto a coarser one
 * (n_to groups, map[p] = coarse index of group p).  This is eq. coeff-gamma /
 * g-notation / eta-gamma (fine -> gamma, weights E^1, B^1, |F^1|) and eq. coeff-Gamma /
 * g2G-notation / eta-Gamma (gamma -> grey, weights E^gamma, |F^gamma|), in the discrete
 * form of eq. mloqd-d-gamma:
 *   phi_P  = <phi>_E,   sig_P = <sig>_E,   emis_P = sum emis (= sigma-bar_B B_P),
 *   sigR_P = <sigR>_|F| per face,
 *   xi_P   = dx_f sum_p (sigR_p - sigR_P) F_p  +  c sum_p (etaR_p E_p,right - etaL_p E_p,left),
 *   etaR_P = xi/(c sum E_p,right) if xi > 0,  etaL_P = -xi/(c sum E_p,left) if xi < 0.
 * Readings: xi carries dx_f (units of the sigma_R dx F term it replaces); the second sum
 * of xi keeps the compensation already applied on the finer level, so that the coarse
 * equations are exactly the sum of the finer ones at the finer solution; at the
 * boundary half faces the face energies of the finer solution are used; C-bar is
 * weighted by the outgoing boundary energies E_face - Ein, which makes the summed
 * boundary condition exact; Ein, Fin, Eold, Fold are sums.  The |F| weight of sigR_P is
 * |F_p| + 1e-6 c (E_p,left + E_p,right)/2: in a group near local equilibrium F_p is a
 * difference of nearly equal terms and carries only rounding noise, which the pure |F|
 * weight would turn into an arbitrary mean; the floor makes the mean well defined and
 * leaves it unchanged wherever the flux is physical.  Any sigR_P keeps the coarse
 * equations exact restrictions (xi compensates), so the converged state does not
 * depend on this choice. */
void orc_restrict(int nx, const double *h, int n_from, int n_to, const int *map,
                  const double *phi, const double *sig, const double *emis, const double *Eold,
                  const double *sigR, const double *etaR, const double *etaL, const double *Fold,
                  const double *phib0, const double *phibX, const double *C0, const double *CX,
                  const double *Ein0, const double *Fin0, const double *EinX, const double *FinX,
                  const double *E, const double *F, const double *Eb0, const double *EbX,
                  double *o_phi, double *o_sig, double *o_emis, double *o_Eold,
                  double *o_sigR, double *o_etaR, double *o_etaL, double *o_Fold,
                  double *o_phib0, double *o_phibX, double *o_C0, double *o_CX,
                  double *o_Ein0, double *o_Fin0, double *o_EinX, double *o_FinX,
                  double *o_Esum)
{
    const double c = orc_c();
    const int nf = nx + 1;
    /* coarse groups are independent (each sums its own fine groups in order) */
#pragma omp parallel for schedule(static)
    for (int P = 0; P < n_to; ++P) {
        for (int i = 0; i < nx; ++i) {
            size_t ci = (size_t)P * nx + i;
            o_phi[ci] = wmean(n_from, map, P, phi + i, nx, E + i, nx, 0);
            o_sig[ci] = wmean(n_from, map, P, sig + i, nx, E + i, nx, 0);
            double se = 0.0, sEo = 0.0, sE = 0.0;
            for (int p = 0; p < n_from; ++p) {
                if (map[p] != P) continue;
                se += emis[(size_t)p * nx + i];
                sEo += Eold[(size_t)p * nx + i];
                sE += E[(size_t)p * nx + i];
            }
            o_emis[ci] = se;
            o_Eold[ci] = sEo;
            o_Esum[ci] = sE;
        }
        for (int f = 0; f <= nx; ++f) {
            size_t cf = (size_t)P * nf + f;
            double dxf = (f == 0) ? 0.5 * h[0] : (f == nx) ? 0.5 * h[nx - 1]
                                               : 0.5 * (h[f - 1] + h[f]);
            double num = 0.0, den = 0.0, sum = 0.0;
            int cnt = 0;
            for (int p = 0; p < n_from; ++p) {
                if (map[p] != P) continue;
                size_t pf = (size_t)p * nf + f;
                double ER = (f == nx) ? EbX[p] : E[(size_t)p * nx + f];
                double EL = (f == 0) ? Eb0[p] : E[(size_t)p * nx + f - 1];
                double wgt = fabs(F[pf]) + orc_flux_floor * c * 0.5 * (EL + ER);
                num += sigR[pf] * wgt;
                den += wgt;
                sum += sigR[pf];
                ++cnt;
            }
            double sR = (den != 0.0) ? num / den : sum / cnt;
            double xi = 0.0, sER = 0.0, sEL = 0.0, sFo = 0.0;
            for (int p = 0; p < n_from; ++p) {
                if (map[p] != P) continue;
                size_t pf = (size_t)p * nf + f;
                double ER = (f == nx) ? EbX[p] : E[(size_t)p * nx + f];
                double EL = (f == 0) ? Eb0[p] : E[(size_t)p * nx + f - 1];
                xi += dxf * (sigR[pf] - sR) * F[pf];
                if (etaR) xi += c * etaR[pf] * ER;
                if (etaL) xi -= c * etaL[pf] * EL;
                sER += ER;
                sEL += EL;
                sFo += Fold[pf];
            }
            o_sigR[cf] = sR;
            o_etaR[cf] = (xi > 0.0 && sER != 0.0) ? xi / (c * sER) : 0.0;
            o_etaL[cf] = (xi < 0.0 && sEL != 0.0) ? -xi / (c * sEL) : 0.0;
            o_Fold[cf] = sFo;
        }
        o_phib0[P] = wmean(n_from, map, P, phib0, 1, Eb0, 1, 0);
        o_phibX[P] = wmean(n_from, map, P, phibX, 1, EbX, 1, 0);
        double *Eout0 = (double *)malloc(sizeof(double) * n_from);
        double *EoutX = (double *)malloc(sizeof(double) * n_from);
        double si0 = 0, sf0 = 0, siX = 0, sfX = 0;
        for (int p = 0; p < n_from; ++p) {
            Eout0[p] = Eb0[p] - Ein0[p];
            EoutX[p] = EbX[p] - EinX[p];
            if (map[p] != P) continue;
            si0 += Ein0[p]; sf0 += Fin0[p]; siX += EinX[p]; sfX += FinX[p];
        }
        o_C0[P] = wmean(n_from, map, P, C0, 1, Eout0, 1, 0);
        o_CX[P] = wmean(n_from, map, P, CX, 1, EoutX, 1, 0);
        o_Ein0[P] = si0; o_Fin0[P] = sf0; o_EinX[P] = siX; o_FinX[P] = sfX;
        free(Eout0);
        free(EoutX);
    }
}

/* Grey LOQD + MEB, one Newton step (Sec. 5, eq. eb-Gamma-d, eq. f-derivative-d).
 * MEB: cv (T - Told)/dt = c sig(T) E - Q(T).  Linearised about T* with E* the current
 * grey energy and the diagonal secant D sigma = (sig(T*) - sig_prev)/(T* - T_prev):
 *   Lambda = cv/dt + Q'(T*) - c D E*,      (reading: clamped to >= (cv/dt + Q')/2)
 *   T      = T* + [c sig* E - Q* - cv (T* - Told)/dt] / Lambda.
 * Substituting T into the grey balance gives an absorption term linear in E:
 *   R = w (c sig* E - Q*) + (1 - w) cv (T* - Told)/dt,   w = (cv/dt)/Lambda,
 * and cv (T - Told)/dt = R holds identically, so each grey solve conserves energy.
 * Readings: D = 0 on the first grey solve of a time step and where T* = T_prev.  The
 * previous grey solve may have been built on another grid (W and F cycles visit a
 * different grid before every grey solve; two-grid and V cycles build every one on the
 * fine grid); sigma-bar then also jumps with the grid while T barely moves, and the
 * quotient is taken only where |T* - T_prev| > secant_cut T* (the caller passes 1e-7 for
 * such a pair, 0 for two solves on the same grid): its relative rounding error is about
 * eps T / |T* - T_prev|, and below 1e-7 the cross-grid quotient would be rounding noise
 * amplified by up to 1e4 and more.  Returns nonzero if a temperature comes out
 * non-positive or non-finite. */
int orc_grey_newton(int nx, const double *h, double dt, double cv,
                    const double *Tstar, const double *Told, const double *Q,
                    const double *dQ, const double *Estar,
                    const double *sig, const double *sig_prev, const double *T_prev, int have_prev,
                    double secant_cut, const double *Eold,
                    const double *phi, const double *sigR, const double *etaR,
                    const double *etaL, const double *Fold,
                    double phib0, double phibX, double C0, double CX,
                    double Ein0, double Fin0, double EinX, double FinX,
                    double *T, double *E, double *F, double *Eb0, double *EbX)
{
    const double c = orc_c();
    double *a = (double *)malloc(sizeof(double) * nx);
    double *s = (double *)malloc(sizeof(double) * nx);
    double *Lam = (double *)malloc(sizeof(double) * nx);
    for (int i = 0; i < nx; ++i) {
        double D = 0.0;
        if (have_prev && Tstar[i] != T_prev[i] &&
            fabs(Tstar[i] - T_prev[i]) > secant_cut * Tstar[i])
            D = (sig[i] - sig_prev[i]) / (Tstar[i] - T_prev[i]);
        double base = cv / dt + dQ[i];
        double L = base - c * D * Estar[i];
        if (L < 0.5 * base) L = 0.5 * base;
        double w = (cv / dt) / L;
        Lam[i] = L;
        a[i] = w * c * sig[i];
        s[i] = w * Q[i] - (1.0 - w) * cv * (Tstar[i] - Told[i]) / dt;
    }
    orc_lo_solve(nx, h, dt, a, s, Eold, phi, sigR, etaR, etaL, Fold,
                 phib0, phibX, C0, CX, Ein0, Fin0, EinX, FinX, E, F, Eb0, EbX);
    int bad = 0;
    for (int i = 0; i < nx; ++i) {
        T[i] = Tstar[i] + (c * sig[i] * E[i] - Q[i] - cv * (Tstar[i] - Told[i]) / dt) / Lam[i];
        if (!(T[i] > 0.0) || !isfinite(T[i])) bad = 1;
    }
    free(a); free(s); free(Lam);
    return bad;
}

/* Cycle schedules S = {gamma_k, k=1..K} (Sec. 4, Fig. 1, Algorithm 3).
 *   V: S empty (two grids; every intermediate grid skipped);
 *   W: S = w(2) with w(Gamma-1) = [Gamma-1], w(g) = w(g+1) + [g] + w(g+1);
 *   F: S = [Gamma-1, Gamma-2, ..., 2].
 * Grid indices are 1-based as in the paper.  Returns K. */
static int wsched(int g, int Gamma, int *S, int k)
{
    if (g == Gamma - 1) { S[k++] = g; return k; }
    k = wsched(g + 1, Gamma, S, k);
    S[k++] = g;
    return wsched(g + 1, Gamma, S, k);
}

int orc_schedule(int type, int Gamma, int *S)
{
    if (Gamma <= 2 || type == 0) return 0;
    if (type == 1) return wsched(2, Gamma, S, 0);
    int K = 0;
    for (int g = Gamma - 1; g >= 2; --g) S[K++] = g;
    return K;
}
