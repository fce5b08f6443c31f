/*
 * physics.c -- oracle: constants, angular quadrature and group physics.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  FP64, single threaded.
 *
 * Paper passages followed:
 *   Sec. 2   Planck function multiplied by 2 pi, group integrals B_g, the group
 *            opacities sigma_B,g and sigma_E,g (Planck-weighted means).
 *   Sec. 3.1 Rosseland group opacity sigma_R,g (dB/dT-weighted harmonic mean).
 *   Sec. 6   Fleck-Cummings opacity sigma(nu,T) = 27/nu^3 (1 - e^{-nu/T}), and the
 *            double S_N Gauss-Legendre angular quadrature.
 * Readings (the paper is silent):
 *   - units cm, sh, keV, GJ; c = 299.792458 cm/sh; aR = 0.01372 GJ cm^-3 keV^-4.
 *   - T_r = T, hence sigma_E,g = sigma_B,g (Algorithm 3 updates the transport
 *     operator from T alone); with the T_r option (orc_set_tr_mode) T_r = (E/aR)^{1/4} from
 *     the latest grey energy and sigma_E,g, sigma_R,g follow Sec. 2 / Sec. 3.1 at (T, T_r).
 *   - the 2-pi-multiplied Planck function is B(nu,T) = CB nu^3/(e^{nu/T}-1) with
 *     CB = 15 aR c / (2 pi^4), so that sum_g B_g = aR c T^4 / 2.
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

static const double PI = 3.14159265358979323846;

double orc_c(void) { return 299.792458; }
double orc_aR(void) { return 0.01372; }
double orc_CB(void) { return 15.0 * orc_aR() * orc_c() / (2.0 * PI * PI * PI * PI); }

/* ---------------------------------------------------------------------------
 * Gauss-Legendre nodes: Newton iteration on P_n(x), evaluated by the three-term
 * Legendre recurrence (Abramowitz & Stegun 8.5.3, 25.4.29).
 * ------------------------------------------------------------------------- */
void orc_gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            if (n == 1) { p0 = 1.0; p1 = z; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        /* recompute derivative at the converged node */
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = pk;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[n - 1 - i] = z;   /* ascending */
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* Double S_N Gauss-Legendre (Sec. 6): an N-point Gauss rule on each half range.
 * Directions m < N have mu in (0,1) ascending; m >= N mirror them (mu < 0).
 * Weights sum to 1 on each half range, 2 in total. */
void orc_double_gl(int N, double *mu, double *w)
{
    double *x = (double *)malloc(sizeof(double) * N);
    double *wx = (double *)malloc(sizeof(double) * N);
    orc_gauss_legendre(N, x, wx);
    for (int k = 0; k < N; ++k) {
        mu[k] = 0.5 * (1.0 + x[k]);
        w[k] = 0.5 * wx[k];
        mu[N + k] = -mu[k];
        w[N + k] = w[k];
    }
    free(x);
    free(wx);
}

/* ---------------------------------------------------------------------------
 * Planck integral P(x) = int_0^x t^3/(e^t - 1) dt  (Debye function, A&S 27.1).
 *   x < 2 : t/(e^t-1) = sum_n B_n t^n / n!  =>  P(x) = sum_n (B_n/n!) x^{n+3}/(n+3),
 *           with B_0 = 1, B_1 = -1/2, B_{2k}/(2k)! = (-1)^{k+1} 2 zeta(2k)/(2 pi)^{2k}.
 *   x >= 2: P(x) = pi^4/15 - sum_{k>=1} e^{-kx}(x^3/k + 3x^2/k^2 + 6x/k^3 + 6/k^4).
 * ------------------------------------------------------------------------- */
#define NBER 31
static double ber_coef[2 * NBER + 2];   /* B_n / n!, n = 0 .. 2*NBER */
static int ber_ready = 0;

static double zeta_even(int s)
{
    /* direct sum plus the Euler-Maclaurin tail; s >= 4 even */
    const int J = 200;
    double sum = 0.0;
    for (int j = J - 1; j >= 1; --j) sum += pow((double)j, -s);
    double Jd = (double)J;
    sum += pow(Jd, 1.0 - s) / (s - 1.0) + 0.5 * pow(Jd, -s) + s * pow(Jd, -s - 1.0) / 12.0
         - s * (s + 1.0) * (s + 2.0) * pow(Jd, -s - 3.0) / 720.0;
    return sum;
}

static void ber_init(void)
{
    if (ber_ready) return;
    for (int n = 0; n < 2 * NBER + 2; ++n) ber_coef[n] = 0.0;
    ber_coef[0] = 1.0;
    ber_coef[1] = -0.5;
    for (int k = 1; k <= NBER; ++k) {
        double z = (k == 1) ? PI * PI / 6.0 : zeta_even(2 * k);
        double v = 2.0 * z / pow(2.0 * PI, 2 * k);
        ber_coef[2 * k] = (k % 2 == 1) ? v : -v;
    }
    ber_ready = 1;
}

static double planck_series(double x)   /* x < 2 */
{
    ber_init();
    double sum = 0.0;
    for (int n = 2 * NBER; n >= 0; --n) sum += ber_coef[n] * pow(x, n + 3) / (n + 3.0);
    return sum;
}

/* e^{xref} * sum_k e^{-k x} (x^3/k + 3x^2/k^2 + 6x/k^3 + 6/k^4), for x >= 2, x >= xref */
static double planck_tail_scaled(double x, double xref)
{
    if (isinf(x)) return 0.0;
    double sum = 0.0;
    for (int k = 1; k < 200; ++k) {
        double kk = (double)k;
        double e = exp(xref - kk * x);
        double term = e * (x * x * x / kk + 3.0 * x * x / (kk * kk) + 6.0 * x / (kk * kk * kk)
                           + 6.0 / (kk * kk * kk * kk));
        sum += term;
        if (term <= 1e-19 * sum) break;
    }
    return sum;
}

double orc_planck_P(double x)
{
    const double P_inf = PI * PI * PI * PI / 15.0;
    if (isinf(x)) return P_inf;
    if (x < 2.0) return planck_series(x);
    return P_inf - planck_tail_scaled(x, 0.0);
}

/* e^{xa} (P(xb) - P(xa)), 0 <= xa < xb <= inf, without cancellation against pi^4/15 */
static double planck_dP_scaled(double xa, double xb)
{
    const double P_inf = PI * PI * PI * PI / 15.0;
    if (xa >= 2.0) return planck_tail_scaled(xa, xa) - planck_tail_scaled(xb, xa);
    double Pa = planck_series(xa);
    double Pb = (xb < 2.0) ? planck_series(xb) : P_inf - planck_tail_scaled(xb, 0.0);
    return exp(xa) * (Pb - Pa);
}

/* x^4 e^{xref}/(e^x - 1) = x^4 e^{xref - x}/(1 - e^{-x});  0 at x = 0 and x = inf */
static double rosseland_edge(double x, double xref)
{
    if (x == 0.0 || isinf(x)) return 0.0;
    return x * x * x * x * exp(xref - x) / (-expm1(-x));
}

/* e^{xa} * int_{xa}^{xb} x^7 e^{2x}/(e^x-1)^3 dx by composite 8-point Gauss-Legendre on
 * panels of width <= 2 over [xa, min(xb, xa + 64)].  The integrand, scaled, is
 * x^7 e^{xa-x} / (1 - e^{-x})^3; the part beyond xa+64 is below 1e-18 relative. */
double orc_rosseland_D_quad(double xa, double xb)
{
    static double gx[8], gw[8];
    static int ready = 0;
    if (!ready) { orc_gauss_legendre(8, gx, gw); ready = 1; }
    double hi = xb < xa + 64.0 ? xb : xa + 64.0;
    int np = (int)ceil((hi - xa) / 2.0);
    if (np < 1) np = 1;
    double width = (hi - xa) / np;
    double sum = 0.0;
    for (int p = 0; p < np; ++p) {
        double a = xa + p * width;
        for (int q = 0; q < 8; ++q) {
            double x = a + 0.5 * width * (1.0 + gx[q]);
            double om = -expm1(-x);
            double v = pow(x, 7) * exp(xa - x) / (om * om * om);
            sum += 0.5 * width * gw[q] * v;
        }
    }
    return sum;
}

/* ---------------------------------------------------------------------------
 * Group physics at temperature T (Sec. 2, Sec. 3.1, Sec. 6).  With x = nu/T:
 *   B_g      = CB T^4 (P(x_{g+1}) - P(x_g))
 *   e_g      = int sigma B dnu = s 27 CB T (e^{-x_g} - e^{-x_{g+1}})   [sigma B = 27 s CB e^{-nu/T}]
 *   sigma_B  = e_g / B_g   (= sigma_E under T_r = T)
 *   sigma_R  = int dB/dT / int (1/sigma) dB/dT = s 27 N_g / (T^3 D_g),
 *     N_g = [-x^4/(e^x-1)] + 4 (P(x_{g+1}) - P(x_g))     (by parts, closed form)
 *     D_g = int x^7 e^{2x}/(e^x-1)^3 dx                   (quadrature)
 * Every ratio is taken between quantities scaled by e^{x_g} so nothing underflows
 * in cold cells; the limit of each ratio is the opacity at the lower group edge.
 * ------------------------------------------------------------------------- */
void orc_group_physics(int G, const double *edges, double T, double s,
                       double *B, double *sigB, double *emis, double *sigR)
{
    const double CB = orc_CB();
    const double T3 = T * T * T;
    for (int g = 0; g < G; ++g) {
        double xa = edges[g] / T;
        double xb = isinf(edges[g + 1]) ? INFINITY : edges[g + 1] / T;
        double dPs = planck_dP_scaled(xa, xb);
        double ea = exp(-xa);
        double one_m = isinf(xb) ? 1.0 : -expm1(-(xb - xa));
        if (B) B[g] = CB * T3 * T * ea * dPs;
        if (emis) emis[g] = s * 27.0 * CB * T * ea * one_m;
        if (sigB) sigB[g] = s * 27.0 * one_m / (T3 * dPs);
        if (sigR) {
            double Ns = rosseland_edge(xa, xa) - rosseland_edge(xb, xa) + 4.0 * dPs;
            double Ds = orc_rosseland_D_quad(xa, xb);
            sigR[g] = s * 27.0 * Ns / (T3 * Ds);
        }
    }
}

/* ---------------------------------------------------------------------------
 * Group opacities at a radiation temperature T_r != T (Sec. 2, sigma_E,g(T, T_r); Sec. 3.1,
 * sigma_R,g(T, T_r)).  With x = nu/T_r and rho = T_r/T (so nu/T = rho x):
 *   sigma_E = int sigma(nu,T) B(nu,T_r) / int B(nu,T_r)
 *           = s 27 J_g / (T_r^3 (P(x_{g+1}) - P(x_g))),  J_g = int (1 - e^{-rho x})/(e^x - 1) dx
 *   sigma_R = int dB/dT|_{T_r} / int (1/sigma(nu,T)) dB/dT|_{T_r}
 *           = s 27 N_g / (T_r^3 D_g),  N_g as at T (at x = nu/T_r),
 *             D_g = int x^7 e^x / ((1 - e^{-rho x}) (e^x - 1)^2) dx
 * J_g and D_g by composite 8-point Gauss-Legendre over [x_g, min(x_{g+1}, x_g + 64)] on
 * panels of width <= 2 (for rho > 1 graded near x = 0, where 1 - e^{-rho x} changes on the
 * scale 1/rho; the last panel takes the remainder up to 1.5 widths), both scaled by e^{x_g}
 * like the T_r = T forms (at rho = 1 the integrands are e^{-x} and x^7 e^{2x}/(e^x - 1)^3).
 * ------------------------------------------------------------------------- */
void orc_group_opacity_tr(int G, const double *edges, double T, double Tr, double s,
                          double *sigE, double *sigR)
{
    static double gx[8], gw[8];
    static int ready = 0;
    if (!ready) { orc_gauss_legendre(8, gx, gw); ready = 1; }
    const double rho = Tr / T;
    const double Tr3 = Tr * Tr * Tr;
    for (int g = 0; g < G; ++g) {
        double xa = edges[g] / Tr;
        double xb = isinf(edges[g + 1]) ? INFINITY : edges[g + 1] / Tr;
        double hi = xb < xa + 64.0 ? xb : xa + 64.0;
        double Js = 0.0, Ds = 0.0;
        /* panels: width 2, except that for rho > 1 the factor 1 - e^{-rho x} varies on the
         * scale 1/rho near x = 0: there the width is max(1/rho, a/2) at the panel start a */
        double a = xa;
        while (a < hi) {
            double wmax = (rho > 1.0) ? fmin(2.0, fmax(1.0 / rho, 0.5 * a)) : 2.0;
            double b = (hi - a <= 1.5 * wmax) ? hi : a + wmax;
            double width = b - a;
            for (int q = 0; q < 8; ++q) {
                double x = a + 0.5 * width * (1.0 + gx[q]);
                double e = exp(xa - x);                 /* e^{xa} e^{-x}   */
                double om = -expm1(-x);                  /* 1 - e^{-x}      */
                double orh = -expm1(-rho * x);           /* 1 - e^{-rho x}  */
                double wq = 0.5 * width * gw[q];
                Js += wq * e * orh / om;                 /* e^{xa} (1-e^{-rho x})/(e^x-1) */
                Ds += wq * pow(x, 7) * e / (orh * om * om);
            }
            a = b;
        }
        double dPs = planck_dP_scaled(xa, xb);
        sigE[g] = s * 27.0 * Js / (Tr3 * dPs);
        double Ns = rosseland_edge(xa, xa) - rosseland_edge(xb, xa) + 4.0 * dPs;
        sigR[g] = s * 27.0 * Ns / (Tr3 * Ds);
    }
}

/* Q(T) = 2 sum_g e_g(T): the emission term of eq. eb-group / eb-Gamma. */
double orc_emission_total(int G, const double *edges, double T, double s)
{
    const double CB = orc_CB();
    double sum = 0.0;
    for (int g = 0; g < G; ++g) {
        double ea = exp(-edges[g] / T);
        double eb = isinf(edges[g + 1]) ? 0.0 : exp(-edges[g + 1] / T);
        sum += s * 27.0 * CB * T * (ea - eb);
    }
    return 2.0 * sum;
}

/* dQ/dT: d/dT [T e^{-nu/T}] = (1 + nu/T) e^{-nu/T} */
double orc_emission_deriv(int G, const double *edges, double T, double s)
{
    const double CB = orc_CB();
    double sum = 0.0;
    for (int g = 0; g < G; ++g) {
        double xa = edges[g] / T;
        double da = (1.0 + xa) * exp(-xa);
        double db = 0.0;
        if (!isinf(edges[g + 1])) {
            double xb = edges[g + 1] / T;
            db = (1.0 + xb) * exp(-xb);
        }
        sum += s * 27.0 * CB * (da - db);
    }
    return 2.0 * sum;
}
