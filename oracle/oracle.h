/*
 * oracle.h -- plain, slow, FP64 CPU oracle of the MLQD method with multigrid in
 * photon frequency (Anistratov, "Nonlinear iterative projection methods with
 * multigrid in photon frequency for thermal radiative transfer", arXiv 2011.05427).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header, table or
 * constant generator with the CUDA library, and the CUDA library never calls it.
 *
 * Everything is double precision, written in the order and
 * notation of the paper (loops over independent groups or cells may run on several
 * threads with OpenMP, with the same results).  Each function names the section /
 * equation it follows.
 * Units: cm, sh (1e-8 s), keV, GJ ("jerk").
 *
 * Array layouts (interface formats, shared with the tests only):
 *   cell arrays      [G][nx]          (group-major, cell fastest)
 *   face arrays      [G][nx+1]        face f sits at x_{f-1/2}; f=0 is x=0, f=nx is x=X
 *   intensity        [M][nx][2][G]    direction, cell, corner (0=left,1=right), group
 *   directions       m < N: mu > 0;   m >= N: mu_m = -mu_{m-N}
 *
 * Parity status of each part is listed in the README block of oracle.py.
 */
#ifndef TRT_ORACLE_H
#define TRT_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- constants (units cm, sh, keV, GJ; paper silent -> standard values) ---- */
double orc_c(void);        /* speed of light  299.792458 cm/sh               */
double orc_aR(void);       /* radiation constant 0.01372 GJ/(cm^3 keV^4)      */
double orc_CB(void);       /* 15 aR c / (2 pi^4): B(nu,T) = CB nu^3/(e^{nu/T}-1) */

/* ---- quadrature (Sec. 6: double S_N Gauss-Legendre) ---- */
void orc_gauss_legendre(int n, double *x, double *w);     /* nodes/weights on [-1,1] */
void orc_double_gl(int N, double *mu, double *w);         /* M=2N directions, sum w = 2 */

/* ---- group physics (Sec. 2, Sec. 3.1, Sec. 6 opacity) ---- */
double orc_planck_P(double x);                             /* int_0^x t^3/(e^t-1) dt */
double orc_rosseland_D_quad(double xa, double xb);         /* int x^7 e^{2x}/(e^x-1)^3, scaled by e^{xa} */
void orc_group_physics(int G, const double *edges, double T, double s,
                       double *B, double *sigB, double *emis, double *sigR);
/* sigma_E,g(T, T_r) and sigma_R,g(T, T_r) (Sec. 2, Sec. 3.1) for a radiation temperature T_r */
void orc_group_opacity_tr(int G, const double *edges, double T, double Tr, double s,
                          double *sigE, double *sigR);
double orc_emission_total(int G, const double *edges, double T, double s);   /* Q = 2 sum_g e_g */
double orc_emission_deriv(int G, const double *edges, double T, double s);   /* dQ/dT          */

/* ---- high-order sweep (eq. rt with implicit Euler, simple corner balance) ---- */
void orc_sweep(int nx, const double *h, int M, const double *mu, const double *w,
               int G, const double *sigE, const double *emis, double inv_cdt,
               const double *I_old, const double *Iin_left, const double *Iin_right,
               double *I_new, double *f, double *fb0, double *fbX, double *C0, double *CX);

/* ---- one low-order QD system (eq. mloqd-d / mloqd-d-gamma, generic level) ---- */
void orc_lo_solve(int nx, const double *h, double dt,
                  const double *a, const double *s, const double *Eold,
                  const double *phi, const double *sigR, const double *etaR,
                  const double *etaL, const double *Fold,
                  double phib0, double phibX, double C0, double CX,
                  double Ein0, double Fin0, double EinX, double FinX,
                  double *E, double *F, double *Eb0, double *EbX);

void orc_tridiag(int n, const double *lo, const double *di, const double *up,
                 const double *rhs, double *x);              /* Thomas, no pivoting */
void orc_fine_face_sigR(int nx, const double *h, int G, const double *sigR_cell,
                        double *sigR_face);                  /* Sec. 5 face average  */

/* ---- restriction of a level onto a coarser one (eqs. coeff-gamma, eta-gamma,
 *      mloqd-d-gamma, coeff-Gamma, eta-Gamma) ---- */
void orc_restrict(int nx, const double *h, int n_from, int n_to, const int *map,
                  /* level coefficients (etaR/etaL may be NULL: zero, as on the fine grid) */
                  const double *phi, const double *sig, const double *emis, const double *Eold,
                  const double *sigR, const double *etaR, const double *etaL, const double *Fold,
                  const double *phib0, const double *phibX, const double *C0, const double *CX,
                  const double *Ein0, const double *Fin0, const double *EinX, const double *FinX,
                  /* level solution used as weights */
                  const double *E, const double *F, const double *Eb0, const double *EbX,
                  /* coarse coefficients (out) */
                  double *o_phi, double *o_sig, double *o_emis, double *o_Eold,
                  double *o_sigR, double *o_etaR, double *o_etaL, double *o_Fold,
                  double *o_phib0, double *o_phibX, double *o_C0, double *o_CX,
                  double *o_Ein0, double *o_Fin0, double *o_EinX, double *o_FinX,
                  double *o_Esum);

/* ---- grey LOQD + MEB, one Newton step (eq. eb-Gamma-d, f-derivative-d) ---- */
int orc_grey_newton(int nx, const double *h, double dt, double cv,
                    const double *Tstar, const double *Told, const double *Q,
                    const double *dQ, const double *Estar,
                    const double *sig, const double *sig_prev, const double *T_prev, int have_prev,
                    double secant_cut, const double *Eold,
                    const double *phi, const double *sigR, const double *etaR,
                    const double *etaL, const double *Fold,
                    double phib0, double phibX, double C0, double CX,
                    double Ein0, double Fin0, double EinX, double FinX,
                    double *T, double *E, double *F, double *Eb0, double *EbX);

/* The |F| floor of the Rosseland weights (default 1e-6: weight |F_p| + floor c E-bar_p) and
 * the secant cut-off of the Newton step between grey solves built on different grids
 * (default 1e-7: D = 0 unless |T* - T_prev| > cut T*), both readings where the paper is
 * silent; settable so that tests can vary them. */
void orc_set_readings(double flux_floor, double secant_cut);

/* Threads of the group-parallel loops (sweep over groups, group physics over cells,
 * group systems, coarse groups of a restriction) when built with OpenMP; n <= 0 leaves the
 * count.  Returns the count in effect (1 without OpenMP).  Results do not depend on it. */
int orc_set_threads(int n);

/* ---- cycle schedules (Sec. 4, Fig. 1, Alg. 3) ---- */
int orc_schedule(int type, int Gamma, int *S);   /* type 0=V, 1=W, 2=F; returns K */

/* ---- whole problem, Algorithm 3 ---- */
typedef struct orc_problem orc_problem;
orc_problem *orc_create(int nx, const double *h, int N, int G, const double *edges,
                        int n_levels, const int *level_groups, double opac_scale, double cv,
                        double T0, double T_left, double T_right);
int orc_step(orc_problem *p, double dt, int cycle_type, int l_max, double eps,
             double eps_inner, int max_outer, int *counters);
void orc_get_state(const orc_problem *p, double *T, double *Eg, double *Fg,
                   double *E, double *F, double *I, double *f);
void orc_set_state(orc_problem *p, const double *T, const double *Eg, const double *Fg,
                   const double *I, const double *f, const double *fb0, const double *fbX,
                   const double *C0, const double *CX);
void orc_destroy(orc_problem *p);
/* T_r option: 0 (default) T_r = T; 1: the opacities sigma_E,g, sigma_R,g are evaluated at
 * (T, T_r) with T_r = (E/aR)^{1/4}, E the latest grey energy of the step (at the step's
 * start the sum of the group energies), the emission at T as before. */
void orc_set_tr_mode(orc_problem *p, int on);

#ifdef __cplusplus
}
#endif
#endif
