/*
 * driver.c -- oracle: one time step of the MLQD method with multigrid in photon
 * frequency (Algorithm 3), on a 1D slab.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  FP64, single threaded.
 *
 * Problem (Sec. 2, Sec. 6): slab [0, X] in cells h_i, groups with edges nu_g (first 0,
 * last possibly inf), material energy eps(T) = cv T, isotropic Planck inflow B_g(T_left)
 * at x=0 (vacuum if T_left <= 0) and B_g(T_right) at x=X, initial state T = T0,
 * I_g = B_g(T0) on every corner and direction, E_g = (1/c) sum w I, F_g = sum w mu I.
 * Grid hierarchy (Sec. 4): n^1 = G > n^2 > ... > n^Gamma = 1, uniform coarsening.
 *
 * Readings of Algorithm 3 (paper silent, garbled or at odds with itself):
 *   - the outer loop stops when BOTH ||T^(s)-T^(s-1)|| <= eps ||T^(s)|| and the same
 *     for the grey E hold (the printed "while A & B" would stop when either holds);
 *   - s = 0 is a low-order phase without a sweep, using f from the previous step;
 *   - the inner loop runs at most l_max cycles per phase, leaving early when T and
 *     grey E change by <= eps_inner (relative, infinity norm) over one cycle;
 *   - T~^[0] = T^(l,s) (the printed T~^[1] is an index typo);
 *   - on a coarse visit the fine opacities are re-evaluated at T~^[k] and averaged
 *     with the fine solution of the current cycle;
 *   - the step ends with T from the last grey solve, E_g and F_g from the last fine
 *     solve, I from the last sweep (I^{j-1} if no sweep ran);
 *   - eps < 0 selects a fixed iteration count: exactly max_outer low-order phases of
 *     exactly l_max cycles (used to compare two implementations step by step).
 * Counters (Sec. 6): N_ti sweeps, N_c cycles, N_lo group-wise low-order solves
 * (every grey solve counts one).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

extern double orc_secant_cut;   /* lo.c: cross-grid secant cut-off (reading) */

#ifdef _OPENMP
#include <omp.h>
#endif

int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

#define MAXLEV 16

struct orc_problem {
    int nx, N, M, G, nlev;
    int ng[MAXLEV];            /* groups per level, ng[0] = G, ng[nlev-1] = 1 */
    int *map[MAXLEV];          /* fine group -> group of level l */
    double *h, *mu, *w, *edges;
    double s, cv;
    double *Iin0, *IinX;       /* isotropic inflow per group */
    double *Ein0, *Fin0, *EinX, *FinX;
    /* state at t^j */
    double *T, *Eg, *Fg, *I, *f, *fb0, *fbX, *C0, *CX;
    double *E, *F;             /* grey energy / flux of the last grey solve */
    int tr_mode;               /* opacities at (T, T_r = (E/aR)^{1/4}) instead of T_r = T */
};

void orc_set_tr_mode(orc_problem *p, int on) { if (p) p->tr_mode = on ? 1 : 0; }

static double *dalloc(size_t n) { return (double *)calloc(n, sizeof(double)); }

orc_problem *orc_create(int nx, const double *h, int N, int G, const double *edges,
                        int n_levels, const int *level_groups, double opac_scale, double cv,
                        double T0, double T_left, double T_right)
{
    if (n_levels < 2 || n_levels > MAXLEV || level_groups[0] != G ||
        level_groups[n_levels - 1] != 1)
        return NULL;
    orc_problem *p = (orc_problem *)calloc(1, sizeof(orc_problem));
    p->nx = nx; p->N = N; p->M = 2 * N; p->G = G; p->nlev = n_levels;
    p->s = opac_scale; p->cv = cv;
    p->h = dalloc(nx); memcpy(p->h, h, sizeof(double) * nx);
    p->edges = dalloc(G + 1); memcpy(p->edges, edges, sizeof(double) * (G + 1));
    p->mu = dalloc(p->M); p->w = dalloc(p->M);
    orc_double_gl(N, p->mu, p->w);
    for (int l = 0; l < n_levels; ++l) {
        p->ng[l] = level_groups[l];
        p->map[l] = (int *)calloc(G, sizeof(int));
        int per = G / level_groups[l];
        for (int g = 0; g < G; ++g) p->map[l][g] = g / per;
    }
    const double c = orc_c();
    p->Iin0 = dalloc(G); p->IinX = dalloc(G);
    if (T_left > 0.0) orc_group_physics(G, edges, T_left, 1.0, p->Iin0, NULL, NULL, NULL);
    if (T_right > 0.0) orc_group_physics(G, edges, T_right, 1.0, p->IinX, NULL, NULL, NULL);
    /* eq. mloqd-bcs inflow moments: E^+ = (1/c) int_0^1 I^+, F^+ = int_0^1 mu I^+,
     * E^- = (1/c) int_{-1}^0 I^-, F^- = int_{-1}^0 mu I^- */
    p->Ein0 = dalloc(G); p->Fin0 = dalloc(G); p->EinX = dalloc(G); p->FinX = dalloc(G);
    for (int g = 0; g < G; ++g)
        for (int m = 0; m < p->M; ++m) {
            if (p->mu[m] > 0) {
                p->Ein0[g] += p->w[m] * p->Iin0[g] / c;
                p->Fin0[g] += p->w[m] * p->mu[m] * p->Iin0[g];
            } else {
                p->EinX[g] += p->w[m] * p->IinX[g] / c;
                p->FinX[g] += p->w[m] * p->mu[m] * p->IinX[g];
            }
        }
    /* initial condition (Sec. 6): T = T0, I = B_g(T0) */
    p->T = dalloc(nx); p->Eg = dalloc((size_t)G * nx); p->Fg = dalloc((size_t)G * (nx + 1));
    p->I = dalloc((size_t)p->M * nx * 2 * G);
    p->f = dalloc((size_t)G * nx); p->fb0 = dalloc(G); p->fbX = dalloc(G);
    p->C0 = dalloc(G); p->CX = dalloc(G);
    p->E = dalloc(nx); p->F = dalloc(nx + 1);
    double *B0 = dalloc(G);
    orc_group_physics(G, edges, T0, 1.0, B0, NULL, NULL, NULL);
    for (int i = 0; i < nx; ++i) p->T[i] = T0;
    for (size_t m = 0; m < (size_t)p->M; ++m)
        for (int i = 0; i < nx; ++i)
            for (int cc = 0; cc < 2; ++cc)
                for (int g = 0; g < G; ++g)
                    p->I[((m * nx + i) * 2 + cc) * G + g] = B0[g];
    for (int g = 0; g < G; ++g) {
        double e0 = 0.0, s0 = 0.0, s2 = 0.0, hm0 = 0.0, hm1 = 0.0, hp0 = 0.0, hp1 = 0.0;
        for (int m = 0; m < p->M; ++m) {
            e0 += p->w[m] * p->mu[m] * B0[g];
            s0 += p->w[m] * B0[g];
            s2 += p->w[m] * p->mu[m] * p->mu[m] * B0[g];
            if (p->mu[m] < 0) { hm0 += p->w[m] * B0[g]; hm1 += p->w[m] * p->mu[m] * B0[g]; }
            else { hp0 += p->w[m] * B0[g]; hp1 += p->w[m] * p->mu[m] * B0[g]; }
        }
        for (int i = 0; i < nx; ++i) {
            p->Eg[(size_t)g * nx + i] = s0 / c;
            p->f[(size_t)g * nx + i] = (s0 != 0.0) ? s2 / s0 : 1.0 / 3.0;
        }
        for (int f = 0; f <= nx; ++f) p->Fg[(size_t)g * (nx + 1) + f] = e0;
        p->fb0[g] = p->fbX[g] = (s0 != 0.0) ? s2 / s0 : 1.0 / 3.0;
        p->C0[g] = (hm0 != 0.0) ? hm1 / hm0 : -0.5;
        p->CX[g] = (hp0 != 0.0) ? hp1 / hp0 : 0.5;
    }
    for (int i = 0; i < nx; ++i) {
        double e = 0.0;
        for (int g = 0; g < G; ++g) e += p->Eg[(size_t)g * nx + i];
        p->E[i] = e;
    }
    free(B0);
    return p;
}

void orc_destroy(orc_problem *p)
{
    if (!p) return;
    for (int l = 0; l < p->nlev; ++l) free(p->map[l]);
    free(p->h); free(p->mu); free(p->w); free(p->edges);
    free(p->Iin0); free(p->IinX); free(p->Ein0); free(p->Fin0); free(p->EinX); free(p->FinX);
    free(p->T); free(p->Eg); free(p->Fg); free(p->I); free(p->f);
    free(p->fb0); free(p->fbX); free(p->C0); free(p->CX); free(p->E); free(p->F);
    free(p);
}

void orc_get_state(const orc_problem *p, double *T, double *Eg, double *Fg,
                   double *E, double *F, double *I, double *f)
{
    size_t nx = p->nx, G = p->G;
    if (T) memcpy(T, p->T, sizeof(double) * nx);
    if (Eg) memcpy(Eg, p->Eg, sizeof(double) * G * nx);
    if (Fg) memcpy(Fg, p->Fg, sizeof(double) * G * (nx + 1));
    if (E) memcpy(E, p->E, sizeof(double) * nx);
    if (F) memcpy(F, p->F, sizeof(double) * (nx + 1));
    if (I) memcpy(I, p->I, sizeof(double) * p->M * nx * 2 * G);
    if (f) memcpy(f, p->f, sizeof(double) * G * nx);
}

void orc_set_state(orc_problem *p, const double *T, const double *Eg, const double *Fg,
                   const double *I, const double *f, const double *fb0, const double *fbX,
                   const double *C0, const double *CX)
{
    size_t nx = p->nx, G = p->G;
    if (T) memcpy(p->T, T, sizeof(double) * nx);
    if (Eg) {
        memcpy(p->Eg, Eg, sizeof(double) * G * nx);
        for (size_t i = 0; i < nx; ++i) {
            double e = 0.0;
            for (size_t g = 0; g < G; ++g) e += Eg[g * nx + i];
            p->E[i] = e;
        }
    }
    if (Fg) memcpy(p->Fg, Fg, sizeof(double) * G * (nx + 1));
    if (I) memcpy(p->I, I, sizeof(double) * p->M * nx * 2 * G);
    if (f) memcpy(p->f, f, sizeof(double) * G * nx);
    if (fb0) memcpy(p->fb0, fb0, sizeof(double) * G);
    if (fbX) memcpy(p->fbX, fbX, sizeof(double) * G);
    if (C0) memcpy(p->C0, C0, sizeof(double) * G);
    if (CX) memcpy(p->CX, CX, sizeof(double) * G);
}

/* group opacities of every cell at temperatures T (Sec. 2) -> [G][nx] */
static void physics_all(const orc_problem *p, const double *T, const double *Erad, double *sig,
                        double *emis, double *sigR_cell)
{
    int nx = p->nx, G = p->G;
    const double aR = orc_aR();
    /* cells are independent: with OpenMP each thread takes whole cells */
#pragma omp parallel
    {
    double *sB = dalloc(G), *em = dalloc(G), *sR = dalloc(G), *sE = dalloc(G);
#pragma omp for schedule(static)
    for (int i = 0; i < nx; ++i) {
        orc_group_physics(G, p->edges, T[i], p->s, NULL, sB, em, sR);
        const double *sEi = sB;   /* sigma_E = sigma_B under T_r = T */
        if (p->tr_mode && Erad[i] > 0.0 && isfinite(Erad[i])) {
            /* T_r from the latest grey energy: E = aR T_r^4 */
            orc_group_opacity_tr(G, p->edges, T[i], pow(Erad[i] / aR, 0.25), p->s, sE, sR);
            sEi = sE;
        }
        for (int g = 0; g < G; ++g) {
            sig[(size_t)g * nx + i] = sEi[g];
            emis[(size_t)g * nx + i] = em[g];
            sigR_cell[(size_t)g * nx + i] = sR[g];
        }
    }
    free(sB); free(em); free(sR); free(sE);
    }
}

static double inf_norm_diff(int n, const double *a, const double *b)
{
    double m = 0.0;
    for (int i = 0; i < n; ++i) if (fabs(a[i] - b[i]) > m) m = fabs(a[i] - b[i]);
    return m;
}
static double inf_norm(int n, const double *a)
{
    double m = 0.0;
    for (int i = 0; i < n; ++i) if (fabs(a[i]) > m) m = fabs(a[i]);
    return m;
}

/* a level's coefficient arrays */
typedef struct {
    double *phi, *sig, *emis, *Eold, *sigR, *etaR, *etaL, *Fold;
    double *phib0, *phibX, *C0, *CX, *Ein0, *Fin0, *EinX, *FinX, *Esum;
    double *E, *F, *Eb0, *EbX;
} level;

static void level_alloc(level *L, int ng, int nx)
{
    L->phi = dalloc((size_t)ng * nx); L->sig = dalloc((size_t)ng * nx);
    L->emis = dalloc((size_t)ng * nx); L->Eold = dalloc((size_t)ng * nx);
    L->Esum = dalloc((size_t)ng * nx); L->E = dalloc((size_t)ng * nx);
    L->sigR = dalloc((size_t)ng * (nx + 1)); L->etaR = dalloc((size_t)ng * (nx + 1));
    L->etaL = dalloc((size_t)ng * (nx + 1)); L->Fold = dalloc((size_t)ng * (nx + 1));
    L->F = dalloc((size_t)ng * (nx + 1));
    L->phib0 = dalloc(ng); L->phibX = dalloc(ng); L->C0 = dalloc(ng); L->CX = dalloc(ng);
    L->Ein0 = dalloc(ng); L->Fin0 = dalloc(ng); L->EinX = dalloc(ng); L->FinX = dalloc(ng);
    L->Eb0 = dalloc(ng); L->EbX = dalloc(ng);
}
static void level_free(level *L)
{
    free(L->phi); free(L->sig); free(L->emis); free(L->Eold); free(L->Esum); free(L->E);
    free(L->sigR); free(L->etaR); free(L->etaL); free(L->Fold); free(L->F);
    free(L->phib0); free(L->phibX); free(L->C0); free(L->CX);
    free(L->Ein0); free(L->Fin0); free(L->EinX); free(L->FinX); free(L->Eb0); free(L->EbX);
}

/* solve every group of a (fine or coarse) level: a = c sig, s = 2 emis (eq. mloqd-d) */
static void level_solve(const orc_problem *p, level *L, int ng, double dt)
{
    int nx = p->nx, nf = nx + 1;
    const double c = orc_c();
    /* the groups' systems are independent: with OpenMP each thread solves whole groups */
#pragma omp parallel
    {
    double *a = dalloc(nx), *s = dalloc(nx);
#pragma omp for schedule(static)
    for (int q = 0; q < ng; ++q) {
        for (int i = 0; i < nx; ++i) {
            a[i] = c * L->sig[(size_t)q * nx + i];
            s[i] = 2.0 * L->emis[(size_t)q * nx + i];
        }
        orc_lo_solve(nx, p->h, dt, a, s, L->Eold + (size_t)q * nx, L->phi + (size_t)q * nx,
                     L->sigR + (size_t)q * nf, L->etaR + (size_t)q * nf,
                     L->etaL + (size_t)q * nf, L->Fold + (size_t)q * nf,
                     L->phib0[q], L->phibX[q], L->C0[q], L->CX[q],
                     L->Ein0[q], L->Fin0[q], L->EinX[q], L->FinX[q],
                     L->E + (size_t)q * nx, L->F + (size_t)q * nf, &L->Eb0[q], &L->EbX[q]);
    }
    free(a); free(s);
    }
}

static void restrict_level(const orc_problem *p, const level *A, int nA, const int *map,
                           level *B, int nB)
{
    orc_restrict(p->nx, p->h, nA, nB, map, A->phi, A->sig, A->emis, A->Eold, A->sigR,
                 A->etaR, A->etaL, A->Fold, A->phib0, A->phibX, A->C0, A->CX,
                 A->Ein0, A->Fin0, A->EinX, A->FinX, A->E, A->F, A->Eb0, A->EbX,
                 B->phi, B->sig, B->emis, B->Eold, B->sigR, B->etaR, B->etaL, B->Fold,
                 B->phib0, B->phibX, B->C0, B->CX, B->Ein0, B->Fin0, B->EinX, B->FinX,
                 B->Esum);
}

/* fine-level coefficients at opacities (sig, emis, sigR_cell) with the current QD
 * factors; E, F of the level are left to the caller */
static void fine_coeffs(const orc_problem *p, level *L, const double *sig, const double *emis,
                        const double *sigR_cell, const double *Eg_old, const double *Fg_old)
{
    size_t nx = p->nx, G = p->G;
    memcpy(L->phi, p->f, sizeof(double) * G * nx);
    memcpy(L->sig, sig, sizeof(double) * G * nx);
    memcpy(L->emis, emis, sizeof(double) * G * nx);
    memcpy(L->Eold, Eg_old, sizeof(double) * G * nx);
    orc_fine_face_sigR(p->nx, p->h, p->G, sigR_cell, L->sigR);
    memset(L->etaR, 0, sizeof(double) * G * (nx + 1));
    memset(L->etaL, 0, sizeof(double) * G * (nx + 1));
    memcpy(L->Fold, Fg_old, sizeof(double) * G * (nx + 1));
    memcpy(L->phib0, p->fb0, sizeof(double) * G); memcpy(L->phibX, p->fbX, sizeof(double) * G);
    memcpy(L->C0, p->C0, sizeof(double) * G); memcpy(L->CX, p->CX, sizeof(double) * G);
    memcpy(L->Ein0, p->Ein0, sizeof(double) * G); memcpy(L->Fin0, p->Fin0, sizeof(double) * G);
    memcpy(L->EinX, p->EinX, sizeof(double) * G); memcpy(L->FinX, p->FinX, sizeof(double) * G);
}

int orc_step(orc_problem *p, double dt, int cycle_type, int l_max, double eps,
             double eps_inner, int max_outer, int *counters)
{
    const int nx = p->nx, G = p->G, M = p->M, Gam = p->nlev;
    const double c = orc_c();
    const size_t nI = (size_t)M * nx * 2 * G;
    int S[1 << 12];
    int K = orc_schedule(cycle_type, Gam, S);
    int fixed = eps < 0.0;
    int n_ti = 0, n_c = 0, n_lo = 0, s_it = 0, status = 0;

    double *Told = dalloc(nx), *Tcur = dalloc(nx), *Tphase = dalloc(nx), *Ttil = dalloc(nx);
    double *Tnew = dalloc(nx), *Tprev = dalloc(nx), *sigprev = dalloc(nx);
    double *Eg_old = dalloc((size_t)G * nx), *Fg_old = dalloc((size_t)G * (nx + 1));
    double *I_old = dalloc(nI);
    double *Ephase = dalloc(nx), *Ecyc = dalloc(nx);
    double *sig = dalloc((size_t)G * nx), *emis = dalloc((size_t)G * nx);
    double *sigRc = dalloc((size_t)G * nx);
    double *Q = dalloc(nx), *dQ = dalloc(nx);
    double *Egrey = dalloc(nx), *Fgrey = dalloc(nx + 1);
    double Eb0g, EbXg;
    level fine, crs, grey;
    level_alloc(&fine, G, nx);
    level_alloc(&crs, G, nx);
    level_alloc(&grey, 1, nx);
    int *zero_map = (int *)calloc(G, sizeof(int));   /* every group -> the grey group */
    int have_prev = 0;

    memcpy(Told, p->T, sizeof(double) * nx);
    memcpy(Tcur, p->T, sizeof(double) * nx);
    memcpy(Eg_old, p->Eg, sizeof(double) * G * nx);
    memcpy(Fg_old, p->Fg, sizeof(double) * G * (nx + 1));
    memcpy(I_old, p->I, sizeof(double) * nI);
    for (int i = 0; i < nx; ++i) {
        double e = 0.0;
        for (int g = 0; g < G; ++g) e += Eg_old[(size_t)g * nx + i];
        Ephase[i] = e;
    }
    memcpy(Egrey, Ephase, sizeof(double) * nx);

    for (;;) {
        /* ---- transport (outer) iteration ---- */
        if (s_it > 0) {
            physics_all(p, Tcur, Egrey, sig, emis, sigRc);
            orc_sweep(nx, p->h, M, p->mu, p->w, G, sig, emis, 1.0 / (c * dt), I_old,
                      p->Iin0, p->IinX, p->I, p->f, p->fb0, p->fbX, p->C0, p->CX);
            ++n_ti;
        }
        memcpy(Tphase, Tcur, sizeof(double) * nx);
        double *Tcyc = Tcur;
        memcpy(Ecyc, Ephase, sizeof(double) * nx);
        for (int l = 0; l < l_max; ++l) {
            /* fine-grid spectrum at T^(l,s) (eq. mloqd-d) */
            physics_all(p, Tcyc, Egrey, sig, emis, sigRc);
            fine_coeffs(p, &fine, sig, emis, sigRc, Eg_old, Fg_old);
            level_solve(p, &fine, G, dt);
            n_lo += G;
            memcpy(Ttil, Tcyc, sizeof(double) * nx);
            for (int k = 0; k <= K; ++k) {
                level *src = &fine;
                int nsrc = G;
                if (k > 0) {
                    /* coarse-grid spectrum on grid gamma_k at T~^[k] */
                    int gam = S[k - 1];
                    int ngam = p->ng[gam - 1];
                    level tmp;
                    physics_all(p, Ttil, Egrey, sig, emis, sigRc);
                    /* fine coefficients at T~, weighted with this cycle's fine solution */
                    level_alloc(&tmp, G, nx);
                    fine_coeffs(p, &tmp, sig, emis, sigRc, Eg_old, Fg_old);
                    memcpy(tmp.E, fine.E, sizeof(double) * G * nx);
                    memcpy(tmp.F, fine.F, sizeof(double) * G * (nx + 1));
                    memcpy(tmp.Eb0, fine.Eb0, sizeof(double) * G);
                    memcpy(tmp.EbX, fine.EbX, sizeof(double) * G);
                    restrict_level(p, &tmp, G, p->map[gam - 1], &crs, ngam);
                    level_free(&tmp);
                    level_solve(p, &crs, ngam, dt);
                    n_lo += ngam;
                    src = &crs;
                    nsrc = ngam;
                } else {
                    /* k = 0: the fine level at T~^[0] = T^(l,s) is the one just solved */
                }
                restrict_level(p, src, nsrc, zero_map, &grey, 1);
                /* grey LOQD + MEB at T~^[k] (eq. eb-Gamma-d) */
                for (int i = 0; i < nx; ++i) {
                    Q[i] = 2.0 * grey.emis[i];
                    dQ[i] = orc_emission_deriv(G, p->edges, Ttil[i], p->s);
                }
                int bad = orc_grey_newton(nx, p->h, dt, p->cv, Ttil, Told, Q, dQ, grey.Esum,
                                          grey.sig, sigprev, Tprev, have_prev,
                                          K == 0 ? 0.0 : orc_secant_cut, grey.Eold,
                                          grey.phi, grey.sigR, grey.etaR, grey.etaL, grey.Fold,
                                          grey.phib0[0], grey.phibX[0], grey.C0[0], grey.CX[0],
                                          grey.Ein0[0], grey.Fin0[0], grey.EinX[0],
                                          grey.FinX[0], Tnew, Egrey, Fgrey, &Eb0g, &EbXg);
                n_lo += 1;
                memcpy(sigprev, grey.sig, sizeof(double) * nx);
                memcpy(Tprev, Ttil, sizeof(double) * nx);
                have_prev = 1;
                memcpy(Ttil, Tnew, sizeof(double) * nx);
                if (bad) { status = 2; goto done; }
            }
            ++n_c;
            int conv_in = inf_norm_diff(nx, Ttil, Tcyc) <= eps_inner * inf_norm(nx, Ttil) &&
                          inf_norm_diff(nx, Egrey, Ecyc) <= eps_inner * inf_norm(nx, Egrey);
            memcpy(Tcyc, Ttil, sizeof(double) * nx);
            memcpy(Ecyc, Egrey, sizeof(double) * nx);
            if (!fixed && conv_in) break;
        }
        /* Tcur now holds T^(s+1) */
        int conv_out = inf_norm_diff(nx, Tcur, Tphase) <= eps * inf_norm(nx, Tcur) &&
                       inf_norm_diff(nx, Ecyc, Ephase) <= eps * inf_norm(nx, Ecyc);
        memcpy(Ephase, Ecyc, sizeof(double) * nx);
        ++s_it;
        if (fixed) {
            if (s_it >= max_outer) break;
        } else {
            if (conv_out) break;
            if (s_it >= max_outer) { status = 1; break; }
        }
    }
done:
    /* end of step: T from the last grey solve, E_g, F_g from the last fine solve */
    memcpy(p->T, Tcur, sizeof(double) * nx);
    memcpy(p->Eg, fine.E, sizeof(double) * G * nx);
    memcpy(p->Fg, fine.F, sizeof(double) * G * (nx + 1));
    memcpy(p->E, Egrey, sizeof(double) * nx);
    memcpy(p->F, Fgrey, sizeof(double) * (nx + 1));
    if (counters) {
        counters[0] = n_ti; counters[1] = n_c; counters[2] = n_lo; counters[3] = s_it;
    }
    free(Told); free(Tcur); free(Tphase); free(Ttil); free(Tnew); free(Tprev); free(sigprev);
    free(Eg_old); free(Fg_old); free(I_old); free(Ephase); free(Ecyc);
    free(sig); free(emis); free(sigRc); free(Q); free(dQ); free(Egrey); free(Fgrey);
    level_free(&fine); level_free(&crs); level_free(&grey);
    free(zero_map);
    return status;
}
