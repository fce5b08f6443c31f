// common.cuh -- internal declarations of the GB300 MLQD library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include "../../include/trt.h"

namespace trt {

constexpr double kC = 299.792458;   // cm / sh
constexpr double kAR = 0.01372;     // GJ / (cm^3 keV^4)
constexpr double kPi = 3.14159265358979323846;
constexpr double kCB = 15.0 * kAR * kC / (2.0 * kPi * kPi * kPi * kPi);
constexpr int kSer = 48;            // power-series terms for the Planck-type integrals, x < 2
constexpr double kXSplit = 2.0;     // series below, exponential tails at and above

// Planck-type integral constants (physics.cu): series coefficients and totals.
struct SeriesTables {
    double pP[kSer];   // P(x)     = x^3 sum pP[n] x^n,   P(x) = int_0^x t^3/(e^t-1)
    double pN[kSer];   // Nt(x)    = x^3 sum pN[n] x^n,   Nt(x) = -x^4/(e^x-1) + 4 P(x)
    double pD[kSer];   // D(x)     = x^5 sum pD[n] x^n,   D(x) = int_0^x t^7 e^{2t}/(e^t-1)^3
    double Pinf;       // pi^4/15
    double Dinf;       // 2520 (zeta(6) + zeta(7))
    double gx[8], gw[8];   // 8-point Gauss-Legendre rule on [-1, 1] (narrow groups)
};
const SeriesTables &host_series();   // host copy (built once)
void gauss_legendre_host(int n, double *x, double *w);   // nodes / weights on [-1, 1]
cudaError_t ensure_tables();         // upload the tables to the current device (once)

// per-group physics at temperature T on host (inflow spectra, initial condition)
void host_group_B(int G, const double *edges, double T, double *B);

// A frequency level seen by the kernels (device pointers).  `fine` marks the fine grid,
// whose coefficients are the raw fields: phi = f, sig = sigma_E, emis = e_g, sigR is the
// CELL Rosseland opacity [G][nx] (faces take its dx-weighted mean), eta = 0.
struct Level {
    int n;
    int fine;
    double *phi, *sig, *emis, *Eold, *Esum;
    double *sigR, *etaR, *etaL, *Fold;
    double *phib0, *phibX, *C0, *CX, *Ein0, *Fin0, *EinX, *FinX;
    double *E, *F, *Eb0, *EbX;
};

// Coefficients of the grey Newton step passed to the grey kernel.
struct GreyArgs {
    const double *Tstar, *Told, *sig_prev, *T_prev;
    double *T, *sig_prev_out, *T_prev_out;
    int have_prev;
    double cv, s, dt;
    double nu_first, nu_last;   // first and last group edge (last may be inf)
    // flags[0] |= 1 when a temperature is non-positive or non-finite (always written);
    // with want_norms, flags[1..6] = max|T-Tcyc|, max|T|, max|E-Ecyc|, max|E|,
    // max|T-Tphase|, max|E-Ephase| (end-of-cycle convergence checks)
    int want_norms;
    const double *Tcyc, *Ecyc, *Tphase, *Ephase;
    double *flags;              // [8], device
};

struct Problem {
    int nx, N, M, G, ldG, nlev, precision;
    int levels[16];
    double s, cv, T0, Tl, Tr;
    double nu_first, nu_last;
    cudaStream_t stream;
    // device constants
    double *h, *edges, *mu, *w, *Iin0, *IinX, *Ein0, *Fin0, *EinX, *FinX;
};

// ---- launchers (each enqueues on p.stream; returns cudaError_t of the launch) ----
cudaError_t launch_opacity(const Problem &p, const double *T, double *sigE, double *emis,
                           double *sigR);
size_t sweep_partial_doubles(const Problem &p);
cudaError_t launch_sweep(const Problem &p, double dt, const double *sigE, const double *emis,
                         const void *I_old, void *I_new, double *part, double *psi_exit,
                         double *f, double *fb0, double *fbX, double *C0, double *CX);
cudaError_t launch_lo_solve(const Problem &p, double dt, const Level &L);
cudaError_t launch_restrict(const Problem &p, const Level &src, Level &dst);
cudaError_t launch_grey(const Problem &p, const Level &g, const GreyArgs &a);
cudaError_t launch_group_sum(const Problem &p, int n, const double *X, double *out);

}  // namespace trt
