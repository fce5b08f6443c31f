// common.cuh -- internal declarations of the GB300 MLQD library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <utility>
#include "../../include/trt.h"

namespace trt {

constexpr double kC = 299.792458;   // cm / sh
constexpr double kAR = 0.01372;     // GJ / (cm^3 keV^4)
constexpr double kPi = 3.14159265358979323846;
constexpr double kCB = 15.0 * kAR * kC / (2.0 * kPi * kPi * kPi * kPi);
constexpr int kSer = 48;            // power-series terms for the Planck-type integrals, x < 2
constexpr double kXSplit = 2.0;     // series below, exponential tails at and above
// secant of the grey Newton step between grey solves built on different grids (W, F
// cycles): taken only where |T* - T_prev| > kSecantCut T* (Sec. 5, eq. f-derivative-d;
// a reading, the paper is silent on the degenerate quotient)
constexpr double kSecantCut = 1e-7;

// Planck-type integral constants (physics.cu): series coefficients and totals.
struct SeriesTables {
    double pP[kSer];   // P(x)     = x^3 sum pP[n] x^n,   P(x) = int_0^x t^3/(e^t-1)
    double pN[kSer];   // Nt(x)    = x^3 sum pN[n] x^n,   Nt(x) = -x^4/(e^x-1) + 4 P(x)
    double pD[kSer];   // D(x)     = x^5 sum pD[n] x^n,   D(x) = int_0^x t^7 e^{2t}/(e^t-1)^3
    double Pinf;       // pi^4/15
    double Dinf;       // 2520 (zeta(6) + zeta(7))
    double tP[65], tD[65];   // tail coefficients 6/k^4 and 5040 k(k+1)/2 / k^8, k = 1..64
    double g3x[3], g3w[3];   // 3-point rule; the centre weight is halved: the symmetric
                             // loop of gauss_group visits the centre once per side
    double g4x[4], g4w[4];   // 4- and 6-point Gauss-Legendre rules on [-1, 1]
    double g6x[6], g6w[6];   // (narrow groups, see group_integrals)
    double g8x[8], g8w[8];   // 8-point rule of the opacities at a radiation temperature
    double e2[32];           // 2^(j/32), j = 0..31 (texp)
    double einv, eL1, eL2;   // 32/ln2 and ln2/32 = eL1 + eL2 (texp)
};
// 1/d in FP64: the hardware's approximate FP64 reciprocal (special-function unit, a
// relative error eps below 2^-19.9 measured, not the FP64 pipe) refined by one third-order
// Newton-Raphson (Householder) step: with e = 1 - d x, x (1 + e + e^2) = (1 - eps^3)/d,
// below FP64 rounding, at 3 FP64 FMAs where an IEEE division costs ~20 on GB300's FP64
// pipe.  Zero, infinite, NaN or subnormal operands (or results) divide; the test reads
// the approximation's biased exponent with integer instructions (an FP64 compare would
// take the FP64 pipe): 1 .. 2018 (|x| < 2^996) is the refined case.  The division sits in
// a function that is never inlined, so that the compiler branches around it instead of
// predicating its FP64 instructions into every call.
#ifdef __CUDA_ARCH__
static __device__ __noinline__ double rcp64_divide(double d) { return 1.0 / d; }
#endif
__host__ __device__ inline double rcp64(double d)
{
#ifdef __CUDA_ARCH__
    double x;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(d));
    const unsigned ex = ((unsigned)__double2hiint(x) >> 20) & 0x7ffu;
    if (ex - 1u >= 2018u) return rcp64_divide(d);
    const double e = fma(-d, x, 1.0);
    return fma(x, fma(e, e, e), x);
#else
    return 1.0 / d;
#endif
}

// e^x by Tang's table-driven method (P. T. P. Tang, "Table-driven implementation of the
// exponential function in IEEE floating-point arithmetic", ACM TOMS 15, 1989): x = (32 m +
// j) ln2/32 + r with |r| <= ln2/64 (two-part constant, exact product k L1), e^x =
// 2^m 2^(j/32) (1 + p(r)), p the degree-6 Taylor polynomial of e^r - 1 (truncation
// r^7/7! < 2e-18).  tab = 2^(j/32), j = 0..31 (SeriesTables::e2, staged in shared memory).
// Within about an ulp.  GB300 runs FP64 compares and FP64 <-> integer conversions on the
// FP64 pipe, so the range tests read the high word of x with integer instructions, the
// rounding of x 32/ln2 adds and subtracts 1.5 2^52 (the integer then sits in the low word
// of the sum), and 2^m is added to the exponent field of the result (normal for |x| < 704,
// where |m| <= 1016): about 12 FP64 operations.  x <= -746 gives 0 (e^x is below half the
// smallest subnormal: the correctly rounded value); anything else outside (-704, 704) and
// NaN call exp() from a function that is never inlined (a branch around the library code,
// not predicated FP64 instructions on every call).
struct ExpConsts {
    double inv, L1, L2;   // 32/ln2; ln2/32 = L1 + L2 with L1 of 31 significant bits
};
static __device__ __noinline__ double texp_library(double x) { return exp(x); }
__device__ inline double texp(double x, const double *tab, const ExpConsts &c)
{
    const int hi = __double2hiint(x);
    const unsigned ahi = (unsigned)hi & 0x7fffffffu;
    if (ahi >= 0x40860000u) {   // |x| >= 704, inf or NaN
        if (hi < 0 && ahi >= 0x40875000u && ahi < 0x7ff00000u) return 0.0;   // -746 >= x > -inf
        return texp_library(x);
    }
    const double kMagic = 6755399441055744.0;   // 1.5 2^52
    const double sk = fma(x, c.inv, kMagic);
    const int k = __double2loint(sk);           // rint(x 32/ln2)
    const double kd = sk - kMagic;
    const double r = fma(-kd, c.L2, fma(-kd, c.L1, x));
    const double q = r * r * (0.5 + r * (1.0 / 6 + r * (1.0 / 24 + r * (1.0 / 120 + r * (1.0 / 720)))));
    const double t = tab[k & 31];
    const double v = fma(t, r + q, t);
    return __longlong_as_double(__double_as_longlong(v) + ((long long)(k >> 5) << 52));
}

// FP32 -> FP64 without the FP64 pipe (GB300 converts there): a normal float is widened
// with integer instructions (sign, exponent rebiased by 1023 - 127 = 896, mantissa shifted
// by 29: exact), a zero keeps its sign; subnormal, infinite and NaN values convert, in a
// function that is never inlined (a branch around the conversion, not a predicated
// conversion on every call).
static __device__ __noinline__ double widen_f32_convert(float q) { return (double)q; }
__device__ inline double widen_f32(float q)
{
    const unsigned u = __float_as_uint(q);
    const unsigned e = (u >> 23) & 0xffu;
    if ((u & 0x7fffffffu) == 0u)
        return __longlong_as_double((long long)((unsigned long long)u << 32));   // +0 or -0
    if (e == 0u || e == 0xffu) return widen_f32_convert(q);
    const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(e + 896u) << 52) |
                                 ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)b);
}

// Programmatic dependent launch for the kernels of one low-order cycle, which run back to
// back on one stream: the launch of kernel k+1 is processed while kernel k drains, and
// k+1's first statement, griddep_wait(), holds every thread until k has completed and its
// writes are visible.  A kernel launched this way must call griddep_wait() before it reads
// or writes global memory (a no-op when the kernel was launched plainly).
#ifdef __CUDACC__
__device__ inline void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

const SeriesTables &host_series();   // host copy (built once)
void gauss_legendre_host(int n, double *x, double *w);   // nodes / weights on [-1, 1]
cudaError_t ensure_tables();         // upload the tables to the current device (once)
cudaError_t launch_fastmath(int n, const double *x, double *ex, double *rc, cudaStream_t st);
// FP64 FMA rate probe: one timed launch of `reps` FMA steps per chain; FMAs executed in *fmas
cudaError_t fp64_probe(int reps, cudaStream_t st, float *ms, long long *fmas);

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
    // the secant of the Newton step is taken where T* != T_prev and |T* - T_prev| >
    // secant_cut T*: 0 when the previous grey solve was built on the same grid (two-grid
    // and V cycles), 1e-7 across grids (W, F: sigma-bar also jumps with the grid)
    double secant_cut;
    // when non-null, the device flag replaces have_prev (read at entry, set to 1 on exit):
    // the batched driver keeps it per slab so that its argument blocks stay fixed
    int *have_prev_dev;
    double cv, s, dt;
    double nu_first, nu_last;   // first and last group edge (last may be inf)
    // flags[0] |= 1 when a temperature is non-positive or non-finite (always written);
    // with want_norms, flags[1..6] = max|T-Tcyc|, max|T|, max|E-Ecyc|, max|E|,
    // max|T-Tphase|, max|E-Ephase| (end-of-cycle convergence checks)
    int want_norms;
    const double *Tcyc, *Ecyc, *Tphase, *Ephase;
    double *flags;              // [8], device
    // the end-of-cycle copies, when non-null (with want_norms): T into T_out, and after the
    // norms have read them, T into Tcyc_out and E into Ecyc_out (the same arrays as Tcyc,
    // Ecyc: each cell's thread reads its old value before it writes the new one)
    double *T_out, *Tcyc_out, *Ecyc_out;
    // inner-loop control of one Algorithm 3 phase on the device (with want_norms), when
    // non-null: ctl[1] counts the cycles that ran, and ctl[0] (the gate that the cycle's
    // kernels of the single-slab driver test at entry) is set once the cycle found a bad
    // temperature or, unless fixed, met the inner test max|T-Tcyc| <= eps_in max|T| and
    // max|E-Ecyc| <= eps_in max|E| -- the host's test, in the same FP64 operations
    int *ctl;
    double eps_in;
    int fixed;
    // set by make_grey_ctx (host, the same IEEE operations): c_v / dt and 54 s C_B, which
    // every cell would otherwise form with an FP64 division on the grey kernel's one SM;
    // the table and constants of texp for the two exponentials of Q'(T) per cell
    double cvdt, k54;
    const double *e2;
    ExpConsts ec;
    // the per-cell Newton terms w c sig*, w Q* - (1 - w) c_v (T* - Told)/dt and 1/Lambda,
    // [3][nx], when the restriction to the grey level already formed them (its second
    // stage, from the same values with the same operations); null: the grey kernel forms
    // them
    const double *pre;
};

inline bool sweep_fp32(int precision) { return (precision & TRT_SWEEP_FP32) != 0; }
inline bool lo_fp32(int precision) { return (precision & TRT_LO_FP32) != 0; }
inline bool lo_pair(int precision) { return (precision & TRT_LO_PAIR) != 0; }
inline bool precision_ok(int precision)
{
    return precision >= 0 && precision <= (TRT_SWEEP_FP32 | TRT_LO_PAIR) &&
           !(lo_fp32(precision) && lo_pair(precision));
}

struct Problem {
    int nx, N, M, G, ldG, nlev, precision;
    int tr_mode = 0;   // opacities at (T, T_r) from the latest grey energy (trt_opacity)
    // single-slab cycle kernels return at entry while *gate != 0 (null: always run); the
    // step driver points it at the phase's inner-loop control word between launches
    const int *gate = nullptr;
    int levels[16];
    double s, cv, T0, Tl, Tr;
    double nu_first, nu_last;
    cudaStream_t stream;
    // device constants
    double *h, *edges, *mu, *w, *Iin0, *IinX, *Ein0, *Fin0, *EinX, *FinX;
    double *ihf;        // [nx+1]: 1/(h_{f-1} + h_f) at interior faces (dx-weighted means)
    double *hf;         // [nx+1]: face half-widths h_0/2, (h_{f-1} + h_f)/2, h_{nx-1}/2
    // constants of the LO rows (lo.cu), so that a row spends no FP64 operation on them: per
    // cell c h and 2 h; per interior face f the weights hf h_{f-1} / (h_{f-1} + h_f) and
    // hf h_f / (h_{f-1} + h_f) of the cell opacities in dx sigma_R,face; and for the step
    // length lo_dt (ensure_lo_consts) h/dt per cell and hf/(c dt) per face
    double *hc, *h2, *fwl, *fwr;
    double *hidt, *dxicdt;
    double lo_dt = 0.0;
    // per-cell terms of the single-slab opacity evaluation (physics.cu): [7][nx] doubles,
    // then nx floats and nx ints
    double *cterm;
    float *dir32;       // [M][4]: |mu|, |mu|/2, w/2, w mu^2/2 rounded once to FP32 (FP32 sweeps)
    double *e2tab;      // [32]: 2^(j/32), the table of texp for kernels outside physics.cu
    int *lo_slot;       // [nx+1]: shared-memory slot k * 32 + l of face/row f in the
                        // partitioned tridiagonal solve (chunk l, row k of the chunk)
    double *rscratch;   // partial sums of the two-stage restriction
    size_t rscratch_doubles;
    // sweep tile: directions per CTA (0 = default) and strip shape index (0 = default)
    int sweep_D = 0, sweep_shape = 0;
    // scratch of the paired FP64 sweep (FP64 handles; null elsewhere): t, s per (|mu|,
    // cell, group) [N][nx][2][ldG], and the pre-scaled inputs [2][nx][ldG] + [nx]
    double *ts64 = nullptr, *tab64 = nullptr;
    // per-group polynomial tables in ln T (Chebyshev fits stored as monomials) of
    // sigma_E T^3, sigma_R T^3 and the emission factor ln(1 - e^{-w}) (null: direct
    // integrals)
    double *otab = nullptr;
    // with TRT_LO_PAIR: the tables with their FP64 coefficients as FP32 pairs, then the G+1
    // group edges as pairs (otab_doubles(G) + G + 1 doubles), and per-cell pair terms of the
    // opacity evaluation [5][nx] (t, 1/T, 1/T^3, 27 s C_B T, h/2); null otherwise
    double *otabp = nullptr, *cpair = nullptr;
    // with TRT_LO_PAIR: the LO row constants as pairs, [8][nx+1] (hf, dxicdt, fwl, fwr per
    // face; hidt, hc, h2, h per cell): the step-independent rows once per handle
    // (launch_lo_pair_consts), hidt and dxicdt with ensure_lo_consts; null otherwise
    double *lopc = nullptr;
};

// opacity tables: ln T in [kTabU0, kTabU0 + kTabNI kTabH), kTabNC coefficients per interval
constexpr int kTabNI = 98, kTabNC = 9;
constexpr double kTabU0 = -9.25, kTabH = 0.125;
constexpr int kTabNF = 3;   // series per interval: sigma_E T^3, sigma_R T^3, ln(1 - e^{-w})
// one (group, interval) entry: the kTabLo low-order monomial coefficients of each series in
// FP64, then its kTabNC - kTabLo high-order ones in FP32 (padded to an even count)
constexpr int kTabLo = 5;
constexpr int kTabHiF = ((kTabNF * (kTabNC - kTabLo) + 1) / 2) * 2;   // floats
constexpr int kTabEntry = kTabNF * kTabLo + kTabHiF / 2;               // doubles
inline size_t otab_doubles(int G) { return (size_t)G * kTabNI * kTabEntry; }
cudaError_t launch_otab_build(const Problem &p);

// ---- launchers (each enqueues on p.stream; returns cudaError_t of the launch) ----
// sig32 / emis32 (may be null): the FP32 sweep's inputs (sigma_E + 1/(c dt)) h/2 and h e/2
// Erad (may be null): per-cell radiation energy; with the T_r option the absorption and
// Rosseland opacities are taken at T_r = (Erad/a_R)^{1/4}
cudaError_t launch_opacity(const Problem &p, const double *T, double *sigE, double *emis,
                           double *sigR, float *sig32 = nullptr, float *emis32 = nullptr,
                           double dt = 0.0, const double *Erad = nullptr);
// the FP32 sweep inputs (sig32, emis32 and the kap32 row after it) from FP64 sigma_E, e_g
cudaError_t launch_prescale32(const Problem &p, double dt, const double *sigE, const double *emis,
                              float *sig32, float *emis32);
size_t sweep_partial_doubles(const Problem &p);
int sweep_shape_count(int precision);
// a kernel exists and fits (shared memory); `batched`: the batched sweep has one too
bool sweep_tile_ok(int precision, int D, int shape, bool batched = false);
void sweep_shape_info(int precision, int shape, int *S, int *NS);
int sweep_group_tiles(int precision, int shape, int D, int ldG);   // CTAs along the groups
int sweep_D_candidates(const Problem &p, int *D);   // fills D[0..n), returns n (<= 3)
// sigE / emis: [G][nx]; FP64 sweeps: double sigma_E, e_g; FP32 sweeps (sigma_fp32 must be
// set): the float pre-scaled (sigma_E + 1/(c dt)) h/2 and h e/2 of launch_opacity or
// launch_prescale32, followed by h/(2 c dt) per cell
cudaError_t launch_sweep(const Problem &p, double dt, const void *sigE, const void *emis,
                         bool sigma_fp32, const void *I_old, void *I_new, double *part,
                         double *psi_exit, double *f, double *fb0, double *fbX, double *C0,
                         double *CX);
cudaError_t launch_lo_solve(const Problem &p, double dt, const Level &L);
// h/dt and hf/(c dt) of the LO rows for step length dt (a launch when dt changed)
cudaError_t ensure_lo_consts(Problem &p, double dt);
// the step-independent pair row constants (Problem::lopc; once per handle, TRT_LO_PAIR)
cudaError_t launch_lo_pair_consts(const Problem &p);
// newton (with pre): the visit's grey Newton arguments; the two-stage restriction to the
// grey level then also forms the per-cell Newton terms into pre ([3][nx]) and sets *formed
// old_key (in/out, may be null): which source's Eold and Fold sums dst holds from this
// step (0: none); the two-stage restriction skips them when it matches src
cudaError_t launch_restrict(const Problem &p, const Level &src, Level &dst,
                            const GreyArgs *newton = nullptr, double *pre = nullptr,
                            bool *formed = nullptr, int *old_key = nullptr);
// the host-formed constants of a grey visit (c_v/dt, 54 s C_B, the exponential's table)
GreyArgs grey_args_ready(const Problem &p, const GreyArgs &a);
size_t restrict_scratch_doubles(int nx, int n_from, int n_to);
cudaError_t launch_grey(const Problem &p, const Level &g, const GreyArgs &a);
cudaError_t launch_group_sum(const Problem &p, int n, const double *X, double *out);

}  // namespace trt
