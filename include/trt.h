/*
 * trt.h -- C ABI of the GB300 (sm_103a) solver for thermal radiative transfer with the
 * multilevel quasidiffusion (QD / VEF) method and multigrid in photon frequency
 * (D. Y. Anistratov, "Nonlinear iterative projection methods with multigrid in photon
 * frequency for thermal radiative transfer", arXiv 2011.05427).
 *
 * Problem (Sec. 2, Sec. 6): 1D slab [0, X]; multigroup RT equation (eq. rt) with the
 * Fleck-Cummings opacity sigma(nu, T) = s 27/nu^3 (1 - e^{-nu/T}); material energy
 * eps = cv T (eq. eb); isotropic Planck inflow at x = 0 and x = X (vacuum when the
 * boundary temperature is <= 0); initial state T = T0, I_g = B_g(T0).
 * Method (Sec. 3-5, Algorithm 3): implicit Euler; simple-corner-balance S_N sweeps;
 * group LOQD equations on a hierarchy of frequency grids visited by V / W / F cycles;
 * effective grey LOQD coupled to the material energy balance, one Newton step per
 * temperature evaluation.
 *
 * Units: cm, sh (1e-8 s), keV, GJ.  c = 299.792458 cm/sh, aR = 0.01372 GJ/(cm^3 keV^4).
 *
 * Conventions for every entry point:
 *   - returns an int status: TRT_OK (0) or a negative TRT_E* code; no exceptions cross
 *     the ABI; after a non-fatal error (EINVAL, ENOTCONVERGED, ENUMERIC) the handle stays
 *     usable and trt_last_error() describes the failure;
 *   - "host" pointers are read or written with plain loads/stores; "device" pointers must
 *     be device memory of the handle's device; the caller owns all memory it passes;
 *   - the library allocates no device memory: all device state lives in the caller's
 *     workspace (trt_workspace_bytes), carved at trt_create; the only allocation the
 *     library makes is a small pinned host buffer per handle for convergence flags;
 *   - all device work is enqueued on the stream given in trt_options (0 = legacy stream);
 *   - array layouts (host and device):
 *       cell arrays     [G][nx]            group-major, cell fastest
 *       face arrays     [G][nx+1]          face f at x_{f-1/2}: f = 0 is x = 0, f = nx is X
 *       intensity       [M][nx][2][ldG]    direction, cell, corner (0 left, 1 right), group
 *                                          (ldG from trt_dims, >= G, padding zero)
 *       directions      m < N: mu_m > 0 ascending; m >= N: mu_m = -mu_{m-N}  (M = 2N)
 */
#ifndef TRT_H
#define TRT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define TRT_OK              0
#define TRT_EINVAL         -1   /* bad argument; nothing was enqueued                   */
#define TRT_ENOTCONVERGED  -2   /* outer loop hit max_outer; the state is the last iterate */
#define TRT_ENUMERIC       -3   /* a temperature came out non-positive or non-finite     */
#define TRT_ETIMEOUT       -4   /* a bounded device wait gave up (trt_mlp.h kernels)     */
#define TRT_ECUDA          -5   /* a CUDA runtime call failed; see trt_last_error        */
#define TRT_ENOSPACE       -6   /* workspace smaller than trt_workspace_bytes            */

/* ---- precision modes (a bit mask) ---- */
#define TRT_FP64         0   /* every step in FP64                                          */
#define TRT_SWEEP_FP32   1   /* HO sweeps (intensity storage and arithmetic) in FP32         */
#define TRT_LO_FP32      2   /* fine and coarse group LOQD solves in FP32                     */
#define TRT_MIXED        3   /* both; opacities, restriction, grey LOQD, MEB Newton and the
                                convergence checks stay FP64                                 */
#define TRT_LO_PAIR      4   /* fine and coarse group LOQD solves in FP32-pair arithmetic
                                (~47 significant bits, FP32's exponent range; FP64 in and
                                out); excludes TRT_LO_FP32; with TRT_SWEEP_FP32: 5           */

/* ---- cycle types (Sec. 4, Fig. 1) ---- */
#define TRT_CYCLE_V 0   /* S empty: two-grid method on any hierarchy                      */
#define TRT_CYCLE_W 1   /* S = w(2), w(Gamma-1) = [Gamma-1], w(g) = w(g+1) + [g] + w(g+1)  */
#define TRT_CYCLE_F 2   /* S = [Gamma-1, ..., 2]                                           */

/* Spatial grid (Sec. 5 mesh), 1 <= n_cells <= 2048 (one warp-partitioned tridiagonal
 * system per group must fit in shared memory).  x_edges: host, n_cells+1 increasing
 * values, or NULL for a uniform mesh over [0, length_cm]. */
typedef struct {
    int n_cells;
    const double *x_edges;
    double length_cm;
    double T_left_keV;    /* isotropic Planck inflow at x = 0; <= 0 means vacuum */
    double T_right_keV;   /* isotropic Planck inflow at x = X; <= 0 means vacuum */
} trt_grid;

/* Angular quadrature (Sec. 6): double Gauss-Legendre, N nodes per half range, M = 2N. */
typedef struct {
    int N;
} trt_angles;

/* Frequency groups (eq. fine-grid, Sec. 4 hierarchy).  edges_keV: host, n_groups+1
 * increasing values, first 0, last may be INFINITY; NULL selects 0, n_groups-2 log-spaced
 * groups in [nu_a, nu_b], [nu_b, inf) (Sec. 6).  level_groups: host, n_levels values
 * n^1 = n_groups > n^2 > ... > n^Gamma = 1, each dividing the previous one (uniform
 * successive coarsening); NULL with n_levels = 0 selects {n_groups, 1}. */
typedef struct {
    int n_groups;
    const double *edges_keV;
    double nu_a, nu_b;
    int n_levels;
    const int *level_groups;
} trt_groups;

/* Opacity model (Sec. 6): sigma(nu, T) = scale * 27 / nu^3 * (1 - exp(-nu/T)) cm^-1.
 * tr_mode = 0: the group opacities at T_r = T (sigma_E,g = sigma_B,g); 1: sigma_E,g(T, T_r)
 * (Sec. 2) and sigma_R,g(T, T_r) (Sec. 3.1) at the radiation temperature T_r = (E/a_R)^{1/4}
 * of the latest grey energy E of the step (at its start the sum of the group energies);
 * single slabs only (trt_create_batch rejects it). */
typedef struct {
    double scale;
    int tr_mode;
} trt_opacity;

/* Options: precision (TRT_FP64 or an OR of TRT_SWEEP_FP32 / TRT_LO_FP32), initial
 * temperature, CUDA stream (cudaStream_t as void*),
 * caller-owned device workspace of at least trt_workspace_bytes bytes (256-B aligned). */
typedef struct {
    int precision;
    double T0_keV;
    void *stream;
    void *workspace;
    size_t workspace_bytes;
} trt_options;

/* Iteration controls of Algorithm 3.  eps: outer tolerance on ||dT||/||T|| and
 * ||dE||/||E|| (infinity norms, both must hold); eps_inner: the same per cycle; l_max:
 * cycles per low-order phase; max_outer: low-order phases per step (the first, s = 0, has
 * no sweep).  eps < 0 runs exactly max_outer phases of exactly l_max cycles. */
typedef struct {
    int type;
    int l_max;
    double eps;
    double eps_inner;
    int max_outer;
} trt_cycle;

/* Per-step counters (Sec. 6): sweeps, cycles, group-wise low-order solves (grey solves
 * count one each), low-order phases; wall time of the step on the host clock; number of
 * the library's kernel launches in the step. */
typedef struct {
    int n_ti, n_c, n_lo, n_outer;
    double ms;
    int status;
    int n_kernels;
} trt_stats;

typedef struct trt_handle trt_handle;

/* Bytes of device workspace trt_create needs for this problem (0 on invalid input). */
size_t trt_workspace_bytes(const trt_grid *grid, const trt_angles *angles,
                           const trt_groups *groups, const trt_options *opt);

/* Validate the problem, carve the workspace, upload constants and the initial state
 * (Sec. 6: T = T0, I = B_g(T0), E_g = (1/c) sum w I, F_g = sum w mu I, isotropic QD
 * factors).  Synchronises the stream before returning.  *out is NULL on failure. */
int trt_create(const trt_grid *grid, const trt_angles *angles, const trt_groups *groups,
               const trt_opacity *opacity, double cv, const trt_options *opt,
               trt_handle **out);

/* One implicit time step of length dt_sh with Algorithm 3.  Blocks on the stream once per
 * cycle to read the convergence flags.  stats may be NULL. */
int trt_step(trt_handle *h, double dt_sh, const trt_cycle *cycle, trt_stats *stats);

/* Copy the state at the current time level to host arrays (any may be NULL):
 * T [nx], E_g [G][nx], F_g [G][nx+1] (last fine solve), grey E [nx], F [nx+1] (last grey
 * solve).  Synchronises the stream. */
int trt_moments(trt_handle *h, double *T, double *Eg, double *Fg, double *E, double *F);

/* Host copy of the intensity [M][nx][2][ldG] as FP64 and the QD factors f_g [G][nx]; either
 * pointer may be NULL (that array is not copied). */
int trt_intensity(trt_handle *h, double *I, double *f);

/* Replace the state (host arrays, any may be NULL): temperature, E_g, F_g, intensity
 * [M][nx][2][ldG] and the QD factors f [G][nx], fb0, fbX, C0 (= C^- at 0), CX (= C^+ at X)
 * [G].  E_g also resets the grey E.  Used for restarts and tests. */
int trt_set_state(trt_handle *h, const double *T, const double *Eg, const double *Fg,
                  const double *I, const double *f, const double *fb0, const double *fbX,
                  const double *C0, const double *CX);

/* Problem dimensions: nx, N, M, G, ldG, number of grids, precision. */
int trt_dims(const trt_handle *h, int *nx, int *N, int *M, int *G, int *ldG, int *n_levels,
             int *precision);

/* Frees host objects only (the workspace belongs to the caller).  NULL is a no-op. */
int trt_destroy(trt_handle *h);

/* Last error message of this handle (or of the last failed create when h is NULL). */
const char *trt_last_error(const trt_handle *h);

/* ======================================================================================
 * Kernel-level entry points (device pointers, the handle's stream and dimensions).  Each
 * runs one step of the hot path on caller-provided device buffers, so that every kernel
 * can be checked on its own against the oracle.  They do not touch the handle's state.
 * ====================================================================================== */

/* Group physics at cell temperatures T [nx] (Sec. 2, Sec. 3.1, Sec. 6): sigma_E (=
 * sigma_B, T_r = T), emission e_g = sigma_B,g B_g and sigma_R, each [G][nx], FP64. */
int trt_k_opacity(trt_handle *h, const double *T, double *sigE, double *emis, double *sigR);

/* One HO sweep (eq. rt, simple corner balance, implicit Euler) of every group and
 * direction with sigma_t = sigE + 1/(c dt) and corner sources emis + I_old/(c dt), inflow
 * from the handle's boundary temperatures, followed by the QD factors (eqs. f_g, c_g).
 * I_old / I_new: [M][nx][2][ldG] in the handle's sweep precision (float when the
 * precision has TRT_SWEEP_FP32, else double).  f [G][nx]; fb0, fbX, C0, CX [G]; all FP64.
 * With TRT_SWEEP_FP32 the FP64 sigE and emis are first rounded once to the step's FP32
 * sweep inputs (sigma_t h/2, h e/2 and h/(2 c dt), in the handle's scratch), so the sweep
 * runs the same kernel and tile on the same inputs as a step would. */
int trt_k_sweep(trt_handle *h, double dt, const double *sigE, const double *emis,
                const void *I_old, void *I_new, double *f, double *fb0, double *fbX,
                double *C0, double *CX);

/* ---- learned closure (not in the paper; include/trt_mlp.h describes the network) ----
 * With a closure set, every trt_step starts its s = 0 low-order phase from QD factors
 * f_g predicted by the MLP from the step's initial state (T, sigma_E,g(T), E_g / E)
 * instead of the previous step's f_g; the sweeps then close the iteration as usual.
 * params (FP32 [TRT_MLP_NPARAM]) and w16 (BF16 copies, trt_mlp_refresh) are the
 * network; scratch (>= trt_mlp_scratch_bytes(G * n_cells, 0) bytes), x (FP32
 * [G * n_cells][3]) and y (FP32 [G * n_cells]) are work buffers.  All caller-owned device
 * memory that must outlive the steps; params 16-byte aligned (TRT_EINVAL otherwise).
 * params = NULL removes the closure. */
int trt_set_closure(trt_handle *h, const float *params, const void *w16, void *scratch,
                    size_t scratch_bytes, float *x, float *y);

/* ---- test aid: the device's exponential and reciprocal helpers ----
 * ex[i] = e^{x[i]} by the table-driven method the opacity kernel uses (Tang 1989) and
 * rc[i] = 1/x[i] by the refined hardware reciprocal, for accuracy tests against the C
 * library.  x, ex, rc: device arrays of n doubles; enqueued on `stream`. */
int trt_k_fastmath(int n, const double *x, double *ex, double *rc, void *stream);

/* ---- measurement aid: the device's FP64 FMA rate (the FP64 kernels' roofline) ----
 * Times one launch of independent FP64 FMA chains (8 per thread, `reps` steps each, as many
 * CTAs of 256 threads as every SM holds at once) with CUDA events on `stream` and writes
 * the rate in TFLOP/s (2 flops per FMA) to *tflops.  No counterpart in the paper.
 * Synchronises the stream. */
int trt_fp64_peak(int reps, void *stream, double *tflops);

/* ---- batched slabs (not in the paper: many independent problems at once) ----
 * n slabs, each as trt_create would take it (grids[s], angles[s], groups[s],
 * opacities[s], cv[s]; one trt_options for all: precision, T0, stream, workspace), step
 * together: trt_step_batch runs Algorithm 3 for every slab in lockstep -- each kernel
 * launch (opacities, sweep, its finalize, every group LOQD solve level, restriction, grey
 * Newton, state copies) covers all slabs taking part in it, through device-side work lists
 * built from per-slab flags; each stage of a step is captured once in a CUDA graph and
 * replayed (a graph needs a non-legacy stream).  Every slab's result is that of
 * trt_step on the same slab.  The learned closure is not available in a batch.
 *   - workspace: one caller-owned device buffer of trt_batch_workspace_bytes; slab s owns
 *     a slice; the batch allocates only pinned host staging buffers;
 *   - stats: n entries (or NULL); the return value is the first failing slab's status;
 *   - trt_batch_slab: the handle of slab s, for trt_moments / trt_intensity / trt_dims
 *     (do not destroy it: trt_destroy_batch does);
 *   - trt_batch_set_tile: directions per CTA D (a power of two dividing every slab's N,
 *     <= 8; 16 with FP32 sweeps, run by the lean sweep shapes only; TRT_EINVAL for a pair
 *     with no kernel or one over the CTA's shared memory) and sweep shape of the
 *     batched sweep; trt_batch_sweep_time: ms per batched
 *     sweep (all slabs, incl. the finalize), CUDA events, QD factors left unchanged. */
typedef struct trt_batch trt_batch;
size_t trt_batch_workspace_bytes(int n, const trt_grid *grids, const trt_angles *angles,
                                 const trt_groups *groups, const trt_options *opt);
int trt_create_batch(int n, const trt_grid *grids, const trt_angles *angles,
                     const trt_groups *groups, const trt_opacity *opacities, const double *cv,
                     const trt_options *opt, trt_batch **out);
int trt_step_batch(trt_batch *b, double dt_sh, const trt_cycle *cycle, trt_stats *stats);
trt_handle *trt_batch_slab(trt_batch *b, int s);
int trt_batch_set_tile(trt_batch *b, int D, int shape);
int trt_batch_sweep_time(trt_batch *b, double dt, int reps, float *ms);
int trt_destroy_batch(trt_batch *b);
const char *trt_batch_last_error(const trt_batch *b);

/* ---- sweep tile selection (a tuning aid; the paper has no counterpart) ----
 * The HO sweep (eq. rt, simple corner balance, Sec. 5) runs one warp per (32 groups,
 * direction); a CTA takes D directions of one sign and walks the cells in strips of S,
 * with NS strip buffers of asynchronous copies.  The best (D, S, NS) depends on the
 * problem's sizes and the precision.
 *
 * trt_sweep_time: the time of the step's own sweep on this handle -- opacities at the
 * current T (FP32 pre-scaled inputs in a FP32-sweep mode), then the sweep of the current
 * intensity into the handle's spare intensity buffer and scratch -- averaged over reps
 * launches (after one warm-up), CUDA events on the handle's stream.  The state (T, E_g,
 * F_g, I, QD factors) is left unchanged; call it between steps.  Needs n_cells >= 3.
 *   *ms: milliseconds per sweep (K2 + its moment finalize).
 * trt_autotune: times every candidate (D, S, NS) with trt_sweep_time and keeps the
 * fastest for later steps.  D, S, NS (may be NULL) receive the choice.
 * Both return TRT_EINVAL on bad arguments, TRT_ECUDA on a launch error. */
int trt_sweep_time(trt_handle *h, double dt, int reps, float *ms);
int trt_autotune(trt_handle *h, double dt, int reps, int *D, int *S, int *NS);
/* Set the sweep tile explicitly: D directions per CTA (a candidate of trt_autotune: the
 * largest power of two <= 4 dividing N, its double if <= 8 and dividing N, and with FP32
 * sweeps 16 if it divides N) and a shape index in [0, trt_sweep_shapes(h)); returns
 * TRT_EINVAL otherwise, and for a pair with no kernel (D = 16 runs on the lean FP32 shapes
 * only) or whose kernel would exceed the shared memory of a CTA; trt_autotune skips such
 * pairs. */
int trt_sweep_shapes(const trt_handle *h);
int trt_set_sweep_tile(trt_handle *h, int D, int shape);
/* The sweep tile the next step uses (after trt_autotune, trt_set_sweep_tile or neither):
 * *D = directions per CTA (0: the library's default for this problem), *shape = shape index.
 * Either pointer may be NULL.  TRT_EINVAL for a NULL handle. */
int trt_get_sweep_tile(const trt_handle *h, int *D, int *shape);

/* One frequency-grid level of the low-order system, device arrays (FP64).
 * fine = 0: a coarse or grey level with the arrays below.
 * fine = 1: the fine grid in its raw form: phi = f_g, sig = sigma_E, emis = e_g, and sigR is
 *           the CELL Rosseland opacity [n][nx] (faces take the dx-weighted mean of their two
 *           cells, boundary half faces the cell value); etaR / etaL are ignored (zero). 
 *   cell [n][nx]: phi (f or f-bar), sig (sigma_E or its average), emis (sum of
 *                 sigma_B B over the group), Eold (E at t^{j-1}), Esum (restriction output)
 *   face [n][nx+1]: sigR, etaR (eta-hat on E right of the face), etaL (eta-check on E left
 *                 of the face), Fold (F at t^{j-1})
 *   bound [n]: phib0, phibX (factor at x=0 / x=X), C0 (C^-), CX (C^+), Ein0, Fin0, EinX,
 *              FinX (inflow moments, eq. mloqd-bcs)
 *   solution: E [n][nx], F [n][nx+1], Eb0, EbX [n] (boundary-face energies). */
typedef struct {
    int n;
    int fine;
    double *phi, *sig, *emis, *Eold, *Esum;
    double *sigR, *etaR, *etaL, *Fold;
    double *phib0, *phibX, *C0, *CX, *Ein0, *Fin0, *EinX, *FinX;
    double *E, *F, *Eb0, *EbX;
} trt_level;

/* Solve every group of a level (eqs. mloqd-d / mloqd-d-gamma with absorption c sig and
 * source 2 emis) in the handle's LO precision; writes E, F, Eb0, EbX. */
int trt_k_lo_solve(trt_handle *h, double dt, trt_level *lv);

/* Test aid: the device arrays of the handle's own levels as the last step left them --
 * which = 0: the fine grid (its sigR field holds cell values, fine = 1), 1: the coarse
 * grid of the last coarse visit (n = its group count), 2: the grey grid (n = 1).  The
 * pointers stay valid while the handle lives; the arrays change with every step. */
int trt_level_view(trt_handle *h, int which, trt_level *out);

/* Restrict level `src` (its coefficients and solution) onto `dst` (dst->n groups, uniform
 * map p -> p / (src->n / dst->n)): eqs. coeff-gamma, eta-gamma, coeff-Gamma, eta-Gamma
 * with the discrete compensation of eq. mloqd-d-gamma.  Writes every coefficient of dst
 * and dst->Esum. */
int trt_k_restrict(trt_handle *h, const trt_level *src, trt_level *dst);

/* Grey LOQD + MEB, one Newton step (eq. eb-Gamma-d, eq. f-derivative-d) on the grey level
 * `g` (g->n == 1) at T* = Tstar [nx], with Q = 2 g->emis, E* = g->Esum, the secant from
 * (sig_prev, T_prev) when have_prev != 0 where T* != T_prev and |T* - T_prev| >
 * secant_cut T* (a step passes 0 when the previous grey solve was built on the same grid,
 * 1e-7 across grids).  Writes T [nx], g->E, g->F, g->Eb0, g->EbX.
 * Returns TRT_ENUMERIC if a temperature is non-positive or non-finite. */
/* The opacities at (T, T_r) of a T_r handle (tr_mode = 1): T [nx], radiation energies
 * Erad [nx] (T_r = (Erad/a_R)^{1/4}; Erad <= 0 or non-finite: T_r = T), outputs as
 * trt_k_opacity.  TRT_EINVAL on a handle without the T_r option. */
int trt_k_opacity_tr(trt_handle *h, const double *T, const double *Erad, double *sigE,
                     double *emis, double *sigR);

int trt_k_grey_newton(trt_handle *h, double dt, const double *Tstar, const double *Told,
                      const double *sig_prev, const double *T_prev, int have_prev,
                      double secant_cut, trt_level *g, double *T);

/* ======================================================================================
 * Allocation-free sweep.  The paper has no counterpart: this exists for callers that can
 * not allocate device memory -- a plug-in inside an application that owns every device
 * allocation and lends it no allocator, or a time loop that must not call cudaMalloc (nor
 * pay its device-wide synchronisation) once it is running.  trt_sweep_noalloc does the
 * work of trt_k_sweep (same kernels, the library's default sweep tile) with no handle and
 * no workspace: every input and output is a plain device pointer of the caller, and the
 * scratch the sweep needs (per-direction-tile angular partial sums, exit intensities and,
 * for FP32 sweeps, the per-direction FP32 constants and the pre-scaled FP32 inputs
 * (sigma_E + 1/(c dt)) h/2, h e/2 that trt_k_sweep forms on an FP32 handle) lives in one
 * file-scope static device array of TRT_STATIC_SCRATCH_BYTES, which every GPU that loads
 * the library keeps until exit.
 *   - sizes: nx cells, N directions per half range (M = 2N), G groups; intensities are
 *     [M][nx][2][ldG] with ldG = G rounded up to a multiple of 32 (float when precision
 *     has TRT_SWEEP_FP32, else double); h [nx], mu, w [M] (layout of trt.h), Iin0, IinX [G]
 *     isotropic inflow intensities, sigE, emis [G][nx] (FP64 in both precisions); outputs
 *     as for trt_k_sweep;
 *   - trt_sweep_noalloc_scratch_bytes gives the scratch a call of either precision needs;
 *     problems whose scratch exceeds the array are rejected with TRT_ENOSPACE before
 *     anything is enqueued;
 *   - the call only enqueues work on `stream` (cudaStream_t as void*) and returns; it
 *     allocates nothing -- no cudaMalloc / cudaFree, no library allocator;
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture;
 *   - all calls share the one array, which keeps whatever the last call left in it (each
 *     call writes every scratch value before it reads it, so nothing needs clearing);
 *     calls that overlap on the GPU -- on different streams, or from different host
 *     threads -- race on it and must be serialised by the caller;
 *   - on failure the message is in trt_sweep_noalloc_error(): the calling thread's last
 *     failure, valid until that thread's next call. */
#define TRT_STATIC_SCRATCH_BYTES (8u << 20)

size_t trt_sweep_noalloc_scratch_bytes(int nx, int N, int G);
int trt_sweep_noalloc(int nx, int N, int G, int precision, double dt, const double *h,
                      const double *mu, const double *w, const double *Iin0,
                      const double *IinX, const double *sigE, const double *emis,
                      const void *I_old, void *I_new, double *f, double *fb0, double *fbX,
                      double *C0, double *CX, void *stream);
const char *trt_sweep_noalloc_error(void);

#ifdef __cplusplus
}
#endif
#endif
