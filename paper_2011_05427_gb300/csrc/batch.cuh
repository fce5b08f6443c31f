// batch.cuh -- argument blocks of the kernels and their batched (many slabs, one launch)
// entry points.
//
// Every kernel has a device body that takes its argument block and explicit block
// coordinates.  The single-slab kernel passes blockIdx; the batched kernel walks a work
// list: an op's metadata in device memory is
//     meta = [n, pre[0..N], gx[0..N), sid[0..N)]      (ints, N = slabs the batch holds)
// where participant j (of n <= N) is slab sid[j] (argument block xs[sid[j]]), owns blocks
// pre[j] .. pre[j+1]-1, and its block l has coordinates (l % gx[j], l / gx[j]).  The
// batched grid is fixed (by the largest work list any step can have) and strides over
// the list, so a CUDA graph of the launches stays valid while the participant set shrinks
// as slabs converge; blocks past pre[n] leave at once.
#pragma once
#include <algorithm>
#include "common.cuh"
#include "pair.cuh"

namespace trt {

// ---- argument blocks ----
struct OpacityArgs {
    int nx, G;
    const double *T, *edges;
    double s;
    double *sigE, *emis, *sigR;
    float *sig32, *emis32;   // FP32 sweep inputs (sigma_E + 1/(c dt)) h/2, h e/2, or null
    float *kap32;            // FP32 sweep input h/(2 c dt) per cell, or null
    const double *h;
    double icdt;
    const double *otab;      // Problem::otab (sigma_E, sigma_R series scaled by 27 s)
    double kE;               // 27 s C_B: the emission factor of the tabulated path
    const double *Erad;      // radiation energy per cell: sigma_E, sigma_R at T_r, or null
    const int *gate;         // Problem::gate (single-slab kernel only)
    double *cterm;           // Problem::cterm: per-cell terms (single-slab kernel only)
    // the pair form (TRT_LO_PAIR), when otabp is non-null: Problem::otabp and ::cpair (the
    // latter single-slab only), and 1/(c dt) split into two floats on the host
    const fpair *otabp;
    fpair *cpair;
    float icdt_h, icdt_l;
};

struct SweepArgs {
    int nx, N, G, ldG, D;
    double icdt;
    const double *h, *mu, *w, *Iin0, *IinX;
    const void *sigE, *emis;   // [G][nx], SR-typed
    const void *I_old;
    void *I_new;
    void *part;       // [n_dt][2][G][nx], R-typed
    void *psi_exit;   // [M][ldG], R-typed
    double *f, *fb0, *fbX, *C0, *CX;
    const float *kap32;   // h/(2 c dt) per cell in FP32 (with the FP32 inputs), or null
    const float *dir32;   // [M][4] |mu|, |mu|/2, w/2, w mu^2/2 in FP32
    double *ts;           // paired FP64 sweep: t, s per (|mu|, cell, group), or null
    double *tab64;        // paired FP64 sweep: its pre-scaled inputs (2 nx ldG + nx), or null
};

struct FinalizeArgs {
    int nx, N, G, ldG, ntile, nb_cell;
    const void *part, *psi_exit;   // R-typed
    const double *mu, *w, *Iin0, *IinX;
    double *f, *fb0, *fbX, *C0, *CX;
};

struct LoCtx {
    int nx;
    double dt, icdt, idt;   // dt, 1/(c dt), 1/dt
    const double *h, *ihf, *hf;
    const double *hc, *h2, *fwl, *fwr, *hidt, *dxicdt;   // Problem's LO row constants
    const int *lo_slot;
    const fpair *pc;   // Problem::lopc (the pair form's row constants), or null
    Level L;
    const double *a_cell, *s_cell;   // grey: explicit absorption / source per cell
    const int *gate;                 // Problem::gate (single-slab kernels only)
};

struct RestrictCtx {
    int nx, r;       // r = members per coarse group
    const double *h, *ihf;
    Level S;         // source level (coefficients + solution)
    Level T;         // target level (written)
    const int *gate;
};

struct Restrict2Ctx {
    int nx, r, nchunk;
    const double *h, *ihf;
    Level S, T;
    double *part;   // [n_to][nchunk][kRP][nx+1]
    const int *gate;
    // the grey visit's per-cell Newton terms, formed by the final stage when newton != 0
    // (single slab, target = the grey level): into pre [3][nx], with the visit's arguments
    int newton;
    GreyArgs ga;
    double *pre;
    // the target's Eold and Fold sums already hold this step's values from this source
    // (they change only between steps): stage 1 neither loads nor sums them, stage 2 keeps
    // them
    int skip_old;
};

struct GreyCtx {
    LoCtx lo;
    GreyArgs a;
    int mmax;
};

struct CopyArgs {
    double *dst;
    const double *src;
    long n;
};

struct GroupSumArgs {
    int n, nx;
    const double *X;
    double *out;
};

// ---- work-list decoding ----
inline size_t bmeta_ints(int N) { return (size_t)3 * N + 2; }

__device__ inline bool bdecode(const int *__restrict__ meta, int N, int b, int &s, int &bx,
                               int &by)
{
    const int n = meta[0];
    const int *pre = meta + 1;
    const int *gx = meta + 2 + N;
    if (n <= 0 || b >= pre[n]) return false;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    const int l = b - pre[lo];
    bx = l % gx[lo];
    by = l / gx[lo];
    s = meta[2 + 2 * N + lo];
    return true;
}

// ---- host-side argument builders (the single-slab launchers use the same) ----
inline int lo_mmax_h(int nx)
{
    return nx < 2 ? 1 : (nx + (std::min(32, nx / 2)) - 1) / std::min(32, nx / 2) + 1;
}
OpacityArgs make_opacity_args(const Problem &p, const double *T, double *sigE, double *emis,
                              double *sigR, float *sig32, float *emis32, double dt,
                              const double *Erad = nullptr);
int opacity_blocks(const Problem &p);
int opacity_gx(const Problem &p);   // blocks along the cells (32 cells x 8 groups each)
SweepArgs make_sweep_args(const Problem &p, double dt, const void *sigE, const void *emis,
                          const void *I_old, void *I_new, double *part, double *psi_exit,
                          double *f, double *fb0, double *fbX, double *C0, double *CX, int D);
FinalizeArgs make_finalize_args(const Problem &p, const SweepArgs &a);
int finalize_blocks(const Problem &p);
int pick_D(const Problem &p);   // directions per CTA of the single-slab sweep
LoCtx make_lo_ctx(const Problem &p, double dt, const Level &L);
// restriction: kind 2 (two-stage) when the source has >= 64 members per coarse group and
// the scratch holds it, else kind 1 with KS row slices per CTA
int restrict_kind(const Problem &p, int n_from, int n_to, int *KS);
RestrictCtx make_restrict_ctx(const Problem &p, const Level &src, const Level &dst);
Restrict2Ctx make_restrict2_ctx(const Problem &p, const Level &src, const Level &dst);
int restrict2_nchunk(int n_from, int n_to);
GreyCtx make_grey_ctx(const Problem &p, const Level &g, const GreyArgs &a);

// ---- batched launchers (grid: CTAs of the fixed grid; stream: the batch's stream) ----
cudaError_t launch_opacity_b(const int *meta, int N, const OpacityArgs *xs, int grid,
                             cudaStream_t st);
// sweep and its finalize: every participant uses the same R/SR types, D and shape
cudaError_t launch_sweep_b(int precision, bool sigma_fp32, int D, int shape, const int *meta,
                           int N, const SweepArgs *xs, int grid, cudaStream_t st);
cudaError_t launch_finalize_b(int precision, const int *meta, int N, const FinalizeArgs *xs,
                              int grid, cudaStream_t st);
cudaError_t launch_lo_solve_b(int precision, int max_nx, const int *meta, int N,
                              const LoCtx *xs, int grid, cudaStream_t st);
cudaError_t launch_restrict_b(int KS, const int *meta, int N, const RestrictCtx *xs, int grid,
                              cudaStream_t st);
cudaError_t launch_restrict_part_b(const int *meta, int N, const Restrict2Ctx *xs, int grid,
                                   cudaStream_t st);
cudaError_t launch_restrict_final_b(const int *meta, int N, const Restrict2Ctx *xs, int grid,
                                    cudaStream_t st);
cudaError_t launch_grey_b(int max_nx, const int *meta, int N, const GreyCtx *xs, int grid,
                          cudaStream_t st);
cudaError_t launch_group_sum_b(const int *meta, int N, const GroupSumArgs *xs, int grid,
                               cudaStream_t st);
cudaError_t launch_copy_b(const int *meta, int N, const CopyArgs *xs, int grid, cudaStream_t st);

}  // namespace trt
