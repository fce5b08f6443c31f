// sweepf.cu -- lean FP32 S_N sweep on the step's pre-scaled FP32 inputs (kernel K2, FP32).
//
// Same discretisation as sweep.cu: eq. rt with implicit Euler (Sec. 5), simple corner
// balance in a 1D slab; per (cell, group, direction) the 2x2 corner system
//   [ a  b ] [psi_L]   [r_L]        a = |mu|/2 + sigma_t h/2,  b = |mu|/2,
//   [-b  a ] [psi_R] = [r_R],       r = (h/2) e_g + (h/(2 c dt)) I^{j-1} (+ |mu| psi_in on
//                                   the inflow corner),
// solved as psi_L = t r_L - s r_R, psi_R = s r_L + t r_R (mu > 0; mirrored for mu < 0)
// with t = a/det, s = b/det, det = a^2 + b^2.  t and s do not depend on the inflow, so the
// recurrence from one cell to the next is two dependent FMAs.
//
// Layout and schedule.  A CTA owns W = 32 GPL consecutive groups (GPL per lane) and D
// directions of one sign (one warp each; D = 4, 8 or 16).  Cells go in strips of S aligned
// to multiples of S from cell 0 (a ragged strip is the last one for mu > 0 and the first
// for mu < 0); each strip's intensity rows (16-byte copies, a warp-wide copy moving 4 / GPL
// rows), sigma_t h/2, h e/2 and h/(2 c dt) arrive by cp.async NS - 1 strips ahead.  Full strips run fully unrolled for one direction sign at a time, so every
// shared-memory operand is a constant offset from a per-strip base; the warp leaves
// psi_L + psi_R of the strip in one of two buffers, and the CTA reduces the previous
// strip's buffer into the two angular moments per (cell, group) right after the one
// barrier per strip -- with two buffers a strip needs a single __syncthreads.  The moment
// sums take the D directions in order with the compensated accumulator of the other FP32
// sweeps.  Every rounding is explicit (__f*_rn), so the single-slab and the batched kernel
// agree bit for bit.
#include <type_traits>
#include "sweep.cuh"

namespace trt {

namespace {

// 1/d for a normal d > 0 with a normal reciprocal (d is the determinant a^2 + b^2 >= mu^2/4
// below 2^126): the hardware approximation (rcp.approx: within 1 ulp per the PTX ISA)
// refined by one Newton-Raphson step x + x (1 - d x), which squares its relative error.
__device__ __forceinline__ float rcp_nr(float d)
{
    float x;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(x) : "f"(d));
    return __fmaf_rn(x, __fmaf_rn(-d, x, 1.f), x);
}

// 16-byte cp.async that bypasses L1 (each intensity row is read once)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}

template <int GPL>
struct Vec;
template <>
struct Vec<1> {
    using T = float;    // one group's value
    using F = float2;   // (sigma_t h/2, h e/2) of one group
    static __device__ __forceinline__ float get(const T &v, int) { return v; }
    static __device__ __forceinline__ float th(const F &f, int) { return f.x; }
    static __device__ __forceinline__ float q(const F &f, int) { return f.y; }
    static __device__ __forceinline__ T make(const float *x) { return x[0]; }
};
template <>
struct Vec<2> {
    using T = float2;
    using F = float4;   // (sigma_t h/2 of both groups, h e/2 of both groups)
    static __device__ __forceinline__ float get(const T &v, int j) { return j ? v.y : v.x; }
    static __device__ __forceinline__ float th(const F &f, int j) { return j ? f.y : f.x; }
    static __device__ __forceinline__ float q(const F &f, int j) { return j ? f.w : f.z; }
    static __device__ __forceinline__ T make(const float *x) { return make_float2(x[0], x[1]); }
};

template <int GPL, int S, int NS, int D>
struct SweepFSmem {
    static constexpr int W = 32 * GPL;          // groups per CTA
    static constexpr int P = W + 32 / S;        // padded moment row: the reduction's
                                                // (group, cell) reads hit 32 distinct banks
    static constexpr int PF = 2 * W + 8;        // field row: per lane GPL x sigma_t h/2 then
                                                // GPL x h e/2 (one vector load per cell)
    static constexpr size_t itile = 0;                                           // [NS][D][S][2][W]
    static constexpr size_t fld = itile + sizeof(float) * NS * D * S * 2 * W;    // [NS][S][PF]
    static constexpr size_t kap = fld + sizeof(float) * NS * S * PF;             // [NS][S]
    static constexpr size_t ps = kap + sizeof(float) * NS * S;                   // [2][D][S][P]
    static constexpr size_t total = ps + sizeof(float) * 2 * D * S * P;
    // CTAs per SM that shared memory allows (228 KB, 1 KB reserved per CTA): the register
    // budget is set to match, so registers never hold residency below it
    static constexpr int minb = (int)(228 * 1024 / (total + 1024)) > 8
                                    ? 8 : (int)(228 * 1024 / (total + 1024));
    static_assert(NS >= 2 && (S & (S - 1)) == 0 && S >= 4 && S <= 32, "strip shape");
    static_assert(((S * P * 4) % 16) == 0 && ((NS * S * 4) % 16) == 0, "16-byte sections");
};

template <int GPL, int S, int NS, int D, bool POS>
__device__ __forceinline__ void sweepf_run(const SweepArgs &a, int dtile, int gt)
{
    using L = SweepFSmem<GPL, S, NS, D>;
    using V = Vec<GPL>;
    using VT = typename V::T;
    using VF = typename V::F;
    constexpr int W = L::W, P = L::P, PF = L::PF, NT = 32 * D;
    constexpr int CH = W / 4;          // 16-byte chunks per intensity row
    constexpr int RPI = 32 / CH;       // rows per warp-wide copy (4 / GPL)
    constexpr int NI = 2 * S / RPI;    // warp-wide copies per full strip
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *itile = reinterpret_cast<float *>(smem_raw + L::itile);
    float *fld = reinterpret_cast<float *>(smem_raw + L::fld);
    float *skap = reinterpret_cast<float *>(smem_raw + L::kap);
    float *ps = reinterpret_cast<float *>(smem_raw + L::ps);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nx = a.nx, G = a.G, ldG = a.ldG;
    const int gb = gt * W;               // the CTA's first group
    const int g0 = gb + GPL * lane;      // this lane's first group in the sweep
    const bool lv = g0 < ldG;            // inside the padded row (ldG is a multiple of 32)
    const int m0 = dtile * D, m = m0 + warp;
    const int rr = lane / CH, ch = lane % CH;   // this lane's row and chunk in the copies
    const bool cv = gb + 4 * ch < ldG;

    const float *__restrict__ sigE = reinterpret_cast<const float *>(a.sigE);
    const float *__restrict__ emis = reinterpret_cast<const float *>(a.emis);
    const float *__restrict__ kap32 = a.kap32;
    float *part = reinterpret_cast<float *>(a.part);
    const size_t lo_off = (size_t)(2 * a.N / D) * 2 * G * nx;   // low parts of the partials
    const unsigned ds = 2u * (unsigned)ldG;   // one cell of one direction, in floats
    const size_t mrow = (size_t)m * nx * ds;
    // copy source of this lane: row rr (cell rr / 2, corner rr % 2), chunk ch
    const float *Isrc = reinterpret_cast<const float *>(a.I_old) + mrow + (rr >> 1) * ds +
                        (rr & 1) * ldG + gb + 4 * ch;
    float *Inew_m = reinterpret_cast<float *>(a.I_new) + mrow + g0;

    const float4 *dir = reinterpret_cast<const float4 *>(a.dir32);
    const float4 dm = dir[m];
    const float am = dm.x, b = dm.y, bb = __fmul_rn(b, b);
    float wt[D], wm[D];   // w/2 and w mu^2/2 of the tile's directions (moment weights)
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const float4 dd = dir[m0 + d];
        wt[d] = dd.z;
        wm[d] = dd.w;
    }
    const double *Iin = POS ? a.Iin0 : a.IinX;
    float psi[GPL];
#pragma unroll
    for (int j = 0; j < GPL; ++j) psi[j] = (g0 + j < G) ? (float)Iin[g0 + j] : 0.f;

    const int nstrip = (nx + S - 1) / S;
    auto range = [&](int st, int &c0, int &ns) {
        c0 = (POS ? st : nstrip - 1 - st) * S;
        ns = min(S, nx - c0);
    };
    // chunks past the padded row are never copied: zero them once in every buffer
    if (!cv) {
        for (int k = 0; k < NS * NI; ++k) {
            const int bf = k / NI, r = (k % NI) * RPI + rr;
            *reinterpret_cast<float4 *>(itile + ((size_t)(bf * D + warp) * S * 2 + r) * W +
                                        4 * ch) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    auto prefetch = [&](int st, int bf) {
        int c0, ns;
        range(st, c0, ns);
        if (cv) {
            float *it = itile + ((size_t)(bf * D + warp) * S * 2 + rr) * W + 4 * ch;
            const float *src = Isrc + (size_t)c0 * ds;
            if (ns == S) {
#pragma unroll
                for (int k = 0; k < NI; ++k)
                    cp_async16(it + k * RPI * W, src + k * (RPI / 2) * ds);
            } else {
                for (int k = 0; k < NI; ++k)
                    if (k * (RPI / 2) + (rr >> 1) < ns)
                        cp_async16(it + k * RPI * W, src + k * (RPI / 2) * ds);
            }
        }
        float *fl = fld + bf * S * PF;
#pragma unroll
        for (int k = 0; k < (W * S + NT - 1) / NT; ++k) {
            const int idx = tid + k * NT;
            if ((W * S) % NT == 0 || idx < W * S) {
                const int gl = idx / S, cc = idx % S;
                const int gg = gb + gl;
                float *slot = fl + cc * PF + (gl / GPL) * 2 * GPL + gl % GPL;
                if (cc < ns && gg < G) {
                    cp_async<4>(slot, sigE + (size_t)gg * nx + c0 + cc);
                    cp_async<4>(slot + GPL, emis + (size_t)gg * nx + c0 + cc);
                } else {
                    slot[0] = 0.f;
                    slot[GPL] = 0.f;
                }
            }
        }
        if (tid < ns) cp_async<4>(skap + bf * S + tid, kap32 + c0 + tid);
        cp_commit();
    };

    // the CTA's angular moments of strip (c0, ns) from buffer pb: one (cell, group) per
    // thread and pass, directions in order; a warp stores S consecutive cells of each of
    // 32 / S groups (one 4 S-byte segment per group)
    auto reduce = [&](const float *pb, int c0, int ns) {
#pragma unroll
        for (int k = 0; k < (W * S + NT - 1) / NT; ++k) {
            const int idx = tid + k * NT;
            if ((W * S) % NT == 0 || idx < W * S) {
                const int gl = idx / S, cc = idx % S;
                const int gg = gb + gl;
                if (cc < ns && gg < G) {
                    Acc<float> s0, s2;
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        const float v = pb[(d * S + cc) * P + gl];
                        s0.add(__fmul_rn(wt[d], v));
                        s2.add(__fmul_rn(wm[d], v));
                    }
                    // the compensated sums as (high, low) pairs: the high parts in the
                    // tile's plane, the low parts (-c) in a second set of planes after
                    // every tile's (the finalize adds them in FP64)
                    const size_t o = ((size_t)(dtile * 2 + 0) * G + gg) * nx + c0 + cc;
                    part[o] = s0.s;
                    part[o + (size_t)G * nx] = s2.s;
                    part[lo_off + o] = -s0.c;
                    part[lo_off + o + (size_t)G * nx] = -s2.c;
                }
            }
        }
    };

    // one cell of the strip: the GPL recurrences of this lane
    auto cell = [&](int cc, float kap, const float *it, const float *fl, float *pw, float *oL,
                    float *oR) {
        const VT IL = *reinterpret_cast<const VT *>(it + cc * 2 * W);
        const VT IR = *reinterpret_cast<const VT *>(it + cc * 2 * W + W);
        const VF f = *reinterpret_cast<const VF *>(fl + cc * PF);
        float pL[GPL], pR[GPL], v[GPL];
#pragma unroll
        for (int j = 0; j < GPL; ++j) {
            const float th = V::th(f, j);
            const float aa = __fadd_rn(b, th);
            const float x = rcp_nr(__fmaf_rn(aa, aa, bb));
            const float t = __fmul_rn(aa, x), s = __fmul_rn(b, x);
            const float kL = __fmaf_rn(kap, V::get(IL, j), V::q(f, j));
            const float kR = __fmaf_rn(kap, V::get(IR, j), V::q(f, j));
            // the outflow is tau psi_in + q with tau = |mu| s = 1 - eps, eps = th (th + |mu|)
            // / det.  In a thin cell (eps < 1/2) it is formed as psi_in + (q - eps psi_in):
            // tau's rounding would otherwise repeat in every cell of a streaming path
            // (coherently where the cells are alike); in a thick cell as s r + t k, whose
            // relative error stays small when tau is.
            const float eps = __fmul_rn(__fmul_rn(th, __fadd_rn(th, am)), x);
            if (POS) {
                const float rL = __fmaf_rn(am, psi[j], kL);
                const float inc = __fadd_rn(psi[j], __fmaf_rn(-eps, psi[j], __fmaf_rn(s, kL, __fmul_rn(t, kR))));
                pR[j] = eps < 0.5f ? inc : __fmaf_rn(s, rL, __fmul_rn(t, kR));
                pL[j] = __fmaf_rn(t, rL, -__fmul_rn(s, kR));
                psi[j] = pR[j];
            } else {
                const float rR = __fmaf_rn(am, psi[j], kR);
                const float inc = __fadd_rn(psi[j], __fmaf_rn(-eps, psi[j], __fmaf_rn(s, kR, __fmul_rn(t, kL))));
                pL[j] = eps < 0.5f ? inc : __fmaf_rn(s, rR, __fmul_rn(t, kL));
                pR[j] = __fmaf_rn(t, rR, -__fmul_rn(s, kL));
                psi[j] = pL[j];
            }
            v[j] = __fadd_rn(pL[j], pR[j]);
        }
        if (lv) {
            *reinterpret_cast<VT *>(oL + cc * ds) = V::make(pL);
            *reinterpret_cast<VT *>(oR + cc * ds) = V::make(pR);
        }
        *reinterpret_cast<VT *>(pw + cc * P) = V::make(v);
    };

    for (int k = 0; k < NS - 1; ++k) {
        if (k < nstrip)
            prefetch(k, k);
        else
            cp_commit();   // empty groups keep the wait count uniform
    }
    int pc0 = 0, pns = 0;   // the previous strip, reduced in this iteration
    for (int st = 0; st < nstrip; ++st) {
        const int bf = st % NS;
        int c0, ns;
        range(st, c0, ns);
        cp_wait<NS - 2>();   // NS - 1 + st groups committed; strip st's is the (st+1)-th
        __syncthreads();     // everyone's copies of strip st landed; strip st - 1 swept
        // into the buffer that held strip st - 1
        if (st + NS - 1 < nstrip)
            prefetch(st + NS - 1, (st + NS - 1) % NS);
        else
            cp_commit();
        if (st > 0) reduce(ps + ((st - 1) & 1) * D * S * P, pc0, pns);
        const float *it = itile + ((size_t)(bf * D + warp) * S) * 2 * W + GPL * lane;
        const float *fl = fld + bf * S * PF + 2 * GPL * lane;
        const float *kp = skap + bf * S;
        float *pw = ps + ((size_t)((st & 1) * D + warp) * S) * P + GPL * lane;
        float *oL = Inew_m + (size_t)c0 * ds, *oR = oL + ldG;
        if (ns == S) {
            float kr[S];   // the strip's h/(2 c dt), four cells per load
#pragma unroll
            for (int k = 0; k < S; k += 4) {
                const float4 k4 = *reinterpret_cast<const float4 *>(kp + k);
                kr[k] = k4.x; kr[k + 1] = k4.y; kr[k + 2] = k4.z; kr[k + 3] = k4.w;
            }
#pragma unroll
            for (int k = 0; k < S; ++k) {
                const int cc = POS ? k : S - 1 - k;
                cell(cc, kr[cc], it, fl, pw, oL, oR);
            }
        } else {
            for (int k = 0; k < ns; ++k) {
                const int cc = POS ? k : ns - 1 - k;
                cell(cc, kp[cc], it, fl, pw, oL, oR);
            }
        }
        pc0 = c0;
        pns = ns;
    }
    __syncthreads();
    reduce(ps + ((nstrip - 1) & 1) * D * S * P, pc0, pns);
    if (lv) {
        float *pe = reinterpret_cast<float *>(a.psi_exit) + (size_t)m * ldG + g0;
        *reinterpret_cast<VT *>(pe) = V::make(psi);
    }
}

template <int GPL, int S, int NS, int D>
__device__ __forceinline__ void sweepf_body(const SweepArgs &a, int dtile, int gt)
{
    if (dtile < a.N / D)
        sweepf_run<GPL, S, NS, D, true>(a, dtile, gt);
    else
        sweepf_run<GPL, S, NS, D, false>(a, dtile, gt);
}

template <int GPL, int S, int NS, int D>
__global__ void __launch_bounds__(32 * D, (SweepFSmem<GPL, S, NS, D>::minb))
k_sweepf(SweepArgs a)
{
    griddep_wait();
    sweepf_body<GPL, S, NS, D>(a, blockIdx.x, blockIdx.y);
}

template <int GPL, int S, int NS, int D>
__global__ void __launch_bounds__(32 * D, (SweepFSmem<GPL, S, NS, D>::minb))
k_sweepf_b(const int *__restrict__ meta, int N, const SweepArgs *__restrict__ xs)
{
    for (int b = blockIdx.x;; b += gridDim.x) {
        int s, bx, by;
        if (!bdecode(meta, N, b, s, bx, by)) break;
        const SweepArgs a = xs[s];
        sweepf_body<GPL, S, NS, D>(a, bx, by);
        __syncthreads();   // shared memory is reused by the next work item
    }
}

template <int GPL, int S, int NS, int D>
cudaError_t launch_f(const SweepArgs *a, int M, int ldG, const int *meta, int N,
                     const SweepArgs *xs, int grid, cudaStream_t st)
{
    constexpr size_t sm = SweepFSmem<GPL, S, NS, D>::total;
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
    constexpr int W = 32 * GPL;
    if (a) {
        cudaError_t e = cudaFuncSetAttribute(k_sweepf<GPL, S, NS, D>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        return launch_pdl(k_sweepf<GPL, S, NS, D>, dim3(M / D, (ldG + W - 1) / W), dim3(32 * D),
                          sm, st, *a);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_sweepf_b<GPL, S, NS, D>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_sweepf_b<GPL, S, NS, D><<<grid, 32 * D, sm, st>>>(meta, N, xs);
    }
    return cudaGetLastError();
}

template <int GPL, int S, int NS>
cudaError_t launch_fd(int D, const SweepArgs *a, int M, int ldG, const int *meta, int N,
                      const SweepArgs *xs, int grid, cudaStream_t st)
{
    switch (D) {
    case 4: return launch_f<GPL, S, NS, 4>(a, M, ldG, meta, N, xs, grid, st);
    case 8: return launch_f<GPL, S, NS, 8>(a, M, ldG, meta, N, xs, grid, st);
    case 16: return launch_f<GPL, S, NS, 16>(a, M, ldG, meta, N, xs, grid, st);
    default: return cudaErrorInvalidConfiguration;
    }
}

}  // namespace

size_t sweepf_smem(int kind, int S, int NS, int D)
{
    auto pick = [&](auto gpl, auto s, auto ns) -> size_t {
        constexpr int G_ = decltype(gpl)::value, S_ = decltype(s)::value, N_ = decltype(ns)::value;
        switch (D) {
        case 4: return SweepFSmem<G_, S_, N_, 4>::total;
        case 8: return SweepFSmem<G_, S_, N_, 8>::total;
        case 16: return SweepFSmem<G_, S_, N_, 16>::total;
        default: return 0;
        }
    };
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    using I3 = std::integral_constant<int, 3>;
    using I4 = std::integral_constant<int, 4>;
    using I8 = std::integral_constant<int, 8>;
    using I16 = std::integral_constant<int, 16>;
    if (kind == 5 && S == 16 && NS == 2) return pick(I1(), I16(), I2());
    if (kind == 5 && S == 8 && NS == 3) return pick(I1(), I8(), I3());
    if (kind == 5 && S == 8 && NS == 2) return pick(I1(), I8(), I2());
    if (kind == 5 && S == 8 && NS == 4) return pick(I1(), I8(), I4());
    if (kind == 6 && S == 8 && NS == 2) return pick(I2(), I8(), I2());
    if (kind == 6 && S == 8 && NS == 4) return pick(I2(), I8(), I4());
    return 0;
}

cudaError_t launch_sweepf(int kind, int S, int NS, const SweepArgs *a, int M, int ldG, int D,
                          const int *meta, int N, const SweepArgs *xs, int grid, cudaStream_t st)
{
    if (kind == 5 && S == 16 && NS == 2)
        return launch_fd<1, 16, 2>(D, a, M, ldG, meta, N, xs, grid, st);
    if (kind == 5 && S == 8 && NS == 3)
        return launch_fd<1, 8, 3>(D, a, M, ldG, meta, N, xs, grid, st);
    if (kind == 5 && S == 8 && NS == 2)
        return launch_fd<1, 8, 2>(D, a, M, ldG, meta, N, xs, grid, st);
    if (kind == 5 && S == 8 && NS == 4)
        return launch_fd<1, 8, 4>(D, a, M, ldG, meta, N, xs, grid, st);
    if (kind == 6 && S == 8 && NS == 2)
        return launch_fd<2, 8, 2>(D, a, M, ldG, meta, N, xs, grid, st);
    if (kind == 6 && S == 8 && NS == 4)
        return launch_fd<2, 8, 4>(D, a, M, ldG, meta, N, xs, grid, st);
    return cudaErrorInvalidConfiguration;
}

}  // namespace trt
