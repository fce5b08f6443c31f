// sweep.cu -- high-order multigroup S_N sweep and QD factors (kernel K2).
//
// Paper: eq. rt with implicit Euler (Sec. 5): sigma_t = sigma_E,g + 1/(c dt), corner
// sources S = e_g + I^{j-1}/(c dt); simple corner balance in a 1D slab (two corners per
// cell, the cell-centre value is the corner average, cell-edge values are upwinded):
//   mu > 0:  (|mu|/2 + sigma_t h/2) psi_L + (|mu|/2) psi_R = (h/2) S_L + |mu| psi_in
//           -(|mu|/2) psi_L + (|mu|/2 + sigma_t h/2) psi_R = (h/2) S_R         out: psi_R
//   mu < 0 mirrors it (inflow on the right corner, out: psi_L).
// Then eq. f_g (cell QD factor from the cell-average intensity) and eq. c_g (boundary
// factors C^- at x = 0 over mu < 0, C^+ at x = X over mu > 0), with the face factors at
// x = 0 and X from the face intensities (inflow from the boundary condition, outflow from
// the sweep); a zero denominator gives the isotropic value (1/3, -1/2, +1/2).
//
// GB300 mapping.  Every (group, direction) pair is an independent recurrence over cells.
// A CTA owns 32 consecutive groups (the lanes: the intensity layout [M][nx][2][ldG] makes
// each warp's corner load one contiguous 128/256-byte line) and D directions of one sign
// (one per warp), so all its warps walk the cells in the same order.  Cells go in strips
// of S: while a strip is swept, cp.async copies the next strip -- each warp's intensity
// tile and the CTA's sigma_E, e_g rows -- into the other half of a double buffer, so the
// serial recurrence never waits on global memory.  Each strip's sigma_t h/2 and
// (h/2) e_g are tabulated once per CTA in shared memory; each warp sweeps the strip and
// leaves psi_L + psi_R in shared memory; the CTA then reduces its D directions into the
// two angular moments per (cell, group) -- the cross-direction reduction costs one
// __syncthreads per strip, not one per cell.  Partial moments of the 2N/D direction tiles
// are summed in a fixed order by the finalize kernel (deterministic).
#include "sweep.cuh"

namespace trt {

namespace {

constexpr int kPadG = 33;   // padded group stride of the strip tables (bank conflicts)
// Tile shape: S cells per strip, NS strip buffers (NS - 1 strips of copies in flight while
// one is swept), D directions per CTA (runtime).  The grid holds one warp per
// (32 groups, direction) -- 2048 warps at 1024 groups x 64 directions, about 13 per SM --
// so the FP32 sweep is bound by how many bytes each warp keeps in flight; the shape is
// picked per problem by timing the candidates (trt_autotune), else the defaults below.



// 1/d.  FP32: the correctly rounded reciprocal.  FP64: the hardware's approximate FP64
// reciprocal x (relative error below 1e-6 = 2^-19.9, measured over [1, 2); special-function
// unit, not the FP64 pipe) refined by one third-order Newton-Raphson (Householder) step:
// with e = 1 - d x, x (1 + e + e^2) = (1 - eps^3)/d, below FP64 rounding (measured 1.1e-16;
// a second-order step leaves 1e-12), at 3 FP64 FMAs instead of the ~20 operations of an
// IEEE division -- FP64 issue rate bounds the FP64 sweep on GB300.
// d here is a determinant (mu/2 + sigma_t h/2)^2 + (mu/2)^2 > 0 of normal FP64 range.
template <typename R>
__device__ inline R recip(R d);
template <>
__device__ inline float recip<float>(float d) { return __frcp_rn(d); }
template <>
__device__ inline double recip<double>(double d)
{
    double x;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(d));
    const double e = fma(-d, x, 1.0);
    return fma(x, fma(e, e, e), x);
}

// shared-memory carve-up of k_sweep (byte offsets, 16-byte aligned sections)
template <typename R, typename SR, int kStrip, int NS>
struct SweepSmem {
    size_t itile, rawS, rawE, sth, sq, skap, ps, swt, total;
    __host__ __device__ SweepSmem(int D)
    {
        auto al = [](size_t x) { return (x + 15) / 16 * 16; };
        size_t o = 0;
        itile = o; o = al(o + sizeof(R) * NS * (size_t)D * kStrip * 2 * 32);
        rawS = o;  o = al(o + sizeof(SR) * NS * kStrip * kPadG);
        rawE = o;  o = al(o + sizeof(SR) * NS * kStrip * kPadG);
        sth = o;   o = al(o + sizeof(R) * kStrip * kPadG);
        sq = o;    o = al(o + sizeof(R) * kStrip * kPadG);
        skap = o;  o = al(o + sizeof(R) * kStrip);
        ps = o;    o = al(o + sizeof(R) * (size_t)D * kStrip * kPadG);
        swt = o;   o = al(o + sizeof(R) * 2 * D);
        total = o;
    }
};

// R: arithmetic and intensity type; SR: type of the fields read.  SR = double: the fields
// are sigma_E and e_g, tabulated per strip as sigma_t h/2 and h e/2 (FP64, one rounding);
// SR = float: the fields already are sigma_t h/2 and h e/2 in FP32 (written by the opacity
// kernel with one rounding each) and are used as staged.
template <typename R, typename SR, int kStrip, int NS>
__device__ void sweep_body(const SweepArgs &a, int dtile, int gt)
{
    constexpr bool kPre = sizeof(SR) == 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int D = a.D;
    const SweepSmem<R, SR, kStrip, NS> L(D);
    R *itile = reinterpret_cast<R *>(smem_raw + L.itile);      // [NS][D][S][2][32]
    SR *rawS = reinterpret_cast<SR *>(smem_raw + L.rawS);      // [NS][S][33] sigma_E
    SR *rawE = reinterpret_cast<SR *>(smem_raw + L.rawE);      // [NS][S][33] e_g
    R *sth = reinterpret_cast<R *>(smem_raw + L.sth);          // [S][33] sigma_t h / 2
    R *sq = reinterpret_cast<R *>(smem_raw + L.sq);            // [S][33] (h/2) e_g
    R *skap = reinterpret_cast<R *>(smem_raw + L.skap);        // [S]     h / (2 c dt)
    R *ps = reinterpret_cast<R *>(smem_raw + L.ps);            // [D][S][33] psi_L + psi_R
    R *swt = reinterpret_cast<R *>(smem_raw + L.swt);          // [D] w/2
    R *swm = swt + D;                                          // [D] w mu^2/2

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nthr = blockDim.x;
    const int tid = threadIdx.x;
    const int g = gt * 32 + lane;
    const int nx = a.nx, G = a.G, ldG = a.ldG;
    const bool pos = dtile < a.N / D;
    const int m = dtile * D + warp;

    const R *__restrict__ Iold = reinterpret_cast<const R *>(a.I_old);
    R *__restrict__ Inew = reinterpret_cast<R *>(a.I_new);
    const SR *__restrict__ sigE = reinterpret_cast<const SR *>(a.sigE);
    const SR *__restrict__ emis = reinterpret_cast<const SR *>(a.emis);
    R *part = reinterpret_cast<R *>(a.part);

    const double mu_d = a.mu[m];
    const R am = (R)fabs(mu_d);
    const R b = (R)(0.5 * fabs(mu_d));
    const R bb = b * b;
    if (lane == 0) {
        swt[warp] = (R)(0.5 * a.w[m]);
        swm[warp] = (R)(0.5 * a.w[m] * mu_d * mu_d);
    }
    R psi_in = (g < G) ? (R)(pos ? a.Iin0[g] : a.IinX[g]) : (R)0;

    const int nstrip = (nx + kStrip - 1) / kStrip;
    const size_t dstride = (size_t)2 * ldG;   // one cell of one direction
    const R *Iold_m = Iold + (size_t)m * nx * dstride + g;
    R *Inew_m = Inew + (size_t)m * nx * dstride + g;

    auto range = [&](int st, int &c0, int &ns) {
        if (pos) {
            c0 = st * kStrip;
            ns = min(kStrip, nx - c0);
        } else {
            const int c1 = nx - st * kStrip;
            c0 = max(c1 - kStrip, 0);
            ns = c1 - c0;
        }
    };
    auto prefetch = [&](int st, int bf) {
        int c0, ns;
        range(st, c0, ns);
        R *it = itile + ((size_t)bf * D + warp) * kStrip * 64 + lane;
        for (int cc = 0; cc < ns; ++cc) {
            cp_async<sizeof(R)>(it + cc * 64, Iold_m + (size_t)(c0 + cc) * dstride);
            cp_async<sizeof(R)>(it + cc * 64 + 32, Iold_m + (size_t)(c0 + cc) * dstride + ldG);
        }
        SR *rs = rawS + bf * kStrip * kPadG, *re = rawE + bf * kStrip * kPadG;
        for (int idx = tid; idx < 32 * kStrip; idx += nthr) {
            const int gl = idx / kStrip, cc = idx - gl * kStrip;
            const int gg = gt * 32 + gl;
            if (cc < ns && gg < G) {
                cp_async<sizeof(SR)>(rs + cc * kPadG + gl, sigE + (size_t)gg * nx + c0 + cc);
                cp_async<sizeof(SR)>(re + cc * kPadG + gl, emis + (size_t)gg * nx + c0 + cc);
            } else {
                rs[cc * kPadG + gl] = (SR)0;
                re[cc * kPadG + gl] = (SR)0;
            }
        }
        cp_commit();
    };

    for (int k = 0; k < NS - 1; ++k) {
        if (k < nstrip)
            prefetch(k, k);
        else
            cp_commit();   // empty groups keep the wait count uniform
    }
    for (int st = 0; st < nstrip; ++st) {
        const int bf = st % NS;
        int c0, ns;
        range(st, c0, ns);
        // the buffer of strip st + NS - 1 last held strip st - 1, consumed before the
        // barrier that ended the previous iteration's sweep
        if (st + NS - 1 < nstrip)
            prefetch(st + NS - 1, (st + NS - 1) % NS);
        else
            cp_commit();
        cp_wait<NS - 1>();   // this thread's copies of strip st have landed
        __syncthreads();     // ... and everyone's
        const SR *rs = rawS + bf * kStrip * kPadG, *re = rawE + bf * kStrip * kPadG;
        if (!kPre) {
            for (int idx = tid; idx < 32 * kStrip; idx += nthr) {
                const int gl = idx / kStrip, cc = idx - gl * kStrip;
                if (cc < ns) {
                    const double hh = 0.5 * a.h[c0 + cc];
                    sth[cc * kPadG + gl] = (R)(hh * ((double)rs[cc * kPadG + gl] + a.icdt));
                    sq[cc * kPadG + gl] = (R)(hh * (double)re[cc * kPadG + gl]);
                }
            }
        }
        if (tid < ns)
            skap[tid] = a.kap32 ? (R)a.kap32[c0 + tid] : (R)(0.5 * a.h[c0 + tid] * a.icdt);
        __syncthreads();
        const R *tth = kPre ? reinterpret_cast<const R *>(rs) : sth;
        const R *tq = kPre ? reinterpret_cast<const R *>(re) : sq;
        const R *it = itile + ((size_t)bf * D + warp) * kStrip * 64 + lane;
        R *psw = ps + warp * kStrip * kPadG;
#pragma unroll 4
        for (int kk = 0; kk < ns; ++kk) {
            const int cc = pos ? kk : ns - 1 - kk;
            const int i = c0 + cc;
            const R IL = it[cc * 64];
            const R IR = it[cc * 64 + 32];
            const R aa = b + tth[cc * kPadG + lane];
            const R inv = recip<R>(aa * aa + bb);
            const R q = tq[cc * kPadG + lane];
            const R kap = skap[cc];
            R pL, pR;
            if (pos) {
                const R rL = q + kap * IL + am * psi_in;
                const R rR = q + kap * IR;
                pL = (aa * rL - b * rR) * inv;
                pR = (aa * rR + b * rL) * inv;
                psi_in = pR;
            } else {
                const R rR = q + kap * IR + am * psi_in;
                const R rL = q + kap * IL;
                pR = (aa * rR - b * rL) * inv;
                pL = (aa * rL + b * rR) * inv;
                psi_in = pL;
            }
            Inew_m[(size_t)i * dstride] = pL;
            Inew_m[(size_t)i * dstride + ldG] = pR;
            psw[cc * kPadG + lane] = pL + pR;
        }
        __syncthreads();
        // angular moments of this tile: sum_d (w/2)(psi_L+psi_R), sum_d (w mu^2/2)(psi_L+psi_R)
        for (int idx = tid; idx < 32 * kStrip; idx += nthr) {
            const int gl = idx / kStrip, cc = idx - gl * kStrip;
            const int gg = gt * 32 + gl;
            if (cc < ns && gg < G) {
                Acc<R> s0, s2;
                for (int d = 0; d < D; ++d) {
                    const R v = ps[(d * kStrip + cc) * kPadG + gl];
                    s0.add(swt[d] * v);
                    s2.add(swm[d] * v);
                }
                const size_t o = ((size_t)(dtile * 2 + 0) * G + gg) * nx + c0 + cc;
                part[o] = s0.s;
                part[o + (size_t)G * nx] = s2.s;
                if (sizeof(R) == 4) {   // FP32: the low parts (-c) after every tile's planes
                    const size_t lo_off = (size_t)(2 * a.N / D) * 2 * G * nx;
                    part[lo_off + o] = -s0.c;
                    part[lo_off + o + (size_t)G * nx] = -s2.c;
                }
            }
        }
    }
    reinterpret_cast<R *>(a.psi_exit)[(size_t)m * ldG + g] = psi_in;
}

template <typename R, typename SR, int kStrip, int NS>
__global__ void __launch_bounds__(256) k_sweep(SweepArgs a)
{
    griddep_wait();
    sweep_body<R, SR, kStrip, NS>(a, blockIdx.x, blockIdx.y);
}

// batched: a persistent grid walks the (slab, direction tile, group tile) work list
template <typename R, typename SR, int kStrip, int NS>
__global__ void __launch_bounds__(256) k_sweep_b(const int *__restrict__ meta, int N,
                                                 const SweepArgs *__restrict__ xs)
{
    for (int b = blockIdx.x;; b += gridDim.x) {
        int s, bx, by;
        if (!bdecode(meta, N, b, s, bx, by)) break;
        const SweepArgs a = xs[s];
        sweep_body<R, SR, kStrip, NS>(a, bx, by);
        __syncthreads();   // shared memory is reused by the next work item
    }
}

// f_g = sum_t A2 / sum_t A0 per (group, cell), in R; boundary factors per group in FP64.
// Blocks [0, nb) with nb = ceil(G / 8) take one group per warp for the boundary factors;
// the blocks after them take one (group, cell) per thread.  The boundary warps come first so
// that their FP64 sums run beside the memory-bound cell blocks instead of after them: lanes
// stride over the directions, then the eight half-range sums meet in a halving exchange
// (lanes l and l ^ 16 trade four sums, then l ^ 8 two, l ^ 4 one, then l ^ 2 and l ^ 1 add
// the last one), which pairs the same lanes in the same order as a full butterfly of every
// sum -- the same totals bit for bit -- with 9 FP64 additions per lane instead of 40; lanes
// 0, 8, 16, 24 then hold the four denominators and form the four factors side by side.
template <typename R>
__device__ void finalize_body(const FinalizeArgs &x, int bx)
{
    const int nx = x.nx, N = x.N, G = x.G, ldG = x.ldG, ntile = x.ntile;
    const R *__restrict__ part = reinterpret_cast<const R *>(x.part);
    const R *__restrict__ psi_exit = reinterpret_cast<const R *>(x.psi_exit);
    const double *__restrict__ mu = x.mu, *__restrict__ w = x.w;
    const double *__restrict__ Iin0 = x.Iin0, *__restrict__ IinX = x.IinX;
    double *f = x.f, *fb0 = x.fb0, *fbX = x.fbX, *C0 = x.C0, *CX = x.CX;
    const int nb = finalize_bnd_blocks_dev(G);
    if (bx >= nb) {
        const long idx = (long)(bx - nb) * blockDim.x + threadIdx.x;
        const long n = (long)G * nx;
        if (idx < n) {
            if constexpr (sizeof(R) == 8) {
                // the tiles summed in order (tile count unrolled where it is a power of two
                // up to 16: every load issued before the first addition), then A2 times the
                // refined reciprocal of A0 (ratio64)
                const double *p = reinterpret_cast<const double *>(part) + idx;
                switch (ntile) {
                case 1: f[idx] = sum_tiles_ratio<1>(p, n); break;
                case 2: f[idx] = sum_tiles_ratio<2>(p, n); break;
                case 4: f[idx] = sum_tiles_ratio<4>(p, n); break;
                case 8: f[idx] = sum_tiles_ratio<8>(p, n); break;
                case 16: f[idx] = sum_tiles_ratio<16>(p, n); break;
                default: {
                    double A0 = 0.0, A2 = 0.0;
                    for (int t = 0; t < ntile; ++t) {
                        A0 += p[(size_t)(t * 2) * n];
                        A2 += p[(size_t)(t * 2 + 1) * n];
                    }
                    f[idx] = (A0 != 0.0) ? ratio64(A2, A0) : 1.0 / 3.0;
                }
                }
            } else {
                // FP32: the tiles' (high, low) pairs summed as unevaluated FP32 sums (an
                // exact two-sum per high part, the low parts added plainly), then the ratio
                // of the two unevaluated sums to about 2^-46 (pair_ratio) instead of the FP32
                // roundings of the partials and of an FP32 division
                const float *p = reinterpret_cast<const float *>(part) + idx;
                switch (ntile) {   // the tile count unrolled: no guards, loads in flight
                case 1: f[idx] = sum_pairs_ratio<1>(p, n); break;
                case 2: f[idx] = sum_pairs_ratio<2>(p, n); break;
                case 4: f[idx] = sum_pairs_ratio<4>(p, n); break;
                case 8: f[idx] = sum_pairs_ratio<8>(p, n); break;
                case 16: f[idx] = sum_pairs_ratio<16>(p, n); break;
                default: {
                    const size_t lo = (size_t)ntile * 2 * n;
                    float S0 = 0.f, E0 = 0.f, S2 = 0.f, E2 = 0.f;
                    for (int t = 0; t < ntile; ++t) {
                        const size_t o = (size_t)(t * 2) * n;
                        two_sum_acc(S0, E0, p[o], p[lo + o]);
                        two_sum_acc(S2, E2, p[o + n], p[lo + o + n]);
                    }
                    f[idx] = pair_ratio(S2, E2, S0, E0);
                }
                }
            }
        }
        return;
    }
    const int lane = threadIdx.x & 31;
    const int g = bx * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (g >= G) return;   // whole warp
    const int M = 2 * N;
    // x = 0: inflow for mu > 0, outflow for mu < 0; x = X: outflow for mu > 0, inflow mu < 0
    // q: a0, a2, ah0, ah1 (face x = 0), b0, b2, bh0, bh1 (face x = X)
    double q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int m = lane; m < M; m += 32) {
        const double wm = w[m], mm = mu[m];
        const double ex = (double)psi_exit[(size_t)m * ldG + g];
        const double p0 = (m < N) ? Iin0[g] : ex;
        const double pX = (m < N) ? ex : IinX[g];
        q[0] += wm * p0;
        q[1] += wm * mm * mm * p0;
        q[4] += wm * pX;
        q[5] += wm * mm * mm * pX;
        if (m >= N) { q[2] += wm * p0; q[3] += wm * mm * p0; }
        else        { q[6] += wm * pX; q[7] += wm * mm * pX; }
    }
    const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
    double r4[4], r2[2];
#pragma unroll
    for (int k = 0; k < 4; ++k) {   // keep sums 4 u16 .. 4 u16 + 3
        const double keep = u16 ? q[k + 4] : q[k], give = u16 ? q[k] : q[k + 4];
        r4[k] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {   // keep 4 u16 + 2 u8 + {0, 1}
        const double keep = u8 ? r4[k + 2] : r4[k], give = u8 ? r4[k] : r4[k + 2];
        r2[k] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
    }
    double r = (u4 ? r2[1] : r2[0]) + __shfl_xor_sync(0xffffffffu, u4 ? r2[0] : r2[1], 4);
    r += __shfl_xor_sync(0xffffffffu, r, 2);
    r += __shfl_xor_sync(0xffffffffu, r, 1);
    // lane l now holds sum (l >> 2) & 7; the numerator of lane 8k's sum is on lane 8k + 4
    const double num = __shfl_down_sync(0xffffffffu, r, 4);
    if ((lane & 7) == 0) {
        const int k = lane >> 3;   // 0: f at x = 0, 1: C^-, 2: f at x = X, 3: C^+
        const double dflt = (k & 1) ? ((k == 1) ? -0.5 : 0.5) : 1.0 / 3.0;
        const double v = (r != 0.0) ? num / r : dflt;
        double *dst = (k == 0) ? fb0 : (k == 1) ? C0 : (k == 2) ? fbX : CX;
        dst[g] = v;
    }
}

template <typename R>
__global__ void k_sweep_finalize(FinalizeArgs x)
{
    griddep_wait();
    finalize_body<R>(x, blockIdx.x);
}

template <typename R>
__global__ void k_sweep_finalize_b(const int *__restrict__ meta, int N,
                                   const FinalizeArgs *__restrict__ xs)
{
    for (int b = blockIdx.x;; b += gridDim.x) {
        int s, bx, by;
        if (!bdecode(meta, N, b, s, bx, by)) break;
        const FinalizeArgs x = xs[s];
        finalize_body<R>(x, bx);
    }
}

// Candidate tile shapes (S, NS, kind); index 0 is the default.  FP32: the lean sweeps of
// sweepf.cu (kind 5: one group per lane, 6: two), which exist for D = 4, 8 and 16, and the
// strip sweep of this file (kind 1), which serves every other tile height (N not a
// multiple of 4).  Measured at 500 cells x 64 directions x 1024 groups: lean one group per
// lane D = 16 (8, 4) 0.100 ms with the finalize, (16, 2) 0.104; two groups per lane
// D = 8 (8, 4) 0.108 (it wins on some batches); the strip sweep D = 8 (16, 2) 0.209.
// FP64 (strip sweep): (8, 2) 1.26 ms, (16, 2) 1.37, (8, 3) 1.37; the paired sweep of
// sweep64.cu (single slab, D = 4) as shapes 3 and 4.
struct Shape {
    int S, NS, V;   // strip cells, strip buffers, kind (1: strip sweep; 5, 6: lean sweep
                    // with one, two groups per lane; 7: paired FP64 sweep)
};
constexpr Shape kShapes32[] = {{8, 4, 5}, {16, 2, 5}, {8, 3, 5}, {8, 2, 5},
                               {8, 2, 6}, {8, 4, 6}, {16, 2, 1}};
constexpr int kStrip32 = 6;   // the FP32 strip sweep's index (tile heights without a lean kernel)
constexpr Shape kShapes64[] = {{8, 2, 1}, {16, 2, 1}, {8, 3, 1}, {8, 2, 7}, {4, 2, 7}};

// largest power of two <= cap dividing N: the direction-tile height D_min that the
// workspace's partial-moment scratch is sized for; D may be D_min or 2 D_min (<= 8)
int base_D(int N, int cap)
{
    for (int D = cap; D >= 1; D >>= 1)
        if (N % D == 0) return D;
    return 1;
}

int finalize_bnd_blocks(int G) { return finalize_bnd_blocks_dev(G); }


// one launch of shape (S, NS): the single-slab grid (direction tiles x group tiles) when
// `a` is given, else the batched persistent grid over the work list (meta, xs)
template <typename R, typename SR, int S, int NS>
cudaError_t launch_shape(const SweepArgs *a, int M, int ldG, int D, const int *meta, int N,
                         const SweepArgs *xs, int grid, cudaStream_t st)
{
    const size_t sm = SweepSmem<R, SR, S, NS>(D).total;
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
    if (a) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep<R, SR, S, NS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        return launch_pdl(k_sweep<R, SR, S, NS>, dim3(M / D, ldG / 32), dim3(32 * D), sm, st, *a);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_sweep_b<R, SR, S, NS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_sweep_b<R, SR, S, NS><<<grid, 32 * D, sm, st>>>(meta, N, xs);
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t dispatch_shape(int shape, const SweepArgs *a, int M, int ldG, int D, const int *meta,
                           int N, const SweepArgs *xs, int grid, cudaStream_t st)
{
    if (sizeof(R) == 4) {   // FP32: pre-scaled FP32 inputs (sigma_t h/2, h e/2)
        const Shape sh = kShapes32[shape];
        if (sh.V >= 5 && (D == 4 || D == 8 || D == 16))
            return launch_sweepf(sh.V, sh.S, sh.NS, a, M, ldG, D, meta, N, xs, grid, st);
        if (D > 8) return cudaErrorInvalidConfiguration;   // 32 D threads: lean sweeps only
        return launch_shape<float, float, 16, 2>(a, M, ldG, D, meta, N, xs, grid, st);
    }
    if (D > 8) return cudaErrorInvalidConfiguration;
    if (kShapes64[shape].V == 7)   // paired sweep: single slab only
        return a ? launch_sweep_pair(kShapes64[shape].S, kShapes64[shape].NS, *a, M, ldG, st)
                 : cudaErrorInvalidConfiguration;
    switch (shape) {
    case 1: return launch_shape<double, double, 16, 2>(a, M, ldG, D, meta, N, xs, grid, st);
    case 2: return launch_shape<double, double, 8, 3>(a, M, ldG, D, meta, N, xs, grid, st);
    default: return launch_shape<double, double, 8, 2>(a, M, ldG, D, meta, N, xs, grid, st);
    }
}

template <typename R>
cudaError_t launch_sweep_t(const Problem &p, const SweepArgs &a)
{
    cudaError_t e = dispatch_shape<R>(p.sweep_shape, &a, p.M, p.ldG, a.D, nullptr, 0, nullptr, 0,
                                      p.stream);
    if (e != cudaSuccess) return e;
    const FinalizeArgs fa = make_finalize_args(p, a);
    cudaError_t ef = launch_pdl(k_sweep_finalize<R>,
                                dim3((unsigned)(fa.nb_cell + finalize_bnd_blocks(p.G))), dim3(256),
                                0, p.stream, fa);
    if (ef != cudaSuccess) return ef;
    return cudaGetLastError();
}

}  // namespace

int pick_D(const Problem &p)
{
    if (p.sweep_D > 0) return p.sweep_D;
    return base_D(p.N, 8);
}

bool sweep_tile_ok(int precision, int D, int shape, bool batched)
{
    if (shape < 0 || shape >= sweep_shape_count(precision) || D < 1) return false;
    if (!sweep_fp32(precision)) {
        if (kShapes64[shape].V == 7)
            return !batched && D == 4 &&
                   pair_sweep_smem(kShapes64[shape].S, kShapes64[shape].NS) <= 227 * 1024;
        return D <= 8;
    }
    const Shape sh = kShapes32[shape];
    if (sh.V >= 5 && (D == 4 || D == 8 || D == 16)) {
        const size_t sm = sweepf_smem(sh.V, sh.S, sh.NS, D);
        return sm > 0 && sm <= 227 * 1024;
    }
    return D <= 8;
}

int sweep_shape_count(int precision)
{
    return sweep_fp32(precision) ? (int)(sizeof(kShapes32) / sizeof(Shape))
                                 : (int)(sizeof(kShapes64) / sizeof(Shape));
}

void sweep_shape_info(int precision, int shape, int *S, int *NS)
{
    const Shape sh = sweep_fp32(precision) ? kShapes32[shape] : kShapes64[shape];
    *S = sh.S;
    *NS = sh.NS;
}

int sweep_group_tiles(int precision, int shape, int D, int ldG)
{
    if (!sweep_fp32(precision)) return ldG / 32;
    const bool lean = kShapes32[shape].V >= 5 && (D == 4 || D == 8 || D == 16);
    return lean && kShapes32[shape].V == 6 ? (ldG + 63) / 64 : ldG / 32;
}

int sweep_D_candidates(const Problem &p, int *D)
{
    const int b = base_D(p.N, 4);
    int n = 0;
    D[n++] = b;
    if (2 * b <= 8 && p.N % (2 * b) == 0) D[n++] = 2 * b;
    // 16 directions per CTA: the lean FP32 sweeps only (half the partial moments of D = 8)
    if (sweep_fp32(p.precision) && p.N % 16 == 0) D[n++] = 16;
    return n;
}

size_t sweep_partial_doubles(const Problem &p)
{
    // sized for the smallest direction tile any shape may use
    return (size_t)(p.M / std::min(base_D(p.N, 4), pick_D(p))) * 2 * p.G * p.nx;
}

SweepArgs make_sweep_args(const Problem &p, double dt, const void *sigE, const void *emis,
                          const void *I_old, void *I_new, double *part, double *psi_exit,
                          double *f, double *fb0, double *fbX, double *C0, double *CX, int D)
{
    SweepArgs a;
    a.nx = p.nx; a.N = p.N; a.G = p.G; a.ldG = p.ldG;
    a.D = D;
    a.icdt = 1.0 / (kC * dt);
    a.h = p.h; a.mu = p.mu; a.w = p.w; a.Iin0 = p.Iin0; a.IinX = p.IinX;
    a.sigE = sigE; a.emis = emis; a.I_old = I_old; a.I_new = I_new;
    a.part = part; a.psi_exit = psi_exit;
    a.f = f; a.fb0 = fb0; a.fbX = fbX; a.C0 = C0; a.CX = CX;
    a.kap32 = nullptr;
    a.dir32 = p.dir32;
    a.ts = p.ts64;
    a.tab64 = p.tab64;
    return a;
}

FinalizeArgs make_finalize_args(const Problem &p, const SweepArgs &a)
{
    FinalizeArgs x;
    x.nx = p.nx; x.N = p.N; x.G = p.G; x.ldG = p.ldG;
    x.ntile = p.M / a.D;
    x.nb_cell = (int)(((long)p.G * p.nx + 255) / 256);
    x.part = a.part; x.psi_exit = a.psi_exit;
    x.mu = p.mu; x.w = p.w; x.Iin0 = p.Iin0; x.IinX = p.IinX;
    x.f = a.f; x.fb0 = a.fb0; x.fbX = a.fbX; x.C0 = a.C0; x.CX = a.CX;
    return x;
}

int finalize_blocks(const Problem &p)
{
    return (int)(((long)p.G * p.nx + 255) / 256) + finalize_bnd_blocks(p.G);
}

cudaError_t launch_sweep(const Problem &p, double dt, const void *sigE, const void *emis,
                         bool sigma_fp32, const void *I_old, void *I_new, double *part,
                         double *psi_exit, double *f, double *fb0, double *fbX, double *C0,
                         double *CX)
{
    SweepArgs a = make_sweep_args(p, dt, sigE, emis, I_old, I_new, part, psi_exit, f, fb0, fbX,
                                  C0, CX, pick_D(p));
    if (!sweep_fp32(p.precision)) return launch_sweep_t<double>(p, a);
    if (!sigma_fp32 || !p.dir32) return cudaErrorInvalidValue;   // FP32 sweeps: FP32 inputs
    // the pre-scaled inputs carry h/(2 c dt) after e (launch_opacity, launch_prescale32)
    a.kap32 = reinterpret_cast<const float *>(emis) + (size_t)p.G * p.nx;
    return launch_sweep_t<float>(p, a);
}

cudaError_t launch_sweep_b(int precision, bool sigma_fp32, int D, int shape, const int *meta,
                           int N, const SweepArgs *xs, int grid, cudaStream_t st)
{
    if (!sweep_fp32(precision))
        return dispatch_shape<double>(shape, nullptr, 0, 0, D, meta, N, xs, grid, st);
    if (!sigma_fp32) return cudaErrorInvalidValue;
    return dispatch_shape<float>(shape, nullptr, 0, 0, D, meta, N, xs, grid, st);
}

cudaError_t launch_finalize_b(int precision, const int *meta, int N, const FinalizeArgs *xs,
                              int grid, cudaStream_t st)
{
    if (sweep_fp32(precision))
        k_sweep_finalize_b<float><<<grid, 256, 0, st>>>(meta, N, xs);
    else
        k_sweep_finalize_b<double><<<grid, 256, 0, st>>>(meta, N, xs);
    return cudaGetLastError();
}

}  // namespace trt
