// sweep64.cu -- paired FP64 S_N sweep (kernel K2, FP64): the directions mu and -mu of one
// |mu| share their corner-system coefficients.
//
// Same discretisation as sweep.cu (eq. rt with implicit Euler, Sec. 5; simple corner
// balance in a 1D slab).  Per (cell, group, direction) the 2 x 2 corner system has
//   a = |mu|/2 + sigma_t h/2,  b = |mu|/2,  t = a/det,  s = b/det,  det = a^2 + b^2,
// and the solution is psi_out = s r_in + t r_out, psi_other = t r_in - s r_out with r the
// corner sources (the inflow corner's carrying |mu| psi_in).  a, b, det, t and s depend on
// |mu|, not on its sign: the sweeps of mu and -mu through a cell use the same t and s.
// On GB300 every FP64 instruction of this kernel holds an FP64 pipe for 64 cycles, and
// forming t and s (the determinant, a refined reciprocal and two products) is 7 of the
// ~17 FP64 instructions of an update, so each pair of directions forms them once.
//
// Schedule (meet in the middle).  A CTA owns 32 groups (the lanes) and D = 4 values of
// |mu|, with two sign groups of D warps: warps 0..D-1 sweep mu > 0 from x = 0, warps
// D..2D-1 sweep mu < 0 from x = X.  Phase 1: each sign group sweeps its first half of the
// slab ([0, mid) for mu > 0, [mid, nx) for mu < 0), forming t and s per cell and storing
// them in a global scratch ts[|mu|][cell][2][ldG]; a CTA barrier; phase 2: each sign group
// sweeps the other half with the t and s the other group stored there.  Every t, s is
// formed once and used twice; the two groups never wait for each other inside a phase.
// Within a sign group cells go in strips of S: intensity rows, the step's pre-scaled
// inputs sigma_t h/2 and h e/2 (FP64, [nx][ldG], written by k_prescale64 before the
// sweep) and, in phase 2, the partner's t, s rows arrive by 16-byte cp.async NS - 1 strips
// ahead; after each strip the group sums its D directions' psi_L + psi_R into the two
// angular moments (a partial tile of D directions per sign, summed in a fixed order by the
// finalize).
#include <type_traits>
#include "sweep.cuh"

namespace trt {

namespace {

constexpr int kPD = 4;   // directions of one sign per CTA (per partial-moment tile)

// 1/d for the determinant d = a^2 + b^2 (normal, > 0): the hardware approximation refined
// by one third-order step (below FP64 rounding; see common.cuh's rcp64)
__device__ __forceinline__ double rcp_det(double d)
{
    double x;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(d));
    const double e = fma(-d, x, 1.0);
    return fma(x, fma(e, e, e), x);
}

__device__ __forceinline__ void cp16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}

// named barrier of one sign group (its D warps)
__device__ __forceinline__ void group_sync(int id)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(32 * kPD) : "memory");
}

template <int S, int NS>
struct PairSmem {
    // per sign group (byte offsets within the group's section):
    static constexpr size_t it = 0;                                 // [NS][D][S][2][32] I_old rows
    static constexpr size_t tb = it + 8ull * NS * kPD * S * 64;     // [NS][D][S][2][32] t, s rows
    static constexpr size_t tq = tb + 8ull * NS * kPD * S * 64;     // [NS][S][2][32] th, q rows
    static constexpr size_t kp = tq + 8ull * NS * S * 64;           // [NS][S] h/(2 c dt)
    static constexpr size_t ps = kp + 8ull * NS * S;                // [D][S][33] psi_L + psi_R
    static constexpr size_t group = ps + 8ull * kPD * S * 33;
    static constexpr size_t total = 2 * group;
};

template <int S, int NS>
__global__ void __launch_bounds__(64 * kPD) k_sweep_pair(SweepArgs a)
{
    griddep_wait();
    using L = PairSmem<S, NS>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sg = warp / kPD, wi = warp % kPD, gtid = tid % (32 * kPD);
    unsigned char *base = smem_raw + sg * L::group;
    double *it = reinterpret_cast<double *>(base + L::it);
    double *tb = reinterpret_cast<double *>(base + L::tb);
    double *tq = reinterpret_cast<double *>(base + L::tq);
    double *kp = reinterpret_cast<double *>(base + L::kp);
    double *ps = reinterpret_cast<double *>(base + L::ps);

    const int nx = a.nx, N = a.N, G = a.G, ldG = a.ldG;
    const int dtile = blockIdx.x, gt = blockIdx.y;
    const int gb = gt * 32, g = gb + lane;
    const int n = dtile * kPD + wi;          // |mu| index
    const int m = sg ? N + n : n;            // direction index (m >= N: mu < 0)
    const int mid = nx / 2;
    const double am = fabs(a.mu[m]), b = 0.5 * am, bb = b * b;
    // moment weights of the group's D directions (w/2, w mu^2/2)
    double wt[kPD], wm[kPD];
#pragma unroll
    for (int d = 0; d < kPD; ++d) {
        const int md = (sg ? N : 0) + dtile * kPD + d;
        wt[d] = 0.5 * a.w[md];
        wm[d] = 0.5 * a.w[md] * a.mu[md] * a.mu[md];
    }
    double psi = (g < G) ? (sg ? a.IinX[g] : a.Iin0[g]) : 0.0;

    const size_t row = 2 * (size_t)ldG;      // one cell of one direction (two corner rows)
    const double *Iold = reinterpret_cast<const double *>(a.I_old) + (size_t)m * nx * row;
    double *Inew = reinterpret_cast<double *>(a.I_new) + (size_t)m * nx * row + g;
    const double *th64 = reinterpret_cast<const double *>(a.sigE);   // [nx][ldG]
    const double *q64 = reinterpret_cast<const double *>(a.emis);    // [nx][ldG], then kap [nx]
    const double *kap64 = q64 + (size_t)nx * ldG;
    double *ts = a.ts + (size_t)n * nx * row;   // this |mu|'s t, s rows
    double *part = reinterpret_cast<double *>(a.part);
    const int tile = sg ? N / kPD + dtile : dtile;
    // this lane's 16-byte chunk of a cell's two 32-double rows: row rr, chunk ch
    const int rr = lane >> 4, ch = lane & 15;

    for (int phase = 0; phase < 2; ++phase) {
        // this group's cells in this phase, in sweep order: mu > 0 ascending over [lo, hi),
        // mu < 0 descending; strips aligned at lo (mu > 0) or hi (mu < 0)
        const bool first = (phase == 0);
        const int lo = (first == (sg == 0)) ? 0 : mid;
        const int hi = (first == (sg == 0)) ? mid : nx;
        const int nst = (hi - lo + S - 1) / S;
        auto range = [&](int st, int &c0, int &ns) {
            if (sg == 0) {
                c0 = lo + st * S;
                ns = min(S, hi - c0);
            } else {
                const int c1 = hi - st * S;
                c0 = max(c1 - S, lo);
                ns = c1 - c0;
            }
        };
        auto prefetch = [&](int st, int bf) {
            int c0, ns;
            range(st, c0, ns);
            double *itw = it + ((size_t)(bf * kPD + wi) * S) * 64;
            double *tbw = tb + ((size_t)(bf * kPD + wi) * S) * 64;
            for (int cc = 0; cc < ns; ++cc) {
                const size_t src = (size_t)(c0 + cc) * row + rr * ldG + gb + 2 * ch;
                cp16(itw + cc * 64 + rr * 32 + 2 * ch, Iold + src);
                if (!first) cp16(tbw + cc * 64 + rr * 32 + 2 * ch, ts + src);
            }
            // th, q rows of the strip: cells wi, wi + D, ... by warp wi of the group
            double *tqb = tq + (size_t)bf * S * 64;
            for (int cc = wi; cc < ns; cc += kPD) {
                const double *srcp = (rr ? q64 : th64) + (size_t)(c0 + cc) * ldG + gb + 2 * ch;
                cp16(tqb + cc * 64 + rr * 32 + 2 * ch, srcp);
            }
            if (gtid < ns) cp_async<8>(kp + bf * S + gtid, kap64 + c0 + gtid);
            cp_commit();
        };
        for (int k = 0; k < NS - 1; ++k) {
            if (k < nst)
                prefetch(k, k);
            else
                cp_commit();
        }
        for (int st = 0; st < nst; ++st) {
            const int bf = st % NS;
            int c0, ns;
            range(st, c0, ns);
            cp_wait<NS - 2>();
            group_sync(1 + sg);   // the strip's copies landed; the last reduction is done
            if (st + NS - 1 < nst)
                prefetch(st + NS - 1, (st + NS - 1) % NS);
            else
                cp_commit();
            const double *itw = it + ((size_t)(bf * kPD + wi) * S) * 64 + lane;
            const double *tbw = tb + ((size_t)(bf * kPD + wi) * S) * 64 + lane;
            const double *tqb = tq + (size_t)bf * S * 64 + lane;
            const double *kpb = kp + bf * S;
            double *psw = ps + (size_t)wi * S * 33 + lane;
            double *tsw = ts + g;
            // one cell: FIRST forms t, s and stores them for the other sign group; POS: the
            // sign of mu (inflow on the left corner)
            auto cell = [&](auto first_c, auto pos_c, int cc) {
                constexpr bool FIRST = decltype(first_c)::value, POS = decltype(pos_c)::value;
                const int c = c0 + cc;
                const double IL = itw[cc * 64], IR = itw[cc * 64 + 32];
                const double q = tqb[cc * 64 + 32];
                const double kap = kpb[cc];
                double t, s;
                if (FIRST) {
                    const double aa = b + tqb[cc * 64];
                    const double x = rcp_det(fma(aa, aa, bb));
                    t = aa * x;
                    s = b * x;
                    tsw[(size_t)c * row] = t;
                    tsw[(size_t)c * row + ldG] = s;
                } else {
                    t = tbw[cc * 64];
                    s = tbw[cc * 64 + 32];
                }
                const double kL = fma(kap, IL, q), kR = fma(kap, IR, q);
                double pL, pR;
                if (POS) {
                    const double rL = fma(am, psi, kL);
                    pR = fma(s, rL, t * kR);
                    pL = fma(t, rL, -(s * kR));
                    psi = pR;
                } else {
                    const double rR = fma(am, psi, kR);
                    pL = fma(s, rR, t * kL);
                    pR = fma(t, rR, -(s * kL));
                    psi = pL;
                }
                Inew[(size_t)c * row] = pL;
                Inew[(size_t)c * row + ldG] = pR;
                psw[cc * 33] = pL + pR;
            };
            // full strips unrolled (the next cells' loads and independent products overlap
            // the recurrence of the current one), ragged strips in a loop
            auto strip = [&](auto first_c, auto pos_c) {
                constexpr bool POS = decltype(pos_c)::value;
                if (ns == S) {
#pragma unroll
                    for (int k = 0; k < S; ++k) cell(first_c, pos_c, POS ? k : S - 1 - k);
                } else {
                    for (int k = 0; k < ns; ++k) cell(first_c, pos_c, POS ? k : ns - 1 - k);
                }
            };
            using T_ = std::true_type;
            using F_ = std::false_type;
            if (first) {
                if (sg == 0) strip(T_(), T_()); else strip(T_(), F_());
            } else {
                if (sg == 0) strip(F_(), T_()); else strip(F_(), F_());
            }
            group_sync(1 + sg);
            // the group's D directions summed per (cell, group) of the strip, in order
            for (int idx = gtid; idx < 32 * S; idx += 32 * kPD) {
                const int gl = idx / S, cc = idx % S;
                const int gg = gb + gl;
                if (cc < ns && gg < G) {
                    double s0 = 0.0, s2 = 0.0;
#pragma unroll
                    for (int d = 0; d < kPD; ++d) {
                        const double v = ps[((size_t)d * S + cc) * 33 + gl];
                        s0 = fma(wt[d], v, s0);
                        s2 = fma(wm[d], v, s2);
                    }
                    const size_t o = ((size_t)(tile * 2) * G + gg) * nx + c0 + cc;
                    part[o] = s0;
                    part[o + (size_t)G * nx] = s2;
                }
            }
        }
        cp_wait<0>();
        // phase 1 -> 2: every t, s of this CTA is stored (global writes before the barrier
        // are visible to the block after it) and every reduction has read ps
        __syncthreads();
    }
    reinterpret_cast<double *>(a.psi_exit)[(size_t)m * ldG + g] = psi;
}

// the paired sweep's pre-scaled FP64 inputs from sigma_E and e_g ([G][nx]): sigma_t h/2 and
// h e/2 as [nx][ldG] (zero in the padding groups), then h/(2 c dt) per cell; a 32 x 32 tile
// through shared memory so that both sides are read and written along rows
__global__ void k_prescale64(int nx, int G, int ldG, const double *__restrict__ h, double icdt,
                             const double *__restrict__ sigE, const double *__restrict__ emis,
                             double *th64, double *q64)
{
    griddep_wait();
    __shared__ double sth[32][33], sq[32][33];
    const int c0 = blockIdx.x * 32, g0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    for (int r = ty; r < 32; r += 8) {   // read along cells: group g0 + r, cell c0 + tx
        const int g = g0 + r, c = c0 + tx;
        double vt = 0.0, vq = 0.0;
        if (g < G && c < nx) {
            const double hh = 0.5 * h[c];
            vt = hh * (sigE[(size_t)g * nx + c] + icdt);
            vq = hh * emis[(size_t)g * nx + c];
        }
        sth[r][tx] = vt;
        sq[r][tx] = vq;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {   // write along groups: cell c0 + r, group g0 + tx
        const int c = c0 + r, g = g0 + tx;
        if (c < nx && g < ldG) {
            th64[(size_t)c * ldG + g] = sth[tx][r];
            q64[(size_t)c * ldG + g] = sq[tx][r];
        }
    }
    if (blockIdx.y == 0 && ty == 0 && c0 + tx < nx)
        q64[(size_t)nx * ldG + c0 + tx] = 0.5 * h[c0 + tx] * icdt;
}

}  // namespace

size_t pair_sweep_smem(int S, int NS)
{
    if (S == 8 && NS == 2) return PairSmem<8, 2>::total;
    if (S == 4 && NS == 2) return PairSmem<4, 2>::total;
    return 0;
}

cudaError_t launch_sweep_pair(int S, int NS, const SweepArgs &a, int M, int ldG, cudaStream_t st)
{
    if (a.D != kPD || a.N % kPD != 0 || !a.ts || !a.tab64) return cudaErrorInvalidConfiguration;
    const double *sigE = reinterpret_cast<const double *>(a.sigE);
    const double *emis = reinterpret_cast<const double *>(a.emis);
    double *tab64 = a.tab64;
    const int nx = a.nx, G = a.G;
    cudaError_t e = launch_pdl(k_prescale64, dim3((nx + 31) / 32, (ldG + 31) / 32), dim3(32, 8),
                               0, st, nx, G, ldG, (const double *)a.h, a.icdt, sigE, emis, tab64,
                               tab64 + (size_t)nx * ldG);
    if (e != cudaSuccess) return e;
    SweepArgs x = a;
    x.sigE = tab64;
    x.emis = tab64 + (size_t)nx * ldG;
    const dim3 grid(M / 2 / kPD, ldG / 32);
    auto go = [&](auto kern, size_t sm) {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sm);
        if (r != cudaSuccess) return r;
        return launch_pdl(kern, grid, dim3(64 * kPD), sm, st, x);
    };
    if (S == 8 && NS == 2) return go(k_sweep_pair<8, 2>, PairSmem<8, 2>::total);
    if (S == 4 && NS == 2) return go(k_sweep_pair<4, 2>, PairSmem<4, 2>::total);
    return cudaErrorInvalidConfiguration;
}

}  // namespace trt
