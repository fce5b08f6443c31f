// physics.cu -- group opacities and Planck integrals at cell temperatures (kernel K1).
//
// Sec. 2 / Sec. 3.1 / Sec. 6 of the paper: with x = nu/T,
//   B_g     = CB T^4 [P(x_{g+1}) - P(x_g)],           P(x) = int_0^x t^3/(e^t-1) dt
//   e_g     = int sigma B = s 27 CB T (e^{-x_g} - e^{-x_{g+1}})   (sigma B = 27 s CB e^{-nu/T})
//   sigma_B = e_g / B_g = sigma_E          (T_r = T; the T_r option: opacity_tr)
//   sigma_R = s 27 N_g / (T^3 D_g),  N_g = [-x^4/(e^x-1) + 4 P(x)],  D_g = [int t^7 e^{2t}/(e^t-1)^3]
// Every per-edge integral is evaluated in closed form: a power series below x = 2 (radius
// of convergence 2 pi; the coefficients follow from t/(e^t-1) = sum B_n t^n / n!), and
// exponentially convergent tails e^{-kx} at and above it, summed with the scale e^{x_g}
// factored out so that cold cells (x ~ 1e5) neither underflow nor lose the ratio.
#include <algorithm>
#include <cmath>
#include <cstring>
#include "batch.cuh"

namespace trt {

__constant__ SeriesTables c_ser;

// Gauss-Legendre nodes on [-1, 1] by Newton's method on the Legendre recurrence.
void gauss_legendre_host(int n, double *x, double *w)
{
    for (int k = 0; k < (n + 1) / 2; ++k) {
        double z = std::cos(kPi * (k + 0.75) / (n + 0.5));
        for (int it = 0; it < 64; ++it) {
            double pm = 1.0, pc = z;
            for (int j = 2; j <= n; ++j) {
                double pn = ((2 * j - 1) * z * pc - (j - 1) * pm) / j;
                pm = pc;
                pc = pn;
            }
            double dp = n * (pm - z * pc) / (1.0 - z * z);
            double dz = pc / dp;
            z -= dz;
            if (std::fabs(dz) <= 1e-16 * std::fabs(z) + 1e-300) break;
        }
        double pm = 1.0, pc = z;
        for (int j = 2; j <= n; ++j) {
            double pn = ((2 * j - 1) * z * pc - (j - 1) * pm) / j;
            pm = pc;
            pc = pn;
        }
        double dp = n * (pm - z * pc) / (1.0 - z * z);
        double wk = 2.0 / ((1.0 - z * z) * dp * dp);
        x[n - 1 - k] = z;
        x[k] = -z;
        w[n - 1 - k] = wk;
        w[k] = wk;
    }
}

static SeriesTables build_tables()
{
    SeriesTables t{};
    for (int k = 1; k <= 64; ++k) {
        const double k4 = (double)k * k * k * k;
        t.tP[k] = 6.0 / k4;
        t.tD[k] = 5040.0 * 0.5 * k * (k + 1.0) / (k4 * k4);
    }
    gauss_legendre_host(3, t.g3x, t.g3w);
    t.g3x[1] = 0.0;
    t.g3w[1] *= 0.5;
    gauss_legendre_host(4, t.g4x, t.g4w);
    gauss_legendre_host(6, t.g6x, t.g6w);
    gauss_legendre_host(8, t.g8x, t.g8w);
    typedef long double LD;
    // c_n = B_n/n!: reciprocal of (e^t-1)/t = sum_k t^k/(k+1)!
    LD c[kSer], fact[kSer + 2];
    fact[0] = 1;
    for (int k = 1; k < kSer + 2; ++k) fact[k] = fact[k - 1] * k;
    c[0] = 1;
    for (int n = 1; n < kSer; ++n) {
        LD s = 0;
        for (int k = 1; k <= n; ++k) s += c[n - k] / fact[k + 1];
        c[n] = -s;
    }
    // psi(t) = phi(t) phi(-t)^2 = t^3 e^{2t}/(e^t-1)^3, phi(t) = t/(e^t-1)
    LD cm[kSer], u[kSer], d[kSer];
    for (int n = 0; n < kSer; ++n) cm[n] = (n % 2) ? -c[n] : c[n];
    for (int n = 0; n < kSer; ++n) {
        LD s = 0;
        for (int k = 0; k <= n; ++k) s += cm[k] * cm[n - k];
        u[n] = s;
    }
    for (int n = 0; n < kSer; ++n) {
        LD s = 0;
        for (int k = 0; k <= n; ++k) s += c[k] * u[n - k];
        d[n] = s;
    }
    for (int n = 0; n < kSer; ++n) {
        t.pP[n] = (double)(c[n] / (n + 3));
        t.pN[n] = (double)(c[n] * (1 - n) / (n + 3));   // -x^3 phi(x) + 4 P(x)
        t.pD[n] = (double)(d[n] / (n + 5));
    }
    const LD pi = 3.141592653589793238462643383279502884L;
    t.Pinf = (double)(pi * pi * pi * pi / 15);
    const LD ln2 = 0.693147180559945309417232121458176568L;
    for (int j = 0; j < 32; ++j) t.e2[j] = (double)exp2l((LD)j / 32);
    const LD L = ln2 / 32;
    double l1 = (double)L;
    uint64_t bits;
    std::memcpy(&bits, &l1, 8);
    bits &= ~((uint64_t(1) << 22) - 1);   // 31 significant bits: k L1 exact for |k| < 2^22
    std::memcpy(&l1, &bits, 8);
    t.eL1 = l1;
    t.eL2 = (double)(L - (LD)l1);
    t.einv = (double)(32 / ln2);
    LD z7 = 0;
    for (long k = 200000; k >= 1; --k) z7 += 1.0L / ((LD)k * k * k * k * k * k * k);
    LD z6 = pi * pi * pi * pi * pi * pi / 945;
    t.Dinf = (double)(2520 * (z6 + z7));
    return t;
}

const SeriesTables &host_series()
{
    static SeriesTables t = build_tables();
    return t;
}

static int g_tables_ready[64] = {0};

cudaError_t ensure_tables()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (g_tables_ready[dev]) return cudaSuccess;
    e = cudaMemcpyToSymbol(c_ser, &host_series(), sizeof(SeriesTables));
    if (e == cudaSuccess) g_tables_ready[dev] = 1;
    return e;
}

// ---------------------------------------------------------------------------------------
// per-edge values
// ---------------------------------------------------------------------------------------
__host__ __device__ inline int series_terms(double x)
{
    return x < 0.125 ? 12 : x < 0.5 ? 18 : x < 1.0 ? 26 : 42;
}

// x < 2: P(x), Nt(x), D(x) by Horner
// The exponential of the group integrals: texp (table-driven, common.cuh) on the device,
// the C library's on the host (inflow spectra and initial state at creation).
struct Mx {
    const double *tab;
    ExpConsts c;
    __host__ __device__ double ex(double x) const
    {
#ifdef __CUDA_ARCH__
        return texp(x, tab, c);
#else
        return std::exp(x);
#endif
    }
};

__host__ __device__ inline void edge_series(double x, const SeriesTables &t, double &P,
                                            double &Nt, double &D)
{
    int n = series_terms(x);
    double sP = 0.0, sN = 0.0, sD = 0.0;
    for (int k = n - 1; k >= 0; --k) {
        sP = fma(sP, x, t.pP[k]);
        sN = fma(sN, x, t.pN[k]);
        sD = fma(sD, x, t.pD[k]);
    }
    double x3 = x * x * x;
    P = x3 * sP;
    Nt = x3 * sN;
    D = x3 * x * x * sD;
}

// x >= 2, every tail scaled by e^{x}:
//   TP = e^x (pi^4/15 - P(x)) = sum_k e^{-(k-1)x} 6 e3(kx)/k^4
//   TN = e^x x^4/(e^x - 1)    = x^4 / (1 - e^{-x})
//   TD = e^x (Dinf - D(x))    = sum_k k(k+1)/2 e^{-(k-1)x} 5040 e7(kx)/k^8
// with e_m(y) = sum_{j<=m} y^j/j!  (integration by parts of t^n e^{-kt}).
__host__ __device__ inline void edge_tail(double x, const SeriesTables &t, const Mx &mx, double &TP,
                                          double &TN, double &TD)
{
    const double e3 = 1.0 + x * (1.0 + x * (0.5 + x * (1.0 / 6.0)));
    const double e7 = 1.0 + x * (1.0 + x * (1.0 / 2 + x * (1.0 / 6 + x * (1.0 / 24 + x * (1.0 / 120
                      + x * (1.0 / 720 + x * (1.0 / 5040)))))));
    double sp = t.tP[1] * e3, sd = t.tD[1] * e7;
    if (x >= 40.0) {   // e^{-x} < 5e-18: one term, and 1 - e^{-x} = 1 in FP64
        TP = sp;
        TD = sd;
        TN = x * x * x * x;
        return;
    }
    const double q = mx.ex(-x);
    double ek = q;
    for (int k = 2; k <= 64 && ek >= 1e-18; ++k) {
        const double y = (double)k * x;
        const double f3 = 1.0 + y * (1.0 + y * (0.5 + y * (1.0 / 6.0)));
        const double f7 = 1.0 + y * (1.0 + y * (1.0 / 2 + y * (1.0 / 6 + y * (1.0 / 24 + y * (1.0 / 120
                          + y * (1.0 / 720 + y * (1.0 / 5040)))))));
        sp += ek * t.tP[k] * f3;
        sd += ek * t.tD[k] * f7;
        ek *= q;
    }
    TP = sp;
    TD = sd;
    TN = x * x * x * x * rcp64(-expm1(-x));
}

// Gauss rule on [xa, xb] for the three scaled integrands x^3 e^{xa-x}/(1-e^{-x}),
// x^4 e^{xa-x}/(1-e^{-x})^2, x^7 e^{xa-x}/(1-e^{-x})^3.  Their nearest singularities
// are the poles x = 2 pi i k, so an n-point rule on a half-width a converges like
// (a/4 pi)^(2n): 3 points reach 1e-16 for xb - xa <= 1/20, 4 points for xb - xa <= 1/4,
// 6 points for xb - xa <= 1.
template <int NP>
__host__ __device__ inline void gauss_group(double xa, double xb, const double *gx,
                                            const double *gw, const Mx &mx, double &dPs,
                                            double &Ns, double &Ds)
{
    // symmetric rule: the points mid -/+ hw xi_j share e^{xa-mid} and e^{+-hw xi_j}, so a
    // pair of points costs one exponential and one reciprocal; e^{-x} follows from
    // e^{-mid} the same way, and 1 - e^{-x} is formed directly where x >= 0.1 (relative
    // error <= eps/x) and by expm1 below
    const double hw = 0.5 * (xb - xa), mid = 0.5 * (xb + xa);
    const double E0 = mx.ex(xa - mid);
    const bool warm = mid - hw < 37.0;              // some point has 1 - e^{-x} != 1
    const double Em = warm ? mx.ex(-mid) : 0.0;
    double sp = 0.0, sn = 0.0, sd = 0.0;
#pragma unroll
    for (int j = NP / 2; j < NP; ++j) {
        const double t = hw * gx[j];
        const double ep = mx.ex(t), em = rcp64(ep);
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const double x = side ? mid + t : mid - t;
            const double ex = side ? E0 * em : E0 * ep;          // e^{xa - x}
            double u = 1.0;                                       // 1/(1 - e^{-x})
            if (warm && x <= 37.0) {
                const double omx = (x >= 0.1) ? 1.0 - Em * (side ? em : ep) : -expm1(-x);
                u = rcp64(omx);
            }
            const double x3 = x * x * x;
            const double eu = gw[j] * ex * x3 * u;
            sp += eu;
            sn += eu * x * u;
            sd += eu * x3 * x * u * u;
        }
    }
    dPs = hw * sp;
    Ns = hw * sn;
    Ds = hw * sd;
}

// e^{xa} [P]_{xa}^{xb}, e^{xa} [Nt]_{xa}^{xb}, e^{xa} [D]_{xa}^{xb}, and 1 - e^{-(xb-xa)}.
// Narrow groups -- xb - xa <= 1 and <= xa/4, where differences of edge values would
// cancel -- integrate the three integrands directly with a Gauss rule (over such a group
// the x^7 factor varies by at most (5/4)^7 and the rest is analytic within 2 pi);
// every other group differences the closed forms.
__host__ __device__ inline void group_integrals(double xa, double xb, bool binf,
                                                const SeriesTables &t, const Mx &mx,
                                                double &dPs, double &Ns, double &Ds,
                                                double &om)
{
    om = binf ? 1.0 : -expm1(-(xb - xa));
    const double w = xb - xa;
    if (!binf && w <= 0.25 * xa && w <= 1.0) {
        if (w <= 0.05)
            gauss_group<3>(xa, xb, t.g3x, t.g3w, mx, dPs, Ns, Ds);
        else if (w <= 0.25)
            gauss_group<4>(xa, xb, t.g4x, t.g4w, mx, dPs, Ns, Ds);
        else
            gauss_group<6>(xa, xb, t.g6x, t.g6w, mx, dPs, Ns, Ds);
        return;
    }
    if (xa >= kXSplit) {
        double TPa, TNa, TDa, TPb = 0.0, TNb = 0.0, TDb = 0.0, r = 0.0;
        edge_tail(xa, t, mx, TPa, TNa, TDa);
        if (!binf) {
            edge_tail(xb, t, mx, TPb, TNb, TDb);
            r = mx.ex(xa - xb);
        }
        dPs = TPa - r * TPb;
        Ns = (TNa - r * TNb) + 4.0 * dPs;
        Ds = TDa - r * TDb;
    } else {
        double Pa, Na, Da, Pb, Nb, Db;
        edge_series(xa, t, Pa, Na, Da);
        if (binf) {
            Pb = t.Pinf;
            Nb = 4.0 * t.Pinf;
            Db = t.Dinf;
        } else if (xb < kXSplit) {
            edge_series(xb, t, Pb, Nb, Db);
        } else {
            double TP, TN, TD;
            edge_tail(xb, t, mx, TP, TN, TD);
            double eb = mx.ex(-xb);
            Pb = t.Pinf - eb * TP;
            Nb = -eb * TN + 4.0 * Pb;
            Db = t.Dinf - eb * TD;
        }
        double ea = mx.ex(xa);
        dPs = ea * (Pb - Pa);
        Ns = ea * (Nb - Na);
        Ds = ea * (Db - Da);
    }
}

void host_group_B(int G, const double *edges, double T, double *B)
{
    const SeriesTables &t = host_series();
    for (int g = 0; g < G; ++g) {
        double xa = edges[g] / T;
        bool binf = std::isinf(edges[g + 1]);
        double xb = binf ? 0.0 : edges[g + 1] / T;
        double dPs, Ns, Ds, om;
        group_integrals(xa, xb, binf, t, Mx{nullptr, ExpConsts{}}, dPs, Ns, Ds, om);
        B[g] = kCB * T * T * T * T * exp(-xa) * dPs;
    }
}

// One interval's series in the local coordinate t in [-1, 1], stored as monomial
// coefficients a_0 .. a_{kTabNC-1} (converted from the Chebyshev fit when the tables are
// built) and summed by Horner's rule: one FMA per term, half the FP64 operations of
// Clenshaw's recurrence on the Chebyshev coefficients.  The conversion is safe for the
// tabulated functions: sum |a_j| <= 1.45 min |p(t)| over every group and interval of the
// 17-, 256-, 1024- and 4096-group structures (the fits' coefficients decay much faster than
// the Chebyshev polynomials' monomial coefficients grow on intervals 0.125 wide in ln T).
// The terms from t^kTabLo on are at most 2.4e-6 of |p| there (1.9e-8 absolute for the
// logarithm of the emission factor), so they are summed in FP32 (a_k stored in FP32,
// between 3e-31 and 7.3e7: normal numbers) and joined to the FP64 Horner sum of the low
// terms; against the direct group integrals the split evaluation stays within 1e-12
// (sigma_E), the direct Rosseland quadrature's own 1.6e-11 (sigma_R) and 4e-14 absolute
// (emission logarithm) -- a CPU emulation of the split on every table entry at 9 points
// per interval -- for 3 FP32 FMAs and one exact conversion in place of 4 FP64 FMAs (the
// tail widened with integer instructions, widen_f32).
__device__ inline double horner(const double *__restrict__ a, const float *__restrict__ b,
                                double t, float tf)
{
    float q = b[kTabNC - kTabLo - 1];
#pragma unroll
    for (int k = kTabNC - kTabLo - 2; k >= 0; --k) q = fmaf(q, tf, b[k]);
    double p = widen_f32(q);
#pragma unroll
    for (int k = kTabLo - 1; k >= 0; --k) p = fma(p, t, a[k]);
    return p;
}

// sigma_E T^3 / (27 s) = (1 - e^{-w}) / [P]  and  sigma_R T^3 / (27 s) = [Nt] / [D] of one
// group at temperature T, the e^{xa}-scaled integrals of group_integrals
__host__ __device__ inline void group_ratios(double T, double ea, double eb, const Mx &mx,
                                             double &A, double &Rr)
{
    const double iT = 1.0 / T;
    const double xa = ea * iT;
    const bool binf = isinf(eb);
    const double xb = binf ? 0.0 : eb * iT;
    double dPs, Ns, Ds, om;
#ifdef __CUDA_ARCH__
    group_integrals(xa, xb, binf, c_ser, mx, dPs, Ns, Ds, om);
#else
    group_integrals(xa, xb, binf, host_series(), mx, dPs, Ns, Ds, om);
#endif
    A = om / dPs;
    Rr = Ns / Ds;
}

// Per-cell terms of the opacity evaluation: T, 1/T, 1/T^3, 27 s C_B T, the table interval
// m and local coordinate t of ln T (m < 0: outside the tables), and with the T_r option
// T_r and T_r / T.  The single-slab kernel reads them from an array that k_cell_terms
// fills once per evaluation (a logarithm and a reciprocal per cell, instead of once per
// block of 8 groups); the batched kernel stages its block's 32 cells with one row (warp),
// rotating with the block over the four sub-partitions.  Both use cell_vals: the same
// operations, the same bits.
struct CellVals {
    double T, iT, iT3, t, kET, Tr, rho;
    float tf;
    int m;
};

__device__ inline CellVals cell_vals(const OpacityArgs &a, int i)
{
    CellVals v;
    const double Ti = a.T[i];
    const double iT = rcp64(Ti);
    v.T = Ti;
    v.iT = iT;
    v.iT3 = iT * iT * iT;
    v.kET = a.kE * Ti;
    int m = -1;
    double t = 0.0;
    if (a.otab) {
        const double z = (log(Ti) - kTabU0) * (1.0 / kTabH);
        if (z >= 0.0 && z < (double)kTabNI) {
            m = min((int)z, kTabNI - 1);
            t = 2.0 * (z - (double)m) - 1.0;
        }
    }
    v.m = m;
    v.t = t;
    v.tf = (float)t;
    v.Tr = Ti;
    v.rho = 1.0;
    if (a.Erad) {   // T_r = (E/a_R)^{1/4}; T_r = T without a usable energy
        const double E = a.Erad[i];
        const double Tr = (E > 0.0 && isfinite(E)) ? sqrt(sqrt(E / kAR)) : Ti;
        v.Tr = Tr;
        v.rho = Tr * iT;
    }
    return v;
}

// the per-cell arrays of the single-slab kernel: [7][nx] doubles (T, 1/T, 1/T^3, t, 27 s
// C_B T, T_r, T_r/T), then tf [nx] floats and m [nx] ints
struct CellArrays {
    double *d;
    float *f;
    int *m;
    int nx;
    __device__ void put(int i, const CellVals &v) const
    {
        d[i] = v.T; d[nx + i] = v.iT; d[2 * nx + i] = v.iT3; d[3 * nx + i] = v.t;
        d[4 * nx + i] = v.kET; d[5 * nx + i] = v.Tr; d[6 * nx + i] = v.rho;
        f[i] = v.tf;
        m[i] = v.m;
    }
    __device__ CellVals get(int i) const
    {
        CellVals v;
        v.T = d[i]; v.iT = d[nx + i]; v.iT3 = d[2 * nx + i]; v.t = d[3 * nx + i];
        v.kET = d[4 * nx + i]; v.Tr = d[5 * nx + i]; v.rho = d[6 * nx + i];
        v.tf = f[i];
        v.m = m[i];
        return v;
    }
};

__device__ inline CellArrays cell_arrays(const OpacityArgs &a)
{
    return CellArrays{a.cterm, reinterpret_cast<float *>(a.cterm + 7 * (size_t)a.nx),
                      reinterpret_cast<int *>(a.cterm + 7 * (size_t)a.nx) + a.nx, a.nx};
}

// the pair form's per-cell terms (TRT_LO_PAIR): t, 1/T, 1/T^3, 27 s C_B T, h/2 split from
// the FP64 terms of cell_vals
struct CellPair {
    fpair t, iT, iT3, kET, hh;
};
__device__ inline CellPair cell_pair(const OpacityArgs &a, int i, const CellVals &v)
{
    return CellPair{fpair(v.t), fpair(v.iT), fpair(v.iT3), fpair(v.kET), fpair(0.5 * a.h[i])};
}

struct CellTerms {
    CellVals v[32];
    CellPair p[32];
};

__device__ inline void stage_cells(const OpacityArgs &a, int i0, CellTerms &ct, int sy)
{
    if ((int)threadIdx.y == (sy & 3)) {
        const int tx = threadIdx.x, i = i0 + tx;
        if (i < a.nx) {
            const CellVals v = cell_vals(a, i);
            ct.v[tx] = v;
            if (a.otabp) ct.p[tx] = cell_pair(a, i, v);
        }
    }
    __syncthreads();
}

// sigma_E,g(T, T_r) and sigma_R,g(T, T_r) (Sec. 2, Sec. 3.1) for sigma = 27 s/nu^3 (1 -
// e^{-nu/T}); with x = nu/T_r and rho = T_r/T:
//   sigma_E = 27 s J / (T_r^3 [P(x_{g+1}) - P(x_g)]),  J = int (1 - e^{-rho x})/(e^x - 1) dx
//   sigma_R = 27 s N / (T_r^3 D),  N the T_r = T numerator at x = nu/T_r,
//             D = int x^7 e^x / ((1 - e^{-rho x}) (e^x - 1)^2) dx
// J and D by the 8-point Gauss rule on panels over [x_g, min(x_{g+1}, x_g + 64)], width 2 or,
// for rho > 1, max(1/rho, a/2) from a panel start a below 4 (1 - e^{-rho x} changes on the
// scale 1/rho near 0), the last panel taking the remainder up to 1.5 widths; both scaled
// by e^{x_g} like the Planck difference, so cold groups neither underflow nor lose the
// ratio.  About 40 FP64 operations per node: far dearer than the tabulated T_r = T path.
__device__ void opacity_tr(double nu_a, double nu_b, bool binf, double Tr, double rho,
                           double k27, const Mx &mx, double &sg, double &sR)
{
    const double iTr = 1.0 / Tr;
    const double xa = nu_a * iTr;
    const double xb = binf ? 0.0 : nu_b * iTr;
    double dPs, Ns, Ds0, om;
    group_integrals(xa, xb, binf, c_ser, mx, dPs, Ns, Ds0, om);
    const double hi = binf ? xa + 64.0 : fmin(xb, xa + 64.0);
    double Js = 0.0, Ds = 0.0, a = xa;
    while (a < hi) {
        const double wmax = (rho > 1.0) ? fmin(2.0, fmax(1.0 / rho, 0.5 * a)) : 2.0;
        const double b = (hi - a <= 1.5 * wmax) ? hi : a + wmax;
        const double hw = 0.5 * (b - a);
        for (int q = 0; q < 8; ++q) {
            const double x = a + hw * (1.0 + c_ser.g8x[q]);
            const double e = exp(xa - x);
            const double o1 = -expm1(-x);
            const double orh = -expm1(-rho * x);
            const double wq = hw * c_ser.g8w[q];
            Js += wq * e * orh / o1;
            const double x2 = x * x, x7 = x2 * x2 * x2 * x;
            Ds += wq * x7 * e / (orh * o1 * o1);
        }
        a = b;
    }
    const double Tr3 = Tr * Tr * Tr;
    sg = k27 * Js / (Tr3 * dPs);
    sR = k27 * Ns / (Tr3 * Ds);
}

// cell i, group g with the cell's terms v; outputs [G][nx] (cells contiguous)
__device__ inline void opacity_body(const OpacityArgs &a, int i, int g, const CellVals &v,
                                    const Mx &mx)
{
    const size_t idx = (size_t)g * a.nx + i;
    const double Ti = v.T, iT = v.iT, iT3 = v.iT3;
    const double xa = a.edges[g] * iT;
    const double eb = a.edges[g + 1];
    const bool binf = isinf(eb);
    double sg, sR, em;
    const int m = v.m;
    if (m >= 0) {
        // tabulated: three polynomials in ln T on the cell's interval (the sigma series carry
        // the factor 27 s, kE = 27 s C_B)
        const double t = v.t;
        const float tf = v.tf;
        const double *c = a.otab + ((size_t)g * kTabNI + m) * kTabEntry;
        const float *ch = reinterpret_cast<const float *>(c + kTabNF * kTabLo);
        constexpr int kh = kTabNC - kTabLo;
        sg = horner(c, ch, t, tf) * iT3;
        sR = horner(c + kTabLo, ch + kh, t, tf) * iT3;
        em = v.kET * mx.ex(horner(c + 2 * kTabLo, ch + 2 * kh, t, tf) - xa);
    } else {
        const double k27 = 27.0 * a.s;
        const double xb = binf ? 0.0 : eb * iT;
        double dPs, Ns, Ds, om;
        group_integrals(xa, xb, binf, c_ser, mx, dPs, Ns, Ds, om);
        sg = k27 * om * iT3 * rcp64(dPs);
        sR = k27 * Ns * iT3 * rcp64(Ds);
        em = k27 * kCB * Ti * mx.ex(-xa) * om;
    }
    if (a.Erad)   // T_r option: absorption and Rosseland opacities at the radiation temperature
        opacity_tr(a.edges[g], eb, binf, v.Tr, v.rho, 27.0 * a.s, mx, sg, sR);
    a.sigE[idx] = sg;
    a.emis[idx] = em;
    a.sigR[idx] = sR;
    if (a.sig32) {   // FP32 sweep inputs: sigma_t h/2 and h e/2, one rounding each
        const double hh = 0.5 * a.h[i];
        a.sig32[idx] = (float)(hh * (sg + a.icdt));
        a.emis32[idx] = (float)(hh * em);
        // and h/(2 c dt) per cell: the sweeps read it instead of forming it in FP64 per strip
        if (g == 0) a.kap32[i] = (float)(hh * a.icdt);
    }
}

// The same quantities in FP32-pair arithmetic (TRT_LO_PAIR; outputs FP64): the three
// Horner sums with their FP64 coefficients as pairs (the FP32 tails as in horner), sigma =
// sum / T^3, and the emission 27 s C_B T e^w, w = (the emission factor's logarithm) -
// nu_g/T, by pr_exp as a pair times 2^k -- the power of two goes into the exponent of the
// FP64 result (pr_join), so e_g keeps FP64's range.  Relative errors: about 1e-14 in the
// opacities, about 3 2^-47 max(1, |w|) in e_g (w's: nu_g, 1/T and their product each
// rounded to a pair; 1.6e-11 at the smallest e_g that FP64 holds, e^-746).  m, tf: the
// cell's table interval (>= 0) and FP32 local coordinate; cells outside the tables and the
// T_r option take opacity_body (the callers' choice).
__device__ inline fpair horner_pair(const fpair *__restrict__ a, const float *__restrict__ b,
                                   fpair t, float tf)
{
    float q = b[kTabNC - kTabLo - 1];
#pragma unroll
    for (int k = kTabNC - kTabLo - 2; k >= 0; --k) q = fmaf(q, tf, b[k]);
    fpair p(q, 0.f);
#pragma unroll
    for (int k = kTabLo - 1; k >= 0; --k) p = fma(p, t, a[k]);
    return p;
}

__device__ inline void opacity_body_pair(const OpacityArgs &a, int i, int g, int m, float tf,
                                         const CellPair &cp, const fpair *e2p)
{
    const size_t idx = (size_t)g * a.nx + i;
    const fpair *c = a.otabp + ((size_t)g * kTabNI + m) * kTabEntry;
    const float *ch = reinterpret_cast<const float *>(c + kTabNF * kTabLo);
    constexpr int kh = kTabNC - kTabLo;
    const fpair sg = horner_pair(c, ch, cp.t, tf) * cp.iT3;
    const fpair sR = horner_pair(c + kTabLo, ch + kh, cp.t, tf) * cp.iT3;
    const fpair xa = a.otabp[(size_t)a.G * kTabNI * kTabEntry + g] * cp.iT;
    int k;
    const fpair em = cp.kET * pr_exp(horner_pair(c + 2 * kTabLo, ch + 2 * kh, cp.t, tf) - xa,
                                     k, e2p);
    a.sigE[idx] = pr_join(sg, 0);
    a.emis[idx] = pr_join(em, k);
    a.sigR[idx] = pr_join(sR, 0);
    if (a.sig32) {   // FP32 sweep inputs: sigma_t h/2 and h e/2, each rounded once from a pair
        const fpair st = (sg + fpair(a.icdt_h, a.icdt_l)) * cp.hh;
        a.sig32[idx] = __fadd_rn(st.h, st.l);
        const fpair eh = em * cp.hh;
        a.emis32[idx] = pr_ldexpf(__fadd_rn(eh.h, eh.l), k);
        if (g == 0) a.kap32[i] = (float)(0.5 * a.h[i] * a.icdt);
    }
}

// the 2^(j/32) table of texp in shared memory (lanes index it with different j)
__device__ inline Mx stage_exp_table(double *s_e2)
{
    if (threadIdx.y == 0 && threadIdx.x < 32) s_e2[threadIdx.x] = c_ser.e2[threadIdx.x];
    __syncthreads();
    return Mx{s_e2, ExpConsts{c_ser.einv, c_ser.eL1, c_ser.eL2}};
}

// the same table as pairs (the pair form); called after stage_exp_table's barrier
__device__ inline void stage_exp_pairs(fpair *s_e2p)
{
    if (threadIdx.y == 0 && threadIdx.x < 32) s_e2p[threadIdx.x] = fpair(c_ser.e2[threadIdx.x]);
    __syncthreads();
}

// the per-cell terms of one evaluation (single slab); the pair form's too
__global__ void k_cell_terms(OpacityArgs a)
{
    griddep_wait();
    if (a.gate && *a.gate) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nx) return;
    const CellVals v = cell_vals(a, i);
    cell_arrays(a).put(i, v);
    if (a.cpair) {
        const CellPair cp = cell_pair(a, i, v);
        const int n = a.nx;
        a.cpair[i] = cp.t;
        a.cpair[n + i] = cp.iT;
        a.cpair[2 * n + i] = cp.iT3;
        a.cpair[3 * n + i] = cp.kET;
        a.cpair[4 * n + i] = cp.hh;
    }
}

// block (32 cells, 8 groups); grid (ceil(nx / 32), ceil(G / 8)); the cells' terms from
// k_cell_terms
__global__ void __launch_bounds__(256) k_opacity(OpacityArgs a)
{
    griddep_wait();
    if (a.gate && *a.gate) return;   // the phase's inner loop has ended (every thread alike)
    __shared__ double s_e2[32];
    __shared__ fpair s_e2p[32];
    const Mx mx = stage_exp_table(s_e2);
    if (a.otabp) stage_exp_pairs(s_e2p);
    const int i = blockIdx.x * 32 + threadIdx.x, g = blockIdx.y * 8 + threadIdx.y;
    if (i >= a.nx || g >= a.G) return;
    const CellArrays ca = cell_arrays(a);
    const int m = ca.m[i];
    if (a.otabp && m >= 0 && !a.Erad) {
        const int n = a.nx;
        const CellPair cp{a.cpair[i], a.cpair[n + i], a.cpair[2 * n + i], a.cpair[3 * n + i],
                          a.cpair[4 * n + i]};
        opacity_body_pair(a, i, g, m, ca.f[i], cp, s_e2p);
    } else {
        opacity_body(a, i, g, ca.get(i), mx);
    }
}

__global__ void __launch_bounds__(256) k_opacity_b(const int *__restrict__ meta, int N,
                                                   const OpacityArgs *__restrict__ xs)
{
    __shared__ double s_e2[32];
    __shared__ fpair s_e2p[32];
    __shared__ CellTerms ct;
    const Mx mx = stage_exp_table(s_e2);
    stage_exp_pairs(s_e2p);
    for (int b = blockIdx.x;; b += gridDim.x) {
        int s, bx, by;
        if (!bdecode(meta, N, b, s, bx, by)) break;
        const OpacityArgs a = xs[s];
        stage_cells(a, bx * 32, ct, b);
        const int i = bx * 32 + threadIdx.x, g = by * 8 + threadIdx.y;
        if (i < a.nx && g < a.G) {
            const CellVals &v = ct.v[threadIdx.x];
            if (a.otabp && v.m >= 0 && !a.Erad)
                opacity_body_pair(a, i, g, v.m, v.tf, ct.p[threadIdx.x], s_e2p);
            else
                opacity_body(a, i, g, v, mx);
        }
        __syncthreads();   // the cell terms are restaged by the next work item
    }
}

// accuracy check of the device helpers: texp and rcp64 of x (test aid)
__global__ void k_fastmath(int n, const double *__restrict__ x, double *__restrict__ ex,
                           double *__restrict__ rc)
{
    __shared__ double s_e2[32];
    const Mx mx = stage_exp_table(s_e2);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    ex[i] = mx.ex(x[i]);
    rc[i] = rcp64(x[i]);
}

cudaError_t launch_fastmath(int n, const double *x, double *ex, double *rc, cudaStream_t st)
{
    cudaError_t e = ensure_tables();
    if (e != cudaSuccess) return e;
    k_fastmath<<<(n + 255) / 256, 256, 0, st>>>(n, x, ex, rc);
    return cudaGetLastError();
}

// FP64 FMA throughput probe: every thread runs 8 independent FMA chains of `reps` steps
// (x <- x * a + b with |a| < 1, so the values stay finite), the chains summed into out so
// that none is dead code.  Grid: as many CTAs of 256 threads as fit on every SM at once
// (one full wave), enough warps on every sub-partition to keep its FP64 pipe issuing.
__global__ void __launch_bounds__(256) k_fp64_probe(int reps, double a, double b, double *out)
{
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 1e-3 * (threadIdx.x + k);
    for (int r = 0; r < reps; ++r) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 123.456) out[0] = s;   // never true for these inputs; keeps the chains live
}

cudaError_t fp64_probe(int reps, cudaStream_t st, float *ms, long long *fmas)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_probe, 256, 0);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, per_sm) * sms;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fp64_probe<<<grid, 256, 0, st>>>(reps / 4, 0.999, 1e-4, nullptr);   // warm-up
    cudaEventRecord(e0, st);
    k_fp64_probe<<<grid, 256, 0, st>>>(reps, 0.999, 1e-4, nullptr);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *fmas = (long long)grid * 256 * 8 * reps;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Tables: one thread per (group, interval) evaluates the three series directly at the
// interval's kTabNC Chebyshev points in ln T (the two opacity ratios times 27 s, so the
// evaluation multiplies by T^-3 only), fits their Chebyshev coefficients and stores them
// converted to monomial coefficients in the interval's coordinate.
__global__ void k_otab_build(int G, const double *__restrict__ edges, double k27,
                             double *__restrict__ tab)
{
    __shared__ double s_e2[32];
    const Mx mx = stage_exp_table(s_e2);
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= G * kTabNI) return;
    const int g = id / kTabNI, m = id - g * kTabNI;
    const double umid = kTabU0 + kTabH * (m + 0.5);
    double fa[kTabNC], fr[kTabNC], fe[kTabNC];
    const bool binf = isinf(edges[g + 1]);
    for (int j = 0; j < kTabNC; ++j) {
        const double th = kPi * (j + 0.5) / kTabNC;
        const double T = exp(umid + 0.5 * kTabH * cos(th));
        group_ratios(T, edges[g], edges[g + 1], mx, fa[j], fr[j]);
        fa[j] *= k27;   // sigma_E T^3 and sigma_R T^3: the series carry the factor 27 s
        fr[j] *= k27;
        // emission factor: e_g = 27 s C_B T e^{-xa} (1 - e^{-w}), w = (nu_b - nu_a)/T
        fe[j] = binf ? 0.0 : log(-expm1(-(edges[g + 1] - edges[g]) / T));
    }
    double ch[kTabNF][kTabNC];   // Chebyshev coefficients (c_0 halved)
    for (int k = 0; k < kTabNC; ++k) {
        double sa = 0.0, sr = 0.0, se = 0.0;
        for (int j = 0; j < kTabNC; ++j) {
            const double ck = cos(kPi * k * (j + 0.5) / kTabNC);
            sa = fma(fa[j], ck, sa);
            sr = fma(fr[j], ck, sr);
            se = fma(fe[j], ck, se);
        }
        const double sc = (k == 0 ? 1.0 : 2.0) / kTabNC;
        ch[0][k] = sa * sc;
        ch[1][k] = sr * sc;
        ch[2][k] = se * sc;
    }
    // monomial coefficients a_j = sum_k c_k [t^j] T_k(t), the highest k first; the
    // coefficients of T_k (integers below 2^11, exact) from T_{k+1} = 2 t T_k - T_{k-1}
    double Tc[kTabNC][kTabNC];
    for (int k = 0; k < kTabNC; ++k)
        for (int j = 0; j < kTabNC; ++j) Tc[k][j] = 0.0;
    Tc[0][0] = 1.0;
    Tc[1][1] = 1.0;
    for (int k = 2; k < kTabNC; ++k)
        for (int j = 0; j < kTabNC; ++j)
            Tc[k][j] = (j > 0 ? 2.0 * Tc[k - 1][j - 1] : 0.0) - Tc[k - 2][j];
    double *c = tab + (size_t)id * kTabEntry;
    float *chi = reinterpret_cast<float *>(c + kTabNF * kTabLo);
    for (int f = 0; f < kTabNF; ++f)
        for (int j = 0; j < kTabNC; ++j) {
            double aj = 0.0;
            for (int k = kTabNC - 1; k >= j; --k) aj = fma(ch[f][k], Tc[k][j], aj);
            if (j < kTabLo)
                c[f * kTabLo + j] = aj;
            else
                chi[f * (kTabNC - kTabLo) + j - kTabLo] = (float)aj;
        }
    if (kTabHiF > kTabNF * (kTabNC - kTabLo)) chi[kTabHiF - 1] = 0.f;
}

// the pair copy of the tables (TRT_LO_PAIR): each entry's FP64 coefficients split into
// pairs, its FP32 tail copied; then the group edges as pairs
__global__ void k_otab_pair(int G, const double *__restrict__ tab,
                            const double *__restrict__ edges, fpair *__restrict__ tp)
{
    const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long n = (long)G * kTabNI * kTabEntry;
    if (id < n) {
        const int j = (int)(id % kTabEntry);
        if (j < kTabNF * kTabLo) tp[id] = fpair(tab[id]);
        else reinterpret_cast<double *>(tp)[id] = tab[id];   // the FP32 tail, bit for bit
    } else if (id < n + G + 1) {
        tp[id] = fpair(edges[id - n]);
    }
}

cudaError_t launch_otab_build(const Problem &p)
{
    if (!p.otab) return cudaSuccess;
    cudaError_t e = ensure_tables();
    if (e != cudaSuccess) return e;
    const int n = p.G * kTabNI;
    k_otab_build<<<(n + 127) / 128, 128, 0, p.stream>>>(p.G, p.edges, 27.0 * p.s, p.otab);
    e = cudaGetLastError();
    if (e != cudaSuccess || !p.otabp) return e;
    const long np = (long)n * kTabEntry + p.G + 1;
    k_otab_pair<<<(unsigned)((np + 255) / 256), 256, 0, p.stream>>>(
        p.G, p.otab, p.edges, reinterpret_cast<fpair *>(p.otabp));
    return cudaGetLastError();
}

OpacityArgs make_opacity_args(const Problem &p, const double *T, double *sigE, double *emis,
                              double *sigR, float *sig32, float *emis32, double dt,
                              const double *Erad)
{
    OpacityArgs a;
    a.Erad = p.tr_mode ? Erad : nullptr;
    a.otab = p.otab;
    a.nx = p.nx; a.G = p.G; a.T = T; a.edges = p.edges; a.s = p.s;
    a.sigE = sigE; a.emis = emis; a.sigR = sigR; a.sig32 = sig32; a.emis32 = emis32;
    a.kap32 = emis32 ? emis32 + (size_t)p.G * p.nx : nullptr;   // carved after emis32
    a.h = p.h;
    a.icdt = (dt > 0) ? 1.0 / (kC * dt) : 0.0;
    a.kE = 27.0 * p.s * kCB;   // the order of the direct path's k27 * kCB
    a.gate = p.gate;
    a.cterm = p.cterm;
    a.otabp = (p.otab && p.otabp) ? reinterpret_cast<const fpair *>(p.otabp) : nullptr;
    a.cpair = reinterpret_cast<fpair *>(p.cpair);
    a.icdt_h = (float)a.icdt;
    a.icdt_l = (float)(a.icdt - (double)a.icdt_h);
    return a;
}

// the FP32 sweep inputs from given FP64 sigma_E and e_g, with the expressions of k_opacity
// (one rounding each): sigma_t h/2, h e/2, then h/(2 c dt) per cell after h e/2
__global__ void k_prescale32(int nx, int G, const double *__restrict__ h, double icdt,
                             const double *__restrict__ sigE, const double *__restrict__ emis,
                             float *sig32, float *emis32)
{
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)G * nx) return;
    const int g = (int)(idx / nx), i = (int)(idx - (long)g * nx);
    const double hh = 0.5 * h[i];
    sig32[idx] = (float)(hh * (sigE[idx] + icdt));
    emis32[idx] = (float)(hh * emis[idx]);
    if (g == 0) emis32[(size_t)G * nx + i] = (float)(hh * icdt);
}

cudaError_t launch_prescale32(const Problem &p, double dt, const double *sigE, const double *emis,
                              float *sig32, float *emis32)
{
    const long n = (long)p.G * p.nx;
    k_prescale32<<<(unsigned)((n + 255) / 256), 256, 0, p.stream>>>(
        p.nx, p.G, p.h, 1.0 / (kC * dt), sigE, emis, sig32, emis32);
    return cudaGetLastError();
}

int opacity_gx(const Problem &p) { return (p.nx + 31) / 32; }
int opacity_blocks(const Problem &p) { return opacity_gx(p) * ((p.G + 7) / 8); }

cudaError_t launch_opacity(const Problem &p, const double *T, double *sigE, double *emis,
                           double *sigR, float *sig32, float *emis32, double dt,
                           const double *Erad)
{
    const OpacityArgs a = make_opacity_args(p, T, sigE, emis, sigR, sig32, emis32, dt, Erad);
    cudaError_t e = launch_pdl(k_cell_terms, dim3((p.nx + 127) / 128), dim3(128), 0, p.stream, a);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_opacity, dim3(opacity_gx(p), (p.G + 7) / 8), dim3(32, 8), 0, p.stream, a);
}

cudaError_t launch_opacity_b(const int *meta, int N, const OpacityArgs *xs, int grid,
                             cudaStream_t st)
{
    k_opacity_b<<<grid, dim3(32, 8), 0, st>>>(meta, N, xs);
    return cudaGetLastError();
}

}  // namespace trt
