// physics.cu -- group opacities and Planck integrals at cell temperatures (kernel K1).
//
// Sec. 2 / Sec. 3.1 / Sec. 6 of the paper: with x = nu/T,
//   B_g     = CB T^4 [P(x_{g+1}) - P(x_g)],           P(x) = int_0^x t^3/(e^t-1) dt
//   e_g     = int sigma B = s 27 CB T (e^{-x_g} - e^{-x_{g+1}})   (sigma B = 27 s CB e^{-nu/T})
//   sigma_B = e_g / B_g = sigma_E          (T_r = T)
//   sigma_R = s 27 N_g / (T^3 D_g),  N_g = [-x^4/(e^x-1) + 4 P(x)],  D_g = [int t^7 e^{2t}/(e^t-1)^3]
// Every per-edge integral is evaluated in closed form: a power series below x = 2 (radius
// of convergence 2 pi; the coefficients follow from t/(e^t-1) = sum B_n t^n / n!), and
// exponentially convergent tails e^{-kx} at and above it, summed with the scale e^{x_g}
// factored out so that cold cells (x ~ 1e5) neither underflow nor lose the ratio.
#include <cmath>
#include "common.cuh"

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
    gauss_legendre_host(8, t.gx, t.gw);
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
__host__ __device__ inline void edge_tail(double x, double &TP, double &TN, double &TD)
{
    double q = exp(-x);
    double ek = 1.0;
    double sp = 0.0, sd = 0.0;
    for (int k = 1; k <= 64; ++k) {
        double kk = (double)k;
        double y = kk * x;
        double e3 = 1.0 + y * (1.0 + y * (0.5 + y * (1.0 / 6.0)));
        double e7 = 1.0 + y * (1.0 + y * (1.0 / 2 + y * (1.0 / 6 + y * (1.0 / 24 + y * (1.0 / 120
                    + y * (1.0 / 720 + y * (1.0 / 5040)))))));
        double k2 = kk * kk, k4 = k2 * k2;
        sp += ek * 6.0 * e3 / k4;
        sd += ek * (0.5 * kk * (kk + 1.0)) * 5040.0 * e7 / (k4 * k4);
        ek *= q;
        if (ek < 1e-18) break;
    }
    TP = sp;
    TD = sd;
    TN = x * x * x * x / (-expm1(-x));
}

// e^{xa} [P]_{xa}^{xb}, e^{xa} [Nt]_{xa}^{xb}, e^{xa} [D]_{xa}^{xb}, and 1 - e^{-(xb-xa)}.
// Narrow groups (xb - xa <= 1) integrate the three integrands directly with the 8-point
// Gauss rule (the differences of edge values would cancel); wide groups difference the
// closed forms.  Scaled integrands: x^3 e^{xa-x}/(1-e^{-x}), x^4 e^{xa-x}/(1-e^{-x})^2,
// x^7 e^{xa-x}/(1-e^{-x})^3.
__host__ __device__ inline void group_integrals(double xa, double xb, bool binf,
                                                const SeriesTables &t, double &dPs,
                                                double &Ns, double &Ds, double &om)
{
    om = binf ? 1.0 : -expm1(-(xb - xa));
    if (!binf && xb - xa <= 1.0) {
        const double hw = 0.5 * (xb - xa), mid = 0.5 * (xb + xa);
        double sp = 0.0, sn = 0.0, sd = 0.0;
        for (int j = 0; j < 8; ++j) {
            const double x = mid + hw * t.gx[j];
            const double u = 1.0 / (-expm1(-x));
            const double e = exp(xa - x) * t.gw[j];
            const double x3 = x * x * x;
            sp += e * x3 * u;
            sn += e * x3 * x * u * u;
            sd += e * x3 * x3 * x * u * u * u;
        }
        dPs = hw * sp;
        Ns = hw * sn;
        Ds = hw * sd;
        return;
    }
    if (xa >= kXSplit) {
        double TPa, TNa, TDa, TPb = 0.0, TNb = 0.0, TDb = 0.0, r = 0.0;
        edge_tail(xa, TPa, TNa, TDa);
        if (!binf) {
            edge_tail(xb, TPb, TNb, TDb);
            r = exp(xa - xb);
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
            edge_tail(xb, TP, TN, TD);
            double eb = exp(-xb);
            Pb = t.Pinf - eb * TP;
            Nb = -eb * TN + 4.0 * Pb;
            Db = t.Dinf - eb * TD;
        }
        double ea = exp(xa);
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
        group_integrals(xa, xb, binf, t, dPs, Ns, Ds, om);
        B[g] = kCB * T * T * T * T * exp(-xa) * dPs;
    }
}

// One thread per (group, cell); outputs [G][nx] (cell fastest, coalesced).
__global__ void __launch_bounds__(256) k_opacity(int nx, int G, const double *__restrict__ T,
                                                 const double *__restrict__ edges, double s,
                                                 double *__restrict__ sigE,
                                                 double *__restrict__ emis,
                                                 double *__restrict__ sigR)
{
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)G * nx) return;
    int g = (int)(idx / nx);
    int i = (int)(idx - (long)g * nx);
    double Ti = T[i];
    double xa = edges[g] / Ti;
    double eb = edges[g + 1];
    bool binf = isinf(eb);
    double xb = binf ? 0.0 : eb / Ti;
    double dPs, Ns, Ds, om;
    group_integrals(xa, xb, binf, c_ser, dPs, Ns, Ds, om);
    double T3 = Ti * Ti * Ti;
    double k27 = 27.0 * s;
    sigE[idx] = k27 * om / (T3 * dPs);
    emis[idx] = k27 * kCB * Ti * exp(-xa) * om;
    sigR[idx] = k27 * Ns / (T3 * Ds);
}

cudaError_t launch_opacity(const Problem &p, const double *T, double *sigE, double *emis,
                           double *sigR)
{
    long n = (long)p.G * p.nx;
    int bs = 256;
    long nb = (n + bs - 1) / bs;
    k_opacity<<<(unsigned)nb, bs, 0, p.stream>>>(p.nx, p.G, T, p.edges, p.s, sigE, emis, sigR);
    return cudaGetLastError();
}

}  // namespace trt
