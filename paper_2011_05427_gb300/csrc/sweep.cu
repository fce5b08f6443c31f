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
// of S: the strip's sigma_t h/2 and (h/2) e_g (read once per CTA from the [G][nx] fields,
// coalesced along cells) are staged in shared memory; each warp sweeps the strip and
// leaves psi_L + psi_R in shared memory; the CTA then reduces its D directions into the
// two angular moments per (cell, group) -- the cross-direction reduction costs one
// __syncthreads per strip, not one per cell.  Partial moments of the 2N/D direction tiles
// are summed in a fixed order by the finalize kernel (deterministic).
#include "common.cuh"

namespace trt {

namespace {

constexpr int kStrip = 32;
constexpr int kPadG = 33;   // padded group stride of the strip tables (bank conflicts)

struct SweepArgs {
    int nx, N, G, ldG, D;
    double icdt;
    const double *h, *mu, *w, *Iin0, *IinX, *sigE, *emis;
    const void *I_old;
    void *I_new;
    double *part;       // [n_dt][2][G][nx]
    double *psi_exit;   // [M][ldG]
};

template <typename R>
struct Acc {   // per-tile angular sum: plain in FP64, compensated (Kahan) in FP32
    R s, c;
    __device__ Acc() : s(0), c(0) {}
    __device__ void add(R v)
    {
        if (sizeof(R) == 8) {
            s += v;
        } else {
            R y = v - c;
            R t = s + y;
            c = (t - s) - y;
            s = t;
        }
    }
};

template <typename R>
__global__ void __launch_bounds__(512) k_sweep(SweepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int D = a.D;
    R *sth = reinterpret_cast<R *>(smem_raw);   // [S][33] sigma_t h / 2
    R *sq = sth + kStrip * kPadG;                 // [S][33] (h/2) e_g
    R *skap = sq + kStrip * kPadG;                // [S]     h / (2 c dt)
    R *ps = skap + kStrip;                        // [D][S][33] psi_L + psi_R
    const size_t off_w = (sizeof(R) * (2 * kStrip * kPadG + kStrip + D * kStrip * kPadG) + 15) / 16 * 16;
    double *swt = reinterpret_cast<double *>(smem_raw + off_w);   // [D] w/2
    double *swm = swt + D;                                        // [D] w mu^2/2

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nthr = blockDim.x;
    const int tid = threadIdx.x;
    const int dtile = blockIdx.x;
    const int gt = blockIdx.y;
    const int g = gt * 32 + lane;
    const int nx = a.nx, G = a.G, ldG = a.ldG;
    const bool pos = dtile < a.N / D;
    const int m = dtile * D + warp;

    const R *__restrict__ Iold = reinterpret_cast<const R *>(a.I_old);
    R *__restrict__ Inew = reinterpret_cast<R *>(a.I_new);

    const double mu_d = a.mu[m];
    const R am = (R)fabs(mu_d);
    const R b = (R)(0.5 * fabs(mu_d));
    const R bb = b * b;
    if (lane == 0) {
        swt[warp] = 0.5 * a.w[m];
        swm[warp] = 0.5 * a.w[m] * mu_d * mu_d;
    }
    R psi_in = (g < G) ? (R)(pos ? a.Iin0[g] : a.IinX[g]) : (R)0;

    const int nstrip = (nx + kStrip - 1) / kStrip;
    const size_t dstride = (size_t)2 * ldG;   // one cell of one direction
    const R *Iold_m = Iold + (size_t)m * nx * dstride + g;
    R *Inew_m = Inew + (size_t)m * nx * dstride + g;

    for (int st = 0; st < nstrip; ++st) {
        int c0, ns;
        if (pos) {
            c0 = st * kStrip;
            ns = min(kStrip, nx - c0);
        } else {
            int c1 = nx - st * kStrip;
            c0 = max(c1 - kStrip, 0);
            ns = c1 - c0;
        }
        __syncthreads();   // previous strip's tables are no longer read
        for (int idx = tid; idx < 32 * kStrip; idx += nthr) {
            int gl = idx / kStrip, cc = idx - gl * kStrip;
            if (cc < ns) {
                int gg = gt * 32 + gl, i = c0 + cc;
                double hi = a.h[i];
                double sg = 0.0, e = 0.0;
                if (gg < G) {
                    sg = a.sigE[(size_t)gg * nx + i];
                    e = a.emis[(size_t)gg * nx + i];
                }
                sth[cc * kPadG + gl] = (R)(0.5 * hi * (sg + a.icdt));
                sq[cc * kPadG + gl] = (R)(0.5 * hi * e);
                if (gl == 0) skap[cc] = (R)(0.5 * hi * a.icdt);
            }
        }
        __syncthreads();
        R *psw = ps + warp * kStrip * kPadG;
#pragma unroll 4
        for (int kk = 0; kk < ns; ++kk) {
            const int cc = pos ? kk : ns - 1 - kk;
            const int i = c0 + cc;
            const R IL = Iold_m[(size_t)i * dstride];
            const R IR = Iold_m[(size_t)i * dstride + ldG];
            const R aa = b + sth[cc * kPadG + lane];
            const R inv = (R)1 / (aa * aa + bb);
            const R q = sq[cc * kPadG + lane];
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
            int gl = idx / kStrip, cc = idx - gl * kStrip;
            int gg = gt * 32 + gl;
            if (cc < ns && gg < G) {
                Acc<R> s0, s2;
                for (int d = 0; d < D; ++d) {
                    R v = ps[(d * kStrip + cc) * kPadG + gl];
                    s0.add((R)swt[d] * v);
                    s2.add((R)swm[d] * v);
                }
                size_t o = ((size_t)(dtile * 2 + 0) * G + gg) * nx + c0 + cc;
                a.part[o] = (double)s0.s;
                a.part[o + (size_t)G * nx] = (double)s2.s;
            }
        }
    }
    a.psi_exit[(size_t)m * ldG + g] = (double)psi_in;
}

// f_g = sum_t A2 / sum_t A0 per (group, cell); boundary factors per group.
__global__ void k_sweep_finalize(int nx, int N, int G, int ldG, int ntile,
                                 const double *__restrict__ part, const double *__restrict__ mu,
                                 const double *__restrict__ w, const double *__restrict__ Iin0,
                                 const double *__restrict__ IinX,
                                 const double *__restrict__ psi_exit, double *__restrict__ f,
                                 double *fb0, double *fbX, double *C0, double *CX)
{
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long n = (long)G * nx;
    if (idx < n) {
        double A0 = 0.0, A2 = 0.0;
        for (int t = 0; t < ntile; ++t) {
            A0 += part[(size_t)(t * 2 + 0) * n + idx];
            A2 += part[(size_t)(t * 2 + 1) * n + idx];
        }
        f[idx] = (A0 != 0.0) ? A2 / A0 : 1.0 / 3.0;
    }
    if (idx < G) {
        const int g = (int)idx, M = 2 * N;
        double s0 = 0, s2 = 0, h0 = 0, h1 = 0;
        for (int m = 0; m < M; ++m) {   // x = 0: inflow for mu > 0, outflow for mu < 0
            double psi = (m < N) ? Iin0[g] : psi_exit[(size_t)m * ldG + g];
            s0 += w[m] * psi;
            s2 += w[m] * mu[m] * mu[m] * psi;
            if (m >= N) { h0 += w[m] * psi; h1 += w[m] * mu[m] * psi; }
        }
        fb0[g] = (s0 != 0.0) ? s2 / s0 : 1.0 / 3.0;
        C0[g] = (h0 != 0.0) ? h1 / h0 : -0.5;
        s0 = s2 = h0 = h1 = 0;
        for (int m = 0; m < M; ++m) {   // x = X: outflow for mu > 0, inflow for mu < 0
            double psi = (m < N) ? psi_exit[(size_t)m * ldG + g] : IinX[g];
            s0 += w[m] * psi;
            s2 += w[m] * mu[m] * mu[m] * psi;
            if (m < N) { h0 += w[m] * psi; h1 += w[m] * mu[m] * psi; }
        }
        fbX[g] = (s0 != 0.0) ? s2 / s0 : 1.0 / 3.0;
        CX[g] = (h0 != 0.0) ? h1 / h0 : 0.5;
    }
}

int pick_D(int N)
{
    for (int D = 8; D >= 1; D >>= 1)
        if (N % D == 0) return D;
    return 1;
}

}  // namespace

size_t sweep_partial_doubles(const Problem &p)
{
    int D = pick_D(p.N);
    return (size_t)(p.M / D) * 2 * p.G * p.nx;
}

cudaError_t launch_sweep(const Problem &p, double dt, const double *sigE, const double *emis,
                         const void *I_old, void *I_new, double *part, double *psi_exit,
                         double *f, double *fb0, double *fbX, double *C0, double *CX)
{
    SweepArgs a;
    a.nx = p.nx; a.N = p.N; a.G = p.G; a.ldG = p.ldG;
    a.D = pick_D(p.N);
    a.icdt = 1.0 / (kC * dt);
    a.h = p.h; a.mu = p.mu; a.w = p.w; a.Iin0 = p.Iin0; a.IinX = p.IinX;
    a.sigE = sigE; a.emis = emis; a.I_old = I_old; a.I_new = I_new;
    a.part = part; a.psi_exit = psi_exit;
    const int ntile = p.M / a.D;
    dim3 grid(ntile, p.ldG / 32);
    dim3 block(32 * a.D);
    cudaError_t e;
    if (p.precision == TRT_FP64) {
        size_t sm = sizeof(double) * (2 * kStrip * kPadG + kStrip + a.D * kStrip * kPadG);
        sm = (sm + 15) / 16 * 16 + sizeof(double) * 2 * a.D;
        e = cudaFuncSetAttribute(k_sweep<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm);
        if (e != cudaSuccess) return e;
        k_sweep<double><<<grid, block, sm, p.stream>>>(a);
    } else {
        size_t sm = sizeof(float) * (2 * kStrip * kPadG + kStrip + a.D * kStrip * kPadG);
        sm = (sm + 15) / 16 * 16 + sizeof(double) * 2 * a.D;
        e = cudaFuncSetAttribute(k_sweep<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm);
        if (e != cudaSuccess) return e;
        k_sweep<float><<<grid, block, sm, p.stream>>>(a);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    long n = (long)p.G * p.nx;
    int bs = 256;
    k_sweep_finalize<<<(unsigned)((n + bs - 1) / bs), bs, 0, p.stream>>>(
        p.nx, p.N, p.G, p.ldG, ntile, part, p.mu, p.w, p.Iin0, p.IinX, psi_exit, f, fb0, fbX,
        C0, CX);
    return cudaGetLastError();
}

}  // namespace trt
