// lo.cu -- low-order QD systems (K3/K4), restriction between frequency grids (K4), grey
// LOQD + material energy balance Newton step (K5).
//
// One group of one level (eq. mloqd-d, eq. mloqd-d-gamma, Sec. 5) is
//   cell i:  (dx_i/dt)(E_i - Eold_i) + F_{i+1/2} - F_{i-1/2} + dx_i a_i E_i = dx_i s_i
//   face f:  (dx_f/(c dt))(F - Fold) + c (phiR E_right - phiL E_left) + sigR dx_f F = 0
// with a = c sigma_E, s = 2 sigma_B B on the group levels; phiR = phi_right + eta-hat,
// phiL = phi_left + eta-check; the boundary faces close a half cell with eq. mloqd-bcs
// (F = c C (E_face - E_in) + F_in, the face energy eliminated).  Eliminating F face by
// face, F_f = GD_f + PL_f E_{f-1} - PR_f E_f, gives a tridiagonal system in E that is
// column diagonally dominant (the dx/dt term), so elimination needs no pivoting.
//
// GB300 mapping.  A warp owns one system.  FP64 throughput on GB300 is a small fraction of
// FP32, so the solver keeps the FP64 work of plain Thomas elimination (one reciprocal per
// row) but splits the serial chain: lane l eliminates its chunk of >= 2 consecutive rows
// (a "modified Thomas" pass down and up the chunk that leaves each row coupled only to the
// chunk's first and last unknowns), the 2 x 32 chunk-boundary unknowns form a tridiagonal
// system solved by parallel cyclic reduction in registers with warp shuffles, and every
// lane back-substitutes its interior rows.  Rows are built on the fly from the level's
// fields; per-warp shared memory holds the chunk coefficients in a [row-in-chunk][lane]
// layout (conflict free).
#include <cmath>
#include "batch.cuh"
#include "pair.cuh"

namespace trt {

namespace {

template <typename R>
__device__ inline R rcpR(R d);
template <>
__device__ inline double rcpR<double>(double d) { return rcp64(d); }
template <>
__device__ inline float rcpR<float>(float d) { return __frcp_rn(d); }
template <>
__device__ inline fpair rcpR<fpair>(fpair d) { return prcp(d); }

// Source terms of a group system (Eold, the emission, Fold, the boundary inflows) and its
// solution (E, F) in the pair form are held scaled by 2^-ks, ks the group's largest source
// exponent (lo_src_exp): the system is linear in them, and FP32's exponent range would
// otherwise cut the small groups' precision (values below 2^-103) or zero them (below
// 2^-126).  The coefficients are not scaled.  FP64 and FP32: ks is unused.
template <typename R>
__device__ inline R src_in(double v, int ks)
{
    if constexpr (is_pair<R>) return pr_split(v, ks);
    else return (R)v;
}
template <typename R>
__device__ inline double sol_out(R v, int ks)
{
    if constexpr (is_pair<R>) return pr_join(v, ks);
    else return (double)v;
}
// row constant j of kind k (the Problem::lopc order: 0 hf, 1 dxicdt, 2 fwl, 3 fwr, 4 hidt,
// 5 hc, 6 h2, 7 h): the pair form reads the pair copy, the others the FP64 array d
template <typename R>
__device__ inline R lc(const LoCtx &x, int k, int j, const double *d)
{
    if constexpr (is_pair<R>) return x.pc[(size_t)k * (x.nx + 1) + j];
    else return (R)d[j];
}
__device__ inline int bexp64(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }
// the largest biased exponent of group q's source terms over this thread's cells and faces
// (threads t, t + nthr, ...); 0 when they are all zero
__device__ inline int lo_src_exp(const LoCtx &x, int q, int t, int nthr)
{
    const int n = x.nx;
    int m = 0;
    for (int i = t; i <= n; i += nthr) {
        if (i < n) {
            m = max(m, bexp64(x.L.Eold[(size_t)q * n + i]));
            m = max(m, bexp64(x.a_cell ? x.s_cell[i] : x.L.emis[(size_t)q * n + i]));
        }
        m = max(m, bexp64(x.L.Fold[(size_t)q * (n + 1) + i]));
    }
    if (t == 0)
        m = max(max(m, max(bexp64(x.L.Ein0[q]), bexp64(x.L.Fin0[q]))),
                max(bexp64(x.L.EinX[q]), bexp64(x.L.FinX[q])));
    return m;
}


__device__ inline double sigR_face(const LoCtx &x, int q, int f)
{
    const int nx = x.nx;
    if (!x.L.fine) return x.L.sigR[(size_t)q * (nx + 1) + f];
    const double *sc = x.L.sigR + (size_t)q * nx;
    if (f == 0) return sc[0];
    if (f == nx) return sc[nx - 1];
    return (sc[f - 1] * x.h[f - 1] + sc[f] * x.h[f]) * x.ihf[f];
}

// F_f = GD + PL E_{f-1} - PR E_f  (boundary faces: the face energy already eliminated).
// kW: GD is instead W = dx/(c dt) / D, the factor of Fold in GD, without the boundary
// inflow terms (the first pass of the pair staging, before the source scale is known).
template <typename R, bool kW = false>
__device__ inline void face_coef(const LoCtx &x, int q, int f, R &PL, R &PR, R &GD, int ks = 0)
{
    const int nx = x.nx;
    const double *phi = x.L.phi + (size_t)q * nx;
    const R dx = lc<R>(x, 0, f, x.hf);
    R phiL, phiR;
    if (f == 0) {
        phiL = (R)x.L.phib0[q];
        phiR = (R)phi[0];
    } else if (f == nx) {
        phiL = (R)phi[nx - 1];
        phiR = (R)x.L.phibX[q];
    } else {
        phiL = (R)phi[f - 1];
        phiR = (R)phi[f];
    }
    if (!x.L.fine) {
        phiL += (R)x.L.etaL[(size_t)q * (nx + 1) + f];
        phiR += (R)x.L.etaR[(size_t)q * (nx + 1) + f];
    }
    const R c = (R)kC;
    R D, Gf;
    if constexpr (!std::is_same<R, float>::value) {
        // dx (1/(c dt) + sigma_R,face) and dx Fold/(c dt) from the row constants: the face
        // opacity's dx-weighted mean folded into one FMA per cell opacity
        const R dxi = lc<R>(x, 1, f, x.dxicdt);
        if (!x.L.fine) {
            D = fma(dx, (R)x.L.sigR[(size_t)q * (nx + 1) + f], dxi);
        } else {
            const double *sc = x.L.sigR + (size_t)q * nx;
            D = (f == 0)    ? fma(dx, (R)sc[0], dxi)
                : (f == nx) ? fma(dx, (R)sc[nx - 1], dxi)
                            : fma(lc<R>(x, 2, f, x.fwl), (R)sc[f - 1],
                                  fma(lc<R>(x, 3, f, x.fwr), (R)sc[f], dxi));
        }
        if constexpr (kW) Gf = dxi;
        else Gf = src_in<R>(x.L.Fold[(size_t)q * (nx + 1) + f], ks) * dxi;
    } else {
        const R icdt = (R)x.icdt;
        D = dx * (icdt + (R)sigR_face(x, q, f));
        Gf = dx * (R)x.L.Fold[(size_t)q * (nx + 1) + f] * icdt;
    }
    if (f == 0) {
        const R iC0 = rcpR<R>((R)x.L.C0[q]);
        D -= phiL * iC0;
        if constexpr (!kW)
            Gf += c * phiL * src_in<R>(x.L.Ein0[q], ks) - phiL * src_in<R>(x.L.Fin0[q], ks) * iC0;
    } else if (f == nx) {
        const R iCX = rcpR<R>((R)x.L.CX[q]);
        D += phiR * iCX;
        if constexpr (!kW)
            Gf += -c * phiR * src_in<R>(x.L.EinX[q], ks) + phiR * src_in<R>(x.L.FinX[q], ks) * iCX;
    }
    const R iD = rcpR<R>(D);
    const R ciD = c * iD;
    PL = phiL * ciD;
    PR = phiR * ciD;
    GD = Gf * iD;
}

// row i of the cell equation: Ap = h (1/dt + a), Dp = h (s + Eold/dt)
template <typename R>
__device__ inline void cell_row(const LoCtx &x, int q, int i, R &Ap, R &Dp, int ks = 0)
{
    const R Eo = src_in<R>(x.L.Eold[(size_t)q * x.nx + i], ks);
    if constexpr (!std::is_same<R, float>::value) {   // from the row constants h/dt, c h, 2 h
        const R hidt = lc<R>(x, 4, i, x.hidt);
        if (x.a_cell) {
            const R hc = lc<R>(x, 7, i, x.h);
            Ap = fma(hc, (R)x.a_cell[i], hidt);
            Dp = fma(hidt, Eo, hc * src_in<R>(x.s_cell[i], ks));
        } else {
            Ap = fma(lc<R>(x, 5, i, x.hc), (R)x.L.sig[(size_t)q * x.nx + i], hidt);
            Dp = fma(hidt, Eo, lc<R>(x, 6, i, x.h2) * src_in<R>(x.L.emis[(size_t)q * x.nx + i], ks));
        }
        return;
    }
    const R hi = (R)x.h[i], idt = (R)x.idt;
    if (x.a_cell) {
        Ap = hi * (idt + (R)x.a_cell[i]);
        Dp = hi * fma(Eo, idt, (R)x.s_cell[i]);
    } else {
        Ap = hi * fma((R)kC, (R)x.L.sig[(size_t)q * x.nx + i], idt);
        Dp = hi * fma(Eo, idt, (R)2 * (R)x.L.emis[(size_t)q * x.nx + i]);
    }
}

// Solve system q with one warp.  sm: 6 * 32 * mmax values of R for this warp.
// Writes E, F, Eb0, EbX of system q.
//   phase A (all lanes, coalesced over cells/faces): face coefficients PL, PR, GD and the
//           row parts dx/dt + dx a, dx s + dx Eold/dt, stored in the chunk layout
//           [row-in-chunk][lane] so that phase B reads conflict free;
//   phase B (each lane its chunk): modified Thomas down and up the chunk;
//   phase C (warp): parallel cyclic reduction of the 2 x 32 chunk-boundary rows;
//   phase D (each lane): back substitution, then the fluxes of its faces.

// Phase A for system q by `nthr` cooperating threads (index `t`): face coefficients and
// row parts into the chunk layout.  n >= 2.
template <typename R>
__device__ void lo_stage(const LoCtx &x, int q, R *sm, int mmax, int t, int nthr, int ks = 0)
{
    const int n = x.nx;
    const int S = 32 * mmax;
    R *PLc = sm, *PRc = sm + S, *GDc = sm + 2 * S, *Ap = sm + 3 * S, *Dp = sm + 5 * S;
    for (int f = t; f <= n; f += nthr) {
        // slot k * 32 + l (chunk l = the lane whose rows hold f, row k of the chunk;
        // face n after the last chunk's last row): a table built with the problem
        const int o = x.lo_slot[f];
        R PL, PR, GD;
        face_coef<R>(x, q, f, PL, PR, GD, ks);
        PLc[o] = PL;
        PRc[o] = PR;
        GDc[o] = GD;
        if (f < n) cell_row<R>(x, q, f, Ap[o], Dp[o], ks);
    }
}

// Phase A in the pair form by the CTA (t = threadIdx.x), with the group's source scale
// (src_in): pass 1 forms the coefficients PL, PR, Ap and the face factor W of Fold (a 7th
// array after the six of the solve) and parks the raw FP64 sources in slots the
// elimination fills later (Fold in GD's, Eold in Dp's, the emission in Cp's) while it
// takes their largest exponent; the CTA's maximum gives ks; pass 2 splits the parked
// sources at that scale into GD and Dp (the boundary faces are formed again whole, with
// their inflow terms).  Each slot is written and read again by one thread, so only the
// reduction needs a barrier.  Returns ks.  n >= 2.
__device__ int lo_stage_pair(const LoCtx &x, int q, fpair *sm, int mmax)
{
    const int n = x.nx;
    const int S = 32 * mmax;
    const int t = threadIdx.x, nthr = blockDim.x;
    fpair *PLc = sm, *PRc = sm + S, *GDc = sm + 2 * S, *Ap = sm + 3 * S, *Cp = sm + 4 * S,
          *Dp = sm + 5 * S, *Wc = sm + 6 * S;
    double *rawF = reinterpret_cast<double *>(GDc), *rawE = reinterpret_cast<double *>(Dp),
           *rawS = reinterpret_cast<double *>(Cp);
    int m = 0;
    for (int f = t; f <= n; f += nthr) {
        const int o = x.lo_slot[f];
        fpair PL, PR, W;
        face_coef<fpair, true>(x, q, f, PL, PR, W);
        PLc[o] = PL;
        PRc[o] = PR;
        Wc[o] = W;
        const double Fo = x.L.Fold[(size_t)q * (n + 1) + f];
        rawF[o] = Fo;
        m = max(m, bexp64(Fo));
        if (f < n) {
            const double Eo = x.L.Eold[(size_t)q * n + f];
            const double sv = x.a_cell ? x.s_cell[f] : x.L.emis[(size_t)q * n + f];
            rawE[o] = Eo;
            rawS[o] = sv;
            m = max(m, max(bexp64(Eo), bexp64(sv)));
            const fpair hidt = lc<fpair>(x, 4, f, x.hidt);
            Ap[o] = x.a_cell ? fma(lc<fpair>(x, 7, f, x.h), (fpair)x.a_cell[f], hidt)
                             : fma(lc<fpair>(x, 5, f, x.hc), (fpair)x.L.sig[(size_t)q * n + f], hidt);
        }
    }
    if (t == 0)
        m = max(max(m, max(bexp64(x.L.Ein0[q]), bexp64(x.L.Fin0[q]))),
                max(bexp64(x.L.EinX[q]), bexp64(x.L.FinX[q])));
    __shared__ int kw[32];
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((t & 31) == 0) kw[t >> 5] = m;
    __syncthreads();
    m = 0;
    for (int w = 0; w < (nthr >> 5); ++w) m = max(m, kw[w]);
    const int ks = (m == 0) ? 0 : m - 1023;
    for (int f = t; f <= n; f += nthr) {
        const int o = x.lo_slot[f];
        if (f == 0 || f == n) {
            fpair PL, PR, GD;
            face_coef<fpair>(x, q, f, PL, PR, GD, ks);
            GDc[o] = GD;
        } else {
            GDc[o] = pr_split(rawF[o], ks) * Wc[o];
        }
        if (f < n) {
            const fpair sv = pr_split(rawS[o], ks);
            const fpair Eo = pr_split(rawE[o], ks);
            Dp[o] = fma(lc<fpair>(x, 4, f, x.hidt), Eo,
                        (x.a_cell ? lc<fpair>(x, 7, f, x.h) : lc<fpair>(x, 6, f, x.h2)) * sv);
        }
    }
    return ks;
}

// Phases B-D of one system by one warp on the staged arrays in sm: the solution x ends in
// the Dp array (chunk layout); nothing is written to global memory.  n >= 2.
template <typename R>
__device__ void tri_solve(R *sm, int n, int mmax)
{
    const int lane = threadIdx.x & 31;
    const int P = min(32, n / 2);
    const bool act = lane < P;
    const int r0 = act ? (lane * n) / P : n;
    const int r1 = act ? ((lane + 1) * n) / P : n;
    const int m = r1 - r0;
    const int S = 32 * mmax;
    R *PLc = sm, *PRc = sm + S, *GDc = sm + 2 * S;
    R *Ap = sm + 3 * S, *Cp = sm + 4 * S, *Dp = sm + 5 * S;
#define CH(arr, k, l) arr[(k) * 32 + (l)]

    R x0 = 0, x1 = 0;
    R A0r = 0, C0r = 0, D0r = 0, A1r = 0, C1r = 0, D1r = 0;   // reduced rows
    if (act) {
        // ---- phase B: rows r0..r1-1, each normalised, coupled to x_{r0} and x_{k+1} ----
        R PLi = CH(PLc, 0, lane), PRi = CH(PRc, 0, lane), GDi = CH(GDc, 0, lane);
        R ap = 0, cp = 0, dp = 0;
        for (int k = 0; k < m; ++k) {
            const int i = r0 + k;
            R PL1, PR1, GD1;
            if (k + 1 < m || lane == P - 1) {
                PL1 = CH(PLc, k + 1, lane); PR1 = CH(PRc, k + 1, lane); GD1 = CH(GDc, k + 1, lane);
            } else {
                PL1 = CH(PLc, 0, lane + 1); PR1 = CH(PRc, 0, lane + 1); GD1 = CH(GDc, 0, lane + 1);
            }
            const R di = CH(Ap, k, lane) + PL1 + PRi;
            const R rh = CH(Dp, k, lane) - GD1 + GDi;
            const R lo = (i > 0) ? -PLi : (R)0;
            const R up = (i < n - 1) ? -PR1 : (R)0;
            if (k < 2) {
                const R r = rcpR<R>(di);
                ap = lo * r;
                cp = up * r;
                dp = rh * r;
            } else {
                const R r = rcpR<R>(di - lo * cp);
                dp = r * (rh - lo * dp);
                ap = -r * lo * ap;
                cp = r * up;
            }
            CH(Ap, k, lane) = ap;
            CH(Cp, k, lane) = cp;
            CH(Dp, k, lane) = dp;
            PLi = PL1;
            PRi = PR1;
            GDi = GD1;
        }
        // backward: rows k = m-3..1 coupled to x_{r0} and x_{r1-1}
        if (m >= 3) {
            for (int k = m - 3; k >= 1; --k) {
                const R ck = CH(Cp, k, lane);
                CH(Dp, k, lane) = CH(Dp, k, lane) - ck * CH(Dp, k + 1, lane);
                CH(Ap, k, lane) = CH(Ap, k, lane) - ck * CH(Ap, k + 1, lane);
                CH(Cp, k, lane) = -ck * CH(Cp, k + 1, lane);
            }
            const R c0 = CH(Cp, 0, lane);
            const R r = rcpR<R>((R)1 - c0 * CH(Ap, 1, lane));
            CH(Dp, 0, lane) = r * (CH(Dp, 0, lane) - c0 * CH(Dp, 1, lane));
            CH(Ap, 0, lane) = r * CH(Ap, 0, lane);
            CH(Cp, 0, lane) = -r * c0 * CH(Cp, 1, lane);
        }
        A0r = CH(Ap, 0, lane); C0r = CH(Cp, 0, lane); D0r = CH(Dp, 0, lane);
        A1r = CH(Ap, m - 1, lane); C1r = CH(Cp, m - 1, lane); D1r = CH(Dp, m - 1, lane);
    }
    // ---- phase C: reduced system rows (first_l, last_l), l = 0..31, PCR with shuffles ----
    // Every row is kept with a unit diagonal (the reduced rows of phase B already are):
    // a level eliminates the neighbours at distance s with the factors -A and -C, then
    // divides the row by its new diagonal -- one reciprocal per row and level instead of
    // one per neighbour, and no diagonals to exchange.
    {
        if (!act) { A0r = C0r = D0r = A1r = C1r = D1r = 0; }
        const unsigned full = 0xffffffffu;
        for (int s = 1; s < 64; s <<= 1) {
            R lA0, lC0, lD0, uA0, uC0, uD0;   // neighbours of slot 0 (unit diagonals)
            R lA1, lC1, lD1, uA1, uC1, uD1;   // neighbours of slot 1
            if (s == 1) {
                R tA = shfl_up(full, A1r, 1), tC = shfl_up(full, C1r, 1);
                R tD = shfl_up(full, D1r, 1);
                R vA = shfl_down(full, A0r, 1), vC = shfl_down(full, C0r, 1);
                R vD = shfl_down(full, D0r, 1);
                if (lane >= 1) { lA0 = tA; lC0 = tC; lD0 = tD; }
                else { lA0 = 0; lC0 = 0; lD0 = 0; }
                uA0 = A1r; uC0 = C1r; uD0 = D1r;
                lA1 = A0r; lC1 = C0r; lD1 = D0r;
                if (lane <= 30) { uA1 = vA; uC1 = vC; uD1 = vD; }
                else { uA1 = 0; uC1 = 0; uD1 = 0; }
            } else {
                const int t = s >> 1;
                R a0 = shfl_up(full, A0r, t), c0 = shfl_up(full, C0r, t);
                R d0 = shfl_up(full, D0r, t);
                R a1 = shfl_up(full, A1r, t), c1 = shfl_up(full, C1r, t);
                R d1 = shfl_up(full, D1r, t);
                R e0 = shfl_down(full, A0r, t), g0 = shfl_down(full, C0r, t);
                R h0 = shfl_down(full, D0r, t);
                R e1 = shfl_down(full, A1r, t), g1 = shfl_down(full, C1r, t);
                R h1 = shfl_down(full, D1r, t);
                if (lane >= t) {
                    lA0 = a0; lC0 = c0; lD0 = d0;
                    lA1 = a1; lC1 = c1; lD1 = d1;
                } else {
                    lA0 = lA1 = 0; lC0 = lC1 = 0; lD0 = lD1 = 0;
                }
                if (lane + t <= 31) {
                    uA0 = e0; uC0 = g0; uD0 = h0;
                    uA1 = e1; uC1 = g1; uD1 = h1;
                } else {
                    uA0 = uA1 = 0; uC0 = uC1 = 0; uD0 = uD1 = 0;
                }
            }
            {
                const R al = -A0r, ga = -C0r;
                const R r = rcpR<R>((R)1 + al * lC0 + ga * uA0);
                const R nA = al * lA0, nC = ga * uC0, nD = D0r + al * lD0 + ga * uD0;
                A0r = nA * r; C0r = nC * r; D0r = nD * r;
            }
            {
                const R al = -A1r, ga = -C1r;
                const R r = rcpR<R>((R)1 + al * lC1 + ga * uA1);
                const R nA = al * lA1, nC = ga * uC1, nD = D1r + al * lD1 + ga * uD1;
                A1r = nA * r; C1r = nC * r; D1r = nD * r;
            }
        }
        x0 = D0r;
        x1 = D1r;
    }
    // ---- phase D: back substitution (E into Dp), then the fluxes ----
    if (act) {
        for (int k = 1; k < m - 1; ++k)
            CH(Dp, k, lane) = CH(Dp, k, lane) - CH(Ap, k, lane) * x0 - CH(Cp, k, lane) * x1;
        CH(Dp, 0, lane) = x0;
        CH(Dp, m - 1, lane) = x1;
    }
    __syncwarp();
#undef CH
}

// The outputs of system q from the solution in the Dp array and the face coefficients:
// E, F (F_f = GD_f + PL_f E_{f-1} - PR_f E_f) and the boundary face energies.  n >= 2.
template <typename R>
__device__ void lo_outputs(const LoCtx &x, int q, R *sm, int mmax, int ks = 0)
{
    const int lane = threadIdx.x & 31;
    const int n = x.nx;
    double *E = x.L.E + (size_t)q * n;
    double *F = x.L.F + (size_t)q * (n + 1);
    const int P = min(32, n / 2);
    const bool act = lane < P;
    const int r0 = act ? (lane * n) / P : n;
    const int r1 = act ? ((lane + 1) * n) / P : n;
    const int m = r1 - r0;
    const int S = 32 * mmax;
    R *PLc = sm, *PRc = sm + S, *GDc = sm + 2 * S;
    R *Ap = sm + 3 * S, *Cp = sm + 4 * S, *Dp = sm + 5 * S;
#define CH(arr, k, l) arr[(k) * 32 + (l)]

    if (act)
        for (int k = 0; k < m; ++k) E[r0 + k] = sol_out<R>(CH(Dp, k, lane), ks);
    if (act) {
        const int mprev = (lane > 0) ? r0 - ((lane - 1) * n) / P : 0;
        const R Eleft0 = (lane > 0) ? CH(Dp, mprev - 1, lane - 1) : (R)0;
        const int kend = (lane == P - 1) ? m : m - 1;
        for (int k = 0; k <= kend; ++k) {
            const int f = r0 + k;
            R Fv = CH(GDc, k, lane);
            if (f > 0) Fv += CH(PLc, k, lane) * ((k == 0) ? Eleft0 : CH(Dp, k - 1, lane));
            if (f < n) Fv -= CH(PRc, k, lane) * CH(Dp, k, lane);
            const double Fd = sol_out<R>(Fv, ks);
            F[f] = Fd;
            if (f == 0) x.L.Eb0[q] = x.L.Ein0[q] + (Fd - x.L.Fin0[q]) / (kC * x.L.C0[q]);
            if (f == n) x.L.EbX[q] = x.L.EinX[q] + (Fd - x.L.FinX[q]) / (kC * x.L.CX[q]);
        }
    }
#undef CH
}

// The outputs of system q by every thread of the CTA, from the solution (chunk layout, in
// the Dp array) and the face coefficients: consecutive threads take consecutive cells and
// faces (coalesced stores), each slot found through the slot table.  The boundary face
// energies as in lo_outputs (the pair form in pair arithmetic, at the source scale).
// n >= 2; called after a barrier that follows the elimination.
template <typename R>
__device__ void lo_outputs_cta(const LoCtx &x, int q, const R *sm, int mmax, int ks)
{
    const int n = x.nx;
    const int S = 32 * mmax;
    const R *PLc = sm, *PRc = sm + S, *GDc = sm + 2 * S, *Dp = sm + 5 * S;
    double *E = x.L.E + (size_t)q * n;
    double *F = x.L.F + (size_t)q * (n + 1);
    for (int f = threadIdx.x; f <= n; f += blockDim.x) {
        const int o = x.lo_slot[f];
        R Fv = GDc[o];
        if (f > 0) Fv += PLc[o] * Dp[x.lo_slot[f - 1]];
        if (f < n) {
            const R Ef = Dp[o];
            Fv -= PRc[o] * Ef;
            E[f] = sol_out<R>(Ef, ks);
        }
        F[f] = sol_out<R>(Fv, ks);
        if (f == 0 || f == n) {
            const double Ein = f == 0 ? x.L.Ein0[q] : x.L.EinX[q];
            const double Fin = f == 0 ? x.L.Fin0[q] : x.L.FinX[q];
            const double Cb = f == 0 ? x.L.C0[q] : x.L.CX[q];
            double Eb;
            if constexpr (is_pair<R>)
                Eb = pr_join(src_in<R>(Ein, ks) +
                                 (Fv - src_in<R>(Fin, ks)) * rcpR<R>((R)kC * (R)Cb), ks);
            else
                Eb = Ein + ((double)Fv - Fin) / (kC * Cb);
            (f == 0 ? x.L.Eb0 : x.L.EbX)[q] = Eb;
        }
    }
}

// staged = true: phase A already done (by the whole block) for n >= 2.
template <typename R>
__device__ void warp_lo_solve(const LoCtx &x, int q, R *sm, int mmax, bool staged = false,
                              int ks = 0)
{
    const int lane = threadIdx.x & 31;
    const int n = x.nx;
    double *E = x.L.E + (size_t)q * n;
    double *F = x.L.F + (size_t)q * (n + 1);

    if (n == 1) {
        if (lane == 0) {
            R PL0, PR0, GD0, PL1, PR1, GD1, Ap0, Dp0;
            face_coef<R>(x, q, 0, PL0, PR0, GD0, ks);
            face_coef<R>(x, q, 1, PL1, PR1, GD1, ks);
            cell_row<R>(x, q, 0, Ap0, Dp0, ks);
            R di = Ap0 + PL1 + PR0;
            R rh = Dp0 - GD1 + GD0;
            R e0 = rh / di;
            E[0] = sol_out<R>(e0, ks);
            R F0 = GD0 - PR0 * e0, F1 = GD1 + PL1 * e0;
            const double F0d = sol_out<R>(F0, ks), F1d = sol_out<R>(F1, ks);
            F[0] = F0d;
            F[1] = F1d;
            x.L.Eb0[q] = x.L.Ein0[q] + (F0d - x.L.Fin0[q]) / (kC * x.L.C0[q]);
            x.L.EbX[q] = x.L.EinX[q] + (F1d - x.L.FinX[q]) / (kC * x.L.CX[q]);
        }
        return;
    }

    // ---- phase A ----
    if (!staged) lo_stage<R>(x, q, sm, mmax, lane, 32, ks);
    __syncwarp();

    tri_solve<R>(sm, n, mmax);
    lo_outputs<R>(x, q, sm, mmax, ks);
#undef CH
}

__host__ __device__ inline int lo_mmax(int nx)
{
    const int P = nx / 2 < 32 ? nx / 2 : 32;
    return nx < 2 ? 1 : (nx + P - 1) / P + 1;
}

// FP32 group solve refined to FP64 accuracy (mixed-precision iterative refinement).  The
// rows are staged in FP64 (s64, by the whole CTA); warp `sw` converts them to FP32 (s32),
// eliminates in FP32 (x0), then kLoRefine times forms the residual r = b - A x of the FP64
// rows in FP64, eliminates A d = r in FP32 and adds d to x in FP64; E = x, and the fluxes
// follow with the FP64 face coefficients.  Each step multiplies the error by about
// cond(A) eps_32 (the plain FP32 solve's error: 3.6e-6 in T on fc_1024, ~5e-5 in E on a
// 1000-cell random level, where one step left 2.6e-9); the eliminations, the part that is
// serial in cells, run on the FP32 pipes.
// Shared memory: 6 S doubles + 6 S floats (S = 32 mmax).
constexpr int kLoRefine = 2;

__device__ void lo_solve_refined(const LoCtx &x, int q, int sw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = x.nx;
    const int mmax = lo_mmax(n);
    const int S = 32 * mmax;
    double *s64 = reinterpret_cast<double *>(smem_raw);
    float *s32 = reinterpret_cast<float *>(s64 + 6 * S);
    if (n < 2) {   // one cell: the FP64 form
        if (threadIdx.x < 32) warp_lo_solve<double>(x, q, s64, mmax, false);
        return;
    }
    lo_stage<double>(x, q, s64, mmax, threadIdx.x, blockDim.x);
    __syncthreads();
    if ((int)(threadIdx.x >> 5) != (sw & ((int)(blockDim.x >> 5) - 1))) return;
    const int lane = threadIdx.x & 31;
    const double *PL = s64, *PR = s64 + S, *GD = s64 + 2 * S, *Ap = s64 + 3 * S;
    double *X0 = s64 + 4 * S;   // x0 in FP64 (the unused Cp slot of s64)
    double *Dp = s64 + 5 * S;   // right-hand sides, then E
    float *pl = s32, *pr = s32 + S, *gd = s32 + 2 * S, *ap = s32 + 3 * S, *cp = s32 + 4 * S,
          *dp = s32 + 5 * S;
    for (int o = lane; o < S; o += 32) {
        pl[o] = (float)PL[o];
        pr[o] = (float)PR[o];
        gd[o] = (float)GD[o];
        ap[o] = (float)Ap[o];
        dp[o] = (float)Dp[o];
    }
    __syncwarp();
    tri_solve<float>(s32, n, mmax);   // x0 in dp
    const int P = min(32, n / 2);
    const bool act = lane < P;
    const int r0 = act ? (lane * n) / P : n;
    const int m = act ? ((lane + 1) * n) / P - r0 : 0;
#define CH(arr, k, l) arr[(k) * 32 + (l)]
    for (int k = 0; k < m; ++k) CH(X0, k, lane) = (double)CH(dp, k, lane);
    __syncwarp();
    for (int step = 0; step < kLoRefine; ++step) {
        // residual of row i = r0 + k (face i+1 is the next slot of the chunk, or the first
        // slot of the next chunk; the last chunk keeps face n in its slot m):
        //   r = (Dp_i - GD_{i+1} + GD_i) - (Ap_i + PL_{i+1} + PR_i) x_i
        //       + PL_i x_{i-1} + PR_{i+1} x_{i+1}
        for (int k = 0; k < m; ++k) {
            const int i = r0 + k;
            const bool wrap = (k + 1 == m) && lane != P - 1;
            const int kn = wrap ? 0 : k + 1, ln = wrap ? lane + 1 : lane;
            const double di = CH(Ap, k, lane) + CH(PL, kn, ln) + CH(PR, k, lane);
            const double rh = CH(Dp, k, lane) - CH(GD, kn, ln) + CH(GD, k, lane);
            double r = rh - di * CH(X0, k, lane);
            if (i > 0) {
                const int mp = (k > 0) ? 0 : r0 - ((lane - 1) * n) / P;   // rows of the chunk before
                r = fma(CH(PL, k, lane), (k > 0) ? CH(X0, k - 1, lane) : CH(X0, mp - 1, lane - 1), r);
            }
            if (i < n - 1) r = fma(CH(PR, kn, ln), CH(X0, kn, ln), r);
            CH(cp, k, lane) = (float)r;
        }
        __syncwarp();
        // the correction system: the same matrix (its FP32 diagonal parts again: the
        // elimination overwrote them), right-hand side r, no face sources
        for (int k = 0; k <= m; ++k) {
            if (k < m) {
                CH(ap, k, lane) = (float)CH(Ap, k, lane);
                CH(dp, k, lane) = CH(cp, k, lane);
            }
            if (k < m || lane == P - 1) CH(gd, k, lane) = 0.f;
        }
        __syncwarp();
        tri_solve<float>(s32, n, mmax);   // the correction in dp
        for (int k = 0; k < m; ++k) CH(X0, k, lane) += (double)CH(dp, k, lane);
        __syncwarp();
    }
    for (int k = 0; k < m; ++k) CH(Dp, k, lane) = CH(X0, k, lane);
    __syncwarp();
#undef CH
    lo_outputs<double>(x, q, s64, mmax);
}

// One system per CTA: all 4 warps stage the rows (phase A: the parallel part, global
// loads and the face coefficients), warp `sw` runs the elimination, and all 4 warps form
// and store the outputs.  The CTA's four warps sit on the SM's four sub-partitions, each
// with its own FP64 pipe; rotating the eliminating warp with the work item spreads the
// serial chains of the CTAs resident on an SM over all four (always warp 0 would queue
// them all on one).
template <typename R>
__device__ void lo_solve_body(const LoCtx &x, int q, int sw)
{
    if constexpr (std::is_same<R, float>::value) {   // FP32 group solves: refined to FP64 accuracy
        lo_solve_refined(x, q, sw);
        return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *sm = reinterpret_cast<R *>(smem_raw);
    const int mmax = lo_mmax(x.nx);
    const bool staged = x.nx >= 2;
    const bool solver = (int)(threadIdx.x >> 5) == (sw & ((int)(blockDim.x >> 5) - 1));
    if (staged) {
        int ks = 0;
        if constexpr (is_pair<R>) ks = lo_stage_pair(x, q, sm, mmax);
        else lo_stage<R>(x, q, sm, mmax, threadIdx.x, blockDim.x);
        __syncthreads();
        if (solver) tri_solve<R>(sm, x.nx, mmax);
        __syncthreads();
        lo_outputs_cta<R>(x, q, sm, mmax, ks);
        return;
    }
    int ks = 0;   // one cell: one lane (the pair form's source scale from every thread)
    if constexpr (is_pair<R>) {
        __shared__ int kw[32];
        int m = lo_src_exp(x, q, threadIdx.x, blockDim.x);
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) kw[threadIdx.x >> 5] = m;
        __syncthreads();
        m = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, kw[w]);
        ks = (m == 0) ? 0 : m - 1023;
    }
    if (solver) warp_lo_solve<R>(x, q, sm, mmax, false, ks);
}

// 7 CTAs per SM (at most 72 registers): one wave of 1064 holds every group of a 1024-group
// level
template <typename R>
__global__ void __launch_bounds__(128, 7) k_lo_solve(LoCtx x)
{
    griddep_wait();
    if (x.gate && *x.gate) return;   // the phase's inner loop has ended
    lo_solve_body<R>(x, blockIdx.x, blockIdx.x);
}

template <typename R>
__global__ void __launch_bounds__(128) k_lo_solve_b(const int *__restrict__ meta, int N,
                                                    const LoCtx *__restrict__ xs)
{
    for (int b = blockIdx.x;; b += gridDim.x) {
        int s, bx, by;
        if (!bdecode(meta, N, b, s, bx, by)) break;
        const LoCtx x = xs[s];
        lo_solve_body<R>(x, bx, b);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// The weighted means below divide (no reciprocal-multiply): the weights (sums of E or of
// boundary energies over a coarse group) reach the subnormal range in cold cells, where
// 1/w overflows while a/w stays finite.
//
// restriction (eqs. coeff-gamma, g-notation, eta-gamma / coeff-Gamma, g2G-notation,
// eta-Gamma, and the discrete compensation of eq. mloqd-d-gamma)
// ---------------------------------------------------------------------------------------
// Per-cell terms of the grey Newton step (Sec. 5, eqs. eb-Gamma and f-derivative-d): from the
// grey opacity sig*, Q* = 2 e* and the group energy sum Esum of cell i at T*, the
// absorption w c sig*, the source w Q* - (1 - w) c_v (T* - Told)/dt and 1/Lambda.  Called
// by the grey kernel on the grey level's arrays, or by the restriction's second stage on
// the same values it writes there (the same operations, the same bits).
__device__ inline void grey_newton_terms(const GreyArgs &a, int have_prev, int i, double sig,
                                         double Q, double Esum, double &sa, double &ss,
                                         double &sL)
{
    const double cvdt = a.cvdt;
    const double k54 = a.k54;
    const double Ts = a.Tstar[i];
    const double iTs = rcp64(Ts);
    double dQ = k54;   // first edge at 0: (1 + x) e^{-x} = 1
    if (a.nu_first != 0.0) {
        const double x1 = a.nu_first * iTs;
        dQ = k54 * (1.0 + x1) * texp(-x1, a.e2, a.ec);
    }
    if (!isinf(a.nu_last)) {
        const double xL = a.nu_last * iTs;
        dQ -= k54 * (1.0 + xL) * texp(-xL, a.e2, a.ec);
    }
    double D = 0.0;
    if (have_prev) {
        const double Tp = a.T_prev[i];
        // T* != T_prev on the encodings (positive finite values: integer instructions, not
        // an FP64 compare); across grids only where |dT| is far above rounding (relative
        // noise ~ eps T/|dT|)
        const bool moved = __double_as_longlong(Ts) != __double_as_longlong(Tp);
        const bool cut = __double_as_longlong(a.secant_cut) != 0ll;
        if (moved && (!cut || fabs(Ts - Tp) > a.secant_cut * Ts))
            D = (sig - a.sig_prev[i]) * rcp64(Ts - Tp);
    }
    const double base = cvdt + dQ;
    double L = base - kC * D * Esum;
    if (L < 0.5 * base) L = 0.5 * base;
    const double iL = rcp64(L);
    const double w = cvdt * iL;
    sa = w * kC * sig;
    ss = w * Q - (1.0 - w) * cvdt * (Ts - a.Told[i]);
    sL = iL;
}

constexpr int kRV1 = 18;   // pass-1 sums
constexpr int kRV2 = 6;    // pass-2 sums


__device__ inline double src_phi_b(const Level &S, int p, int side)
{
    return side == 0 ? S.phib0[p] : S.phibX[p];
}

// block (32, KS <= 16); grid (ceil((nx+1)/32), n_to)
__device__ void restrict_body(const RestrictCtx &x, int bx, int by)
{
    extern __shared__ __align__(16) double rsm[];
    const int tx = threadIdx.x, ty = threadIdx.y, KS = blockDim.y;
    const int nx = x.nx, nf = nx + 1;
    const int i = bx * 32 + tx;   // cell index and face index
    const int P = by;
    const int pb = P * x.r;
    const Level &S = x.S;
    double v[kRV1];
#pragma unroll
    for (int k = 0; k < kRV1; ++k) v[k] = 0.0;
    // ---- pass 1 ----
    for (int p = pb + ty; p < pb + x.r; p += KS) {
        if (i < nx) {
            size_t c = (size_t)p * nx + i;
            double E = S.E[c];
            double ph = S.phi[c], sg = S.sig[c];
            v[0] += ph * E; v[1] += ph; v[2] += sg * E; v[3] += sg;
            v[4] += S.emis[c]; v[5] += S.Eold[c]; v[6] += E;
        }
        if (i <= nx) {
            double Fp = S.F[(size_t)p * nf + i];
            double sR;
            if (S.fine) {
                const double *sc = S.sigR + (size_t)p * nx;
                sR = (i == 0) ? sc[0] : (i == nx) ? sc[nx - 1]
                     : (sc[i - 1] * x.h[i - 1] + sc[i] * x.h[i]) * x.ihf[i];
            } else {
                sR = S.sigR[(size_t)p * nf + i];
            }
            // |F| weight with a floor 1e-6 c E-bar: groups in local equilibrium carry
            // rounding-noise fluxes that must not decide the mean
            double ER = (i == nx) ? S.EbX[p] : S.E[(size_t)p * nx + i];
            double EL = (i == 0) ? S.Eb0[p] : S.E[(size_t)p * nx + i - 1];
            double wF = fabs(Fp) + 1e-6 * kC * 0.5 * (EL + ER);
            v[7] += sR * wF; v[8] += sR; v[9] += wF;
        }
        if (i == 0 || i == nx) {
            const int side = (i == 0) ? 0 : 1;
            double Eb = side == 0 ? S.Eb0[p] : S.EbX[p];
            double Ein = side == 0 ? S.Ein0[p] : S.EinX[p];
            double Fin = side == 0 ? S.Fin0[p] : S.FinX[p];
            double Cb = side == 0 ? S.C0[p] : S.CX[p];
            double ph = src_phi_b(S, p, side);
            double Eo = Eb - Ein;
            v[10] += ph * Eb; v[11] += ph; v[12] += Eb;
            v[13] += Cb * Eo; v[14] += Cb; v[15] += Eo;
            v[16] += Ein; v[17] += Fin;
        }
    }
    // reduce over ty
    if (KS > 1) {
        double *red = rsm + ((size_t)ty * 32 + tx) * kRV1;
        for (int k = 0; k < kRV1; ++k) red[k] = v[k];
        __syncthreads();
        if (ty == 0) {
            for (int y = 1; y < KS; ++y) {
                const double *o = rsm + ((size_t)y * 32 + tx) * kRV1;
                for (int k = 0; k < kRV1; ++k) v[k] += o[k];
            }
            double *bc = rsm + (size_t)tx * kRV1;
            for (int k = 0; k < kRV1; ++k) bc[k] = v[k];
        }
        __syncthreads();
        if (ty != 0) {
            const double *bc = rsm + (size_t)tx * kRV1;
            for (int k = 0; k < kRV1; ++k) v[k] = bc[k];
        }
        __syncthreads();
    }
    const double rn = (double)x.r;
    const double sRP = (v[9] != 0.0) ? v[7] / v[9] : v[8] / rn;
    // ---- pass 2 (faces): xi, eta sums, side energies, Fold ----
    double u[kRV2];
#pragma unroll
    for (int k = 0; k < kRV2; ++k) u[k] = 0.0;
    if (i <= nx) {
        const double dxf = (i == 0) ? 0.5 * x.h[0] : (i == nx) ? 0.5 * x.h[nx - 1]
                                               : 0.5 * (x.h[i - 1] + x.h[i]);
        for (int p = pb + ty; p < pb + x.r; p += KS) {
            size_t fp = (size_t)p * nf + i;
            double Fp = S.F[fp];
            double sR;
            if (S.fine) {
                const double *sc = S.sigR + (size_t)p * nx;
                sR = (i == 0) ? sc[0] : (i == nx) ? sc[nx - 1]
                     : (sc[i - 1] * x.h[i - 1] + sc[i] * x.h[i]) * x.ihf[i];
            } else {
                sR = S.sigR[fp];
            }
            double ER = (i == nx) ? S.EbX[p] : S.E[(size_t)p * nx + i];
            double EL = (i == 0) ? S.Eb0[p] : S.E[(size_t)p * nx + i - 1];
            u[0] += dxf * (sR - sRP) * Fp;
            if (!S.fine) {
                u[1] += S.etaR[fp] * ER;
                u[2] += S.etaL[fp] * EL;
            }
            u[3] += ER; u[4] += EL; u[5] += S.Fold[fp];
        }
    }
    if (KS > 1) {
        double *red = rsm + ((size_t)ty * 32 + tx) * kRV2;
        for (int k = 0; k < kRV2; ++k) red[k] = u[k];
        __syncthreads();
        if (ty == 0) {
            for (int y = 1; y < KS; ++y) {
                const double *o = rsm + ((size_t)y * 32 + tx) * kRV2;
                for (int k = 0; k < kRV2; ++k) u[k] += o[k];
            }
        }
    }
    if (ty != 0) return;
    const Level &T = x.T;
    if (i < nx) {
        size_t c = (size_t)P * nx + i;
        (T.phi)[c] = (v[6] != 0.0) ? v[0] / v[6] : v[1] / rn;
        (T.sig)[c] = (v[6] != 0.0) ? v[2] / v[6] : v[3] / rn;
        (T.emis)[c] = v[4];
        (T.Eold)[c] = v[5];
        T.Esum[c] = v[6];
    }
    if (i <= nx) {
        size_t f = (size_t)P * nf + i;
        double xi = u[0] + kC * (u[1] - u[2]);
        (T.sigR)[f] = sRP;
        (T.etaR)[f] = (xi > 0.0 && u[3] != 0.0) ? xi / (kC * u[3]) : 0.0;
        (T.etaL)[f] = (xi < 0.0 && u[4] != 0.0) ? -xi / (kC * u[4]) : 0.0;
        (T.Fold)[f] = u[5];
    }
    if (i == 0 || i == nx) {
        double phb = (v[12] != 0.0) ? v[10] / v[12] : v[11] / rn;
        double Cb = (v[15] != 0.0) ? v[13] / v[15] : v[14] / rn;
        if (i == 0) {
            (T.phib0)[P] = phb;
            (T.C0)[P] = Cb;
            (T.Ein0)[P] = v[16];
            (T.Fin0)[P] = v[17];
        } else {
            (T.phibX)[P] = phb;
            (T.CX)[P] = Cb;
            (T.EinX)[P] = v[16];
            (T.FinX)[P] = v[17];
        }
    }
}

// Two-stage restriction for wide coarse groups (r >= 64 members): stage 1 sums chunks of
// kChunk members per (coarse group, cell / face) into partial vectors with many CTAs;
// stage 2 adds the chunks in a fixed order and forms the coefficients.  Sums stage 1 does
// not form: the member energies on either side of an interior face (sum E_R at face i is
// sum E at cell i, sum E_L is sum E at cell i - 1: the same terms in the same order, so
// the same bits), and the plain means that replace a weighted mean whose weights sum to
// zero (formed by stage 2 from the members in that rare case).  Every stage-1 addition is
// an FP64 operation, the pipe that bounds these kernels on GB300.  The compensation
// is summed in one pass, xi = dx (sum sigR F - sigR-bar sum F) + c (sum etaR E_R -
// sum etaL E_L), which is the two-pass sum up to rounding relative to the sigR dx F terms.
constexpr int kChunk = 64;
constexpr int kRP = 25;
constexpr int kPartRows = 8;   // rows (warps) of a stage-1 block: kChunk / kPartRows members each
constexpr size_t kPartSmem = sizeof(double) * kPartRows * 32 * (kRP + 1);


// block (32, kPartRows); grid (ceil((nx+1)/32), n_to * nchunk); kPartSmem bytes of dynamic
// shared memory
__device__ void restrict_part_body(const Restrict2Ctx &x, int bx, int by)
{
    extern __shared__ __align__(16) double red_raw[];
    double (*red)[32][kRP + 1] = reinterpret_cast<double (*)[32][kRP + 1]>(red_raw);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nx = x.nx, nf = nx + 1;
    const int i = bx * 32 + tx;
    const int P = by / x.nchunk, ch = by - P * x.nchunk;
    const int pb = P * x.r + ch * kChunk;
    const int pe = min(pb + kChunk, P * x.r + x.r);
    const Level &S = x.S;
    double v[kRP];
#pragma unroll
    for (int k = 0; k < kRP; ++k) v[k] = 0.0;
    for (int p = pb + ty; p < pe; p += kPartRows) {
        if (i < nx) {
            const size_t c = (size_t)p * nx + i;
            const double E = S.E[c];
            v[0] += S.phi[c] * E; v[2] += S.sig[c] * E;
            v[4] += S.emis[c];
            if (!x.skip_old) v[5] += S.Eold[c];
            v[6] += E;
        }
        if (i <= nx) {
            const size_t fp = (size_t)p * nf + i;
            const double Fp = S.F[fp];
            double sR;
            if (S.fine) {
                const double *sc = S.sigR + (size_t)p * nx;
                sR = (i == 0) ? sc[0] : (i == nx) ? sc[nx - 1]
                     : (sc[i - 1] * x.h[i - 1] + sc[i] * x.h[i]) * x.ihf[i];
            } else {
                sR = S.sigR[fp];
            }
            const double ER = (i == nx) ? S.EbX[p] : S.E[(size_t)p * nx + i];
            const double EL = (i == 0) ? S.Eb0[p] : S.E[(size_t)p * nx + i - 1];
            const double wF = fabs(Fp) + 1e-6 * kC * 0.5 * (EL + ER);
            v[7] += sR * wF; v[9] += wF; v[10] += sR * Fp; v[11] += Fp;
            if (!S.fine) {
                v[12] += S.etaR[fp] * ER;
                v[13] += S.etaL[fp] * EL;
            }
            if (i == nx) v[14] += ER;
            if (i == 0) v[15] += EL;
            if (!x.skip_old) v[16] += S.Fold[fp];
        }
        if (i == 0 || i == nx) {
            const int side = (i == 0) ? 0 : 1;
            const double Eb = side == 0 ? S.Eb0[p] : S.EbX[p];
            const double Ein = side == 0 ? S.Ein0[p] : S.EinX[p];
            const double Fin = side == 0 ? S.Fin0[p] : S.FinX[p];
            const double Cb = side == 0 ? S.C0[p] : S.CX[p];
            const double ph = side == 0 ? S.phib0[p] : S.phibX[p];
            const double Eo = Eb - Ein;
            v[17] += ph * Eb; v[18] += ph; v[19] += Eb;
            v[20] += Cb * Eo; v[21] += Cb; v[22] += Eo;
            v[23] += Ein; v[24] += Fin;
        }
    }
#pragma unroll
    for (int k = 0; k < kRP; ++k) red[ty][tx][k] = v[k];
    __syncthreads();
    // the rows' partials, value k by row k % kPartRows: the additions are spread over the
    // warps (all four sub-partitions' FP64 pipes); same order as a sum by one row
    if (i <= nx) {
        double *o = x.part + ((size_t)(P * x.nchunk + ch) * kRP) * nf + i;
        for (int k = ty; k < kRP; k += kPartRows) {
            double a = red[0][tx][k];
#pragma unroll
            for (int y = 1; y < kPartRows; ++y) a += red[y][tx][k];
            o[(size_t)k * nf] = a;
        }
    }
}

// block (32, kRP); grid (ceil((nx+1)/32), n_to): thread (tx, k) adds value k of position
// tx over the chunks in a fixed order; then rows 0 .. 3 (one warp each, on four
// sub-partitions) form the coefficients: row 0 the E-weighted cell means, row 1 the copied
// cell sums, row 2 the face opacity and compensation, row 3 the boundary means.
__device__ void restrict_final_body(const Restrict2Ctx &x, int bx, int by)
{
    __shared__ double sv[kRP][33];
    const int nx = x.nx, nf = nx + 1;
    const int tx = threadIdx.x, k = threadIdx.y;
    const int i = bx * 32 + tx;
    const int P = by;
    if (i <= nx) {
        double acc = 0.0;
        // sum E_L at the block's first face (i > 0) is sum E at cell i - 1 of the block before
        const int kk = (k == 15 && tx == 0 && i > 0) ? 6 : k;
        const int ii = (kk != k) ? i - 1 : i;
        const double *o = x.part + ((size_t)P * x.nchunk * kRP + kk) * nf + ii;
        for (int ch = 0; ch < x.nchunk; ++ch) acc += o[(size_t)ch * kRP * nf];
        sv[k][tx] = acc;
    }
    __syncthreads();
    if (k > 3 || i > nx) return;
    const double rn = (double)x.r;
    const Level &T = x.T;
    const Level &S = x.S;
    const int p0 = P * x.r;
    if (k == 0 && i < nx) {
        const size_t c = (size_t)P * nx + i;
        const double E = sv[6][tx];
        double ph = 0.0, sg = 0.0;
        if (E != 0.0) {
            ph = sv[0][tx] / E;
            sg = sv[2][tx] / E;
        } else {   // no energy in the coarse group: plain means of the members
            for (int p = p0; p < p0 + x.r; ++p) {
                ph += S.phi[(size_t)p * nx + i];
                sg += S.sig[(size_t)p * nx + i];
            }
            ph /= rn;
            sg /= rn;
        }
        T.phi[c] = ph;
        T.sig[c] = sg;
        if (x.newton) {   // target = the grey level: the visit's Newton terms of cell i
            double sa, ss, sL;
            grey_newton_terms(x.ga, x.ga.have_prev, i, sg, 2.0 * sv[4][tx], sv[6][tx], sa, ss,
                              sL);
            x.pre[i] = sa;
            x.pre[nx + i] = ss;
            x.pre[2 * (size_t)nx + i] = sL;
        }
    } else if (k == 1) {
        if (i < nx) {
            const size_t c = (size_t)P * nx + i;
            T.emis[c] = sv[4][tx];
            if (!x.skip_old) T.Eold[c] = sv[5][tx];
            T.Esum[c] = sv[6][tx];
        }
        if (!x.skip_old) T.Fold[(size_t)P * nf + i] = sv[16][tx];
    } else if (k == 2) {
        const double v14 = (i < nx) ? sv[6][tx] : sv[14][tx];
        const double v15 = (i > 0 && tx > 0) ? sv[6][tx - 1] : sv[15][tx];
        const double dxf = (i == 0) ? 0.5 * x.h[0] : (i == nx) ? 0.5 * x.h[nx - 1]
                                                : 0.5 * (x.h[i - 1] + x.h[i]);
        double sRP = 0.0;
        if (sv[9][tx] != 0.0) {
            sRP = sv[7][tx] / sv[9][tx];
        } else {   // no flux weight: plain mean of the members' face opacities
            for (int p = p0; p < p0 + x.r; ++p) {
                if (S.fine) {
                    const double *sc = S.sigR + (size_t)p * nx;
                    sRP += (i == 0) ? sc[0] : (i == nx) ? sc[nx - 1]
                           : (sc[i - 1] * x.h[i - 1] + sc[i] * x.h[i]) * x.ihf[i];
                } else {
                    sRP += S.sigR[(size_t)p * nf + i];
                }
            }
            sRP /= rn;
        }
        const double xi = dxf * (sv[10][tx] - sRP * sv[11][tx]) + kC * (sv[12][tx] - sv[13][tx]);
        const size_t f = (size_t)P * nf + i;
        T.sigR[f] = sRP;
        T.etaR[f] = (xi > 0.0 && v14 != 0.0) ? xi / (kC * v14) : 0.0;
        T.etaL[f] = (xi < 0.0 && v15 != 0.0) ? -xi / (kC * v15) : 0.0;
    } else if (k == 3 && (i == 0 || i == nx)) {
        const double phb = (sv[19][tx] != 0.0) ? sv[17][tx] / sv[19][tx] : sv[18][tx] / rn;
        const double Cb = (sv[22][tx] != 0.0) ? sv[20][tx] / sv[22][tx] : sv[21][tx] / rn;
        if (i == 0) {
            T.phib0[P] = phb; T.C0[P] = Cb; T.Ein0[P] = sv[23][tx]; T.Fin0[P] = sv[24][tx];
        } else {
            T.phibX[P] = phb; T.CX[P] = Cb; T.EinX[P] = sv[23][tx]; T.FinX[P] = sv[24][tx];
        }
    }
}

// ---------------------------------------------------------------------------------------
// grey LOQD + MEB: one Newton step on the grey level (single CTA)
// ---------------------------------------------------------------------------------------

// Block-wide maxima of non-negative values on their IEEE encodings: for x >= 0 (and +inf)
// the order of the doubles is the unsigned order of their bit patterns, so the reduction
// runs on the integer pipes (a warp-wide FP64 max takes a sub-partition's FP64 pipe for 64
// cycles on GB300).  NaN maps to 0, the value fmax would keep.  red: kGreyRed slots, at
// least 32 per value; the maxima are returned to thread 0 (each warp reduces its lanes by
// shuffles, then warp 0 reduces the warps' results the same way).
constexpr int kGreyNV = 7;
constexpr int kGreyRed = 32 * kGreyNV;

__device__ inline unsigned long long nn_bits(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return ((b & 0x7fffffffffffffffull) > 0x7ff0000000000000ull) ? 0ull : b;
}

__device__ inline unsigned long long umax64(unsigned long long a, unsigned long long b)
{
    return a > b ? a : b;
}

__device__ inline void block_max_bits(unsigned long long (&v)[kGreyNV], unsigned long long *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < kGreyNV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] = umax64(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < kGreyNV; ++k) red[k * 32 + warp] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < kGreyNV; ++k) {
            unsigned long long r = (lane < nw) ? red[k * 32 + lane] : 0ull;
            for (int o = 16; o > 0; o >>= 1) r = umax64(r, __shfl_xor_sync(0xffffffffu, r, o));
            v[k] = r;
        }
    }
}

__device__ inline void grey_newton_cell(const GreyArgs &a, const Level &g, int have_prev, int i,
                                        double &sa, double &ss, double &sL)
{
    grey_newton_terms(a, have_prev, i, g.sig[i], 2.0 * g.emis[i], g.Esum[i], sa, ss, sL);
}

// The grey level's tridiagonal system (n >= 2) by P = min(128, n/2, block) threads: GB300
// runs a warp's FP64 instructions on its own sub-partition's FP64 pipe only, so the group
// systems' one-warp partitioned elimination (32 chunks of ~16 rows: a serial chain of ~500
// FP64 instructions at 64 cycles each) would keep the SM's other three pipes idle for
// ~20 us on the grey level, where a single system is solved at a time.  Here every
// thread eliminates a chunk of ~4 rows (the modified Thomas pass down and up the chunk of
// tri_solve: rows coupled only to the chunk's first and last unknowns), the 2P chunk-
// boundary rows are solved by parallel cyclic reduction in shared memory (rows kept with
// unit diagonals, ceil(log2 2P) levels of one block barrier each), and every thread
// back-substitutes its chunk's interior.  sm: PL, PR, GD [n + 1], Ap, Cp, Dp [n], then the
// reduced rows' A, C, D in two buffers [2][3][2P].  All threads of the block call it; the
// solution is left in Dp.
__host__ __device__ inline int grey_chunks(int n, int block)
{
    int P = n / 2;
    if (P > 128) P = 128;
    if (P > block) P = block;
    return P < 1 ? 1 : P;
}

__device__ void grey_tri_solve(const LoCtx &x, double *sm, int n)
{
    const int P = grey_chunks(n, (int)blockDim.x), nr = 2 * P;
    double *PL = sm, *PR = PL + (n + 1), *GD = PR + (n + 1);
    double *Ap = GD + (n + 1), *Cp = Ap + n, *Dp = Cp + n;
    double *rb = Dp + n;   // [2][3][nr]
    const int t = threadIdx.x;
    for (int f = t; f <= n; f += blockDim.x) {
        double pl, pr, gd;
        face_coef<double>(x, 0, f, pl, pr, gd);
        PL[f] = pl;
        PR[f] = pr;
        GD[f] = gd;
        if (f < n) cell_row<double>(x, 0, f, Ap[f], Dp[f]);
    }
    __syncthreads();
    const int r0 = (t < P) ? (int)(((long long)t * n) / P) : n;
    const int r1 = (t < P) ? (int)(((long long)(t + 1) * n) / P) : n;
    const int m = r1 - r0;
    if (t < P) {
        // down the chunk: row k >= 1 coupled to x_{r0} (a) and x_{r0+k+1} (c); row 0 to
        // x_{r0-1} and x_{r0+1}
        double PLi = PL[r0], PRi = PR[r0], GDi = GD[r0];
        double ap = 0.0, cp = 0.0, dp = 0.0;
        for (int k = 0; k < m; ++k) {
            const int i = r0 + k;
            const double PL1 = PL[i + 1], PR1 = PR[i + 1], GD1 = GD[i + 1];
            const double di = Ap[i] + PL1 + PRi;
            const double rh = Dp[i] - GD1 + GDi;
            const double lo = (i > 0) ? -PLi : 0.0;
            const double up = (i < n - 1) ? -PR1 : 0.0;
            if (k < 2) {
                const double r = rcp64(di);
                ap = lo * r;
                cp = up * r;
                dp = rh * r;
            } else {
                const double r = rcp64(di - lo * cp);
                dp = r * (rh - lo * dp);
                ap = -r * lo * ap;
                cp = r * up;
            }
            Ap[i] = ap;
            Cp[i] = cp;
            Dp[i] = dp;
            PLi = PL1;
            PRi = PR1;
            GDi = GD1;
        }
        // up the chunk: rows 1 .. m-2 coupled to x_{r0} and x_{r1-1}; row 0 to x_{r0-1}
        // and x_{r1-1}
        if (m >= 3) {
            for (int k = m - 3; k >= 1; --k) {
                const int i = r0 + k;
                const double ck = Cp[i];
                Dp[i] = Dp[i] - ck * Dp[i + 1];
                Ap[i] = Ap[i] - ck * Ap[i + 1];
                Cp[i] = -ck * Cp[i + 1];
            }
            const double c0 = Cp[r0];
            const double r = rcp64(1.0 - c0 * Ap[r0 + 1]);
            Dp[r0] = r * (Dp[r0] - c0 * Dp[r0 + 1]);
            Ap[r0] = r * Ap[r0];
            Cp[r0] = -r * c0 * Cp[r0 + 1];
        }
        // reduced rows 2t (the chunk's first row) and 2t + 1 (its last)
        rb[2 * t] = Ap[r0];
        rb[nr + 2 * t] = Cp[r0];
        rb[2 * nr + 2 * t] = Dp[r0];
        rb[2 * t + 1] = Ap[r1 - 1];
        rb[nr + 2 * t + 1] = Cp[r1 - 1];
        rb[2 * nr + 2 * t + 1] = Dp[r1 - 1];
    }
    __syncthreads();
    // parallel cyclic reduction of the 2P reduced rows: a level eliminates the neighbours at
    // distance s with the factors -A and -C and divides by the new diagonal
    int cur = 0;
    for (int s = 1; s < nr; s <<= 1) {
        const double *A = rb + (size_t)cur * 3 * nr, *C = A + nr, *D = C + nr;
        double *nA = rb + (size_t)(cur ^ 1) * 3 * nr, *nC = nA + nr, *nD = nC + nr;
        if (t < P) {
#pragma unroll
            for (int j = 2 * t; j <= 2 * t + 1; ++j) {
                const bool hl = j >= s, hu = j + s < nr;
                const double lA = hl ? A[j - s] : 0.0, lC = hl ? C[j - s] : 0.0;
                const double lD = hl ? D[j - s] : 0.0;
                const double uA = hu ? A[j + s] : 0.0, uC = hu ? C[j + s] : 0.0;
                const double uD = hu ? D[j + s] : 0.0;
                const double al = -A[j], ga = -C[j];
                const double r = rcp64(1.0 + al * lC + ga * uA);
                nA[j] = al * lA * r;
                nC[j] = ga * uC * r;
                nD[j] = (D[j] + al * lD + ga * uD) * r;
            }
        }
        cur ^= 1;
        __syncthreads();
    }
    // back substitution of the chunk's interior rows
    if (t < P) {
        const double *D = rb + (size_t)cur * 3 * nr + 2 * nr;
        const double x0 = D[2 * t], x1 = D[2 * t + 1];
        for (int k = 1; k < m - 1; ++k) {
            const int i = r0 + k;
            Dp[i] = Dp[i] - Ap[i] * x0 - Cp[i] * x1;
        }
        Dp[r0] = x0;
        Dp[r1 - 1] = x1;
    }
    __syncthreads();
}

// the grey level's outputs from the solution in Dp (grey_tri_solve's layout): E, the face
// fluxes F_f = GD_f + PL_f E_{f-1} - PR_f E_f and the boundary face energies
__device__ void grey_outputs(const LoCtx &x, const double *sm, int n)
{
    const double *PL = sm, *PR = PL + (n + 1), *GD = PR + (n + 1);
    const double *Dp = GD + (n + 1) + 2 * n;
    for (int f = threadIdx.x; f <= n; f += blockDim.x) {
        if (f < n) x.L.E[f] = Dp[f];
        double Fv = GD[f];
        if (f > 0) Fv += PL[f] * Dp[f - 1];
        if (f < n) Fv -= PR[f] * Dp[f];
        x.L.F[f] = Fv;
        if (f == 0) x.L.Eb0[0] = x.L.Ein0[0] + (Fv - x.L.Fin0[0]) * rcp64(kC * x.L.C0[0]);
        if (f == n) x.L.EbX[0] = x.L.EinX[0] + (Fv - x.L.FinX[0]) * rcp64(kC * x.L.CX[0]);
    }
}

// T at cell i from the grey solution E; the bad-value test and the norms' terms
__device__ inline void grey_update_cell(const GreyArgs &a, const Level &g, int i, double sL,
                                        double E, unsigned long long (&v)[kGreyNV])
{
    const unsigned long long kInfBits = 0x7ff0000000000000ull;
    const double cvdt = a.cvdt;
    const double Ts = a.Tstar[i];
    const double T = Ts + (kC * g.sig[i] * E - 2.0 * g.emis[i] - cvdt * (Ts - a.Told[i])) * sL;
    a.T[i] = T;
    const long long tb = __double_as_longlong(T);
    const unsigned long long eb = (unsigned long long)__double_as_longlong(E) & 0x7fffffffffffffffull;
    // T > 0 and finite: sign clear, not zero, below the infinity encoding
    if (tb <= 0 || (unsigned long long)tb >= kInfBits || eb >= kInfBits) v[0] = 1ull;
    if (a.want_norms) {
        v[1] = umax64(v[1], nn_bits(fabs(T - a.Tcyc[i])));
        v[2] = umax64(v[2], nn_bits(fabs(T)));
        v[3] = umax64(v[3], nn_bits(fabs(E - a.Ecyc[i])));
        v[4] = umax64(v[4], nn_bits(fabs(E)));
        v[5] = umax64(v[5], nn_bits(fabs(T - a.Tphase[i])));
        v[6] = umax64(v[6], nn_bits(fabs(E - a.Ephase[i])));
        if (a.T_out) a.T_out[i] = T;
        if (a.Tcyc_out) a.Tcyc_out[i] = T;
        if (a.Ecyc_out) a.Ecyc_out[i] = E;
    }
}

__device__ void grey_body(const GreyCtx &x)
{
    const int have_prev = x.a.have_prev_dev ? *x.a.have_prev_dev : x.a.have_prev;
    extern __shared__ __align__(16) double gsm[];
    const int nx = x.lo.nx;
    double *sa = gsm;            // absorption w c sig*
    double *ss = sa + nx;        // source w Q* - (1-w) cv (T* - Told)/dt
    double *sL = ss + nx;        // 1 / Lambda
    double *red = sL + nx;       // [kGreyRed] block maxima
    double *wsm = red + kGreyRed;   // solver scratch (grey_tri_solve)
    const GreyArgs &a = x.a;
    const Level &g = x.lo.L;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        if (a.pre) {   // formed by the restriction before this kernel
            sa[i] = a.pre[i];
            ss[i] = a.pre[nx + i];
            sL[i] = a.pre[2 * (size_t)nx + i];
        } else {
            grey_newton_cell(a, g, have_prev, i, sa[i], ss[i], sL[i]);
        }
        a.sig_prev_out[i] = g.sig[i];
        a.T_prev_out[i] = a.Tstar[i];
    }
    __syncthreads();
    LoCtx lc = x.lo;
    lc.a_cell = sa;
    lc.s_cell = ss;
    const double *Esol = wsm + 3 * (size_t)(nx + 1) + 2 * (size_t)nx;   // grey_tri_solve's Dp
    if (nx >= 2) {
        grey_tri_solve(lc, wsm, nx);
        grey_outputs(lc, wsm, nx);
    } else {
        if (threadIdx.x < 32) warp_lo_solve<double>(lc, 0, wsm, x.mmax, false);
        __syncthreads();
        Esol = g.E;
    }
    // v: bad flag, max|T - Tcyc|, max|T|, max|E - Ecyc|, max|E|, max|T - Tphase|,
    // max|E - Ephase| as non-negative encodings (flags[0 .. 6])
    unsigned long long v[kGreyNV] = {};
    for (int i = threadIdx.x; i < nx; i += blockDim.x) grey_update_cell(a, g, i, sL[i], Esol[i], v);
    block_max_bits(v, reinterpret_cast<unsigned long long *>(red));
    if (threadIdx.x == 0) {
        if (v[0] != 0ull) a.flags[0] = 1.0;
        if (a.want_norms) {
            a.flags[1] = __longlong_as_double((long long)v[1]);
            a.flags[2] = __longlong_as_double((long long)v[2]);
            a.flags[3] = __longlong_as_double((long long)v[3]);
            a.flags[4] = __longlong_as_double((long long)v[4]);
            a.flags[5] = __longlong_as_double((long long)v[5]);
            a.flags[6] = __longlong_as_double((long long)v[6]);
            if (a.ctl) {   // inner-loop control: this cycle ran; does the phase go on?
                const double f1 = __longlong_as_double((long long)v[1]);
                const double f2 = __longlong_as_double((long long)v[2]);
                const double f3 = __longlong_as_double((long long)v[3]);
                const double f4 = __longlong_as_double((long long)v[4]);
                const bool conv_in = f1 <= a.eps_in * f2 && f3 <= a.eps_in * f4;
                a.ctl[1] += 1;
                // a bad temperature of this visit or of an earlier visit of the cycle
                if (v[0] != 0ull || a.flags[0] != 0.0 || (!a.fixed && conv_in)) a.ctl[0] = 1;
            }
        }
    }
    if (a.have_prev_dev && threadIdx.x == 0) *a.have_prev_dev = 1;   // after the reduction's barriers
}

// out_i = sum_q X[q][i]: block of 256 threads = 32 cells x 8 rows; row y sums the groups
// q = y (mod 8) of its cell, then one row adds the 8 partials in row order (fixed order,
// deterministic).  A single pass over the groups per cell would leave 32 cells per warp
// and few warps per SM on a serial FP64 chain.
__device__ void group_sum_body(const GroupSumArgs &a, int bx)
{
    __shared__ double part[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int i = bx * 32 + tx;
    double s = 0.0;
    if (i < a.nx)
        for (int q = ty; q < a.n; q += 8) s += a.X[(size_t)q * a.nx + i];
    part[ty][tx] = s;
    __syncthreads();
    if (ty == (bx & 7) && i < a.nx) {
        double t = part[0][tx];
        for (int y = 1; y < 8; ++y) t += part[y][tx];
        a.out[i] = t;
    }
}

// entry points: the single-slab kernels pass blockIdx; the batched ones walk a work list
// (single-slab entry points: return at entry while the driver's gate is set)
__global__ void __launch_bounds__(512) k_restrict(RestrictCtx x)
{
    griddep_wait();
    if (x.gate && *x.gate) return;
    restrict_body(x, blockIdx.x, blockIdx.y);
}
__global__ void __launch_bounds__(32 * kPartRows) k_restrict_part(Restrict2Ctx x)
{
    griddep_wait();
    if (x.gate && *x.gate) return;
    restrict_part_body(x, blockIdx.x, blockIdx.y);
}
__global__ void __launch_bounds__(32 * kRP, 1) k_restrict_final(Restrict2Ctx x)
{
    griddep_wait();
    if (x.gate && *x.gate) return;
    restrict_final_body(x, blockIdx.x, blockIdx.y);
}
__global__ void __launch_bounds__(1024) k_grey(GreyCtx x)
{
    griddep_wait();
    if (x.lo.gate && *x.lo.gate) return;
    grey_body(x);
}
__global__ void __launch_bounds__(256) k_group_sum(GroupSumArgs a) { group_sum_body(a, blockIdx.x); }

#define TRT_BATCHED(name, Ctx, bounds, call)                                                  \
    __global__ void __launch_bounds__(bounds) name(const int *__restrict__ meta, int N,        \
                                                   const Ctx *__restrict__ xs)                 \
    {                                                                                          \
        for (int b = blockIdx.x;; b += gridDim.x) {                                            \
            int s, bx, by;                                                                     \
            if (!bdecode(meta, N, b, s, bx, by)) break;                                        \
            const Ctx x = xs[s];                                                               \
            call;                                                                              \
            __syncthreads();                                                                   \
        }                                                                                      \
    }
TRT_BATCHED(k_restrict_b, RestrictCtx, 512, restrict_body(x, bx, by))
TRT_BATCHED(k_restrict_part_b, Restrict2Ctx, 32 * kPartRows, restrict_part_body(x, bx, by))
TRT_BATCHED(k_restrict_final_b, Restrict2Ctx, 32 * kRP, restrict_final_body(x, bx, by))
TRT_BATCHED(k_grey_b, GreyCtx, 1024, grey_body(x))
TRT_BATCHED(k_group_sum_b, GroupSumArgs, 256, group_sum_body(x, bx))
#undef TRT_BATCHED

__global__ void __launch_bounds__(256) k_copy_b(const int *__restrict__ meta, int N,
                                                const CopyArgs *__restrict__ xs)
{
    for (int b = blockIdx.x;; b += gridDim.x) {
        int s, bx, by;
        if (!bdecode(meta, N, b, s, bx, by)) break;
        const CopyArgs c = xs[s];
        const long i = (long)bx * blockDim.x + threadIdx.x;
        if (i < c.n) c.dst[i] = c.src[i];
    }
}

}  // namespace

namespace {
// h/dt per cell and hf/(c dt) per face (for step length dt); with pc (the pair form) the
// same two rows of Problem::lopc
__global__ void k_lo_consts(int nx, const double *__restrict__ h, const double *__restrict__ hf,
                            double idt, double icdt, double *hidt, double *dxicdt, fpair *pc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t n1 = (size_t)nx + 1;
    if (i < nx) {
        const double v = h[i] * idt;
        hidt[i] = v;
        if (pc) pc[4 * n1 + i] = fpair(v);
    }
    if (i <= nx) {
        const double v = hf[i] * icdt;
        dxicdt[i] = v;
        if (pc) pc[n1 + i] = fpair(v);
    }
}

// the step-independent rows of Problem::lopc ([8][nx+1] pairs): hf, fwl, fwr (faces), hc,
// h2, h (cells); once per handle
__global__ void k_lo_pair_consts(int nx, const double *__restrict__ h, const double *__restrict__ hf,
                                 const double *__restrict__ hc, const double *__restrict__ h2,
                                 const double *__restrict__ fwl, const double *__restrict__ fwr,
                                 fpair *pc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t n1 = (size_t)nx + 1;
    if (i < nx) {
        pc[5 * n1 + i] = fpair(hc[i]);
        pc[6 * n1 + i] = fpair(h2[i]);
        pc[7 * n1 + i] = fpair(h[i]);
    }
    if (i <= nx) {
        pc[i] = fpair(hf[i]);
        pc[2 * n1 + i] = fpair(fwl[i]);
        pc[3 * n1 + i] = fpair(fwr[i]);
    }
}

}  // namespace

cudaError_t launch_lo_pair_consts(const Problem &p)
{
    if (!p.lopc) return cudaSuccess;
    k_lo_pair_consts<<<(p.nx + 1 + 255) / 256, 256, 0, p.stream>>>(
        p.nx, p.h, p.hf, p.hc, p.h2, p.fwl, p.fwr, reinterpret_cast<fpair *>(p.lopc));
    return cudaGetLastError();
}

cudaError_t ensure_lo_consts(Problem &p, double dt)
{
    if (p.lo_dt == dt) return cudaSuccess;
    k_lo_consts<<<(p.nx + 1 + 255) / 256, 256, 0, p.stream>>>(
        p.nx, p.h, p.hf, 1.0 / dt, 1.0 / (kC * dt), p.hidt, p.dxicdt,
        reinterpret_cast<fpair *>(p.lopc));
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) p.lo_dt = dt;
    return e;
}

// (the LO row constants hidt, dxicdt must be those of dt: ensure_lo_consts first)
LoCtx make_lo_ctx(const Problem &p, double dt, const Level &L)
{
    LoCtx x;
    x.nx = p.nx; x.dt = dt; x.icdt = 1.0 / (kC * dt); x.idt = 1.0 / dt; x.h = p.h; x.ihf = p.ihf;
    x.hf = p.hf;
    x.hc = p.hc; x.h2 = p.h2; x.fwl = p.fwl; x.fwr = p.fwr; x.hidt = p.hidt; x.dxicdt = p.dxicdt;
    x.lo_slot = p.lo_slot;
    x.pc = reinterpret_cast<const fpair *>(p.lopc);
    x.L = L;
    x.a_cell = nullptr; x.s_cell = nullptr;
    x.gate = p.gate;
    return x;
}

// shared memory of one LO solve; the FP32 form with refinement keeps both copies of the
// rows and falls back to the FP64 form where they do not fit (n_x above ~3100)
static size_t lo_smem(int precision, int nx)
{
    const size_t S = 32 * (size_t)lo_mmax(nx);
    if (lo_fp32(precision) && 6 * S * (sizeof(double) + sizeof(float)) <= 227 * 1024)
        return 6 * S * (sizeof(double) + sizeof(float));
    if (lo_pair(precision)) return 7 * S * sizeof(double);   // + the face factors of Fold
    return 6 * S * sizeof(double);
}
static bool lo_refined(int precision, int nx)
{
    return lo_fp32(precision) && 6 * 32 * (size_t)lo_mmax(nx) * 12 <= 227 * 1024;
}

cudaError_t launch_lo_solve(const Problem &p, double dt, const Level &L)
{
    const LoCtx x = make_lo_ctx(p, dt, L);
    const size_t sm = lo_smem(p.precision, p.nx);
    const unsigned nb = (unsigned)L.n;
    cudaError_t e;
    if (lo_pair(p.precision)) {
        e = cudaFuncSetAttribute(k_lo_solve<fpair>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm);
        if (e != cudaSuccess) return e;
        return launch_pdl(k_lo_solve<fpair>, dim3(nb), dim3(128), sm, p.stream, x);
    } else if (!lo_refined(p.precision, p.nx)) {
        e = cudaFuncSetAttribute(k_lo_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm);
        if (e != cudaSuccess) return e;
        return launch_pdl(k_lo_solve<double>, dim3(nb), dim3(128), sm, p.stream, x);
    } else {
        e = cudaFuncSetAttribute(k_lo_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm);
        if (e != cudaSuccess) return e;
        return launch_pdl(k_lo_solve<float>, dim3(nb), dim3(128), sm, p.stream, x);
    }
}

cudaError_t launch_lo_solve_b(int precision, int max_nx, const int *meta, int N,
                              const LoCtx *xs, int grid, cudaStream_t st)
{
    const size_t sm = lo_smem(precision, max_nx);
    cudaError_t e;
    if (lo_pair(precision)) {
        e = cudaFuncSetAttribute(k_lo_solve_b<fpair>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm);
        if (e != cudaSuccess) return e;
        k_lo_solve_b<fpair><<<grid, 128, sm, st>>>(meta, N, xs);
    } else if (!lo_refined(precision, max_nx)) {
        e = cudaFuncSetAttribute(k_lo_solve_b<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm);
        if (e != cudaSuccess) return e;
        k_lo_solve_b<double><<<grid, 128, sm, st>>>(meta, N, xs);
    } else {
        e = cudaFuncSetAttribute(k_lo_solve_b<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm);
        if (e != cudaSuccess) return e;
        k_lo_solve_b<float><<<grid, 128, sm, st>>>(meta, N, xs);
    }
    return cudaGetLastError();
}

size_t restrict_scratch_doubles(int nx, int n_from, int n_to)
{
    const int r = n_from / n_to;
    if (r < 64) return 0;
    const int nchunk = (r + kChunk - 1) / kChunk;
    return (size_t)n_to * nchunk * kRP * (nx + 1);
}

int restrict2_nchunk(int n_from, int n_to) { return (n_from / n_to + kChunk - 1) / kChunk; }

int restrict_kind(const Problem &p, int n_from, int n_to, int *KS)
{
    const size_t need = restrict_scratch_doubles(p.nx, n_from, n_to);
    if (need > 0 && p.rscratch && need <= p.rscratch_doubles) return 2;
    const int r = n_from / n_to;
    int k = 1;
    while (k < 16 && k * 4 <= r) k *= 2;   // <= 512 threads: the register file holds them
    *KS = k;
    return 1;
}

RestrictCtx make_restrict_ctx(const Problem &p, const Level &src, const Level &dst)
{
    RestrictCtx x;
    x.nx = p.nx; x.r = src.n / dst.n; x.h = p.h; x.ihf = p.ihf; x.S = src; x.T = dst;
    x.gate = p.gate;
    return x;
}

Restrict2Ctx make_restrict2_ctx(const Problem &p, const Level &src, const Level &dst)
{
    Restrict2Ctx y;
    y.nx = p.nx; y.r = src.n / dst.n; y.nchunk = restrict2_nchunk(src.n, dst.n);
    y.h = p.h; y.ihf = p.ihf; y.S = src; y.T = dst; y.part = p.rscratch;
    y.gate = p.gate;
    y.newton = 0;
    y.ga = GreyArgs{};
    y.pre = nullptr;
    y.skip_old = 0;
    return y;
}

static size_t restrict_smem(int KS) { return (KS > 1) ? sizeof(double) * KS * 32 * kRV1 : 0; }

cudaError_t launch_restrict(const Problem &p, const Level &src, Level &dst,
                            const GreyArgs *newton, double *pre, bool *formed, int *old_key)
{
    int KS = 1;
    if (formed) *formed = false;
    const int key = 2 * src.n + (src.fine ? 1 : 0);
    if (restrict_kind(p, src.n, dst.n, &KS) == 2) {
        Restrict2Ctx y = make_restrict2_ctx(p, src, dst);
        if (old_key) {
            y.skip_old = (*old_key == key) ? 1 : 0;
            *old_key = key;
        }
        if (newton && pre && dst.n == 1 && !newton->have_prev_dev) {
            y.newton = 1;
            y.ga = *newton;
            y.pre = pre;
            if (formed) *formed = true;
        }
        dim3 g1((p.nx + 1 + 31) / 32, dst.n * y.nchunk);
        cudaError_t e = cudaFuncSetAttribute(k_restrict_part,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kPartSmem);
        if (e != cudaSuccess) return e;
        e = launch_pdl(k_restrict_part, g1, dim3(32, kPartRows), kPartSmem, p.stream, y);
        if (e != cudaSuccess) return e;
        return launch_pdl(k_restrict_final, dim3((p.nx + 1 + 31) / 32, dst.n), dim3(32, kRP), 0,
                          p.stream, y);
    }
    if (old_key) *old_key = 0;   // the one-stage form sums them in another order
    const RestrictCtx x = make_restrict_ctx(p, src, dst);
    dim3 grid((p.nx + 1 + 31) / 32, dst.n);
    const size_t sm = restrict_smem(KS);
    cudaError_t e = cudaFuncSetAttribute(k_restrict, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_restrict, grid, dim3(32, KS), sm, p.stream, x);
}

cudaError_t launch_restrict_b(int KS, const int *meta, int N, const RestrictCtx *xs, int grid,
                              cudaStream_t st)
{
    const size_t sm = restrict_smem(KS);
    cudaError_t e = cudaFuncSetAttribute(k_restrict_b, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    k_restrict_b<<<grid, dim3(32, KS), sm, st>>>(meta, N, xs);
    return cudaGetLastError();
}

cudaError_t launch_restrict_part_b(const int *meta, int N, const Restrict2Ctx *xs, int grid,
                                   cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(k_restrict_part_b,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kPartSmem);
    if (e != cudaSuccess) return e;
    k_restrict_part_b<<<grid, dim3(32, kPartRows), kPartSmem, st>>>(meta, N, xs);
    return cudaGetLastError();
}

cudaError_t launch_restrict_final_b(const int *meta, int N, const Restrict2Ctx *xs, int grid,
                                    cudaStream_t st)
{
    k_restrict_final_b<<<grid, dim3(32, kRP), 0, st>>>(meta, N, xs);
    return cudaGetLastError();
}

GreyArgs grey_args_ready(const Problem &p, const GreyArgs &a)
{
    GreyArgs r = a;
    r.cvdt = a.cv / a.dt;
    r.k54 = 54.0 * a.s * kCB;
    const SeriesTables &t = host_series();
    r.e2 = p.e2tab;
    r.ec = ExpConsts{t.einv, t.eL1, t.eL2};
    return r;
}

GreyCtx make_grey_ctx(const Problem &p, const Level &g, const GreyArgs &a)
{
    GreyCtx x;
    x.lo = make_lo_ctx(p, a.dt, g);
    x.a = grey_args_ready(p, a);
    x.mmax = lo_mmax(p.nx);
    return x;
}

static void grey_launch_shape(int nx, int &bs, size_t &sm)
{
    bs = std::min(1024, std::max(32, (nx + 31) / 32 * 32));
    // Newton terms, block maxima, then grey_tri_solve's rows and reduced rows
    sm = sizeof(double) * (3 * (size_t)nx + kGreyRed + 3 * (size_t)(nx + 1) + 3 * (size_t)nx +
                           6 * 256);
}

cudaError_t launch_grey(const Problem &p, const Level &g, const GreyArgs &a)
{
    const GreyCtx x = make_grey_ctx(p, g, a);
    int bs;
    size_t sm;
    grey_launch_shape(p.nx, bs, sm);
    cudaError_t e = cudaFuncSetAttribute(k_grey, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_grey, dim3(1), dim3(bs), sm, p.stream, x);
}

cudaError_t launch_grey_b(int max_nx, const int *meta, int N, const GreyCtx *xs, int grid,
                          cudaStream_t st)
{
    int bs;
    size_t sm;
    grey_launch_shape(max_nx, bs, sm);
    cudaError_t e = cudaFuncSetAttribute(k_grey_b, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    k_grey_b<<<grid, bs, sm, st>>>(meta, N, xs);
    return cudaGetLastError();
}

cudaError_t launch_group_sum(const Problem &p, int n, const double *X, double *out)
{
    GroupSumArgs a;
    a.n = n; a.nx = p.nx; a.X = X; a.out = out;
    k_group_sum<<<(p.nx + 31) / 32, 256, 0, p.stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_group_sum_b(const int *meta, int N, const GroupSumArgs *xs, int grid,
                               cudaStream_t st)
{
    k_group_sum_b<<<grid, 256, 0, st>>>(meta, N, xs);
    return cudaGetLastError();
}

cudaError_t launch_copy_b(const int *meta, int N, const CopyArgs *xs, int grid, cudaStream_t st)
{
    k_copy_b<<<grid, 256, 0, st>>>(meta, N, xs);
    return cudaGetLastError();
}

}  // namespace trt
