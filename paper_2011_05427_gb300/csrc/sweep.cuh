// sweep.cuh -- pieces shared by the FP64/FP32 strip sweeps (sweep.cu) and the lean FP32
// sweep (sweepf.cu): the per-tile angular accumulator and the cp.async wrappers.
#pragma once
#include "batch.cuh"

namespace trt {

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

// a / b for b != 0: a times the hardware reciprocal of b refined by one third-order step
// (below FP64 rounding) while that reciprocal is a normal number of moderate exponent,
// else the IEEE division (in a function that is never inlined: a branch around it, not
// predicated FP64 instructions); the exponent test runs on integer instructions
static __device__ __noinline__ double div64_slow(double a, double b) { return a / b; }
__device__ inline double ratio64(double a, double b)
{
    double x;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(b));
    const unsigned ex = ((unsigned)__double2hiint(x) >> 20) & 0x7ffu;
    if (ex - 1u >= 2018u) return div64_slow(a, b);
    const double e = fma(-b, x, 1.0);
    return a * fma(x, fma(e, e, e), x);
}

// (S2 + E2) / (S0 + E0) for unevaluated FP32 sums (|E| far below |S|) in FP32 arithmetic:
// q = S2/S0 rounded, the remainder (S2 + E2) - q (S0 + E0) with the exact product q S0 =
// ph + pl (S2 - ph is exact: ph is within a rounding of S2), d = remainder / (S0 + E0), and
// q + d widened to FP64 (one FP64 addition): within about 2^-46 of the quotient.  Zero,
// subnormal or non-finite S0 go to the FP64 form (a function never inlined); zero sums
// give 1/3.
static __device__ __noinline__ double pair_ratio_fp64(float S2, float E2, float S0, float E0)
{
    const double a0 = (double)S0 + (double)E0, a2 = (double)S2 + (double)E2;
    return (a0 != 0.0) ? a2 / a0 : 1.0 / 3.0;
}
__device__ inline double pair_ratio(float S2, float E2, float S0, float E0)
{
    const unsigned e = (__float_as_uint(S0) >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return pair_ratio_fp64(S2, E2, S0, E0);
    const float q = __fdiv_rn(S2, S0);
    const float ph = __fmul_rn(q, S0);
    const float pl = __fmaf_rn(q, S0, -ph);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(S2, ph), pl), __fsub_rn(E2, __fmul_rn(q, E0)));
    const float d = __fdiv_rn(r, __fadd_rn(S0, E0));
    return widen_f32(q) + widen_f32(d);
}

// f of one (group, cell) from NT direction tiles of FP64 partial moments (tile t's at
// p[2 t n] and p[(2 t + 1) n]).  GB300 adds FP64 numbers at 1/64 of the FP32 rate, so the
// tiles are added as fixed-point integers on the integer pipes: every value's significand
// (hidden bit included) shifted to the largest exponent emax of the element's 2 NT values
// and summed exactly in 64 bits (at most 16 values below 2^53: no overflow); each value
// loses only its bits below 2^(emax - 52), so each sum is within NT units of the largest
// value's last place -- order-independent, no FP64 addition.  A2/A0 then is the ratio of
// the two integer sums (the common scale cancels): two conversions and A2 times the refined
// reciprocal of A0.  Subnormal values enter with their own significand at the least
// exponent (exactly their value); a zero zeroth sum gives 1/3; elements holding an infinity
// or NaN take the FP64 sum (in tile order) and division.
static __device__ __noinline__ double sum_tiles_ratio_fp64(const double *__restrict__ p,
                                                           size_t n, int nt)
{
    double A0 = 0.0, A2 = 0.0;
    for (int t = 0; t < nt; ++t) {
        A0 += p[(size_t)(2 * t) * n];
        A2 += p[(size_t)(2 * t + 1) * n];
    }
    return (A0 != 0.0) ? A2 / A0 : 1.0 / 3.0;
}
__device__ inline long long fixed_point(unsigned long long b, int emax)
{
    int e = (int)((b >> 52) & 0x7ffull);
    unsigned long long M = b & 0xfffffffffffffull;
    if (e == 0)
        e = 1;   // subnormal (or zero): significand without the hidden bit, exponent 1
    else
        M |= 1ull << 52;
    const int d = emax - e;
    if (d > 63) return 0;
    const long long v = (long long)(M >> d);
    return (b >> 63) ? -v : v;
}
template <int NT>
__device__ inline double sum_tiles_ratio(const double *__restrict__ p, size_t n)
{
    unsigned long long b0[NT], b2[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        b0[t] = (unsigned long long)__double_as_longlong(p[(size_t)(2 * t) * n]);
        b2[t] = (unsigned long long)__double_as_longlong(p[(size_t)(2 * t + 1) * n]);
    }
    int emax = 1;   // subnormal values count at exponent 1
#pragma unroll
    for (int t = 0; t < NT; ++t)
        emax = max(emax, max((int)((b0[t] >> 52) & 0x7ffull), (int)((b2[t] >> 52) & 0x7ffull)));
    if (emax == 0x7ff) return sum_tiles_ratio_fp64(p, n, NT);
    long long S0 = 0, S2 = 0;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        S0 += fixed_point(b0[t], emax);
        S2 += fixed_point(b2[t], emax);
    }
    if (S0 == 0) return 1.0 / 3.0;
    return ratio64(__ll2double_rn(S2), __ll2double_rn(S0));
}

// forward declaration (defined below)
__device__ inline void two_sum_acc(float &S, float &E, float hi, float lo);

// f of one (group, cell) from NT direction tiles of FP32 (high, low) partial moments: p
// points at tile 0's zeroth moment, tile t's moments at p[2 t n] and p[(2 t + 1) n], their
// low parts NT 2 n further; every load is issued before the first addition
template <int NT>
__device__ inline double sum_pairs_ratio(const float *__restrict__ p, size_t n)
{
    float h0[NT], h2[NT], l0[NT], l2[NT];
    const size_t lo = (size_t)NT * 2 * n;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        h0[t] = p[(size_t)(2 * t) * n];
        h2[t] = p[(size_t)(2 * t + 1) * n];
        l0[t] = p[lo + (size_t)(2 * t) * n];
        l2[t] = p[lo + (size_t)(2 * t + 1) * n];
    }
    float S0 = 0.f, E0 = 0.f, S2 = 0.f, E2 = 0.f;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        two_sum_acc(S0, E0, h0[t], l0[t]);
        two_sum_acc(S2, E2, h2[t], l2[t]);
    }
    return pair_ratio(S2, E2, S0, E0);
}

// (S, E) += hi + lo for unevaluated FP32 sums S + E: hi enters by an exact two-sum (Knuth),
// its rounding error and lo go to E
__device__ inline void two_sum_acc(float &S, float &E, float hi, float lo)
{
    const float s = __fadd_rn(S, hi);
    const float bb = __fsub_rn(s, S);
    const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bb)), __fsub_rn(hi, bb));
    S = s;
    E = __fadd_rn(E, __fadd_rn(err, lo));
}

// cp.async (global -> shared, completion per issuing thread): the next strip's data is
// in flight while the current strip is swept.
template <int B>
__device__ inline void cp_async(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(B));
}
__device__ inline void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ inline void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// boundary-factor blocks of the sweep's finalize: one warp per group, 8 per block
__host__ __device__ inline int finalize_bnd_blocks_dev(int G) { return (G + 7) / 8; }

// the lean FP32 sweep of a shape kind (5: one group per lane, 6: two), strip S, buffers NS:
// the single-slab grid when `a` is given, else the persistent grid over the work list;
// cudaErrorInvalidConfiguration for a tile height D it has no kernel for (D = 4, 8, 16)
// shared memory of a lean sweep kernel (0: no such kernel)
size_t sweepf_smem(int kind, int S, int NS, int D);
// the paired FP64 sweep of sweep64.cu (single slab, D = 4 directions of each sign per CTA;
// strip S, buffers NS): k_prescale64 of the raw sigma_E, e_g of `a` into a.tab64, then the
// sweep; shared memory of a shape (0: no such kernel)
size_t pair_sweep_smem(int S, int NS);
cudaError_t launch_sweep_pair(int S, int NS, const SweepArgs &a, int M, int ldG, cudaStream_t st);
cudaError_t launch_sweepf(int kind, int S, int NS, const SweepArgs *a, int M, int ldG, int D,
                          const int *meta, int N, const SweepArgs *xs, int grid, cudaStream_t st);

}  // namespace trt
