// pair.cuh -- FP32-pair ("double-float") arithmetic for the low-order kernels.
//
// A value is the unevaluated sum h + l of two floats with |l| <= ulp(h): about 47
// significant bits over FP32's exponent range.  GB300 issues FP32 FMAs at 64 times its
// FP64 rate (a warp-wide FP64 instruction holds a sub-partition's FP64 pipe for 64
// cycles), and a pair operation costs 6 to 15 FP32 instructions, so work that is bound by
// the FP64 pipe runs several times faster in pairs.  The operations are built from the
// error-free transformations of T. J. Dekker ("A floating-point technique for extending
// the available precision", Numer. Math. 18, 1971: the exact product a b = p + e as
// e = fma(a, b, -p), and the fast two-sum for |a| >= |b|) and D. E. Knuth (TAOCP vol. 2,
// Sec. 4.2.2: the two-sum of any two floats).  Additions take the "sloppy" form (the low
// parts are added in FP32): its error is below 2^-46 (|a| + |b|), the bound of an FP64
// addition's inputs at this precision.  Every FP32 operation is written with an explicit
// rounding intrinsic, so the compiler neither contracts nor reorders them.
//
// Conversions from FP64 use integer instructions only (GB300 converts FP64 <-> FP32 on
// the FP64 pipe): h takes the sign, the rebiased exponent and the top 23 fraction bits of
// the double; the remaining 29 fraction bits, rounded to 23, are read as the mantissa of a
// float against the power of two that their unit place has, minus that power (exact).
// |x| in [2^-103, 2^127) splits this way (relative error below 2^-47); below that h alone
// holds x truncated to 24 bits, and below 2^-126 (zeros included) x is a signed zero --
// the pair form has FP32's normal exponent range, so a kernel that holds values of one
// linear system in pairs scales them by a power of two first (an offset of the exponent
// in the same integer instructions); |x| >= 2^128 becomes inf, inf and NaN stay so.  Back
// to FP64: both parts widen with integer instructions (subnormal parts as zero), then one
// FP64 addition.  Nothing here calls a function: an opaque call would keep the compiler
// from issuing later loads ahead of it.
#pragma once
#include <cuda_runtime.h>
#include <type_traits>
#include "common.cuh"

namespace trt {

struct __align__(8) fpair {
    float h, l;
    fpair() = default;
    __device__ constexpr fpair(float a, float b) : h(a), l(b) {}
    __device__ constexpr fpair(int v) : h((float)v), l(0.f) {}   // small integer constants
    __device__ explicit fpair(double x);
    __device__ explicit operator double() const;
};

template <typename R>
constexpr bool is_pair = std::is_same<R, fpair>::value;

// |a| >= |b| (or a == 0): s + e = a + b exactly
__device__ inline fpair pr_fast_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return fpair(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// any a, b: s + e = a + b exactly
__device__ inline fpair pr_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return fpair(s, e);
}

__device__ inline fpair operator+(fpair a, fpair b)
{
    const fpair s = pr_two_sum(a.h, b.h);
    return pr_fast_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ inline fpair operator-(fpair a) { return fpair(-a.h, -a.l); }
__device__ inline fpair operator-(fpair a, fpair b) { return a + (-b); }
__device__ inline fpair operator*(fpair a, fpair b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return pr_fast_sum(p, e);
}
// a b + c with one normalisation
__device__ inline fpair fma(fpair a, fpair b, fpair c)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    const fpair s = pr_two_sum(p, c.h);
    return pr_fast_sum(s.h, __fadd_rn(s.l, __fadd_rn(e, c.l)));
}
using ::fma;

// 1/b: the hardware's approximate FP32 reciprocal (relative error below 2^-22), one FP32
// Newton step (q within about an ulp of 1/b.h), then the pair step q (1 + e), e = 1 - b q:
// 1 - b.h q is a multiple of ulp(b.h) ulp(q) below 2^-22 in magnitude and so exact in one
// FMA; the step's truncation e^2 is below 2^-46.  No branch: |b.h| must lie in the normal
// range (the diagonals of the low-order systems do).
__device__ inline fpair prcp(fpair b)
{
    float q;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(q) : "f"(b.h));
    q = __fmaf_rn(q, __fmaf_rn(-b.h, q, 1.f), q);
    float e = __fmaf_rn(-b.h, q, 1.f);
    e = __fmaf_rn(-b.l, q, e);
    return pr_fast_sum(q, __fmul_rn(q, e));
}
__device__ inline fpair operator/(fpair a, fpair b) { return a * prcp(b); }
__device__ inline fpair &operator+=(fpair &a, fpair b) { return a = a + b; }
__device__ inline fpair &operator-=(fpair &a, fpair b) { return a = a - b; }
__device__ inline fpair &operator*=(fpair &a, fpair b) { return a = a * b; }

// x 2^-k as a pair (|k| < 1024)
__device__ inline fpair pr_split(double x, int k)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const int e0 = (int)((hw >> 20) & 0x7ffu);
    const unsigned s = hw & 0x80000000u;
    if (e0 == 0x7ff)   // inf, NaN (a quiet NaN keeps the sign)
        return fpair(__uint_as_float(s | 0x7f800000u | (((hw & 0xfffffu) | lw) ? 0x400000u : 0u)),
                     0.f);
    const int e = (e0 == 0) ? 0 : e0 - k;          // biased exponent of x 2^-k (0: zero)
    if (e < 920 || e > 1150) {   // outside [2^-103, 2^128)
        if (e < 920)   // below: h alone (FP32 precision), zero below 2^-126
            return fpair(__uint_as_float(e >= 897 ? s | ((unsigned)(e - 896) << 23) |
                                                        ((hw & 0xfffffu) << 3) | (lw >> 29)
                                                  : s),
                         0.f);
        return fpair(__uint_as_float(s | 0x7f800000u), 0.f);   // |x 2^-k| >= 2^128: inf
    }
    const float h = __uint_as_float(s | ((unsigned)(e - 896) << 23) | ((hw & 0xfffffu) << 3) |
                                    (lw >> 29));
    // bits 28..0 of the fraction, rounded to 23 (a carry into bit 23 is the next power of
    // two, still exact), against 2^(e-1023-46) = the float of biased exponent e - 919
    const unsigned eb = (unsigned)(e - 919) << 23;
    const unsigned m = ((lw & 0x1fffffffu) + 32u) >> 6;
    const float lo = __fsub_rn(__uint_as_float(eb + m), __uint_as_float(eb));
    return fpair(h, __uint_as_float(__float_as_uint(lo) | s));
}
__device__ inline fpair::fpair(double x)
{
    const fpair v = pr_split(x, 0);
    h = v.h;
    l = v.l;
}
// q 2^k in FP64 with integer instructions; subnormal q, and results below FP64's normal
// range, as zero; inf and NaN stay so, results above FP64's range are inf
__device__ inline double pr_widen(float q, int k)
{
    const unsigned u = __float_as_uint(q);
    const int e = (int)((u >> 23) & 0xffu);
    const unsigned long long sg = (unsigned long long)(u & 0x80000000u) << 32;
    const int E = e + 896 + k;
    if (e == 0 || E <= 0) return __longlong_as_double((long long)sg);
    if (e == 0xff || E >= 2047)
        return __longlong_as_double((long long)(sg | 0x7ff0000000000000ull |
                                                ((e == 0xff && (u & 0x7fffffu)) ? 1ull << 51 : 0ull)));
    return __longlong_as_double((long long)(sg | ((unsigned long long)E << 52) |
                                            ((unsigned long long)(u & 0x7fffffu) << 29)));
}
// (h + l) 2^k in FP64: one FP64 addition
__device__ inline double pr_join(fpair a, int k) { return pr_widen(a.h, k) + pr_widen(a.l, k); }
__device__ inline fpair::operator double() const { return pr_join(*this, 0); }

// q 2^k in FP32 with integer instructions; results below FP32's normal range as zero,
// above it inf
__device__ inline float pr_ldexpf(float q, int k)
{
    const unsigned u = __float_as_uint(q);
    const int e = (int)((u >> 23) & 0xffu);
    if (e == 0 || e == 0xff) return q;
    const int E = e + k;
    if (E <= 0) return __uint_as_float(u & 0x80000000u);
    if (E >= 255) return __uint_as_float((u & 0x80000000u) | 0x7f800000u);
    return __uint_as_float((u & 0x807fffffu) | ((unsigned)E << 23));
}

// e^w = ew 2^k (|w| < 9e4; w.h <= -1e4 gives ew = 0): the table-driven reduction of P. T. P.
// Tang (ACM TOMS 15, 1989) in pair arithmetic.  w = n ln2/32 + r with n = rint(w 32/ln2)
// (FP32 rounding by adding 1.5 2^23: n sits in the low bits) and ln2/32 = L1 + L2 + L3,
// L1 = 177/2^13 (8 significant bits: n L1 is exact in FP32 for |n| < 2^16), L2 and L3 the
// next two FP32 parts (ln2/32 to 1.6e-18 relative).  w.h - n L1 is exact (Sterbenz); its
// difference with the exact product n L2 and the sum with w.l are two-sums; the remaining
// parts (each below 1e-7) add in FP32, 6e-15 of r's scale at most.  Then e^r - 1 = r + r^2 P,
// P = 1/2 + Q, Q = r/6 + r^2/24 + r^3/120 + r^4/720 in FP32 from r.h (|Q| < 1.9e-3: its
// rounding is 1e-10 of P, below 1e-14 of e^r; the dropped r^7/5040 is 3e-18), and
// ew = 2^(j/32) (1 + (e^r - 1)), j = n mod 32, k = (n - j)/32; tab holds 2^(j/32) as pairs.
// The relative error of ew is about 2^-46 plus that of w itself (2^-47 |w|).
__device__ inline fpair pr_exp(fpair w, int &k, const fpair *tab)
{
    if (w.h <= -1e4f) { k = 0; return fpair(0.f, 0.f); }
    const float kMagic = 12582912.f;   // 1.5 2^23
    const float sk = __fmaf_rn(w.h, 46.16624069213867f, kMagic);
    const int n = __float_as_int(sk) - 0x4b400000;
    const float nf = __fsub_rn(sk, kMagic);
    const float L1 = 0x1.62p-6f, L2 = 0x1.c85fep-15f, L3 = -0x1.718432p-40f;
    const float a = __fmaf_rn(-nf, L1, w.h);          // exact
    const float p2 = __fmul_rn(nf, L2);
    const float e2 = __fmaf_rn(nf, L2, -p2);           // n L2 = p2 + e2 exactly
    const fpair d = pr_two_sum(a, -p2);
    const fpair s1 = pr_two_sum(d.h, w.l);
    const float tail = __fsub_rn(__fsub_rn(__fadd_rn(d.l, s1.l), e2), __fmul_rn(nf, L3));
    const fpair r = pr_fast_sum(s1.h, tail);
    const float u = r.h;
    const float Q = __fmul_rn(u, __fmaf_rn(u, __fmaf_rn(u, __fmaf_rn(u, 1.f / 720, 1.f / 120),
                                                         1.f / 24),
                                          1.f / 6));
    const fpair em1 = fma(r * r, pr_fast_sum(0.5f, Q), r);
    const fpair t = tab[n & 31];
    k = n >> 5;
    return fma(t, em1, t);
}

// warp shuffles of either number type
template <typename R>
__device__ inline R shfl_up(unsigned m, R v, int d)
{
    if constexpr (is_pair<R>)
        return fpair(__shfl_up_sync(m, v.h, d), __shfl_up_sync(m, v.l, d));
    else
        return __shfl_up_sync(m, v, d);
}
template <typename R>
__device__ inline R shfl_down(unsigned m, R v, int d)
{
    if constexpr (is_pair<R>)
        return fpair(__shfl_down_sync(m, v.h, d), __shfl_down_sync(m, v.l, d));
    else
        return __shfl_down_sync(m, v, d);
}

}  // namespace trt
