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
