// mlp.cu -- the learned closure's network on the tensor cores: a BF16 GEMM on tcgen05
// (tensor memory accumulators, shared-memory operand descriptors, mbarrier-tracked
// commits) with fused epilogues, and the MLP's forward, backward, Adam and feature
// kernels built on it.  The paper has no learned component; see include/trt_mlp.h.
//
// GEMM tile: 128 rows x 256 columns per CTA, K in chunks of 64 through two shared-memory
// stages.  Four warps copy each chunk with cp.async into the canonical no-swizzle K-major
// layout of the tensor core (8-row x 16-byte core matrices, 128 contiguous bytes each; the
// 8 core matrices of a row group along K are adjacent, 128 bytes apart, and row groups are
// 1024 bytes apart -- either reading of the two descriptor strides stays inside the stage);
// one thread issues four tcgen05.mma (M 128, N 256, K 16) per chunk and commits them to
// the stage's mbarrier, which releases the stage for the chunk after next.  The 128 x 256
// FP32 accumulator lives in 256 tensor-memory columns; in the epilogue thread t owns row
// t (tensor-memory lane t) and reads its 256 values 32 at a time with tcgen05.ld.
#include <algorithm>
#include <cuda_bf16.h>
#include <stdint.h>
#include "common.cuh"
#include "../../include/trt_mlp.h"

namespace trt {

namespace {

typedef __nv_bfloat16 bf16;

constexpr int BM = 128, BN = 256, BK = 64;
constexpr int A_STAGE = BM * BK * 2;   // 16 KB
constexpr int B_STAGE = BN * BK * 2;   // 32 KB
constexpr int GEMM_SMEM = 2 * (A_STAGE + B_STAGE) + 256;
// core-matrix (row group r, K group k) of a stage at (r * 8 + k) * 128: leading-dimension
// (K) byte offset 128, stride-dimension (row group) byte offset 1024
constexpr uint32_t LBO = 128, SBO = 1024;
// instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9,
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);
constexpr unsigned long long WAIT_NS = 1000000000ull;   // one second

__device__ int g_mlp_err = 0;

__device__ inline uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline unsigned long long gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ inline void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count));
}

__device__ inline bool mbar_test(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait on a phase of an mbarrier: false after WAIT_NS without completion
__device__ inline bool mbar_wait(uint64_t *bar, unsigned parity)
{
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = gtime();
    while (!mbar_test(bar, parity))
        if (gtime() - t0 > WAIT_NS) return false;
    return true;
}

__device__ inline void cp16(void *dst, const void *src, unsigned bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(su32(dst)), "l"(src),
                 "r"(bytes));
}
__device__ inline void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ inline void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ inline void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ inline void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// shared-memory operand descriptor: start >> 4 (bits 0-13), leading-dimension byte offset
// >> 4 (16-29), stride-dimension byte offset >> 4 (32-45), descriptor version 1 (46-47),
// base offset 0, no swizzle (61-63 = 0)
__device__ inline uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
           ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

__device__ inline void umma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(IDESC), "r"(acc));
}

__device__ inline void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     su32(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 tensor-memory lanes (one per thread)
__device__ inline void tmem_ld32(uint32_t taddr, float *v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// the same load without its wait (two loads may be in flight before one wait), and the
// wait tied to the loaded registers so that no use of them is scheduled before it
__device__ inline void tmem_ld32_issue(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
}
__device__ inline void tmem_wait_tied(uint32_t (&r)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}
__device__ inline void reg_tie(uint32_t (&r)[32])
{
    asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]));
}

struct Epi {
    const float *bias;
    int relu;
    const bf16 *mask;
    float *out32;
    bf16 *out16, *out16T;
    int ldT;
    // head: z = sum_n act[n] w[n] + b, y = sigmoid(z); with a target, also
    // dz = scale (y - t) y (1 - y), sq = (y - t)^2, dact = dz w[n] [act > 0]
    const float *head_w;
    const float *head_b;   // device pointer to the head's bias
    float *head_y;
    const float *target;
    float scale;
    float *dz, *sq;
    bf16 *dact16, *dact16T;
};

__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, const bf16 *__restrict__ A,
                                              const bf16 *__restrict__ B, Epi e)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sA = sm;
    unsigned char *sB = sm + 2 * A_STAGE;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + 2 * (A_STAGE + B_STAGE));
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 2);
    int *sfail = reinterpret_cast<int *>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int nk = K / BK;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        *sfail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(tslot)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tslot;

    // chunk c of A (128 x 64) and B (256 x 64) into stage st in 16-byte pieces: piece p
    // is row p & 7 of core matrix (row group p >> 6, K group (p >> 3) & 7), i.e. shared
    // offset 16 p (conflict-free); rows of A past M are zero-filled
    auto load = [&](int c, int st) {
        const int k0 = c * BK;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int p = tid + 128 * j;
            const int r8 = p & 7, ki = (p >> 3) & 7, mi = p >> 6;
            const int row = m0 + mi * 8 + r8;
            const bf16 *src = A + (size_t)min(row, M - 1) * K + k0 + ki * 8;
            cp16(sA + st * A_STAGE + p * 16, src, row < M ? 16u : 0u);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int p = tid + 128 * j;
            const int r8 = p & 7, ki = (p >> 3) & 7, ni = p >> 6;
            const bf16 *src = B + (size_t)(n0 + ni * 8 + r8) * K + k0 + ki * 8;
            cp16(sB + st * B_STAGE + p * 16, src, 16u);
        }
    };

    load(0, 0);
    cp_commit();
    if (nk > 1) load(1, 1);
    cp_commit();
    bool ok = true;
    for (int c = 0; c < nk; ++c) {
        const int st = c & 1;
        if (c + 1 < nk)
            cp_wait<1>();
        else
            cp_wait<0>();
        fence_async_smem();   // this thread's copies -> visible to the tensor core
        __syncthreads();
        if (*sfail) { ok = false; break; }
        if (tid == 0) {
            tc_after();
            const uint32_t a0 = su32(sA + st * A_STAGE), b0 = su32(sB + st * B_STAGE);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)   // K = 16 per instruction: 2 core matrices
                umma(tmem, sdesc(a0 + kk * 2 * LBO, LBO, SBO), sdesc(b0 + kk * 2 * LBO, LBO, SBO),
                     (c | kk) != 0);
            umma_commit(&bar[st]);
        }
        if (c + 2 < nk) {
            // stage st takes chunk c + 2 once the MMAs of chunk c have read it
            if (!mbar_wait(&bar[st], (c >> 1) & 1)) *sfail = 1;
            __syncthreads();
            if (*sfail) { ok = false; break; }
            load(c + 2, st);
            cp_commit();
        }
    }
    if (ok && !mbar_wait(&bar[(nk - 1) & 1], ((nk - 1) >> 1) & 1)) ok = false;
    ok = !__syncthreads_or(!ok);   // CTA-uniform: the tensor-memory loads are warp-collective
    if (!ok) {
        cp_wait<0>();
        if (lane == 0) atomicExch(&g_mlp_err, TRT_ETIMEOUT);
    }
    tc_after();

    const int row = m0 + tid;
    if (ok) {
        float dot = 0.f;
        for (int ch = 0; ch < BN / 32; ++ch) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + ch * 32, v);
            if (row >= M) continue;
            const int nb = n0 + ch * 32;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                float a = v[j];
                if (e.bias) a += e.bias[nb + j];
                if (e.relu) a = fmaxf(a, 0.f);
                v[j] = a;
            }
            if (e.mask) {
                const uint4 *mk = reinterpret_cast<const uint4 *>(e.mask + (size_t)row * N + nb);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint4 u = mk[q];
                    const bf16 *hb = reinterpret_cast<const bf16 *>(&u);
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (!(__bfloat162float(hb[j]) > 0.f)) v[q * 8 + j] = 0.f;
                }
            }
            if (e.out32) {
                float4 *o = reinterpret_cast<float4 *>(e.out32 + (size_t)row * N + nb);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
            if (e.out16) {
                uint4 *o = reinterpret_cast<uint4 *>(e.out16 + (size_t)row * N + nb);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint4 u;
                    bf16 *hb = reinterpret_cast<bf16 *>(&u);
#pragma unroll
                    for (int j = 0; j < 8; ++j) hb[j] = __float2bfloat16_rn(v[q * 8 + j]);
                    o[q] = u;
                }
            }
            if (e.out16T) {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    e.out16T[(size_t)(nb + j) * e.ldT + row] = __float2bfloat16_rn(v[j]);
            }
            if (e.head_w) {
#pragma unroll
                for (int j = 0; j < 32; ++j) dot = fmaf(v[j], e.head_w[nb + j], dot);
            }
        }
        float dz = 0.f;
        if (e.head_w && row < M) {
            const float z = dot + *e.head_b;
            const float y = 1.f / (1.f + __expf(-z));
            if (e.head_y) e.head_y[row] = y;
            if (e.target) {
                const float d = y - e.target[row];
                dz = e.scale * d * y * (1.f - y);
                e.dz[row] = dz;
                e.sq[row] = 0.5f * e.scale * d * d;
            }
        }
        if (e.head_w && e.target) {
            // second pass over the accumulator (all threads: the loads are warp-collective)
            // for the gradient of the last hidden layer, dz w4 [h3 > 0]
            for (int ch = 0; ch < BN / 32; ++ch) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + ch * 32, v);
                if (row >= M) continue;
                const int nb = n0 + ch * 32;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float a = v[j] + (e.bias ? e.bias[nb + j] : 0.f);
                    const bf16 gb = __float2bfloat16_rn((a > 0.f) ? dz * e.head_w[nb + j] : 0.f);
                    e.dact16[(size_t)row * N + nb + j] = gb;
                    e.dact16T[(size_t)(nb + j) * e.ldT + row] = gb;
                }
            }
        }
    }
    tc_before();
    __syncthreads();
    if (warp == 0) {
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
    }
}

// ---- fused inference: the whole network in one persistent kernel ----
// One CTA per SM, 320 threads: two groups of four warps, a producer warp and an MMA warp.
// Each iteration takes 256 rows; group g (warps 4g .. 4g+3, thread = row = tensor-memory
// lane) owns rows 128 g .. 128 g + 127 of it, its activation tile A_g in shared memory and
// its 128 x 256 FP32 accumulator in tensor-memory columns 256 g .. 256 g + 255.  One thread
// (warp 8) streams the weights; one thread (warp 9) issues every MMA, in the order
//   layer 2 of group 0, layer 2 of group 1, layer 3 of group 0, layer 3 of group 1,
// so that while the tensor core multiplies for one group the other group's warps run its
// CUDA-core phase (layer 1, a ReLU/bias epilogue, the sigmoid head): the two groups work
// half a period apart and the MMAs of one hide the epilogues of the other.
//   Weights: 32-wide K chunks (16 KB, 256 rows x 32 K of W2 or W3) through a four-slot
// ring.  trt_mlp_refresh stores each chunk contiguously in the order the tensor core
// reads it (core matrices of 8 rows x 16 bytes; K groups 4096 bytes apart, row groups 128
// bytes apart), so one cp.async.bulk of 16 KB moves a chunk and completes on the slot's
// `full` mbarrier; the MMAs reading a slot commit to its `empty` mbarrier, which releases
// it for the chunk S later.  Every chunk is used by one group's layer, so each weight is
// streamed twice per 256 rows (from L2: the whole 256 KB image stays resident there).
//   The MMA thread never waits for a slot to drain (that is the producer's wait), so the
// tensor core always has the next chunk's MMAs queued behind the running ones.
//   Hand-offs: a group arrives on act[g] (128 arrivals) when A_g holds the next layer's
// input (after a proxy fence: the MMAs read it through the async proxy); the MMA thread
// commits the last MMA of a layer to acc[g], which the group waits on before it reads
// the accumulator.  Small parameters (layer-1 weights, biases, head) sit in shared
// memory.  Every mbarrier wait is bounded (one second); a wait that runs out stops the
// kernel's work and sets the device error flag (trt_mlp_status).
constexpr int FA_BYTES = 128 * 256 * 2;   // one activation tile
constexpr int FK = 32;                    // K width of a weight chunk
constexpr int FNC = 256 / FK;             // chunks per layer
constexpr int FW_BYTES = 256 * FK * 2;    // one weight chunk
constexpr int F_SLOTS = 4;
constexpr uint32_t FW_LBO = 4096, FW_SBO = 128;   // weight chunk: K groups, row groups
// small parameters in shared memory: W1^T [3][256], b1, b2, b3, w4, b4 (1793 floats)
constexpr int FP_W1 = 0, FP_B1 = 768, FP_B2 = 1024, FP_B3 = 1280, FP_W4 = 1536, FP_B4 = 1792;
constexpr int FP_BYTES = 1796 * 4;
constexpr int F_NBAR = 2 * F_SLOTS + 4;   // full[S], empty[S], act[2], acc[2]
constexpr int F_SMEM = 2 * FA_BYTES + F_SLOTS * FW_BYTES + FP_BYTES + 8 * F_NBAR + 32;
constexpr uint32_t FA_SBO = 4096;         // activation tiles: 32 K groups per row group
constexpr int F_THREADS = 320;

__device__ inline void mbar_init_n(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count));
}
__device__ inline void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ inline void mbar_expect(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)),
                 "r"(bytes)
                 : "memory");
}
// packed FP32 pairs (Blackwell f32x2 arithmetic: two lanes' worth of FP32 per instruction)
__device__ inline float2 fma2(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;"
        : "=l"(*reinterpret_cast<unsigned long long *>(&d))
        : "l"(*reinterpret_cast<const unsigned long long *>(&a)),
          "l"(*reinterpret_cast<const unsigned long long *>(&b)),
          "l"(*reinterpret_cast<const unsigned long long *>(&c)));
    return d;
}
__device__ inline float2 add2(float2 a, float2 b)
{
    float2 d;
    asm("add.rn.f32x2 %0, %1, %2;"
        : "=l"(*reinterpret_cast<unsigned long long *>(&d))
        : "l"(*reinterpret_cast<const unsigned long long *>(&a)),
          "l"(*reinterpret_cast<const unsigned long long *>(&b)));
    return d;
}
// relu of two FP32 values rounded to BF16 (nearest even) in one word, v.x in the low half:
// rounding keeps the sign, so rounding after the clamp equals clamping after rounding
__device__ inline uint32_t relu_bf16x2(float2 v)
{
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(v.y), "f"(v.x));
    return d;
}

// one contiguous bulk copy global -> this CTA's shared memory, completing (bytes) on `bar`
__device__ inline void bulk_copy(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}

__global__ void __launch_bounds__(F_THREADS, 1) k_mlp_fused(int rows, const float *__restrict__ x,
                                                            const float *__restrict__ P,
                                                            const bf16 *__restrict__ Wimg,
                                                            float *__restrict__ y)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sW = sm + 2 * FA_BYTES;   // F_SLOTS weight chunks
    float *sP = reinterpret_cast<float *>(sW + F_SLOTS * FW_BYTES);
    uint64_t *bar = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(sP) + FP_BYTES);
    uint64_t *full = bar, *empty = bar + F_SLOTS, *act = bar + 2 * F_SLOTS, *acc = act + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + F_NBAR);
    int *sfail = reinterpret_cast<int *>(tslot + 1);
    int *sprod = sfail + 1, *scons = sfail + 2;   // chunks copied / expected (failure drain)

    const int tid = threadIdx.x, warp = tid >> 5;
    const int ntiles = (rows + 255) / 256;
    const int mine = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (tid == 0) {
        for (int k = 0; k < F_SLOTS; ++k) {
            mbar_init_n(&full[k], 1);
            mbar_init_n(&empty[k], 1);   // the commit of the MMAs that read the slot
        }
        for (int g = 0; g < 2; ++g) {
            mbar_init_n(&act[g], 128);
            mbar_init_n(&acc[g], 1);
        }
        *sfail = 0;
        *sprod = 0;
        *scons = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         su32(tslot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid < 256) {   // small parameters (W1 transposed; float4 runs b1, b2, b3 + w4)
        const float4 *gp = reinterpret_cast<const float4 *>(P);
        float4 *d = reinterpret_cast<float4 *>(sP);
        for (int k = 0; k < 3; ++k) sP[FP_W1 + k * 256 + tid] = __ldg(P + TRT_MLP_W1 + 3 * tid + k);
        if (tid < 64) d[FP_B1 / 4 + tid] = __ldg(gp + TRT_MLP_B1 / 4 + tid);     // b1
        if (tid < 64) d[FP_B2 / 4 + tid] = __ldg(gp + TRT_MLP_B2 / 4 + tid);     // b2
        if (tid < 128) d[FP_B3 / 4 + tid] = __ldg(gp + TRT_MLP_B3 / 4 + tid);    // b3, w4
        if (tid == 0) sP[FP_B4] = __ldg(P + TRT_MLP_B4);
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = *tslot;
    bool ok = true;

    const int Q = 4 * FNC * mine;   // weight chunks: 4 layer-jobs of FNC chunks per iteration
    if (warp == 8) {
        // ---------------- producer thread ----------------
        if ((tid & 31) == 0) {
            int q = 0;
            for (; q < Q; ++q) {   // chunk q: job q / FNC, K chunk q % FNC, slot q % S
                if (q >= F_SLOTS && !mbar_wait(&empty[q % F_SLOTS], ((q - F_SLOTS) / F_SLOTS) & 1)) {
                    *sfail = 1;
                    break;
                }
                const int layer = (q / FNC) % 4 >= 2 ? 1 : 0;
                bulk_copy(sW + (q % F_SLOTS) * FW_BYTES,
                          Wimg + layer * 65536 + (q % FNC) * (FW_BYTES / 2), FW_BYTES,
                          &full[q % F_SLOTS]);
            }
            *sprod = q;
        }
    } else if (warp == 9) {
        // ---------------- MMA thread ----------------
        if ((tid & 31) == 0) {
            unsigned pact = 0;   // bit g: parity of act[g]'s next phase
            int q = 0;
            for (int it = 0; it < mine && ok; ++it) {
                for (int job = 0; job < 4 && ok; ++job) {
                    const int g = job & 1;
                    if (!mbar_wait(&act[g], (pact >> g) & 1u)) { ok = false; break; }
                    pact ^= 1u << g;
                    tc_after();
                    const uint32_t a0 = su32(sm + g * FA_BYTES);
                    const uint32_t d = tmem + (uint32_t)(g * 256);
                    for (int c = 0; c < FNC; ++c, ++q) {
                        // chunk q's bytes (the copy may land first: the phase completes
                        // once both the arrival and the bytes are in)
                        mbar_expect(&full[q % F_SLOTS], FW_BYTES);
                        if (!mbar_wait(&full[q % F_SLOTS], (q / F_SLOTS) & 1)) {
                            ok = false;
                            ++q;
                            break;
                        }
                        const uint32_t w0 = su32(sW + (q % F_SLOTS) * FW_BYTES);
#pragma unroll
                        for (int kk = 0; kk < FK / 16; ++kk) {
                            const uint64_t bd = sdesc(w0 + kk * 2 * FW_LBO, FW_LBO, FW_SBO);
                            const uint32_t ka = (c * (FK / 8) + kk * 2) * 128;
                            umma(d, sdesc(a0 + ka, LBO, FA_SBO), bd, (c | kk) != 0);
                        }
                        // the slot is free for chunk q + S once the MMAs reading it are done
                        umma_commit(&empty[q % F_SLOTS]);
                    }
                    if (!ok) break;
                    umma_commit(&acc[g]);   // the group's accumulator is complete
                }
            }
            if (!ok) *sfail = 1;
            *scons = q;   // chunks whose bytes this CTA has expected
        }
    } else {
        // ---------------- a group of four warps: 128 rows ----------------
        const int g = warp >> 2, r = tid & 127;
        unsigned char *myA = sm + g * FA_BYTES;
        const uint32_t tb = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(g * 256);
        // A tile element (row, k) offset: core matrix (row / 8, k / 8), row % 8 at 16 bytes
        auto a_off = [](int row, int k8) { return (row >> 3) * FA_SBO + k8 * 128 + (row & 7) * 16; };
        unsigned pacc = 0;
        auto wait_acc = [&]() {
            if (!mbar_wait(&acc[g], pacc)) {
                *sfail = 1;
                return false;
            }
            pacc ^= 1u;
            tc_after();
            return true;
        };
        auto hand_off = [&]() {   // A_g holds the next layer's input
            tc_before();
            fence_async_smem();
            mbar_arrive(&act[g]);
        };
        float xn0 = 0.f, xn1 = 0.f, xn2 = 0.f;   // this tile's inputs (0 past the last row)
        {
            const int row = (int)blockIdx.x * 256 + g * 128 + r;
            if (mine > 0 && row < rows) {
                xn0 = x[3 * row];
                xn1 = x[3 * row + 1];
                xn2 = x[3 * row + 2];
            }
        }
        for (int it = 0; it < mine && ok; ++it) {
            const int row = ((int)blockIdx.x + it * (int)gridDim.x) * 256 + g * 128 + r;
            const bool rv = row < rows;
            // ---- layer 1: h1 = relu(W1 x + b1) ----
            {
                const float2 X0 = make_float2(xn0, xn0), X1 = make_float2(xn1, xn1),
                             X2 = make_float2(xn2, xn2);
                // 8 columns per step: W1^T rows and b1 as broadcast float4 reads of shared
                // memory, pairs of columns by packed FP32 FMAs, ReLU fused in the BF16 pack
                const float4 *pw0 = reinterpret_cast<const float4 *>(sP + FP_W1);
                const float4 *pw1 = reinterpret_cast<const float4 *>(sP + FP_W1 + 256);
                const float4 *pw2 = reinterpret_cast<const float4 *>(sP + FP_W1 + 512);
                const float4 *pb = reinterpret_cast<const float4 *>(sP + FP_B1);
#pragma unroll 4
                for (int k8 = 0; k8 < 32; ++k8) {
                    uint4 u;
                    uint32_t *hw = reinterpret_cast<uint32_t *>(&u);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float4 b = pb[k8 * 2 + h], w0 = pw0[k8 * 2 + h],
                                     w1 = pw1[k8 * 2 + h], w2 = pw2[k8 * 2 + h];
                        float2 a = make_float2(b.x, b.y), c = make_float2(b.z, b.w);
                        a = fma2(make_float2(w0.x, w0.y), X0, a);
                        c = fma2(make_float2(w0.z, w0.w), X0, c);
                        a = fma2(make_float2(w1.x, w1.y), X1, a);
                        c = fma2(make_float2(w1.z, w1.w), X1, c);
                        a = fma2(make_float2(w2.x, w2.y), X2, a);
                        c = fma2(make_float2(w2.z, w2.w), X2, c);
                        hw[2 * h] = relu_bf16x2(a);
                        hw[2 * h + 1] = relu_bf16x2(c);
                    }
                    *reinterpret_cast<uint4 *>(myA + a_off(r, k8)) = u;
                }
            }
            // the next tile's inputs, in flight during the two layers
            {
                const int nrow = row + (int)gridDim.x * 256;
                if (it + 1 < mine && nrow < rows) {
                    xn0 = x[3 * nrow];
                    xn1 = x[3 * nrow + 1];
                    xn2 = x[3 * nrow + 2];
                }
            }
            hand_off();
            if (!(ok = wait_acc())) break;
            // ---- epilogue of layer 2: h2 = relu(acc + b2) over h1 ----
            for (int ch = 0; ch < 8; ch += 2) {   // 64 columns per tensor-memory wait
                uint32_t ra[32], rb[32];
                tmem_ld32_issue(tb + ch * 32, ra);
                tmem_ld32_issue(tb + ch * 32 + 32, rb);
                tmem_wait_tied(ra);
                reg_tie(rb);
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const uint32_t *rr = half ? rb : ra;
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        const float4 *b2 = reinterpret_cast<const float4 *>(sP + FP_B2) + (ch + half) * 8 + qq * 2;
                        const float4 p0 = b2[0], p1 = b2[1];
                        const uint32_t *vq = rr + qq * 8;
                        uint4 u;
                        u.x = relu_bf16x2(add2(make_float2(__uint_as_float(vq[0]), __uint_as_float(vq[1])), make_float2(p0.x, p0.y)));
                        u.y = relu_bf16x2(add2(make_float2(__uint_as_float(vq[2]), __uint_as_float(vq[3])), make_float2(p0.z, p0.w)));
                        u.z = relu_bf16x2(add2(make_float2(__uint_as_float(vq[4]), __uint_as_float(vq[5])), make_float2(p1.x, p1.y)));
                        u.w = relu_bf16x2(add2(make_float2(__uint_as_float(vq[6]), __uint_as_float(vq[7])), make_float2(p1.z, p1.w)));
                        *reinterpret_cast<uint4 *>(myA + a_off(r, (ch + half) * 4 + qq)) = u;
                    }
                }
            }
            hand_off();
            if (!(ok = wait_acc())) break;
            // ---- epilogue of layer 3 and the head: y = sigmoid(w4 . relu(acc + b3) + b4) ----
            float2 dot = make_float2(0.f, 0.f);   // even and odd columns
            for (int ch = 0; ch < 8; ch += 2) {   // 64 columns per tensor-memory wait
                uint32_t ra[32], rb[32];
                tmem_ld32_issue(tb + ch * 32, ra);
                tmem_ld32_issue(tb + ch * 32 + 32, rb);
                tmem_wait_tied(ra);
                reg_tie(rb);
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const uint32_t *rr = half ? rb : ra;
#pragma unroll
                    for (int j4 = 0; j4 < 8; ++j4) {
                        const float4 b3 = reinterpret_cast<const float4 *>(sP + FP_B3)[(ch + half) * 8 + j4];
                        const float4 w4 = reinterpret_cast<const float4 *>(sP + FP_W4)[(ch + half) * 8 + j4];
                        float2 a = add2(make_float2(__uint_as_float(rr[4 * j4]), __uint_as_float(rr[4 * j4 + 1])),
                                        make_float2(b3.x, b3.y));
                        float2 c = add2(make_float2(__uint_as_float(rr[4 * j4 + 2]), __uint_as_float(rr[4 * j4 + 3])),
                                        make_float2(b3.z, b3.w));
                        a = make_float2(fmaxf(a.x, 0.f), fmaxf(a.y, 0.f));
                        c = make_float2(fmaxf(c.x, 0.f), fmaxf(c.y, 0.f));
                        dot = fma2(a, make_float2(w4.x, w4.y), dot);
                        dot = fma2(c, make_float2(w4.z, w4.w), dot);
                    }
                }
            }
            if (rv) y[row] = 1.f / (1.f + __expf(-((dot.x + dot.y) + sP[FP_B4])));
        }
    }
    tc_before();
    __syncthreads();
    if (*sfail && tid == 0) {
        atomicExch(&g_mlp_err, TRT_ETIMEOUT);
        // let the producer's copies in flight land (bounded): expect what the MMA thread
        // did not, then wait
        for (int r = *scons; r < *sprod; ++r) {
            mbar_expect(&full[r % F_SLOTS], FW_BYTES);
            mbar_wait(&full[r % F_SLOTS], (r / F_SLOTS) & 1);
        }
    }
    __syncthreads();   // the drain above ends before TMEM is released
    if (warp == 0) {
        tc_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

int g_num_sms = 0;

cudaError_t mlp_fused(int rows, const float *x, const float *P, const bf16 *W, float *y,
                      cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t r = cudaFuncSetAttribute(k_mlp_fused,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, F_SMEM);
        if (r != cudaSuccess) return r;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        attr = true;
    }
    if (reinterpret_cast<uintptr_t>(P) & 15) return cudaErrorMisalignedAddress;   // float4 loads
    // one persistent CTA per SM, no more CTAs than row tiles (a CTA left for a second wave
    // would double the time)
    const int ntiles = (rows + 255) / 256;
    const int grid = std::max(1, std::min(ntiles, g_num_sms > 0 ? g_num_sms : 148));
    k_mlp_fused<<<grid, F_THREADS, F_SMEM, st>>>(rows, x, P, (const bf16 *)(W + 4 * 65536), y);
    return cudaGetLastError();
}

cudaError_t gemm(int M, int N, int K, const bf16 *A, const bf16 *B, const Epi &e,
                 cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaError_t r = cudaFuncSetAttribute(k_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             GEMM_SMEM);
        if (r != cudaSuccess) return r;
        attr = true;
    }
    dim3 grid((M + BM - 1) / BM, N / BN);
    k_gemm<<<grid, 128, GEMM_SMEM, st>>>(M, N, K, A, B, e);
    return cudaGetLastError();
}

// ---- MLP pieces on CUDA cores ----

// h1 = relu(W1 x + b1) per row (FP32), stored BF16 row-major and optionally transposed
__global__ void k_layer1(int R, const float *__restrict__ x, const float *__restrict__ P,
                         bf16 *__restrict__ h1, bf16 *__restrict__ h1T, int ldT)
{
    __shared__ float w[TRT_MLP_HIDDEN * 4];
    for (int i = threadIdx.x; i < TRT_MLP_HIDDEN; i += blockDim.x) {
        w[4 * i + 0] = P[TRT_MLP_W1 + 3 * i + 0];
        w[4 * i + 1] = P[TRT_MLP_W1 + 3 * i + 1];
        w[4 * i + 2] = P[TRT_MLP_W1 + 3 * i + 2];
        w[4 * i + 3] = P[TRT_MLP_B1 + i];
    }
    __syncthreads();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const float x0 = x[3 * r], x1 = x[3 * r + 1], x2 = x[3 * r + 2];
    uint4 *o = reinterpret_cast<uint4 *>(h1 + (size_t)r * TRT_MLP_HIDDEN);
    for (int q = 0; q < TRT_MLP_HIDDEN / 8; ++q) {
        uint4 u;
        bf16 *hb = reinterpret_cast<bf16 *>(&u);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = q * 8 + j;
            float a = w[4 * c + 3];
            a = fmaf(w[4 * c + 0], x0, a);
            a = fmaf(w[4 * c + 1], x1, a);
            a = fmaf(w[4 * c + 2], x2, a);
            hb[j] = __float2bfloat16_rn(fmaxf(a, 0.f));
            if (h1T) h1T[(size_t)c * ldT + r] = hb[j];
        }
        o[q] = u;
    }
}

// out[c] = sum_r a[r][c] * (wr ? wr[r * ws + wo] : 1), c < ncol; a is BF16 or FP32 with row
// stride lda; fixed summation order: 8 row slices per column, then the slices in order
template <typename T>
__global__ void k_colsum(int R, int ncol, const T *__restrict__ a, int lda,
                         const float *__restrict__ wr, int ws, int wo, float *__restrict__ out)
{
    __shared__ float part[8][33];
    const int cl = threadIdx.x & 31, sl = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + cl;
    float s = 0.f;
    if (c < ncol)
        for (int r = sl; r < R; r += 8) {
            const float v = (float)a[(size_t)r * lda + c];
            s = fmaf(v, wr ? wr[(size_t)r * ws + wo] : 1.f, s);
        }
    part[sl][cl] = s;
    __syncthreads();
    if (sl == 0 && c < ncol) {
        float t = 0.f;
        for (int k = 0; k < 8; ++k) t += part[k][cl];
        out[c] = t;
    }
}

// dW1[c][k] = sum_r d1[r][c] x[r][k]: one column sum per (c, k), written at stride 3
__global__ void k_dw1(int R, const float *__restrict__ d1, const float *__restrict__ x,
                      float *__restrict__ g)
{
    __shared__ float part[8][33];
    const int cl = threadIdx.x & 31, sl = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + cl, k = blockIdx.y;
    float s = 0.f;
    for (int r = sl; r < R; r += 8) s = fmaf(d1[(size_t)r * TRT_MLP_HIDDEN + c], x[3 * r + k], s);
    part[sl][cl] = s;
    __syncthreads();
    if (sl == 0) {
        float t = 0.f;
        for (int q = 0; q < 8; ++q) t += part[q][cl];
        g[TRT_MLP_W1 + 3 * c + k] = t;
    }
}

// W2, W3 (BF16), their transposes and their streaming images (the 16 KB chunks of the
// fused kernel, each laid out as it lands in shared memory) from the FP32 parameters
__global__ void k_refresh(const float *__restrict__ P, bf16 *__restrict__ w16)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;   // 2 x 65536
    if (idx >= 2 * 65536) return;
    const int layer = idx >> 16, o = (idx >> 8) & 255, i = idx & 255;
    const float v = P[(layer ? TRT_MLP_W3 : TRT_MLP_W2) + o * 256 + i];
    const bf16 b = __float2bfloat16_rn(v);
    w16[layer * 65536 + o * 256 + i] = b;                 // W [out][in]
    w16[(2 + layer) * 65536 + i * 256 + o] = b;           // W^T [in][out]
    const int c = i >> 5, kg = (i >> 3) & 3, j = i & 7;   // chunk, K group, element
    w16[(4 + layer) * 65536 + c * 8192 + kg * 2048 + o * 8 + j] = b;
}

__global__ void k_adam(int n, float *__restrict__ P, const float *__restrict__ g,
                       float *__restrict__ m, float *__restrict__ v, float lr, float b1,
                       float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_features(int nx, int G, const double *__restrict__ T,
                           const double *__restrict__ sigE, const double *__restrict__ Eg,
                           const double *__restrict__ Ecell, float *__restrict__ x)
{
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)G * nx) return;
    const int i = (int)(idx % nx);
    const double t = fmax(T[i], 1e-30);
    const double s = fmax(sigE[idx], 1e-300);
    const double r = fmax(Eg[idx], 1e-300) / fmax(Ecell[i], 1e-300);
    x[3 * idx + 0] = (float)((log(t) + 3.5) * 0.5);
    x[3 * idx + 1] = (float)((log(s) - 10.0) * 0.1);
    x[3 * idx + 2] = (float)((log(r) + 10.0) * 0.1);
}

inline size_t al256(size_t x) { return (x + 255) / 256 * 256; }

struct Scratch {
    bf16 *h1, *h1T, *h2, *h2T, *h3, *d3, *d3T, *d2, *d2T;
    float *d1, *dz, *sq;
    size_t bytes;
};

Scratch carve_scratch(void *base, int R, int training)
{
    Scratch s{};
    char *p = reinterpret_cast<char *>(base);
    size_t o = 0;
    const size_t hb = al256((size_t)R * TRT_MLP_HIDDEN * sizeof(bf16));
    auto take = [&](size_t n) { char *q = p ? p + o : nullptr; o += n; return q; };
    s.h1 = reinterpret_cast<bf16 *>(take(hb));
    s.h2 = reinterpret_cast<bf16 *>(take(hb));
    if (training) {
        s.h1T = reinterpret_cast<bf16 *>(take(hb));
        s.h2T = reinterpret_cast<bf16 *>(take(hb));
        s.h3 = reinterpret_cast<bf16 *>(take(hb));
        s.d3 = reinterpret_cast<bf16 *>(take(hb));
        s.d3T = reinterpret_cast<bf16 *>(take(hb));
        s.d2 = reinterpret_cast<bf16 *>(take(hb));
        s.d2T = reinterpret_cast<bf16 *>(take(hb));
        s.d1 = reinterpret_cast<float *>(take(al256((size_t)R * TRT_MLP_HIDDEN * sizeof(float))));
        s.dz = reinterpret_cast<float *>(take(al256((size_t)R * sizeof(float))));
        s.sq = reinterpret_cast<float *>(take(al256((size_t)R * sizeof(float))));
    }
    s.bytes = o;
    return s;
}

bool al16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

}  // namespace trt

using namespace trt;

extern "C" {

int trt_gemm_bf16(int M, int N, int K, const void *A, const void *B, const float *bias, int relu,
                  const void *mask, float *out32, void *out16, void *out16T, int ldT,
                  void *stream)
{
    if (M < 1 || N < BN || N % BN || K < BK || K % BK || !A || !B) return TRT_EINVAL;
    if (out16T && ldT < M) return TRT_EINVAL;
    if (!al16(A) || !al16(B) || !al16(mask) || !al16(out32) || !al16(out16)) return TRT_EINVAL;
    Epi e{};
    e.bias = bias;
    e.relu = relu;
    e.mask = reinterpret_cast<const bf16 *>(mask);
    e.out32 = out32;
    e.out16 = reinterpret_cast<bf16 *>(out16);
    e.out16T = reinterpret_cast<bf16 *>(out16T);
    e.ldT = ldT;
    cudaError_t r = gemm(M, N, K, reinterpret_cast<const bf16 *>(A),
                         reinterpret_cast<const bf16 *>(B), e, reinterpret_cast<cudaStream_t>(stream));
    return r == cudaSuccess ? TRT_OK : TRT_ECUDA;
}

size_t trt_mlp_scratch_bytes(int rows, int training)
{
    if (rows < 1) return 0;
    return carve_scratch(nullptr, rows, training).bytes;
}

int trt_mlp_refresh(const float *params, void *w16, void *stream)
{
    if (!params || !w16) return TRT_EINVAL;
    k_refresh<<<512, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        params, reinterpret_cast<bf16 *>(w16));
    return cudaGetLastError() == cudaSuccess ? TRT_OK : TRT_ECUDA;
}

int trt_mlp_forward_fused(int rows, const float *x, const float *params, const void *w16,
                          float *y, void *stream)
{
    if (rows < 1 || !x || !params || !w16 || !y) return TRT_EINVAL;
    if (reinterpret_cast<uintptr_t>(params) & 15) return TRT_EINVAL;
    return mlp_fused(rows, x, params, reinterpret_cast<const bf16 *>(w16), y,
                     reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
               ? TRT_OK
               : TRT_ECUDA;
}

int trt_mlp_forward(int rows, const float *x, const float *params, const void *w16,
                    void *scratch, size_t scratch_bytes, float *y, void *stream)
{
    if (rows < 1 || !x || !params || !w16 || !scratch || !y) return TRT_EINVAL;
    Scratch s = carve_scratch(scratch, rows, 0);
    if (scratch_bytes < s.bytes || !al16(scratch)) return TRT_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const bf16 *W = reinterpret_cast<const bf16 *>(w16);
    k_layer1<<<(rows + 127) / 128, 128, 0, st>>>(rows, x, params, s.h1, nullptr, 0);
    if (cudaGetLastError() != cudaSuccess) return TRT_ECUDA;
    Epi e2{};
    e2.bias = params + TRT_MLP_B2;
    e2.relu = 1;
    e2.out16 = s.h2;
    if (gemm(rows, 256, 256, s.h1, W, e2, st) != cudaSuccess) return TRT_ECUDA;
    Epi e3{};
    e3.bias = params + TRT_MLP_B3;
    e3.relu = 1;
    e3.head_w = params + TRT_MLP_W4;
    e3.head_b = params + TRT_MLP_B4;
    e3.head_y = y;
    if (gemm(rows, 256, 256, s.h2, W + 65536, e3, st) != cudaSuccess) return TRT_ECUDA;
    return TRT_OK;
}

int trt_mlp_grad(int rows, const float *x, const float *target, const float *params,
                 const void *w16, void *scratch, size_t scratch_bytes, float *grad, float *loss,
                 void *stream)
{
    if (rows < 128 || rows % 128 || !x || !target || !params || !w16 || !scratch || !grad ||
        !loss)
        return TRT_EINVAL;
    Scratch s = carve_scratch(scratch, rows, 1);
    if (scratch_bytes < s.bytes || !al16(scratch)) return TRT_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const bf16 *W = reinterpret_cast<const bf16 *>(w16);
    const bf16 *W2 = W, *W3 = W + 65536, *W2T = W + 2 * 65536, *W3T = W + 3 * 65536;
#define CKL(x)                                            \
    do {                                                  \
        if ((x) != cudaSuccess) return TRT_ECUDA;         \
    } while (0)
    k_layer1<<<(rows + 127) / 128, 128, 0, st>>>(rows, x, params, s.h1, s.h1T, rows);
    CKL(cudaGetLastError());
    Epi e2{};
    e2.bias = params + TRT_MLP_B2;
    e2.relu = 1;
    e2.out16 = s.h2;
    e2.out16T = s.h2T;
    e2.ldT = rows;
    CKL(gemm(rows, 256, 256, s.h1, W2, e2, st));
    Epi e3{};
    e3.bias = params + TRT_MLP_B3;
    e3.relu = 1;
    e3.out16 = s.h3;
    e3.head_w = params + TRT_MLP_W4;
    e3.head_b = params + TRT_MLP_B4;
    e3.target = target;
    e3.scale = 2.f / rows;
    e3.dz = s.dz;
    e3.sq = s.sq;
    e3.dact16 = s.d3;
    e3.dact16T = s.d3T;
    e3.ldT = rows;
    CKL(gemm(rows, 256, 256, s.h2, W3, e3, st));
    // d2 = (d3 W3) [h2 > 0];  dW3 = d3^T h2
    Epi eb{};
    eb.mask = s.h2;
    eb.out16 = s.d2;
    eb.out16T = s.d2T;
    eb.ldT = rows;
    CKL(gemm(rows, 256, 256, s.d3, W3T, eb, st));
    Epi ew{};
    ew.out32 = grad + TRT_MLP_W3;
    CKL(gemm(256, 256, rows, s.d3T, s.h2T, ew, st));
    // d1 = (d2 W2) [h1 > 0];  dW2 = d2^T h1
    Epi e1{};
    e1.mask = s.h1;
    e1.out32 = s.d1;
    CKL(gemm(rows, 256, 256, s.d2, W2T, e1, st));
    Epi ew2{};
    ew2.out32 = grad + TRT_MLP_W2;
    CKL(gemm(256, 256, rows, s.d2T, s.h1T, ew2, st));
    // biases, W1, w4, b4, loss: fixed-order column sums over the rows
    k_colsum<bf16><<<8, 256, 0, st>>>(rows, 256, s.d3, 256, nullptr, 0, 0, grad + TRT_MLP_B3);
    k_colsum<bf16><<<8, 256, 0, st>>>(rows, 256, s.d2, 256, nullptr, 0, 0, grad + TRT_MLP_B2);
    k_colsum<float><<<8, 256, 0, st>>>(rows, 256, s.d1, 256, nullptr, 0, 0, grad + TRT_MLP_B1);
    k_colsum<bf16><<<8, 256, 0, st>>>(rows, 256, s.h3, 256, s.dz, 1, 0, grad + TRT_MLP_W4);
    k_colsum<float><<<1, 256, 0, st>>>(rows, 1, s.dz, 1, nullptr, 0, 0, grad + TRT_MLP_B4);
    k_colsum<float><<<1, 256, 0, st>>>(rows, 1, s.sq, 1, nullptr, 0, 0, loss);
    k_dw1<<<dim3(8, 3), 256, 0, st>>>(rows, s.d1, x, grad);
    CKL(cudaGetLastError());
#undef CKL
    return TRT_OK;
}

int trt_mlp_adam(float *params, const float *grad, float *m, float *v, int t, float lr,
                 float beta1, float beta2, float eps, void *w16, void *stream)
{
    if (!params || !grad || !m || !v || t < 1 || !w16) return TRT_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
    k_adam<<<(TRT_MLP_NPARAM + 255) / 256, 256, 0, st>>>(TRT_MLP_NPARAM, params, grad, m, v, lr,
                                                         beta1, beta2, eps, c1, c2);
    if (cudaGetLastError() != cudaSuccess) return TRT_ECUDA;
    return trt_mlp_refresh(params, w16, stream);
}

int trt_mlp_features(int nx, int G, const double *T, const double *sigE, const double *Eg,
                     const double *E, float *x, void *stream)
{
    if (nx < 1 || G < 1 || !T || !sigE || !Eg || !E || !x) return TRT_EINVAL;
    const long n = (long)G * nx;
    k_features<<<(unsigned)((n + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        nx, G, T, sigE, Eg, E, x);
    return cudaGetLastError() == cudaSuccess ? TRT_OK : TRT_ECUDA;
}

int trt_mlp_status(void)
{
    int v = 0, zero = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return TRT_ECUDA;
    if (cudaMemcpyFromSymbol(&v, g_mlp_err, sizeof(int)) != cudaSuccess) return TRT_ECUDA;
    if (cudaMemcpyToSymbol(g_mlp_err, &zero, sizeof(int)) != cudaSuccess) return TRT_ECUDA;
    return v;
}

}  // extern "C"
