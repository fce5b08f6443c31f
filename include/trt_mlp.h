/*
 * trt_mlp.h -- C ABI of the learned closure: a small MLP that predicts the group QD
 * factors f_g (eq. f_g) at the start of a time step, and the BF16 tensor-core GEMM it is
 * built on.
 *
 * The paper has no learned component.  Algorithm 3 starts every time step with an s = 0
 * low-order phase that uses the previous step's QD factors f_g^{j-1}; here those factors
 * may instead come from the MLP (a warm start).  The transport sweep still closes the
 * iteration, so the converged answer is the plain method's to within the iteration
 * tolerance; the MLP only changes where the iteration starts.
 *
 * Network (per (cell i, group g) row):
 *   x = (x0, x1, x2) = ((ln T_i + 3.5)/2, (ln sigma_E,g,i - 10)/10,
 *                       (ln(E_g,i / E_i) + 10)/10)                         (FP32)
 *   h1 = relu(W1 x + b1)            256, FP32 arithmetic, stored BF16
 *   h2 = relu(W2 h1 + b2)           256, BF16 x BF16 -> FP32 on tensor cores, stored BF16
 *   h3 = relu(W3 h2 + b3)           256, same
 *   y  = sigmoid(w4 . h3 + b4)      f_g,i in (0, 1), FP32
 * Parameters are one FP32 vector (the master copy, caller-owned device memory) at the
 * offsets below; W are row-major [out][in].  The tensor-core layers read BF16 copies
 * (W2, W3 and their transposes) made by trt_mlp_refresh.
 *
 * Ownership: every pointer is caller-owned device memory; nothing is allocated; all work
 * is enqueued on `stream` (cudaStream_t as void*, NULL = legacy stream) and the calls
 * return without synchronising.  Return codes are those of trt.h (TRT_EINVAL for bad
 * sizes or NULL pointers, checked before anything is enqueued; TRT_ECUDA for a launch
 * error).  A kernel whose wait on a tensor-core completion exceeds one second records
 * TRT_ETIMEOUT in the error word read by trt_mlp_status.
 */
#ifndef TRT_MLP_H
#define TRT_MLP_H

#include <stddef.h>
#include "trt.h"   /* status codes */

#ifdef __cplusplus
extern "C" {
#endif

#define TRT_MLP_HIDDEN 256
#define TRT_MLP_W1 0        /* [256][3]                  */
#define TRT_MLP_B1 768      /* [256]                     */
#define TRT_MLP_W2 1024     /* [256][256]                */
#define TRT_MLP_B2 66560    /* [256]                     */
#define TRT_MLP_W3 66816    /* [256][256]                */
#define TRT_MLP_B3 132352   /* [256]                     */
#define TRT_MLP_W4 132608   /* [256]                     */
#define TRT_MLP_B4 132864   /* [1]                       */
#define TRT_MLP_NPARAM 132868
/* BF16 copies made by trt_mlp_refresh, 65536 each: W2, W3, W2^T, W3^T, and W2, W3 again
 * in the order trt_mlp_forward_fused streams them (per 32-wide K chunk c, 8-wide K group
 * kg and output n: element (n, k = 32 c + 8 kg + j) at 8192 c + 2048 kg + 8 n + j) */
#define TRT_MLP_W16_ELEMS (6 * 65536)

/* C = A B^T on the tensor cores (tcgen05.mma kind::f16, BF16 inputs, FP32 accumulation
 * in tensor memory), with a fused epilogue applied per element:
 *   a = C[m][n] + bias[n]  (bias may be NULL);  relu: a = max(a, 0);
 *   mask (BF16 [M][N], may be NULL): a = (mask[m][n] > 0) ? a : 0;
 *   out32 [M][N] FP32, out16 [M][N] BF16, out16T [N][ldT] BF16 (transposed) -- each may
 *   be NULL.
 * A is BF16 [M][K] row-major, B is BF16 [N][K] row-major (both K-contiguous).  M >= 1,
 * N a multiple of 256, K a multiple of 64; A, B, mask and the outputs 16-byte aligned;
 * ldT >= M. */
int trt_gemm_bf16(int M, int N, int K, const void *A, const void *B, const float *bias,
                  int relu, const void *mask, float *out32, void *out16, void *out16T,
                  int ldT, void *stream);

/* Device scratch (bytes) for trt_mlp_forward / trt_mlp_grad over `rows` rows. */
size_t trt_mlp_scratch_bytes(int rows, int training);

/* BF16 copies of W2 and W3 (their transposes and their streaming images) from the FP32
 * parameters. */
int trt_mlp_refresh(const float *params, void *w16, void *stream);

/* Inference: x [rows][3] FP32 -> y [rows] FP32 (sigmoid outputs).  rows >= 1. */
int trt_mlp_forward(int rows, const float *x, const float *params, const void *w16,
                    void *scratch, size_t scratch_bytes, float *y, void *stream);

/* Inference in one persistent kernel (one CTA per SM in clusters of two, 256 rows per
 * iteration as two 128-row groups half a period apart, both hidden layers on the tensor
 * cores with the activations kept in shared memory and the weights streamed in 32-wide K
 * chunks from the image trt_mlp_refresh keeps in w16); same arithmetic and result as
 * trt_mlp_forward up to the order of the FP32 accumulation.  Needs no scratch.  params must be 16-byte aligned (the
 * biases and the first and last layers' weights are read as float4): TRT_EINVAL otherwise. */
int trt_mlp_forward_fused(int rows, const float *x, const float *params, const void *w16,
                          float *y, void *stream);

/* Loss L = (1/rows) sum_r (y_r - t_r)^2 and its gradient with respect to every parameter
 * (grad [TRT_MLP_NPARAM] FP32, overwritten; *loss a device float).  rows a multiple of
 * 128.  The backward pass rounds the layer gradients to BF16 before each tensor-core
 * product, as the forward pass rounds the activations. */
int trt_mlp_grad(int rows, const float *x, const float *target, const float *params,
                 const void *w16, void *scratch, size_t scratch_bytes, float *grad,
                 float *loss, void *stream);

/* One Adam step (Kingma & Ba, bias-corrected, step number t >= 1) on the FP32
 * parameters, then trt_mlp_refresh. */
int trt_mlp_adam(float *params, const float *grad, float *m, float *v, int t, float lr,
                 float beta1, float beta2, float eps, void *w16, void *stream);

/* Closure features of the rows (g, i), g-major ([G][nx], the layout of f_g):
 * T [nx], sigE [G][nx], Eg [G][nx], E = sum_g E_g [nx] (FP64) -> x [G*nx][3] FP32. */
int trt_mlp_features(int nx, int G, const double *T, const double *sigE, const double *Eg,
                     const double *E, float *x, void *stream);

/* Error word of the MLP kernels on the current device: 0, or TRT_ETIMEOUT after a wait
 * on a tensor-core completion gave up (the kernel then skipped its remaining work and
 * released its tensor memory).  Synchronises the device; clears the word. */
int trt_mlp_status(void);

#ifdef __cplusplus
}
#endif
#endif
