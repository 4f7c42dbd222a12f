/*
 * mlp.h -- C ABI of the surrogate network (libmlp) that pre-screens GA
 * candidates before the full simulator evaluates them.
 *
 * The paper evaluates every candidate with the simulator ("The Main GA Loop",
 * Eq. final_fit_fun); this library adds a learned pre-screen on top of that
 * loop.  Network: 45 protocol features (15 fraction slots x (dose, wait, mask),
 * zero-padded to 48) -> 256 -> 256 -> 256 -> 1, GELU (erf form) after every
 * hidden layer, trained with mean squared error and Adam.  Weights are FP32
 * masters with BF16 copies; every matrix product runs on the tensor cores
 * (tcgen05) with BF16 operands and FP32 accumulation.
 *
 * Conventions as in sim.h: the caller owns all memory (one device workspace,
 * borrowed for the context's lifetime), work is enqueued on the given stream,
 * calls marked "synchronises" report device-side errors.  Return values are
 * sim_status codes (0 ok, -1 bad argument, -2 workspace too small, -3 CUDA
 * error, -4 a bounded device wait timed out).
 * Batch sizes must be multiples of 128 and at most the context's batch_max.
 */
#ifndef GPUGA_MLP_H
#define GPUGA_MLP_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { MLP_IN = 45, MLP_IN_PAD = 48, MLP_HIDDEN = 256 };

typedef struct mlp_ctx mlp_ctx;

/* Number of FP32 parameters, in the order W1 (256 x 48, row-major, columns
 * 45..47 unused), b1, W2 (256 x 256), b2, W3, b3, w4 (256), b4. */
int mlp_num_params(void);

/* Device workspace for batches of up to batch_max rows (multiple of 128). */
int mlp_workspace_size(int batch_max, size_t* bytes);

/* Create a network with weights drawn from a scaled uniform (He-style fan-in
 * scaling, seeded counter-based generator on the host), Adam moments zero. */
int mlp_create(int batch_max, uint64_t seed, void* d_workspace, size_t bytes, void* cuda_stream, mlp_ctx** out);

/* y[B] (device, FP32) = network(X[B x 45]) (device, FP32, row-major). */
int mlp_forward(mlp_ctx* ctx, const float* d_X, int B, float* d_y);

/* One Adam step on the mean squared error between network(X) and targets t[B]
 * (device, FP32); *loss (host, may be NULL) receives the loss before the step
 * (synchronises when loss != NULL). */
int mlp_train_step(mlp_ctx* ctx, const float* d_X, const float* d_t, int B, float lr, float* loss);

/* Gradient of the loss with respect to every parameter (device, FP32, the
 * order of mlp_num_params) without updating the weights; *loss as above. */
int mlp_gradients(mlp_ctx* ctx, const float* d_X, const float* d_t, int B, float* d_grad, float* loss);

/* Copy the FP32 parameters to / from host memory (mlp_num_params floats).
 * Setting them also refreshes the BF16 copies and zeroes the Adam moments.
 * Synchronises. */
int mlp_get_params(mlp_ctx* ctx, float* host);
int mlp_set_params(mlp_ctx* ctx, const float* host);

/* C[M x N] (device FP32) = A[M x K] * B[N x K]^T (device BF16, row-major)
 * on the tensor cores, operands staged by TMA; M a multiple of 128, N a
 * multiple of 16 up to 256, K a multiple of 16, d_A, d_B and d_C 16-byte
 * aligned (-1 otherwise).  d_status (device u32) is set non-zero if a bounded wait
 * timed out.  Asynchronous. */
int mlp_gemm_bf16(const void* d_A, const void* d_B, float* d_C, int M, int N, int K, uint32_t* d_status,
                  void* cuda_stream);

/* Failure-path probe (no counterpart in the paper): one CTA waits on an
 * mbarrier that nothing arrives at, polling at most spin_limit times (1 ..
 * 2^26), and then writes 1 to *d_status (device u32) exactly as a timed-out
 * GEMM wait would.  Lets callers and tests check that a device-side timeout is
 * reported and leaves the context usable.  Asynchronous. */
int mlp_wait_probe(uint32_t spin_limit, uint32_t* d_status, void* cuda_stream);

void mlp_destroy(mlp_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
