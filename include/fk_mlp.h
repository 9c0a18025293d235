/*
 * fk_mlp.h -- C ABI of the surface-charge surrogate's tensor-core kernels.
 *
 * The surrogate is a small multilayer perceptron that maps the parameters
 * of a run of the 1D2V flashover model (Sun et al., arXiv 2303.14119: the
 * applied field E_y of Sec. 2, the SEE parameters delta_max, A_max and T_se
 * of Eqs. 8-15, the injected current J of Eq. 7 and the gap h_max) to the
 * run's surface-charge history sigma(t) (Eq. 18) and its saturation time
 * (the convergence test of Sec. 2).  The paper has no surrogate; the
 * network's dense layers run on GB300's tensor cores through the calls
 * declared here.  Conventions as in fk.h: status codes, no aborts, device
 * memory owned by whoever allocated it, fk_last_error(NULL) for messages of
 * calls without a handle.
 */
#ifndef FK_MLP_H
#define FK_MLP_H

#include <stdint.h>

#include "fk.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Dense-layer primitive: C = A * B^T on the tensor cores (tcgen05), bf16
 * operands, FP32 accumulation, FP32 result.
 *   A: device, bf16 bit patterns, [M][lda] row-major (K contiguous);
 *   B: device, bf16, [N][ldb] row-major (K contiguous);
 *   C: device, FP32, [M][ldc].
 * Requirements: 1 <= N <= 256, K a multiple of 16, lda and ldb multiples of
 * 8 and >= K, ldc >= N, A and B 16-byte aligned; any M >= 1.  err_dev: a
 * device int the kernel sets to 1 if a bounded internal wait ran out (the
 * result is then undefined); it is never cleared by the call.
 * Stream-ordered and asynchronous on cuda_stream (NULL = legacy default).
 * Errors: FK_EINVAL for a shape or pointer outside the rules, FK_ECUDA if
 * the launch fails. */
fk_status fk_gemm_bf16_tn(const void *A, int64_t lda, const void *B, int64_t ldb, float *C,
                          int64_t ldc, int32_t M, int32_t N, int32_t K, int32_t *err_dev,
                          void *cuda_stream);

/* ---- The network --------------------------------------------------------
 * n_in inputs -> depth hidden layers of `width` units with GELU (exact erf
 * form) -> n_out linear outputs.  Parameters are FP32 masters, one flat
 * vector layer by layer: W [out][in] row-major, then b [out].  Every matrix
 * product runs on the tensor cores with bf16 operands (inputs, weights,
 * hidden activations and back-propagated gradients rounded to bf16, round
 * to nearest even) and FP32 accumulation; biases, pre-activations, outputs,
 * gradients and the Adam state stay FP32.  Loss: (1/n) sum over samples and
 * outputs of w_o (y - t)^2 with per-output weights w (NULL = all 1). */
typedef struct fk_mlp fk_mlp;

typedef struct {
  int32_t n_in;      /* 1..256 */
  int32_t width;     /* multiple of 16, 16..256 */
  int32_t depth;     /* hidden layers, 1..32 */
  int32_t n_out;     /* 1..256 */
  int32_t max_batch; /* samples per forward / gradient call and per training batch, 1..2^20 */
  int32_t device;    /* CUDA device ordinal */
} fk_mlp_desc;

/* Create a network with all parameters zero.  cuda_stream: stream for its
 * work, or NULL for one it owns.  FK_EINVAL for a bad description. */
fk_status fk_mlp_create(const fk_mlp_desc *desc, void *cuda_stream, fk_mlp **out);
fk_status fk_mlp_destroy(fk_mlp *mlp);

/* Number of parameters of the flat vector. */
fk_status fk_mlp_param_count(const fk_mlp *mlp, int64_t *count);

/* Copy the parameters in (host FP32, finite; resets the Adam state) or out. */
fk_status fk_mlp_set_params(fk_mlp *mlp, const float *params);
fk_status fk_mlp_get_params(fk_mlp *mlp, float *params);

/* y[n][n_out] = network(x[n][n_in]) for any n >= 0 (host FP32 arrays,
 * processed max_batch rows at a time; synchronises). */
fk_status fk_mlp_forward(fk_mlp *mlp, const float *x, int64_t n, float *y);

/* Loss and its gradient with respect to the parameters (flat layout, host
 * FP32; grad may be NULL) on n <= max_batch samples x[n][n_in] with targets
 * t[n][n_out] and output weights w[n_out] (NULL = 1).  Synchronises. */
fk_status fk_mlp_loss_grad(fk_mlp *mlp, const float *x, const float *t, const float *w,
                           int64_t n, double *loss, float *grad);

/* Adam training (beta1 0.9, beta2 0.999, eps 1e-8, constant learning rate
 * lr) on a data set of n samples copied to the device: `epochs` passes, each
 * over the samples in an order drawn from seed and the epoch (SplitMix64
 * Fisher-Yates), in batches of `batch` <= max_batch.  epoch_loss[epochs]
 * (may be NULL) receives each epoch's mean training loss over the batches
 * as they were met.  Deterministic for equal inputs.  Continues the Adam
 * state of earlier calls (fk_mlp_set_params resets it). */
fk_status fk_mlp_train(fk_mlp *mlp, const float *x, const float *t, const float *w, int64_t n,
                       int32_t batch, int32_t epochs, float lr, uint64_t seed,
                       double *epoch_loss);

/* Text of the last error on this network; NULL: errors of fk_mlp_create. */
const char *fk_mlp_last_error(const fk_mlp *mlp);

#ifdef __cplusplus
}
#endif

#endif /* FK_MLP_H */
