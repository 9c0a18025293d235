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

#ifdef __cplusplus
}
#endif

#endif /* FK_MLP_H */
