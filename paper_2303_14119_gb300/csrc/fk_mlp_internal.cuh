// Internal declarations of the surrogate's dense-layer kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fk {

enum GemmEpilogue {
  kEpiF32 = 0,       // C = acc (+ bias)                          FP32 [M][N]
  kEpiBiasGelu = 1,  // C = z = acc + bias (FP32); H = gelu(z) (bf16), Ht = H^T
  kEpiGeluBack = 2,  // H = acc * gelu'(Zin) (bf16), Ht = H^T
};

// C = A * B^T: A [M][lda] and B [N][ldb] bf16 (bit patterns), K-major.
struct GemmArgs {
  const uint16_t* A;
  long long lda;
  const uint16_t* B;
  long long ldb;
  int M, N, K;
  float* C;
  long long ldc;
  const float* bias;  // [N] or null
  uint16_t* H;        // bf16 output [M][ldh]
  long long ldh;
  uint16_t* Ht;       // bf16 transposed output [N][ldht] (or null)
  long long ldht;
  const float* Zin;   // FP32 pre-activation [M][ldz] (kEpiGeluBack)
  long long ldz;
  int m_valid;        // rows >= m_valid write zeros to H / Ht
  int* err;           // set to 1 if a bounded wait ran out
};

// Elementwise and reduction kernels of training and inference.
// Rows [0, n) of the gathered batch come from samples idx[r] of the data
// set (FP32 [*][n_in]); rows >= n are zero.  X [bp][in_p] and its
// transpose Xt [in_p][bp] in bf16; T [bp][out_p] FP32 (when t_src is set).
cudaError_t launch_gather(const float* x_src, const float* t_src, const int* idx, int n, int bp,
                          int n_in, int in_p, int n_out, int out_p, uint16_t* X, uint16_t* Xt,
                          float* T, cudaStream_t s);
// dY = 2 w (Y - T) / n_total for rows < n (bf16, both layouts), zero
// elsewhere; loss_rows[r] = sum_o w_o (Y - T)^2 (FP64, rows < n).
cudaError_t launch_loss_grad(const float* Y, const float* T, const float* w, int n, int bp,
                             int out_p, double inv_n, uint16_t* dY, uint16_t* dYt,
                             double* loss_rows, cudaStream_t s);
// out[r] = sum over columns [0, n) of the bf16 row r of M [rows][ld] (FP32,
// fixed order).
cudaError_t launch_row_sums(const uint16_t* M, long long ld, int rows, int n, float* out,
                            cudaStream_t s);
// *acc += scale * sum_{r < n} loss_rows[r] (one block, fixed order)
cudaError_t launch_loss_reduce(const double* loss_rows, int n, double scale, double* acc,
                               cudaStream_t s);
// Adam on count FP32 parameters (bias-corrected step t >= 1)
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, long long count, float lr,
                        float b1, float b2, float eps, int t, cudaStream_t s);
// bf16 copies of a layer's FP32 weights W [N][K]: Wb [N][K] and Wt [K][N]
cudaError_t launch_pack_weights(const float* W, int N, int K, uint16_t* Wb, uint16_t* Wt,
                                cudaStream_t s);

// nullptr if the shape is supported, else the reason
const char* gemm_shape_error(const GemmArgs& g);
cudaError_t launch_gemm(const GemmArgs& g, int epi, cudaStream_t s);

}  // namespace fk
