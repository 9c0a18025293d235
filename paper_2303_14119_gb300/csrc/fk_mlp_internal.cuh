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

// nullptr if the shape is supported, else the reason
const char* gemm_shape_error(const GemmArgs& g);
cudaError_t launch_gemm(const GemmArgs& g, int epi, cudaStream_t s);

}  // namespace fk
