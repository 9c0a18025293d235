// Dense layers of the surface-charge surrogate on the tensor cores:
// C = A * B^T with bf16 A [M][K] and B [N][K] (both K-major), FP32
// accumulation in tensor memory (tcgen05.mma, operands in shared memory),
// and the epilogues the surrogate's training needs (bias, GELU and its
// derivative, bf16 copies in both layouts).
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include <string>

#include "fk_internal.cuh"
#include "fk_mlp.h"
#include "fk_mlp_internal.cuh"
#include "fk_tc.cuh"

namespace fk {

namespace {

constexpr int kMTile = 128;   // rows per CTA (one MMA M)
constexpr int kNTile = 64;    // columns per CTA (one MMA N at most)
constexpr int kNMax = 256;    // the largest N the entry points accept
constexpr int kKChunk = 64;   // K per stage (4 MMAs of K = 16)
constexpr int kGemmStages = 4;     // stages of the ring: K chunks in flight
constexpr int kGemmThreads = 128;  // 4 warps: one per 32-lane slice of tensor memory
constexpr int kCoreBytes = 128;    // one 8 x 16-byte core matrix
// a tile: [rows/8 row groups][kKChunk/8 K groups] core matrices
constexpr int kLboBytes = kCoreBytes;                        // next core matrix along K
constexpr int kSboBytes = (kKChunk / 8) * kCoreBytes;        // next 8-row group
constexpr int kATileBytes = kMTile * kKChunk * 2;            // 16 KB
constexpr int kBTileBytes = kNTile * kKChunk * 2;            // 8 KB
constexpr int kGemmStageBytes = kATileBytes + kBTileBytes;   // 24 KB
// dynamic shared memory per CTA: the ring (two CTAs fit on an SM, with 2 x
// 64 of its 512 tensor-memory columns)
constexpr int kGemmSmem = kGemmStages * kGemmStageBytes;

__device__ __forceinline__ uint16_t f32_to_bf16(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
// GELU with the exact (erf) form and its derivative
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
         z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// 16-byte asynchronous copy global -> shared (cp.async); zeros when !full
// (no byte of src is read then; src stays a valid address)
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool full) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc::smem_u32(dst)), "l"(src),
               "r"(full ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
// wait until at most n of this thread's copy groups are still pending
__device__ __forceinline__ void cp_async_wait(int n) {
  switch (n) {
    case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
  }
}

// Queue the copy of rows [r0, r0 + rows) x K columns [k0, k0 + kKChunk) of a
// K-major bf16 matrix into the core-matrix layout; zeros outside
// [0, nrows) x [0, K).
__device__ __forceinline__ void stage_tile(unsigned char* dst, const uint16_t* src, long long ld,
                                           int r0, int rows, int nrows, int k0, int K) {
  const int vecs = rows * (kKChunk / 8);
  for (int v = threadIdx.x; v < vecs; v += kGemmThreads) {
    const int r = v / (kKChunk / 8), kc = v - (v / (kKChunk / 8)) * (kKChunk / 8);
    const int gr = r0 + r, gk = k0 + kc * 8;
    const bool in = gr < nrows && gk < K;
    cp_async16(dst + ((r >> 3) * (kKChunk / 8) + kc) * kCoreBytes + (r & 7) * 16,
               in ? src + (long long)gr * ld + gk : src, in);
  }
}

// One CTA: rows [m0, m0 + 128) x columns [n0, n0 + Nc) of C.  The K chunks
// stream through a ring of kGemmStages shared-memory stages: every thread
// queues its part of a chunk's copies (cp.async) up to kGemmStages chunks
// ahead; once a chunk has landed, one thread issues its four MMAs and
// commits them to the stage's mbarrier, whose phase frees the stage for
// the chunk kGemmStages later.  Each output element sums its K terms in
// the same order whatever the grid, so results are deterministic.
template <int EPI>
__global__ void __launch_bounds__(kGemmThreads) gemm_tn_kernel(const __grid_constant__ GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar[kGemmStages];
  __shared__ uint32_t s_taddr;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kMTile;
  const int n0 = blockIdx.y * kNTile;
  const int N = g.N;
  const int Nc = min(kNTile, (N + 15) / 16 * 16 - n0);  // this CTA's columns, a multiple of 16
  const uint32_t ncols = Nc <= 32 ? 32u : 64u;
  if (warp == 0) {
    tc::tmem_alloc(&s_taddr, ncols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int q = 0; q < kGemmStages; q++) tc::mbar_init(&bar[q], 1);
    tc::fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = s_taddr;
  const uint32_t idesc = tc::idesc_bf16_f32(kMTile, Nc);
  const int nch = (g.K + kKChunk - 1) / kKChunk;
  auto stage = [&](int c) {
    unsigned char* sA = smem + (c % kGemmStages) * kGemmStageBytes;
    stage_tile(sA, g.A, g.lda, m0, kMTile, g.M, c * kKChunk, g.K);
    stage_tile(sA + kATileBytes, g.B, g.ldb, n0, Nc, N, c * kKChunk, g.K);
    cp_async_commit();
  };
  for (int c = 0; c < min(kGemmStages, nch); c++) stage(c);
  uint32_t parity = 0;  // bit q: the phase of stage q's mbarrier to wait for
  bool ok = true;
  for (int c = 0; c < nch && ok; c++) {
    const int q = c % kGemmStages;
    // chunk c's copies (later chunks' groups may still be in flight)
    cp_async_wait(min(nch, c + kGemmStages) - 1 - c);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      const uint32_t a0 = tc::smem_u32(smem + q * kGemmStageBytes), b0 = a0 + kATileBytes;
      for (int kk = 0; kk < kKChunk / 16; kk++) {
        // K step of 16 = two core matrices along K
        const uint64_t ad = tc::smem_desc(a0 + kk * 2 * kLboBytes, kLboBytes, kSboBytes);
        const uint64_t bd = tc::smem_desc(b0 + kk * 2 * kLboBytes, kLboBytes, kSboBytes);
        tc::mma_bf16(taddr, ad, bd, idesc, (c > 0 || kk > 0) ? 1u : 0u);
      }
      tc::mma_commit(&bar[q]);
    }
    if (c + kGemmStages < nch || c == nch - 1) {
      // the stage is free (or, after the last chunk, D is complete) once
      // its MMAs have run
      ok = tc::mbar_wait(&bar[q], (parity >> q) & 1u);
      parity ^= 1u << q;
      tc::fence_after_sync();
      if (!__syncthreads_and(ok)) ok = false;
      if (ok && c + kGemmStages < nch) stage(c + kGemmStages);
    }
  }
  cp_async_wait(0);  // nothing left in flight into shared memory
  if (ok) {
    // epilogue: warp w holds rows m0 + 32 w + lane (tensor-memory lanes)
    const int row = m0 + warp * 32 + lane;
    const bool live = row < g.M;
    for (int c0 = 0; c0 < Nc; c0 += 16) {
      uint32_t r[16];
      tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
      tc::tmem_wait_ld();
      if (!live) continue;
#pragma unroll
      for (int e = 0; e < 16; e++) {
        const int col = n0 + c0 + e;
        if (col >= N) break;
        float v = __uint_as_float(r[e]);
        if (EPI == kEpiF32) {
          if (g.bias) v += g.bias[col];
          g.C[(long long)row * g.ldc + col] = v;
        } else if (EPI == kEpiBiasGelu) {
          const float z = v + (g.bias ? g.bias[col] : 0.f);
          g.C[(long long)row * g.ldc + col] = z;
          const uint16_t h = row < g.m_valid ? f32_to_bf16(gelu(z)) : (uint16_t)0;
          g.H[(long long)row * g.ldh + col] = h;
          if (g.Ht) g.Ht[(long long)col * g.ldht + row] = h;
        } else {  // kEpiGeluBack
          const float d = row < g.m_valid ? v * gelu_grad(g.Zin[(long long)row * g.ldz + col]) : 0.f;
          const uint16_t h = f32_to_bf16(d);
          g.H[(long long)row * g.ldh + col] = h;
          if (g.Ht) g.Ht[(long long)col * g.ldht + row] = h;
        }
      }
    }
  } else if (tid == 0) {
    atomicOr(g.err, 1);
    // a second bounded wait for MMAs still in flight before the memory is
    // freed: the last chunk's commit completes after every earlier one
    const int q = (nch - 1) % kGemmStages;
    tc::mbar_wait(&bar[q], (parity >> q) & 1u);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(taddr, ncols);
  }
}

template <int EPI>
cudaError_t launch_gemm_epi(const GemmArgs& g, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(gemm_tn_kernel<EPI>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem);
  if (e != cudaSuccess) return e;
  const dim3 grid((g.M + kMTile - 1) / kMTile, ((g.N + 15) / 16 * 16 + kNTile - 1) / kNTile);
  gemm_tn_kernel<EPI><<<grid, kGemmThreads, kGemmSmem, s>>>(g);
  return cudaGetLastError();
}

constexpr int kEwThreads = 256;

__global__ void gather_kernel(const float* __restrict__ x_src, const float* __restrict__ t_src,
                              const int* __restrict__ idx, int n, int bp, int n_in, int in_p,
                              int n_out, int out_p, uint16_t* X, uint16_t* Xt, float* T) {
  const long long e = (long long)blockIdx.x * kEwThreads + threadIdx.x;
  if (e < (long long)bp * in_p) {
    const int r = (int)(e / in_p), c = (int)(e - (e / in_p) * in_p);
    const float v = (r < n && c < n_in) ? x_src[(long long)idx[r] * n_in + c] : 0.f;
    const uint16_t h = f32_to_bf16(v);
    X[(long long)r * in_p + c] = h;
    Xt[(long long)c * bp + r] = h;
  }
  if (t_src && e < (long long)bp * out_p) {
    const int r = (int)(e / out_p), c = (int)(e - (e / out_p) * out_p);
    T[e] = (r < n && c < n_out) ? t_src[(long long)idx[r] * n_out + c] : 0.f;
  }
}

__global__ void loss_grad_kernel(const float* __restrict__ Y, const float* __restrict__ T,
                                 const float* __restrict__ w, int n, int bp, int out_p,
                                 double inv_n, uint16_t* dY, uint16_t* dYt, double* loss_rows) {
  const long long e = (long long)blockIdx.x * kEwThreads + threadIdx.x;
  if (e < (long long)bp * out_p) {
    const int r = (int)(e / out_p), c = (int)(e - (e / out_p) * out_p);
    float d = 0.f;
    if (r < n) d = (float)(2.0 * (double)w[c] * ((double)Y[e] - (double)T[e]) * inv_n);
    const uint16_t h = f32_to_bf16(d);
    dY[e] = h;
    dYt[(long long)c * bp + r] = h;
  }
  if (e < n) {  // one thread per sample row: its weighted squared error
    double acc = 0.0;
    for (int c = 0; c < out_p; c++) {
      const double dd = (double)Y[e * out_p + c] - (double)T[e * out_p + c];
      acc += (double)w[c] * dd * dd;
    }
    loss_rows[e] = acc;
  }
}

template <typename T>
__device__ __forceinline__ T block_reduce_sum(T v, T* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  T r = 0;
  if (w == 0) {
    r = l < (int)(blockDim.x >> 5) ? sh[l] : (T)0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;  // thread 0
}

__global__ void row_sums_kernel(const uint16_t* __restrict__ M, long long ld, int n, float* out) {
  __shared__ float sh[32];
  const uint16_t* row = M + (long long)blockIdx.x * ld;
  float acc = 0.f;
  for (int c = threadIdx.x; c < n; c += kEwThreads) acc += __uint_as_float((uint32_t)row[c] << 16);
  acc = block_reduce_sum(acc, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = acc;
}

__global__ void loss_reduce_kernel(const double* __restrict__ rows, int n, double scale,
                                   double* acc) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int r = threadIdx.x; r < n; r += kEwThreads) v += rows[r];
  v = block_reduce_sum(v, sh);
  if (threadIdx.x == 0) *acc += scale * v;
}

__global__ void adam_kernel(float* p, const float* __restrict__ g, float* m, float* v,
                            long long count, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  const long long e = (long long)blockIdx.x * kEwThreads + threadIdx.x;
  if (e >= count) return;
  const float gg = g[e];
  const float mm = b1 * m[e] + (1.f - b1) * gg;
  const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
  m[e] = mm;
  v[e] = vv;
  p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

__global__ void pack_weights_kernel(const float* __restrict__ W, int N, int K, uint16_t* Wb,
                                    uint16_t* Wt) {
  const long long e = (long long)blockIdx.x * kEwThreads + threadIdx.x;
  if (e >= (long long)N * K) return;
  const int r = (int)(e / K), c = (int)(e - (e / K) * K);
  const uint16_t h = f32_to_bf16(W[e]);
  Wb[e] = h;
  Wt[(long long)c * N + r] = h;
}

inline int ew_blocks(long long count) { return (int)((count + kEwThreads - 1) / kEwThreads); }

}  // namespace

cudaError_t launch_gather(const float* x_src, const float* t_src, const int* idx, int n, int bp,
                          int n_in, int in_p, int n_out, int out_p, uint16_t* X, uint16_t* Xt,
                          float* T, cudaStream_t s) {
  const long long cnt = (long long)bp * (in_p > out_p ? in_p : out_p);
  gather_kernel<<<ew_blocks(cnt), kEwThreads, 0, s>>>(x_src, t_src, idx, n, bp, n_in, in_p,
                                                      n_out, out_p, X, Xt, T);
  return cudaGetLastError();
}

cudaError_t launch_loss_grad(const float* Y, const float* T, const float* w, int n, int bp,
                             int out_p, double inv_n, uint16_t* dY, uint16_t* dYt,
                             double* loss_rows, cudaStream_t s) {
  loss_grad_kernel<<<ew_blocks((long long)bp * out_p), kEwThreads, 0, s>>>(
      Y, T, w, n, bp, out_p, inv_n, dY, dYt, loss_rows);
  return cudaGetLastError();
}

cudaError_t launch_row_sums(const uint16_t* M, long long ld, int rows, int n, float* out,
                            cudaStream_t s) {
  row_sums_kernel<<<rows, kEwThreads, 0, s>>>(M, ld, n, out);
  return cudaGetLastError();
}

cudaError_t launch_loss_reduce(const double* loss_rows, int n, double scale, double* acc,
                               cudaStream_t s) {
  loss_reduce_kernel<<<1, kEwThreads, 0, s>>>(loss_rows, n, scale, acc);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, long long count, float lr,
                        float b1, float b2, float eps, int t, cudaStream_t s) {
  // bias corrections 1 - beta^t in FP64: in FP32, 1 - 0.999^t loses about
  // nine bits to cancellation at small t
  const float c1 = (float)(1.0 - pow((double)b1, (double)t));
  const float c2 = (float)(1.0 - pow((double)b2, (double)t));
  adam_kernel<<<ew_blocks(count), kEwThreads, 0, s>>>(p, g, m, v, count, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_pack_weights(const float* W, int N, int K, uint16_t* Wb, uint16_t* Wt,
                                cudaStream_t s) {
  pack_weights_kernel<<<ew_blocks((long long)N * K), kEwThreads, 0, s>>>(W, N, K, Wb, Wt);
  return cudaGetLastError();
}

// Shape rules checked on the host before any launch.
const char* gemm_shape_error(const GemmArgs& g) {
  if (g.M < 1 || g.N < 1 || g.K < 1) return "M, N and K must be >= 1";
  if (g.N > kNMax) return "N must be <= 256";
  if (g.K % 16) return "K must be a multiple of 16";
  if (g.lda < g.K || g.ldb < g.K || g.lda % 8 || g.ldb % 8)
    return "lda and ldb must be >= K and multiples of 8 (16-byte rows)";
  if (((uintptr_t)g.A | (uintptr_t)g.B) & 15) return "A and B must be 16-byte aligned";
  return nullptr;
}

cudaError_t launch_gemm(const GemmArgs& g, int epi, cudaStream_t s) {
  if (epi == kEpiF32) return launch_gemm_epi<kEpiF32>(g, s);
  if (epi == kEpiBiasGelu) return launch_gemm_epi<kEpiBiasGelu>(g, s);
  return launch_gemm_epi<kEpiGeluBack>(g, s);
}

}  // namespace fk

extern "C" fk_status fk_gemm_bf16_tn(const void* A, int64_t lda, const void* B, int64_t ldb,
                                     float* C, int64_t ldc, int32_t M, int32_t N, int32_t K,
                                     int32_t* err_dev, void* cuda_stream) {
  fk::GemmArgs g{};
  g.A = static_cast<const uint16_t*>(A);
  g.B = static_cast<const uint16_t*>(B);
  g.lda = lda;
  g.ldb = ldb;
  g.C = C;
  g.ldc = ldc;
  g.M = M;
  g.N = N;
  g.K = K;
  g.m_valid = M;
  g.err = err_dev;
  if (!A || !B || !C || !err_dev) {
    fk::set_thread_error("fk_gemm_bf16_tn: A, B, C and err must be device pointers");
    return FK_EINVAL;
  }
  if (const char* why = fk::gemm_shape_error(g)) {
    fk::set_thread_error((std::string("fk_gemm_bf16_tn: ") + why).c_str());
    return FK_EINVAL;
  }
  if (ldc < N) {
    fk::set_thread_error("fk_gemm_bf16_tn: ldc must be >= N");
    return FK_EINVAL;
  }
  const cudaError_t e = fk::launch_gemm(g, fk::kEpiF32, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) {
    fk::set_thread_error((std::string("fk_gemm_bf16_tn: ") + cudaGetErrorString(e)).c_str());
    return FK_ECUDA;
  }
  return FK_OK;
}
