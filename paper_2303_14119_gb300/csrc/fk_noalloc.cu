// fk_density_moment_noalloc: the density moment n_e(x) of a distribution
// that already lives in device memory, computed without allocating any
// memory.  Its scratch (the per-plane partial sums of a two-pass,
// fixed-order reduction) is a file-scope __device__ array of fixed size
// that every GPU loading this library holds until the process exits.
#include <mutex>
#include <string>

#include "fk_internal.cuh"

namespace {

constexpr int kUnits = 16;  // partial sums per x-plane
constexpr int kThreads = 256;

// Scratch shared by every call: FK_NOALLOC_MAX_PARTIALS doubles (1 MiB).
static __device__ __align__(256) double g_noalloc_partials[FK_NOALLOC_MAX_PARTIALS];

// In host code the name g_noalloc_partials is only a host-side stand-in;
// the kernels get the device address looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch[kMaxDevices] = {};

// Pass 1: block (k, u) sums its slice of plane k in a fixed tree order.
__global__ void __launch_bounds__(kThreads)
moment_partials(const double* __restrict__ f, long long plane, double* partials) {
  __shared__ double sh[kThreads / 32];
  const int k = blockIdx.x / kUnits, u = blockIdx.x - (blockIdx.x / kUnits) * kUnits;
  const long long per = (plane + kUnits - 1) / kUnits;
  const long long lo = (long long)u * per;
  const long long hi = lo + per < plane ? lo + per : plane;
  const double* p = f + (long long)k * plane;
  double s = 0.0;
  for (long long c = lo + threadIdx.x; c < hi; c += kThreads) s += p[c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; w++) t += sh[w];
    partials[blockIdx.x] = t;  // every slot used by this call is written here
  }
}

// Pass 2: n_e[k] = dv1 dv2 * (sum of plane k's partials, in unit order).
__global__ void moment_finish(const double* partials, int nx, double dvv, double* n_e) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nx) return;
  double s = 0.0;
  for (int u = 0; u < kUnits; u++) s += partials[k * kUnits + u];
  n_e[k] = s * dvv;
}

}  // namespace

extern "C" fk_status fk_density_moment_noalloc(const double* f_dev, int32_t nx, int32_t nv1,
                                               int32_t nv2, double dv1, double dv2,
                                               double* n_e_dev, void* cuda_stream) {
  if (!f_dev || !n_e_dev) {
    fk::set_thread_error("fk_density_moment_noalloc: f and n_e must be device pointers");
    return FK_EINVAL;
  }
  if (nx < 1 || nv1 < 1 || nv2 < 1 || !(dv1 > 0.0) || !(dv2 > 0.0)) {
    fk::set_thread_error("fk_density_moment_noalloc: need nx, nv1, nv2 >= 1 and dv1, dv2 > 0");
    return FK_EINVAL;
  }
  if ((long long)nx * kUnits > FK_NOALLOC_MAX_PARTIALS) {
    fk::set_thread_error(("fk_density_moment_noalloc: nx = " + std::to_string(nx) +
                          " exceeds the scratch limit of " +
                          std::to_string(FK_NOALLOC_MAX_PARTIALS / kUnits) + " planes")
                             .c_str());
    return FK_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    fk::set_thread_error("fk_density_moment_noalloc: no usable current CUDA device");
    return FK_ECUDA;
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch[dev]) {
      // first call on this device (with it current): look up the device
      // address of the scratch array
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
      if (e != cudaSuccess) {
        fk::set_thread_error((std::string("fk_density_moment_noalloc: cudaGetSymbolAddress: ") +
                              cudaGetErrorString(e))
                                 .c_str());
        return FK_ECUDA;
      }
      g_scratch[dev] = static_cast<double*>(ptr);
    }
    scratch = g_scratch[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const long long plane = (long long)nv1 * nv2;
  moment_partials<<<nx * kUnits, kThreads, 0, s>>>(f_dev, plane, scratch);
  moment_finish<<<(nx + 255) / 256, 256, 0, s>>>(scratch, nx, dv1 * dv2, n_e_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    fk::set_thread_error((std::string("fk_density_moment_noalloc: launch: ") +
                          cudaGetErrorString(e))
                             .c_str());
    return FK_ECUDA;
  }
  return FK_OK;
}
