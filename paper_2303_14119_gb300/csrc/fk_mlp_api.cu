// Host side of the surrogate network (include/fk_mlp.h): parameter buffers,
// the forward and backward passes as sequences of tensor-core GEMMs with
// fused epilogues, Adam training on a device-resident data set.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "fk_internal.cuh"
#include "fk_mlp.h"
#include "fk_mlp_internal.cuh"

using namespace fk;

namespace {

thread_local std::string g_mlp_create_error;

int round_up(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

struct fk_mlp {
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int n_in = 0, width = 0, depth = 0, n_out = 0, max_batch = 0;
  int in_p = 0, out_p = 0, bp_max = 0, L = 0;
  std::vector<int> K, N;               // padded input / output widths per layer
  std::vector<size_t> woff, boff;      // offsets (floats) into the padded parameter buffers
  size_t np = 0;                       // padded parameter count
  float *d_p = nullptr, *d_g = nullptr, *d_m = nullptr, *d_v = nullptr;
  std::vector<uint16_t*> Wb, Wt;       // bf16 weights [N][K] and transposes [K][N]
  std::vector<uint16_t*> H, Ht;        // activations: H[l] [bp][K_l], Ht[l] [K_l][bp]
  std::vector<float*> Z;               // pre-activations of the hidden layers [bp][width]
  float *d_Y = nullptr, *d_T = nullptr, *d_w = nullptr;
  uint16_t *d_dY = nullptr, *d_dYt = nullptr;
  uint16_t *d_dZ[2] = {nullptr, nullptr}, *d_dZt[2] = {nullptr, nullptr};
  double *d_lrow = nullptr, *d_loss = nullptr;
  int* d_err = nullptr;
  int* d_idx = nullptr;                // gather indices of the current batch
  float *d_xin = nullptr, *d_tin = nullptr;  // staging of host inputs [bp][n_in], [bp][n_out]
  long long adam_t = 0;
  std::vector<void*> owned;
  std::string err;
};

namespace {

fk_status mfail(fk_mlp* m, fk_status s, const std::string& msg) {
  if (m)
    m->err = msg;
  else
    g_mlp_create_error = msg;
  return s;
}

fk_status mcuda(fk_mlp* m, cudaError_t e, const char* what) {
  return mfail(m, e == cudaErrorMemoryAllocation ? FK_ENOMEM : FK_ECUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

#define MK_CUDA(m, call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return mcuda((m), e_, #call);   \
  } while (0)

template <typename P>
cudaError_t malloc_owned(fk_mlp* m, P** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
  if (e == cudaSuccess) {
    m->owned.push_back(q);
    *p = static_cast<P*>(q);
  }
  return e;
}

void free_mlp(fk_mlp* m) {
  if (!m) return;
  cudaSetDevice(m->dev);
  if (m->stream) cudaStreamSynchronize(m->stream);
  for (void* p : m->owned) cudaFree(p);
  if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
  delete m;
}

// Public layout (per layer: W [N][K] then b [N], unpadded) <-> padded device
// layout (per layer: W [N_p][K_p] then b [N_p]).
void layer_dims(const fk_mlp* m, int q, int* n, int* k) {
  *k = q == 0 ? m->n_in : m->width;
  *n = q == m->L - 1 ? m->n_out : m->width;
}

long long public_count(const fk_mlp* m) {
  long long c = 0;
  for (int q = 0; q < m->L; q++) {
    int n, k;
    layer_dims(m, q, &n, &k);
    c += (long long)n * k + n;
  }
  return c;
}

void to_padded(const fk_mlp* m, const float* pub, std::vector<float>& pad) {
  pad.assign(m->np, 0.f);
  size_t pos = 0;
  for (int q = 0; q < m->L; q++) {
    int n, k;
    layer_dims(m, q, &n, &k);
    for (int r = 0; r < n; r++)
      for (int c = 0; c < k; c++) pad[m->woff[q] + (size_t)r * m->K[q] + c] = pub[pos++];
    for (int r = 0; r < n; r++) pad[m->boff[q] + r] = pub[pos++];
  }
}

void from_padded(const fk_mlp* m, const std::vector<float>& pad, float* pub) {
  size_t pos = 0;
  for (int q = 0; q < m->L; q++) {
    int n, k;
    layer_dims(m, q, &n, &k);
    for (int r = 0; r < n; r++)
      for (int c = 0; c < k; c++) pub[pos++] = pad[m->woff[q] + (size_t)r * m->K[q] + c];
    for (int r = 0; r < n; r++) pub[pos++] = pad[m->boff[q] + r];
  }
}

fk_status pack_all(fk_mlp* m) {
  for (int q = 0; q < m->L; q++)
    MK_CUDA(m, launch_pack_weights(m->d_p + m->woff[q], m->N[q], m->K[q], m->Wb[q], m->Wt[q],
                                   m->stream));
  return FK_OK;
}

}  // namespace

namespace {

GemmArgs gemm_args(fk_mlp* m) {
  GemmArgs g{};
  g.err = m->d_err;
  return g;
}

// Forward pass over bp rows (n live) from H[0] / Ht[0]: hidden layers with
// the bias + GELU epilogue (Z kept for the backward pass), output layer with
// the bias epilogue into Y.
fk_status forward_pass(fk_mlp* m, int n, int bp) {
  for (int q = 0; q < m->L; q++) {
    GemmArgs g = gemm_args(m);
    g.A = m->H[q];
    g.lda = m->K[q];
    g.B = m->Wb[q];
    g.ldb = m->K[q];
    g.M = bp;
    g.N = m->N[q];
    g.K = m->K[q];
    g.bias = m->d_p + m->boff[q];
    g.m_valid = n;
    if (q < m->L - 1) {
      g.C = m->Z[q];
      g.ldc = m->N[q];
      g.H = m->H[q + 1];
      g.ldh = m->N[q];
      g.Ht = m->Ht[q + 1];
      g.ldht = bp;
      MK_CUDA(m, launch_gemm(g, kEpiBiasGelu, m->stream));
    } else {
      g.C = m->d_Y;
      g.ldc = m->out_p;
      MK_CUDA(m, launch_gemm(g, kEpiF32, m->stream));
    }
  }
  return FK_OK;
}

// Backward pass: dL/dY from Y and T, then per layer (last first) the weight
// gradient dZ^T H, the bias gradient (row sums of dZ^T) and, below the
// first layer, dZ of the layer beneath through W and gelu'.
fk_status backward_pass(fk_mlp* m, int n, int bp, double inv_n) {
  MK_CUDA(m, launch_loss_grad(m->d_Y, m->d_T, m->d_w, n, bp, m->out_p, inv_n, m->d_dY, m->d_dYt,
                              m->d_lrow, m->stream));
  const uint16_t* dz = m->d_dY;    // [bp][N_q]
  const uint16_t* dzt = m->d_dYt;  // [N_q][bp]
  int cur = 0;
  for (int q = m->L - 1; q >= 0; q--) {
    GemmArgs g = gemm_args(m);
    g.A = dzt;
    g.lda = bp;
    g.B = m->Ht[q];
    g.ldb = bp;
    g.M = m->N[q];
    g.N = m->K[q];
    g.K = bp;
    g.C = m->d_g + m->woff[q];
    g.ldc = m->K[q];
    g.m_valid = m->N[q];
    MK_CUDA(m, launch_gemm(g, kEpiF32, m->stream));
    MK_CUDA(m, launch_row_sums(dzt, bp, m->N[q], n, m->d_g + m->boff[q], m->stream));
    if (q == 0) break;
    GemmArgs d = gemm_args(m);
    d.A = dz;
    d.lda = m->N[q];
    d.B = m->Wt[q];
    d.ldb = m->N[q];
    d.M = bp;
    d.N = m->K[q];
    d.K = m->N[q];
    d.Zin = m->Z[q - 1];
    d.ldz = m->K[q];
    d.H = m->d_dZ[cur];
    d.ldh = m->K[q];
    d.Ht = m->d_dZt[cur];
    d.ldht = bp;
    d.m_valid = n;
    MK_CUDA(m, launch_gemm(d, kEpiGeluBack, m->stream));
    dz = m->d_dZ[cur];
    dzt = m->d_dZt[cur];
    cur ^= 1;
  }
  return FK_OK;
}

// Copy n host rows of x (and t) into the staging buffers and gather them
// into H[0] / Ht[0] (and T).
fk_status load_rows(fk_mlp* m, const float* x, const float* t, int n, int bp) {
  MK_CUDA(m, cudaMemcpyAsync(m->d_xin, x, (size_t)n * m->n_in * sizeof(float),
                             cudaMemcpyHostToDevice, m->stream));
  if (t)
    MK_CUDA(m, cudaMemcpyAsync(m->d_tin, t, (size_t)n * m->n_out * sizeof(float),
                               cudaMemcpyHostToDevice, m->stream));
  MK_CUDA(m, launch_gather(m->d_xin, t ? m->d_tin : nullptr, m->d_idx, n, bp, m->n_in, m->in_p,
                           m->n_out, m->out_p, m->H[0], m->Ht[0], m->d_T, m->stream));
  return FK_OK;
}

fk_status set_loss_weights(fk_mlp* m, const float* w) {
  std::vector<float> wp(m->out_p, 0.f);
  for (int o = 0; o < m->n_out; o++) wp[o] = w ? w[o] : 1.f;
  MK_CUDA(m, cudaMemcpyAsync(m->d_w, wp.data(), m->out_p * sizeof(float), cudaMemcpyHostToDevice,
                             m->stream));
  MK_CUDA(m, cudaStreamSynchronize(m->stream));
  return FK_OK;
}

fk_status check_err(fk_mlp* m) {
  int e = 0;
  MK_CUDA(m, cudaMemcpyAsync(&e, m->d_err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  MK_CUDA(m, cudaStreamSynchronize(m->stream));
  if (e) return mfail(m, FK_ETIMEOUT, "a bounded wait inside a tensor-core GEMM ran out");
  return FK_OK;
}

uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

fk_status fk_mlp_create(const fk_mlp_desc* desc, void* cuda_stream, fk_mlp** out) {
  g_mlp_create_error.clear();
  if (!desc || !out) return mfail(nullptr, FK_EINVAL, "desc and out must not be NULL");
  *out = nullptr;
  const fk_mlp_desc& d = *desc;
  if (d.n_in < 1 || d.n_in > 256 || d.n_out < 1 || d.n_out > 256)
    return mfail(nullptr, FK_EINVAL, "need 1 <= n_in, n_out <= 256");
  if (d.width < 16 || d.width > 256 || d.width % 16)
    return mfail(nullptr, FK_EINVAL, "width must be a multiple of 16 in [16, 256]");
  if (d.depth < 1 || d.depth > 32) return mfail(nullptr, FK_EINVAL, "need 1 <= depth <= 32");
  if (d.max_batch < 1 || d.max_batch > (1 << 20))
    return mfail(nullptr, FK_EINVAL, "need 1 <= max_batch <= 2^20");
  fk_mlp* m = new (std::nothrow) fk_mlp();
  if (!m) return mfail(nullptr, FK_ENOMEM, "host allocation failed");
  m->dev = d.device;
  m->n_in = d.n_in;
  m->width = d.width;
  m->depth = d.depth;
  m->n_out = d.n_out;
  m->max_batch = d.max_batch;
  m->in_p = round_up(d.n_in, 16);
  m->out_p = round_up(d.n_out, 16);
  m->bp_max = round_up(d.max_batch, 128);
  m->L = d.depth + 1;
  size_t pos = 0;
  for (int q = 0; q < m->L; q++) {
    const int k = q == 0 ? m->in_p : m->width;
    const int n = q == m->L - 1 ? m->out_p : m->width;
    m->K.push_back(k);
    m->N.push_back(n);
    m->woff.push_back(pos);
    pos += (size_t)n * k;
    m->boff.push_back(pos);
    pos += n;
  }
  m->np = pos;
#define CREATE_M(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) {                             \
      const fk_status s_ = mcuda(nullptr, e_, #call);    \
      free_mlp(m);                                       \
      return s_;                                         \
    }                                                    \
  } while (0)
  CREATE_M(cudaSetDevice(m->dev));
  if (cuda_stream) {
    m->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    CREATE_M(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking));
    m->own_stream = true;
  }
  const size_t bp = m->bp_max;
  CREATE_M(malloc_owned(m, &m->d_p, m->np * sizeof(float)));
  CREATE_M(malloc_owned(m, &m->d_g, m->np * sizeof(float)));
  CREATE_M(malloc_owned(m, &m->d_m, m->np * sizeof(float)));
  CREATE_M(malloc_owned(m, &m->d_v, m->np * sizeof(float)));
  m->Wb.assign(m->L, nullptr);
  m->Wt.assign(m->L, nullptr);
  m->H.assign(m->L, nullptr);
  m->Ht.assign(m->L, nullptr);
  m->Z.assign(m->L - 1, nullptr);
  for (int q = 0; q < m->L; q++) {
    CREATE_M(malloc_owned(m, &m->Wb[q], (size_t)m->N[q] * m->K[q] * 2));
    CREATE_M(malloc_owned(m, &m->Wt[q], (size_t)m->N[q] * m->K[q] * 2));
    CREATE_M(malloc_owned(m, &m->H[q], bp * m->K[q] * 2));
    CREATE_M(malloc_owned(m, &m->Ht[q], bp * m->K[q] * 2));
    if (q < m->L - 1) CREATE_M(malloc_owned(m, &m->Z[q], bp * m->width * sizeof(float)));
  }
  CREATE_M(malloc_owned(m, &m->d_Y, bp * m->out_p * sizeof(float)));
  CREATE_M(malloc_owned(m, &m->d_T, bp * m->out_p * sizeof(float)));
  CREATE_M(malloc_owned(m, &m->d_w, m->out_p * sizeof(float)));
  CREATE_M(malloc_owned(m, &m->d_dY, bp * m->out_p * 2));
  CREATE_M(malloc_owned(m, &m->d_dYt, bp * m->out_p * 2));
  for (int c = 0; c < 2; c++) {
    CREATE_M(malloc_owned(m, &m->d_dZ[c], bp * m->width * 2));
    CREATE_M(malloc_owned(m, &m->d_dZt[c], bp * m->width * 2));
  }
  CREATE_M(malloc_owned(m, &m->d_lrow, bp * sizeof(double)));
  CREATE_M(malloc_owned(m, &m->d_loss, sizeof(double)));
  CREATE_M(malloc_owned(m, &m->d_err, sizeof(int)));
  CREATE_M(malloc_owned(m, &m->d_idx, bp * sizeof(int)));
  CREATE_M(malloc_owned(m, &m->d_xin, bp * m->n_in * sizeof(float)));
  CREATE_M(malloc_owned(m, &m->d_tin, bp * m->n_out * sizeof(float)));
  CREATE_M(cudaMemsetAsync(m->d_p, 0, m->np * sizeof(float), m->stream));
  CREATE_M(cudaMemsetAsync(m->d_m, 0, m->np * sizeof(float), m->stream));
  CREATE_M(cudaMemsetAsync(m->d_v, 0, m->np * sizeof(float), m->stream));
  CREATE_M(cudaMemsetAsync(m->d_err, 0, sizeof(int), m->stream));
  {
    std::vector<int> iota(bp);
    for (size_t r = 0; r < bp; r++) iota[r] = (int)r;
    CREATE_M(cudaMemcpyAsync(m->d_idx, iota.data(), bp * sizeof(int), cudaMemcpyHostToDevice,
                             m->stream));
    CREATE_M(cudaStreamSynchronize(m->stream));
  }
#undef CREATE_M
  fk_status s = pack_all(m);
  if (s == FK_OK) s = set_loss_weights(m, nullptr);
  if (s != FK_OK) {
    g_mlp_create_error = m->err;
    free_mlp(m);
    return s;
  }
  *out = m;
  return FK_OK;
}

fk_status fk_mlp_destroy(fk_mlp* m) {
  free_mlp(m);
  return FK_OK;
}

fk_status fk_mlp_param_count(const fk_mlp* m, int64_t* count) {
  if (!m || !count) return FK_EINVAL;
  *count = public_count(m);
  return FK_OK;
}

fk_status fk_mlp_set_params(fk_mlp* m, const float* params) {
  if (!m || !params) return FK_EINVAL;
  const long long n = public_count(m);
  for (long long q = 0; q < n; q++)
    if (!isfinite(params[q])) return mfail(m, FK_EINVAL, "parameters must be finite");
  std::vector<float> pad;
  to_padded(m, params, pad);
  MK_CUDA(m, cudaSetDevice(m->dev));
  MK_CUDA(m, cudaMemcpyAsync(m->d_p, pad.data(), m->np * sizeof(float), cudaMemcpyHostToDevice,
                             m->stream));
  MK_CUDA(m, cudaMemsetAsync(m->d_m, 0, m->np * sizeof(float), m->stream));
  MK_CUDA(m, cudaMemsetAsync(m->d_v, 0, m->np * sizeof(float), m->stream));
  m->adam_t = 0;
  fk_status s = pack_all(m);
  if (s != FK_OK) return s;
  MK_CUDA(m, cudaStreamSynchronize(m->stream));  // the padded copy goes out of scope
  return FK_OK;
}

fk_status fk_mlp_get_params(fk_mlp* m, float* params) {
  if (!m || !params) return FK_EINVAL;
  MK_CUDA(m, cudaSetDevice(m->dev));
  std::vector<float> pad(m->np);
  MK_CUDA(m, cudaMemcpyAsync(pad.data(), m->d_p, m->np * sizeof(float), cudaMemcpyDeviceToHost,
                             m->stream));
  MK_CUDA(m, cudaStreamSynchronize(m->stream));
  from_padded(m, pad, params);
  return FK_OK;
}

fk_status fk_mlp_forward(fk_mlp* m, const float* x, int64_t n, float* y) {
  if (!m || (n > 0 && (!x || !y)) || n < 0) return m ? mfail(m, FK_EINVAL, "bad arguments") : FK_EINVAL;
  MK_CUDA(m, cudaSetDevice(m->dev));
  for (int64_t r0 = 0; r0 < n; r0 += m->max_batch) {
    const int nb = (int)std::min<int64_t>(m->max_batch, n - r0);
    const int bp = round_up(nb, 128);
    fk_status s = load_rows(m, x + r0 * m->n_in, nullptr, nb, bp);
    if (s == FK_OK) s = forward_pass(m, nb, bp);
    if (s != FK_OK) return s;
    MK_CUDA(m, cudaMemcpy2DAsync(y + r0 * m->n_out, m->n_out * sizeof(float), m->d_Y,
                                 m->out_p * sizeof(float), m->n_out * sizeof(float), nb,
                                 cudaMemcpyDeviceToHost, m->stream));
    MK_CUDA(m, cudaStreamSynchronize(m->stream));
  }
  return check_err(m);
}

fk_status fk_mlp_loss_grad(fk_mlp* m, const float* x, const float* t, const float* w, int64_t n,
                           double* loss, float* grad) {
  if (!m) return FK_EINVAL;
  if (!x || !t || n < 1 || n > m->max_batch)
    return mfail(m, FK_EINVAL, "need x, t and 1 <= n <= max_batch");
  MK_CUDA(m, cudaSetDevice(m->dev));
  fk_status s = set_loss_weights(m, w);
  const int bp = round_up((int)n, 128);
  if (s == FK_OK) s = load_rows(m, x, t, (int)n, bp);
  if (s == FK_OK) s = forward_pass(m, (int)n, bp);
  if (s == FK_OK) s = backward_pass(m, (int)n, bp, 1.0 / (double)n);
  if (s != FK_OK) return s;
  MK_CUDA(m, cudaMemsetAsync(m->d_loss, 0, sizeof(double), m->stream));
  MK_CUDA(m, launch_loss_reduce(m->d_lrow, (int)n, 1.0 / (double)n, m->d_loss, m->stream));
  double l = 0.0;
  MK_CUDA(m, cudaMemcpyAsync(&l, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  std::vector<float> pad;
  if (grad) {
    pad.resize(m->np);
    MK_CUDA(m, cudaMemcpyAsync(pad.data(), m->d_g, m->np * sizeof(float), cudaMemcpyDeviceToHost,
                               m->stream));
  }
  MK_CUDA(m, cudaStreamSynchronize(m->stream));
  if (loss) *loss = l;
  if (grad) from_padded(m, pad, grad);
  return check_err(m);
}

fk_status fk_mlp_train(fk_mlp* m, const float* x, const float* t, const float* w, int64_t n,
                       int32_t batch, int32_t epochs, float lr, uint64_t seed,
                       double* epoch_loss) {
  if (!m) return FK_EINVAL;
  if (!x || !t || n < 1 || n > (int64_t)1 << 30 || batch < 1 || batch > m->max_batch ||
      epochs < 0 || !(lr > 0.f) || !isfinite(lr))
    return mfail(m, FK_EINVAL,
                 "need x, t, 1 <= n, 1 <= batch <= max_batch, epochs >= 0 and lr > 0");
  MK_CUDA(m, cudaSetDevice(m->dev));
  fk_status s = set_loss_weights(m, w);
  if (s != FK_OK) return s;
  float *dx = nullptr, *dt = nullptr;
  int* dperm = nullptr;
  double* dl = nullptr;
  auto release = [&]() {
    cudaStreamSynchronize(m->stream);
    if (dx) cudaFree(dx);
    if (dt) cudaFree(dt);
    if (dperm) cudaFree(dperm);
    if (dl) cudaFree(dl);
  };
#define TRAIN_CUDA(call)                     \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) {                 \
      const fk_status s_ = mcuda(m, e_, #call); \
      release();                             \
      return s_;                             \
    }                                        \
  } while (0)
  TRAIN_CUDA(cudaMalloc(&dx, (size_t)n * m->n_in * sizeof(float)));
  TRAIN_CUDA(cudaMalloc(&dt, (size_t)n * m->n_out * sizeof(float)));
  TRAIN_CUDA(cudaMalloc(&dperm, (size_t)n * sizeof(int)));
  TRAIN_CUDA(cudaMalloc(&dl, (size_t)std::max(epochs, 1) * sizeof(double)));
  TRAIN_CUDA(cudaMemcpyAsync(dx, x, (size_t)n * m->n_in * sizeof(float), cudaMemcpyHostToDevice,
                             m->stream));
  TRAIN_CUDA(cudaMemcpyAsync(dt, t, (size_t)n * m->n_out * sizeof(float), cudaMemcpyHostToDevice,
                             m->stream));
  TRAIN_CUDA(cudaMemsetAsync(dl, 0, (size_t)std::max(epochs, 1) * sizeof(double), m->stream));
  std::vector<int> perm(n);
  for (int ep = 0; ep < epochs; ep++) {
    // sample order of this epoch: Fisher-Yates driven by SplitMix64 outputs
    for (int64_t q = 0; q < n; q++) perm[q] = (int)q;
    const uint64_t base = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(ep + 1);
    for (int64_t q = n - 1; q > 0; q--) {
      const uint64_t r = mix64(base + 0x9E3779B97F4A7C15ull * (uint64_t)(q + 1));
      std::swap(perm[q], perm[r % (uint64_t)(q + 1)]);
    }
    TRAIN_CUDA(cudaMemcpyAsync(dperm, perm.data(), (size_t)n * sizeof(int),
                               cudaMemcpyHostToDevice, m->stream));
    for (int64_t off = 0; off < n; off += batch) {
      const int nb = (int)std::min<int64_t>(batch, n - off);
      const int bp = round_up(nb, 128);
      TRAIN_CUDA(launch_gather(dx, dt, dperm + off, nb, bp, m->n_in, m->in_p, m->n_out, m->out_p,
                               m->H[0], m->Ht[0], m->d_T, m->stream));
      s = forward_pass(m, nb, bp);
      if (s == FK_OK) s = backward_pass(m, nb, bp, 1.0 / (double)nb);
      if (s != FK_OK) {
        release();
        return s;
      }
      TRAIN_CUDA(launch_loss_reduce(m->d_lrow, nb, 1.0 / (double)n, dl + ep, m->stream));
      m->adam_t += 1;
      TRAIN_CUDA(launch_adam(m->d_p, m->d_g, m->d_m, m->d_v, (long long)m->np, lr, 0.9f, 0.999f,
                             1e-8f, (int)std::min<long long>(m->adam_t, 1 << 30), m->stream));
      s = pack_all(m);
      if (s != FK_OK) {
        release();
        return s;
      }
    }
    // the host permutation is rewritten next epoch: its copy must be done
    TRAIN_CUDA(cudaStreamSynchronize(m->stream));
  }
#undef TRAIN_CUDA
  if (epoch_loss && epochs > 0)
    cudaMemcpyAsync(epoch_loss, dl, (size_t)epochs * sizeof(double), cudaMemcpyDeviceToHost,
                    m->stream);
  release();
  return check_err(m);
}

const char* fk_mlp_last_error(const fk_mlp* m) {
  return m ? m->err.c_str() : g_mlp_create_error.c_str();
}

}  // extern "C"
