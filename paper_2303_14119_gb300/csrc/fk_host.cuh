// Host-side definition of the grid object, shared by the grid API and the
// batch API (internal; the public ABI is include/fk.h).
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <string>
#include <vector>

#include "fk_internal.cuh"

struct fk_grid {
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t cap_stream = nullptr;
  fk_grid_desc desc{};
  int prec = FK_F64;
  int nx = 0, nv1 = 0, nv2 = 0, pitch = 0;
  size_t esize = 8;
  double dx = 0, dv1 = 0, dv2 = 0, dt = 0;
  fk::Params prm{};
  fk::Params* d_prm = nullptr;
  fk::DevState* d_st = nullptr;
  void* d_f[2] = {nullptr, nullptr};
  int enq_cur = 0;            // buffer the next enqueued step reads
  int base_cur = 0;           // buffer that held state base_step
  long long base_step = 0;
  fk::Tables tab{};
  fk::Partials part{};
  fk::Geom geom{};
  int tile_cap = 0;   // whole-CTA v1 tiles of at most this many rows (0: the plan's most)
  int env_direct = -1, env_no_half = -1;  // FK_STEP_KERNEL / FK_STREAM_HALF at creation
  int part_cap = 0;   // tiles the partial-sum buffers hold
  bool use_stream = true;  // streaming kernel (else the direct-load kernel)
  double *d_ne = nullptr, *d_Ex = nullptr, *d_c1 = nullptr, *d_hist = nullptr;
  float* d_c1_32 = nullptr;
  fk::FinScratch fin{};
  void* d_stage = nullptr;
  // pinned read-back buffer of the getters: DevState, then n_e and E_x [nx]
  void* h_stage = nullptr;
  // physics parameters as last set
  double Ey = 0, Ex_ext = 0;
  int self_consistent = 1;
  double delta_max = 0, A_max = 1, k_s = 1, T_se = 1;
  int see_enabled = 0;
  double J = 0, x_lo = 0, x_hi = 0, T_fe = 1;
  double T_e = 2.0, ln_lambda = 10.0;  // BGK collisions (off until switched on)
  double *d_bgk = nullptr;             // [2][nx] per-plane collision coefficients
  float* d_bgk32 = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  unsigned known_flags = 0;
  // kernel timing
  bool timing = false;
  std::vector<cudaEvent_t> ev;  // pairs: 2*r = start, 2*r+1 = stop
  int ev_used = 0;              // pairs recorded since the last read
  // batch that steps this grid: while set, calls that change the state are
  // refused and the getters wait for the batch's last enqueued step
  int scheme = 0;             // kSchemeUnsplit or kSchemeLie
  void* d_f3 = nullptr;       // intermediate state of the split steps
  // the split steps' passes on the streaming kernel: the parameters of an
  // x pass (c_2 = 0, no source band, no collisions), zeros for the c_1 of
  // an x pass and the c_x of the velocity pass (one array of
  // max(nx, nv1) doubles, which read as floats are zeros too), c_x / 2 of
  // a Strang half pass, and the velocity-edge partials the last Strang
  // pass writes aside (the velocity pass's are the step's)
  fk::Params prm_x{};
  fk::Params* d_prm_x = nullptr;
  double* d_zero = nullptr;
  double* d_cx_half = nullptr;
  float* d_cx32_half = nullptr;
  double* d_lv_aside = nullptr;
  fk::DevState* d_st_mid = nullptr;  // Strang step: wall fluxes after the velocity pass
  fk_batch* batch = nullptr;
  cudaEvent_t batch_done = nullptr;
  std::string err;
};

namespace fk {

// An NVTX range over a host call (tracing: profilers and timeline tools
// show each fk_step / batch step as a named range; free without a tool).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Passes of the direct-load step kernel: a whole step, the moments of f_in
// only, and the passes of the split steps: x-advection with the wall and
// vacuum boundaries (over dt; over dt/2 without partial sums; over dt/2
// writing every partial sum but the velocity-edge loss, the last pass of a
// Strang step), and v1, v2 advection, source and collisions.
enum StepPass {
  kPassFull = 0,
  kPassMoments = 1,
  kPassX = 2,
  kPassV = 3,
  kPassXHalf = 4,
  kPassXHalfLast = 5
};
cudaError_t launch_step_pass(const StepArgs& a, int precision, int mode, cudaStream_t s);

// Time schemes of a grid (fk_set_scheme).
enum Scheme { kSchemeUnsplit = 0, kSchemeLie = 1, kSchemeStrang = 2 };

// Finalize mode of a Strang step, beside the modes of FinalizeMode: the wall
// and vacuum terms of f^n weigh dt/2 (the other half came from the state
// after the velocity pass, folded by launch_strang_mid).
constexpr int kModeStepStrang = 3;
// Strang step, after the velocity pass: fold its wall and vacuum partial
// sums (those of the state the second x half-pass acts on), add dt/2 of
// them to the surface charge and the ledger in a.st, and write that state's
// Gamma_see and the flags into *mid, the state block of the second x
// half-pass.
cudaError_t launch_strang_mid(const StepArgs& a, DevState* mid, cudaStream_t s);

// Per-step arguments of the grid with f^n in buffer cur.
StepArgs make_args(fk_grid* g, int cur);
// Synchronise the grid's stream (after the batch that steps it, if any),
// read the device scalars and re-base the buffer bookkeeping.
fk_status sync_state(fk_grid* g, DevState* out);
// The same, also reading n_e and E_x [nx] into the host arrays given
// (either may be NULL): one wait for all the copies.
fk_status sync_state_with(fk_grid* g, DevState* out, double* n_e, double* Ex);
// Cap the v1 rows of the grid's whole-CTA tiles (0: the shared-memory plan's
// most) and re-plan its work decomposition; the grid must be idle.  The
// partial-sum buffers grow if the new plan has more tiles; captured graphs
// are dropped.
fk_status replan_tiles(fk_grid* g, int cap);
// Device (host: pinned host) allocation through the failure-injection test
// hook: with FK_TEST_FAIL_ALLOC=<n> in the environment, the n-th allocation
// since the last alloc_hook_reset() (called at the start of fk_create_grid
// and fk_batch_create) fails with cudaErrorMemoryAllocation.
cudaError_t hooked_alloc(void** p, size_t bytes, bool host = false);
void alloc_hook_reset();
// dst[i] = s * src[i] and dst32[i] = s * src32[i] for i < n.
cudaError_t launch_scale_tables(const double* src, const float* src32, double s, int n,
                                double* dst, float* dst32, cudaStream_t st);
// Status for sticky device flags (FK_OK if none); sets the grid's message.
fk_status flags_status(fk_grid* g, unsigned flags);

}  // namespace fk
