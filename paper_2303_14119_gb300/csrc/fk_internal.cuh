// Internal declarations shared by the CUDA translation units of the library.
// Not part of the public ABI (include/fk.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "fk.h"

namespace fk {

// CODATA 2018 values (SI).
constexpr double kQe = 1.602176634e-19;    // elementary charge, C
constexpr double kMe = 9.1093837015e-31;   // electron mass, kg
constexpr double kEps0 = 8.8541878128e-12; // vacuum permittivity, F/m
constexpr double kPi = 3.14159265358979323846;

// Sticky device error bits (fk_dev_state::flags).
enum : unsigned {
  kFlagCfl = 1u,
  kFlagNumeric = 2u,
  kFlagTimeout = 4u,
  kFlagNegative = 8u,
  kFlagBounds = 16u,  // FK_DEBUG_BOUNDS builds: an index check failed
};

// Default limit of a bounded wait inside a kernel: cycles (about 2 s).
constexpr long long kWaitLimitCycles = 4000000000LL;

// Run parameters read by the kernels from device memory, so that captured
// CUDA graphs stay valid when a setter changes them.
struct Params {
  double dx, dv1, dv2, dt;
  double Ey, Ex_ext;
  double c2;      // signed v2-Courant number a2 dt / dv2
  double cx_max;  // max_i |v1_i| dt / dx
  double inj;     // injected electrons per m^2 per s (J/e, 0 if off)
  double sat_tol;
  // host-computed coefficients of the finalize kernel (no division on the
  // device): E_x = sigma * ex_sigma - ex_n * (sum of n below + n_k / 2),
  // c_1 = c1_per_ex * E_x, density scale dv1 dv2, loss scale dx dv1 dv2 / dt
  double ex_sigma, ex_n, c1_per_ex, dvv, lv_scale;
  long long sat_window;
  long long hist_cap;
  // electron-electron BGK collisions (Eqs. 3-5): relaxation rate of plane k
  // is nu_k = bgk_c n_k / dt, i.e. dt nu_k = bgk_c * n_k
  double bgk_c;
  // electron reflection at the dielectric: a fraction refl of each incident
  // flux element returns at the mirrored v1 (symmetric v1 grid)
  double refl;
  int collisions;
  int self_consistent;
  int see_enabled;
  int band_lo, band_hi; // source planes [band_lo, band_hi)
  // failure-detection test knobs, read from the environment at grid
  // creation (off by default): the limit of the streaming kernel's bounded
  // waits (cycles), and a pipeline item (>= 0) whose plane copy the unit of
  // tile 0, chunk 0 does not issue, so that the waits on it run out
  int withhold_item;
  long long wait_limit;
};

// Mutable per-run scalars, device resident.
struct DevState {
  double sigma, sigma0;
  // fluxes and totals of the current state
  double g_pe, g_see, g_vac, n_tot, n0;
  // cumulative ledger terms
  double cum_emit, cum_see, cum_pe, cum_vac, cum_lv, cum_inj;
  long long step, sat_step, hist_count;
  unsigned flags;
  unsigned pad;
};

// Per work-unit partial sums written by the step kernel's epilogue; the
// finalize kernel reduces them in a fixed order.
struct Partials {
  double* n;    // [nx][nu] sum of f^{n+1} over the unit's cells
  double* lv;   // [nx][nu] sum over downwind velocity-edge cells of |c| f^n
  double* pe;   // [nu]     sum over x = 0 cells with v1 < 0 of -v1 f^{n+1}
  double* see;  // [nu]     same weighted by delta
  double* vac;  // [nu]     sum over x = nx-1 cells with v1 > 0 of v1 f^{n+1}
  int nu;       // units (tiles) per plane
};

// Velocity-space tables.  2D tables use the row pitch of f (zero padding).
struct Tables {
  double* v1;     // [nv1] cell-centre normal velocities
  double* cx;     // [nv1] signed x-Courant numbers v1 dt / dx
  float* cx32;    // [nv1] the same rounded to FP32
  double* delta;  // [nv1][pitch] SEE yield, zero where v1 >= 0
  double* gse;    // [nv1][pitch] emission shape, unit flux
  double* src;    // [nv1][pitch] dt (J/e)/W g_fe, added on source planes
  float* src32;   // same rounded to FP32
  double* gfe_raw;// [nv1][pitch] scratch for the source shape
  // the source shape is separable (Maxwellian in v1 times half-Maxwellian
  // in v2, normalised per factor): src(i, j) = srow32[i] * scol32[j]
  float* srow32;  // [nv1] dt (J/e)/W times the normalised v1 factor
  float* scol32;  // [pitch] normalised v2 factor, zero for v2 <= 0 and padding
  double* tsum;   // [tables_scratch_doubles()] normalisation partials and norms
  // equilibrium of Eq. 5 at T_e, separable and normalised per factor on the
  // grid: f_e0(i, j) = m1[i] * m2[j] with sum_i m1 dv1 = sum_j m2 dv2 = 1
  double* m1;     // [nv1]
  double* m2;     // [pitch] (zero on padding)
  float* m1_32;
  float* m2_32;
  // for the wall sums of FP32 grids' half units, as FP32 pairs x = x.x +
  // x.y: x.x = x rounded to FP32, x.y = the rest rounded to FP32
  float2* v1p;     // [nv1] v1
  float2* deltap;  // [nv1][pitch] delta
};

// Work decomposition shared by the step kernels and the finalize kernel.
// v1 rows split at i_neg: rows [0, i_neg) have v1 <= 0 (upwind in x is
// k+1, march toward -x), rows [i_neg, nv1) have v1 > 0 (upwind k-1, march
// toward +x).  Each half is cut into tiles of at most ti rows; a tile never
// straddles the split, so one x-upwind direction holds for the whole tile.
// The march along x is cut into chunks; one CTA of the streaming kernel
// owns one (tile, chunk) unit.
struct Geom {
  int ti_neg, ti_pos;  // rows per tile in each half (last tile may be short)
  int i_neg;           // first row with v1 > 0
  int t_neg, n_tiles;  // tiles in the lower half, tiles in total
  int chunk_len, n_chunks;
  int stage_elems;     // elements of one shared-memory stage
  int half;            // 1: units run two to a CTA, one per half (thin tiles)
};

__host__ __device__ inline void tile_rows(const Geom& g, int nv1, int t, int* i0, int* i1,
                                          int* dir) {
  if (t < g.t_neg) {
    *i0 = t * g.ti_neg;
    *i1 = (*i0 + g.ti_neg < g.i_neg) ? *i0 + g.ti_neg : g.i_neg;
    *dir = -1;
  } else {
    const int u = t - g.t_neg;
    *i0 = g.i_neg + u * g.ti_pos;
    *i1 = (*i0 + g.ti_pos < nv1) ? *i0 + g.ti_pos : nv1;
    *dir = 1;
  }
}

struct alignas(16) StepArgs {
  const void* f_in;
  void* f_out;
  int nx, nv1, nv2, pitch;  // pitch = row stride of f in elements (>= nv2)
  const double* c1;         // [nx] signed v1-Courant numbers of f^n
  const float* c1_32;       // [nx] the same rounded to FP32
  const Params* prm;
  DevState* st;
  // BGK coefficients of the state being stepped, written by the finalize
  // kernel: bgk[k] = dt nu_k, bgk[nx + k] = dt nu_k n_k (zero when off)
  double* bgk;      // [2][nx]
  float* bgk32;     // [2][nx] the same rounded to FP32
  Tables tab;
  Partials part;
  Geom geom;
};

// Scratch of the finalize kernel: per-plane in-block prefix of n, per-block
// sums, and the counter that elects the last block (zero between launches).
struct FinScratch {
  double* pre;   // [nx]
  double* bsum;  // [blocks]
  double* blv;   // [blocks]
  int* counter;  // [1]
};

// Outputs of the finalize kernel for one grid.
struct FinOut {
  double* ne;     // [nx] n_e of the new state
  double* Ex;     // [nx] E_x
  double* c1;     // [nx] v1-Courant numbers for the next step
  float* c1_32;   // [nx] the same rounded to FP32
  double* hist;   // [hist_cap][FK_HISTORY_COLS] history ring
  FinScratch fs;
};

// One grid of a batch: the step kernel's arguments (with the batch's
// x-chunking) and the finalize kernel's outputs.
struct BatchInst {
  StepArgs a;
  FinOut o;
};

// Launchers (return the launch error).
cudaError_t launch_tables(const Tables& t, int nv1, int nv2, int pitch,
                          double v1_min, double v2_min, double dv1, double dv2,
                          double dt, double dx, double delta_max, double A_max,
                          double k_s, double T_se, double T_fe, double J_over_eW,
                          double T_e, cudaStream_t s);
int tables_scratch_doubles();
// Direct-load step (and moments-only evaluation): one block per (plane, tile).
cudaError_t launch_step(const StepArgs& a, int precision, int moments_only, cudaStream_t s);
// Streaming step: one CTA per (tile, chunk), bulk-async staged planes.
cudaError_t launch_step_stream(const StepArgs& a, int precision, bool bgk, cudaStream_t s);
// Rows per tile of the streaming kernel for this precision and row pitch
// so that two CTAs fit on an SM (half: a unit on half a CTA, two units per
// CTA; 0 if a row does not fit); the shared memory of one unit, of one
// half-CTA region and of a CTA of grid geometry gm; resident CTAs per SM of
// the kernels of a unit layout (kLayoutWhole, kLayoutHalf) or of all.
int stream_tile_rows(int precision, int pitch, int smem_per_sm, int reserved_per_block,
                     bool half);
size_t stream_smem_bytes(int precision, int stage_elems, int pitch);
size_t stream_half_bytes(int precision, int stage_elems, int pitch);
size_t stream_cta_smem_bytes(int precision, const Geom& gm, int pitch);
enum StreamLayout { kLayoutAll = 0, kLayoutWhole = 1, kLayoutHalf = 2 };
int stream_ctas_per_sm(int precision, size_t smem_bytes, int layout);
// Batched streaming step: one launch over the whole-CTA units, CTA b
// running units[b] = (grid index into inst, tile + n_tiles * chunk of that
// grid) with smem_bytes >= every such grid's stream_smem_bytes; then one
// launch over the half units, CTA b running pairs[b] = (grid, unit, grid2,
// unit2; grid2 < 0: the second half idle), each half in a region of
// half_bytes.  padded: some grid has pitch > nv2.
cudaError_t launch_step_stream_batch(const BatchInst* inst, const int2* units, int n_units,
                                     const int4* pairs, int n_pairs, int precision, bool padded,
                                     bool bgk, size_t smem_bytes, int half_bytes,
                                     cudaStream_t s);
// Batched finalize (step mode) over n_entries entries: the first n_multi
// are (grid, block) pairs, one CTA each, listing blocks 0 ..
// finalize_blocks(nx) - 1 of every grid with more than one; the rest are
// (grid, -1), one warp each, four to a CTA, for the grids of one block.
cudaError_t launch_finalize_batch(const BatchInst* inst, const int2* blocks, int n_multi,
                                  int n_entries, cudaStream_t s);
int finalize_batch_ctas(int n_multi, int n_entries);
int finalize_blocks(int nx);
cudaError_t launch_finalize(const StepArgs& a, double* ne, double* Ex, double* c1,
                            float* c1_32, double* hist, const FinScratch& fs, int mode,
                            cudaStream_t s);
cudaError_t launch_convert(const void* src, void* dst, size_t rows, int nv2, int pitch,
                           int to_f32, cudaStream_t s);

enum FinalizeMode { kModeStep = 0, kModeRefresh = 1, kModeReset = 2 };

// Error text for calls without a grid (read back by fk_last_error(NULL)).
void set_thread_error(const char* msg);

}  // namespace fk
