// Host side of the C ABI declared in include/fk.h: the grid object, its
// device buffers, parameter tables, CUDA-graph replay of the step loop and
// the synchronising getters.
//
// Paper: Sun et al., arXiv 2303.14119, Sec. 2 (model, boundary conditions,
// surface charge, convergence test).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "fk_host.cuh"

using namespace fk;

namespace {

thread_local std::string g_create_error;

constexpr int kGraphSteps = 32;  // steps per captured graph (even)
constexpr int kMaxTimed = 8192;  // step-kernel launches timed between reads
constexpr size_t kStageElems = size_t(1) << 23;  // FP64 staging chunk, 64 MB

}  // namespace

void fk::set_thread_error(const char* msg) { g_create_error = msg; }


namespace {

fk_status fail(fk_grid* g, fk_status s, const std::string& msg) {
  if (g)
    g->err = msg;
  else
    g_create_error = msg;
  return s;
}

fk_status cuda_fail(fk_grid* g, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(g, e == cudaErrorMemoryAllocation ? FK_ENOMEM : FK_ECUDA, m);
}

#define FK_CUDA(g, call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail((g), e_, #call); \
  } while (0)

}  // namespace

fk_status fk::flags_status(fk_grid* g, unsigned flags) {
  if (flags & kFlagBounds)
    return fail(g, FK_EBOUNDS, "an index of the step kernel fell outside its buffer (debug-bounds build)");
  if (flags & kFlagTimeout) return fail(g, FK_ETIMEOUT, "a bounded wait inside the step kernel ran out");
  if (flags & kFlagNegative)
    return fail(g, FK_ENEGATIVE, "f has a negative value (the state set, or a step beyond rounding)");
  if (flags & kFlagNumeric) return fail(g, FK_ENUMERIC, "a moment or flux became non-finite");
  if (flags & kFlagCfl)
    return fail(g, FK_ECFL, "|c_x| + |c_1| + |c_2| exceeds 1: the explicit upwind step is unstable");
  return FK_OK;
}

namespace {

}  // namespace

StepArgs fk::make_args(fk_grid* g, int cur) {
  StepArgs a{};
  a.f_in = g->d_f[cur];
  a.f_out = g->d_f[cur ^ 1];
  a.nx = g->nx;
  a.nv1 = g->nv1;
  a.nv2 = g->nv2;
  a.pitch = g->pitch;
  a.c1 = g->d_c1;
  a.c1_32 = g->d_c1_32;
  a.geom = g->geom;
  a.prm = g->d_prm;
  a.st = g->d_st;
  a.bgk = g->d_bgk;
  a.bgk32 = g->d_bgk32;
  a.tab = g->tab;
  a.part = g->part;
  return a;
}

namespace {

fk_status upload_params(fk_grid* g) {
  FK_CUDA(g, cudaMemcpyAsync(g->d_prm, &g->prm, sizeof(Params), cudaMemcpyHostToDevice, g->stream));
  if (g->d_prm_x) {  // an x pass of a split step: advection in x and the wall only
    g->prm_x = g->prm;
    g->prm_x.c2 = 0.0;
    g->prm_x.band_lo = g->prm_x.band_hi = 0;
    g->prm_x.collisions = 0;
    FK_CUDA(g, cudaMemcpyAsync(g->d_prm_x, &g->prm_x, sizeof(Params), cudaMemcpyHostToDevice,
                               g->stream));
  }
  return FK_OK;
}

// Synchronise, read the device scalars, and re-base the buffer bookkeeping
// on the last valid state.
}  // namespace

fk_status fk::sync_state(fk_grid* g, DevState* out) {
  return sync_state_with(g, out, nullptr, nullptr);
}

fk_status fk::sync_state_with(fk_grid* g, DevState* out, double* n_e, double* Ex) {
  FK_CUDA(g, cudaSetDevice(g->dev));
  if (g->batch_done) FK_CUDA(g, cudaStreamWaitEvent(g->stream, g->batch_done, 0));
  // every copy lands in the grid's pinned buffer; one wait for all of them
  DevState* hst = static_cast<DevState*>(g->h_stage);
  double* hv = reinterpret_cast<double*>(hst + 1);  // n_e, then E_x
  const size_t vb = (size_t)g->nx * sizeof(double);
  FK_CUDA(g, cudaMemcpyAsync(hst, g->d_st, sizeof(DevState), cudaMemcpyDeviceToHost, g->stream));
  if (n_e) FK_CUDA(g, cudaMemcpyAsync(hv, g->d_ne, vb, cudaMemcpyDeviceToHost, g->stream));
  if (Ex) FK_CUDA(g, cudaMemcpyAsync(hv + g->nx, g->d_Ex, vb, cudaMemcpyDeviceToHost, g->stream));
  FK_CUDA(g, cudaStreamSynchronize(g->stream));
  *out = *hst;
  if (n_e) memcpy(n_e, hv, vb);
  if (Ex) memcpy(Ex, hv + g->nx, vb);
  const long long adv = out->step - g->base_step;
  g->base_cur = (int)((g->base_cur + (adv & 1)) & 1);
  g->base_step = out->step;
  g->enq_cur = g->base_cur;
  g->known_flags = out->flags;
  return FK_OK;
}

namespace {
fk_status plan_geometry(fk_grid* g);
}  // namespace

namespace {
thread_local long long g_alloc_calls = 0;
}  // namespace

void fk::alloc_hook_reset() { g_alloc_calls = 0; }

cudaError_t fk::hooked_alloc(void** p, size_t bytes, bool host) {
  const char* e = getenv("FK_TEST_FAIL_ALLOC");
  if (e && *e) {
    const long long n = atoll(e);
    if (n > 0 && ++g_alloc_calls == n) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
  }
  return host ? cudaMallocHost(p, bytes) : cudaMalloc(p, bytes);
}

fk_status fk::replan_tiles(fk_grid* g, int cap) {
  // on any failure the grid keeps its previous plan and buffers
  const Geom old_geom = g->geom;
  const int old_cap = g->tile_cap;
  const bool old_stream = g->use_stream;
  auto restore = [&](fk_status s) {
    g->geom = old_geom;
    g->tile_cap = old_cap;
    g->use_stream = old_stream;
    return s;
  };
  g->tile_cap = cap;
  const fk_status s = plan_geometry(g);
  if (s != FK_OK) return restore(s);
  if (g->use_stream != old_stream) return restore(fail(g, FK_EINVAL, "the tile plan does not fit"));
  const int nu = g->geom.n_tiles;
  if (nu > g->part_cap) {  // more tiles: larger partial-sum buffers (the grid is idle)
    const size_t nparts = (size_t)g->nx * nu;
    const size_t sizes[5] = {nparts, nparts, (size_t)nu, (size_t)nu, (size_t)nu};
    double* nb[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    for (int q = 0; q < 5; q++) {
      cudaError_t e = hooked_alloc(reinterpret_cast<void**>(&nb[q]), sizes[q] * sizeof(double));
      if (e == cudaSuccess) e = cudaMemsetAsync(nb[q], 0, sizes[q] * sizeof(double), g->stream);
      if (e != cudaSuccess) {
        for (double* p : nb)
          if (p) cudaFree(p);
        return restore(cuda_fail(g, e, "allocating the partial sums of the tile plan"));
      }
    }
    const cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) {
      for (double* p : nb) cudaFree(p);
      return restore(cuda_fail(g, e, "cudaStreamSynchronize"));
    }
    double** bufs[5] = {&g->part.n, &g->part.lv, &g->part.pe, &g->part.see, &g->part.vac};
    for (int q = 0; q < 5; q++) {
      if (*bufs[q]) cudaFree(*bufs[q]);
      *bufs[q] = nb[q];
    }
    g->part_cap = nu;
  }
  g->part.nu = nu;
  for (int p = 0; p < 2; p++)  // captured with the old decomposition
    if (g->graph[p]) {
      cudaGraphExecDestroy(g->graph[p]);
      g->graph[p] = nullptr;
    }
  return FK_OK;
}

namespace {

// Evaluate the current state: moments of f, then finalize in `mode`.
fk_status evaluate(fk_grid* g, int mode) {
  StepArgs a = make_args(g, g->enq_cur);
  FK_CUDA(g, launch_step(a, g->prec, 1, g->stream));
  FK_CUDA(g, launch_finalize(a, g->d_ne, g->d_Ex, g->d_c1, g->d_c1_32, g->d_hist, g->fin, mode,
                             g->stream));
  return FK_OK;
}

// One step: the step kernel then the finalize kernel on stream s.
cudaError_t enqueue_step(fk_grid* g, int cur, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) {
  StepArgs a = make_args(g, cur);
  cudaError_t e = cudaSuccess;
  if (ev0) e = cudaEventRecord(ev0, s);
  if (e == cudaSuccess) {
    if (g->scheme != kSchemeUnsplit && g->use_stream) {
      // the split steps' passes on the streaming kernel: an x pass is the
      // fused step with c_1 = c_2 = 0, no source and no collisions (c_x / 2
      // for a Strang half pass); the velocity pass is the fused step with
      // c_x = 0.  Partial sums a pass writes that a later pass writes again
      // are overwritten; the last Strang pass sets its velocity-edge loss
      // (zero) aside, the step's is the velocity pass's.
      const bool bgk = g->prm.collisions != 0;
      float* const zero32 = reinterpret_cast<float*>(g->d_zero);
      StepArgs xp = a, vp = a;
      xp.prm = g->d_prm_x;
      xp.c1 = g->d_zero;
      xp.c1_32 = zero32;
      vp.tab.cx = g->d_zero;
      vp.tab.cx32 = zero32;
      if (g->scheme == kSchemeLie) {
        xp.f_out = g->d_f3;
        vp.f_in = g->d_f3;
        e = launch_step_stream(xp, g->prec, false, s);
        if (e == cudaSuccess) e = launch_step_stream(vp, g->prec, bgk, s);
      } else {
        xp.tab.cx = g->d_cx_half;
        xp.tab.cx32 = g->d_cx32_half;
        StepArgs x2 = xp;
        vp.f_in = a.f_out;
        vp.f_out = g->d_f3;
        x2.f_in = g->d_f3;
        x2.st = g->d_st_mid;
        x2.part.lv = g->d_lv_aside;
        e = launch_step_stream(xp, g->prec, false, s);
        if (e == cudaSuccess) e = launch_step_stream(vp, g->prec, bgk, s);
        if (e == cudaSuccess) e = launch_strang_mid(vp, g->d_st_mid, s);
        if (e == cudaSuccess) e = launch_step_stream(x2, g->prec, false, s);
      }
    } else if (g->scheme == kSchemeLie) {
      // x-advection of f^n into the intermediate buffer, then the velocity
      // step of that state into f^{n+1} (both direct-load passes)
      StepArgs ax = a, av = a;
      ax.f_out = g->d_f3;
      av.f_in = g->d_f3;
      e = launch_step_pass(ax, g->prec, kPassX, s);
      if (e == cudaSuccess) e = launch_step_pass(av, g->prec, kPassV, s);
    } else if (g->scheme == kSchemeStrang) {
      // x over dt/2 into the other state buffer, the velocity step of that
      // into the third buffer, the wall fluxes of the result (and dt/2 of
      // them into sigma and the ledger), x over dt/2 of it back into the
      // other buffer with the inflow of those fluxes
      StepArgs x1 = a, av = a, x2 = a;
      av.f_in = a.f_out;
      av.f_out = g->d_f3;
      x2.f_in = g->d_f3;
      x2.st = g->d_st_mid;
      e = launch_step_pass(x1, g->prec, kPassXHalf, s);
      if (e == cudaSuccess) e = launch_step_pass(av, g->prec, kPassV, s);
      if (e == cudaSuccess) e = launch_strang_mid(av, g->d_st_mid, s);
      if (e == cudaSuccess) e = launch_step_pass(x2, g->prec, kPassXHalfLast, s);
    } else {
      e = g->use_stream ? launch_step_stream(a, g->prec, g->prm.collisions != 0, s)
                        : launch_step(a, g->prec, 0, s);
    }
  }
  if (e == cudaSuccess && ev1) e = cudaEventRecord(ev1, s);
  if (e == cudaSuccess)
    e = launch_finalize(a, g->d_ne, g->d_Ex, g->d_c1, g->d_c1_32, g->d_hist, g->fin,
                        g->scheme == kSchemeStrang ? kModeStepStrang : kModeStep, s);
  return e;
}

// Calls that change a grid's state are refused while a batch steps it.
#define FK_NOT_IN_BATCH(g)                                                          \
  do {                                                                              \
    if ((g)->batch)                                                                 \
      return fail((g), FK_ESTATE, "the grid is stepped by a batch: destroy the batch first"); \
  } while (0)

fk_status clear_flags(fk_grid* g, unsigned mask) {
  // flags live in DevState; clear with a read-modify-write through the host
  DevState st;
  fk_status s = sync_state(g, &st);
  if (s != FK_OK) return s;
  st.flags &= ~mask;
  FK_CUDA(g, cudaMemcpyAsync(&g->d_st->flags, &st.flags, sizeof(unsigned), cudaMemcpyHostToDevice,
                             g->stream));
  g->known_flags = st.flags;
  return FK_OK;
}

fk_status rebuild_tables(fk_grid* g) {
  const double W = (g->prm.band_hi - g->prm.band_lo) * g->dx;
  const double j_over_ew = (g->J > 0.0 && W > 0.0) ? g->J / kQe / W : 0.0;
  FK_CUDA(g, launch_tables(g->tab, g->nv1, g->nv2, g->pitch, g->desc.v1_min, g->desc.v2_min,
                           g->dv1, g->dv2, g->dt, g->dx, g->delta_max, g->A_max, g->k_s,
                           g->T_se, g->T_fe, j_over_ew, g->T_e, g->stream));
  return FK_OK;
}

// The failure-detection test knobs from the environment (off by default).
void test_knobs(Params* p) {
  p->wait_limit = kWaitLimitCycles;
  p->withhold_item = -1;
  if (const char* w = getenv("FK_TEST_WAIT_CYCLES")) {
    const long long v = atoll(w);
    if (v > 0) p->wait_limit = v;
  }
  if (const char* q = getenv("FK_TEST_WITHHOLD_COPY")) {
    const int v = atoi(q);
    if (v >= 0) p->withhold_item = v;
  }
}

// Parameters changed: rebuild tables, re-evaluate the current state and
// rewrite its history row.  Clears a CFL flag (the new fields may fix it).
fk_status refresh(fk_grid* g, bool tables) {
  fk_status s = clear_flags(g, kFlagCfl);
  if (s != FK_OK) return s;
  if ((s = upload_params(g)) != FK_OK) return s;
  if (tables && (s = rebuild_tables(g)) != FK_OK) return s;
  return evaluate(g, kModeRefresh);
}

void free_grid(fk_grid* g) {
  if (!g) return;
  cudaSetDevice(g->dev);
  if (g->stream) cudaStreamSynchronize(g->stream);
  for (int p = 0; p < 2; p++)
    if (g->graph[p]) cudaGraphExecDestroy(g->graph[p]);
  void* ptrs[] = {g->d_prm, g->d_st, g->d_f[0], g->d_f[1], g->tab.v1, g->tab.cx,
                  g->tab.cx32, g->tab.delta, g->tab.gse, g->tab.src, g->tab.src32,
                  g->tab.gfe_raw, g->tab.srow32, g->tab.scol32, g->tab.tsum, g->tab.m1, g->tab.m2,
                  g->tab.m1_32, g->tab.m2_32, g->tab.v1p, g->tab.deltap,
                  g->d_bgk, g->d_bgk32, g->part.n, g->part.lv,
                  g->part.pe, g->part.see,
                  g->part.vac, g->d_ne, g->d_Ex, g->d_c1, g->d_c1_32, g->d_hist,
                  g->d_stage, g->d_f3, g->d_st_mid, g->d_prm_x, g->d_zero, g->d_cx_half,
                  g->d_cx32_half, g->d_lv_aside, g->fin.pre, g->fin.bsum, g->fin.blv,
                  g->fin.counter};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (g->h_stage) cudaFreeHost(g->h_stage);
  for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
  if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
  delete g;
}

template <typename P>
cudaError_t dalloc(P** p, size_t bytes) {
  return hooked_alloc(reinterpret_cast<void**>(p), bytes ? bytes : 16);
}

// The buffers a time scheme needs beyond the two state buffers: a third
// buffer of f for the split steps, and the Strang step's second state block.
fk_status split_buffers(fk_grid* g, int scheme) {
  if (scheme != kSchemeUnsplit && !g->d_f3)
    FK_CUDA(g, dalloc(&g->d_f3, (size_t)g->nx * g->nv1 * g->pitch * g->esize));
  if (scheme == kSchemeStrang && !g->d_st_mid) {
    FK_CUDA(g, dalloc(&g->d_st_mid, sizeof(DevState)));
    FK_CUDA(g, cudaMemsetAsync(g->d_st_mid, 0, sizeof(DevState), g->stream));
  }
  if (scheme != kSchemeUnsplit && g->use_stream && !g->d_prm_x) {
    // the passes run on the streaming kernel (the tables of c_x are final
    // since creation, the parameters are re-uploaded with every setter)
    const size_t nz = (size_t)std::max(g->nx, g->nv1);
    FK_CUDA(g, dalloc(&g->d_zero, nz * sizeof(double)));
    FK_CUDA(g, cudaMemsetAsync(g->d_zero, 0, nz * sizeof(double), g->stream));
    FK_CUDA(g, dalloc(&g->d_cx_half, g->nv1 * sizeof(double)));
    FK_CUDA(g, dalloc(&g->d_cx32_half, g->nv1 * sizeof(float)));
    FK_CUDA(g, launch_scale_tables(g->tab.cx, g->tab.cx32, 0.5, g->nv1, g->d_cx_half,
                                   g->d_cx32_half, g->stream));
    // at most one tile per v1 row
    FK_CUDA(g, dalloc(&g->d_lv_aside, (size_t)g->nx * g->nv1 * sizeof(double)));
    FK_CUDA(g, dalloc(&g->d_prm_x, sizeof(Params)));
    const fk_status s = upload_params(g);
    if (s != FK_OK) return s;
  }
  return FK_OK;
}

fk_status build_graph(fk_grid* g, int parity) {
  cudaStream_t cs = g->cap_stream;
  FK_CUDA(g, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  int cur = parity;
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < kGraphSteps && e == cudaSuccess; s++) {
    e = enqueue_step(g, cur, cs, nullptr, nullptr);
    cur ^= 1;
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(g, e, "capturing the step graph");
  }
  if (e2 != cudaSuccess) return cuda_fail(g, e2, "cudaStreamEndCapture");
  cudaError_t e3 = cudaGraphInstantiate(&g->graph[parity], graph, 0);
  cudaGraphDestroy(graph);
  if (e3 != cudaSuccess) return cuda_fail(g, e3, "cudaGraphInstantiate");
  return FK_OK;
}

// Tiles of v1 rows (never straddling the sign change of v1) and chunks of
// x-planes: one streaming unit per (tile, chunk), about one wave of them.
// Where each sign half of the v1 rows fits the tile of a half-CTA unit,
// units run two to a CTA (FK_STREAM_HALF=0 keeps one unit per CTA).
fk_status plan_geometry(fk_grid* g) {
  if (g->env_direct < 0) {  // the environment's choices hold for the grid's life
    const char* env = getenv("FK_STEP_KERNEL");
    const char* env_half = getenv("FK_STREAM_HALF");
    g->env_direct = env && strcmp(env, "direct") == 0;
    g->env_no_half = env_half && strcmp(env_half, "0") == 0;
  }
  FK_CUDA(g, cudaSetDevice(g->dev));
  int sms = 0, smem_sm = 0, reserved = 0;
  FK_CUDA(g, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->dev));
  FK_CUDA(g, cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, g->dev));
  FK_CUDA(g, cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, g->dev));
  int ti_max = stream_tile_rows(g->prec, g->pitch, smem_sm, reserved, false);
  g->use_stream = ti_max > 0 && !g->env_direct;
  if (!g->use_stream) ti_max = std::max(1, 4096 / g->pitch);
  int i_neg = 0;
  for (int i = 0; i < g->nv1; i++)
    if (g->desc.v1_min + ((double)i + 0.5) * g->dv1 <= 0.0) i_neg++;
  Geom& m = g->geom;
  m.i_neg = i_neg;
  m.half = 0;
  if (g->use_stream && !g->env_no_half) {
    const int ti_half = stream_tile_rows(g->prec, g->pitch, smem_sm, reserved, true);
    if (ti_half > 0 && std::max(i_neg, g->nv1 - i_neg) <= ti_half) {
      m.half = 1;
      ti_max = ti_half;
    }
  }
  if (g->use_stream && !m.half && g->tile_cap > 0) ti_max = std::min(ti_max, g->tile_cap);
  auto split = [&](int rows, int* nt, int* ti) {
    if (rows <= 0) {
      *nt = 0;
      *ti = 1;
      return;
    }
    *nt = (rows + ti_max - 1) / ti_max;
    *ti = (rows + *nt - 1) / *nt;
  };
  int t_pos = 0;
  split(i_neg, &m.t_neg, &m.ti_neg);
  split(g->nv1 - i_neg, &t_pos, &m.ti_pos);
  m.n_tiles = m.t_neg + t_pos;
  m.stage_elems = (std::max(m.ti_neg, m.ti_pos) + (g->use_stream ? 1 : 2)) * g->pitch;
  m.n_chunks = 1;
  m.chunk_len = g->nx;
  if (g->use_stream) {
    const int per_sm = stream_ctas_per_sm(g->prec, stream_cta_smem_bytes(g->prec, m, g->pitch),
                                          m.half ? kLayoutHalf : kLayoutWhole);
    if (per_sm <= 0) {
      g->use_stream = false;
      m.half = 0;
    } else {
      // about one wave: (tiles x chunks) units for the resident slots, and
      // at least 4 planes per chunk (the upwind plane is loaded once per chunk)
      const int slots = sms * per_sm * (m.half ? 2 : 1);
      const int nc = std::max(1, std::min(slots / m.n_tiles, (g->nx + 3) / 4));
      m.chunk_len = (g->nx + nc - 1) / nc;
      m.n_chunks = (g->nx + m.chunk_len - 1) / m.chunk_len;
    }
  }
  return FK_OK;
}

}  // namespace

extern "C" {

fk_status fk_create_grid(const fk_grid_desc* desc, void* cuda_stream, fk_grid** out) {
  g_create_error.clear();
  alloc_hook_reset();
  if (!desc || !out) return fail(nullptr, FK_EINVAL, "desc and out must not be NULL");
  *out = nullptr;
  const fk_grid_desc& d = *desc;
  if (d.nx < 2 || d.nv1 < 2 || d.nv2 < 2)
    return fail(nullptr, FK_EINVAL, "nx, nv1, nv2 must be >= 2");
  if (d.nv1 > (1 << 16) || d.nv2 > (1 << 16) || d.nx > 8192)
    return fail(nullptr, FK_EINVAL, "grid too large: nx <= 8192, nv1, nv2 <= 65536");
  if (!(d.h_max > 0) || !(d.v1_min < d.v1_max) || !(d.v2_min < d.v2_max) ||
      !isfinite(d.h_max) || !isfinite(d.v1_min) || !isfinite(d.v1_max) ||
      !isfinite(d.v2_min) || !isfinite(d.v2_max))
    return fail(nullptr, FK_EINVAL, "need h_max > 0, v1_min < v1_max, v2_min < v2_max, finite");
  if (!(d.dt > 0) && !(d.cfl > 0))
    return fail(nullptr, FK_EINVAL, "need dt > 0 or cfl > 0");
  if (d.precision != FK_F64 && d.precision != FK_F32)
    return fail(nullptr, FK_EINVAL, "precision must be FK_F64 or FK_F32");
  if (d.history_capacity < 0) return fail(nullptr, FK_EINVAL, "history_capacity must be >= 0");

  fk_grid* g = new (std::nothrow) fk_grid();
  if (!g) return fail(nullptr, FK_ENOMEM, "host allocation failed");
  g->desc = d;
  g->dev = d.device;
  g->prec = d.precision;
  g->nx = d.nx;
  g->nv1 = d.nv1;
  g->nv2 = d.nv2;
  g->esize = d.precision == FK_F32 ? 4 : 8;
  const int align = (int)(16 / g->esize);  // 16-byte rows
  g->pitch = (d.nv2 + align - 1) / align * align;
  g->dx = d.h_max / d.nx;
  g->dv1 = (d.v1_max - d.v1_min) / d.nv1;
  g->dv2 = (d.v2_max - d.v2_min) / d.nv2;
  const double vmax = fmax(fabs(d.v1_min), fabs(d.v1_max));
  g->dt = d.dt > 0 ? d.dt : d.cfl * g->dx / vmax;
  double cx_max = 0.0;
  for (int i = 0; i < d.nv1; i++)
    cx_max = fmax(cx_max, fabs(d.v1_min + (i + 0.5) * g->dv1) * g->dt / g->dx);

  Params& p = g->prm;
  p.dx = g->dx;
  p.dv1 = g->dv1;
  p.dv2 = g->dv2;
  p.dt = g->dt;
  p.Ey = 0;
  p.Ex_ext = 0;
  p.c2 = 0;
  p.cx_max = cx_max;
  p.inj = 0;
  p.sat_tol = 1e-3;
  // Gauss's law from the wall (E_x(0) = sigma / (2 eps0), space charge -e n)
  // and the v1-Courant number c_1 = a1 dt / dv1 with a1 = -e E_x / m_e
  p.ex_sigma = 1.0 / (2.0 * kEps0);
  p.ex_n = kQe / kEps0 * g->dx;
  p.c1_per_ex = -kQe / kMe * g->dt / g->dv1;
  p.dvv = g->dv1 * g->dv2;
  p.lv_scale = g->dx * g->dv1 * g->dv2 / g->dt;
  p.sat_window = 10000;
  p.hist_cap = d.history_capacity > 0 ? d.history_capacity : 65536;
  p.self_consistent = 1;
  p.see_enabled = 0;
  p.collisions = 0;
  p.bgk_c = 0.0;
  p.refl = 0.0;
  p.band_lo = p.band_hi = 0;
  if (p.sat_window >= p.hist_cap) p.sat_window = p.hist_cap - 1;
  test_knobs(&p);
  if (cx_max > 1.0 + 1e-12) {
    delete g;
    return fail(nullptr, FK_ECFL, "max |v1| dt / dx exceeds 1");
  }

#define CREATE_CUDA(call)                                     \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) {                                  \
      fk_status s_ = cuda_fail(nullptr, e_, #call);           \
      free_grid(g);                                           \
      return s_;                                              \
    }                                                         \
  } while (0)

  CREATE_CUDA(cudaSetDevice(g->dev));
  if (cuda_stream) {
    g->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    CREATE_CUDA(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
    g->own_stream = true;
  }
  CREATE_CUDA(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
  const size_t nv = (size_t)d.nv1 * g->pitch;  // 2D tables use the row pitch
  const size_t fbytes = (size_t)d.nx * d.nv1 * g->pitch * g->esize;
  {
    fk_status gs = plan_geometry(g);
    if (gs != FK_OK) {
      g_create_error = g->err;
      free_grid(g);
      return gs;
    }
  }
  g->part.nu = g->geom.n_tiles;
  g->part_cap = g->part.nu;
  const size_t nparts = (size_t)d.nx * g->part.nu;
  CREATE_CUDA(dalloc(&g->d_prm, sizeof(Params)));
  CREATE_CUDA(dalloc(&g->d_st, sizeof(DevState)));
  CREATE_CUDA(hooked_alloc(&g->h_stage, sizeof(DevState) + 2 * (size_t)d.nx * sizeof(double),
                           true));
  CREATE_CUDA(dalloc(&g->d_f[0], fbytes));
  CREATE_CUDA(dalloc(&g->d_f[1], fbytes));
  CREATE_CUDA(dalloc(&g->tab.v1, d.nv1 * sizeof(double)));
  CREATE_CUDA(dalloc(&g->tab.cx, d.nv1 * sizeof(double)));
  CREATE_CUDA(dalloc(&g->tab.cx32, d.nv1 * sizeof(float)));
  CREATE_CUDA(dalloc(&g->tab.delta, nv * sizeof(double)));
  CREATE_CUDA(dalloc(&g->tab.gse, nv * sizeof(double)));
  CREATE_CUDA(dalloc(&g->tab.src, nv * sizeof(double)));
  CREATE_CUDA(dalloc(&g->tab.src32, nv * sizeof(float)));
  CREATE_CUDA(dalloc(&g->tab.gfe_raw, nv * sizeof(double)));
  CREATE_CUDA(dalloc(&g->tab.srow32, d.nv1 * sizeof(float)));
  CREATE_CUDA(dalloc(&g->tab.scol32, g->pitch * sizeof(float)));
  CREATE_CUDA(dalloc(&g->tab.tsum, tables_scratch_doubles() * sizeof(double)));
  CREATE_CUDA(dalloc(&g->tab.m1, d.nv1 * sizeof(double)));
  CREATE_CUDA(dalloc(&g->tab.m2, g->pitch * sizeof(double)));
  CREATE_CUDA(dalloc(&g->tab.m1_32, d.nv1 * sizeof(float)));
  CREATE_CUDA(dalloc(&g->tab.m2_32, g->pitch * sizeof(float)));
  CREATE_CUDA(dalloc(&g->tab.v1p, d.nv1 * sizeof(float2)));
  CREATE_CUDA(dalloc(&g->tab.deltap, nv * sizeof(float2)));
  CREATE_CUDA(dalloc(&g->d_bgk, 2 * (size_t)d.nx * sizeof(double)));
  CREATE_CUDA(dalloc(&g->d_bgk32, 2 * (size_t)d.nx * sizeof(float)));
  CREATE_CUDA(cudaMemsetAsync(g->d_bgk, 0, 2 * (size_t)d.nx * sizeof(double), g->stream));
  CREATE_CUDA(cudaMemsetAsync(g->d_bgk32, 0, 2 * (size_t)d.nx * sizeof(float), g->stream));
  CREATE_CUDA(dalloc(&g->part.n, nparts * sizeof(double)));
  CREATE_CUDA(dalloc(&g->part.lv, nparts * sizeof(double)));
  CREATE_CUDA(dalloc(&g->part.pe, g->part.nu * sizeof(double)));
  CREATE_CUDA(dalloc(&g->part.see, g->part.nu * sizeof(double)));
  CREATE_CUDA(dalloc(&g->part.vac, g->part.nu * sizeof(double)));
  CREATE_CUDA(dalloc(&g->d_ne, d.nx * sizeof(double)));
  CREATE_CUDA(dalloc(&g->d_Ex, d.nx * sizeof(double)));
  CREATE_CUDA(dalloc(&g->d_c1, d.nx * sizeof(double)));
  CREATE_CUDA(dalloc(&g->d_c1_32, d.nx * sizeof(float)));
  CREATE_CUDA(dalloc(&g->fin.pre, d.nx * sizeof(double)));
  CREATE_CUDA(dalloc(&g->fin.bsum, finalize_blocks(d.nx) * sizeof(double)));
  CREATE_CUDA(dalloc(&g->fin.blv, finalize_blocks(d.nx) * sizeof(double)));
  CREATE_CUDA(dalloc(&g->fin.counter, sizeof(int)));
  CREATE_CUDA(cudaMemsetAsync(g->fin.counter, 0, sizeof(int), g->stream));
  CREATE_CUDA(dalloc(&g->d_hist, (size_t)p.hist_cap * FK_HISTORY_COLS * sizeof(double)));
  CREATE_CUDA(cudaMemsetAsync(g->d_f[0], 0, fbytes, g->stream));
  CREATE_CUDA(cudaMemsetAsync(g->d_f[1], 0, fbytes, g->stream));
  CREATE_CUDA(cudaMemsetAsync(g->d_st, 0, sizeof(DevState), g->stream));
  CREATE_CUDA(cudaMemsetAsync(g->part.pe, 0, g->part.nu * sizeof(double), g->stream));
  CREATE_CUDA(cudaMemsetAsync(g->part.see, 0, g->part.nu * sizeof(double), g->stream));
  CREATE_CUDA(cudaMemsetAsync(g->part.vac, 0, g->part.nu * sizeof(double), g->stream));
  CREATE_CUDA(cudaMemsetAsync(g->part.lv, 0, nparts * sizeof(double), g->stream));
#undef CREATE_CUDA
  fk_status s = upload_params(g);
  if (s == FK_OK) s = rebuild_tables(g);
  if (s == FK_OK) s = evaluate(g, kModeReset);
  if (s == FK_OK) {
    DevState st;
    s = sync_state(g, &st);
  }
  if (s != FK_OK) {
    g_create_error = g->err;
    free_grid(g);
    return s;
  }
  *out = g;
  return FK_OK;
}

fk_status fk_destroy_grid(fk_grid* g) {
  if (g) FK_NOT_IN_BATCH(g);
  free_grid(g);
  return FK_OK;
}

fk_status fk_set_fields(fk_grid* g, double Ey, int self_consistent, double Ex_external) {
  if (!g) return FK_EINVAL;
  FK_NOT_IN_BATCH(g);
  if (!(Ey <= 0.0) || !isfinite(Ey) || !isfinite(Ex_external))
    return fail(g, FK_EINVAL, "E_y must be finite and <= 0 (cathode on the left); E_x finite");
  g->Ey = Ey;
  g->Ex_ext = Ex_external;
  g->self_consistent = self_consistent ? 1 : 0;
  g->prm.Ey = Ey;
  g->prm.Ex_ext = Ex_external;
  g->prm.self_consistent = g->self_consistent;
  g->prm.c2 = (-kQe * Ey / kMe) * g->dt / g->dv2;
  return refresh(g, false);  // the tables do not depend on the fields
}

fk_status fk_set_see(fk_grid* g, double delta_max, double A_max_eV, double k_s, double T_se_eV,
                     int enabled) {
  if (!g) return FK_EINVAL;
  FK_NOT_IN_BATCH(g);
  if (!(delta_max >= 0.0) || !(A_max_eV > 0.0) || !(k_s >= 0.0) || !(T_se_eV > 0.0) ||
      !isfinite(delta_max) || !isfinite(A_max_eV) || !isfinite(k_s) || !isfinite(T_se_eV))
    return fail(g, FK_EINVAL, "need delta_max >= 0, A_max > 0, k_s >= 0, T_se > 0");
  g->delta_max = delta_max;
  g->A_max = A_max_eV;
  g->k_s = k_s;
  g->T_se = T_se_eV;
  g->see_enabled = enabled ? 1 : 0;
  g->prm.see_enabled = g->see_enabled;
  return refresh(g, true);
}

fk_status fk_set_source(fk_grid* g, double J, double x_lo, double x_hi, double T_fe_eV) {
  if (!g) return FK_EINVAL;
  FK_NOT_IN_BATCH(g);
  if (!(J >= 0.0) || !(x_lo <= x_hi) || !(T_fe_eV > 0.0) || !isfinite(J) || !isfinite(T_fe_eV))
    return fail(g, FK_EINVAL, "need J >= 0, x_lo <= x_hi, T_fe > 0");
  int lo = -1, hi = -1;
  for (int k = 0; k < g->nx; k++) {
    const double x = (k + 0.5) * g->dx;
    if (x >= x_lo && x <= x_hi) {
      if (lo < 0) lo = k;
      hi = k + 1;
    }
  }
  if (J > 0.0 && lo < 0) return fail(g, FK_EINVAL, "no cell centre lies in [x_lo, x_hi]");
  g->J = J;
  g->x_lo = x_lo;
  g->x_hi = x_hi;
  g->T_fe = T_fe_eV;
  if (J > 0.0) {
    g->prm.band_lo = lo;
    g->prm.band_hi = hi;
    g->prm.inj = J / kQe;
  } else {
    g->prm.band_lo = g->prm.band_hi = 0;
    g->prm.inj = 0.0;
  }
  return refresh(g, true);
}

fk_status fk_fowler_nordheim(double E, double phi_V, double* log_J, double* J) {
  if (!(E > 0.0) || !(phi_V > 0.0) || !isfinite(E) || !isfinite(phi_V))
    return fail(nullptr, FK_EINVAL, "fk_fowler_nordheim: need E > 0 and phi > 0, finite");
  // Eq. 6 with the work function W = e phi (J) and Planck's constant
  // h = 6.62607015e-34 J s; ln J keeps the exponent from underflowing
  const double h = 6.62607015e-34;
  const double W = kQe * phi_V;
  const double ln_pre = log(kQe * kQe * kQe / (8.0 * kPi * h * W));
  const double B = 8.0 * kPi * sqrt(2.0 * kMe * W * W * W) / (3.0 * kQe * h);
  const double lj = ln_pre + 2.0 * log(E) - B / E;
  if (log_J) *log_J = lj;
  if (J) *J = exp(lj);  // 0 when it underflows
  return FK_OK;
}

fk_status fk_set_source_fn(fk_grid* g, double E_ctj, double phi_V, double x_lo, double x_hi,
                           double T_fe_eV) {
  if (!g) return FK_EINVAL;
  double J = 0.0;
  if (fk_fowler_nordheim(E_ctj, phi_V, nullptr, &J) != FK_OK)
    return fail(g, FK_EINVAL, "need E_ctj > 0 and phi > 0");
  return fk_set_source(g, J, x_lo, x_hi, T_fe_eV);
}

fk_status fk_set_collisions(fk_grid* g, double T_e_eV, double ln_lambda, int enabled) {
  if (!g) return FK_EINVAL;
  FK_NOT_IN_BATCH(g);
  if (!(T_e_eV > 0.0) || !(ln_lambda >= 0.0) || !isfinite(T_e_eV) || !isfinite(ln_lambda))
    return fail(g, FK_EINVAL, "need T_e > 0 and ln(Lambda) >= 0, finite");
  g->T_e = T_e_eV;
  g->ln_lambda = ln_lambda;
  // Eq. 4 without n_e, times dt: dt nu_ee(x) = bgk_c * n_e(x)
  const double T = T_e_eV * kQe;
  const double per_n = kQe * kQe * kQe * kQe * ln_lambda /
                       (12.0 * pow(kPi, 1.5) * kEps0 * kEps0 * sqrt(kMe) * pow(T, 1.5));
  g->prm.bgk_c = g->dt * per_n;
  const int on = enabled ? 1 : 0;
  if (on != g->prm.collisions) {
    // the captured graphs hold the step kernel of the other variant
    FK_CUDA(g, cudaStreamSynchronize(g->stream));
    for (int q = 0; q < 2; q++)
      if (g->graph[q]) {
        cudaGraphExecDestroy(g->graph[q]);
        g->graph[q] = nullptr;
      }
  }
  g->prm.collisions = on;
  if (!on) {
    FK_CUDA(g, cudaMemsetAsync(g->d_bgk, 0, 2 * (size_t)g->nx * sizeof(double), g->stream));
    FK_CUDA(g, cudaMemsetAsync(g->d_bgk32, 0, 2 * (size_t)g->nx * sizeof(float), g->stream));
  }
  return refresh(g, true);  // tables (equilibrium factors) and coefficients of the state
}

fk_status fk_set_reflection(fk_grid* g, double R_f) {
  if (!g) return FK_EINVAL;
  FK_NOT_IN_BATCH(g);
  if (!(R_f >= 0.0 && R_f <= 1.0)) return fail(g, FK_EINVAL, "need 0 <= R_f <= 1");
  if (R_f > 0.0 && fabs(g->desc.v1_min + g->desc.v1_max) > 1e-12 * fabs(g->desc.v1_max))
    return fail(g, FK_EINVAL, "reflection needs a v1 grid symmetric about 0");
  g->prm.refl = R_f;
  return refresh(g, false);  // the state's Gamma_see changes with R_f
}

fk_status fk_set_scheme(fk_grid* g, int scheme) {
  if (!g) return FK_EINVAL;
  FK_NOT_IN_BATCH(g);
  if (scheme != FK_SCHEME_UNSPLIT && scheme != FK_SCHEME_LIE && scheme != FK_SCHEME_STRANG)
    return fail(g, FK_EINVAL,
                "scheme must be FK_SCHEME_UNSPLIT, FK_SCHEME_LIE or FK_SCHEME_STRANG");
  FK_CUDA(g, cudaSetDevice(g->dev));
  {
    const fk_status bs = split_buffers(g, scheme);
    if (bs != FK_OK) return bs;
  }
  if (scheme != g->scheme) {
    // the captured graphs hold the other scheme's kernels
    FK_CUDA(g, cudaStreamSynchronize(g->stream));
    for (int q = 0; q < 2; q++)
      if (g->graph[q]) {
        cudaGraphExecDestroy(g->graph[q]);
        g->graph[q] = nullptr;
      }
  }
  g->scheme = scheme;
  return FK_OK;
}

fk_status fk_set_convergence(fk_grid* g, int64_t window, double rel_tol) {
  if (!g) return FK_EINVAL;
  FK_NOT_IN_BATCH(g);
  if (window < 1 || window >= g->prm.hist_cap || !(rel_tol >= 0.0))
    return fail(g, FK_EINVAL, "need 1 <= window < history_capacity and rel_tol >= 0");
  g->prm.sat_window = window;
  g->prm.sat_tol = rel_tol;
  return upload_params(g);
}

fk_status fk_step(fk_grid* g, int64_t n) {
  if (!g) return FK_EINVAL;
  const NvtxRange range("fk_step");
  FK_NOT_IN_BATCH(g);
  if (n < 0) return fail(g, FK_EINVAL, "n must be >= 0");
  if (g->known_flags) return flags_status(g, g->known_flags);
  FK_CUDA(g, cudaSetDevice(g->dev));
  while (n > 0) {
    if (g->timing) {
      const bool rec = g->ev_used < kMaxTimed;
      FK_CUDA(g, enqueue_step(g, g->enq_cur, g->stream, rec ? g->ev[2 * g->ev_used] : nullptr,
                              rec ? g->ev[2 * g->ev_used + 1] : nullptr));
      if (rec) g->ev_used++;
      g->enq_cur ^= 1;
      n -= 1;
    } else if (n >= kGraphSteps) {
      if (!g->graph[g->enq_cur]) {
        fk_status s = build_graph(g, g->enq_cur);
        if (s != FK_OK) return s;
      }
      FK_CUDA(g, cudaGraphLaunch(g->graph[g->enq_cur], g->stream));
      n -= kGraphSteps;  // even: the current buffer is unchanged
    } else {
      FK_CUDA(g, enqueue_step(g, g->enq_cur, g->stream, nullptr, nullptr));
      g->enq_cur ^= 1;
      n -= 1;
    }
  }
  return FK_OK;
}

fk_status fk_sync(fk_grid* g) {
  if (!g) return FK_EINVAL;
  DevState st;
  fk_status s = sync_state(g, &st);
  if (s != FK_OK) return s;
  return flags_status(g, st.flags);
}

fk_status fk_moments(fk_grid* g, double* n_e, double* Ex, double* gamma_pe, double* gamma_see) {
  if (!g) return FK_EINVAL;
  DevState st;
  fk_status s = sync_state_with(g, &st, n_e, Ex);
  if (s != FK_OK) return s;
  if (gamma_pe) *gamma_pe = st.g_pe;
  if (gamma_see) *gamma_see = st.g_see;
  return flags_status(g, st.flags);
}

fk_status fk_surface_charge(fk_grid* g, double* sigma) {
  if (!g || !sigma) return FK_EINVAL;
  DevState st;
  fk_status s = sync_state(g, &st);
  if (s != FK_OK) return s;
  *sigma = st.sigma;
  return flags_status(g, st.flags);
}

fk_status fk_history(fk_grid* g, double* out, int64_t max_rows, int64_t* rows) {
  if (!g || !rows || (max_rows > 0 && !out)) return FK_EINVAL;
  DevState st;
  fk_status s = sync_state(g, &st);
  if (s != FK_OK) return s;
  const long long cap = g->prm.hist_cap;
  // rows 0..step are stored (the ring keeps the last cap of them)
  const long long total = st.step + 1;
  long long n = std::min<long long>(std::min<long long>(max_rows, total), cap);
  if (n < 0) n = 0;
  const long long first = total - n;
  for (long long r = 0; r < n;) {
    const long long slot = (first + r) % cap;
    const long long run = std::min<long long>(n - r, cap - slot);
    FK_CUDA(g, cudaMemcpy(out + r * FK_HISTORY_COLS, g->d_hist + slot * FK_HISTORY_COLS,
                          run * FK_HISTORY_COLS * sizeof(double), cudaMemcpyDeviceToHost));
    r += run;
  }
  *rows = n;
  return flags_status(g, st.flags);
}

fk_status fk_ledger(fk_grid* g, double* out) {
  if (!g || !out) return FK_EINVAL;
  DevState st;
  fk_status s = sync_state(g, &st);
  if (s != FK_OK) return s;
  out[0] = st.n_tot;
  out[1] = st.n0;
  out[2] = st.cum_emit;
  out[3] = st.cum_pe;
  out[4] = st.cum_vac;
  out[5] = st.cum_lv;
  out[6] = st.cum_inj;
  out[7] = st.sigma0;
  out[8] = st.cum_see;
  return flags_status(g, st.flags);
}

fk_status fk_step_count(fk_grid* g, int64_t* step, int64_t* saturated_step) {
  if (!g) return FK_EINVAL;
  DevState st;
  fk_status s = sync_state(g, &st);
  if (s != FK_OK) return s;
  if (step) *step = st.step;
  if (saturated_step) *saturated_step = st.sat_step;
  return flags_status(g, st.flags);
}

fk_status fk_get_f(fk_grid* g, double* host_f) {
  if (!g || !host_f) return FK_EINVAL;
  DevState st;
  fk_status s = sync_state(g, &st);
  if (s != FK_OK) return s;
  const void* src = g->d_f[g->base_cur];
  const size_t rows = (size_t)g->nx * g->nv1;
  if (g->prec == FK_F64) {
    FK_CUDA(g, cudaMemcpy2D(host_f, g->nv2 * sizeof(double), src, g->pitch * sizeof(double),
                            g->nv2 * sizeof(double), rows, cudaMemcpyDeviceToHost));
  } else {
    if (!g->d_stage) FK_CUDA(g, dalloc(&g->d_stage, kStageElems * sizeof(double)));
    const size_t rows_per = std::max<size_t>(1, kStageElems / g->nv2);
    for (size_t r0 = 0; r0 < rows; r0 += rows_per) {
      const size_t nr = std::min(rows_per, rows - r0);
      FK_CUDA(g, launch_convert(static_cast<const float*>(src) + r0 * g->pitch, g->d_stage, nr,
                                g->nv2, g->pitch, 0, g->stream));
      FK_CUDA(g, cudaMemcpyAsync(host_f + r0 * g->nv2, g->d_stage, nr * g->nv2 * sizeof(double),
                                 cudaMemcpyDeviceToHost, g->stream));
      FK_CUDA(g, cudaStreamSynchronize(g->stream));
    }
  }
  return flags_status(g, st.flags);
}

fk_status fk_set_f(fk_grid* g, const double* host_f) {
  if (!g || !host_f) return FK_EINVAL;
  FK_NOT_IN_BATCH(g);
  DevState st;
  fk_status s = sync_state(g, &st);
  if (s != FK_OK) return s;
  void* dst = g->d_f[0];
  const size_t rows = (size_t)g->nx * g->nv1;
  if (g->prec == FK_F64) {
    FK_CUDA(g, cudaMemcpy2DAsync(dst, g->pitch * sizeof(double), host_f, g->nv2 * sizeof(double),
                                 g->nv2 * sizeof(double), rows, cudaMemcpyHostToDevice, g->stream));
  } else {
    if (!g->d_stage) FK_CUDA(g, dalloc(&g->d_stage, kStageElems * sizeof(double)));
    const size_t rows_per = std::max<size_t>(1, kStageElems / g->nv2);
    for (size_t r0 = 0; r0 < rows; r0 += rows_per) {
      const size_t nr = std::min(rows_per, rows - r0);
      FK_CUDA(g, cudaMemcpyAsync(g->d_stage, host_f + r0 * g->nv2, nr * g->nv2 * sizeof(double),
                                 cudaMemcpyHostToDevice, g->stream));
      FK_CUDA(g, launch_convert(g->d_stage, static_cast<float*>(dst) + r0 * g->pitch, nr, g->nv2,
                                g->pitch, 1, g->stream));
      FK_CUDA(g, cudaStreamSynchronize(g->stream));  // staging buffer reuse
    }
  }
  g->base_cur = g->enq_cur = 0;
  g->base_step = 0;
  // every sticky flag belongs to the replaced state
  FK_CUDA(g, cudaMemsetAsync(&g->d_st->flags, 0, sizeof(unsigned), g->stream));
  g->known_flags = 0;
  s = evaluate(g, kModeReset);
  if (s != FK_OK) return s;
  if ((s = sync_state(g, &st)) != FK_OK) return s;
  return flags_status(g, st.flags);
}

fk_status fk_get_f32(fk_grid* g, float* host_f) {
  if (!g || !host_f) return FK_EINVAL;
  if (g->prec != FK_F32) return fail(g, FK_EINVAL, "fk_get_f32 needs an FP32 grid");
  DevState st;
  fk_status s = sync_state(g, &st);
  if (s != FK_OK) return s;
  // one strided copy from the row-pitch layout to the dense host array
  FK_CUDA(g, cudaMemcpy2DAsync(host_f, g->nv2 * sizeof(float), g->d_f[g->base_cur],
                               g->pitch * sizeof(float), g->nv2 * sizeof(float),
                               (size_t)g->nx * g->nv1, cudaMemcpyDeviceToHost, g->stream));
  FK_CUDA(g, cudaStreamSynchronize(g->stream));
  return flags_status(g, st.flags);
}

fk_status fk_set_f32(fk_grid* g, const float* host_f) {
  if (!g || !host_f) return FK_EINVAL;
  FK_NOT_IN_BATCH(g);
  if (g->prec != FK_F32) return fail(g, FK_EINVAL, "fk_set_f32 needs an FP32 grid");
  DevState st;
  fk_status s = sync_state(g, &st);
  if (s != FK_OK) return s;
  FK_CUDA(g, cudaMemcpy2DAsync(g->d_f[0], g->pitch * sizeof(float), host_f,
                               g->nv2 * sizeof(float), g->nv2 * sizeof(float),
                               (size_t)g->nx * g->nv1, cudaMemcpyHostToDevice, g->stream));
  g->base_cur = g->enq_cur = 0;
  g->base_step = 0;
  FK_CUDA(g, cudaMemsetAsync(&g->d_st->flags, 0, sizeof(unsigned), g->stream));
  g->known_flags = 0;
  s = evaluate(g, kModeReset);
  if (s != FK_OK) return s;
  if ((s = sync_state(g, &st)) != FK_OK) return s;
  return flags_status(g, st.flags);
}

fk_status fk_set_surface_charge(fk_grid* g, double sigma) {
  if (!g || !isfinite(sigma)) return g ? fail(g, FK_EINVAL, "sigma must be finite") : FK_EINVAL;
  FK_NOT_IN_BATCH(g);
  DevState st;
  fk_status s = sync_state(g, &st);
  if (s != FK_OK) return s;
  FK_CUDA(g, cudaMemcpyAsync(&g->d_st->sigma, &sigma, sizeof(double), cudaMemcpyHostToDevice,
                             g->stream));
  FK_CUDA(g, cudaMemsetAsync(&g->d_st->flags, 0, sizeof(unsigned), g->stream));
  g->known_flags = 0;
  g->base_step = 0;  // the reset below restarts the step count
  s = evaluate(g, kModeReset);
  if (s != FK_OK) return s;
  if ((s = sync_state(g, &st)) != FK_OK) return s;
  return flags_status(g, st.flags);
}

// ---- checkpoints: everything a continued run depends on, so that a grid
// restored from a checkpoint steps on bit for bit as the original would.
namespace {

struct StateHeader {
  char magic[8];
  int32_t nx, nv1, nv2, precision, pitch, scheme;
  int64_t hist_cap, f_bytes;
  // parameters as set (the tables are rebuilt from them)
  double Ey, Ex_ext, delta_max, A_max, k_s, T_se, J, x_lo, x_hi, T_fe, T_e, ln_lambda;
  int32_t self_consistent, see_enabled;
  Params prm;
  DevState st;
};
constexpr char kStateMagic[8] = {'F', 'K', 'S', 'T', 'A', 'T', 'E', '1'};

size_t f_bytes(const fk_grid* g) { return (size_t)g->nx * g->nv1 * g->pitch * g->esize; }

// bytes after the header: f, then ne, Ex, c1 (double [nx]), c1_32 (float
// [nx]), bgk (double [2 nx]), bgk32 (float [2 nx]), history ring
size_t state_bytes(const fk_grid* g) {
  return sizeof(StateHeader) + f_bytes(g) + 3 * g->nx * sizeof(double) + g->nx * sizeof(float) +
         2 * g->nx * sizeof(double) + 2 * g->nx * sizeof(float) +
         (size_t)g->prm.hist_cap * FK_HISTORY_COLS * sizeof(double);
}

}  // namespace

fk_status fk_get_state(fk_grid* g, void* buf, size_t* len) {
  if (!g || !len) return FK_EINVAL;
  const size_t need = state_bytes(g);
  if (!buf) {
    *len = need;
    return FK_OK;
  }
  if (*len < need) {
    *len = need;
    return fail(g, FK_EINVAL, "checkpoint buffer too small (size returned in *len)");
  }
  DevState st;
  fk_status s = sync_state(g, &st);
  if (s != FK_OK) return s;
  StateHeader h;
  memset(&h, 0, sizeof h);
  memcpy(h.magic, kStateMagic, 8);
  h.nx = g->nx;
  h.nv1 = g->nv1;
  h.nv2 = g->nv2;
  h.precision = g->prec;
  h.pitch = g->pitch;
  h.scheme = g->scheme;
  h.hist_cap = g->prm.hist_cap;
  h.f_bytes = (int64_t)f_bytes(g);
  h.Ey = g->Ey;
  h.Ex_ext = g->Ex_ext;
  h.delta_max = g->delta_max;
  h.A_max = g->A_max;
  h.k_s = g->k_s;
  h.T_se = g->T_se;
  h.J = g->J;
  h.x_lo = g->x_lo;
  h.x_hi = g->x_hi;
  h.T_fe = g->T_fe;
  h.T_e = g->T_e;
  h.ln_lambda = g->ln_lambda;
  h.self_consistent = g->self_consistent;
  h.see_enabled = g->see_enabled;
  memcpy(&h.prm, &g->prm, sizeof(Params));
  memcpy(&h.st, &st, sizeof(DevState));
  unsigned char* p = static_cast<unsigned char*>(buf);
  memcpy(p, &h, sizeof h);
  p += sizeof h;
  struct Part {
    const void* src;
    size_t bytes;
  } parts[] = {{g->d_f[g->base_cur], f_bytes(g)},
               {g->d_ne, g->nx * sizeof(double)},
               {g->d_Ex, g->nx * sizeof(double)},
               {g->d_c1, g->nx * sizeof(double)},
               {g->d_c1_32, g->nx * sizeof(float)},
               {g->d_bgk, 2 * g->nx * sizeof(double)},
               {g->d_bgk32, 2 * g->nx * sizeof(float)},
               {g->d_hist, (size_t)g->prm.hist_cap * FK_HISTORY_COLS * sizeof(double)}};
  for (const Part& q : parts) {
    FK_CUDA(g, cudaMemcpy(p, q.src, q.bytes, cudaMemcpyDeviceToHost));
    p += q.bytes;
  }
  *len = need;
  return FK_OK;  // a frozen (flagged) state is a valid checkpoint too
}

fk_status fk_set_state(fk_grid* g, const void* buf, size_t len) {
  if (!g || !buf) return FK_EINVAL;
  FK_NOT_IN_BATCH(g);
  StateHeader h;
  if (len < sizeof h) return fail(g, FK_EINVAL, "checkpoint too short");
  memcpy(&h, buf, sizeof h);
  if (memcmp(h.magic, kStateMagic, 8) != 0) return fail(g, FK_EINVAL, "not a checkpoint of this library");
  if (h.nx != g->nx || h.nv1 != g->nv1 || h.nv2 != g->nv2 || h.precision != g->prec ||
      h.pitch != g->pitch || h.hist_cap != g->prm.hist_cap || h.f_bytes != (int64_t)f_bytes(g))
    return fail(g, FK_EINVAL,
                "checkpoint of another grid (shape, precision or history capacity differ)");
  if (len < state_bytes(g)) return fail(g, FK_EINVAL, "checkpoint truncated");
  if (h.scheme != kSchemeUnsplit && h.scheme != kSchemeLie && h.scheme != kSchemeStrang)
    return fail(g, FK_EINVAL, "checkpoint with an unknown time scheme");
  DevState cur;
  fk_status s = sync_state(g, &cur);
  if (s != FK_OK) return s;
  {
    const fk_status bs = split_buffers(g, h.scheme);
    if (bs != FK_OK) return bs;
  }
  // graphs were captured for the old kernel variants
  for (int q = 0; q < 2; q++)
    if (g->graph[q]) {
      cudaGraphExecDestroy(g->graph[q]);
      g->graph[q] = nullptr;
    }
  g->scheme = h.scheme;
  g->Ey = h.Ey;
  g->Ex_ext = h.Ex_ext;
  g->delta_max = h.delta_max;
  g->A_max = h.A_max;
  g->k_s = h.k_s;
  g->T_se = h.T_se;
  g->J = h.J;
  g->x_lo = h.x_lo;
  g->x_hi = h.x_hi;
  g->T_fe = h.T_fe;
  g->T_e = h.T_e;
  g->ln_lambda = h.ln_lambda;
  g->self_consistent = h.self_consistent;
  g->see_enabled = h.see_enabled;
  {
    // the test knobs are the grid's own, not the checkpoint's
    const long long wl = g->prm.wait_limit;
    const int wi = g->prm.withhold_item;
    memcpy(&g->prm, &h.prm, sizeof(Params));
    g->prm.wait_limit = wl;
    g->prm.withhold_item = wi;
  }
  if ((s = upload_params(g)) != FK_OK) return s;
  if ((s = rebuild_tables(g)) != FK_OK) return s;
  const unsigned char* p = static_cast<const unsigned char*>(buf) + sizeof h;
  struct Part {
    void* dst;
    size_t bytes;
  } parts[] = {{g->d_f[0], f_bytes(g)},
               {g->d_ne, g->nx * sizeof(double)},
               {g->d_Ex, g->nx * sizeof(double)},
               {g->d_c1, g->nx * sizeof(double)},
               {g->d_c1_32, g->nx * sizeof(float)},
               {g->d_bgk, 2 * g->nx * sizeof(double)},
               {g->d_bgk32, 2 * g->nx * sizeof(float)},
               {g->d_hist, (size_t)g->prm.hist_cap * FK_HISTORY_COLS * sizeof(double)}};
  for (const Part& q : parts) {
    FK_CUDA(g, cudaMemcpyAsync(q.dst, p, q.bytes, cudaMemcpyHostToDevice, g->stream));
    p += q.bytes;
  }
  FK_CUDA(g, cudaMemcpyAsync(g->d_st, &h.st, sizeof(DevState), cudaMemcpyHostToDevice, g->stream));
  FK_CUDA(g, cudaStreamSynchronize(g->stream));
  g->base_cur = g->enq_cur = 0;
  g->base_step = h.st.step;
  g->known_flags = h.st.flags;
  return FK_OK;
}

fk_status fk_grid_info(const fk_grid* g, double* out) {
  if (!g || !out) return FK_EINVAL;
  out[0] = g->dx;
  out[1] = g->dv1;
  out[2] = g->dv2;
  out[3] = g->dt;
  out[4] = g->prm.c2;
  out[5] = g->prm.cx_max;
  out[6] = g->use_stream ? 1.0 : 0.0;
  out[7] = g->geom.n_tiles;
  out[8] = g->geom.n_chunks;
  out[9] = g->geom.chunk_len;
  out[10] = g->geom.half ? 2.0 : 1.0;
  out[11] = std::max(g->geom.ti_neg, g->geom.ti_pos);
  out[12] = g->tile_cap;
  return FK_OK;
}

fk_status fk_set_tile_rows(fk_grid* g, int32_t max_rows) {
  if (!g) return FK_EINVAL;
  FK_NOT_IN_BATCH(g);
  if (max_rows < 0) return fail(g, FK_EINVAL, "max_rows must be >= 0");
  DevState st;
  const fk_status s = sync_state(g, &st);  // the grid's work is done
  if (s != FK_OK) return s;
  return replan_tiles(g, max_rows);
}

fk_status fk_set_kernel_timing(fk_grid* g, int enabled) {
  if (!g) return FK_EINVAL;
  FK_NOT_IN_BATCH(g);
  FK_CUDA(g, cudaSetDevice(g->dev));
  if (enabled && g->ev.empty()) {
    g->ev.resize(2 * kMaxTimed, nullptr);
    for (auto& e : g->ev) FK_CUDA(g, cudaEventCreate(&e));
  }
  FK_CUDA(g, cudaStreamSynchronize(g->stream));
  g->timing = enabled != 0;
  g->ev_used = 0;
  return FK_OK;
}

fk_status fk_kernel_timing(fk_grid* g, int64_t* launches, double* total_ms) {
  if (!g || !launches || !total_ms) return FK_EINVAL;
  FK_CUDA(g, cudaSetDevice(g->dev));
  FK_CUDA(g, cudaStreamSynchronize(g->stream));
  double tot = 0.0;
  for (int r = 0; r < g->ev_used; r++) {
    float ms = 0.f;
    FK_CUDA(g, cudaEventElapsedTime(&ms, g->ev[2 * r], g->ev[2 * r + 1]));
    tot += ms;
  }
  *launches = g->ev_used;
  *total_ms = tot;
  g->ev_used = 0;
  return FK_OK;
}

const char* fk_last_error(const fk_grid* g) {
  return g ? g->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
