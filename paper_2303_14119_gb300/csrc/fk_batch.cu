// Batched stepping of many independent grids (the parameter scans of
// Sec. 3 of Sun et al., arXiv 2303.14119, run as one sweep): per batch step
// one launch of the streaming step kernel over the work units of every grid
// and one launch of the finalize kernel over every grid's planes, replayed
// 32 steps per CUDA graph; an autotuner for the x-chunk length per size
// bucket.  The C ABI is declared in include/fk.h.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "fk_host.cuh"

using namespace fk;

namespace {

thread_local std::string g_batch_create_error;

constexpr int kBatchGraphSteps = 32;  // steps per captured graph (even)
constexpr int kBatchMaxTimed = 8192;  // step-kernel launches timed between reads
constexpr int kMinChunk = 4;          // fewest planes per x-chunk the planner picks
constexpr double kDefaultWaves = 4.0; // default plan: about this many CTA waves

// Where one grid's moments live, and where its n_e / E_x go in a packed slot.
struct MomentSrc {
  const DevState* st;
  const double* ne;
  const double* ex;
  long long off;  // planes of the grids before it
  int nx;
  int pad;
};

}  // namespace

struct fk_batch {
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t cap_stream = nullptr;
  int prec = FK_F64;
  bool padded = false;  // some grid has row padding (pitch > nv2)
  bool bgk = false;     // some grid has collisions on (the kernel variant with the term)
  int n = 0;
  std::vector<fk_grid*> grids;
  std::vector<int> cur0;       // buffer holding each grid's f at batch step 0
  std::vector<int> chunk_len;  // planes per x-chunk, per grid
  std::vector<int> bucket;     // size bucket per grid
  int n_buckets = 0;
  long long steps = 0;         // batch steps enqueued
  double cells = 0;            // phase-space cells of all grids
  BatchInst* d_inst = nullptr; // [2][n]: grid arguments for even / odd batch steps
  int2* d_units = nullptr;     // [max_units] whole-CTA work units, largest first
  int n_units = 0, max_units = 0;
  int4* d_pairs = nullptr;     // [max_pairs] CTAs of two half units, largest first
  int n_pairs = 0, max_pairs = 0;
  int2* d_fblk = nullptr;      // [n_fblk] finalize entries: n_fmulti (grid, block)
  int n_fblk = 0;               // pairs of the grids of several finalize blocks,
  int n_fmulti = 0;             // then (grid, -1) for those of one
  size_t smem = 0;             // dynamic shared memory per CTA (whole-CTA units)
  int half_bytes = 0;          // shared memory of one half unit's region
  int per_sm = 0, sms = 0;      // CTAs per SM (the smaller of the two layouts), SMs
  int per_sm_whole = 0, per_sm_half = 0;  // CTAs per SM of each unit layout's launch
  bool dirty = true;           // units / arguments must be re-uploaded
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  cudaEvent_t done = nullptr;  // recorded after the last enqueued batch step
  bool timing = false;
  std::vector<cudaEvent_t> ev; // pairs around the step kernel
  int ev_used = 0;
  // pipelined moment read-back (fk_batch_moments_enqueue / _collect): two
  // slots, each (sigma, Gamma_pe, Gamma_see) of every grid, then n_e and
  // E_x of every grid, packed on the device by one gather kernel and
  // brought to pinned host memory by one copy, both on copy_stream, so that
  // they run beside the next step kernel; the next finalize (the first
  // kernel to overwrite what the gather reads) waits for `pending`
  void* h_slot[2] = {nullptr, nullptr};
  double* d_slot[2] = {nullptr, nullptr};
  cudaEvent_t gathered[2] = {nullptr, nullptr};  // the gather kernel has run
  cudaEvent_t slot_ev[2] = {nullptr, nullptr};   // the slot's copy has landed
  bool slot_full[2] = {false, false};
  size_t sum_nx = 0;
  MomentSrc* d_msrc = nullptr;  // [n] where each grid's moments live
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t fin_ev = nullptr;   // the batch's work up to an enqueue
  cudaEvent_t pending = nullptr;  // the last gather, not yet waited for
  std::string err;
};

namespace {

fk_status bfail(fk_batch* b, fk_status s, const std::string& msg) {
  if (b)
    b->err = msg;
  else
    g_batch_create_error = msg;
  return s;
}

fk_status bcuda_fail(fk_batch* b, cudaError_t e, const char* what) {
  return bfail(b, e == cudaErrorMemoryAllocation ? FK_ENOMEM : FK_ECUDA,
               std::string(what) + ": " + cudaGetErrorString(e));
}

#define BK_CUDA(b, call)                                      \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return bcuda_fail((b), e_, #call); \
  } while (0)

// Pack every grid's sigma, Gamma_pe and Gamma_see (3 doubles per grid), then
// the n_e of all grids, then their E_x, into out; block i copies grid i.
__global__ void __launch_bounds__(256)
gather_moments_kernel(const MomentSrc* __restrict__ src, int n, long long sum_nx,
                      double* __restrict__ out) {
  const MomentSrc m = src[blockIdx.x];
  if (threadIdx.x == 0) {
    out[3 * (size_t)blockIdx.x] = m.st->sigma;
    out[3 * (size_t)blockIdx.x + 1] = m.st->g_pe;
    out[3 * (size_t)blockIdx.x + 2] = m.st->g_see;
  }
  double* ne = out + 3 * (size_t)n + m.off;
  double* ex = ne + sum_nx;
  for (int k = threadIdx.x; k < m.nx; k += blockDim.x) {
    ne[k] = m.ne[k];
    ex[k] = m.ex[k];
  }
}

int chunks_of(int nx, int len) { return (nx + len - 1) / len; }

// Equal chunks of at most len planes.
int even_chunk_len(int nx, int len) {
  len = std::max(1, std::min(len, nx));
  const int nc = chunks_of(nx, len);
  return (nx + nc - 1) / nc;
}

// Grid i's geometry with the batch's x-chunking.
Geom batch_geom(const fk_batch* b, int i) {
  Geom gm = b->grids[i]->geom;
  gm.chunk_len = b->chunk_len[i];
  gm.n_chunks = chunks_of(b->grids[i]->nx, gm.chunk_len);
  return gm;
}

// Cells a unit reads: its rows x pitch over its planes plus the upwind plane
// loaded first (every chunk but the first along the march).
long long unit_cells(const fk_grid* g, const Geom& gm, int t, int c) {
  int i0, i1, dir;
  tile_rows(gm, g->nv1, t, &i0, &i1, &dir);
  const int s0 = c * gm.chunk_len;
  const int s1 = std::min(g->nx, s0 + gm.chunk_len);
  if (s0 >= s1 || i0 >= i1) return 0;
  return (long long)(i1 - i0) * g->pitch * (s1 - s0 + (s0 > 0 ? 1 : 0));
}

// Work units of the current chunking, largest first (ties in grid, tile,
// chunk order), so that the block scheduler hands out the long units before
// the short ones that fill the last wave.
std::vector<int2> plan_units(const fk_batch* b) {
  struct U {
    long long cells;
    int inst, local;
  };
  std::vector<U> us;
  for (int i = 0; i < b->n; i++) {
    const Geom gm = batch_geom(b, i);
    for (int c = 0; c < gm.n_chunks; c++)
      for (int t = 0; t < gm.n_tiles; t++) {
        const long long w = unit_cells(b->grids[i], gm, t, c);
        if (w > 0) us.push_back({w, i, t + gm.n_tiles * c});
      }
  }
  std::stable_sort(us.begin(), us.end(), [](const U& x, const U& y) { return x.cells > y.cells; });
  std::vector<int2> out(us.size());
  for (size_t q = 0; q < us.size(); q++) out[q] = make_int2(us[q].inst, us[q].local);
  return out;
}

// Split a unit list into the whole-CTA units and the CTAs of half units,
// two to a CTA in list order (so that a pair's units are of about the same
// size; the second half of a last odd one stays idle).
void split_units(const fk_batch* b, const std::vector<int2>& units, std::vector<int2>* whole,
                 std::vector<int4>* pairs) {
  whole->clear();
  pairs->clear();
  bool open = false;  // the last pair's second half is free
  for (const int2& u : units) {
    if (!b->grids[u.x]->geom.half) {
      whole->push_back(u);
    } else if (open) {
      pairs->back().z = u.x;
      pairs->back().w = u.y;
      open = false;
    } else {
      pairs->push_back(make_int4(u.x, u.y, -1, 0));
      open = true;
    }
  }
}

// Default chunking: units of about (all cells) / (kDefaultWaves x resident
// CTAs), at least kMinChunk planes, one chunk if the grid is smaller.
void default_chunks(fk_batch* b) {
  bool all_half = true;
  for (const fk_grid* g : b->grids) all_half = all_half && g->geom.half;
  const double slots =
      (double)b->sms * (all_half ? 2.0 * b->per_sm_half : (double)b->per_sm_whole);  // unit slots
  const double target = b->cells / (kDefaultWaves * slots);
  for (int i = 0; i < b->n; i++) {
    const fk_grid* g = b->grids[i];
    const double per_tile = (double)g->nx * g->nv1 * g->pitch / g->geom.n_tiles;
    int nc = (int)lround(per_tile / std::max(target, 1.0));
    nc = std::max(1, std::min(nc, std::max(1, g->nx / kMinChunk)));
    b->chunk_len[i] = (g->nx + nc - 1) / nc;
  }
}

// Size buckets: grids with the same power-of-two class of plane size and nx.
void assign_buckets(fk_batch* b) {
  std::map<std::pair<int, int>, int> ids;
  for (int i = 0; i < b->n; i++) {
    const fk_grid* g = b->grids[i];
    const int lp = (int)floor(log2((double)g->nv1 * g->pitch));
    const int lx = (int)floor(log2((double)g->nx));
    auto it = ids.find({lp, lx});
    if (it == ids.end()) it = ids.emplace(std::make_pair(lp, lx), (int)ids.size()).first;
    b->bucket[i] = it->second;
  }
  b->n_buckets = (int)ids.size();
}

}  // namespace

namespace {

void drop_graphs(fk_batch* b) {
  for (int p = 0; p < 2; p++)
    if (b->graph[p]) {
      cudaGraphExecDestroy(b->graph[p]);
      b->graph[p] = nullptr;
    }
}

// Shared memory per CTA and CTAs per SM of the batch's two launches, from
// its grids' current tile plans; false if a plan does not fit an SM.
bool batch_resources(fk_batch* b) {
  b->smem = 0;
  b->half_bytes = 0;
  bool any_whole = false, any_half = false;
  for (const fk_grid* g : b->grids) {
    if (g->geom.half)
      b->half_bytes = std::max(
          b->half_bytes, (int)stream_half_bytes(g->prec, g->geom.stage_elems, g->pitch));
    else
      b->smem = std::max(b->smem, stream_smem_bytes(g->prec, g->geom.stage_elems, g->pitch));
    (g->geom.half ? any_half : any_whole) = true;
  }
  b->per_sm_whole = any_whole ? stream_ctas_per_sm(b->prec, b->smem, kLayoutWhole) : 1 << 30;
  b->per_sm_half =
      any_half ? stream_ctas_per_sm(b->prec, 2 * (size_t)b->half_bytes, kLayoutHalf) : 1 << 30;
  b->per_sm = std::min(b->per_sm_whole, b->per_sm_half);
  return b->per_sm > 0;
}

// Upload both parities' grid arguments and the unit list of the current
// chunking (after the batch's earlier work: the buffers may be in use).
fk_status upload_plan(fk_batch* b) {
  std::vector<BatchInst> h(2 * (size_t)b->n);
  for (int p = 0; p < 2; p++)
    for (int i = 0; i < b->n; i++) {
      fk_grid* g = b->grids[i];
      BatchInst& bi = h[(size_t)p * b->n + i];
      bi.a = make_args(g, b->cur0[i] ^ p);
      bi.a.geom = batch_geom(b, i);
      bi.o = FinOut{g->d_ne, g->d_Ex, g->d_c1, g->d_c1_32, g->d_hist, g->fin};
    }
  std::vector<int2> units;
  std::vector<int4> pairs;
  split_units(b, plan_units(b), &units, &pairs);
  BK_CUDA(b, cudaStreamSynchronize(b->stream));
  drop_graphs(b);
  if ((int)units.size() > b->max_units) {
    if (b->d_units) BK_CUDA(b, cudaFree(b->d_units));
    b->d_units = nullptr;
    b->max_units = 0;
    BK_CUDA(b, hooked_alloc(reinterpret_cast<void**>(&b->d_units), units.size() * sizeof(int2)));
    b->max_units = (int)units.size();
  }
  if ((int)pairs.size() > b->max_pairs) {
    if (b->d_pairs) BK_CUDA(b, cudaFree(b->d_pairs));
    b->d_pairs = nullptr;
    b->max_pairs = 0;
    BK_CUDA(b, hooked_alloc(reinterpret_cast<void**>(&b->d_pairs), pairs.size() * sizeof(int4)));
    b->max_pairs = (int)pairs.size();
  }
  b->n_units = (int)units.size();
  b->n_pairs = (int)pairs.size();
  BK_CUDA(b, cudaMemcpyAsync(b->d_inst, h.data(), h.size() * sizeof(BatchInst),
                             cudaMemcpyHostToDevice, b->stream));
  if (b->n_units)
    BK_CUDA(b, cudaMemcpyAsync(b->d_units, units.data(), units.size() * sizeof(int2),
                               cudaMemcpyHostToDevice, b->stream));
  if (b->n_pairs)
    BK_CUDA(b, cudaMemcpyAsync(b->d_pairs, pairs.data(), pairs.size() * sizeof(int4),
                               cudaMemcpyHostToDevice, b->stream));
  BK_CUDA(b, cudaStreamSynchronize(b->stream));  // the host vectors go out of scope
  b->dirty = false;
  return FK_OK;
}

// One batch step whose grids read the buffers of parity p: the batched step
// kernel (optionally between two events) then the batched finalize.
cudaError_t enqueue_batch_step(fk_batch* b, int p, cudaStream_t s, cudaEvent_t ev0,
                               cudaEvent_t ev1) {
  const BatchInst* inst = b->d_inst + (size_t)p * b->n;
  cudaError_t e = cudaSuccess;
  if (ev0) e = cudaEventRecord(ev0, s);
  if (e == cudaSuccess)
    e = launch_step_stream_batch(inst, b->d_units, b->n_units, b->d_pairs, b->n_pairs, b->prec,
                                 b->padded, b->bgk, b->smem, b->half_bytes, s);
  if (e == cudaSuccess && ev1) e = cudaEventRecord(ev1, s);
  // a moment gather queued before this step may still read the moments and
  // scalars the finalize overwrites (never inside a capture: the graph's
  // launch waits instead)
  if (e == cudaSuccess && b->pending && s == b->stream) {
    e = cudaStreamWaitEvent(s, b->pending, 0);
    b->pending = nullptr;
  }
  if (e == cudaSuccess) e = launch_finalize_batch(inst, b->d_fblk, b->n_fmulti, b->n_fblk, s);
  return e;
}

fk_status build_batch_graph(fk_batch* b, int parity) {
  cudaStream_t cs = b->cap_stream;
  BK_CUDA(b, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < kBatchGraphSteps && e == cudaSuccess; s++)
    e = enqueue_batch_step(b, (parity + s) & 1, cs, nullptr, nullptr);
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return bcuda_fail(b, e, "capturing the batch step graph");
  }
  if (e2 != cudaSuccess) return bcuda_fail(b, e2, "cudaStreamEndCapture");
  const cudaError_t e3 = cudaGraphInstantiate(&b->graph[parity], graph, 0);
  cudaGraphDestroy(graph);
  if (e3 != cudaSuccess) return bcuda_fail(b, e3, "cudaGraphInstantiate");
  return FK_OK;
}

// Enqueue n steps (graphs of kBatchGraphSteps where possible; direct launches
// with event pairs in timing mode) and mark the batch's progress.
fk_status enqueue_steps(fk_batch* b, long long n) {
  if (b->dirty) {
    const fk_status s = upload_plan(b);
    if (s != FK_OK) return s;
  }
  while (n > 0) {
    const int p = (int)(b->steps & 1);
    if (b->timing) {
      const bool rec = b->ev_used < kBatchMaxTimed;
      BK_CUDA(b, enqueue_batch_step(b, p, b->stream, rec ? b->ev[2 * b->ev_used] : nullptr,
                                    rec ? b->ev[2 * b->ev_used + 1] : nullptr));
      if (rec) b->ev_used++;
      b->steps += 1;
      n -= 1;
    } else if (n >= kBatchGraphSteps) {
      if (!b->graph[p]) {
        const fk_status s = build_batch_graph(b, p);
        if (s != FK_OK) return s;
      }
      if (b->pending) {
        BK_CUDA(b, cudaStreamWaitEvent(b->stream, b->pending, 0));
        b->pending = nullptr;
      }
      BK_CUDA(b, cudaGraphLaunch(b->graph[p], b->stream));
      b->steps += kBatchGraphSteps;  // even: the parity is unchanged
      n -= kBatchGraphSteps;
    } else {
      BK_CUDA(b, enqueue_batch_step(b, p, b->stream, nullptr, nullptr));
      b->steps += 1;
      n -= 1;
    }
  }
  BK_CUDA(b, cudaEventRecord(b->done, b->stream));
  return FK_OK;
}

// Release the grids (re-based on their device step counters) and free.
void free_batch(fk_batch* b) {
  if (!b) return;
  cudaSetDevice(b->dev);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->copy_stream) cudaStreamSynchronize(b->copy_stream);  // a gather or copy in flight
  drop_graphs(b);
  for (fk_grid* g : b->grids) {
    if (!g || g->batch != b) continue;
    g->batch = nullptr;
    g->batch_done = nullptr;
    DevState st;
    sync_state(g, &st);
  }
  void* ptrs[] = {b->d_inst, b->d_units, b->d_pairs, b->d_fblk};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  if (b->done) cudaEventDestroy(b->done);
  for (int q = 0; q < 2; q++) {
    if (b->h_slot[q]) cudaFreeHost(b->h_slot[q]);
    if (b->d_slot[q]) cudaFree(b->d_slot[q]);
    if (b->gathered[q]) cudaEventDestroy(b->gathered[q]);
    if (b->slot_ev[q]) cudaEventDestroy(b->slot_ev[q]);
  }
  if (b->d_msrc) cudaFree(b->d_msrc);
  if (b->fin_ev) cudaEventDestroy(b->fin_ev);
  if (b->copy_stream) cudaStreamDestroy(b->copy_stream);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

// Read every grid's device scalars into its pinned read-back buffer (all
// copies enqueued, one wait) and return them there.
fk_status read_states(fk_batch* b, std::vector<const DevState*>* st) {
  st->resize(b->n);
  for (int i = 0; i < b->n; i++) {
    fk_grid* g = b->grids[i];
    BK_CUDA(b, cudaMemcpyAsync(g->h_stage, g->d_st, sizeof(DevState), cudaMemcpyDeviceToHost,
                               b->stream));
    (*st)[i] = static_cast<const DevState*>(g->h_stage);
  }
  BK_CUDA(b, cudaStreamSynchronize(b->stream));
  return FK_OK;
}

}  // namespace

extern "C" {

fk_status fk_batch_create(fk_grid* const* grids, int32_t n, void* cuda_stream, fk_batch** out) {
  g_batch_create_error.clear();
  alloc_hook_reset();
  if (!grids || !out || n < 1)
    return bfail(nullptr, FK_EINVAL, "grids and out must not be NULL and n must be >= 1");
  *out = nullptr;
  std::vector<fk_grid*> gs(grids, grids + n);
  for (int i = 0; i < n; i++) {
    fk_grid* g = gs[i];
    const std::string who = "grid " + std::to_string(i);
    if (!g) return bfail(nullptr, FK_EINVAL, who + " is NULL");
    if (g->batch) return bfail(nullptr, FK_ESTATE, who + " already belongs to a batch");
    if (g->dev != gs[0]->dev) return bfail(nullptr, FK_EINVAL, who + " is on another device");
    if (g->prec != gs[0]->prec) return bfail(nullptr, FK_EINVAL, who + " has another precision");
    if (!g->use_stream)
      return bfail(nullptr, FK_EINVAL, who + " uses the direct-load step kernel (rows too wide)");
    if (g->scheme != kSchemeUnsplit)
      return bfail(nullptr, FK_EINVAL, who + " uses a split time scheme (steps alone only)");
  }
  {
    std::vector<fk_grid*> sorted(gs);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
      return bfail(nullptr, FK_EINVAL, "a grid appears twice");
  }
  fk_batch* b = new (std::nothrow) fk_batch();
  if (!b) return bfail(nullptr, FK_ENOMEM, "host allocation failed");
  b->dev = gs[0]->dev;
  b->prec = gs[0]->prec;
  b->n = n;
  b->grids = gs;
  b->cur0.assign(n, 0);
  b->chunk_len.assign(n, 1);
  b->bucket.assign(n, 0);

#define CREATE_B(call)                                          \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) {                                    \
      const fk_status s_ = bcuda_fail(nullptr, e_, #call);      \
      free_batch(b);                                            \
      return s_;                                                \
    }                                                           \
  } while (0)

  CREATE_B(cudaSetDevice(b->dev));
  if (cuda_stream) {
    b->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    CREATE_B(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    b->own_stream = true;
  }
  CREATE_B(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  CREATE_B(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming));
  CREATE_B(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->dev));
  std::vector<int2> fblk, fone;
  for (int i = 0; i < n; i++) {
    fk_grid* g = gs[i];
    if (g->pitch != g->nv2) b->padded = true;
    if (g->prm.collisions) b->bgk = true;
    b->cells += (double)g->nx * g->nv1 * g->nv2;
    if (finalize_blocks(g->nx) == 1)
      fone.push_back(make_int2(i, -1));
    else
      for (int q = 0; q < finalize_blocks(g->nx); q++) fblk.push_back(make_int2(i, q));
    DevState st;
    const fk_status s = sync_state(g, &st);  // the grid's own work is done
    if (s != FK_OK) {
      g_batch_create_error = "grid " + std::to_string(i) + ": " + g->err;
      free_batch(b);
      return s;
    }
    b->cur0[i] = g->enq_cur;
  }
  if (!batch_resources(b)) {
    free_batch(b);
    return bfail(nullptr, FK_EINVAL, "the grids' shared-memory plans do not fit an SM");
  }
  b->n_fmulti = (int)fblk.size();
  fblk.insert(fblk.end(), fone.begin(), fone.end());
  b->n_fblk = (int)fblk.size();
  CREATE_B(hooked_alloc(reinterpret_cast<void**>(&b->d_inst), 2 * (size_t)n * sizeof(BatchInst)));
  CREATE_B(hooked_alloc(reinterpret_cast<void**>(&b->d_fblk), fblk.size() * sizeof(int2)));
  CREATE_B(cudaMemcpy(b->d_fblk, fblk.data(), fblk.size() * sizeof(int2),
                      cudaMemcpyHostToDevice));
#undef CREATE_B
  default_chunks(b);
  assign_buckets(b);
  fk_status s = upload_plan(b);
  if (s != FK_OK) {
    g_batch_create_error = b->err;
    free_batch(b);
    return s;
  }
  for (fk_grid* g : gs) {
    g->batch = b;
    g->batch_done = b->done;
  }
  *out = b;
  return FK_OK;
}

fk_status fk_batch_destroy(fk_batch* b) {
  free_batch(b);
  return FK_OK;
}

fk_status fk_batch_step(fk_batch* b, int64_t n) {
  if (!b) return FK_EINVAL;
  const NvtxRange range("fk_batch_step");
  if (n < 0) return bfail(b, FK_EINVAL, "n must be >= 0");
  BK_CUDA(b, cudaSetDevice(b->dev));
  return enqueue_steps(b, n);
}

fk_status fk_batch_sync(fk_batch* b, int32_t* status) {
  if (!b) return FK_EINVAL;
  BK_CUDA(b, cudaSetDevice(b->dev));
  std::vector<const DevState*> st;
  const fk_status rs = read_states(b, &st);
  if (rs != FK_OK) return rs;
  fk_status first = FK_OK;
  for (int i = 0; i < b->n; i++) {
    fk_grid* g = b->grids[i];
    const fk_status s = flags_status(g, st[i]->flags);
    if (status) status[i] = s;
    if (s != FK_OK && first == FK_OK) {
      first = s;
      b->err = "grid " + std::to_string(i) + ": " + g->err;
    }
  }
  return first;
}

fk_status fk_batch_scalars(fk_batch* b, double* sigma, int64_t* step, int64_t* sat_step,
                           int32_t* status) {
  if (!b) return FK_EINVAL;
  BK_CUDA(b, cudaSetDevice(b->dev));
  std::vector<const DevState*> st;
  const fk_status rs = read_states(b, &st);
  if (rs != FK_OK) return rs;
  for (int i = 0; i < b->n; i++) {
    if (sigma) sigma[i] = st[i]->sigma;
    if (step) step[i] = st[i]->step;
    if (sat_step) sat_step[i] = st[i]->sat_step;
    if (status) status[i] = flags_status(b->grids[i], st[i]->flags);
  }
  return FK_OK;
}

fk_status fk_batch_moments(fk_batch* b, double* sigma, double* gamma_pe, double* gamma_see,
                           double* n_e, double* Ex) {
  if (!b) return FK_EINVAL;
  BK_CUDA(b, cudaSetDevice(b->dev));
  // every copy lands in its grid's pinned buffer (DevState, n_e, E_x), all
  // enqueued on the batch's stream; one wait for all of them
  for (int i = 0; i < b->n; i++) {
    fk_grid* g = b->grids[i];
    DevState* hst = static_cast<DevState*>(g->h_stage);
    double* hv = reinterpret_cast<double*>(hst + 1);
    const size_t vb = (size_t)g->nx * sizeof(double);
    BK_CUDA(b, cudaMemcpyAsync(hst, g->d_st, sizeof(DevState), cudaMemcpyDeviceToHost, b->stream));
    if (n_e) BK_CUDA(b, cudaMemcpyAsync(hv, g->d_ne, vb, cudaMemcpyDeviceToHost, b->stream));
    if (Ex) BK_CUDA(b, cudaMemcpyAsync(hv + g->nx, g->d_Ex, vb, cudaMemcpyDeviceToHost, b->stream));
  }
  BK_CUDA(b, cudaStreamSynchronize(b->stream));
  size_t off = 0;
  for (int i = 0; i < b->n; i++) {
    fk_grid* g = b->grids[i];
    const DevState* hst = static_cast<const DevState*>(g->h_stage);
    const double* hv = reinterpret_cast<const double*>(hst + 1);
    const size_t vb = (size_t)g->nx * sizeof(double);
    if (sigma) sigma[i] = hst->sigma;
    if (gamma_pe) gamma_pe[i] = hst->g_pe;
    if (gamma_see) gamma_see[i] = hst->g_see;
    if (n_e) memcpy(n_e + off, hv, vb);
    if (Ex) memcpy(Ex + off, hv + g->nx, vb);
    off += g->nx;
  }
  return FK_OK;
}

fk_status fk_batch_moments_enqueue(fk_batch* b, int32_t slot) {
  if (!b) return FK_EINVAL;
  if (slot != 0 && slot != 1) return bfail(b, FK_EINVAL, "slot must be 0 or 1");
  BK_CUDA(b, cudaSetDevice(b->dev));
  if (!b->d_msrc) {  // first use: the grids' source pointers and the side stream
    std::vector<MomentSrc> src(b->n);
    size_t nx = 0;
    for (int i = 0; i < b->n; i++) {
      const fk_grid* g = b->grids[i];
      src[i] = MomentSrc{g->d_st, g->d_ne, g->d_Ex, (long long)nx, g->nx, 0};
      nx += g->nx;
    }
    b->sum_nx = nx;
    BK_CUDA(b, cudaStreamCreateWithFlags(&b->copy_stream, cudaStreamNonBlocking));
    BK_CUDA(b, cudaEventCreateWithFlags(&b->fin_ev, cudaEventDisableTiming));
    BK_CUDA(b, hooked_alloc(reinterpret_cast<void**>(&b->d_msrc), src.size() * sizeof(MomentSrc)));
    BK_CUDA(b, cudaMemcpy(b->d_msrc, src.data(), src.size() * sizeof(MomentSrc),
                          cudaMemcpyHostToDevice));
  }
  const size_t bytes = (3 * (size_t)b->n + 2 * b->sum_nx) * sizeof(double);
  if (!b->h_slot[slot]) {  // first use of the slot: its buffers and events
    BK_CUDA(b, hooked_alloc(&b->h_slot[slot], bytes, true));
    BK_CUDA(b, hooked_alloc(reinterpret_cast<void**>(&b->d_slot[slot]), bytes));
    BK_CUDA(b, cudaEventCreateWithFlags(&b->gathered[slot], cudaEventDisableTiming));
    BK_CUDA(b, cudaEventCreateWithFlags(&b->slot_ev[slot], cudaEventDisableTiming));
  }
  if (b->slot_full[slot]) return bfail(b, FK_ESTATE, "slot holds uncollected moments");
  // the slot's previous copy has landed (it was collected), so its device
  // buffer is free; the gather reads the state of the work enqueued so far
  // (and only reads it: the next step kernel may run beside it)
  BK_CUDA(b, cudaEventRecord(b->fin_ev, b->stream));
  BK_CUDA(b, cudaStreamWaitEvent(b->copy_stream, b->fin_ev, 0));
  gather_moments_kernel<<<b->n, 256, 0, b->copy_stream>>>(b->d_msrc, b->n,
                                                          (long long)b->sum_nx, b->d_slot[slot]);
  BK_CUDA(b, cudaGetLastError());
  BK_CUDA(b, cudaEventRecord(b->gathered[slot], b->copy_stream));
  b->pending = b->gathered[slot];  // gathers run in order: the last covers the earlier ones
  BK_CUDA(b, cudaMemcpyAsync(b->h_slot[slot], b->d_slot[slot], bytes, cudaMemcpyDeviceToHost,
                             b->copy_stream));
  BK_CUDA(b, cudaEventRecord(b->slot_ev[slot], b->copy_stream));
  b->slot_full[slot] = true;
  return FK_OK;
}

fk_status fk_batch_moments_collect(fk_batch* b, int32_t slot, double* sigma, double* gamma_pe,
                                   double* gamma_see, double* n_e, double* Ex) {
  if (!b) return FK_EINVAL;
  if (slot != 0 && slot != 1) return bfail(b, FK_EINVAL, "slot must be 0 or 1");
  if (!b->slot_full[slot]) return bfail(b, FK_ESTATE, "nothing enqueued in this slot");
  BK_CUDA(b, cudaSetDevice(b->dev));
  BK_CUDA(b, cudaEventSynchronize(b->slot_ev[slot]));
  b->slot_full[slot] = false;
  const double* hs = static_cast<const double*>(b->h_slot[slot]);
  const double* hne = hs + 3 * (size_t)b->n;
  const double* hex = hne + b->sum_nx;
  for (int i = 0; i < b->n; i++) {
    if (sigma) sigma[i] = hs[3 * (size_t)i];
    if (gamma_pe) gamma_pe[i] = hs[3 * (size_t)i + 1];
    if (gamma_see) gamma_see[i] = hs[3 * (size_t)i + 2];
  }
  if (n_e) memcpy(n_e, hne, b->sum_nx * sizeof(double));
  if (Ex) memcpy(Ex, hex, b->sum_nx * sizeof(double));
  return FK_OK;
}

fk_status fk_batch_get_chunks(const fk_batch* b, int32_t* chunk_len) {
  if (!b || !chunk_len) return FK_EINVAL;
  for (int i = 0; i < b->n; i++) chunk_len[i] = b->chunk_len[i];
  return FK_OK;
}

fk_status fk_batch_set_chunks(fk_batch* b, const int32_t* chunk_len) {
  if (!b || !chunk_len) return FK_EINVAL;
  for (int i = 0; i < b->n; i++)
    b->chunk_len[i] = std::max(1, std::min((int)chunk_len[i], b->grids[i]->nx));
  b->dirty = true;
  return FK_OK;
}

fk_status fk_batch_info(const fk_batch* b, double* out) {
  if (!b || !out) return FK_EINVAL;
  // the units and CTAs of the chunking in force (planned on the host)
  std::vector<int2> whole;
  std::vector<int4> pairs;
  split_units(b, plan_units(b), &whole, &pairs);
  int halves = 2 * (int)pairs.size();
  if (!pairs.empty() && pairs.back().z < 0) halves -= 1;
  out[0] = b->n;
  out[1] = (double)whole.size() + halves;
  out[2] = finalize_batch_ctas(b->n_fmulti, b->n_fblk);
  out[3] = (double)std::max(b->smem, 2 * (size_t)b->half_bytes);
  out[4] = b->per_sm;
  out[5] = b->cells;
  out[6] = b->n_buckets;
  out[7] = (double)b->steps;
  out[8] = (double)whole.size();
  out[9] = (double)pairs.size();
  return FK_OK;
}

namespace {

// Cells per tile plane that the tile search of fk_batch_autotune_tiles tries
// beside each grid's current tiles (rows = cells / pitch, at least 4).
constexpr int kTileCellTargets[] = {5120, 4096};

// The autotuner (fk_batch_autotune; tiles: fk_batch_autotune_tiles).
fk_status autotune(fk_batch* b, int32_t steps_per_trial, int64_t* steps_taken, bool tiles) {
  if (!b) return FK_EINVAL;
  const NvtxRange range(tiles ? "fk_batch_autotune_tiles" : "fk_batch_autotune");
  if (steps_per_trial < 1) return bfail(b, FK_EINVAL, "steps_per_trial must be >= 1");
  BK_CUDA(b, cudaSetDevice(b->dev));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BK_CUDA(b, cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return bcuda_fail(b, ce, "cudaEventCreate");
  }
  long long taken = 0;
  // one trial: steps_per_trial real batch steps of the current chunking,
  // timed on the batch's stream
  auto trial = [&](float* ms) -> fk_status {
    if (b->dirty) {
      const fk_status s = upload_plan(b);
      if (s != FK_OK) return s;
    }
    BK_CUDA(b, cudaEventRecord(e0, b->stream));
    for (int q = 0; q < steps_per_trial; q++) {
      BK_CUDA(b, enqueue_batch_step(b, (int)(b->steps & 1), b->stream, nullptr, nullptr));
      b->steps += 1;
    }
    BK_CUDA(b, cudaEventRecord(e1, b->stream));
    BK_CUDA(b, cudaEventRecord(b->done, b->stream));
    BK_CUDA(b, cudaEventSynchronize(e1));
    BK_CUDA(b, cudaEventElapsedTime(ms, e0, e1));
    taken += steps_per_trial;
    return FK_OK;
  };
  // every grid of bucket q with the tile-row cap caps[i] (the batch is idle
  // after a trial).  A grid whose re-plan fails keeps its plan; the batch's
  // shared memory and slots follow whatever plans the grids hold.
  auto set_caps = [&](int q, const std::vector<int>& caps) -> fk_status {
    fk_status first = FK_OK;
    bool changed = false;
    for (int i = 0; i < b->n; i++)
      if (b->bucket[i] == q && b->grids[i]->tile_cap != caps[i]) {
        const fk_status s = replan_tiles(b->grids[i], caps[i]);
        if (s == FK_OK) {
          changed = true;
        } else if (first == FK_OK) {
          first = s;
          b->err = b->grids[i]->err;
        }
      }
    if (changed) {
      b->dirty = true;
      if (!batch_resources(b) && first == FK_OK)
        first = bfail(b, FK_EINVAL, "a tile plan does not fit an SM");
    }
    return first;
  };
  fk_status s = FK_OK;
  float best = 0.f, ms = 0.f;
  // buckets by their cells, largest first
  std::vector<double> bcells(b->n_buckets, 0.0);
  std::vector<int> bmax_nx(b->n_buckets, 1);
  for (int i = 0; i < b->n; i++) {
    const fk_grid* g = b->grids[i];
    bcells[b->bucket[i]] += (double)g->nx * g->nv1 * g->pitch;
    bmax_nx[b->bucket[i]] = std::max(bmax_nx[b->bucket[i]], g->nx);
  }
  std::vector<int> order(b->n_buckets);
  for (int q = 0; q < b->n_buckets; q++) order[q] = q;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return bcells[x] > bcells[y]; });
  s = trial(&ms);  // warm-up (first touch of the plan)
  if (s == FK_OK) s = trial(&best);
  std::vector<int> keep = b->chunk_len;
  std::vector<int> keep_caps(b->n);
  for (int i = 0; i < b->n; i++) keep_caps[i] = b->grids[i]->tile_cap;
  for (size_t oi = 0; oi < order.size() && s == FK_OK; oi++) {
    const int q = order[oi];
    bool half_bucket = true;
    for (int i = 0; i < b->n; i++)
      if (b->bucket[i] == q) half_bucket = half_bucket && b->grids[i]->geom.half;
    // tile plans: the grids' current ones, then (tile search, whole-CTA
    // buckets) caps of about kTileCellTargets cells per tile plane where
    // they cut a grid's tiles
    std::vector<std::vector<int>> plans(1, keep_caps);
    if (tiles && !half_bucket)
      for (const int cells : kTileCellTargets) {
        std::vector<int> caps = keep_caps;
        bool cuts = false;
        for (int i = 0; i < b->n; i++)
          if (b->bucket[i] == q && !b->grids[i]->geom.half) {  // half units keep their tiles
            const fk_grid* g = b->grids[i];
            caps[i] = std::max(4, cells / g->pitch);
            cuts |= caps[i] < std::max(g->geom.ti_neg, g->geom.ti_pos);
          }
        if (cuts) plans.push_back(caps);
      }
    for (size_t pi = 0; pi < plans.size() && s == FK_OK; pi++) {
      if (pi > 0) {  // a new tile plan: time it at the best chunking so far first
        s = set_caps(q, plans[pi]);
        if (s == FK_OK) s = trial(&ms);
        if (s == FK_OK && ms < best) {
          best = ms;
          keep_caps = plans[pi];
        }
      }
      // candidate chunk lengths: powers of two from kMinChunk up to the
      // bucket's largest x range, and the lengths whose chunk count gives the
      // bucket about a whole number k of waves of unit slots (equal units
      // otherwise leave the last wave part-empty)
      std::vector<int> cand;
      for (int L = kMinChunk;; L *= 2) {
        cand.push_back(std::min(L, bmax_nx[q]));
        if (L >= bmax_nx[q]) break;
      }
      double row_units = 0.0;  // units of one chunk of every grid in the bucket
      for (int i = 0; i < b->n; i++)
        if (b->bucket[i] == q) row_units += b->grids[i]->geom.n_tiles;
      // unit slots of the launch the bucket's units run in
      const double slots =
          (double)b->sms * (half_bucket ? 2.0 * b->per_sm_half : (double)b->per_sm_whole);
      for (int k = 1; k <= 12 && row_units > 0.0; k++) {
        const int c = std::max(1, (int)std::lround(k * slots / row_units));
        const int L = (bmax_nx[q] + c - 1) / c;
        if (L >= kMinChunk && L <= bmax_nx[q]) cand.push_back(L);
      }
      std::sort(cand.begin(), cand.end());
      cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
      for (size_t ci = 0; ci < cand.size() && s == FK_OK; ci++) {
        const int Lc = cand[ci];
        bool changed = false;
        for (int i = 0; i < b->n; i++)
          if (b->bucket[i] == q) {
            const int len = even_chunk_len(b->grids[i]->nx, Lc);
            changed |= len != b->chunk_len[i];
            b->chunk_len[i] = len;
          }
        if (changed) {
          b->dirty = true;
          s = trial(&ms);
          if (s == FK_OK && ms < best) {
            best = ms;
            keep = b->chunk_len;
            keep_caps = plans[pi];
          }
        }
        b->chunk_len = keep;
        b->dirty = true;
      }
    }
    if (s == FK_OK) s = set_caps(q, keep_caps);  // the bucket's best tile plan
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (steps_taken) *steps_taken = taken;
  return s;
}

}  // namespace

fk_status fk_batch_autotune(fk_batch* b, int32_t steps_per_trial, int64_t* steps_taken) {
  return autotune(b, steps_per_trial, steps_taken, false);
}

fk_status fk_batch_autotune_tiles(fk_batch* b, int32_t steps_per_trial, int64_t* steps_taken) {
  return autotune(b, steps_per_trial, steps_taken, true);
}

fk_status fk_batch_set_kernel_timing(fk_batch* b, int enabled) {
  if (!b) return FK_EINVAL;
  BK_CUDA(b, cudaSetDevice(b->dev));
  if (enabled && b->ev.empty()) {
    b->ev.resize(2 * kBatchMaxTimed, nullptr);
    for (auto& e : b->ev) BK_CUDA(b, cudaEventCreate(&e));
  }
  BK_CUDA(b, cudaStreamSynchronize(b->stream));
  b->timing = enabled != 0;
  b->ev_used = 0;
  return FK_OK;
}

fk_status fk_batch_kernel_timing(fk_batch* b, int64_t* launches, double* total_ms) {
  if (!b || !launches || !total_ms) return FK_EINVAL;
  BK_CUDA(b, cudaSetDevice(b->dev));
  BK_CUDA(b, cudaStreamSynchronize(b->stream));
  double tot = 0.0;
  for (int r = 0; r < b->ev_used; r++) {
    float ms = 0.f;
    BK_CUDA(b, cudaEventElapsedTime(&ms, b->ev[2 * r], b->ev[2 * r + 1]));
    tot += ms;
  }
  *launches = b->ev_used;
  *total_ms = tot;
  b->ev_used = 0;
  return FK_OK;
}

const char* fk_batch_last_error(const fk_batch* b) {
  return b ? b->err.c_str() : g_batch_create_error.c_str();
}

}  // extern "C"
