// Streaming step kernel: one explicit upwind step of Eq. 2 (Sun et al.,
// arXiv 2303.14119, Sec. 2) over the whole phase-space grid, one read of
// f^n and one write of f^{n+1} per cell.
//
// Decomposition.  A CTA owns one unit = (tile of v1 rows [i0, i1) times all
// v2 cells, chunk of consecutive x-planes), or two units of thin tiles, one
// per half of the CTA.  All rows of a tile have the same sign of v1, so the
// x-upwind neighbour of plane k is plane k - dir for the whole tile; the
// unit marches through its chunk in the direction dir, and every consumer
// thread keeps the previous plane's input values of its own cells in
// registers: the x-neighbour never comes from memory twice.
//
// Pipeline.  Planes arrive in shared memory through cp.async.bulk copies
// (the TMA engine) into a ring of stages (kStages for a whole-CTA unit,
// kHalfStages for a half-CTA unit, whose planes are small).  Each stage holds the
// tile's rows plus the one v1 halo row on the upwind side of that plane's
// c_1.  Warp roles:
//  - consumer warps (kWarps): wait until a stage is full, update their cells
//    (FP32/INT work only on the FP32 path), store f^{n+1}, sum it per warp,
//    and release the stage;
//  - the producer warp: when a stage is released, read what the partial
//    sums of its plane need (the warp sums; the outflow of f^n through the
//    downwind velocity edges, still in the stage), refill the stage, then
//    fold them into the per-(plane, tile) partial sums (on x = 0 and
//    x = h_max with the wall fluxes of Eqs. 12-14 and the vacuum outflow
//    of f^{n+1}).
// There is no block-wide barrier inside the march.
//
// Per cell: f' = f + |c_x|(f_ux - f) + |c_1|(f_u1 - f) + |c_2|(f_u2 - f) + dt S
// (FP32: increment form) or the convex form of the same sum (FP64).
#include <type_traits>
#include <stdint.h>

#include "fk_internal.cuh"

namespace fk {

namespace {

constexpr int kThreads = 224;            // consumer threads of a whole-CTA unit (7 warps)
constexpr int kWarps = kThreads / 32;    // its consumer warps; one producer warp follows
constexpr int kBlock = kThreads + 32;
// Thin tiles (few cells per plane) run two units per CTA, each on one half:
// 3 consumer warps and its own producer warp, stages and mbarriers.
constexpr int kHalfThreads = 96;
constexpr int kHalfBlock = kHalfThreads + 32;
static_assert(2 * kHalfBlock == kBlock, "two half units fill one CTA");
constexpr int kStages = 4;      // stages of a whole-CTA unit
constexpr int kHalfStages = 4;  // stages of a half-CTA unit
static_assert(kHalfStages <= 32, "a producer lane per stage");
// stages of a unit on NT consumer threads
template <int NT>
__host__ __device__ constexpr int unit_stages() { return NT == kThreads ? kStages : kHalfStages; }
constexpr int kVecPerThread = 8;         // 16-byte vectors per consumer thread and plane
constexpr int kHalfVecPerThread32 = 3;   // the same for half units of FP32 grids
// vectors per consumer thread and plane of a unit on NT threads, element size E
template <int NT, int E>
__host__ __device__ constexpr int unit_vectors() {
  return (NT == kHalfThreads && E == 4) ? kHalfVecPerThread32 : kVecPerThread;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) accesses to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with the given parity; false if it did not complete
// within *limit cycles (read only when the first try fails).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const long long* limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long lim = *limit;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > lim) return false;
  return true;
}

template <typename T>
struct alignas(16) Vec {
  static constexpr int N = 16 / sizeof(T);
  T e[N];
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T upd(T f, T fx, T fv, T fw, T ax, T a1, T a2, T s, T d);
template <>
__device__ __forceinline__ float upd<float>(float f, float fx, float fv, float fw, float ax,
                                            float a1, float a2, float s, float) {
  const float inc = fmaf(a2, fw - f, fmaf(a1, fv - f, fmaf(ax, fx - f, s)));
  return f + inc;
}
template <>
__device__ __forceinline__ double upd<double>(double f, double fx, double fv, double fw,
                                              double ax, double a1, double a2, double s,
                                              double d) {
  // every weight is >= 0 under the CFL condition: nothing cancels
  return fma(a2, fw, fma(a1, fv, fma(ax, fx, fma(d, f, s))));
}

template <typename T>
__host__ __device__ constexpr size_t stage_bytes(int stage_elems) {
  return ((size_t)stage_elems * sizeof(T) + 127) / 128 * 128;
}
// The dynamic shared memory of both kernels starts with a slot for the
// unit's StepArgs (filled by the batched kernel), so that one tile plan fits
// a grid stepped alone or in a batch.  After the slot and the stages come:
// mbarriers full[NS], empty[NS] (NS stages); warp sums [NS][kWarps][4]
// (a half unit uses the first 3 warps of each stage)
// (density, wall primary flux, wall secondary flux, vacuum outflow); for
// FP64 grids the per-stage diagonal 1 - |c_x| - |c_1| - |c_2| (- dt nu) of
// every tile row [NS][kMaxTileRows] double, for FP32 grids the
// separable source factors of the tile rows [kMaxTileRows] and of the row
// cells [pitch] (float); the BGK equilibrium factors of Eq. 5 (FP32 grids:
// m1 of the tile rows [kMaxTileRows] and m2 [pitch], float; FP64 grids:
// dt nu_k n_k m1 per stage and tile row [NS][kMaxTileRows] and m2
// [pitch], double); control words: the sticky flags and a withheld
// pipeline item (ints), the wait limit (long long, at byte 8).
constexpr int kArgsBytes = 384;  // a multiple of 128: the stages stay 128-byte aligned
static_assert(sizeof(StepArgs) <= kArgsBytes && sizeof(StepArgs) % 8 == 0,
              "StepArgs must fit its shared-memory slot");
constexpr int kWs = 4;
constexpr int kMaxTileRows = 64;  // also bounds the per-stage row tables
template <typename T, int NS>
__host__ __device__ constexpr size_t tail_main_bytes(int pitch) {
  return sizeof(T) == 8 ? NS * kMaxTileRows * sizeof(double)
                        : ((size_t)(kMaxTileRows + pitch) * sizeof(float) + 15) / 16 * 16;
}
template <typename T, int NS>
__host__ __device__ constexpr size_t tail_bgk_bytes(int pitch) {
  return sizeof(T) == 8 ? (NS * kMaxTileRows + (size_t)pitch) * sizeof(double)
                        : ((size_t)(kMaxTileRows + pitch) * sizeof(float) + 15) / 16 * 16;
}
template <typename T, int NS>
__host__ __device__ constexpr size_t tail_bytes(int pitch) {
  return kArgsBytes + 2 * NS * sizeof(uint64_t) + NS * kWarps * kWs * sizeof(double) +
         tail_main_bytes<T, NS>(pitch) + tail_bgk_bytes<T, NS>(pitch) + 16;
}

// Exact split of a double x with 2^-126 <= |x| < 2^128 into hi + lo floats:
// hi keeps the top 24 significant bits (truncated), lo the remaining 29
// rounded to 24 bits, so hi + lo = x to about 2^-47 relative.  Integer and
// FP32 operations only: none of this runs on GB300's narrow FP64 pipe.
// Smaller magnitudes (and zero) give 0 + 0, negligible in a sum of
// phase-space densities; |x| >= 2^128, infinities and NaN give a NaN hi, so
// the sum they enter is flagged as non-finite.
__device__ __forceinline__ void split_double(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int h32 = (unsigned int)(b >> 32);
  const int E = (int)((h32 >> 20) & 0x7FF);
  const unsigned int sign = h32 & 0x80000000u;
  const unsigned int m23 = (unsigned int)(b >> 29) & 0x7FFFFFu;
  const bool ok = E >= 897 && E <= 1150;  // hi is a normal float
  const unsigned int out_of_range = E > 1150 ? 0x7FC00000u : 0u;  // quiet NaN
  hi = __int_as_float(ok ? (sign | ((unsigned int)(E - 896) << 23) | m23) : out_of_range);
  const unsigned int r29 = (unsigned int)b & 0x1FFFFFFFu;
  // scale 2^(E-1075) as a float: exponent field E - 948 (0 below 2^-74)
  const float scale = __int_as_float(E >= 949 ? ((unsigned int)(E - 948) << 23) : 0u);
  const float l = __uint2float_rn(r29) * scale;
  lo = ok ? (sign ? -l : l) : 0.f;
}
// Debug-bounds build (-DFK_DEBUG_BOUNDS): the step kernel checks the index
// of each shared- and global-memory access and of each bulk copy against its
// buffer first; a failed check sets kFlagBounds in the grid's state and the
// access is skipped (a skipped copy still completes its stage's phase).  In
// the release build every check is the constant true.
#ifdef FK_DEBUG_BOUNDS
__device__ __forceinline__ bool in_bounds(bool ok, DevState* st) {
  if (!ok) atomicOr(&st->flags, kFlagBounds);
  return ok;
}
#else
__device__ __forceinline__ constexpr bool in_bounds(bool, DevState*) { return true; }
#endif

// s + c += x, exactly in s (TwoSum), the rounding error collected in c
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float x) {
  const float t = s + x;
  const float bp = t - s;
  c += (s - (t - bp)) + (x - bp);
  s = t;
}

// FP32 pairs x.x + x.y, for the wall sums of FP32 grids' half units:
// the leading product of a pair by a float or a pair is exact (TwoProd
// with a fused multiply-add), sums take TwoSum of the leading parts and add
// the trailing parts (Dekker 1971; Knuth, TAOCP Vol. 2, 4.2.2), about 44
// bits in all, on the FP32 pipe instead of GB300's narrow FP64 one.
__device__ __forceinline__ float2 pair_mul(float2 a, float b) {
  const float p = a.x * b;
  float e = fmaf(a.x, b, -p);
  e = fmaf(a.y, b, e);
  return make_float2(p, e);
}
__device__ __forceinline__ float2 pair_mul(float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  return make_float2(p, e);
}
__device__ __forceinline__ void pair_acc(float2& s, float2 x) {
  two_sum_acc(s.x, s.y, x.x);
  s.y += x.y;
}
// sum over the warp, valid in lane 0
__device__ __forceinline__ float2 pair_warp_sum(float2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_down_sync(0xffffffffu, v.x, o);
    const float ol = __shfl_down_sync(0xffffffffu, v.y, o);
    two_sum_acc(v.x, v.y, oh);
    v.y += ol;
  }
  return v;
}

// Wall (x = 0, v1 < 0: Eqs. 12-14) or vacuum (x = h_max, v1 > 0) sums of
// f^{n+1} over this consumer thread's cells of one plane, read back from
// its own stores; returns whether one of those cells is negative.  Called
// only on those two planes of a march, so the main loop carries no FP64
// instruction for them.
template <typename T>
__device__ __noinline__ bool wall_terms(const T* oplane, const double* v1tab,
                                        const double* delta, int tid, int nthreads, int i0,
                                        int rows, int nv2, int pitch, bool wall, double* out3) {
  constexpr int VEC = 16 / sizeof(T);
  const int QV = pitch / VEC;
  double pe = 0.0, see = 0.0, vac = 0.0;
  bool neg = false;
  for (int m = 0; m < kVecPerThread; m++) {
    const int v = tid + nthreads * m;
    if (v >= rows * QV) break;
    const int r = v / QV, q = v - (v / QV) * QV;
    const int i = i0 + r;
    const double v1 = v1tab[i];
    for (int e = 0; e < VEC && q * VEC + e < nv2; e++) {
      const size_t c = (size_t)i * pitch + q * VEC + e;
      const double fn = (double)oplane[c];
      neg = neg || fn < 0.0;
      if (wall) {
        const double g = -v1 * fn;  // Eq. 13 without dv1 dv2
        pe += g;
        see += delta[c] * g;  // Eq. 12
      } else {
        vac += v1 * fn;
      }
    }
  }
  out3[0] = pe;
  out3[1] = see;
  out3[2] = vac;
  return neg;  // a value of the plane is negative
}

// The same sums for the half-CTA units of FP32 grids, in FP32 pairs (v1
// and delta as pairs, exact leading products) and folded over the warp
// (out3 valid in lane 0): thin tiles run three CTAs to an SM, and there the
// FP64 instructions of the two boundary planes held up whole units.
__device__ __noinline__ bool wall_terms_pairs(const float* oplane, const float2* v1p,
                                              const float2* deltap, int tid, int nthreads,
                                              int i0, int rows, int nv2, int pitch, bool wall,
                                              double* out3) {
  const int QV = pitch / 4;
  float2 pe = make_float2(0.f, 0.f), see = pe, vac = pe;
  bool neg = false;
  for (int m = 0; m < kVecPerThread; m++) {
    const int v = tid + nthreads * m;
    if (v >= rows * QV) break;
    const int r = v / QV, q = v - (v / QV) * QV;
    const int i = i0 + r;
    const float2 v1 = v1p[i];
    for (int e = 0; e < 4 && q * 4 + e < nv2; e++) {
      const size_t c = (size_t)i * pitch + q * 4 + e;
      const float fn = oplane[c];
      neg = neg || fn < 0.f;
      const float2 g = pair_mul(v1, fn);
      if (wall) {
        const float2 mg = make_float2(-g.x, -g.y);  // Eq. 13 without dv1 dv2
        pair_acc(pe, mg);
        pair_acc(see, pair_mul(deltap[c], mg));  // Eq. 12
      } else {
        pair_acc(vac, g);
      }
    }
  }
  pe = pair_warp_sum(pe);
  see = pair_warp_sum(see);
  vac = pair_warp_sum(vac);
  out3[0] = (double)pe.x + (double)pe.y;
  out3[1] = (double)see.x + (double)see.y;
  out3[2] = (double)vac.x + (double)vac.y;
  return neg;  // a value of the thread's cells is negative
}

// Barrier over the threads of one unit: the whole CTA (barrier 0), or one
// half of it (named barrier 1 or 2, kHalfBlock threads).
template <int NT>
__device__ __forceinline__ void unit_sync(int bar) {
  if constexpr (NT == kThreads) {
    __syncthreads();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(NT + 32) : "memory");
  }
}

// A pointer field of the step arguments read where it is used.  SA: the
// arguments sit in the CTA's shared memory (batched kernels), and a read
// there at each use (an LDS) keeps the pointer out of the registers of the
// march; otherwise they are kernel parameters, which instructions take
// directly.
template <bool SA, typename X>
__device__ __forceinline__ X arg_at_use(const X& field) {
  static_assert(sizeof(X) == 8, "pointer fields");
  if constexpr (SA) {
    unsigned long long v;
    asm volatile("ld.shared.b64 %0, [%1];"
                 : "=l"(v)
                 : "r"((unsigned)__cvta_generic_to_shared(&field)));
    return reinterpret_cast<X>(v);
  } else {
    return field;
  }
}

// One unit (tile t, chunk) of a grid on NT consumer threads (kThreads, or
// kHalfThreads for a half-CTA unit) plus a producer warp; tid: the thread's
// index within the unit, bar: the unit's barrier; smem is the unit's shared
// memory past its argument slot.  BGK: the grid has the electron-electron
// collision term of Eq. 3 switched on.  SA: a is in shared memory.
template <typename T, bool PADDED, bool BGK, int NT, bool SA>
__device__ __forceinline__ void stream_unit(const StepArgs& a, const int t, const int chunk,
                                            unsigned char* smem, const int tid, const int bar) {
  constexpr int NW = NT / 32;  // consumer warps
  constexpr int NS = unit_stages<NT>();  // stages of the ring
  constexpr int VEC = Vec<T>::N;
  constexpr int M = unit_vectors<NT, (int)sizeof(T)>();
  // per-plane pointer reads from the shared-memory arguments at their use
  // where the march runs out of registers (half units, the collision
  // variant); elsewhere the pointers stay in registers (measured faster)
  constexpr bool SAU = SA && (NT == kHalfThreads || BGK);
  // compact index arithmetic (an item's plane in one multiply-add, 32-bit
  // stage and plane sizes): faster in the half-unit, padded-row and
  // collision variants, 1 % slower in the plain whole-CTA one (measured)
  constexpr bool COMPACT = NT == kHalfThreads || PADDED || BGK;
  using StageSz = std::conditional_t<COMPACT, unsigned, size_t>;  // < 227 KB
  using PlaneSz = std::conditional_t<COMPACT, int, size_t>;
  const Geom& gm = a.geom;
  const StageSz sbytes = (StageSz)stage_bytes<T>(gm.stage_elems);
  unsigned char* stage_base = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NS * sbytes);
  uint64_t* empty = full + NS;
  double* wsum = reinterpret_cast<double*>(empty + NS);  // [NS][kWarps][kWs]
  double* dgl = wsum + NS * kWarps * kWs;  // [NS][kMaxTileRows], FP64
  float* srow_s = reinterpret_cast<float*>(dgl);  // [kMaxTileRows], FP32
  float* scol_s = srow_s + kMaxTileRows;          // [pitch], FP32
  unsigned char* bgk_base = reinterpret_cast<unsigned char*>(dgl) + tail_main_bytes<T, NS>(a.pitch);
  double* dgs = reinterpret_cast<double*>(bgk_base);  // [NS][kMaxTileRows], FP64
  double* m2d = dgs + NS * kMaxTileRows;         // [pitch], FP64
  float* m1_s = reinterpret_cast<float*>(bgk_base);   // [kMaxTileRows], FP32
  float* m2_s = m1_s + kMaxTileRows;                  // [pitch], FP32
  int* ctl = reinterpret_cast<int*>(bgk_base + tail_bgk_bytes<T, NS>(a.pitch));

  const int lane = tid & 31, warp = tid >> 5;
  const int nt = gm.n_tiles;
  const int nx = a.nx, nv1 = a.nv1, nv2 = a.nv2, pitch = a.pitch;
  int i0, i1, dir;
  tile_rows(gm, nv1, t, &i0, &i1, &dir);
  const int s0 = chunk * gm.chunk_len;
  const int s1 = min(nx, s0 + gm.chunk_len);
  if (s0 >= s1 || i0 >= i1) return;  // uniform over the block
  // the tile fits its row tables and a stage holds it with its halo row
  if (!in_bounds(i0 >= 0 && i1 <= nv1 && i1 - i0 <= kMaxTileRows &&
                     (i1 - i0 + 1) * pitch <= gm.stage_elems,
                 a.st))
    return;  // uniform over the block

  // march: step s visits plane k(s); the upwind plane of the first one is
  // loaded first ("prime" item) unless it lies outside the domain
  const int k_first = dir > 0 ? s0 : nx - 1 - s0;
  const int k_up = k_first - dir;
  const bool prime = k_up >= 0 && k_up < nx;
  const int n_items = (s1 - s0) + (prime ? 1 : 0);
  // item q visits plane k_first + dir (q - 1) after a prime item (q = 0:
  // k_up), plane k_first + dir q without one
  const int k_item0 = prime ? k_up : k_first;
  auto item_plane = [&](int q) -> int {
    if constexpr (COMPACT) {
      return k_item0 + dir * q;
    } else {
      const int s = s0 + q - (prime ? 1 : 0);
      if (s < s0) return k_up;
      return dir > 0 ? s : nx - 1 - s;
    }
  };

  if (sizeof(T) == 4) {  // source factors of this tile (FP32 grids)
    for (int r = tid; r < i1 - i0; r += NT + 32) srow_s[r] = a.tab.srow32[i0 + r];
    for (int j = tid; j < pitch; j += NT + 32) scol_s[j] = a.tab.scol32[j];
  }
  if (BGK) {  // factors of the collision equilibrium (Eq. 5)
    if (sizeof(T) == 4) {
      for (int r = tid; r < i1 - i0; r += NT + 32) m1_s[r] = a.tab.m1_32[i0 + r];
      for (int j = tid; j < pitch; j += NT + 32) m2_s[j] = a.tab.m2_32[j];
    } else {
      for (int j = tid; j < pitch; j += NT + 32) m2d[j] = a.tab.m2[j];
    }
  }
  long long* wlim = reinterpret_cast<long long*>(ctl + 2);  // bounded waits' limit (cycles)
  if (tid == 0) {
    ctl[0] = (int)a.st->flags;
    // test knob: the pipeline item whose copy this unit does not issue
    ctl[1] = (t == 0 && chunk == 0) ? a.prm->withhold_item : -1;
    *wlim = a.prm->wait_limit;
    for (int s = 0; s < NS; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NT);
    }
    fence_mbar_init();
  }
  unit_sync<NT>(bar);
  if (ctl[0]) return;  // sticky error: freeze the state (uniform)

  const Params& p = *a.prm;
  const T* __restrict__ fin = static_cast<const T*>(a.f_in);
  T* __restrict__ fout = static_cast<T*>(a.f_out);
  // cells of a plane (below 2^31, as a streamed row holds at most one
  // unit's cells, 7168, and nv1 <= 65536)
  const PlaneSz plane = (PlaneSz)nv1 * pitch;
  const int QV = pitch / VEC;  // vectors per row
  const int stage_n = gm.stage_elems;     // elements of a stage
  const size_t f_n = (size_t)nx * plane;  // elements of f
  const int rows = i1 - i0;

  if (warp == NW) {
    // ============================ producer warp ============================
    // Per item q: wait until every consumer released the stage of item
    // q - NS, read what its partial sums need from that stage and from
    // the warp sums (gather), refill the stage with item q (issue), then
    // reduce and store the partial sums of item q - NS (finish): the
    // reductions run while the copy is in flight.
    //
    // c_1 (FP32 copy) of item q sits in lane q % 32 of c1w (items wbase ..
    // wbase + 31) or of c1n (the next 32 items, loaded a window ahead);
    // lane st of c1slot / a1slot holds c_1 and |c_1| (FP64 grids) of the
    // item in stage st.
    const T a2t = (T)fabs(p.c2);
    const bool has_a2 = p.c2 != 0.0;
    float c1w = lane < n_items ? a.c1_32[item_plane(lane)] : 0.f;
    float c1n = lane + 32 < n_items ? a.c1_32[item_plane(lane + 32)] : 0.f;
    int wbase = 0;
    float c1slot = 0.f;
    double a1slot = 0.0;
    // all 32 lanes: where the upwind v1 halo row lies outside the velocity
    // grid, fill its slot with zeros (zero inflow through the v1 edge) so
    // the consumers read a neighbour row without a bounds test; then lane 0
    // copies plane k's tile rows plus the halo row inside the grid
    auto issue = [&](int q) {
      if (q == wbase + 32) {  // next window; prefetch the one after
        c1w = c1n;
        wbase += 32;
        c1n = wbase + 32 + lane < n_items ? a.c1_32[item_plane(wbase + 32 + lane)] : 0.f;
      }
      const int k = item_plane(q);
      const float c1 = __shfl_sync(0xffffffffu, c1w, q & 31);
      const int st = q % NS;
      if (lane == st) c1slot = c1;
      T* stage = reinterpret_cast<T*>(stage_base + st * sbytes);
      // stage layout: the tile's rows start at row 1 when the halo lies
      // above (c_1 > 0), at row 0 otherwise (halo, if any, at row `rows`)
      int zrow = -1;
      if (c1 > 0.f && i0 == 0) zrow = 0;
      if (c1 < 0.f && i1 == nv1) zrow = rows;
      if (zrow >= 0 && in_bounds((zrow + 1) * pitch <= stage_n, a.st)) {
        float4* z = reinterpret_cast<float4*>(stage + (size_t)zrow * pitch);
        const int n16 = pitch * (int)sizeof(T) / 16;
        for (int c = lane; c < n16; c += 32) z[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        // a later bulk copy (async proxy) may land on these bytes when c_1
        // changes sign: order the zero stores (generic proxy) before it
        fence_proxy_async_smem();
      }
      if (sizeof(T) == 8) {
        // FP64 diagonal of the convex update per tile row, once per plane
        // here rather than per vector in the consumers
        const double a1 = c1 == 0.f ? 0.0 : fabs(a.c1[k]);
        if (lane == st) a1slot = a1;
        double db = 1.0 - a1 - fabs(p.c2);
        if (BGK) db -= a.bgk[k];  // the loss part of the collision term, dt nu_k f
        for (int r = lane; r < rows; r += 32) dgl[st * kMaxTileRows + r] = db - fabs(a.tab.cx[i0 + r]);
        if (BGK) {  // its gain part per tile row: dt nu_k n_k m1[i]
          const double sk = a.bgk[nx + k];
          for (int r = lane; r < rows; r += 32) dgs[st * kMaxTileRows + r] = sk * a.tab.m1[i0 + r];
        }
      }
      __syncwarp();
      if (lane == 0 && q != ctl[1]) {  // ctl[1]: a withheld item (test knob), else -1
        int lo = i0, hi = i1;
        if (c1 > 0.f && i0 > 0) lo = i0 - 1;  // v1 halo row on the upwind side
        if (c1 < 0.f && i1 < nv1) hi = i1 + 1;
        const int dofs = (lo - i0 + (c1 > 0.f ? 1 : 0)) * pitch;  // in the stage
        const size_t sofs = (size_t)k * plane + (size_t)lo * pitch;  // in f
        T* dst = stage + dofs;
        const T* src = fin + sofs;
        const uint32_t bytes = (uint32_t)((hi - lo) * pitch * sizeof(T));
        if (in_bounds(k >= 0 && k < nx && lo >= 0 && hi <= nv1 && dofs >= 0 &&
                          dofs + (hi - lo) * pitch <= stage_n &&
                          sofs + (size_t)(hi - lo) * pitch <= f_n,
                      a.st)) {
          mbar_expect_tx(&full[st], bytes);  // release: the zero row is visible too
          bulk_g2s(dst, src, bytes, &full[st]);
        } else {
          mbar_expect_tx(&full[st], 0);  // no data: the stage's phase completes
        }
      }
    };
    // What the partial sums of a consumed compute item need from its stage
    // and from the warp sums, read before the stage is refilled.
    struct Gathered {
      int k;       // plane (-1: the prime item, no sums)
      T lvt;       // this lane's share of the velocity-edge outflow
      float wsf;   // lane w < NW, FP32 grids: warp w's density sum
      double ws[kWs];  // lane w < NW: warp w's sums (all four on a wall plane)
    };
    auto gather = [&](int q) -> Gathered {
      Gathered g;
      g.k = -1;
      g.lvt = (T)0;
      g.wsf = 0.f;
#pragma unroll
      for (int i = 0; i < kWs; i++) g.ws[i] = 0.0;
      if (prime && q == 0) return g;
      const int k = item_plane(q);
      const int st = q % NS;
      g.k = k;
      const T* sb = reinterpret_cast<const T*>(stage_base + st * sbytes);
      const float c1f = __shfl_sync(0xffffffffu, c1slot, st);
      const double a1d = sizeof(T) == 8 ? __shfl_sync(0xffffffffu, a1slot, st) : 0.0;
      // ledger: outflow of f^n through the downwind velocity edges, summed
      // in the grid's precision (a ledger diagnostic: FP32 grids keep FP64
      // instructions off this per-plane path)
      const T a1t = sizeof(T) == 4 ? (T)fabsf(c1f) : (T)a1d;
      const int erow = (c1f > 0.f && i1 == nv1) ? nv1 - 1 : ((c1f < 0.f && i0 == 0) ? 0 : -1);
      const int rb = c1f > 0.f ? 1 : 0;  // stage row of the tile's first row
      if (erow >= 0 && in_bounds(erow - i0 + rb >= 0 && (erow - i0 + rb + 1) * pitch <= stage_n,
                                 a.st)) {
        const T* r = sb + (size_t)(erow - i0 + rb) * pitch;
        for (int j = lane; j < nv2; j += 32) g.lvt += a1t * r[j];
      }
      if (has_a2 && in_bounds((rows - 1 + rb) * pitch + nv2 <= stage_n, a.st))
        for (int r = lane; r < rows; r += 32) g.lvt += a2t * sb[(size_t)(r + rb) * pitch + nv2 - 1];
      if (lane < NW) {
        const double* ws = wsum + (st * kWarps + lane) * kWs;
        // FP32 grids hand over their warp's density sum as a float
        g.ws[0] = sizeof(T) == 4 ? (double)0 : ws[0];
        if constexpr (sizeof(T) == 4) g.wsf = *reinterpret_cast<const float*>(ws);
        if (k == 0 || k == nx - 1) {
#pragma unroll
          for (int i = 1; i < kWs; i++) g.ws[i] = ws[i];
        }
      }
      return g;
    };
    // fold the gathered sums (the warps' in a fixed order) and store them
    auto finish = [&](const Gathered& g) {
      if (g.k < 0) return;
      const int k = g.k;
      const double lv = (double)warp_sum(g.lvt);
      double sum[kWs] = {0.0, 0.0, 0.0, 0.0};
      const bool wall = k == 0 || k == nx - 1;
      float sumf = 0.f;  // FP32 grids: the warps' density sums, added in FP32
#pragma unroll
      for (int w = 0; w < NW; w++) {
        if constexpr (sizeof(T) == 4)
          sumf += __shfl_sync(0xffffffffu, g.wsf, w);
        else
          sum[0] += __shfl_sync(0xffffffffu, g.ws[0], w);
        if (wall) {
#pragma unroll
          for (int i = 1; i < kWs; i++) sum[i] += __shfl_sync(0xffffffffu, g.ws[i], w);
        }
      }
      if constexpr (sizeof(T) == 4) sum[0] = (double)sumf;  // one conversion per plane
      if (lane == 0 && in_bounds(k >= 0 && k < nx && t >= 0 && t < nt, a.st)) {
        a.part.n[(size_t)k * nt + t] = sum[0];
        a.part.lv[(size_t)k * nt + t] = lv;
        if (k == 0) {
          a.part.pe[t] = sum[1];
          a.part.see[t] = sum[2];
        }
        if (k == nx - 1) a.part.vac[t] = sum[3];
      }
    };
    int issued = 0;
    bool ok = true;
    for (int q = 0; q < n_items; q++) {
      Gathered g{};
      g.k = -1;
      if (q >= NS) {
        // stage reuse: wait until every consumer thread released item q - NS
        ok = __all_sync(0xffffffffu,
                        mbar_wait(&empty[q % NS], (uint32_t)(((q / NS) - 1) & 1), wlim));
        if (!ok) break;
        g = gather(q - NS);
        __syncwarp();  // the stage is read by every lane before it is refilled
      }
      issue(q);
      issued = q + 1;
      finish(g);
    }
    for (int q = max(0, issued - NS); q < issued && ok; q++) {
      ok = __all_sync(0xffffffffu, mbar_wait(&empty[q % NS], (uint32_t)((q / NS) & 1), wlim));
      if (ok) finish(gather(q));
    }
    if (!ok && lane == 0) {
      atomicOr(&a.st->flags, kFlagTimeout);
      // copies still in flight land before the CTA leaves (a withheld
      // item's copy was never issued: nothing to wait for)
      for (int q = max(0, issued - NS); q < issued; q++)
        if (q != ctl[1]) mbar_wait(&full[q % NS], (uint32_t)((q / NS) & 1), wlim);
    }
    return;
  }

  // ============================ consumer warps =============================
  // this thread's cells: vectors v = tid + NT*m of the tile, fixed for
  // the whole march; per vector its offset in a stage and in a plane
  int soff[M];  // offset from the tile's first cell (low 24 bits) and row (top byte)
  const int gbase = i0 * pitch;  // the tile's first cell in a plane
  // bit m: vector m exists / starts a row; zleft bit 16 + m: vector m is
  // the last of a padded row (pitch > nv2: only a row's last vector holds
  // padding, its elements from nv2 - (pitch - VEC) on)
  unsigned valid = 0, zleft = 0;
  T ax[M];
  T xr[M][VEC];
#pragma unroll
  for (int m = 0; m < M; m++) {
    const int v = tid + NT * m;
    soff[m] = 0;
    ax[m] = (T)0;
    if (v < rows * QV) {
      const int r = v / QV, qv = v - r * QV;
      valid |= 1u << m;
      if (qv == 0) zleft |= 1u << m;
      if (PADDED && qv == QV - 1 && pitch != nv2) zleft |= 1u << (16 + m);
      soff[m] = (r * pitch + qv * VEC) | (r << 24);
      const T cx = sizeof(T) == 8 ? (T)a.tab.cx[i0 + r] : (T)a.tab.cx32[i0 + r];
      ax[m] = cx < (T)0 ? -cx : cx;
    }
#pragma unroll
    for (int e = 0; e < VEC; e++) xr[m][e] = (T)0;
  }
  if (!prime && dir > 0) {
    // first plane is x = 0 with v1 > 0: the upwind value is the re-emitted
    // distribution Gamma_see g_se of Eq. 15 (zero for the vacuum side)
    // (plus, with reflection, refl times the incident f^n of the mirror
    // cell at -v1 on the same plane)
    const double gsee = a.st->g_see;
    const double refl = p.refl;
#pragma unroll
    for (int m = 0; m < M; m++) {
      if (!(valid >> m & 1)) continue;
      const int r = soff[m] >> 24;
      const int c0 = (soff[m] & 0xFFFFFF) - r * pitch;
#pragma unroll
      for (int e = 0; e < VEC; e++) {
        double g = gsee * a.tab.gse[(soff[m] & 0xFFFFFF) + gbase + e];
        if (refl > 0.0)
          g += refl * (double)fin[(size_t)(nv1 - 1 - (i0 + r)) * pitch + c0 + e];
        xr[m][e] = (T)g;
      }
    }
  }
  const T c2 = (T)p.c2;
  const T a2 = c2 < (T)0 ? -c2 : c2;
  // the source band in registers: the march's stores could alias Params
  const int band_lo = p.band_lo, band_hi = p.band_hi;
  const T* srcbase = sizeof(T) == 8 ? (const T*)a.tab.src : (const T*)a.tab.src32;

  for (int q = 0; q < n_items; q++) {
    const int st = q % NS;
    const bool compute = !(prime && q == 0);
    const int k = item_plane(q);
    // per-plane values and the source row (L2-resident table) are fetched
    // before waiting for the stage, so their latency overlaps the wait
    const float c1f = arg_at_use<SAU>(a.c1_32)[k];
    const T a1 =
        c1f == 0.f ? (T)0 : (sizeof(T) == 8 ? (T)fabs(arg_at_use<SAU>(a.c1)[k]) : (T)fabsf(c1f));
    const bool band = compute && k >= band_lo && k < band_hi;
    // source term: FP32 grids rebuild it from the separable factors in
    // shared memory, FP64 grids load the 2D table in the update loop
    // collision term (Eq. 3) of FP32 grids: dt nu_k and dt nu_k n_k (FP64
    // grids take it from the producer's row tables)
    T bgk_a = (T)0, bgk_s = (T)0;
    if (BGK && sizeof(T) == 4) {
      const float* b32 = arg_at_use<SAU>(a.bgk32);
      bgk_a = (T)b32[k];
      bgk_s = (T)b32[nx + k];
    }
    const bool ok = mbar_wait(&full[st], (uint32_t)((q / NS) & 1), wlim);
    if (__any_sync(0xffffffffu, !ok)) {
      if (lane == 0) atomicOr(&a.st->flags, kFlagTimeout);
      return;
    }
    // the tile's first row sits at stage row 1 when this plane's halo lies
    // above (c_1 > 0), at row 0 otherwise
    const int sbo = c1f > 0.f ? pitch : 0;  // sb's offset in the stage
    const T* sb = reinterpret_cast<const T*>(stage_base + st * sbytes) + sbo;
    if (!compute) {
#pragma unroll
      for (int m = 0; m < M; m++) {
        if (!(valid >> m & 1)) continue;
        if (!in_bounds(sbo + (int)(soff[m] & 0xFFFFFF) + VEC <= stage_n, a.st)) continue;
        const Vec<T> own = *reinterpret_cast<const Vec<T>*>(sb + (soff[m] & 0xFFFFFF));
#pragma unroll
        for (int e = 0; e < VEC; e++) xr[m][e] = own.e[e];
      }
    } else {
      // v1 upwind row: one row up (c_1 > 0), one down (c_1 < 0) or none;
      // the direction comes from the FP32 copy, as in the producer, so the
      // row read is always one that was copied or zero-filled
      const int nboff = c1f > 0.f ? -pitch : (c1f < 0.f ? pitch : 0);
      const double* dg = dgl + st * kMaxTileRows;
      T sum_n = (T)0;
      float sh_ = 0.f, sc_ = 0.f, sl_ = 0.f;  // FP64 grids: compensated FP32 sum
      T* oplane = (SAU ? static_cast<T*>(arg_at_use<SAU>(a.f_out)) : fout) + (size_t)k * plane;
#pragma unroll
      for (int m = 0; m < M; m++) {
        if (NT * m >= rows * QV) break;  // no thread of the unit has vector m (uniform)
        const int so = soff[m] & 0xFFFFFF;
        Vec<T> own;
        if ((valid >> m & 1) && in_bounds(sbo + so + VEC <= stage_n, a.st))
          own = *reinterpret_cast<const Vec<T>*>(sb + so);
        else
#pragma unroll
          for (int e = 0; e < VEC; e++) own.e[e] = (T)0;
        // v2 upwind (c_2 >= 0 since E_y <= 0): element j-1
        T left = __shfl_up_sync(0xffffffffu, own.e[VEC - 1], 1);
        if (!(valid >> m & 1)) continue;
        if (zleft >> m & 1)
          left = (T)0;
        else if (lane == 0)
          left = in_bounds(sbo + so - 1 >= 0, a.st) ? sb[so - 1] : (T)0;
        Vec<T> nb;
        if (in_bounds(sbo + so + nboff >= 0 && sbo + so + nboff + VEC <= stage_n, a.st))
          nb = *reinterpret_cast<const Vec<T>*>(sb + so + nboff);
        else
#pragma unroll
          for (int e = 0; e < VEC; e++) nb.e[e] = (T)0;
        const T d = sizeof(T) == 8 ? (T)dg[soff[m] >> 24] : (T)0;  // unused on FP32 grids
        Vec<T> src;
#pragma unroll
        for (int e = 0; e < VEC; e++) src.e[e] = (T)0;
        if (band) {
          if constexpr (sizeof(T) == 4) {
            const int r = soff[m] >> 24;
            const float sr = srow_s[r];
            const Vec<float> sc =
                *reinterpret_cast<const Vec<float>*>(scol_s + (so - r * pitch));
#pragma unroll
            for (int e = 0; e < VEC; e++) src.e[e] = sr * sc.e[e];
          } else {
            src = *reinterpret_cast<const Vec<T>*>(srcbase + so + gbase);
          }
        }
        if (BGK) {  // gain dt nu_k n_k m1[i] m2[j] of the collision term
          const int r = soff[m] >> 24;
          const int c0 = so - r * pitch;  // column of the vector's first cell
          if constexpr (sizeof(T) == 4) {
            const float ms = bgk_s * m1_s[r];
            const Vec<float> mv = *reinterpret_cast<const Vec<float>*>(m2_s + c0);
#pragma unroll
            for (int e = 0; e < VEC; e++) src.e[e] = fmaf(ms, mv.e[e], src.e[e]);
          } else {
            const double ms = dgs[st * kMaxTileRows + r];
            const Vec<double> mv = *reinterpret_cast<const Vec<double>*>(m2d + c0);
#pragma unroll
            for (int e = 0; e < VEC; e++) src.e[e] = fma(ms, mv.e[e], src.e[e]);
          }
        }
        Vec<T> out;
#pragma unroll
        for (int e = 0; e < VEC; e++) {
          const T f = own.e[e];
          const T fw = e == 0 ? left : own.e[e - 1];
          T se = src.e[e];
          if (BGK && sizeof(T) == 4) se = fmaf(-(float)bgk_a, (float)f, (float)se);  // loss dt nu f
          T fn = upd<T>(f, xr[m][e], nb.e[e], fw, ax[m], a1, a2, se, d);
          if (PADDED && (zleft >> (16 + m) & 1) && e >= nv2 - (pitch - VEC))
            fn = (T)0;  // row padding stays zero
          out.e[e] = fn;
          xr[m][e] = f;  // x-upwind value for the next plane is f^n here
          if (sizeof(T) == 4) {
            sum_n += fn;
          } else {
            float h, l;
            split_double((double)fn, h, l);
            two_sum_acc(sh_, sc_, h);
            sl_ += l;
          }
        }
        if (in_bounds((size_t)k * plane + gbase + so + VEC <= f_n, a.st))
          __stcs(reinterpret_cast<float4*>(oplane + so + gbase),
                 *reinterpret_cast<const float4*>(&out));
      }
      // warp sum of this plane's f^{n+1} (an FP32 grid sums its 32 lanes in
      // FP32; everything above a warp is FP64)
      double* wsl = wsum + (st * kWarps + warp) * kWs;
      if (sizeof(T) == 4) {
        const T ws = warp_sum(sum_n);
        if (lane == 0) *reinterpret_cast<float*>(wsl) = ws;  // the producer converts once
      } else {
        // fold the lanes' (hi, error) pairs in FP32 with TwoSum, convert once
        float lo = sc_ + sl_;
        for (int o = 16; o > 0; o >>= 1) {
          const float oh = __shfl_down_sync(0xffffffffu, sh_, o);
          const float ol = __shfl_down_sync(0xffffffffu, lo, o);
          float c = 0.f;
          two_sum_acc(sh_, c, oh);
          lo += ol + c;
        }
        if (lane == 0) wsl[0] = (double)sh_ + (double)lo;
      }
      const bool wall = k == 0 && dir < 0, vout = k == nx - 1 && dir > 0;
      if (wall || vout) {  // uniform over the block
        double b3[3];
        if constexpr (sizeof(T) == 4 && NT == kHalfThreads) {
          const bool neg = wall_terms_pairs(oplane, a.tab.v1p, a.tab.deltap, tid, NT, i0, rows,
                                            nv2, pitch, wall, b3);
          if (__any_sync(0xffffffffu, neg) && lane == 0) atomicOr(&a.st->flags, kFlagNegative);
          if (lane == 0) {
            wsl[1] = b3[0];
            wsl[2] = b3[1];
            wsl[3] = b3[2];
          }
        } else {
          const bool neg =
              wall_terms<T>(oplane, a.tab.v1, a.tab.delta, tid, NT, i0, rows, nv2, pitch, wall, b3);
          if (__any_sync(0xffffffffu, neg) && lane == 0) atomicOr(&a.st->flags, kFlagNegative);
          const double w1 = warp_sum(b3[0]), w2 = warp_sum(b3[1]), w3 = warp_sum(b3[2]);
          if (lane == 0) {
            wsl[1] = w1;
            wsl[2] = w2;
            wsl[3] = w3;
          }
        }
      } else if (k == 0 || k == nx - 1) {
        if (lane == 0) wsl[1] = wsl[2] = wsl[3] = 0.0;
      }
    }
    mbar_arrive(&empty[st]);  // this thread is done with stage st
  }
}

// Shared memory of one unit: argument slot, stages and tail.  A CTA of two
// half units holds two such regions, each rounded up to 128 bytes.
template <typename T, int NS>
__host__ __device__ constexpr size_t unit_smem_bytes(int stage_elems, int pitch) {
  return NS * stage_bytes<T>(stage_elems) + tail_bytes<T, NS>(pitch);
}
template <typename T>
__host__ __device__ constexpr size_t half_region_bytes(int stage_elems, int pitch) {
  return (unit_smem_bytes<T, kHalfStages>(stage_elems, pitch) + 127) / 128 * 128;
}

// One grid, whole-CTA units: CTA b runs tile b % n_tiles of chunk
// b / n_tiles.
template <typename T, bool PADDED, bool BGK>
__global__ void __launch_bounds__(kBlock, 2) step_stream_kernel(const __grid_constant__ StepArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int nt = a.geom.n_tiles;
  stream_unit<T, PADDED, BGK, kThreads, false>(a, blockIdx.x % nt, blockIdx.x / nt, smem + kArgsBytes,
                                        threadIdx.x, 0);
}

// One grid, half units: CTA b runs units 2b and 2b + 1 on its two halves,
// each in a region of half_region_bytes.
template <typename T, bool PADDED, bool BGK>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 3 : 2)
step_stream_half_kernel(const __grid_constant__ StepArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int nt = a.geom.n_tiles;
  const int h = threadIdx.x / kHalfBlock;
  const int u = 2 * blockIdx.x + h;
  if (u >= nt * a.geom.n_chunks) return;
  unsigned char* region = smem + h * half_region_bytes<T>(a.geom.stage_elems, a.pitch);
  stream_unit<T, PADDED, BGK, kHalfThreads, false>(a, u % nt, u / nt, region + kArgsBytes,
                                            threadIdx.x - h * kHalfBlock, 1 + h);
}

// Many grids in one launch, whole-CTA units: CTA b copies the arguments of
// grid units[b].x into the slot at the start of its shared memory and runs
// that grid's unit units[b].y = tile + n_tiles * chunk.
template <typename T, bool PADDED, bool BGK>
__global__ void __launch_bounds__(kBlock, 2)
step_stream_batch_kernel(const BatchInst* __restrict__ inst, const int2* __restrict__ units) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int2 u = units[blockIdx.x];
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&inst[u.x].a);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(smem);
  for (int w = threadIdx.x; w < (int)(sizeof(StepArgs) / 8); w += blockDim.x) dst[w] = src[w];
  __syncthreads();
  const StepArgs& a = *reinterpret_cast<const StepArgs*>(smem);
  const int nt = a.geom.n_tiles;
  stream_unit<T, PADDED, BGK, kThreads, true>(a, u.y % nt, u.y / nt, smem + kArgsBytes, threadIdx.x, 0);
}

// Many grids in one launch, half units: CTA b runs unit pairs[b].y of grid
// pairs[b].x on threads [0, kHalfBlock) and unit pairs[b].w of grid
// pairs[b].z (none if pairs[b].z < 0) on the rest, each half in a region of
// half_bytes whose slot receives that grid's arguments.
template <typename T, bool PADDED, bool BGK>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 3 : 2)
step_stream_batch_half_kernel(const BatchInst* __restrict__ inst, const int4* __restrict__ pairs,
                              int half_bytes) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int4 c = pairs[blockIdx.x];
  const int h = threadIdx.x / kHalfBlock, ht = threadIdx.x - h * kHalfBlock;
  const int g = h ? c.z : c.x, u = h ? c.w : c.y;
  unsigned char* region = smem + (size_t)h * half_bytes;
  if (g >= 0) {
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&inst[g].a);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(region);
    for (int w = ht; w < (int)(sizeof(StepArgs) / 8); w += kHalfBlock) dst[w] = src[w];
  }
  __syncthreads();
  if (g < 0) return;  // the idle half of a CTA with one unit
  const StepArgs& a = *reinterpret_cast<const StepArgs*>(region);
  const int nt = a.geom.n_tiles;
  stream_unit<T, PADDED, BGK, kHalfThreads, true>(a, u % nt, u / nt, region + kArgsBytes, ht, 1 + h);
}

}  // namespace

int stream_tile_rows(int precision, int pitch, int smem_per_sm, int reserved_per_block,
                     bool half) {
  const int esize = precision == FK_F32 ? 4 : 8;
  const int vec = 16 / esize;
  const int cells = half ? kHalfThreads * (esize == 4 ? unit_vectors<kHalfThreads, 4>()
                                                    : unit_vectors<kHalfThreads, 8>()) * vec
                         : kThreads * kVecPerThread * vec;
  if (pitch > cells) return 0;
  int rows = cells / pitch;
  if (rows > kMaxTileRows) rows = kMaxTileRows;
  // two CTAs per SM: each unit holds its stages (kStages, or kHalfStages for
  // a half unit) of (rows + 1) * pitch elements (a half unit gets half of
  // its CTA, less the region's rounding)
  const int ns = half ? kHalfStages : kStages;
  const long tail =
      (long)(precision == FK_F32
                 ? (half ? tail_bytes<float, kHalfStages>(pitch) : tail_bytes<float, kStages>(pitch))
                 : (half ? tail_bytes<double, kHalfStages>(pitch)
                         : tail_bytes<double, kStages>(pitch)));
  const long cta = (long)smem_per_sm / 2 - reserved_per_block;
  const long budget = (half ? cta / 2 - 127 : cta) - tail;
  const long stage = budget / ns / 128 * 128;
  const long fit = stage / ((long)pitch * esize) - 1;  // one halo slot per stage
  if (fit < rows) rows = (int)fit;
  return rows > 0 ? rows : 0;
}

size_t stream_smem_bytes(int precision, int stage_elems, int pitch) {
  return precision == FK_F32 ? unit_smem_bytes<float, kStages>(stage_elems, pitch)
                             : unit_smem_bytes<double, kStages>(stage_elems, pitch);
}

size_t stream_half_bytes(int precision, int stage_elems, int pitch) {
  return precision == FK_F32 ? half_region_bytes<float>(stage_elems, pitch)
                             : half_region_bytes<double>(stage_elems, pitch);
}

size_t stream_cta_smem_bytes(int precision, const Geom& gm, int pitch) {
  return gm.half ? 2 * stream_half_bytes(precision, gm.stage_elems, pitch)
                 : stream_smem_bytes(precision, gm.stage_elems, pitch);
}

namespace {
// allow the device's largest opt-in shared memory for kernel k and ask how
// many CTAs of smem_bytes fit on an SM
// allow the device's largest opt-in shared memory for kernel k and ask how
// many CTAs of smem_bytes fit on an SM; *best keeps the smallest answer of
// the kernels that count (count = false: the attribute is only set)
template <typename K>
cudaError_t fit_kernel(K k, int optin, size_t smem_bytes, bool count, int* best) {
  int n = 0;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kBlock, smem_bytes);
  if (e == cudaSuccess && count && n < *best) *best = n;
  return e;
}
template <typename T, bool P, bool B>
cudaError_t fit_four(int optin, size_t smem_bytes, bool whole, bool half, int* best) {
  cudaError_t e = fit_kernel(step_stream_kernel<T, P, B>, optin, smem_bytes, whole, best);
  if (e == cudaSuccess) e = fit_kernel(step_stream_batch_kernel<T, P, B>, optin, smem_bytes, whole, best);
  if (e == cudaSuccess) e = fit_kernel(step_stream_half_kernel<T, P, B>, optin, smem_bytes, half, best);
  if (e == cudaSuccess)
    e = fit_kernel(step_stream_batch_half_kernel<T, P, B>, optin, smem_bytes, half, best);
  return e;
}
template <typename T>
int ctas_per_sm(int optin, size_t smem_bytes, int layout) {
  const bool whole = layout != kLayoutHalf, half = layout != kLayoutWhole;
  int best = 1 << 30;
  cudaError_t e = fit_four<T, false, false>(optin, smem_bytes, whole, half, &best);
  if (e == cudaSuccess) e = fit_four<T, true, false>(optin, smem_bytes, whole, half, &best);
  if (e == cudaSuccess) e = fit_four<T, false, true>(optin, smem_bytes, whole, half, &best);
  if (e == cudaSuccess) e = fit_four<T, true, true>(optin, smem_bytes, whole, half, &best);
  return e == cudaSuccess ? best : 0;
}
}  // namespace

int stream_ctas_per_sm(int precision, size_t smem_bytes, int layout) {
  // the attribute is per kernel, shared by every grid and batch: allow the
  // device's largest opt-in size on every variant, and ask the occupancy of
  // this size (the smallest over the single-grid and batched variants of
  // the layout asked for; the half-unit kernels of FP32 grids fit more
  // CTAs on an SM than the whole-CTA ones)
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  if (smem_bytes > (size_t)optin) return 0;
  return precision == FK_F32 ? ctas_per_sm<float>(optin, smem_bytes, layout)
                             : ctas_per_sm<double>(optin, smem_bytes, layout);
}

namespace {
template <typename T, bool BGK>
void launch_single(const StepArgs& a, int grid, size_t smem, bool padded, bool half,
                   cudaStream_t s) {
  if (half) {
    if (padded)
      step_stream_half_kernel<T, true, BGK><<<grid, kBlock, smem, s>>>(a);
    else
      step_stream_half_kernel<T, false, BGK><<<grid, kBlock, smem, s>>>(a);
  } else {
    if (padded)
      step_stream_kernel<T, true, BGK><<<grid, kBlock, smem, s>>>(a);
    else
      step_stream_kernel<T, false, BGK><<<grid, kBlock, smem, s>>>(a);
  }
}
template <typename T, bool BGK>
void launch_batch(const BatchInst* inst, const int2* units, int n_units, size_t smem,
                  const int4* pairs, int n_pairs, int half_bytes, bool padded, cudaStream_t s) {
  if (n_units > 0) {
    if (padded)
      step_stream_batch_kernel<T, true, BGK><<<n_units, kBlock, smem, s>>>(inst, units);
    else
      step_stream_batch_kernel<T, false, BGK><<<n_units, kBlock, smem, s>>>(inst, units);
  }
  if (n_pairs > 0) {
    const size_t hs = 2 * (size_t)half_bytes;
    if (padded)
      step_stream_batch_half_kernel<T, true, BGK><<<n_pairs, kBlock, hs, s>>>(inst, pairs, half_bytes);
    else
      step_stream_batch_half_kernel<T, false, BGK><<<n_pairs, kBlock, hs, s>>>(inst, pairs, half_bytes);
  }
}
}  // namespace

cudaError_t launch_step_stream(const StepArgs& a, int precision, bool bgk, cudaStream_t s) {
  const int units = a.geom.n_tiles * a.geom.n_chunks;
  const bool half = a.geom.half != 0;
  const int grid = half ? (units + 1) / 2 : units;
  const size_t smem = stream_cta_smem_bytes(precision, a.geom, a.pitch);
  const bool padded = a.pitch != a.nv2;
  if (precision == FK_F32) {
    if (bgk)
      launch_single<float, true>(a, grid, smem, padded, half, s);
    else
      launch_single<float, false>(a, grid, smem, padded, half, s);
  } else {
    if (bgk)
      launch_single<double, true>(a, grid, smem, padded, half, s);
    else
      launch_single<double, false>(a, grid, smem, padded, half, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_step_stream_batch(const BatchInst* inst, const int2* units, int n_units,
                                     const int4* pairs, int n_pairs, int precision, bool padded,
                                     bool bgk, size_t smem_bytes, int half_bytes,
                                     cudaStream_t s) {
  if (n_units <= 0 && n_pairs <= 0) return cudaSuccess;
  if (precision == FK_F32) {
    if (bgk)
      launch_batch<float, true>(inst, units, n_units, smem_bytes, pairs, n_pairs, half_bytes,
                                padded, s);
    else
      launch_batch<float, false>(inst, units, n_units, smem_bytes, pairs, n_pairs, half_bytes,
                                 padded, s);
  } else {
    if (bgk)
      launch_batch<double, true>(inst, units, n_units, smem_bytes, pairs, n_pairs, half_bytes,
                                 padded, s);
    else
      launch_batch<double, false>(inst, units, n_units, smem_bytes, pairs, n_pairs, half_bytes,
                                  padded, s);
  }
  return cudaGetLastError();
}

}  // namespace fk
