// Set-up tables, the fused upwind step (direct-load variant), the finalize
// kernel (moments -> surface charge, field, Courant numbers, ledger,
// history) and the precision conversion used by fk_set_f / fk_get_f.
//
// Paper: Sun et al., arXiv 2303.14119, Sec. 2.
#include <math.h>

#include "fk_host.cuh"

namespace fk {

// ---------------------------------------------------------------------------
// Deterministic block reductions: fixed shuffle tree, fixed warp order.
template <int NT>
__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = l < NT / 32 ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

template <int NT>
__device__ double block_max(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = l < NT / 32 ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_down_sync(0xffffffffu, r, o));
  }
  return r;
}

// ---------------------------------------------------------------------------
// Tables, in three launches with deterministic sums:
//  1. kTabBlocks blocks over the cells: delta (SEE yield of Eqs. 8-11 where
//     v1 < 0), the raw Eq. 15 emission shape and the raw Eq. 7 source shape,
//     and per-block partial sums of their normalisations;
//  2. one block: the partials folded in block order, the 1D tables (v1, c_x)
//     and the separable source factors;
//  3. kTabBlocks blocks: gse scaled to unit flux sum v1 g dv1 dv2, src = dt
//     (J/e)/W times the source shape scaled to unit density.
// The per-cell special functions run in FP64 on every SM (GB300's FP64 rate
// per SM is small, so one block would take milliseconds).
constexpr int kTabBlocks = 256;
constexpr int kTabThreads = 256;
constexpr int kTabFoldThreads = 1024;

// x as an FP32 pair (hi, lo): hi = x rounded to FP32, lo = x - hi rounded.
__device__ __forceinline__ float2 split_pair(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}

// Cell centre lo + (i + 1/2) h with separate roundings (no fused multiply-
// add), so the velocity grid is bit-identical to a host computation.
__device__ __forceinline__ double cell_centre(double lo, int i, double h) {
  return __dadd_rn(lo, __dmul_rn((double)i + 0.5, h));
}

__global__ void __launch_bounds__(kTabThreads)
tables_cells_kernel(Tables t, int nv1, int nv2, int pitch, double v1_min, double v2_min,
                    double dv1, double dv2, double dmax, double amax, double ks, double Tse,
                    double Tfe) {
  __shared__ double sh[32];
  double s_se = 0.0, s_fe = 0.0;
  const int ncell = nv1 * pitch;
  for (int c = blockIdx.x * kTabThreads + threadIdx.x; c < ncell; c += kTabBlocks * kTabThreads) {
    const int i = c / pitch, j = c - (c / pitch) * pitch;
    double d = 0.0, gs = 0.0, gf = 0.0;
    if (j < nv2) {
      const double v1 = cell_centre(v1_min, i, dv1);
      const double v2 = cell_centre(v2_min, j, dv2);
      const double vv = v1 * v1 + v2 * v2;
      if (v1 < 0.0) {
        const double A = 0.5 * kMe * vv / kQe;                             // Eq. 10, eV
        const double al = atan(fabs(v2 / v1));                             // Eq. 11
        const double z = 1.284 * A / (amax * (1.0 + ks * al * al / kPi));  // Eq. 9
        if (z > 0.0)
          d = 1.526 * dmax * (1.0 + ks * al * al / (2.0 * kPi)) *
              (1.0 - exp(-pow(z, 1.725))) / pow(z, 0.725);  // Eq. 8
      }
      gs = v1 > 0.0 ? exp(-kMe * vv / (2.0 * Tse * kQe)) : 0.0;  // Eq. 15 shape
      s_se += v1 * gs;
      gf = v2 > 0.0 ? exp(-kMe * vv / (2.0 * Tfe * kQe)) : 0.0;  // Eq. 7 shape
      s_fe += gf;
    }
    t.delta[c] = d;
    t.gse[c] = gs;
    t.gfe_raw[c] = gf;
  }
  s_se = block_sum<kTabThreads>(s_se, sh);
  __syncthreads();
  s_fe = block_sum<kTabThreads>(s_fe, sh);
  if (threadIdx.x == 0) {
    t.tsum[2 * blockIdx.x] = s_se;
    t.tsum[2 * blockIdx.x + 1] = s_fe;
  }
}

__global__ void __launch_bounds__(kTabFoldThreads)
tables_fold_kernel(Tables t, int nv1, int nv2, int pitch, double v1_min, double v2_min,
                   double dv1, double dv2, double dt, double dx, double Tfe, double j_over_ew,
                   double Te) {
  __shared__ double sh[32];
  __shared__ double norms[6];
  // block partials in block order (one per thread, kTabBlocks <= threads)
  const int b = threadIdx.x;
  double s_se = b < kTabBlocks ? t.tsum[2 * b] : 0.0;
  double s_fe = b < kTabBlocks ? t.tsum[2 * b + 1] : 0.0;
  s_se = block_sum<kTabFoldThreads>(s_se, sh);
  __syncthreads();
  s_fe = block_sum<kTabFoldThreads>(s_fe, sh);
  for (int i = threadIdx.x; i < nv1; i += blockDim.x) {
    const double v1 = cell_centre(v1_min, i, dv1);
    t.v1[i] = v1;
    t.v1p[i] = split_pair(v1);
    t.cx[i] = __ddiv_rn(__dmul_rn(v1, dt), dx);
    t.cx32[i] = (float)t.cx[i];
  }
  // separable factors of the source shape (FP32 step kernel)
  double s1 = 0.0, s2 = 0.0;
  for (int i = threadIdx.x; i < nv1; i += blockDim.x) {
    const double v1 = cell_centre(v1_min, i, dv1);
    s1 += exp(-kMe * v1 * v1 / (2.0 * Tfe * kQe));
  }
  for (int j = threadIdx.x; j < nv2; j += blockDim.x) {
    const double v2 = cell_centre(v2_min, j, dv2);
    s2 += v2 > 0.0 ? exp(-kMe * v2 * v2 / (2.0 * Tfe * kQe)) : 0.0;
  }
  __syncthreads();
  s1 = block_sum<kTabFoldThreads>(s1, sh);
  __syncthreads();
  s2 = block_sum<kTabFoldThreads>(s2, sh);
  if (threadIdx.x == 0) {
    norms[0] = s_se * dv1 * dv2;
    norms[1] = s_fe * dv1 * dv2;
    norms[2] = s1 * dv1;
    norms[3] = s2 * dv2;
    t.tsum[2 * kTabBlocks] = norms[0];
    t.tsum[2 * kTabBlocks + 1] = norms[1];
  }
  __syncthreads();
  const double nfe = norms[1], n1 = norms[2], n2 = norms[3];
  const bool on = nfe > 0.0 && n1 > 0.0 && n2 > 0.0;
  for (int i = threadIdx.x; i < nv1; i += blockDim.x) {
    const double v1 = cell_centre(v1_min, i, dv1);
    t.srow32[i] = on ? (float)(dt * j_over_ew * exp(-kMe * v1 * v1 / (2.0 * Tfe * kQe)) / n1) : 0.f;
  }
  for (int j = threadIdx.x; j < pitch; j += blockDim.x) {
    double g = 0.0;
    if (on && j < nv2) {
      const double v2 = cell_centre(v2_min, j, dv2);
      g = v2 > 0.0 ? exp(-kMe * v2 * v2 / (2.0 * Tfe * kQe)) / n2 : 0.0;
    }
    t.scol32[j] = (float)g;
  }
  // factors of the BGK equilibrium of Eq. 5 at T_e (no drift), each
  // normalised on the grid to unit integral
  double e1 = 0.0, e2 = 0.0;
  for (int i = threadIdx.x; i < nv1; i += blockDim.x) {
    const double v1 = cell_centre(v1_min, i, dv1);
    e1 += exp(-kMe * v1 * v1 / (2.0 * Te * kQe));
  }
  for (int j = threadIdx.x; j < nv2; j += blockDim.x) {
    const double v2 = cell_centre(v2_min, j, dv2);
    e2 += exp(-kMe * v2 * v2 / (2.0 * Te * kQe));
  }
  __syncthreads();
  e1 = block_sum<kTabFoldThreads>(e1, sh);
  __syncthreads();
  e2 = block_sum<kTabFoldThreads>(e2, sh);
  if (threadIdx.x == 0) {
    norms[4] = e1 * dv1;
    norms[5] = e2 * dv2;
  }
  __syncthreads();
  const double ne1 = norms[4], ne2 = norms[5];
  for (int i = threadIdx.x; i < nv1; i += blockDim.x) {
    const double v1 = cell_centre(v1_min, i, dv1);
    const double m = exp(-kMe * v1 * v1 / (2.0 * Te * kQe)) / ne1;
    t.m1[i] = m;
    t.m1_32[i] = (float)m;
  }
  for (int j = threadIdx.x; j < pitch; j += blockDim.x) {
    double m = 0.0;
    if (j < nv2) {
      const double v2 = cell_centre(v2_min, j, dv2);
      m = exp(-kMe * v2 * v2 / (2.0 * Te * kQe)) / ne2;
    }
    t.m2[j] = m;
    t.m2_32[j] = (float)m;
  }
}

__global__ void __launch_bounds__(kTabThreads)
tables_scale_kernel(Tables t, int ncell, double dt, double j_over_ew) {
  const double nse = t.tsum[2 * kTabBlocks], nfe = t.tsum[2 * kTabBlocks + 1];
  for (int c = blockIdx.x * kTabThreads + threadIdx.x; c < ncell; c += kTabBlocks * kTabThreads) {
    t.gse[c] = nse > 0.0 ? t.gse[c] / nse : 0.0;
    t.deltap[c] = split_pair(t.delta[c]);
    const double s = nfe > 0.0 ? dt * j_over_ew * (t.gfe_raw[c] / nfe) : 0.0;
    t.src[c] = s;
    t.src32[c] = (float)s;
  }
}

int tables_scratch_doubles() { return 2 * kTabBlocks + 2; }

__global__ void scale_tables_kernel(const double* src, const float* src32, double s, int n,
                                    double* dst, float* dst32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    dst[i] = s * src[i];
    dst32[i] = (float)s * src32[i];
  }
}

cudaError_t launch_scale_tables(const double* src, const float* src32, double s, int n,
                                double* dst, float* dst32, cudaStream_t st) {
  scale_tables_kernel<<<(n + 255) / 256, 256, 0, st>>>(src, src32, s, n, dst, dst32);
  return cudaGetLastError();
}

cudaError_t launch_tables(const Tables& t, int nv1, int nv2, int pitch, double v1_min,
                          double v2_min, double dv1, double dv2, double dt, double dx,
                          double delta_max, double A_max, double k_s, double T_se,
                          double T_fe, double j_over_ew, double T_e, cudaStream_t s) {
  tables_cells_kernel<<<kTabBlocks, kTabThreads, 0, s>>>(t, nv1, nv2, pitch, v1_min, v2_min, dv1,
                                                         dv2, delta_max, A_max, k_s, T_se, T_fe);
  tables_fold_kernel<<<1, kTabFoldThreads, 0, s>>>(t, nv1, nv2, pitch, v1_min, v2_min, dv1, dv2,
                                                   dt, dx, T_fe, j_over_ew, T_e);
  tables_scale_kernel<<<kTabBlocks, kTabThreads, 0, s>>>(t, nv1 * pitch, dt, j_over_ew);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Direct-load step kernel.  One block per (plane k, tile t): the tile's rows
// [i0, i1) times all v2 cells.  Every neighbour is a plain load (L1/L2 catch
// the re-reads).  Used for the moments-only evaluation of a state and as the
// step for grids whose rows do not fit the streaming kernel's tiles.
//
// Per cell, with c_x = v1 dt/dx, c_1 = a1(x) dt/dv1, c_2 = a2 dt/dv2 and the
// upwind neighbour f_u in each direction (zero beyond a velocity edge or the
// vacuum side, Gamma_see g_se at the wall for v1 > 0):
//   f' = f - |c_x|(f - f_ux) - |c_1|(f - f_u1) - |c_2|(f - f_u2) + dt S
// which is the donor-cell flux difference of Eq. 2 written per cell.
constexpr int kStepThreads = 256;

template <typename T>
__device__ __forceinline__ T update_cell(T f, T fx, T fv, T fw, T ax, T a1, T a2, T s);

template <>
__device__ __forceinline__ double update_cell<double>(double f, double fx, double fv,
                                                      double fw, double ax, double a1,
                                                      double a2, double s) {
  // convex form: (1 - ax - a1 - a2) f + ax fx + a1 fv + a2 fw + s; every
  // weight is >= 0 under the CFL condition, so nothing cancels
  const double d = 1.0 - ax - a1 - a2;
  return fma(a2, fw, fma(a1, fv, fma(ax, fx, fma(d, f, s))));
}

template <>
__device__ __forceinline__ float update_cell<float>(float f, float fx, float fv, float fw,
                                                    float ax, float a1, float a2, float s) {
  // increment form: one rounding of f per step dominates the error
  const float inc = fmaf(a2, fw - f, fmaf(a1, fv - f, fmaf(ax, fx - f, s)));
  return f + inc;
}

// Per-thread accumulator of the density moment: FP64 grids add in FP64;
// FP32 grids keep a compensated FP32 sum (TwoSum: the running sum and its
// rounding errors), converted to FP64 once per thread.
template <typename T>
struct DensityAcc;
template <>
struct DensityAcc<double> {
  double s = 0.0;
  __device__ void add(double x) { s += x; }
  __device__ double value() const { return s; }
};
template <>
struct DensityAcc<float> {
  float s = 0.f, c = 0.f;
  __device__ void add(float x) {
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
  }
  __device__ double value() const { return (double)s + (double)c; }
};

template <typename T>
__global__ void __launch_bounds__(kStepThreads)
step_direct_kernel(StepArgs a, int mode) {
  __shared__ double sh[32];
  __shared__ unsigned s_flags;
  const int nt = a.part.nu;
  const int k = blockIdx.x / nt;
  const int t = blockIdx.x - k * nt;
  const Params& p = *a.prm;
  if (threadIdx.x == 0) s_flags = a.st->flags;
  __syncthreads();
  // mode: kPassFull, kPassMoments (moments of f_in only), kPassX (x-advection
  // with the wall and vacuum boundaries only), kPassV (v1, v2 advection,
  // source and collisions only): these two make the Lie-split step;
  // kPassXHalf and kPassXHalfLast (x-advection over dt/2, the second one
  // writing the partial sums of its output) with kPassV make the Strang step
  const bool moments_only = mode == kPassMoments;
  const bool xlast = mode == kPassXHalfLast;
  const bool xpass = mode == kPassX || mode == kPassXHalf || xlast, vpass = mode == kPassV;
  const T xscale = (mode == kPassXHalf || xlast) ? (T)0.5 : (T)1;  // dt/2: exact halving
  if (!moments_only && s_flags) return;  // sticky error: freeze the state
  const T* __restrict__ fin = static_cast<const T*>(a.f_in);
  T* __restrict__ fout = static_cast<T*>(a.f_out);
  const int nx = a.nx, nv1 = a.nv1, nv2 = a.nv2, pitch = a.pitch;
  const size_t plane = (size_t)nv1 * pitch;
  int i0, i1, dir;
  tile_rows(a.geom, nv1, t, &i0, &i1, &dir);
  // per-plane coefficients in the arithmetic type (no FP64 work per cell
  // on the FP32 path)
  const T c1 = xpass ? (T)0 : (sizeof(T) == 8 ? (T)a.c1[k] : (T)a.c1_32[k]);
  const T c2 = xpass ? (T)0 : (T)p.c2;
  const T a1 = c1 < (T)0 ? -c1 : c1, a2 = c2 < (T)0 ? -c2 : c2;
  const double gsee = a.st->g_see;
  const bool band = !xpass && k >= p.band_lo && k < p.band_hi;
  // BGK relaxation of this plane (Eq. 3): dt nu_k and dt nu_k n_k
  const bool coll = !xpass && p.collisions != 0;
  const T ca = coll ? (sizeof(T) == 8 ? (T)a.bgk[k] : (T)a.bgk32[k]) : (T)0;
  const T cs = coll ? (sizeof(T) == 8 ? (T)a.bgk[nx + k] : (T)a.bgk32[nx + k]) : (T)0;
  const int ncell = (i1 - i0) * nv2;
  DensityAcc<T> s_n;
  double s_lv = 0.0, s_pe = 0.0, s_see = 0.0, s_vac = 0.0;
  int neg = 0;  // a value written (or, moments only, read) is negative
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    const int i = i0 + c / nv2;
    const int j = c - (c / nv2) * nv2;
    const size_t idx = (size_t)k * plane + (size_t)i * pitch + j;
    const size_t tix = (size_t)i * pitch + j;
    const T f = fin[idx];
    T fn = f;
    if (!moments_only) {
      const T cx =
          vpass ? (T)0 : xscale * (sizeof(T) == 8 ? (T)a.tab.cx[i] : (T)a.tab.cx32[i]);
      T fx = (T)0;
      if (cx > (T)0)
        fx = k > 0 ? fin[idx - plane]
                   : (T)(gsee * a.tab.gse[tix] +
                         (p.refl > 0.0 ? p.refl * (double)fin[(size_t)(nv1 - 1 - i) * pitch + j]
                                       : 0.0));
      else if (cx < (T)0)
        fx = k < nx - 1 ? fin[idx + plane] : (T)0;
      T fv = (T)0;
      if (c1 > (T)0)
        fv = i > 0 ? fin[idx - pitch] : (T)0;
      else if (c1 < (T)0)
        fv = i < nv1 - 1 ? fin[idx + pitch] : (T)0;
      T fw = (T)0;
      if (c2 > (T)0)
        fw = j > 0 ? fin[idx - 1] : (T)0;
      else if (c2 < (T)0)
        fw = j < nv2 - 1 ? fin[idx + 1] : (T)0;
      T s = (T)0;
      if (band) s = sizeof(T) == 8 ? (T)a.tab.src[tix] : (T)a.tab.src32[tix];
      fn = update_cell<T>(f, fx, fv, fw, cx < (T)0 ? -cx : cx, a1, a2, s);
      if (coll) {
        const T m = sizeof(T) == 8 ? (T)(a.tab.m1[i] * a.tab.m2[j])
                                   : (T)a.tab.m1_32[i] * (T)a.tab.m2_32[j];
        fn += cs * m - ca * f;
      }
      fout[idx] = fn;
      // loss through the downwind velocity edges, from f^n (ledger)
      if ((c1 > (T)0 && i == nv1 - 1) || (c1 < (T)0 && i == 0)) s_lv += (double)a1 * (double)f;
      if ((c2 > (T)0 && j == nv2 - 1) || (c2 < (T)0 && j == 0)) s_lv += (double)a2 * (double)f;
    }
    s_n.add(fn);
    neg |= fn < (T)0;
    if (k == 0 && dir < 0) {
      const double g = -a.tab.v1[i] * (double)fn;  // Eq. 13 without dv1 dv2
      s_pe += g;
      s_see += a.tab.delta[tix] * g;  // Eq. 12
    }
    if (k == nx - 1 && dir > 0) s_vac += a.tab.v1[i] * (double)fn;
  }
  if (__syncthreads_or(neg) && threadIdx.x == 0) atomicOr(&a.st->flags, kFlagNegative);
  // the velocity pass (and the last pass of a Strang step) writes the
  // partial sums (uniform)
  if (xpass && !xlast) return;
  const double n_tot = block_sum<kStepThreads>(s_n.value(), sh);
  s_lv = block_sum<kStepThreads>(s_lv, sh);
  if (k == 0) {
    s_pe = block_sum<kStepThreads>(s_pe, sh);
    s_see = block_sum<kStepThreads>(s_see, sh);
  }
  if (k == nx - 1) s_vac = block_sum<kStepThreads>(s_vac, sh);
  if (threadIdx.x == 0) {
    a.part.n[(size_t)k * nt + t] = n_tot;
    if (!xlast) a.part.lv[(size_t)k * nt + t] = s_lv;  // Strang: the velocity pass's
    if (k == 0) {
      a.part.pe[t] = s_pe;
      a.part.see[t] = s_see;
    }
    if (k == nx - 1) a.part.vac[t] = s_vac;
  }
}

cudaError_t launch_step_pass(const StepArgs& a, int precision, int mode, cudaStream_t s) {
  const int nblk = a.nx * a.part.nu;
  if (precision == FK_F32)
    step_direct_kernel<float><<<nblk, kStepThreads, 0, s>>>(a, mode);
  else
    step_direct_kernel<double><<<nblk, kStepThreads, 0, s>>>(a, mode);
  return cudaGetLastError();
}

cudaError_t launch_step(const StepArgs& a, int precision, int moments_only, cudaStream_t s) {
  return launch_step_pass(a, precision, moments_only ? kPassMoments : kPassFull, s);
}

// ---------------------------------------------------------------------------
// Finalize, after every step kernel (and after a moments-only evaluation).
//
// Phase A, one thread per x-plane over kFinBlocks-sized blocks: the plane's
// density n_k from its tile partials (fixed order), the velocity-edge loss,
// and the exclusive prefix of n within the block.  Phase B, run by the last
// block to finish (a counter in FinScratch decides which; its sums are in a
// fixed order, so the result does not depend on which block it is):
//  - step mode: ledger += dt * (fluxes of f^n), sigma^{n+1} = sigma^n +
//    e dt (Gamma_see^n - Gamma_pe^n)  (Eq. 18 summed with Eq. 14), step++;
//    in the Strang step mode the wall and vacuum terms of f^n weigh dt/2
//    (the other half was added after the velocity pass);
//  - the fluxes of the new state (Eqs. 12-14), N, and the history row;
//  - E_x from Gauss's law integrated from the wall, E_x(0) = sigma/(2 eps0)
//    (the Poisson problem of Sec. 2), c_1 = -e E_x dt / (m_e dv1);
//  - CFL and finiteness checks (sticky flags) and the convergence test
//    (Sec. 2, paragraph after Eq. 18).
// Spreading phase A over many SMs matters on GB300, whose FP64 rate per SM
// is a small fraction of its FP32 rate.
constexpr int kFinThreads = 128;
constexpr int kFinMaxBlocks = 64;  // nx <= 8192

// Block blk of nblk finalizing one grid.
__device__ __forceinline__ void finalize_body(const StepArgs& a, const FinOut& o, const int blk,
                                              const int nblk, const int mode) {
  double* const ne = o.ne;
  double* const Ex = o.Ex;
  double* const c1 = o.c1;
  float* const c1_32 = o.c1_32;
  double* const hist = o.hist;
  const FinScratch& fs = o.fs;
  __shared__ double sh[32];
  __shared__ double wscan[kFinThreads / 32];
  __shared__ int s_last;
  __shared__ double bc[4];
  __shared__ double boff[kFinMaxBlocks];  // phase B: sum of n over blocks below
  const Params& p = *a.prm;
  DevState* st = a.st;
  const bool stepping = mode == kModeStep || mode == kModeStepStrang;
  if (stepping && st->flags) return;
  const int nx = a.nx, nu = a.part.nu;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int k = blk * kFinThreads + t;
  // ---- phase A
  double nk = 0.0, lk = 0.0;
  if (k < nx) {
    // loads batched ahead of the (fixed-order) adds: in-order issue would
    // otherwise serialise one L2 round trip per partial
    const double* pn = a.part.n + (size_t)k * nu;
    const double* pl = a.part.lv + (size_t)k * nu;
    double sn = 0.0, sl = 0.0;
    int u = 0;
    for (; u + 8 <= nu; u += 8) {
      double xn[8], xl[8];
#pragma unroll
      for (int q = 0; q < 8; q++) {
        xn[q] = pn[u + q];
        xl[q] = pl[u + q];
      }
#pragma unroll
      for (int q = 0; q < 8; q++) {
        sn += xn[q];
        sl += xl[q];
      }
    }
    for (; u < nu; u++) {
      sn += pn[u];
      sl += pl[u];
    }
    nk = sn * p.dvv;
    lk = sl;
    ne[k] = nk;
  }
  double incl = nk;
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  double excl = __shfl_up_sync(0xffffffffu, incl, 1);
  if (lane == 0) excl = 0.0;
  if (lane == 31) wscan[w] = incl;
  __syncthreads();
  double woff = 0.0;
  for (int q = 0; q < w; q++) woff += wscan[q];
  if (k < nx) fs.pre[k] = woff + excl;  // sum of n over the block's planes below k
  const double btot = block_sum<kFinThreads>(nk, sh);
  const double blv = block_sum<kFinThreads>(lk, sh);
  if (t == 0) {
    fs.bsum[blk] = btot;
    fs.blv[blk] = blv;
    __threadfence();
    s_last = atomicAdd(fs.counter, 1) == nblk - 1;
  }
  __syncthreads();
  if (!s_last) return;
  // ---- phase B (last block)
  __threadfence();
  const int nb = nblk;
  if (w == 0) {
    // block totals and their exclusive prefix, wall-flux tile partials:
    // lane-strided loads, fixed shuffle trees (other blocks' results are
    // read past L1 with __ldcg)
    const double b0 = lane < nb ? __ldcg(fs.bsum + lane) : 0.0;
    const double b1 = lane + 32 < nb ? __ldcg(fs.bsum + lane + 32) : 0.0;
    double l = (lane < nb ? __ldcg(fs.blv + lane) : 0.0) +
               (lane + 32 < nb ? __ldcg(fs.blv + lane + 32) : 0.0);
    double i0s = b0, i1s = b1;  // inclusive scans of the two halves
    for (int o = 1; o < 32; o <<= 1) {
      const double y0 = __shfl_up_sync(0xffffffffu, i0s, o);
      const double y1 = __shfl_up_sync(0xffffffffu, i1s, o);
      if (lane >= o) {
        i0s += y0;
        i1s += y1;
      }
    }
    const double half = __shfl_sync(0xffffffffu, i0s, 31);
    if (lane < nb) boff[lane] = i0s - b0;
    if (lane + 32 < nb) boff[lane + 32] = half + i1s - b1;
    const double ntot_raw = half + __shfl_sync(0xffffffffu, i1s, 31);
    double pe = 0.0, see = 0.0, vac = 0.0;
    for (int u = lane; u < nu; u += 32) {
      pe += a.part.pe[u];
      see += a.part.see[u];
      vac += a.part.vac[u];
    }
    for (int o = 16; o > 0; o >>= 1) {
      l += __shfl_down_sync(0xffffffffu, l, o);
      pe += __shfl_down_sync(0xffffffffu, pe, o);
      see += __shfl_down_sync(0xffffffffu, see, o);
      vac += __shfl_down_sync(0xffffffffu, vac, o);
    }
    if (lane == 0) {
      *fs.counter = 0;  // ready for the next launch
      DevState d = *st;  // one batch of loads, updated in registers
      const double ntot = ntot_raw * p.dx;
      pe *= p.dvv;
      // secondaries come from the absorbed part (1 - refl) of the primaries;
      // with SEE off every absorbed primary is deposited
      see = p.see_enabled ? see * p.dvv * (1.0 - p.refl) : 0.0;
      vac *= p.dvv;
      if (stepping) {
        const double lv = l * p.lv_scale;
        const double hw = mode == kModeStepStrang ? 0.5 * p.dt : p.dt;  // wall terms' share
        d.cum_emit += hw * (d.g_see + p.refl * d.g_pe);  // secondaries and reflected
        d.cum_see += hw * d.g_see;
        d.cum_pe += hw * d.g_pe;
        d.cum_vac += hw * d.g_vac;
        d.cum_lv += p.dt * lv;
        d.cum_inj += p.dt * p.inj;
        d.sigma += kQe * hw * (d.g_see - (1.0 - p.refl) * d.g_pe);
        d.step += 1;
      }
      if (mode == kModeReset) {
        d.step = 0;
        d.hist_count = 0;
        d.sat_step = -1;
        d.cum_emit = d.cum_see = d.cum_pe = d.cum_vac = d.cum_lv = d.cum_inj = 0.0;
        d.sigma0 = d.sigma;
        d.n0 = ntot;
      }
      d.g_pe = pe;
      d.g_see = see;
      d.g_vac = vac;
      d.n_tot = ntot;
      if (!isfinite(pe) || !isfinite(see) || !isfinite(vac) || !isfinite(ntot) ||
          !isfinite(d.sigma))
        d.flags |= kFlagNumeric;
      *st = d;  // one batch of stores
      bc[0] = d.sigma;
    }
  }
  __syncthreads();
  const double e_wall = bc[0] * p.ex_sigma;
  // E_x at cell centres and the v1-Courant numbers.  The planes' prefix
  // sums and densities (other blocks' results) are loaded kLd at a time, and
  // the coefficients once, ahead of the stores, past which the compiler
  // cannot move a load.
  const bool self_cons = p.self_consistent, coll = p.collisions;
  const double ex_n = p.ex_n, ex_ext = p.Ex_ext, c1_per_ex = p.c1_per_ex, bgk_c = p.bgk_c;
  const double cx_max = p.cx_max, ac2 = fabs(p.c2), dt = p.dt, sat_tol = p.sat_tol;
  const long long cap = p.hist_cap, window = p.sat_window;
  double cmax = 0.0, ex0 = 0.0;
  constexpr int kLd = 8;
  for (int k0 = t; k0 < nx; k0 += kLd * kFinThreads) {
    double pre_l[kLd], ne_l[kLd];
#pragma unroll
    for (int j = 0; j < kLd; j++) {
      const int kk = k0 + j * kFinThreads;
      pre_l[j] = kk < nx ? __ldcg(fs.pre + kk) : 0.0;
      ne_l[j] = kk < nx ? __ldcg(ne + kk) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < kLd; j++) {
      const int kk = k0 + j * kFinThreads;
      if (kk >= nx) break;
      const double below = boff[kk / kFinThreads] + pre_l[j];
      const double n_k = ne_l[j];
      const double e = self_cons ? e_wall - ex_n * (below + 0.5 * n_k) : ex_ext;
      if (kk == 0) ex0 = e;
      Ex[kk] = e;
      const double c = c1_per_ex * e;
      c1[kk] = c;
      c1_32[kk] = (float)c;
      double cfl = fabs(c);
      if (coll) {
        // BGK coefficients of the new state (Eqs. 3-4): dt nu_k = bgk_c n_k
        const double ak = n_k > 0.0 ? bgk_c * n_k : 0.0;
        a.bgk[kk] = ak;
        a.bgk[nx + kk] = ak * n_k;
        a.bgk32[kk] = (float)ak;
        a.bgk32[nx + kk] = (float)(ak * n_k);
        cfl += ak;  // the collision term takes part in the positivity bound
      }
      cmax = fmax(cmax, cfl);
    }
  }
  cmax = block_max<kFinThreads>(cmax, sh);
  __syncthreads();
  if (t == 0) {
    DevState d = *st;
    if (cmax + cx_max + ac2 > 1.0 + 1e-12) d.flags |= kFlagCfl;
    const long long row = d.step;
    double rr[FK_HISTORY_COLS] = {(double)row, (double)row * dt, d.sigma, d.g_pe,
                                  d.g_see, d.g_vac, d.n_tot, ex0};
    double* r = hist + (size_t)(row % cap) * FK_HISTORY_COLS;
    for (int q = 0; q < FK_HISTORY_COLS; q++) r[q] = rr[q];
    if (row + 1 > d.hist_count) d.hist_count = row + 1;
    if (stepping && d.sat_step < 0 && row >= window && window < cap) {
      const double* o = hist + (size_t)((row - window) % cap) * FK_HISTORY_COLS;
      bool ok = true;
      for (int q = 2; q <= 4; q++)
        if (!(fabs(rr[q] - o[q]) <= sat_tol * fabs(rr[q]))) ok = false;
      if (ok) d.sat_step = row;
    }
    st->flags = d.flags;
    st->hist_count = d.hist_count;
    st->sat_step = d.sat_step;
  }
}

__global__ void __launch_bounds__(kFinThreads)
finalize_kernel(const __grid_constant__ StepArgs a, const __grid_constant__ FinOut o, int mode) {
  finalize_body(a, o, blockIdx.x, gridDim.x, mode);
}

// One grid of at most kFinThreads planes (one finalize block) in step mode,
// on one warp: the arithmetic of finalize_body run with a single block, in
// the same fixed order -- each plane's partials in order, per 32-plane group
// the warp scan and shuffle trees of that group's warp, the group totals
// folded as block_sum's warp 0 folds them, phase B's scans over one block
// total -- so the new state is bit for bit the one finalize_body gives.
// A single block needs no last-block election, so the atomic counter, the
// fences and the round trip of the prefix sums through FinScratch go, and
// the group values stay in registers.
__device__ __forceinline__ void finalize_warp_body(const StepArgs& a, const FinOut& o,
                                                   const int lane) {
  constexpr int G = kFinThreads / 32;  // 32-plane groups
  const Params& p = *a.prm;
  DevState* st = a.st;
  if (st->flags) return;
  const int nx = a.nx, nu = a.part.nu;
  // ---- phase A
  double nk[G], lk[G];
#pragma unroll
  for (int g = 0; g < G; g++) {
    const int k = 32 * g + lane;
    nk[g] = 0.0;
    lk[g] = 0.0;
    if (k < nx) {
      const double* pn = a.part.n + (size_t)k * nu;
      const double* pl = a.part.lv + (size_t)k * nu;
      double sn = 0.0, sl = 0.0;
      int u = 0;
      for (; u + 8 <= nu; u += 8) {
        double xn[8], xl[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
          xn[q] = pn[u + q];
          xl[q] = pl[u + q];
        }
#pragma unroll
        for (int q = 0; q < 8; q++) {
          sn += xn[q];
          sl += xl[q];
        }
      }
      for (; u < nu; u++) {
        sn += pn[u];
        sl += pl[u];
      }
      nk[g] = sn * p.dvv;
      lk[g] = sl;
      o.ne[k] = nk[g];
    }
  }
  double pre[G];
  double woff = 0.0, btot = 0.0, blv = 0.0;
#pragma unroll
  for (int g = 0; g < G; g++) {
    // a group past the last plane: its sums are +0 (lane g keeps 0.0) and
    // its scan feeds no plane
    if (32 * g >= nx) break;
    double incl = nk[g];
    for (int d = 1; d < 32; d <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    double excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 0.0;
    pre[g] = woff + excl;
    woff += __shfl_sync(0xffffffffu, incl, 31);
    double vn = nk[g], vl = lk[g];
    for (int d = 16; d > 0; d >>= 1) {
      vn += __shfl_down_sync(0xffffffffu, vn, d);
      vl += __shfl_down_sync(0xffffffffu, vl, d);
    }
    vn = __shfl_sync(0xffffffffu, vn, 0);
    vl = __shfl_sync(0xffffffffu, vl, 0);
    if (lane == g) {
      btot = vn;
      blv = vl;
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    btot += __shfl_down_sync(0xffffffffu, btot, d);
    blv += __shfl_down_sync(0xffffffffu, blv, d);
  }
  // ---- phase B: finalize_body's last-block work with one block total
  // (valid in lane 0), the other lanes' entries zero
  const double b0 = lane == 0 ? btot : 0.0;
  double l = (lane == 0 ? blv : 0.0) + 0.0;
  double i0s = b0;
  for (int d = 1; d < 32; d <<= 1) {
    const double y0 = __shfl_up_sync(0xffffffffu, i0s, d);
    if (lane >= d) i0s += y0;
  }
  const double half = __shfl_sync(0xffffffffu, i0s, 31);
  const double boff0 = __shfl_sync(0xffffffffu, i0s - b0, 0);
  const double ntot_raw = half + 0.0;  // the empty second half of the scan
  double pe = 0.0, see = 0.0, vac = 0.0;
  for (int u = lane; u < nu; u += 32) {
    pe += a.part.pe[u];
    see += a.part.see[u];
    vac += a.part.vac[u];
  }
  for (int d = 16; d > 0; d >>= 1) {
    l += __shfl_down_sync(0xffffffffu, l, d);
    pe += __shfl_down_sync(0xffffffffu, pe, d);
    see += __shfl_down_sync(0xffffffffu, see, d);
    vac += __shfl_down_sync(0xffffffffu, vac, d);
  }
  DevState d = *st;
  if (lane == 0) {
    const double ntot = ntot_raw * p.dx;
    pe *= p.dvv;
    see = p.see_enabled ? see * p.dvv * (1.0 - p.refl) : 0.0;
    vac *= p.dvv;
    const double lv = l * p.lv_scale;
    d.cum_emit += p.dt * (d.g_see + p.refl * d.g_pe);
    d.cum_see += p.dt * d.g_see;
    d.cum_pe += p.dt * d.g_pe;
    d.cum_vac += p.dt * d.g_vac;
    d.cum_lv += p.dt * lv;
    d.cum_inj += p.dt * p.inj;
    d.sigma += kQe * p.dt * (d.g_see - (1.0 - p.refl) * d.g_pe);
    d.step += 1;
    d.g_pe = pe;
    d.g_see = see;
    d.g_vac = vac;
    d.n_tot = ntot;
    if (!isfinite(pe) || !isfinite(see) || !isfinite(vac) || !isfinite(ntot) ||
        !isfinite(d.sigma))
      d.flags |= kFlagNumeric;
    *st = d;
  }
  const double e_wall = __shfl_sync(0xffffffffu, d.sigma, 0) * p.ex_sigma;
  double cmax = 0.0, ex0 = 0.0;
#pragma unroll
  for (int g = 0; g < G; g++) {
    const int kk = 32 * g + lane;
    if (kk >= nx) continue;
    const double below = boff0 + pre[g];
    const double n_k = nk[g];
    const double e = p.self_consistent ? e_wall - p.ex_n * (below + 0.5 * n_k) : p.Ex_ext;
    if (g == 0) ex0 = e;
    o.Ex[kk] = e;
    const double c = p.c1_per_ex * e;
    o.c1[kk] = c;
    o.c1_32[kk] = (float)c;
    double cfl = fabs(c);
    if (p.collisions) {
      const double ak = n_k > 0.0 ? p.bgk_c * n_k : 0.0;
      a.bgk[kk] = ak;
      a.bgk[nx + kk] = ak * n_k;
      a.bgk32[kk] = (float)ak;
      a.bgk32[nx + kk] = (float)(ak * n_k);
      cfl += ak;
    }
    cmax = fmax(cmax, cfl);
  }
  for (int q = 16; q > 0; q >>= 1) cmax = fmax(cmax, __shfl_down_sync(0xffffffffu, cmax, q));
  if (lane == 0) {
    if (cmax + p.cx_max + fabs(p.c2) > 1.0 + 1e-12) d.flags |= kFlagCfl;
    const long long row = d.step;
    const long long cap = p.hist_cap;
    double rr[FK_HISTORY_COLS] = {(double)row, (double)row * p.dt, d.sigma, d.g_pe,
                                  d.g_see, d.g_vac, d.n_tot, ex0};
    double* r = o.hist + (size_t)(row % cap) * FK_HISTORY_COLS;
    for (int q = 0; q < FK_HISTORY_COLS; q++) r[q] = rr[q];
    if (row + 1 > d.hist_count) d.hist_count = row + 1;
    if (d.sat_step < 0 && row >= p.sat_window && p.sat_window < cap) {
      const double* h = o.hist + (size_t)((row - p.sat_window) % cap) * FK_HISTORY_COLS;
      bool ok = true;
      for (int q = 2; q <= 4; q++)
        if (!(fabs(rr[q] - h[q]) <= p.sat_tol * fabs(rr[q]))) ok = false;
      if (ok) d.sat_step = row;
    }
    st->flags = d.flags;
    st->hist_count = d.hist_count;
    st->sat_step = d.sat_step;
  }
}

// Many grids in one launch (step mode).  Blocks below n_multi run
// finalize_body: block b is block blocks[b].y of grid blocks[b].x, and each
// grid elects its own last block with its own counter.  The grids of one
// finalize block (entries blocks[n_multi ..], y = -1) go four to a block,
// one warp each.
__global__ void __launch_bounds__(kFinThreads)
finalize_batch_kernel(const BatchInst* __restrict__ inst, const int2* __restrict__ blocks,
                      int n_multi, int n_entries) {
  constexpr int G = kFinThreads / 32;
  __shared__ BatchInst bi[G];
  if ((int)blockIdx.x < n_multi) {
    const int2 m = blocks[blockIdx.x];
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(inst + m.x);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&bi[0]);
    for (int w = threadIdx.x; w < (int)(sizeof(BatchInst) / 8); w += blockDim.x) dst[w] = src[w];
    __syncthreads();
    finalize_body(bi[0].a, bi[0].o, m.y, (bi[0].a.nx + kFinThreads - 1) / kFinThreads, kModeStep);
    return;
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = n_multi + ((int)blockIdx.x - n_multi) * G + w;
  if (q >= n_entries) return;
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(inst + blocks[q].x);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(&bi[w]);
  for (int i = lane; i < (int)(sizeof(BatchInst) / 8); i += 32) dst[i] = src[i];
  __syncwarp();
  finalize_warp_body(bi[w].a, bi[w].o, lane);
}

// Strang step, after the velocity pass (one warp): fold the wall and vacuum
// partial sums of the velocity pass's output as the finalize kernel folds
// those of a new state, add dt/2 of the resulting fluxes to the ledger and
// the surface charge (Eqs. 12-14, 18), and hand Gamma_see of that state and
// the sticky flags to the second x half-pass through *mid.
__global__ void strang_mid_kernel(const __grid_constant__ StepArgs a, DevState* mid) {
  const Params& p = *a.prm;
  DevState* st = a.st;
  const int lane = threadIdx.x;
  const unsigned flags = st->flags;
  double pe = 0.0, see = 0.0, vac = 0.0;
  for (int u = lane; u < a.part.nu; u += 32) {
    pe += a.part.pe[u];
    see += a.part.see[u];
    vac += a.part.vac[u];
  }
  for (int o = 16; o > 0; o >>= 1) {
    pe += __shfl_down_sync(0xffffffffu, pe, o);
    see += __shfl_down_sync(0xffffffffu, see, o);
    vac += __shfl_down_sync(0xffffffffu, vac, o);
  }
  if (lane != 0) return;
  mid->flags = flags;
  if (flags) return;  // frozen state: the passes do nothing either
  pe *= p.dvv;
  see = p.see_enabled ? see * p.dvv * (1.0 - p.refl) : 0.0;
  vac *= p.dvv;
  mid->g_see = see;
  const double h = 0.5 * p.dt;
  st->cum_emit += h * (see + p.refl * pe);
  st->cum_see += h * see;
  st->cum_pe += h * pe;
  st->cum_vac += h * vac;
  st->sigma += kQe * h * (see - (1.0 - p.refl) * pe);
}

cudaError_t launch_strang_mid(const StepArgs& a, DevState* mid, cudaStream_t s) {
  strang_mid_kernel<<<1, 32, 0, s>>>(a, mid);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const StepArgs& a, double* ne, double* Ex, double* c1,
                            float* c1_32, double* hist, const FinScratch& fs, int mode,
                            cudaStream_t s) {
  const int nb = (a.nx + kFinThreads - 1) / kFinThreads;
  const FinOut o{ne, Ex, c1, c1_32, hist, fs};
  finalize_kernel<<<nb, kFinThreads, 0, s>>>(a, o, mode);
  return cudaGetLastError();
}

int finalize_batch_ctas(int n_multi, int n_entries) {
  return n_multi + (n_entries - n_multi + kFinThreads / 32 - 1) / (kFinThreads / 32);
}

cudaError_t launch_finalize_batch(const BatchInst* inst, const int2* blocks, int n_multi,
                                  int n_entries, cudaStream_t s) {
  const int n_ctas = finalize_batch_ctas(n_multi, n_entries);
  if (n_ctas <= 0) return cudaSuccess;
  finalize_batch_kernel<<<n_ctas, kFinThreads, 0, s>>>(inst, blocks, n_multi, n_entries);
  return cudaGetLastError();
}

int finalize_blocks(int nx) { return (nx + kFinThreads - 1) / kFinThreads; }

// ---------------------------------------------------------------------------
// FP64 rows <-> FP32 rows with a row pitch (host arrays are dense FP64).
__global__ void convert_kernel(const void* src, void* dst, size_t rows, int nv2, int pitch,
                               int to_f32) {
  const size_t n = rows * (size_t)nv2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t r = e / nv2, j = e - (e / nv2) * nv2;
    if (to_f32)
      static_cast<float*>(dst)[r * pitch + j] = (float)static_cast<const double*>(src)[e];
    else
      static_cast<double*>(dst)[e] = (double)static_cast<const float*>(src)[r * pitch + j];
  }
}

cudaError_t launch_convert(const void* src, void* dst, size_t rows, int nv2, int pitch,
                           int to_f32, cudaStream_t s) {
  const size_t n = rows * (size_t)nv2;
  size_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  convert_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, dst, rows, nv2, pitch, to_f32);
  return cudaGetLastError();
}

}  // namespace fk
