/*
 * fk.h -- C ABI of the GB300 library that advances the electron velocity
 * distribution f(x, v1, v2) of the 1D2V continuum-kinetic model of vacuum
 * surface flashover (Sun et al., arXiv 2303.14119).
 *
 * Model (Sec. 2): x is the coordinate normal to the insulator, x = 0 the
 * dielectric surface and x = h_max the vacuum side; v1 = v_x is the normal
 * velocity and v2 = v_y the tangential velocity along the applied field E_y.
 * One time step is an explicit, first-order upwind, finite-volume update of
 * Eq. 2 (advection in x, v1 and v2 plus the field-emission source of Eq. 7),
 * with the secondary-electron wall boundary of Eqs. 12-16, the absorbing
 * vacuum boundary of Eq. 17, the surface-charge update of Eq. 18 and the
 * normal field E_x from the 1D Poisson problem stated after Eq. 2.
 *
 * Conventions shared by every call:
 *  - Grids are uniform and cell-centred: x_k = (k + 1/2) dx, v1_i = v1_min +
 *    (i + 1/2) dv1, v2_j likewise.  Host arrays of f are FP64, C order
 *    [k][i][j] (v2 fastest), nx * nv1 * nv2 elements.
 *  - SI units throughout, except energies and temperatures in eV.
 *  - Every call returns an fk_status.  Nothing aborts and no C++ exception
 *    crosses the boundary.  After a failure, fk_last_error() describes it.
 *  - The library owns all device memory of a grid; it allocates it in
 *    fk_create_grid and frees it in fk_destroy_grid.  Host buffers passed in
 *    are owned by the caller and are only read or written during the call
 *    (copies complete before the call returns).
 *  - Work is ordered on the grid's CUDA stream.  fk_step only enqueues;
 *    the getters synchronise that stream.  Errors detected on the device
 *    (CFL violation, non-finite sums, a pipeline wait that ran out, negative
 *    f) are sticky: the step that meets one leaves f at the last valid
 *    state, later steps do nothing, and the next getter or fk_sync returns
 *    the status.  Where f is checked for negative values: every cell of a
 *    state set with fk_set_f / fk_set_f32 (the call returns FK_ENEGATIVE),
 *    every cell a direct-load pass writes, and the wall and vacuum planes of
 *    every streaming step or split-scheme pass on the streaming kernel.  The
 *    interior of a streaming pass is not checked per cell: with f >= 0 and
 *    the Courant sum (checked every step) at most 1, its update is a sum of
 *    non-negative terms.
 *  - Range of f.  FP64 grids: the streaming step sums f^{n+1} for n_e through
 *    an exact split of each value into two FP32 parts, which covers
 *    2^-126 <= |f| < 2^128 (about 1.2e-38 to 3.4e38); smaller magnitudes
 *    count as 0 in n_e, and larger ones, infinities and NaN make the sum
 *    non-finite, so the step reports FK_ENUMERIC.  FP32 grids store f in
 *    FP32; their half-CTA units sum the wall fluxes v1 f in FP32 pairs, so
 *    |f| max|v1| must stay below 3.4e38 (above it the flux is non-finite and
 *    the step reports FK_ENUMERIC).
 *  - Failure-detection test knobs (off by default, read at fk_create_grid):
 *    FK_TEST_WAIT_CYCLES=<n> sets the limit of the streaming kernel's bounded
 *    waits to n cycles (default about 2 s); FK_TEST_WITHHOLD_COPY=<q> makes
 *    the work unit of tile 0, chunk 0 skip the plane copy of its pipeline
 *    item q, so that the waits on it run out and the step reports
 *    FK_ETIMEOUT (every copy that was issued still lands before the kernel
 *    leaves).  FK_TEST_FAIL_ALLOC=<n> (read at each allocation) makes the
 *    n-th device or pinned allocation since the start of the last
 *    fk_create_grid or fk_batch_create fail, so that the call returns
 *    FK_ENOMEM after freeing what it allocated.
 *  - Builds: the release library, and a debug-bounds build (compiled with
 *    FK_DEBUG_BOUNDS) whose streaming step kernel checks every index before
 *    the access and reports a failed check as FK_EBOUNDS instead.
 *  - Calls on one grid must not run concurrently from several threads.
 *    Distinct grids are independent.
 */
#ifndef FK_H
#define FK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fk_grid fk_grid; /* opaque, library-owned */
typedef struct fk_batch fk_batch; /* opaque, library-owned; see fk_batch_create */

typedef enum {
  FK_OK = 0,
  FK_EINVAL = 1,   /* an argument is out of range or NULL */
  FK_ENOMEM = 2,   /* device or host allocation failed */
  FK_ECUDA = 3,    /* a CUDA runtime call failed (message in fk_last_error) */
  FK_ECFL = 4,     /* |c_x| + |c_1| + |c_2| > 1 somewhere: the explicit
                      upwind step would not keep f >= 0 */
  FK_ENUMERIC = 5, /* a moment or flux became NaN or infinite */
  FK_ETIMEOUT = 6, /* a bounded wait inside a kernel ran out */
  FK_ESTATE = 7,   /* call not valid in the grid's current state */
  FK_ENEGATIVE = 8, /* f has a negative value: a state set with one, or a
                      step that produced one beyond rounding */
  FK_EBOUNDS = 9   /* debug-bounds build (FK_DEBUG_BOUNDS) only: an index of
                      the streaming step kernel fell outside its buffer; the
                      access was skipped */
} fk_status;

typedef enum {
  FK_F64 = 0, /* f stored and advected in FP64 */
  FK_F32 = 1  /* f stored and advected in FP32; moments, fluxes, surface
                 charge, field and ledger stay FP64 */
} fk_precision;

/* Grid description.
 * 2 <= nx <= 8192 and 2 <= nv1, nv2 <= 65536 cells; h_max > 0 (m); v1_min < v1_max, v2_min < v2_max
 * (m/s); dt > 0 (s), or dt <= 0 to take dt = cfl * dx / max(|v1_min|,
 * |v1_max|) with cfl > 0; history_capacity = rows kept in the device history
 * ring (0 selects 65536).  Sec. 2, paragraph on default parameters: the
 * paper sets the grid and the time step by the CFL conditions. */
typedef struct {
  int32_t nx, nv1, nv2;
  int32_t precision; /* fk_precision */
  double h_max;
  double v1_min, v1_max, v2_min, v2_max;
  double dt;
  double cfl;
  int64_t history_capacity;
  int32_t device; /* CUDA device ordinal */
  int32_t reserved;
} fk_grid_desc;

/* Create a grid with f = 0 and sigma = 0 everywhere (Sec. 2: the simulation
 * starts with no space or surface charge), no applied field, E_x
 * self-consistent, secondary emission and source switched off.
 * cuda_stream: a cudaStream_t to order the grid's work on, or NULL for a
 * stream the grid creates and owns.  On success *out receives the grid.
 * Returns FK_EINVAL for a bad description, FK_ECFL if the x-Courant number
 * max|v1| dt/dx exceeds 1, FK_ENOMEM / FK_ECUDA on device failures. */
fk_status fk_create_grid(const fk_grid_desc *desc, void *cuda_stream, fk_grid **out);

/* Release the grid and all its device memory.  NULL is accepted. */
fk_status fk_destroy_grid(fk_grid *grid);

/* Fields of Sec. 2 (text after Eq. 2).  Ey (V/m) is the applied tangential
 * field, constant and <= 0 (cathode on the left).  self_consistent != 0:
 * E_x(x) from the 1D Poisson problem with E_x = sigma/(2 eps0) at the
 * dielectric and V = 0 at the vacuum side, i.e. Gauss's law integrated from
 * the wall over the electron space charge -e n_e; otherwise E_x = Ex_external
 * everywhere.  Acceleration of electrons: a = -e E / m_e. */
fk_status fk_set_fields(fk_grid *grid, double Ey, int self_consistent, double Ex_external);

/* Secondary electron emission, Sec. 2, Eqs. 8-16.  The yield matrix
 * delta(i, j) of Eqs. 8-11 (delta_max, A_max in eV, smoothness k_s >= 0) is
 * built once over the grid cells with v1 < 0.  Each step the primary flux
 * dGamma_pe = -v1 f(x=0) dv1 dv2 (Eq. 13) and Gamma_see = sum delta dGamma_pe
 * (Eqs. 12, 14) are re-emitted at x = 0 into v1 > 0 as the half-Maxwellian
 * of Eq. 15 at temperature T_se (eV), normalised on the grid so that the
 * emitted flux equals Gamma_see.  enabled = 0 switches re-emission off
 * (delta treated as 0; every primary is then deposited on the surface). */
fk_status fk_set_see(fk_grid *grid, double delta_max, double A_max_eV, double k_s,
                     double T_se_eV, int enabled);

/* Field-emission source of Eq. 7: J (A/m^2, >= 0, 0 switches it off)
 * injected uniformly on the cells whose centres lie in [x_lo, x_hi] (m),
 * with a velocity shape that is Maxwellian in v1 and half-Maxwellian on
 * v2 > 0 at temperature T_fe (eV), normalised on the grid so that exactly
 * J/e electrons per m^2 per s are injected.  FK_EINVAL if J > 0 and no cell
 * centre lies in the band. */
fk_status fk_set_source(fk_grid *grid, double J, double x_lo, double x_hi, double T_fe_eV);

/* Fowler-Nordheim field emission, Eq. 6: the current density J (A/m^2) at
 * the emitter field E (V/m, > 0) for a work function e phi (phi in V, > 0),
 * without field enhancement or image-charge correction.  *log_J receives
 * ln J (finite even where J underflows), *J = exp(ln J) (0 on underflow);
 * either may be NULL.  Host-side, needs no grid.  At the paper's E = |E_y|
 * of a few MV/m the exponent is about -1e4, so J is exactly 0 in FP64. */
fk_status fk_fowler_nordheim(double E, double phi_V, double *log_J, double *J);

/* fk_set_source with J from Eq. 6 at the field E_ctj (V/m) and work function
 * phi (V): the source of Eq. 7 fed by field emission at the cathode triple
 * junction.  A J that underflows switches the source off. */
fk_status fk_set_source_fn(fk_grid *grid, double E_ctj, double phi_V, double x_lo, double x_hi,
                           double T_fe_eV);

/* Electron-electron Coulomb collisions, Eqs. 3-5: the BGK term
 * nu_ee(x) (n_e(x) f_e0 - f) with nu_ee from Eq. 4 at the electron
 * temperature T_e (eV, > 0; the paper's default is 2 eV) and Coulomb
 * logarithm ln_lambda (>= 0; the paper's value is 10), n_e(x) the density of
 * the state being stepped, and f_e0 the equilibrium of Eq. 5 (Maxwellian at
 * T_e, no drift) normalised on the grid so that the term moves no density.
 * It enters the same forward-Euler step as the advection; dt nu_ee counts
 * toward the Courant bound (FK_ECFL).  enabled = 0 (the default) switches
 * it off. */
fk_status fk_set_collisions(fk_grid *grid, double T_e_eV, double ln_lambda, int enabled);

/* Electron reflection at the dielectric (Sec. 2, text after Eq. 17): a
 * fraction R_f (0..1) of each incident primary flux element dGamma_pe(i, j)
 * returns specularly at (-v1_i, v2_j); only the rest, (1 - R_f), is absorbed
 * and emits secondaries with yield delta(i, j) (Eqs. 12-14), so Gamma_see
 * and the charging of Eq. 18 scale with (1 - R_f), and the ledger's emitted
 * term counts secondaries plus reflected electrons.  R_f > 0 needs a v1 grid
 * symmetric about 0 (each cell's mirror is a cell); FK_EINVAL otherwise.
 * Default 0. */
fk_status fk_set_reflection(fk_grid *grid, double R_f);

/* Time scheme of fk_step.  FK_SCHEME_UNSPLIT (the default): one forward-
 * Euler step with every flux from f^n, fused into one pass over f.
 * FK_SCHEME_LIE: Lie splitting -- x-advection of f^n (with the wall and
 * vacuum boundaries) over dt, then the velocity step (v1, v2 advection,
 * source, collisions) of that intermediate state over dt, both with the
 * fields of f^n; the surface charge and the wall ledger terms come from f^n
 * as in the unsplit step.  FK_SCHEME_STRANG: Strang splitting --
 * x-advection over dt/2, the velocity step over dt with the fields of f^n,
 * x-advection over dt/2; each x half-step takes its wall fluxes (Eqs. 12-15)
 * from its own input state, so the surface charge and the wall ledger terms
 * take dt/2 of the fluxes of f^n and dt/2 of those of the state after the
 * velocity step.  Sec. 2 states only an explicit upwind update; the split
 * forms run as two (Lie) or three (Strang) passes over f through one more
 * buffer of f: each pass is the streaming step kernel with the other terms'
 * coefficients zeroed (the direct-load kernel on grids too wide for it),
 * and grids using them cannot join a batch.  FK_EINVAL for another value;
 * FK_ESTATE while the grid is in a batch. */
#define FK_SCHEME_UNSPLIT 0
#define FK_SCHEME_LIE 1
#define FK_SCHEME_STRANG 2
fk_status fk_set_scheme(fk_grid *grid, int scheme);

/* Convergence test of Sec. 2 (paragraph after Eq. 18): the run is saturated
 * at the first step n >= window with |q_n - q_{n-window}| <= rel_tol |q_n|
 * for q = sigma, Gamma_pe and Gamma_see.  Defaults: window 10000, rel_tol
 * 1e-3.  FK_EINVAL unless 1 <= window < history_capacity and rel_tol >= 0. */
fk_status fk_set_convergence(fk_grid *grid, int64_t window, double rel_tol);

/* Advance n >= 0 time steps (forward Euler, all fluxes from f^n; Eq. 18
 * updates sigma for the next step's E_x).  Stream-ordered and asynchronous:
 * it returns once the work is enqueued.  Returns a sticky device error seen
 * by an earlier synchronising call (FK_ECFL, FK_ENUMERIC, FK_ETIMEOUT). */
fk_status fk_step(fk_grid *grid, int64_t n);

/* Wait for the grid's stream and report any sticky device error. */
fk_status fk_sync(fk_grid *grid);

/* Moments of the current state (synchronises).  n_e[nx] (m^-3) and Ex[nx]
 * (V/m) at cell centres; *gamma_pe and *gamma_see (m^-2 s^-1) of Eqs. 13-14
 * evaluated on the x = 0 plane.  Any pointer may be NULL. */
fk_status fk_moments(fk_grid *grid, double *n_e, double *Ex, double *gamma_pe,
                     double *gamma_see);

/* Surface charge density sigma_e (C/m^2) of the current state, Eq. 18. */
fk_status fk_surface_charge(fk_grid *grid, double *sigma);

/* Per-step history (Fig. 3 quantities), one row of FK_HISTORY_COLS doubles
 * per state: step, time (s), sigma (C/m^2), Gamma_pe, Gamma_see, Gamma_vac
 * (m^-2 s^-1), areal electron count N = sum n_e dx (m^-2), E_x at the first
 * cell centre (V/m).  Copies the most recent min(max_rows, stored) rows,
 * oldest first, into out[rows][FK_HISTORY_COLS]; *rows receives the count. */
#define FK_HISTORY_COLS 8
fk_status fk_history(fk_grid *grid, double *out, int64_t max_rows, int64_t *rows);

/* Conservation ledger since the last reset (fk_set_f, fk_set_surface_charge
 * or creation), FK_LEDGER_LEN doubles: N, N0, emitted, primary (wall),
 * vacuum, velocity-edge loss, injected, sigma0, secondary -- the six
 * cumulative terms are time integrals (m^-2) of the fluxes of each step's
 * starting state, so that N - N0 = emitted - primary - vacuum - loss +
 * injected and (sigma - sigma0)/e = secondary - primary up to rounding. */
#define FK_LEDGER_LEN 9
fk_status fk_ledger(fk_grid *grid, double *out);

/* Step index of the current state and the first saturated step (-1 if the
 * convergence test has not passed). */
fk_status fk_step_count(fk_grid *grid, int64_t *step, int64_t *saturated_step);

/* Copy f of the current state to host FP64 [nx][nv1][nv2] (synchronises). */
fk_status fk_get_f(fk_grid *grid, double *host_f);

/* Replace f (host FP64 [nx][nv1][nv2], values finite) and restart the run at
 * step 0: history cleared, ledger baseline taken from the new state.  An FP32
 * grid rounds each value to nearest. */
fk_status fk_set_f(fk_grid *grid, const double *host_f);

/* FP32 grids only (FK_EINVAL otherwise): fk_get_f and fk_set_f with host
 * arrays in the grid's own storage type, float [nx][nv1][nv2]: one strided
 * copy each way, no conversion and half the bytes of the FP64 forms. */
fk_status fk_get_f32(fk_grid *grid, float *host_f);
fk_status fk_set_f32(fk_grid *grid, const float *host_f);

/* Replace sigma (C/m^2) and restart the run at step 0 like fk_set_f. */
fk_status fk_set_surface_charge(fk_grid *grid, double sigma);

/* Checkpoints.  fk_get_state writes the whole run into a host buffer the
 * caller owns: f in its storage precision, the surface charge, fluxes,
 * ledger, step and sticky flags, the fields and Courant numbers of the
 * current state, the history ring and every parameter set on the grid.
 * Call it with buf = NULL to get the size in *len; a smaller *len returns
 * FK_EINVAL with the size in *len.  fk_set_state restores such a buffer
 * into a grid created with the same description (shape, precision,
 * history capacity; FK_EINVAL otherwise): the restored grid then steps on
 * exactly -- bit for bit -- as the original would have.  Both synchronise. */
fk_status fk_get_state(fk_grid *grid, void *buf, size_t *len);
fk_status fk_set_state(fk_grid *grid, const void *buf, size_t len);

/* Grid facts, FK_INFO_LEN doubles: dx, dv1, dv2, dt (s), c2 (signed
 * v2-Courant number a2 dt/dv2), max |c_x|, step kernel (1 streaming,
 * 0 direct-load), v1-row tiles per plane, x-chunks, planes per chunk,
 * work units per CTA of the streaming kernel (2 where each sign half of the
 * v1 rows fits the tile of a half-CTA unit, else 1; the environment
 * variable FK_STREAM_HALF=0 at grid creation keeps 1), v1 rows of the
 * largest tile, the tile-row cap of fk_set_tile_rows (0: none).
 * Host-side, no synchronisation. */
#define FK_INFO_LEN 13
fk_status fk_grid_info(const fk_grid *grid, double *out);

/* Work decomposition of the streaming step kernel's whole-CTA units: cap
 * the v1 rows of a tile at max_rows (>= 1), or 0 for the default plan (the
 * most rows for which two CTAs fit on an SM).  Grids whose sign halves run
 * as half-CTA units keep their tiles.  Waits for the grid's pending work,
 * keeps its state and re-plans its tiles (and x-chunks); the next fk_step
 * recaptures its graphs.  The per-cell update does not depend on the
 * tiles, but n_e(x) (Eq. 14) is summed per (plane, tile) before the planes'
 * FP64 fold, so the tile plan sets the rounding of n_e, E_x and everything
 * after them: two grids step bit for bit alike only with the same plan.
 * FK_EINVAL for max_rows < 0, FK_ESTATE while a batch steps the grid. */
fk_status fk_set_tile_rows(fk_grid *grid, int32_t max_rows);

/* Kernel timing (tracing).  enabled != 0: later fk_step calls launch each
 * step directly (no graph replay) and record a CUDA event pair around every
 * launch of the fused step kernel on the grid's stream; enabled = 0 returns
 * to graph replay.  Switching discards pending records. */
fk_status fk_set_kernel_timing(fk_grid *grid, int enabled);

/* Synchronise and report the step-kernel launches recorded since the last
 * call (at most 8192 are kept; later ones are counted but not timed):
 * *launches = launches timed, *total_ms = sum of their durations (ms).
 * The records are consumed. */
fk_status fk_kernel_timing(fk_grid *grid, int64_t *launches, double *total_ms);

/* Density moment without allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc themselves or
 * let a library do it -- code that runs while a stream is being captured
 * into a CUDA graph (allocation is not allowed there), applications whose
 * device memory is owned by their own pool allocator, and loops that cannot
 * afford the device-wide synchronisation an allocation may cause.
 *
 * Computes n_e[k] = dv1 dv2 * sum_{i,j} f[k][i][j] for k < nx from a
 * distribution the caller already holds in device memory (f_dev: FP64,
 * dense [nx][nv1][nv2]) into the caller's device array n_e_dev[nx], both on
 * cuda_stream (NULL = the legacy default stream).  Stream-ordered and
 * asynchronous; it allocates nothing.  Its scratch is one fixed array of
 * FK_NOALLOC_MAX_PARTIALS doubles (1 MiB) in the library's device memory,
 * held by every GPU that loads the library until the process exits, so
 * nx <= FK_NOALLOC_MAX_PARTIALS / 16 = 8192; larger nx returns FK_EINVAL
 * with the limit in fk_last_error(NULL).  Every call shares that array and
 * overwrites the slots it uses before reading them, so nothing needs
 * clearing; calls that overlap on the GPU (different streams or devices
 * sharing one context) race on it and must be ordered by the caller.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.
 * The address is kept for the life of the process: after a reset of the
 * device's primary context (cudaDeviceReset) the entry point must not be
 * called again in that process.
 * Errors: FK_EINVAL (NULL pointer, non-positive size or spacing, nx above
 * the limit), FK_ECUDA (no current device, lookup or launch failure). */
#define FK_NOALLOC_MAX_PARTIALS 131072
fk_status fk_density_moment_noalloc(const double *f_dev, int32_t nx, int32_t nv1, int32_t nv2,
                                    double dv1, double dv2, double *n_e_dev, void *cuda_stream);

/* ---- Batched stepping of many grids (parameter sweeps) --------------------
 * The paper's design studies (Sec. 3: scans over E_y, delta_max, A_max and
 * T_se, each point a separate run) are many small independent runs.  A batch
 * steps a set of existing grids together: every batch step is one launch of
 * the streaming step kernel over the work units (v1-row tile x x-chunk) of
 * all grids, largest units first (a second launch runs the units of grids
 * whose thin tiles go two to a CTA), followed by ONE launch of the finalize
 * kernel over all grids' planes, replayed 32 steps per CUDA graph.  Each
 * grid's arithmetic is exactly that of fk_step on the same grid: the x-chunk
 * split (the only thing the batch chooses) changes which CTA updates a cell,
 * not how, so a batch step and fk_step give bitwise identical states.
 *
 * Ownership and state rules:
 *  - The batch borrows the grids; the caller keeps ownership.  While a grid
 *    belongs to a batch, every call that changes it (fk_step, the setters,
 *    fk_set_f, fk_set_f32, fk_set_surface_charge, fk_set_collisions, fk_set_reflection,
 *    fk_set_scheme, fk_set_state, fk_set_kernel_timing and
 *    fk_destroy_grid) returns FK_ESTATE; the getters work and see every
 *    batch step enqueued before them.  fk_batch_destroy releases the grids.
 *  - A grid that meets a sticky device error (FK_ECFL, FK_ENUMERIC,
 *    FK_ETIMEOUT) freezes at its last valid state; the other grids go on.
 *    fk_batch_sync reports each grid's status.
 *  - Work is ordered on the batch's stream. */

/* Create a batch of n >= 1 distinct grids, none already in a batch, all on
 * one device, all of one precision, all using the streaming step kernel
 * (fk_grid_info's kernel entry is 1).  Waits for each grid's pending work.
 * cuda_stream: stream for the batch's work, or NULL for one it owns.
 * Errors: FK_EINVAL (NULL, n < 1, duplicates, mixed device or precision, a
 * grid on the direct-load kernel), FK_ESTATE (a grid already in a batch),
 * FK_ENOMEM / FK_ECUDA. */
fk_status fk_batch_create(fk_grid *const *grids, int32_t n, void *cuda_stream, fk_batch **out);

/* Wait for the batch's work, release its grids (each re-synchronised so it
 * can be stepped alone again) and free the batch.  NULL is accepted. */
fk_status fk_batch_destroy(fk_batch *batch);

/* Advance every grid of the batch by n >= 0 steps (stream-ordered,
 * asynchronous; frozen grids stay frozen).  Returns FK_OK unless the work
 * could not be enqueued. */
fk_status fk_batch_step(fk_batch *batch, int64_t n);

/* Wait for the batch's stream and read each grid's sticky status into
 * status[i] (may be NULL).  Returns FK_OK if every grid is OK, else the
 * status of the first grid that is not (its message in fk_batch_last_error). */
fk_status fk_batch_sync(fk_batch *batch, int32_t *status);

/* Per-grid scalars of the current states after the batch's enqueued work
 * (one synchronisation for all grids): sigma[i] (C/m^2), step[i], the first
 * saturated step sat_step[i] (-1 if none) and the sticky status[i]; any
 * array may be NULL.  Frozen grids report their last valid state. */
fk_status fk_batch_scalars(fk_batch *batch, double *sigma, int64_t *step, int64_t *sat_step,
                           int32_t *status);

/* Moments of every grid's current state after the batch's enqueued work,
 * read with one synchronisation for all grids (the batch form of
 * fk_moments and fk_surface_charge): sigma[i] (C/m^2, Eq. 18),
 * gamma_pe[i] and gamma_see[i] (m^-2 s^-1, Eqs. 13-14), and n_e and E_x at
 * the cell centres of every grid in batch order, grid i's nx_i values
 * starting at offset nx_0 + ... + nx_{i-1} of n_e and Ex.  Any pointer may
 * be NULL.  Frozen grids report their last valid state. */
fk_status fk_batch_moments(fk_batch *batch, double *sigma, double *gamma_pe, double *gamma_see,
                           double *n_e, double *Ex);

/* Pipelined form of fk_batch_moments, so that a loop can read the moments
 * of step n while step n + 1 runs.  fk_batch_moments_enqueue queues, after
 * the work enqueued on the batch's stream so far, one small kernel that
 * packs every grid's sigma, Gamma_pe, Gamma_see, n_e and E_x into one of two
 * device slots and one copy of that slot into its pinned host twin (slot 0
 * or 1), both on a copy stream the batch owns (buffers, events and the copy
 * stream are allocated on first use), and returns at once.  The next batch
 * step's step kernel runs beside them; its finalize, the first kernel to
 * overwrite what the packing kernel reads, waits for that kernel (not for
 * the copy).  fk_batch_moments_collect waits for that slot's copy only (not
 * for later work) and unpacks it as fk_batch_moments does.  A slot holds one
 * set: enqueue on a full slot, or collect from an empty one, returns
 * FK_ESTATE.  The values are those of the state after the work enqueued
 * before the call; sticky device errors are reported by fk_batch_sync. */
fk_status fk_batch_moments_enqueue(fk_batch *batch, int32_t slot);
fk_status fk_batch_moments_collect(fk_batch *batch, int32_t slot, double *sigma,
                                   double *gamma_pe, double *gamma_see, double *n_e, double *Ex);

/* Autotuner: picks the x-chunk length (planes per work unit) of every size
 * bucket of the batch -- grids grouped by plane size and nx, each a power of
 * two -- by timing real steps: one trial of steps_per_trial >= 1 batch steps
 * per candidate length (powers of two from 4 planes up to the whole x range,
 * and the lengths that give the bucket about 1 to 12 whole waves of the
 * GPU's unit slots), bucket by bucket, largest bucket first, keeping the
 * fastest.  The trials advance every grid
 * (bitwise as fk_batch_step would); *steps_taken (may be NULL) receives how
 * many steps they took.  The v1-row tile of each grid is fixed by its shared-
 * memory plan: the most rows for which two CTAs fit on an SM, or, where each
 * sign half of the v1 rows fits a half-CTA unit, one such half per tile. */
fk_status fk_batch_autotune(fk_batch *batch, int32_t steps_per_trial, int64_t *steps_taken);

/* The same search, and for every bucket whose grids run whole-CTA units
 * also the v1 tile: besides each grid's current tiles, caps of about 5120
 * and 4096 cells per tile plane (rows = cells / pitch, at least 4; only
 * where they cut the grid's tiles), each timed at the chunk candidates.
 * The grids keep the tile caps found, as after fk_set_tile_rows (their
 * fk_grid_info reports them); the trials' steps advance the grids with the
 * plans tried.  Afterwards a grid in the batch steps bit for bit as the same
 * state stepped alone with the same tile cap. */
fk_status fk_batch_autotune_tiles(fk_batch *batch, int32_t steps_per_trial,
                                  int64_t *steps_taken);

/* Read (chunk_len[n]) or set the planes per x-chunk of every grid.  Set:
 * each value is clamped to [1, nx]; the next fk_batch_step uses it. */
fk_status fk_batch_get_chunks(const fk_batch *batch, int32_t *chunk_len);
fk_status fk_batch_set_chunks(fk_batch *batch, const int32_t *chunk_len);

/* Batch facts, FK_BATCH_INFO_LEN doubles: grids, work units of one batch
 * step, CTAs of the finalize launch (one per 128 planes of a grid with more
 * than 128, one per four grids of at most 128), dynamic shared memory per
 * CTA (bytes), CTAs per SM, phase-space cells of all grids, size buckets,
 * batch steps enqueued, CTAs of whole-CTA units, CTAs of half units (two to
 * a CTA).  A batch step launches the step kernel once per nonzero CTA
 * count, then the finalize kernel.  Host-side, no synchronisation. */
#define FK_BATCH_INFO_LEN 10
fk_status fk_batch_info(const fk_batch *batch, double *out);

/* Kernel timing for the batch, as fk_set_kernel_timing / fk_kernel_timing:
 * with enabled != 0 every batch step is launched directly with an event
 * pair around the batched step kernel. */
fk_status fk_batch_set_kernel_timing(fk_batch *batch, int enabled);
fk_status fk_batch_kernel_timing(fk_batch *batch, int64_t *launches, double *total_ms);

/* Text of the last error on this batch ("" if none); NULL: errors of
 * fk_batch_create on the calling thread. */
const char *fk_batch_last_error(const fk_batch *batch);

/* Text of the last error on this grid ("" if none).  grid may be NULL for
 * errors of fk_create_grid on the calling thread.  Valid until the next call
 * on the same grid. */
const char *fk_last_error(const fk_grid *grid);

#ifdef __cplusplus
}
#endif

#endif /* FK_H */
