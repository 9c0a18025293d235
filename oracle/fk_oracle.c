/*
 * fk_oracle.c -- plain FP64 CPU oracle for one explicit time step of the
 * 1D2V continuum-kinetic model of vacuum surface flashover
 * (Sun et al., arXiv 2303.14119, Sec. 2).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg load this library.  It shares
 * no code, header, table or constant with the CUDA library; both sides are
 * fed the same seeded inputs from a separate generator module.
 *
 * It is written to be read against the paper, not to be fast: every face
 * flux is evaluated on its own from its definition (each interior face is
 * evaluated twice), every sum is a serial loop, every number is a double.
 * Built with -fopenmp, the loops over x-planes run on several threads; a
 * sum over planes is then taken from per-plane partials added in plane
 * order, as the serial build does, so both builds give the same bits.
 *
 * One step n -> n+1, in the order of Sec. 2:
 *   1. fields from the current state: the density moment n_k, the normal
 *      field E_x from the 1D Poisson problem with E_x(0) = sigma/(2 eps0)
 *      (Neumann, dielectric side) and V(h_max) = 0 (Dirichlet, vacuum side),
 *      and the constant tangential field E_y;
 *   2. wall fluxes from the x = 0 plane of f^n (Eqs. 12-14);
 *   3. one forward-Euler, first-order upwind (donor-cell) update of every
 *      cell of Eq. 2 with all face fluxes taken from f^n: advection in x, v1
 *      and v2, the cathode-triple-junction source of Eq. 7; the wall inflow
 *      for v1 > 0 is the re-emitted half-Maxwellian of Eq. 15, the vacuum
 *      side absorbs (Eq. 17);
 *   4. the surface-charge update of Eq. 18 (used by the next step's E_x);
 *   5. moments of f^{n+1}, history row, conservation ledger and the
 *      convergence test stated at the end of Sec. 2.
 *
 * Readings taken where the paper is silent (cited as R1..R14 below):
 *   R1 unsplit forward Euler, all fluxes from f^n;
 *   R2 first-order donor cell upwind;
 *   R3 uniform cell-centred grids in x, v1, v2;
 *   R4 Gamma_see^n (from f^n) feeds the inflow of the same step, sigma^{n+1}
 *      feeds E_x of the next step;
 *   R5 the emission shape of Eq. 15 is renormalised on the grid so that the
 *      discrete emitted flux equals Gamma_see exactly;
 *   R6 the source of Eq. 7 acts on the cells whose centres lie in
 *      [x_lo, x_hi], with width W = (number of such cells) * dx, and its
 *      velocity shape (full Maxwellian in v1, half Maxwellian on v2 > 0)
 *      renormalised on the grid to unit density;
 *   R7 E_x at cell centres from Gauss's law integrated from the wall;
 *   R8 sign conventions: electron charge -e, acceleration a = -e E / m_e;
 *   R9 velocity-grid edges have zero inflow; what leaves through them is
 *      counted as a loss in the ledger;
 *   R10 the convergence test compares each history row with the row
 *      `window` steps earlier (relative change <= tol for sigma, Gamma_pe
 *      and Gamma_see);
 *   R11 the electron-electron BGK term of Eqs. 3-5 (off unless switched on)
 *      uses the electron temperature T_e as a fixed parameter (listed with
 *      the default parameters of Sec. 2, 2 eV) and n_e(x) of f^n, so that
 *      nu_ee(x) = n_e e^4 ln(Lambda) / (12 pi^1.5 eps0^2 sqrt(m_e) T_e^1.5);
 *      the equilibrium of Eq. 5 (no drift) is renormalised on the grid to
 *      unit density, so the term changes no plane's density; it enters the
 *      same forward-Euler step as the advection (R1), and the Courant sum
 *      includes dt nu_ee;
 *   R12 electron reflection at the dielectric (Sec. 2, after Eq. 17, off
 *      unless set): a fraction R_f of each incident flux element
 *      dGamma_pe(i, j) returns specularly at (-v1_i, v2_j) -- the mirror cell
 *      of a v1 grid symmetric about 0 -- and only the rest, (1 - R_f), is
 *      absorbed and induces SEE with yield delta(i, j); the surface charge
 *      changes by e dt (1 - R_f) sum (delta - 1) dGamma_pe;
 *   R13 Lie splitting (off unless set): the step is an x-advection of f^n
 *      (with the wall and vacuum boundaries of R4, R5, R12) followed by the
 *      velocity step (v1, v2 advection, source, collisions) of that
 *      intermediate state, both over dt and with the fields of f^n; the
 *      surface charge and the wall and vacuum ledger terms come from f^n as
 *      in the unsplit step, the velocity-edge loss from the intermediate
 *      state;
 *   R14 Strang splitting (off unless set): an x-advection over dt/2, the
 *      velocity step over dt, and a second x-advection over dt/2.  The
 *      velocity step uses the fields and collision rates of f^n, as in R13.
 *      Each x half-step takes its wall fluxes (Eqs. 12-15, with R12) from its
 *      own input state, so that what leaves through the wall and what the
 *      surface charge receives stay the same.  The surface charge and the
 *      wall and vacuum ledger terms therefore take dt/2 of the fluxes of
 *      f^n and dt/2 of those of the second half-step's input.  The
 *      velocity-edge loss comes from the state the velocity step acts on.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA 2018 values (SI). */
#define OR_QE 1.602176634e-19    /* elementary charge, C */
#define OR_ME 9.1093837015e-31   /* electron mass, kg */
#define OR_EPS0 8.8541878128e-12 /* vacuum permittivity, F/m */
#define OR_PI 3.14159265358979323846
#define OR_H 6.62607015e-34      /* Planck constant, J s (exact in SI) */

enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_ECFL = 4 };

enum { OR_HIST_COLS = 8 }; /* step, t, sigma, g_pe, g_see, g_vac, N, Ex(0) */

typedef struct {
  /* grid (R3) */
  int nx, nv1, nv2;
  double h_max, v1_min, v1_max, v2_min, v2_max;
  double dx, dv1, dv2, dt;
  double *x, *v1, *v2;
  /* f^n and the buffer that receives f^{n+1}; index (k*nv1 + i)*nv2 + j */
  double *f, *f_next;
  /* fields */
  double Ey, Ex_ext;
  int self_consistent;
  /* secondary emission */
  double delta_max, A_max, k_s, T_se;
  int see_enabled;
  double *delta; /* SEEY matrix, Eqs. 8-11; zero where v1 >= 0 */
  double *g_se;  /* emission shape of Eq. 15, zero where v1 <= 0 */
  /* source */
  double J, x_lo, x_hi, T_fe;
  int n_band;
  double *g_fe; /* source velocity shape of Eq. 7 */
  /* electron-electron collisions, Eqs. 3-5 (R11) */
  int collisions;
  double T_e, ln_lambda;
  double *g_e0; /* equilibrium of Eq. 5, unit density on the grid */
  /* electron reflection at the dielectric (R12) */
  double refl;
  /* time splitting (R13): 0 unsplit, 1 Lie (x, then velocity) */
  int scheme;
  double *f_tmp;
  /* state */
  double sigma;
  int64_t step;
  /* quantities evaluated on the current state */
  double *ne, *Ex, *a1;
  double *plane_sum; /* per-plane partials of sums over planes */
  double a2;
  double g_pe, g_see, g_emit, g_vac, l_v, n_tot;
  /* ledger */
  double n0, sigma0, cum_emit, cum_see, cum_pe, cum_vac, cum_lv, cum_inj;
  /* history */
  double *hist;
  int64_t hist_rows, hist_cap;
  int64_t sat_window;
  double sat_tol;
  int64_t sat_step;
} or_state;

static double pos(double a) { return a > 0.0 ? a : 0.0; }
static double neg(double a) { return a < 0.0 ? a : 0.0; }
static size_t cell(const or_state *s, int k, int i, int j) {
  return ((size_t)k * (size_t)s->nv1 + (size_t)i) * (size_t)s->nv2 + (size_t)j;
}
static size_t vcell(const or_state *s, int i, int j) {
  return (size_t)i * (size_t)s->nv2 + (size_t)j;
}

/* ------------------------------------------------------------------ */
/* Secondary-electron yield, Eqs. 8-9 (Sec. 2).  A in eV, alpha in rad. */
double oracle_seey(double A_eV, double alpha, double delta_max, double A_max,
                   double k_s) {
  double z = 1.284 * A_eV / (A_max * (1.0 + k_s * alpha * alpha / OR_PI));
  if (z <= 0.0) return 0.0; /* the yield vanishes as the incident energy -> 0 */
  return 1.526 * delta_max * (1.0 + k_s * alpha * alpha / (2.0 * OR_PI)) *
         (1.0 - exp(-pow(z, 1.725))) / pow(z, 0.725);
}

/* Incident energy in eV, Eq. 10, and incidence angle, Eq. 11. */
double oracle_incident_energy_eV(double v1, double v2) {
  return 0.5 * OR_ME * (v1 * v1 + v2 * v2) / OR_QE;
}
double oracle_incidence_angle(double v1, double v2) {
  return atan(fabs(v2 / v1));
}

/* SEEY matrix over the velocity grid (Sec. 2, text after Eq. 11: SEE only
 * for v1 < 0; computed once and reused every step). */
static void build_delta(or_state *s) {
  for (int i = 0; i < s->nv1; i++)
    for (int j = 0; j < s->nv2; j++) {
      double d = 0.0;
      if (s->v1[i] < 0.0) {
        double A = oracle_incident_energy_eV(s->v1[i], s->v2[j]);
        double al = oracle_incidence_angle(s->v1[i], s->v2[j]);
        d = oracle_seey(A, al, s->delta_max, s->A_max, s->k_s);
      }
      s->delta[vcell(s, i, j)] = d;
    }
}

/* Re-emission shape, Eq. 15 with the flux definition Eq. 16.  The continuum
 * prefactor of Eq. 15 is replaced by the discrete normalisation (R5):
 * sum_{v1>0} v1 g_se dv1 dv2 = 1, so that the emitted flux is Gamma_see. */
static void build_gse(or_state *s) {
  double T = s->T_se * OR_QE; /* temperature in J */
  double norm = 0.0;
  for (int i = 0; i < s->nv1; i++)
    for (int j = 0; j < s->nv2; j++) {
      double g = 0.0;
      if (s->v1[i] > 0.0)
        g = exp(-OR_ME * (s->v1[i] * s->v1[i] + s->v2[j] * s->v2[j]) / (2.0 * T));
      s->g_se[vcell(s, i, j)] = g;
      norm += s->v1[i] * g * s->dv1 * s->dv2;
    }
  for (int i = 0; i < s->nv1; i++)
    for (int j = 0; j < s->nv2; j++)
      s->g_se[vcell(s, i, j)] = norm > 0.0 ? s->g_se[vcell(s, i, j)] / norm : 0.0;
}

/* Continuum-normalised Eq. 15 for unit Gamma_see (used only by tests that
 * pin the prefactor against Eq. 16). */
double oracle_emission_continuum(double v1, double v2, double T_se_eV) {
  double T = T_se_eV * OR_QE;
  if (v1 <= 0.0) return 0.0;
  return 1.0 / sqrt(2.0 * OR_PI) * pow(OR_ME / T, 1.5) *
         exp(-(OR_ME * v1 * v1 + OR_ME * v2 * v2) / (2.0 * T));
}

/* Field-emission source shape of Eq. 7: full Maxwellian in v1, half
 * Maxwellian on v2 > 0 (toward the anode), temperature T_fe, renormalised on
 * the grid to unit density (R6). */
static void build_gfe(or_state *s) {
  double T = s->T_fe * OR_QE;
  double norm = 0.0;
  for (int i = 0; i < s->nv1; i++)
    for (int j = 0; j < s->nv2; j++) {
      double g = 0.0;
      if (s->v2[j] > 0.0)
        g = exp(-OR_ME * (s->v1[i] * s->v1[i] + s->v2[j] * s->v2[j]) / (2.0 * T));
      s->g_fe[vcell(s, i, j)] = g;
      norm += g * s->dv1 * s->dv2;
    }
  for (int i = 0; i < s->nv1; i++)
    for (int j = 0; j < s->nv2; j++)
      s->g_fe[vcell(s, i, j)] = norm > 0.0 ? s->g_fe[vcell(s, i, j)] / norm : 0.0;
}

/* Equilibrium VDF of Eq. 5 at T_e, renormalised on the grid to unit
 * density (R11). */
static void build_ge0(or_state *s) {
  double T = s->T_e * OR_QE;
  double norm = 0.0;
  for (int i = 0; i < s->nv1; i++)
    for (int j = 0; j < s->nv2; j++) {
      double g = OR_ME / (2.0 * OR_PI * T) *
                 exp(-(OR_ME * s->v1[i] * s->v1[i] + OR_ME * s->v2[j] * s->v2[j]) / (2.0 * T));
      s->g_e0[vcell(s, i, j)] = g;
      norm += g * s->dv1 * s->dv2;
    }
  for (int i = 0; i < s->nv1; i++)
    for (int j = 0; j < s->nv2; j++)
      s->g_e0[vcell(s, i, j)] = norm > 0.0 ? s->g_e0[vcell(s, i, j)] / norm : 0.0;
}

/* Eq. 4: electron-electron collision frequency (1/s) at density n (m^-3),
 * temperature T_e (eV) and Coulomb logarithm ln_lambda. */
double oracle_nu_ee(double n, double T_e_eV, double ln_lambda) {
  const double T = T_e_eV * OR_QE;
  return n * pow(OR_QE, 4) * ln_lambda /
         (12.0 * pow(OR_PI, 1.5) * OR_EPS0 * OR_EPS0 * sqrt(OR_ME) * pow(T, 1.5));
}

/* BGK relaxation rate of plane k of the current state (0 when off). */
static double nu_plane(const or_state *s, int k) {
  if (!s->collisions || !(s->ne[k] > 0.0)) return 0.0;
  return oracle_nu_ee(s->ne[k], s->T_e, s->ln_lambda);
}

static int in_band(const or_state *s, int k) {
  return s->J != 0.0 && s->x[k] >= s->x_lo && s->x[k] <= s->x_hi;
}

/* Source term S_CTJ of Eq. 7 at cell (k, i, j): (J/e)/W * shape. */
static double source(const or_state *s, int k, int i, int j) {
  if (!in_band(s, k) || s->n_band == 0) return 0.0;
  double W = (double)s->n_band * s->dx;
  return s->J / OR_QE / W * s->g_fe[vcell(s, i, j)];
}

/* ------------------------------------------------------------------ */
/* Step 1: density moment and fields of the current state. */
static void evaluate_fields(or_state *s) {
#pragma omp parallel for schedule(static)
  for (int k = 0; k < s->nx; k++) {
    double n = 0.0;
    for (int i = 0; i < s->nv1; i++)
      for (int j = 0; j < s->nv2; j++) n += s->f[cell(s, k, i, j)] * s->dv1 * s->dv2;
    s->ne[k] = n;
  }
  /* R7: Gauss's law integrated from the wall, where E_x = sigma/(2 eps0);
   * space charge -e n.  Cell-centred: the cell's own charge counts half. */
  double below = 0.0; /* sum_{m<k} n_m */
  for (int k = 0; k < s->nx; k++) {
    if (s->self_consistent)
      s->Ex[k] = s->sigma / (2.0 * OR_EPS0) -
                 OR_QE / OR_EPS0 * s->dx * (below + 0.5 * s->ne[k]);
    else
      s->Ex[k] = s->Ex_ext;
    below += s->ne[k];
    s->a1[k] = -OR_QE * s->Ex[k] / OR_ME; /* R8 */
  }
  s->a2 = -OR_QE * s->Ey / OR_ME;
}

/* Step 2: wall fluxes, Eqs. 12-14, from the plane x = 0 of f^n. */
static void evaluate_wall(or_state *s) {
  double gpe = 0.0, gsee = 0.0;
  for (int i = 0; i < s->nv1; i++) {
    if (!(s->v1[i] < 0.0)) continue;
    for (int j = 0; j < s->nv2; j++) {
      double dG = -s->v1[i] * s->f[cell(s, 0, i, j)] * s->dv1 * s->dv2; /* Eq. 13 */
      gpe += dG;
      /* Eqs. 12, 14 on the absorbed part (R12) */
      if (s->see_enabled) gsee += (1.0 - s->refl) * s->delta[vcell(s, i, j)] * dG;
    }
  }
  s->g_pe = gpe;
  s->g_see = gsee;
}

/* Face fluxes of the donor-cell scheme (R2).  A face is named by the index
 * of the cell on its upper side; face 0 is the lower domain edge.        */

/* x face kf between cells kf-1 and kf; kf = 0 is the dielectric wall,
 * kf = nx the vacuum boundary. */
static double flux_x(const or_state *s, int kf, int i, int j) {
  double v = s->v1[i];
  double lower, upper;
  if (kf == 0) { /* Eq. 15: inflow from the wall carries the SE distribution */
    lower = s->g_see * s->g_se[vcell(s, i, j)];
    /* R12: plus the specularly reflected part of the incident distribution */
    if (s->refl > 0.0 && v > 0.0) lower += s->refl * s->f[cell(s, 0, s->nv1 - 1 - i, j)];
  } else {
    lower = s->f[cell(s, kf - 1, i, j)];
  }
  if (kf == s->nx) /* Eq. 17: nothing enters from the vacuum side */
    upper = 0.0;
  else
    upper = s->f[cell(s, kf, i, j)];
  return pos(v) * lower + neg(v) * upper;
}

/* v1 face if between cells if-1 and if, at position k (R9 at the edges). */
static double flux_v1(const or_state *s, int k, int iface, int j) {
  double a = s->a1[k];
  double lower = iface == 0 ? 0.0 : s->f[cell(s, k, iface - 1, j)];
  double upper = iface == s->nv1 ? 0.0 : s->f[cell(s, k, iface, j)];
  return pos(a) * lower + neg(a) * upper;
}

/* v2 face jf between cells jf-1 and jf (R9 at the edges). */
static double flux_v2(const or_state *s, int k, int i, int jface) {
  double a = s->a2;
  double lower = jface == 0 ? 0.0 : s->f[cell(s, k, i, jface - 1)];
  double upper = jface == s->nv2 ? 0.0 : s->f[cell(s, k, i, jface)];
  return pos(a) * lower + neg(a) * upper;
}

/* Boundary fluxes of the current state used by the ledger. */
/* Outflow through the velocity-grid edges (R9) of the state in s->f. */
static double edge_loss(const or_state *s) {
#pragma omp parallel for schedule(static)
  for (int k = 0; k < s->nx; k++) {
    double p = 0.0;
    for (int j = 0; j < s->nv2; j++)
      p += (flux_v1(s, k, s->nv1, j) - flux_v1(s, k, 0, j)) * s->dx * s->dv2;
    for (int i = 0; i < s->nv1; i++)
      p += (flux_v2(s, k, i, s->nv2) - flux_v2(s, k, i, 0)) * s->dx * s->dv1;
    s->plane_sum[k] = p;
  }
  double lv = 0.0;
  for (int k = 0; k < s->nx; k++) lv += s->plane_sum[k];
  return lv;
}

static void evaluate_boundaries(or_state *s) {
  double emit = 0.0, vac = 0.0;
  for (int i = 0; i < s->nv1; i++)
    for (int j = 0; j < s->nv2; j++) {
      if (s->v1[i] > 0.0) emit += flux_x(s, 0, i, j) * s->dv1 * s->dv2;
      vac += flux_x(s, s->nx, i, j) * s->dv1 * s->dv2;
    }
  const double lv = edge_loss(s);
  double ntot = 0.0;
  for (int k = 0; k < s->nx; k++) ntot += s->ne[k] * s->dx;
  s->g_emit = emit;
  s->g_vac = vac;
  s->l_v = lv;
  s->n_tot = ntot;
}

static void evaluate_state(or_state *s) {
  evaluate_fields(s);
  evaluate_wall(s);
  evaluate_boundaries(s);
}

static int write_history_row(or_state *s, int64_t row) {
  if (row >= s->hist_cap) {
    int64_t cap = s->hist_cap ? 2 * s->hist_cap : 1024;
    while (cap <= row) cap *= 2;
    double *h = (double *)realloc(s->hist, (size_t)cap * OR_HIST_COLS * sizeof(double));
    if (!h) return OR_ENOMEM;
    s->hist = h;
    s->hist_cap = cap;
  }
  double *r = s->hist + (size_t)row * OR_HIST_COLS;
  r[0] = (double)s->step;
  r[1] = (double)s->step * s->dt;
  r[2] = s->sigma;
  r[3] = s->g_pe;
  r[4] = s->g_see;
  r[5] = s->g_vac;
  r[6] = s->n_tot;
  r[7] = s->Ex[0];
  if (row + 1 > s->hist_rows) s->hist_rows = row + 1;
  return OR_OK;
}

/* Convergence test stated at the end of Sec. 2 (R10). */
static void check_saturation(or_state *s) {
  int64_t m = s->hist_rows - 1;
  if (s->sat_step >= 0 || m < s->sat_window) return;
  const double *now = s->hist + (size_t)m * OR_HIST_COLS;
  const double *old = s->hist + (size_t)(m - s->sat_window) * OR_HIST_COLS;
  for (int c = 2; c <= 4; c++)
    if (!(fabs(now[c] - old[c]) <= s->sat_tol * fabs(now[c]))) return;
  s->sat_step = s->step;
}

/* Reset the run to the current (f, sigma): step 0, empty history, ledger
 * baseline taken from the current state. */
static int reset_run(or_state *s) {
  s->step = 0;
  s->hist_rows = 0;
  s->sat_step = -1;
  evaluate_state(s);
  s->n0 = s->n_tot;
  s->sigma0 = s->sigma;
  s->cum_emit = s->cum_see = s->cum_pe = s->cum_vac = s->cum_lv = s->cum_inj = 0.0;
  return write_history_row(s, 0);
}

/* Parameters changed: re-evaluate the current state, rewrite its row. */
static int refresh(or_state *s) {
  evaluate_state(s);
  return write_history_row(s, s->hist_rows > 0 ? s->hist_rows - 1 : 0);
}

/* ------------------------------------------------------------------ */
void oracle_destroy(or_state *s) {
  if (!s) return;
  free(s->x); free(s->v1); free(s->v2);
  free(s->f); free(s->f_next); free(s->f_tmp);
  free(s->delta); free(s->g_se); free(s->g_fe); free(s->g_e0);
  free(s->ne); free(s->Ex); free(s->a1); free(s->plane_sum);
  free(s->hist);
  free(s);
}

/* Grid set-up.  dt <= 0 selects dt = cfl * dx / max(|v1_min|, |v1_max|). */
or_state *oracle_create(int nx, int nv1, int nv2, double h_max, double v1_min,
                        double v1_max, double v2_min, double v2_max, double dt,
                        double cfl) {
  if (nx < 2 || nv1 < 2 || nv2 < 2 || !(h_max > 0.0) || !(v1_min < v1_max) ||
      !(v2_min < v2_max))
    return NULL;
  if (!(dt > 0.0) && !(cfl > 0.0)) return NULL;
  or_state *s = (or_state *)calloc(1, sizeof(or_state));
  if (!s) return NULL;
  s->nx = nx; s->nv1 = nv1; s->nv2 = nv2;
  s->h_max = h_max;
  s->v1_min = v1_min; s->v1_max = v1_max; s->v2_min = v2_min; s->v2_max = v2_max;
  s->dx = h_max / nx;
  s->dv1 = (v1_max - v1_min) / nv1;
  s->dv2 = (v2_max - v2_min) / nv2;
  double vmax = fmax(fabs(v1_min), fabs(v1_max));
  s->dt = dt > 0.0 ? dt : cfl * s->dx / vmax;
  size_t ncell = (size_t)nx * nv1 * nv2, nv = (size_t)nv1 * nv2;
  s->x = (double *)malloc(nx * sizeof(double));
  s->v1 = (double *)malloc(nv1 * sizeof(double));
  s->v2 = (double *)malloc(nv2 * sizeof(double));
  s->f = (double *)calloc(ncell, sizeof(double));
  s->f_next = (double *)calloc(ncell, sizeof(double));
  s->f_tmp = (double *)calloc(ncell, sizeof(double));
  s->delta = (double *)calloc(nv, sizeof(double));
  s->g_se = (double *)calloc(nv, sizeof(double));
  s->g_fe = (double *)calloc(nv, sizeof(double));
  s->g_e0 = (double *)calloc(nv, sizeof(double));
  s->ne = (double *)calloc(nx, sizeof(double));
  s->Ex = (double *)calloc(nx, sizeof(double));
  s->a1 = (double *)calloc(nx, sizeof(double));
  s->plane_sum = (double *)calloc(nx, sizeof(double));
  if (!s->plane_sum || !s->x || !s->v1 || !s->v2 || !s->f || !s->f_next || !s->f_tmp || !s->delta || !s->g_se ||
      !s->g_fe || !s->g_e0 || !s->ne || !s->Ex || !s->a1) {
    oracle_destroy(s);
    return NULL;
  }
  for (int k = 0; k < nx; k++) s->x[k] = (k + 0.5) * s->dx;
  for (int i = 0; i < nv1; i++) s->v1[i] = v1_min + (i + 0.5) * s->dv1;
  for (int j = 0; j < nv2; j++) s->v2[j] = v2_min + (j + 0.5) * s->dv2;
  /* defaults: no applied field, self-consistent E_x, no SEE, no source */
  s->self_consistent = 1;
  s->delta_max = 0.0; s->A_max = 1.0; s->k_s = 1.0; s->T_se = 1.0;
  s->T_fe = 1.0;
  s->T_e = 2.0; s->ln_lambda = 10.0; /* Sec. 2 defaults; collisions off */
  build_ge0(s);
  s->sat_window = 10000;
  s->sat_tol = 1e-3;
  if (reset_run(s) != OR_OK) { oracle_destroy(s); return NULL; }
  return s;
}

int oracle_set_fields(or_state *s, double Ey, int self_consistent, double Ex_ext) {
  if (!(Ey <= 0.0)) return OR_EINVAL; /* Sec. 2: E_y is negative (cathode left) */
  s->Ey = Ey;
  s->self_consistent = self_consistent ? 1 : 0;
  s->Ex_ext = Ex_ext;
  return refresh(s);
}

int oracle_set_see(or_state *s, double delta_max, double A_max_eV, double k_s,
                   double T_se_eV, int enabled) {
  if (!(delta_max >= 0.0) || !(A_max_eV > 0.0) || !(k_s >= 0.0) || !(T_se_eV > 0.0))
    return OR_EINVAL;
  s->delta_max = delta_max; s->A_max = A_max_eV; s->k_s = k_s; s->T_se = T_se_eV;
  s->see_enabled = enabled ? 1 : 0;
  build_delta(s);
  build_gse(s);
  return refresh(s);
}

int oracle_set_source(or_state *s, double J, double x_lo, double x_hi, double T_fe_eV) {
  if (!(J >= 0.0) || !(x_lo <= x_hi) || !(T_fe_eV > 0.0)) return OR_EINVAL;
  s->J = J; s->x_lo = x_lo; s->x_hi = x_hi; s->T_fe = T_fe_eV;
  s->n_band = 0;
  for (int k = 0; k < s->nx; k++) s->n_band += in_band(s, k);
  if (J > 0.0 && s->n_band == 0) return OR_EINVAL;
  build_gfe(s);
  return refresh(s);
}

/* Electron-electron collisions of Eqs. 3-5 (R11). */
int oracle_set_collisions(or_state *s, double T_e_eV, double ln_lambda, int enabled) {
  if (!(T_e_eV > 0.0) || !(ln_lambda >= 0.0)) return OR_EINVAL;
  s->T_e = T_e_eV;
  s->ln_lambda = ln_lambda;
  s->collisions = enabled ? 1 : 0;
  build_ge0(s);
  return refresh(s);
}

/* Electron reflection at the dielectric (R12); R_f > 0 needs a v1 grid
 * symmetric about 0. */
int oracle_set_reflection(or_state *s, double R_f) {
  if (!(R_f >= 0.0 && R_f <= 1.0)) return OR_EINVAL;
  if (R_f > 0.0 && fabs(s->v1_min + s->v1_max) > 1e-12 * fabs(s->v1_max)) return OR_EINVAL;
  s->refl = R_f;
  return refresh(s);
}

/* Time splitting: 0 unsplit, 1 Lie (R13), 2 Strang (R14). */
int oracle_set_scheme(or_state *s, int scheme) {
  if (scheme != 0 && scheme != 1 && scheme != 2) return OR_EINVAL;
  s->scheme = scheme;
  return OR_OK;
}

int oracle_set_convergence(or_state *s, int64_t window, double tol) {
  if (window < 1 || !(tol >= 0.0)) return OR_EINVAL;
  s->sat_window = window;
  s->sat_tol = tol;
  return OR_OK;
}

/* Replace the state (f, sigma); the run restarts at step 0. */
int oracle_set_state(or_state *s, const double *f, double sigma) {
  memcpy(s->f, f, (size_t)s->nx * s->nv1 * s->nv2 * sizeof(double));
  s->sigma = sigma;
  return reset_run(s);
}

/* Largest sum of |Courant numbers| over the grid for the current state. */
double oracle_courant_sum(const or_state *s) {
  double cx = 0.0, c1 = 0.0;
  for (int i = 0; i < s->nv1; i++) cx = fmax(cx, fabs(s->v1[i]) * s->dt / s->dx);
  for (int k = 0; k < s->nx; k++) c1 = fmax(c1, fabs(s->a1[k]) * s->dt / s->dv1);
  double cb = 0.0;
  for (int k = 0; k < s->nx; k++) cb = fmax(cb, nu_plane(s, k) * s->dt);
  return cx + c1 + fabs(s->a2) * s->dt / s->dv2 + cb;
}

/* Steps 3-5 for one time step (R1, R4). */
/* Step 3 (R1): every cell of f^n updated with all face fluxes from f^n. */
static void unsplit_update(or_state *s) {
  const double dt = s->dt;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < s->nx; k++) {
    const double nu = nu_plane(s, k);
    for (int i = 0; i < s->nv1; i++)
      for (int j = 0; j < s->nv2; j++) {
        double dFx = flux_x(s, k + 1, i, j) - flux_x(s, k, i, j);
        double dFv1 = flux_v1(s, k, i + 1, j) - flux_v1(s, k, i, j);
        double dFv2 = flux_v2(s, k, i, j + 1) - flux_v2(s, k, i, j);
        /* Eq. 3: nu_ee (n_e f_e0 - f), from f^n */
        double coll = nu * (s->ne[k] * s->g_e0[vcell(s, i, j)] - s->f[cell(s, k, i, j)]);
        s->f_next[cell(s, k, i, j)] = s->f[cell(s, k, i, j)] - dt / s->dx * dFx -
                                      dt / s->dv1 * dFv1 - dt / s->dv2 * dFv2 +
                                      dt * source(s, k, i, j) + dt * coll;
      }
  }
}

/* x-advection over h of the state in s->f into out, with the wall inflow of
 * Eq. 15 from s->g_see (the wall fluxes of that state). */
static void x_pass(or_state *s, double h, double *out) {
#pragma omp parallel for schedule(static)
  for (int k = 0; k < s->nx; k++)
    for (int i = 0; i < s->nv1; i++)
      for (int j = 0; j < s->nv2; j++) {
        double dFx = flux_x(s, k + 1, i, j) - flux_x(s, k, i, j);
        out[cell(s, k, i, j)] = s->f[cell(s, k, i, j)] - h / s->dx * dFx;
      }
}

/* Velocity step over h of the state in s->f into out, with the fields and
 * collision rates of f^n (s->a1, s->ne). */
static void v_pass(or_state *s, double h, double *out) {
#pragma omp parallel for schedule(static)
  for (int k = 0; k < s->nx; k++) {
    const double nu = nu_plane(s, k);
    for (int i = 0; i < s->nv1; i++)
      for (int j = 0; j < s->nv2; j++) {
        double dFv1 = flux_v1(s, k, i + 1, j) - flux_v1(s, k, i, j);
        double dFv2 = flux_v2(s, k, i, j + 1) - flux_v2(s, k, i, j);
        double coll = nu * (s->ne[k] * s->g_e0[vcell(s, i, j)] - s->f[cell(s, k, i, j)]);
        out[cell(s, k, i, j)] = s->f[cell(s, k, i, j)] - h / s->dv1 * dFv1 -
                                h / s->dv2 * dFv2 + h * source(s, k, i, j) + h * coll;
      }
  }
}

/* R13: x-advection of f^n into f_next, then the velocity step of that
 * intermediate state (the flux helpers read s->f, so it stands in for f^n
 * meanwhile) into f_tmp, copied back to f_next.  *lv receives the
 * velocity-edge loss of the intermediate state. */
static void lie_update(or_state *s, double *lv) {
  double *fn = s->f;
  x_pass(s, s->dt, s->f_next);
  s->f = s->f_next;
  v_pass(s, s->dt, s->f_tmp);
  *lv = edge_loss(s);
  s->f = fn;
  memcpy(s->f_next, s->f_tmp, (size_t)s->nx * s->nv1 * s->nv2 * sizeof(double));
}

/* Charge deposited per unit time by the wall fluxes of the state in s->f
 * (the sum of Eq. 18 without e dt). */
static double wall_charge_rate(const or_state *s) {
  double dsig = 0.0;
  for (int i = 0; i < s->nv1; i++) {
    if (!(s->v1[i] < 0.0)) continue;
    for (int j = 0; j < s->nv2; j++) {
      double dG = -s->v1[i] * s->f[cell(s, 0, i, j)] * s->dv1 * s->dv2;
      double d = s->see_enabled ? s->delta[vcell(s, i, j)] : 0.0;
      dsig += (1.0 - s->refl) * (d - 1.0) * dG; /* R12: reflected electrons deposit nothing */
    }
  }
  return dsig;
}

/* Boundary terms of the second x half-step of a Strang step. */
typedef struct {
  double emit, see, pe, vac, dsig;
} half_wall;

/* R14: Strang, x over dt/2, velocity over dt, x over dt/2.  The first x
 * half-step takes the wall fluxes of f^n, the second those of its own
 * input (Eqs. 12-15 on that state), returned in *w2 for sigma and the
 * ledger; *lv receives the velocity-edge loss of the state the velocity
 * step acts on.  f_next receives f^{n+1}; s->f and the wall fluxes of f^n
 * are left as they were. */
static void strang_update(or_state *s, double *lv, half_wall *w2) {
  const double h = 0.5 * s->dt;
  double *fn = s->f, *f1 = s->f_next, *f2 = s->f_tmp;
  const double g_pe = s->g_pe, g_see = s->g_see;
  x_pass(s, h, f1);
  s->f = f1;
  v_pass(s, s->dt, f2);
  *lv = edge_loss(s);
  s->f = f2;
  evaluate_wall(s); /* Gamma_pe, Gamma_see of the second half-step's input */
  w2->pe = s->g_pe;
  w2->see = s->g_see;
  w2->emit = w2->vac = 0.0;
  for (int i = 0; i < s->nv1; i++)
    for (int j = 0; j < s->nv2; j++) {
      if (s->v1[i] > 0.0) w2->emit += flux_x(s, 0, i, j) * s->dv1 * s->dv2;
      w2->vac += flux_x(s, s->nx, i, j) * s->dv1 * s->dv2;
    }
  w2->dsig = wall_charge_rate(s);
  x_pass(s, h, f1);
  s->f = fn;
  s->g_pe = g_pe;
  s->g_see = g_see;
}

static int one_step(or_state *s) {
  if (oracle_courant_sum(s) > 1.0 + 1e-12) return OR_ECFL;
  const double dt = s->dt;
  double lv_step = s->l_v; /* loss of the state the velocity advection acts on */
  /* share of the step's dt carried by the boundary terms of f^n */
  const double hn = s->scheme == 2 ? 0.5 * dt : dt;
  half_wall w2 = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (s->scheme == 2)
    strang_update(s, &lv_step, &w2);
  else if (s->scheme == 1)
    lie_update(s, &lv_step);
  else
    unsplit_update(s);
  /* ledger: fluxes of state n times dt */
#pragma omp parallel for schedule(static)
  for (int k = 0; k < s->nx; k++) {
    double p = 0.0;
    for (int i = 0; i < s->nv1; i++)
      for (int j = 0; j < s->nv2; j++) p += source(s, k, i, j) * s->dx * s->dv1 * s->dv2;
    s->plane_sum[k] = p;
  }
  double inj = 0.0;
  for (int k = 0; k < s->nx; k++) inj += s->plane_sum[k];
  s->cum_emit += hn * s->g_emit;
  s->cum_see += hn * s->g_see;
  s->cum_pe += hn * s->g_pe;
  s->cum_vac += hn * s->g_vac;
  s->cum_lv += dt * lv_step;
  s->cum_inj += dt * inj;
  /* Eq. 18: sigma^{n+1} = sigma^n + e dt sum_{v1<0} (delta - 1) dGamma_pe */
  s->sigma += OR_QE * hn * wall_charge_rate(s);
  if (s->scheme == 2) { /* the second x half-step's boundary terms (R14) */
    s->cum_emit += hn * w2.emit;
    s->cum_see += hn * w2.see;
    s->cum_pe += hn * w2.pe;
    s->cum_vac += hn * w2.vac;
    s->sigma += OR_QE * hn * w2.dsig;
  }
  double *t = s->f;
  s->f = s->f_next;
  s->f_next = t;
  s->step += 1;
  evaluate_state(s);
  int rc = write_history_row(s, s->hist_rows);
  if (rc != OR_OK) return rc;
  check_saturation(s);
  return OR_OK;
}

int oracle_step(or_state *s, int64_t n) {
  for (int64_t m = 0; m < n; m++) {
    int rc = one_step(s);
    if (rc != OR_OK) return rc;
  }
  return OR_OK;
}

/* Threads of the OpenMP build (n >= 1 sets the count); returns the count
 * the loops over planes use.  The serial build always returns 1. */
int oracle_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Getters. */
void oracle_get_f(const or_state *s, double *out) {
  memcpy(out, s->f, (size_t)s->nx * s->nv1 * s->nv2 * sizeof(double));
}
double oracle_surface_charge(const or_state *s) { return s->sigma; }
void oracle_moments(const or_state *s, double *ne, double *Ex, double *g_pe,
                    double *g_see) {
  if (ne) memcpy(ne, s->ne, s->nx * sizeof(double));
  if (Ex) memcpy(Ex, s->Ex, s->nx * sizeof(double));
  if (g_pe) *g_pe = s->g_pe;
  if (g_see) *g_see = s->g_see;
}
/* grid facts: dx, dv1, dv2, dt, a2, n_band, step, sat_step */
void oracle_info(const or_state *s, double *out) {
  out[0] = s->dx; out[1] = s->dv1; out[2] = s->dv2; out[3] = s->dt;
  out[4] = s->a2; out[5] = (double)s->n_band; out[6] = (double)s->step;
  out[7] = (double)s->sat_step;
}
/* Ledger: N, N0, cum_emit, cum_pe, cum_vac, cum_lv, cum_inj, sigma0, cum_see */
void oracle_ledger(const or_state *s, double *out) {
  out[0] = s->n_tot; out[1] = s->n0; out[2] = s->cum_emit; out[3] = s->cum_pe;
  out[4] = s->cum_vac; out[5] = s->cum_lv; out[6] = s->cum_inj; out[7] = s->sigma0;
  out[8] = s->cum_see;
}
/* Boundary fluxes of the current state: emit, vac, l_v, a1[] (per x). */
void oracle_boundary_fluxes(const or_state *s, double *out) {
  out[0] = s->g_emit; out[1] = s->g_vac; out[2] = s->l_v;
}
void oracle_accel(const or_state *s, double *a1) {
  memcpy(a1, s->a1, s->nx * sizeof(double));
}
int64_t oracle_history(const or_state *s, double *out, int64_t max_rows) {
  int64_t n = s->hist_rows < max_rows ? s->hist_rows : max_rows;
  int64_t first = s->hist_rows - n; /* the most recent rows, oldest first */
  memcpy(out, s->hist + (size_t)first * OR_HIST_COLS, (size_t)n * OR_HIST_COLS * sizeof(double));
  return n;
}
void oracle_tables(const or_state *s, double *delta, double *g_se, double *g_fe) {
  size_t nv = (size_t)s->nv1 * s->nv2;
  if (delta) memcpy(delta, s->delta, nv * sizeof(double));
  if (g_se) memcpy(g_se, s->g_se, nv * sizeof(double));
  if (g_fe) memcpy(g_fe, s->g_fe, nv * sizeof(double));
}
void oracle_grid(const or_state *s, double *x, double *v1, double *v2) {
  if (x) memcpy(x, s->x, s->nx * sizeof(double));
  if (v1) memcpy(v1, s->v1, s->nv1 * sizeof(double));
  if (v2) memcpy(v2, s->v2, s->nv2 * sizeof(double));
}

/* ------------------------------------------------------------------ */
/* SEEA single-particle saturation (Sec. 3, Eqs. 19-20).  Validation only. */

/* A1: the incident energy at which a normally incident electron produces
 * exactly one secondary, i.e. the first crossover delta(A, 0) = 1 of Eq. 8,
 * found by bisection on (0, A_max].  Returns -1 if delta_max <= 1. */
double oracle_first_crossover(double delta_max, double A_max_eV, double k_s) {
  if (oracle_seey(A_max_eV, 0.0, delta_max, A_max_eV, k_s) <= 1.0) return -1.0;
  double lo = 0.0, hi = A_max_eV;
  for (int it = 0; it < 200; it++) {
    double mid = 0.5 * (lo + hi);
    if (oracle_seey(mid, 0.0, delta_max, A_max_eV, k_s) < 1.0) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* Eq. 6, the Fowler-Nordheim current density J (A/m^2) at the field E
 * (V/m) for a work function e phi (phi in V), returned as ln J so that the
 * exponent -B/E (about -1.1e4 at 5 MV/m) does not underflow:
 *   J = e^3 E^2 / (8 pi h W) exp(-8 pi sqrt(2 m_e W^3) / (3 e h E)),  W = e phi. */
double oracle_fn_log_current(double E, double phi_V) {
  const double W = OR_QE * phi_V;
  const double pre = OR_QE * OR_QE * OR_QE / (8.0 * OR_PI * OR_H * W);
  const double B = 8.0 * OR_PI * sqrt(2.0 * OR_ME * W * W * W) / (3.0 * OR_QE * OR_H);
  return log(pre) + 2.0 * log(E) - B / E;
}

/* Eq. 20: saturated surface charge of the SEEA theory, A0, A1 in eV. */
double oracle_sigma_eq20(double Ey, double A0_eV, double A1_eV) {
  return 2.0 * OR_EPS0 * fabs(Ey) * pow(0.5 * (A1_eV / A0_eV - 1.0), -0.5);
}

/* Time of flight of a normally emitted secondary (Sec. 3, text before
 * Eq. 19): t_ef = 2 sqrt(2 A0 / m_e) / |a_x|. */
double oracle_time_of_flight(double A0_eV, double ax) {
  return 2.0 * sqrt(2.0 * A0_eV * OR_QE / OR_ME) / fabs(ax);
}
