"""ctypes binding of the plain FP64 CPU oracle (``fk_oracle.c``).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the smoke check and
the benchmark's CPU-baseline leg import this package.  The CUDA library never
does, and the oracle never imports the CUDA package.

The oracle advances the electron distribution f(x, v1, v2) of the 1D2V
flashover model (Sec. 2 of arXiv 2303.14119) one explicit upwind step at a
time, in FP64, with serial sums.  ``build()`` compiles the C source with gcc
(``-O2 -ffp-contract=off`` so that x86 and Arm hosts give the same bits)
twice: the serial checker ``liboracle_fk.so`` and an OpenMP build
``liboracle_fk_omp.so`` whose loops over x-planes run on several threads and
whose sums over planes are added in plane order, so that both give the same
bits (``Oracle(..., threads=n)`` selects the threaded build).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fk_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_fk.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_fk_omp.so")
_lock = threading.Lock()
_libs = {}

HIST_COLS = 8  # step, t, sigma, gamma_pe, gamma_see, gamma_vac, N, Ex(0)
OK, EINVAL, ENOMEM, ECFL = 0, 1, 2, 4

# Physical constants (CODATA 2018), for tests that need them in Python.
QE = 1.602176634e-19
ME = 9.1093837015e-31
EPS0 = 8.8541878128e-12


def build(force: bool = False) -> str:
    """Compile ``fk_oracle.c`` into ``liboracle_fk.so`` (serial) and
    ``liboracle_fk_omp.so`` (OpenMP) where stale."""
    with _lock:
        for lib, extra in ((_LIB, []), (_LIB_OMP, ["-fopenmp"])):
            if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
                tmp = lib + ".tmp%d" % os.getpid()
                subprocess.check_call(
                    ["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared", *extra,
                     _SRC, "-o", tmp, "-lm"])
                os.replace(tmp, lib)
    return _LIB


def _load(omp: bool = False):
    key = bool(omp)
    if key in _libs:
        return _libs[key]
    build()
    lib = C.CDLL(_LIB_OMP if omp else _LIB)
    P, D, I, I64 = C.c_void_p, C.c_double, C.c_int, C.c_int64
    dp = C.POINTER(C.c_double)
    sig = {
        "oracle_create": (P, [I, I, I, D, D, D, D, D, D, D]),
        "oracle_destroy": (None, [P]),
        "oracle_set_fields": (I, [P, D, I, D]),
        "oracle_set_see": (I, [P, D, D, D, D, I]),
        "oracle_set_source": (I, [P, D, D, D, D]),
        "oracle_set_convergence": (I, [P, I64, D]),
        "oracle_set_state": (I, [P, dp, D]),
        "oracle_step": (I, [P, I64]),
        "oracle_get_f": (None, [P, dp]),
        "oracle_surface_charge": (D, [P]),
        "oracle_moments": (None, [P, dp, dp, dp, dp]),
        "oracle_info": (None, [P, dp]),
        "oracle_ledger": (None, [P, dp]),
        "oracle_boundary_fluxes": (None, [P, dp]),
        "oracle_accel": (None, [P, dp]),
        "oracle_history": (I64, [P, dp, I64]),
        "oracle_tables": (None, [P, dp, dp, dp]),
        "oracle_grid": (None, [P, dp, dp, dp]),
        "oracle_courant_sum": (D, [P]),
        "oracle_seey": (D, [D, D, D, D, D]),
        "oracle_incident_energy_eV": (D, [D, D]),
        "oracle_incidence_angle": (D, [D, D]),
        "oracle_emission_continuum": (D, [D, D, D]),
        "oracle_first_crossover": (D, [D, D, D]),
        "oracle_sigma_eq20": (D, [D, D, D]),
        "oracle_time_of_flight": (D, [D, D]),
        "oracle_fn_log_current": (D, [D, D]),
        "oracle_nu_ee": (D, [D, D, D]),
        "oracle_set_collisions": (I, [P, D, D, I]),
        "oracle_set_reflection": (I, [P, D]),
        "oracle_set_scheme": (I, [P, I]),
        "oracle_threads": (I, [I]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _libs[key] = lib
    return lib


def threads(n: int = 0) -> int:
    """Set (n >= 1) and return the thread count of the OpenMP build."""
    return _load(True).oracle_threads(int(n))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# Scalar helpers (Eqs. 8-11, 15, 19-20).
def seey(A_eV, alpha, delta_max, A_max, k_s=1.0):
    return _load().oracle_seey(A_eV, alpha, delta_max, A_max, k_s)


def incident_energy_eV(v1, v2):
    return _load().oracle_incident_energy_eV(v1, v2)


def incidence_angle(v1, v2):
    return _load().oracle_incidence_angle(v1, v2)


def emission_continuum(v1, v2, T_se_eV):
    return _load().oracle_emission_continuum(v1, v2, T_se_eV)


def first_crossover(delta_max, A_max, k_s=1.0):
    return _load().oracle_first_crossover(delta_max, A_max, k_s)


def sigma_eq20(Ey, A0_eV, A1_eV):
    return _load().oracle_sigma_eq20(Ey, A0_eV, A1_eV)


def time_of_flight(A0_eV, ax):
    return _load().oracle_time_of_flight(A0_eV, ax)


def nu_ee(n, T_e_eV, ln_lambda=10.0):
    """Eq. 4: electron-electron collision frequency (1/s)."""
    return _load().oracle_nu_ee(n, T_e_eV, ln_lambda)


def fn_log_current(E, phi_V):
    """ln of the Eq. 6 Fowler-Nordheim current density (A/m^2)."""
    return _load().oracle_fn_log_current(E, phi_V)


class OracleError(RuntimeError):
    pass


class Oracle:
    """One oracle grid.  Method names follow the C-ABI of the CUDA library."""

    def __init__(self, nx, nv1, nv2, h_max, v1_min, v1_max, v2_min, v2_max, dt=0.0, cfl=0.4,
                 threads=None):
        """threads: None for the serial build (the checker); n >= 1 for the
        OpenMP build on n threads (0: its default count)."""
        lib = _load(threads is not None)
        if threads is not None:
            lib.oracle_threads(int(threads))
        self.threads = 1 if threads is None else lib.oracle_threads(0)
        self._lib = lib
        self._h = lib.oracle_create(int(nx), int(nv1), int(nv2), float(h_max), float(v1_min),
                                    float(v1_max), float(v2_min), float(v2_max), float(dt),
                                    float(cfl))
        if not self._h:
            raise OracleError("oracle_create rejected the grid")
        self.shape = (int(nx), int(nv1), int(nv2))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.oracle_destroy(self._h)
            self._h = None

    __del__ = close

    def _chk(self, rc, what):
        if rc != OK:
            raise OracleError("%s failed with status %d" % (what, rc))

    def set_fields(self, Ey, self_consistent=True, Ex_ext=0.0):
        self._chk(self._lib.oracle_set_fields(self._h, float(Ey), int(bool(self_consistent)),
                                              float(Ex_ext)), "set_fields")

    def set_see(self, delta_max, A_max_eV, k_s=1.0, T_se_eV=2.0, enabled=True):
        self._chk(self._lib.oracle_set_see(self._h, float(delta_max), float(A_max_eV), float(k_s),
                                           float(T_se_eV), int(bool(enabled))), "set_see")

    def set_source(self, J, x_lo, x_hi, T_fe_eV):
        self._chk(self._lib.oracle_set_source(self._h, float(J), float(x_lo), float(x_hi),
                                              float(T_fe_eV)), "set_source")

    def set_collisions(self, T_e_eV=2.0, ln_lambda=10.0, enabled=True):
        self._chk(self._lib.oracle_set_collisions(self._h, float(T_e_eV), float(ln_lambda),
                                                  int(bool(enabled))), "set_collisions")

    def set_reflection(self, R_f):
        self._chk(self._lib.oracle_set_reflection(self._h, float(R_f)), "set_reflection")

    def set_scheme(self, scheme):
        """0: unsplit step, 1: Lie splitting (x, then velocity), 2: Strang
        splitting (x over dt/2, velocity over dt, x over dt/2)."""
        self._chk(self._lib.oracle_set_scheme(self._h, int(scheme)), "set_scheme")

    def set_convergence(self, window, tol):
        self._chk(self._lib.oracle_set_convergence(self._h, int(window), float(tol)),
                  "set_convergence")

    def set_state(self, f, sigma=0.0):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.shape)
        self._chk(self._lib.oracle_set_state(self._h, _ptr(f), float(sigma)), "set_state")

    def step(self, n=1):
        self._chk(self._lib.oracle_step(self._h, int(n)), "step")

    def step_status(self, n=1):
        return self._lib.oracle_step(self._h, int(n))

    def get_f(self):
        out = np.empty(self.shape, dtype=np.float64)
        self._lib.oracle_get_f(self._h, _ptr(out))
        return out

    def surface_charge(self):
        return self._lib.oracle_surface_charge(self._h)

    def moments(self):
        nx = self.shape[0]
        ne = np.empty(nx)
        ex = np.empty(nx)
        gpe = np.empty(1)
        gsee = np.empty(1)
        self._lib.oracle_moments(self._h, _ptr(ne), _ptr(ex), _ptr(gpe), _ptr(gsee))
        return ne, ex, float(gpe[0]), float(gsee[0])

    def info(self):
        out = np.empty(8)
        self._lib.oracle_info(self._h, _ptr(out))
        return dict(dx=out[0], dv1=out[1], dv2=out[2], dt=out[3], a2=out[4],
                    n_band=int(out[5]), step=int(out[6]), sat_step=int(out[7]))

    def ledger(self):
        out = np.empty(9)
        self._lib.oracle_ledger(self._h, _ptr(out))
        keys = ["N", "N0", "emit", "pe", "vac", "lv", "inj", "sigma0", "see"]
        return dict(zip(keys, out.tolist()))

    def boundary_fluxes(self):
        out = np.empty(3)
        self._lib.oracle_boundary_fluxes(self._h, _ptr(out))
        return dict(emit=out[0], vac=out[1], lv=out[2])

    def accel(self):
        a = np.empty(self.shape[0])
        self._lib.oracle_accel(self._h, _ptr(a))
        return a

    def history(self, max_rows=None):
        if max_rows is None:
            max_rows = self.info()["step"] + 1
        out = np.empty((int(max_rows), HIST_COLS))
        n = self._lib.oracle_history(self._h, _ptr(out), int(max_rows))
        return out[:n]

    def tables(self):
        nv = self.shape[1] * self.shape[2]
        d, gse, gfe = np.empty(nv), np.empty(nv), np.empty(nv)
        self._lib.oracle_tables(self._h, _ptr(d), _ptr(gse), _ptr(gfe))
        sh = self.shape[1:]
        return d.reshape(sh), gse.reshape(sh), gfe.reshape(sh)

    def grid(self):
        x, v1, v2 = np.empty(self.shape[0]), np.empty(self.shape[1]), np.empty(self.shape[2])
        self._lib.oracle_grid(self._h, _ptr(x), _ptr(v1), _ptr(v2))
        return x, v1, v2

    def courant_sum(self):
        return self._lib.oracle_courant_sum(self._h)
