"""Python binding of the C ABI in ``include/fk.h`` (ctypes, marshalling only).

Every function here has the name of the C entry point it calls and does
nothing but convert arguments and results; every step of the solver runs in
the CUDA kernels of ``libflashkin.so``.  There is no CPU path: if the library
is missing or cannot load, importing the binding's functions raises.

Host arrays are numpy FP64 arrays (any contiguous buffer works; a pinned
torch CPU tensor viewed with ``.numpy()`` makes the copies asynchronous-
capable).  Streams are passed as raw ``cudaStream_t`` integers, e.g.
``torch.cuda.current_stream().cuda_stream``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

(FK_OK, FK_EINVAL, FK_ENOMEM, FK_ECUDA, FK_ECFL, FK_ENUMERIC, FK_ETIMEOUT, FK_ESTATE,
 FK_ENEGATIVE, FK_EBOUNDS) = range(10)
FK_F64, FK_F32 = 0, 1
FK_SCHEME_UNSPLIT, FK_SCHEME_LIE, FK_SCHEME_STRANG = 0, 1, 2
FK_HISTORY_COLS = 8
FK_LEDGER_LEN = 9
STATUS_NAMES = {0: "FK_OK", 1: "FK_EINVAL", 2: "FK_ENOMEM", 3: "FK_ECUDA", 4: "FK_ECFL",
                5: "FK_ENUMERIC", 6: "FK_ETIMEOUT", 7: "FK_ESTATE", 8: "FK_ENEGATIVE",
                9: "FK_EBOUNDS"}


class fk_grid_desc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("nv1", C.c_int32), ("nv2", C.c_int32),
                ("precision", C.c_int32), ("h_max", C.c_double), ("v1_min", C.c_double),
                ("v1_max", C.c_double), ("v2_min", C.c_double), ("v2_max", C.c_double),
                ("dt", C.c_double), ("cfl", C.c_double), ("history_capacity", C.c_int64),
                ("device", C.c_int32), ("reserved", C.c_int32)]


class fk_mlp_desc(C.Structure):
    _fields_ = [("n_in", C.c_int32), ("width", C.c_int32), ("depth", C.c_int32),
                ("n_out", C.c_int32), ("max_batch", C.c_int32), ("device", C.c_int32)]


class FkError(RuntimeError):
    def __init__(self, status, what, message):
        self.status = status
        super().__init__("%s: %s (%s)" % (what, STATUS_NAMES.get(status, status), message))


_lib = None


def library_path() -> str:
    """Path of the library load() takes (the FK_LIBRARY variant)."""
    return _build.LIBS.get(os.environ.get("FK_LIBRARY", "release") or "release", _build.LIB)


def load(build_if_missing: bool = True):
    """Load ``libflashkin.so`` (building it first if it is missing or stale
    and nvcc is available); with FK_LIBRARY=bounds in the environment, the
    debug-bounds build ``libflashkin_bounds.so`` instead.  Raises if it
    cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    variant = os.environ.get("FK_LIBRARY", "release") or "release"
    if variant not in _build.LIBS:
        raise ImportError("FK_LIBRARY must be one of %s" % sorted(_build.LIBS))
    path = _build.LIBS[variant]
    if build_if_missing and (not os.path.exists(path) or _build.stale(variant)):
        _build.build(variant=variant)
    if not os.path.exists(path):
        raise ImportError("%s is not built; run paper_2303_14119_gb300._build.build()"
                          % os.path.basename(path))
    lib = C.CDLL(path)
    P, D, I, I64 = C.c_void_p, C.c_double, C.c_int, C.c_int64
    dp = C.POINTER(C.c_double)
    fp = C.POINTER(C.c_float)
    i64p = C.POINTER(C.c_int64)
    sig = {
        "fk_create_grid": [C.POINTER(fk_grid_desc), P, C.POINTER(P)],
        "fk_destroy_grid": [P],
        "fk_set_fields": [P, D, I, D],
        "fk_set_see": [P, D, D, D, D, I],
        "fk_set_source": [P, D, D, D, D],
        "fk_set_convergence": [P, I64, D],
        "fk_fowler_nordheim": [D, D, dp, dp],
        "fk_set_collisions": [P, D, D, I],
        "fk_set_reflection": [P, D],
        "fk_set_scheme": [P, I],
        "fk_get_f32": [P, fp],
        "fk_set_f32": [P, fp],
        "fk_get_state": [P, P, C.POINTER(C.c_size_t)],
        "fk_set_state": [P, P, C.c_size_t],
        "fk_set_source_fn": [P, D, D, D, D, D],
        "fk_step": [P, I64],
        "fk_sync": [P],
        "fk_moments": [P, dp, dp, dp, dp],
        "fk_surface_charge": [P, dp],
        "fk_history": [P, dp, I64, i64p],
        "fk_ledger": [P, dp],
        "fk_step_count": [P, i64p, i64p],
        "fk_get_f": [P, dp],
        "fk_set_f": [P, dp],
        "fk_set_surface_charge": [P, D],
        "fk_grid_info": [P, dp],
        "fk_set_kernel_timing": [P, I],
        "fk_set_tile_rows": [P, C.c_int32],
        "fk_kernel_timing": [P, i64p, dp],
        "fk_batch_create": [C.POINTER(P), C.c_int32, P, C.POINTER(P)],
        "fk_batch_destroy": [P],
        "fk_batch_step": [P, I64],
        "fk_batch_sync": [P, C.POINTER(C.c_int32)],
        "fk_batch_autotune": [P, C.c_int32, i64p],
        "fk_batch_autotune_tiles": [P, C.c_int32, i64p],
        "fk_batch_get_chunks": [P, C.POINTER(C.c_int32)],
        "fk_batch_set_chunks": [P, C.POINTER(C.c_int32)],
        "fk_batch_info": [P, dp],
        "fk_batch_scalars": [P, dp, i64p, i64p, C.POINTER(C.c_int32)],
        "fk_batch_moments": [P, dp, dp, dp, dp, dp],
        "fk_batch_moments_enqueue": [P, C.c_int32],
        "fk_batch_moments_collect": [P, C.c_int32, dp, dp, dp, dp, dp],
        "fk_batch_set_kernel_timing": [P, I],
        "fk_batch_kernel_timing": [P, i64p, dp],
        "fk_gemm_bf16_tn": [P, I64, P, I64, P, I64, C.c_int32, C.c_int32, C.c_int32, P, P],
        "fk_mlp_create": [C.POINTER(fk_mlp_desc), P, C.POINTER(P)],
        "fk_mlp_destroy": [P],
        "fk_mlp_param_count": [P, i64p],
        "fk_mlp_set_params": [P, fp],
        "fk_mlp_get_params": [P, fp],
        "fk_mlp_forward": [P, fp, I64, fp],
        "fk_mlp_loss_grad": [P, fp, fp, fp, I64, dp, fp],
        "fk_mlp_train": [P, fp, fp, fp, I64, C.c_int32, C.c_int32, C.c_float, C.c_uint64, dp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.restype = C.c_int
        fn.argtypes = args
    lib.fk_last_error.restype = C.c_char_p
    lib.fk_last_error.argtypes = [P]
    lib.fk_batch_last_error.restype = C.c_char_p
    lib.fk_batch_last_error.argtypes = [P]
    lib.fk_mlp_last_error.restype = C.c_char_p
    lib.fk_mlp_last_error.argtypes = [P]
    _lib = lib
    return lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(status, what, handle=None):
    if status != FK_OK:
        msg = load().fk_last_error(handle).decode(errors="replace")
        raise FkError(status, what, msg)


def _f64(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != n:
        raise ValueError("expected %d elements, got %d" % (n, a.size))
    return a


# --- the C entry points, one Python function each --------------------------
def fk_create_grid(nx, nv1, nv2, h_max, v1_min, v1_max, v2_min, v2_max, dt=0.0, cfl=0.4,
                   precision=FK_F64, history_capacity=0, device=0, stream=None):
    d = fk_grid_desc(int(nx), int(nv1), int(nv2), int(precision), float(h_max), float(v1_min),
                     float(v1_max), float(v2_min), float(v2_max), float(dt), float(cfl),
                     int(history_capacity), int(device), 0)
    h = C.c_void_p()
    st = load().fk_create_grid(C.byref(d), C.c_void_p(stream) if stream else None, C.byref(h))
    _check(st, "fk_create_grid")
    return h.value


def fk_destroy_grid(g):
    _check(load().fk_destroy_grid(g), "fk_destroy_grid", g)


def fk_set_fields(g, Ey, self_consistent=True, Ex_external=0.0):
    _check(load().fk_set_fields(g, float(Ey), int(bool(self_consistent)), float(Ex_external)),
           "fk_set_fields", g)


def fk_set_see(g, delta_max, A_max_eV, k_s=1.0, T_se_eV=2.0, enabled=True):
    _check(load().fk_set_see(g, float(delta_max), float(A_max_eV), float(k_s), float(T_se_eV),
                             int(bool(enabled))), "fk_set_see", g)


def fk_set_source(g, J, x_lo, x_hi, T_fe_eV):
    _check(load().fk_set_source(g, float(J), float(x_lo), float(x_hi), float(T_fe_eV)),
           "fk_set_source", g)


def fk_fowler_nordheim(E, phi_V):
    """(ln J, J) of Eq. 6 in A/m^2."""
    lj, j = np.empty(1), np.empty(1)
    _check(load().fk_fowler_nordheim(float(E), float(phi_V), _dp(lj), _dp(j)),
           "fk_fowler_nordheim")
    return float(lj[0]), float(j[0])


def fk_set_source_fn(g, E_ctj, phi_V, x_lo, x_hi, T_fe_eV):
    _check(load().fk_set_source_fn(g, float(E_ctj), float(phi_V), float(x_lo), float(x_hi),
                                   float(T_fe_eV)), "fk_set_source_fn", g)


def fk_set_collisions(g, T_e_eV=2.0, ln_lambda=10.0, enabled=True):
    _check(load().fk_set_collisions(g, float(T_e_eV), float(ln_lambda), int(bool(enabled))),
           "fk_set_collisions", g)


def fk_set_reflection(g, R_f):
    _check(load().fk_set_reflection(g, float(R_f)), "fk_set_reflection", g)


def fk_get_state(g):
    """The grid's checkpoint as bytes."""
    n = C.c_size_t(0)
    _check(load().fk_get_state(g, None, C.byref(n)), "fk_get_state", g)
    buf = (C.c_ubyte * n.value)()
    _check(load().fk_get_state(g, buf, C.byref(n)), "fk_get_state", g)
    return bytes(buf)


def fk_set_state(g, state):
    buf = (C.c_ubyte * len(state)).from_buffer_copy(state)
    _check(load().fk_set_state(g, buf, len(state)), "fk_set_state", g)


def fk_set_scheme(g, scheme):
    _check(load().fk_set_scheme(g, int(scheme)), "fk_set_scheme", g)


def fk_set_convergence(g, window, rel_tol):
    _check(load().fk_set_convergence(g, int(window), float(rel_tol)), "fk_set_convergence", g)


def fk_step(g, n=1):
    _check(load().fk_step(g, int(n)), "fk_step", g)


def fk_step_status(g, n=1):
    """fk_step returning the raw status instead of raising."""
    return load().fk_step(g, int(n))


def fk_sync(g):
    _check(load().fk_sync(g), "fk_sync", g)


def fk_sync_status(g):
    return load().fk_sync(g)


def fk_moments(g, nx, n_e=None, Ex=None):
    n_e = np.empty(nx) if n_e is None else n_e
    Ex = np.empty(nx) if Ex is None else Ex
    gpe = np.empty(1)
    gsee = np.empty(1)
    _check(load().fk_moments(g, _dp(n_e), _dp(Ex), _dp(gpe), _dp(gsee)), "fk_moments", g)
    return n_e, Ex, float(gpe[0]), float(gsee[0])


def fk_surface_charge(g):
    s = np.empty(1)
    _check(load().fk_surface_charge(g, _dp(s)), "fk_surface_charge", g)
    return float(s[0])


def fk_history(g, max_rows):
    out = np.empty((int(max_rows), FK_HISTORY_COLS))
    rows = C.c_int64()
    _check(load().fk_history(g, _dp(out), int(max_rows), C.byref(rows)), "fk_history", g)
    return out[: rows.value]


def fk_ledger(g):
    out = np.empty(FK_LEDGER_LEN)
    _check(load().fk_ledger(g, _dp(out)), "fk_ledger", g)
    keys = ["N", "N0", "emit", "pe", "vac", "lv", "inj", "sigma0", "see"]
    return dict(zip(keys, out.tolist()))


def fk_step_count(g):
    s, sat = C.c_int64(), C.c_int64()
    _check(load().fk_step_count(g, C.byref(s), C.byref(sat)), "fk_step_count", g)
    return s.value, sat.value


def fk_get_f(g, shape, out=None):
    n = int(np.prod(shape))
    out = np.empty(shape, dtype=np.float64) if out is None else out
    if out.dtype != np.float64 or out.size != n or not out.flags.c_contiguous:
        raise ValueError("out must be a contiguous FP64 array of %d elements" % n)
    _check(load().fk_get_f(g, _dp(out)), "fk_get_f", g)
    return out


def fk_set_f(g, f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    _check(load().fk_set_f(g, _dp(f)), "fk_set_f", g)


def fk_get_f32(g, shape, out=None):
    n = int(np.prod(shape))
    out = np.empty(shape, dtype=np.float32) if out is None else out
    if out.dtype != np.float32 or out.size != n or not out.flags.c_contiguous:
        raise ValueError("out must be a contiguous FP32 array of %d elements" % n)
    _check(load().fk_get_f32(g, out.ctypes.data_as(C.POINTER(C.c_float))), "fk_get_f32", g)
    return out


def fk_set_f32(g, f):
    f = np.ascontiguousarray(f, dtype=np.float32)
    _check(load().fk_set_f32(g, f.ctypes.data_as(C.POINTER(C.c_float))), "fk_set_f32", g)


def fk_set_surface_charge(g, sigma):
    _check(load().fk_set_surface_charge(g, float(sigma)), "fk_set_surface_charge", g)


FK_INFO_LEN = 13


def fk_grid_info(g):
    out = np.empty(FK_INFO_LEN)
    _check(load().fk_grid_info(g, _dp(out)), "fk_grid_info", g)
    return dict(dx=out[0], dv1=out[1], dv2=out[2], dt=out[3], c2=out[4], cx_max=out[5],
                kernel="stream" if out[6] else "direct", n_tiles=int(out[7]),
                n_chunks=int(out[8]), chunk_len=int(out[9]), units_per_cta=int(out[10]),
                tile_rows=int(out[11]), tile_cap=int(out[12]))


def fk_set_tile_rows(g, max_rows):
    _check(load().fk_set_tile_rows(g, int(max_rows)), "fk_set_tile_rows", g)


def fk_set_kernel_timing(g, enabled):
    _check(load().fk_set_kernel_timing(g, int(bool(enabled))), "fk_set_kernel_timing", g)


def fk_kernel_timing(g):
    n = C.c_int64()
    ms = np.empty(1)
    _check(load().fk_kernel_timing(g, C.byref(n), _dp(ms)), "fk_kernel_timing", g)
    return n.value, float(ms[0])


def fk_last_error(g=None):
    return load().fk_last_error(g).decode(errors="replace")


class Grid:
    """Owning handle around one ``fk_grid``; methods call the entry points
    above with the grid's shape filled in."""

    def __init__(self, nx, nv1, nv2, h_max, v1_min, v1_max, v2_min, v2_max, dt=0.0, cfl=0.4,
                 precision=FK_F64, history_capacity=0, device=0, stream=None):
        self.h = fk_create_grid(nx, nv1, nv2, h_max, v1_min, v1_max, v2_min, v2_max, dt, cfl,
                                precision, history_capacity, device, stream)
        self.shape = (int(nx), int(nv1), int(nv2))
        self.precision = precision

    def close(self):
        if getattr(self, "h", None):
            fk_destroy_grid(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_fields(self, Ey, self_consistent=True, Ex_external=0.0):
        fk_set_fields(self.h, Ey, self_consistent, Ex_external)

    def set_see(self, delta_max, A_max_eV, k_s=1.0, T_se_eV=2.0, enabled=True):
        fk_set_see(self.h, delta_max, A_max_eV, k_s, T_se_eV, enabled)

    def set_source(self, J, x_lo, x_hi, T_fe_eV):
        fk_set_source(self.h, J, x_lo, x_hi, T_fe_eV)

    def set_source_fn(self, E_ctj, phi_V, x_lo, x_hi, T_fe_eV):
        fk_set_source_fn(self.h, E_ctj, phi_V, x_lo, x_hi, T_fe_eV)

    def set_collisions(self, T_e_eV=2.0, ln_lambda=10.0, enabled=True):
        fk_set_collisions(self.h, T_e_eV, ln_lambda, enabled)

    def set_reflection(self, R_f):
        fk_set_reflection(self.h, R_f)

    def checkpoint(self):
        return fk_get_state(self.h)

    def restore(self, state):
        fk_set_state(self.h, state)

    def set_scheme(self, scheme):
        fk_set_scheme(self.h, scheme)

    def set_convergence(self, window, rel_tol):
        fk_set_convergence(self.h, window, rel_tol)

    def step(self, n=1):
        fk_step(self.h, n)

    def sync(self):
        fk_sync(self.h)

    def moments(self):
        return fk_moments(self.h, self.shape[0])

    def surface_charge(self):
        return fk_surface_charge(self.h)

    def history(self, max_rows):
        return fk_history(self.h, max_rows)

    def ledger(self):
        return fk_ledger(self.h)

    def step_count(self):
        return fk_step_count(self.h)

    def get_f(self, out=None):
        return fk_get_f(self.h, self.shape, out)

    def set_f(self, f):
        fk_set_f(self.h, f)

    def get_f32(self, out=None):
        return fk_get_f32(self.h, self.shape, out)

    def set_f32(self, f):
        fk_set_f32(self.h, f)

    def set_state(self, f, sigma):
        fk_set_f(self.h, f)
        fk_set_surface_charge(self.h, sigma)

    def set_surface_charge(self, sigma):
        fk_set_surface_charge(self.h, sigma)

    def info(self):
        return fk_grid_info(self.h)

    def set_kernel_timing(self, enabled):
        fk_set_kernel_timing(self.h, enabled)

    def set_tile_rows(self, max_rows):
        fk_set_tile_rows(self.h, max_rows)

    def kernel_timing(self):
        return fk_kernel_timing(self.h)


# --- tensor-core dense layer (include/fk_mlp.h) ---------------------------
def fk_gemm_bf16_tn(A_ptr, lda, B_ptr, ldb, C_ptr, ldc, M, N, K, err_ptr, stream=None):
    """C = A * B^T on the tensor cores; every pointer a raw device address
    (e.g. ``tensor.data_ptr()``), A and B bf16, C FP32, err an int32."""
    _check(load().fk_gemm_bf16_tn(C.c_void_p(A_ptr), int(lda), C.c_void_p(B_ptr), int(ldb),
                                  C.c_void_p(C_ptr), int(ldc), int(M), int(N), int(K),
                                  C.c_void_p(err_ptr), C.c_void_p(stream) if stream else None),
           "fk_gemm_bf16_tn")


# --- the surrogate network (include/fk_mlp.h) ------------------------------
def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _f32(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if n is not None and a.size != n:
        raise ValueError("expected %d elements, got %d" % (n, a.size))
    return a


def _mcheck(status, what, handle=None):
    if status != FK_OK:
        msg = load().fk_mlp_last_error(handle).decode(errors="replace")
        raise FkError(status, what, msg)


def fk_mlp_create(n_in, width, depth, n_out, max_batch, device=0, stream=None):
    d = fk_mlp_desc(int(n_in), int(width), int(depth), int(n_out), int(max_batch), int(device))
    h = C.c_void_p()
    st = load().fk_mlp_create(C.byref(d), C.c_void_p(stream) if stream else None, C.byref(h))
    _mcheck(st, "fk_mlp_create")
    return h.value


def fk_mlp_destroy(h):
    _mcheck(load().fk_mlp_destroy(h), "fk_mlp_destroy", h)


def fk_mlp_param_count(h):
    n = C.c_int64()
    _mcheck(load().fk_mlp_param_count(h, C.byref(n)), "fk_mlp_param_count", h)
    return n.value


def fk_mlp_set_params(h, params):
    p = _f32(params, fk_mlp_param_count(h))
    _mcheck(load().fk_mlp_set_params(h, _fp(p)), "fk_mlp_set_params", h)


def fk_mlp_get_params(h):
    p = np.empty(fk_mlp_param_count(h), dtype=np.float32)
    _mcheck(load().fk_mlp_get_params(h, _fp(p)), "fk_mlp_get_params", h)
    return p


def fk_mlp_forward(h, x, n_out):
    x = _f32(x)
    n = x.shape[0]
    y = np.empty((n, n_out), dtype=np.float32)
    _mcheck(load().fk_mlp_forward(h, _fp(x), int(n), _fp(y)), "fk_mlp_forward", h)
    return y


def fk_mlp_loss_grad(h, x, t, w=None, grad=True):
    x, t = _f32(x), _f32(t)
    wv = _f32(w) if w is not None else None
    loss = np.empty(1)
    g = np.empty(fk_mlp_param_count(h), dtype=np.float32) if grad else None
    _mcheck(load().fk_mlp_loss_grad(h, _fp(x), _fp(t), _fp(wv) if wv is not None else None,
                                    int(x.shape[0]), _dp(loss), _fp(g) if grad else None),
            "fk_mlp_loss_grad", h)
    return float(loss[0]), g


def fk_mlp_train(h, x, t, w=None, batch=256, epochs=1, lr=1e-3, seed=0):
    x, t = _f32(x), _f32(t)
    wv = _f32(w) if w is not None else None
    el = np.empty(max(int(epochs), 1))
    _mcheck(load().fk_mlp_train(h, _fp(x), _fp(t), _fp(wv) if wv is not None else None,
                                int(x.shape[0]), int(batch), int(epochs), float(lr),
                                int(seed) & 0xFFFFFFFFFFFFFFFF, _dp(el)), "fk_mlp_train", h)
    return el[:int(epochs)]


def fk_mlp_last_error(h=None):
    return load().fk_mlp_last_error(h).decode(errors="replace")


class Mlp:
    """Owning handle around one ``fk_mlp``."""

    def __init__(self, n_in, width, depth, n_out, max_batch, device=0, stream=None):
        self.h = fk_mlp_create(n_in, width, depth, n_out, max_batch, device, stream)
        self.n_in, self.width, self.depth, self.n_out = n_in, width, depth, n_out

    def close(self):
        if getattr(self, "h", None):
            fk_mlp_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def param_count(self):
        return fk_mlp_param_count(self.h)

    def set_params(self, p):
        fk_mlp_set_params(self.h, p)

    def get_params(self):
        return fk_mlp_get_params(self.h)

    def forward(self, x):
        return fk_mlp_forward(self.h, x, self.n_out)

    def loss_grad(self, x, t, w=None, grad=True):
        return fk_mlp_loss_grad(self.h, x, t, w, grad)

    def train(self, x, t, w=None, batch=256, epochs=1, lr=1e-3, seed=0):
        return fk_mlp_train(self.h, x, t, w, batch, epochs, lr, seed)


# --- batches ---------------------------------------------------------------
FK_BATCH_INFO_LEN = 10


def _bcheck(status, what, handle=None):
    if status != FK_OK:
        msg = load().fk_batch_last_error(handle).decode(errors="replace")
        raise FkError(status, what, msg)


def fk_batch_create(grids, stream=None):
    """grids: sequence of grid handles (ints from fk_create_grid)."""
    n = len(grids)
    arr = (C.c_void_p * max(n, 1))(*[C.c_void_p(g) for g in grids])
    h = C.c_void_p()
    st = load().fk_batch_create(arr, int(n), C.c_void_p(stream) if stream else None, C.byref(h))
    _bcheck(st, "fk_batch_create")
    return h.value


def fk_batch_destroy(b):
    _bcheck(load().fk_batch_destroy(b), "fk_batch_destroy", b)


def fk_batch_step(b, n=1):
    _bcheck(load().fk_batch_step(b, int(n)), "fk_batch_step", b)


def fk_batch_sync(b, n):
    """Per-grid statuses (list of ints); never raises for a grid's sticky
    device error (the list reports it)."""
    out = (C.c_int32 * n)()
    st = load().fk_batch_sync(b, out)
    if st in (FK_EINVAL, FK_ECUDA, FK_ENOMEM):
        _bcheck(st, "fk_batch_sync", b)
    return list(out)


def fk_batch_scalars(b, n):
    """(sigma, step, sat_step, status) arrays of the batch's n grids."""
    sig = np.empty(n)
    st = np.empty(n, dtype=np.int64)
    sat = np.empty(n, dtype=np.int64)
    status = np.empty(n, dtype=np.int32)
    _bcheck(load().fk_batch_scalars(b, _dp(sig), st.ctypes.data_as(C.POINTER(C.c_int64)),
                                    sat.ctypes.data_as(C.POINTER(C.c_int64)),
                                    status.ctypes.data_as(C.POINTER(C.c_int32))),
            "fk_batch_scalars", b)
    return sig, st, sat, status


def fk_batch_moments(b, n, n_e=None, Ex=None, sigma=None, gamma_pe=None, gamma_see=None):
    """Every grid's sigma, Gamma_pe, Gamma_see (arrays of n) and n_e, E_x
    (concatenated in batch order) with one synchronisation; output arrays
    may be passed in (FP64, C-contiguous) to avoid allocation."""
    sigma = np.empty(n) if sigma is None else sigma
    gamma_pe = np.empty(n) if gamma_pe is None else gamma_pe
    gamma_see = np.empty(n) if gamma_see is None else gamma_see
    _bcheck(load().fk_batch_moments(b, _dp(sigma), _dp(gamma_pe), _dp(gamma_see),
                                    _dp(n_e) if n_e is not None else None,
                                    _dp(Ex) if Ex is not None else None),
            "fk_batch_moments", b)
    return sigma, gamma_pe, gamma_see, n_e, Ex


def fk_batch_moments_enqueue(b, slot):
    _bcheck(load().fk_batch_moments_enqueue(b, int(slot)), "fk_batch_moments_enqueue", b)


def fk_batch_moments_collect(b, n, slot, n_e=None, Ex=None, sigma=None, gamma_pe=None,
                             gamma_see=None):
    """The moments queued in `slot` by fk_batch_moments_enqueue (waits for
    those copies only); arrays as fk_batch_moments."""
    sigma = np.empty(n) if sigma is None else sigma
    gamma_pe = np.empty(n) if gamma_pe is None else gamma_pe
    gamma_see = np.empty(n) if gamma_see is None else gamma_see
    _bcheck(load().fk_batch_moments_collect(b, int(slot), _dp(sigma), _dp(gamma_pe),
                                            _dp(gamma_see),
                                            _dp(n_e) if n_e is not None else None,
                                            _dp(Ex) if Ex is not None else None),
            "fk_batch_moments_collect", b)
    return sigma, gamma_pe, gamma_see, n_e, Ex


def fk_batch_autotune(b, steps_per_trial=2):
    taken = C.c_int64()
    _bcheck(load().fk_batch_autotune(b, int(steps_per_trial), C.byref(taken)),
            "fk_batch_autotune", b)
    return taken.value


def fk_batch_autotune_tiles(b, steps_per_trial=2):
    taken = C.c_int64()
    _bcheck(load().fk_batch_autotune_tiles(b, int(steps_per_trial), C.byref(taken)),
            "fk_batch_autotune_tiles", b)
    return taken.value


def fk_batch_get_chunks(b, n):
    out = (C.c_int32 * n)()
    _bcheck(load().fk_batch_get_chunks(b, out), "fk_batch_get_chunks", b)
    return list(out)


def fk_batch_set_chunks(b, chunk_len):
    arr = (C.c_int32 * len(chunk_len))(*[int(c) for c in chunk_len])
    _bcheck(load().fk_batch_set_chunks(b, arr), "fk_batch_set_chunks", b)


def fk_batch_info(b):
    out = np.empty(FK_BATCH_INFO_LEN)
    _bcheck(load().fk_batch_info(b, _dp(out)), "fk_batch_info", b)
    return dict(grids=int(out[0]), units=int(out[1]), finalize_ctas=int(out[2]),
                smem_bytes=int(out[3]), ctas_per_sm=int(out[4]), cells=float(out[5]),
                buckets=int(out[6]), steps=int(out[7]), whole_ctas=int(out[8]),
                half_ctas=int(out[9]),
                step_launches=int(out[8] > 0) + int(out[9] > 0))


def fk_batch_set_kernel_timing(b, enabled):
    _bcheck(load().fk_batch_set_kernel_timing(b, int(bool(enabled))),
            "fk_batch_set_kernel_timing", b)


def fk_batch_kernel_timing(b):
    n = C.c_int64()
    ms = np.empty(1)
    _bcheck(load().fk_batch_kernel_timing(b, C.byref(n), _dp(ms)), "fk_batch_kernel_timing", b)
    return n.value, float(ms[0])


def fk_batch_last_error(b=None):
    return load().fk_batch_last_error(b).decode(errors="replace")


class Batch:
    """Owning handle around one ``fk_batch`` over existing ``Grid`` objects
    (which must outlive it)."""

    def __init__(self, grids, stream=None):
        self.grids = list(grids)
        self.h = fk_batch_create([g.h for g in self.grids], stream)

    def close(self):
        if getattr(self, "h", None):
            fk_batch_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def step(self, n=1):
        fk_batch_step(self.h, n)

    def sync(self):
        return fk_batch_sync(self.h, len(self.grids))

    def autotune(self, steps_per_trial=2, tiles=False):
        """Chunk lengths per size bucket (tiles: and the v1 tile rows of the
        whole-CTA buckets); returns the steps the trials took."""
        if tiles:
            return fk_batch_autotune_tiles(self.h, steps_per_trial)
        return fk_batch_autotune(self.h, steps_per_trial)

    def scalars(self):
        return fk_batch_scalars(self.h, len(self.grids))

    def moments(self, n_e=None, Ex=None, sigma=None, gamma_pe=None, gamma_see=None):
        """(sigma, gamma_pe, gamma_see, n_e, Ex) of every grid, one wait;
        n_e and Ex are filled only when given (length sum of nx)."""
        return fk_batch_moments(self.h, len(self.grids), n_e, Ex, sigma, gamma_pe, gamma_see)

    def moments_enqueue(self, slot):
        fk_batch_moments_enqueue(self.h, slot)

    def moments_collect(self, slot, n_e=None, Ex=None, sigma=None, gamma_pe=None,
                        gamma_see=None):
        return fk_batch_moments_collect(self.h, len(self.grids), slot, n_e, Ex, sigma,
                                        gamma_pe, gamma_see)

    def chunks(self):
        return fk_batch_get_chunks(self.h, len(self.grids))

    def set_chunks(self, chunk_len):
        fk_batch_set_chunks(self.h, chunk_len)

    def info(self):
        return fk_batch_info(self.h)

    def set_kernel_timing(self, enabled):
        fk_batch_set_kernel_timing(self.h, enabled)

    def kernel_timing(self):
        return fk_batch_kernel_timing(self.h)


FK_NOALLOC_MAX_PARTIALS = 131072
_noalloc_ready = False


def fk_density_moment_noalloc(f_dev_ptr, nx, nv1, nv2, dv1, dv2, n_e_dev_ptr, stream=None):
    """Density moment of a caller-held device array without any allocation
    by the library (see include/fk.h): f_dev_ptr and n_e_dev_ptr are raw
    device addresses, e.g. ``tensor.data_ptr()`` of CUDA tensors."""
    global _noalloc_ready
    lib = load()
    fn = lib.fk_density_moment_noalloc
    if not _noalloc_ready:
        fn.restype = C.c_int
        fn.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double,
                       C.c_void_p, C.c_void_p]
        _noalloc_ready = True
    _check(fn(C.c_void_p(f_dev_ptr), int(nx), int(nv1), int(nv2), float(dv1), float(dv2),
              C.c_void_p(n_e_dev_ptr), C.c_void_p(stream) if stream else None),
           "fk_density_moment_noalloc")
