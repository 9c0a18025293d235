"""The C-ABI library loads, exports every entry point include/fk.h declares,
and rejects invalid grids on the host before touching a GPU."""
import ctypes as C
import os
import re

import pytest

from paper_2303_14119_gb300 import fk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(fk_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ("fk_create_grid", "fk_destroy_grid", "fk_set_fields", "fk_set_see",
                     "fk_set_source", "fk_step", "fk_moments", "fk_surface_charge",
                     "fk_history", "fk_ledger", "fk_get_f", "fk_set_f", "fk_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = fk.load()
    missing = [n for n in declared_entry_points() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_constants_match_the_header():
    """Every integer #define of include/fk.h has the binding's value."""
    text = open(os.path.join(ROOT, "include", "fk.h")).read()
    defs = dict(re.findall(r"^#define\s+(FK_[A-Z0-9_]+)\s+(\d+)\s*$", text, flags=re.M))
    assert "FK_INFO_LEN" in defs and "FK_HISTORY_COLS" in defs
    for name, value in defs.items():
        if hasattr(fk, name):
            assert getattr(fk, name) == int(value), name


def _desc(**kw):
    d = dict(nx=8, nv1=6, nv2=6, precision=0, h_max=20e-6, v1_min=-6e7, v1_max=6e7,
             v2_min=-3e7, v2_max=3e7, dt=0.0, cfl=0.4, history_capacity=0, device=0, reserved=0)
    d.update(kw)
    return fk.fk_grid_desc(**d)


@pytest.mark.parametrize("bad", [dict(nx=1), dict(nv1=1), dict(nv2=0), dict(h_max=0.0),
                                 dict(v1_min=1.0, v1_max=1.0), dict(v2_min=2.0, v2_max=1.0),
                                 dict(dt=0.0, cfl=0.0), dict(precision=7),
                                 dict(history_capacity=-1), dict(h_max=float("nan"))])
def test_invalid_descriptions_rejected_on_host(bad):
    lib = fk.load()
    h = C.c_void_p()
    st = lib.fk_create_grid(C.byref(_desc(**bad)), None, C.byref(h))
    assert st == fk.FK_EINVAL
    assert h.value is None
    assert lib.fk_last_error(None)


def test_x_courant_above_one_rejected_on_host():
    lib = fk.load()
    h = C.c_void_p()
    st = lib.fk_create_grid(C.byref(_desc(dt=1e-12)), None, C.byref(h))
    assert st == fk.FK_ECFL


def test_null_arguments():
    lib = fk.load()
    assert lib.fk_create_grid(None, None, None) == fk.FK_EINVAL
    assert lib.fk_destroy_grid(None) == fk.FK_OK
    assert lib.fk_step(None, 1) == fk.FK_EINVAL
    assert lib.fk_sync(None) == fk.FK_EINVAL
    assert lib.fk_set_tile_rows(None, 16) == fk.FK_EINVAL


def test_batch_create_rejects_bad_arguments_on_host():
    lib = fk.load()
    h = C.c_void_p()
    assert lib.fk_batch_create(None, 1, None, C.byref(h)) == fk.FK_EINVAL
    arr = (C.c_void_p * 2)(None, None)
    assert lib.fk_batch_create(arr, 0, None, C.byref(h)) == fk.FK_EINVAL
    assert lib.fk_batch_create(arr, -3, None, C.byref(h)) == fk.FK_EINVAL
    assert lib.fk_batch_create(arr, 2, None, C.byref(h)) == fk.FK_EINVAL
    assert h.value is None
    assert "NULL" in lib.fk_batch_last_error(None).decode()


def test_batch_calls_reject_null_handles():
    lib = fk.load()
    n = C.c_int64()
    d = C.c_double()
    assert lib.fk_batch_step(None, 1) == fk.FK_EINVAL
    assert lib.fk_batch_sync(None, None) == fk.FK_EINVAL
    assert lib.fk_batch_autotune(None, 1, C.byref(n)) == fk.FK_EINVAL
    assert lib.fk_batch_autotune_tiles(None, 1, C.byref(n)) == fk.FK_EINVAL
    assert lib.fk_batch_get_chunks(None, None) == fk.FK_EINVAL
    assert lib.fk_batch_set_chunks(None, None) == fk.FK_EINVAL
    assert lib.fk_batch_info(None, C.byref(d)) == fk.FK_EINVAL
    assert lib.fk_batch_kernel_timing(None, C.byref(n), C.byref(d)) == fk.FK_EINVAL
    assert lib.fk_batch_destroy(None) == fk.FK_OK


def test_fowler_nordheim_host_function_matches_the_oracle():
    import math
    import oracle
    for E in (1e6, 5e6, 3e9, 1e10):
        for phi in (2.5, 4.08, 4.5):
            lj, j = fk.fk_fowler_nordheim(E, phi)
            ref = oracle.fn_log_current(E, phi)
            assert abs(lj - ref) <= 1e-12 * abs(ref)
            assert j == (math.exp(lj))
    assert fk.fk_fowler_nordheim(5e6, 4.08)[1] == 0.0
    lib = fk.load()
    import ctypes as Ct
    d = Ct.c_double()
    assert lib.fk_fowler_nordheim(0.0, 4.0, Ct.byref(d), None) == fk.FK_EINVAL
    assert lib.fk_fowler_nordheim(1e9, -1.0, None, None) == fk.FK_EINVAL


def test_debug_bounds_build_compiles_and_exports_every_symbol():
    """The FK_DEBUG_BOUNDS variant builds (nvcc cross-compiles without a GPU)
    and exports the same entry points; loading it makes no device call."""
    from paper_2303_14119_gb300 import _build
    path = _build.build(variant="bounds")
    lib = C.CDLL(path)
    missing = [n for n in declared_entry_points() if not hasattr(lib, n)]
    assert not missing, missing
