"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle.

Tolerances (the stated numeric targets, and the bounds rounding gives them):
  FP64 path: relative L1 of f <= 1e-12 after one step from the same state;
  FP32 path: relative L1 of f <= 1e-5 after 1000 steps; surface charge 1e-4.
Scalars (sigma, fluxes, moments) of the FP64 path agree to 1e-12 relative
per step.  Multi-step FP64 runs are compared with the looser bound the
per-step rounding differences grow to (stated per test).
"""
import numpy as np
import pytest

import oracle
from oracle import EPS0, ME, QE
from paper_2303_14119_gb300 import fk, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fk.load()


def rel_l1(a, b):
    den = np.abs(b).sum()
    return np.abs(a - b).sum() / den if den > 0 else np.abs(a - b).sum()


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def edge_errors(a, b, floor=1e-6):
    """Max-relative errors of a against b on the parts of phase space a
    global norm could hide: the wall plane x = 0, and the velocity-edge
    rows (first and last v1 row, first and last v2 column) over all planes;
    each normalised by the largest |b| of that part, or by `floor` times the
    largest |b| of the whole state where the part holds less than that (a
    part the distribution has not reached holds only round-off, FP64
    values far below the smallest normal FP32)."""
    scale = floor * np.abs(b).max()
    parts = {"x=0 plane": (a[0], b[0]),
             "v1 edge rows": (a[:, [0, -1], :], b[:, [0, -1], :]),
             "v2 edge columns": (a[:, :, [0, -1]], b[:, :, [0, -1]])}
    out = {}
    for name, (pa, pb) in parts.items():
        den = max(np.abs(pb).max(), scale)
        out[name] = float(np.abs(pa - pb).max() / den) if den > 0 else float(np.abs(pa).max())
    return out


def check_edges(a, b, tol, what=""):
    errs = edge_errors(a, b)
    print("%s edge max-relative errors: %s" % (what, {k: "%.2e" % v for k, v in errs.items()}))
    for name, e in errs.items():
        assert e <= tol, (name, e)


# ----------------------------------------------------------------- set-ups
def make_pair(shape, prec=fk.FK_F64, h=20e-6, V1=6e7, V2=3e7, cfl=0.4, dt=0.0,
              history_capacity=0):
    nx, nv1, nv2 = shape
    g = fk.Grid(nx, nv1, nv2, h, -V1, V1, -V2, V2, dt=dt, cfl=cfl, precision=prec,
                history_capacity=history_capacity)
    o = oracle.Oracle(nx, nv1, nv2, h, -V1, V1, -V2, V2, dt=dt, cfl=cfl)
    return g, o


def both(g, o, name, *args):
    getattr(g, name)(*args)
    getattr(o, name)(*args)


def strong_physics(g, o, shape, seed=1, h=20e-6, V1=6e7, V2=3e7, c1f=0.25, c2f=0.2):
    """Every term active with large Courant numbers: E_x self-consistent and
    changing sign across x (|c_1| up to about c1f), large E_y (c_2 = c2f),
    SEE with a spread emission shape, a strong source.  Returns (f0, sigma0)."""
    nx, nv1, nv2 = shape
    info = o.info()
    a2 = c2f * info["dv2"] / info["dt"]
    both(g, o, "set_fields", -a2 * ME / QE, True, 0.0)
    both(g, o, "set_see", 3.0, 400.0, 1.0, 400.0)
    both(g, o, "set_source", 1e7, 0.2 * h, 0.7 * h, 300.0)
    emax = c1f * info["dv1"] / info["dt"] * ME / QE
    sigma = 2 * EPS0 * emax * 0.8
    n_tot = 1.6 * emax * EPS0 / QE
    amp = 2 * n_tot / (h * 2 * V1 * 2 * V2)
    f0 = synth.random_f(shape, seed, amp)
    return f0, sigma


def workload_physics(g, o, w):
    both(g, o, "set_fields", w["Ey"], True, 0.0)
    both(g, o, "set_see", w["delta_max"], w["A_max"], w["k_s"], w["T_se"])
    both(g, o, "set_source", w["J"], w["x_lo"], w["x_hi"], w["T_fe"])


def compare_state(g, o, tol_f, tol_s):
    fg, fo = g.get_f(), o.get_f()
    assert rel_l1(fg, fo) <= tol_f, rel_l1(fg, fo)
    assert rel(g.surface_charge(), o.surface_charge()) <= tol_s
    ne_g, ex_g, pe_g, see_g = g.moments()
    ne_o, ex_o, pe_o, see_o = o.moments()
    assert rel_l1(ne_g, ne_o) <= tol_s
    assert np.abs(ex_g - ex_o).max() <= tol_s * np.abs(ex_o).max()
    assert rel(pe_g, pe_o) <= tol_s
    assert rel(see_g, see_o) <= tol_s if see_o != 0 else see_g == 0


SHAPES = [(2, 2, 2), (4, 4, 5), (7, 9, 11), (16, 12, 10), (33, 200, 46), (12, 64, 81)]


# ----------------------------------------------------------------- FP64
@pytest.mark.parametrize("shape", SHAPES)
def test_fp64_per_step_parity_all_terms(shape):
    g, o = make_pair(shape)
    f0, sigma = strong_physics(g, o, shape)
    g.set_state(f0, sigma)
    for _ in range(4):
        o.set_state(g.get_f(), g.surface_charge())  # same starting state
        assert o.courant_sum() <= 1.0
        g.step(1)
        o.step(1)
        compare_state(g, o, 1e-12, 1e-12)
    g.close()


@pytest.mark.parametrize("kernel", ["stream", "direct"])
@pytest.mark.parametrize("prec,tol", [(fk.FK_F64, 1e-12), (fk.FK_F32, 2e-7)])
def test_both_step_kernels_per_step(kernel, prec, tol, monkeypatch):
    """The streaming kernel and the direct-load kernel against the oracle."""
    if kernel == "direct":
        monkeypatch.setenv("FK_STEP_KERNEL", "direct")
    else:
        monkeypatch.delenv("FK_STEP_KERNEL", raising=False)
    shape = (21, 70, 36)
    g, o = make_pair(shape, prec=prec)
    f0, sigma = strong_physics(g, o, shape, seed=12)
    g.set_state(f0, sigma)
    for _ in range(3):
        o.set_state(g.get_f(), g.surface_charge())
        g.step(1)
        o.step(1)
        assert rel_l1(g.get_f(), o.get_f()) <= tol
        assert rel(g.surface_charge(), o.surface_charge()) <= 1e-12
        assert rel(g.moments()[2], o.moments()[2]) <= 1e-12 if prec == fk.FK_F64 else True
    g.close()


def test_fp64_multi_step_parity_and_ledger():
    shape = (16, 12, 10)
    g, o = make_pair(shape)
    f0, sigma = strong_physics(g, o, shape, seed=3)
    g.set_state(f0, sigma)
    o.set_state(f0, sigma)
    g.step(60)
    o.step(60)
    compare_state(g, o, 1e-11, 1e-11)
    lg, lo = g.ledger(), o.ledger()
    for key in ("N", "N0", "pe", "vac", "lv", "inj", "see", "sigma0"):
        assert rel(lg[key], lo[key]) <= 1e-11, key
    assert rel(lg["emit"], lo["emit"]) <= 1e-11
    hg, ho = g.history(100), o.history(100)
    assert hg.shape == ho.shape == (61, 8)
    assert np.array_equal(hg[:, 0], ho[:, 0])
    for c in range(1, 8):
        assert np.all(np.abs(hg[:, c] - ho[:, c]) <= 1e-11 * np.abs(ho[:, c]).max() + 1e-300)
    # conservation on the device itself
    rhs = lg["emit"] - lg["pe"] - lg["vac"] - lg["lv"] + lg["inj"]
    scale = max(abs(v) for v in lg.values() if v)
    assert abs((lg["N"] - lg["N0"]) - rhs) < 1e-12 * scale
    g.close()


def test_small_workload_fp64_2000_steps():
    """64 x 48 x 48, E_y = -1e6 V/m, delta_max 3, A_max 400 eV, T_se 2 eV,
    J = 1 A/m^2 on [10, 15] um, f0 = 1e-6 relative noise, dt at CFL 0.4."""
    w = synth.WORKLOADS["small_64x48x48"]
    shape = (w["nx"], w["nv1"], w["nv2"])
    g, o = make_pair(shape, cfl=w["cfl"])
    workload_physics(g, o, w)
    f0 = synth.initial_f(shape, w["seed"], w["noise_rel"], w["J"], w["T_fe"])
    g.set_f(f0)
    o.set_state(f0, 0.0)
    g.step(w["steps"])
    o.step(w["steps"])
    compare_state(g, o, 1e-10, 1e-10)
    hg, ho = g.history(w["steps"] + 1), o.history(w["steps"] + 1)
    assert np.allclose(hg[:, 2:5], ho[:, 2:5], rtol=1e-10, atol=1e-10 * np.abs(ho[:, 2:5]).max())
    assert g.step_count()[0] == w["steps"]
    g.close()


def test_graph_replay_matches_single_steps_bitwise():
    shape = (20, 16, 12)
    g1, o = make_pair(shape)
    f0, sigma = strong_physics(g1, o, shape, seed=9)
    g2, _ = make_pair(shape)
    strong_physics(g2, o, shape, seed=9)
    g1.set_state(f0, sigma)
    g2.set_state(f0, sigma)
    g1.step(64 + 3)  # two graph replays + 3 single steps
    for _ in range(67):
        g2.step(1)
    assert np.array_equal(g1.get_f(), g2.get_f())
    assert g1.surface_charge() == g2.surface_charge()
    g1.close()
    g2.close()


def test_determinism_bitwise():
    shape = (33, 200, 46)
    outs = []
    for _ in range(2):
        g, o = make_pair(shape)
        f0, sigma = strong_physics(g, o, shape, seed=4)
        g.set_state(f0, sigma)
        g.step(40)
        outs.append((g.get_f(), g.surface_charge(), g.history(41)))
        g.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]
    assert np.array_equal(outs[0][2], outs[1][2])


def test_external_field_and_no_see():
    shape = (10, 8, 6)
    g, o = make_pair(shape)
    info = o.info()
    ex = -0.3 * info["dv1"] / info["dt"] * ME / QE
    both(g, o, "set_fields", -1e9, False, ex)
    both(g, o, "set_see", 3.0, 400.0, 1.0, 2.0, False)
    f0 = synth.random_f(shape, 2, 1.0)
    g.set_state(f0, 1e-6)
    o.set_state(f0, 1e-6)
    g.step(5)
    o.step(5)
    compare_state(g, o, 1e-12, 1e-12)
    assert g.moments()[3] == 0.0
    g.close()


def test_zero_state_stays_zero_without_source():
    g, o = make_pair((6, 6, 6))
    g.set_fields(-1e6)
    g.set_see(3.0, 400.0)
    g.step(10)
    assert not g.get_f().any()
    assert g.surface_charge() == 0.0
    g.close()


def test_cfl_violation_is_reported_and_state_frozen():
    shape = (8, 8, 8)
    g, o = make_pair(shape)
    f0 = synth.random_f(shape, 5, 1.0)
    g.set_state(f0, 0.0)
    info = o.info()
    a2 = 0.9 * info["dv2"] / info["dt"]  # c2 = 0.9, plus c_x up to 0.35
    g.set_fields(-a2 * ME / QE)
    assert fk.fk_step_status(g.h, 5) == fk.FK_OK  # enqueued; device refuses
    assert fk.fk_sync_status(g.h) == fk.FK_ECFL
    assert "unstable" in fk.fk_last_error(g.h)
    assert fk.fk_step_status(g.h, 1) == fk.FK_ECFL
    # state is the one before the refused steps
    g.set_fields(-1e3)
    assert g.step_count()[0] == 0
    assert np.array_equal(g.get_f(), f0)
    g.close()


def test_nonfinite_input_is_reported():
    shape = (6, 4, 4)
    g, _ = make_pair(shape)
    f0 = np.ones(shape)
    f0[2, 1, 1] = np.nan
    with pytest.raises(fk.FkError) as ei:
        g.set_f(f0)
    assert ei.value.status == fk.FK_ENUMERIC
    g.close()


# ----------------------------------------------------------------- FP32
def test_fp32_per_step_parity():
    shape = (33, 200, 46)
    g, o = make_pair(shape, prec=fk.FK_F32)
    f0, sigma = strong_physics(g, o, shape, seed=6)
    g.set_state(f0, sigma)
    o.set_state(g.get_f(), sigma)  # the FP32-rounded state
    g.step(1)
    o.step(1)
    assert rel_l1(g.get_f(), o.get_f()) <= 2e-7
    assert rel(g.surface_charge(), o.surface_charge()) <= 1e-12  # FP64 accumulation
    g.close()


def test_fp32_small_workload_1000_steps():
    w = synth.WORKLOADS["small_64x48x48"]
    shape = (w["nx"], w["nv1"], w["nv2"])
    g, o = make_pair(shape, prec=fk.FK_F32, cfl=w["cfl"])
    workload_physics(g, o, w)
    f0 = synth.initial_f(shape, w["seed"], w["noise_rel"], w["J"], w["T_fe"])
    g.set_f(f0)
    o.set_state(f0, 0.0)
    g.step(1000)
    o.step(1000)
    fg, fo = g.get_f(), o.get_f()
    assert rel_l1(fg, fo) <= 1e-5
    check_edges(fg, fo, 1e-4, "small workload FP32, 1000 steps:")
    assert rel(g.surface_charge(), o.surface_charge()) <= 1e-4
    _, _, pe_g, see_g = g.moments()
    _, _, pe_o, see_o = o.moments()
    assert rel(pe_g, pe_o) <= 1e-4 and rel(see_g, see_o) <= 1e-4
    g.close()


def test_fp32_strong_1000_steps():
    shape = (16, 24, 20)
    g, o = make_pair(shape, prec=fk.FK_F32)
    f0, sigma = strong_physics(g, o, shape, seed=8, c1f=0.05, c2f=0.2)  # stays within CFL
    g.set_state(f0, sigma)
    o.set_state(g.get_f(), sigma)
    g.step(1000)
    o.step(1000)
    fg, fo = g.get_f(), o.get_f()
    assert rel_l1(fg, fo) <= 1e-5
    check_edges(fg, fo, 1e-4, "strong state FP32, 1000 steps:")
    assert rel(g.surface_charge(), o.surface_charge()) <= 1e-4
    g.close()


# ----------------------------------------------------------------- full size
def test_full_size_fp64_one_step_parity():
    """1024 x 256 x 256 in the launch configuration the benchmark times:
    every cell of one step compared with the oracle from the same state."""
    w = synth.WORKLOADS["full_1024x256x256"]
    shape = (w["nx"], w["nv1"], w["nv2"])
    g, o = make_pair(shape, cfl=w["cfl"])
    f0, sigma = strong_physics(g, o, shape, seed=11)
    g.set_state(f0, sigma)
    g.step(3)
    o.set_state(g.get_f(), g.surface_charge())
    g.step(1)
    o.step(1)
    compare_state(g, o, 1e-12, 1e-12)
    g.close()


def test_full_size_fp32_against_fp64_gpu():
    """FP32 path against the FP64 path at 1024 x 256 x 256, 1000 steps of the
    workload physics from the same f0 (both on the GPU): the stated FP32
    bound (1e-5 relative L1 after 1000 steps), and the wall plane and the
    velocity-edge rows element by element."""
    w = synth.WORKLOADS["full_1024x256x256"]
    shape = (w["nx"], w["nv1"], w["nv2"])
    f0 = synth.initial_f(shape, w["seed"], w["noise_rel"], w["J"], w["T_fe"])
    res = []
    for prec in (fk.FK_F64, fk.FK_F32):
        g = fk.Grid(*shape, w["h_max"], -w["v1_span"], w["v1_span"], -w["v2_span"],
                    w["v2_span"], cfl=w["cfl"], precision=prec)
        g.set_fields(w["Ey"])
        g.set_see(w["delta_max"], w["A_max"], w["k_s"], w["T_se"])
        g.set_source(w["J"], w["x_lo"], w["x_hi"], w["T_fe"])
        g.set_f(f0)
        g.step(1000)
        res.append((g.get_f(), g.surface_charge(), g.ledger()))
        g.close()
    e = rel_l1(res[1][0], res[0][0])
    print("1024x256x256 FP32 vs FP64 after 1000 steps: rel L1 %.3e" % e)
    assert e <= 1e-5
    check_edges(res[1][0], res[0][0], 1e-4, "1024x256x256 FP32 vs FP64, 1000 steps:")
    assert rel(res[1][1], res[0][1]) <= 1e-4
    assert rel(res[1][2]["N"], res[0][2]["N"]) <= 1e-5


# ----------------------------------------------------------------- 2048 x 384 x 384
def test_large_fp32_against_fp64_gpu():
    """Mixed-precision workload 2048 x 384 x 384 (302 M cells), E_y = -2e6 V/m:
    FP32 f with FP64 accumulators against the FP64 path over the workload's
    10000 steps, both on the GPU from the same f0, compared after 1000 steps
    (the stated bound, 1e-5 relative L1) and after 10000 (the growth of the
    difference over the whole run; the same bound holds)."""
    w = synth.WORKLOADS["large_2048x384x384"]
    shape = (w["nx"], w["nv1"], w["nv2"])
    f0 = synth.initial_f(shape, w["seed"], w["noise_rel"], w["J"], w["T_fe"])
    grids = []
    for prec in (fk.FK_F64, fk.FK_F32):
        g = fk.Grid(*shape, w["h_max"], -w["v1_span"], w["v1_span"], -w["v2_span"],
                    w["v2_span"], cfl=w["cfl"], precision=prec, history_capacity=16384)
        g.set_fields(w["Ey"])
        g.set_see(w["delta_max"], w["A_max"], w["k_s"], w["T_se"])
        g.set_source(w["J"], w["x_lo"], w["x_hi"], w["T_fe"])
        g.set_f(f0)
        grids.append(g)
    del f0
    out = np.empty(shape)
    for steps in (1000, w["steps"]):
        for g in grids:
            g.step(steps - g.step_count()[0])
        f64 = grids[0].get_f()
        f32 = grids[1].get_f(out)
        e = rel_l1(f32, f64)
        print("2048x384x384 FP32 vs FP64 after %d steps: rel L1 %.3e, sigma %.3e" %
              (steps, e, rel(grids[1].surface_charge(), grids[0].surface_charge())))
        assert e <= 1e-5
        check_edges(f32, f64, 1e-4, "2048x384x384 after %d steps:" % steps)
        del f64
        assert rel(grids[1].surface_charge(), grids[0].surface_charge()) <= 1e-4
    h64, h32 = (g.history(w["steps"] + 1) for g in grids)
    for c in (3, 4, 6):  # Gamma_pe, Gamma_see, N histories
        assert np.abs(h32[:, c] - h64[:, c]).max() <= 1e-4 * np.abs(h64[:, c]).max()
    for g in grids:
        g.close()


def test_coarse_copy_fp32_against_oracle():
    """The 4x-coarsened copy of the mixed-precision workload, 512 x 96 x 96,
    FP32 path against the FP64 oracle (its threaded build) for 1000 steps."""
    import os
    w = synth.WORKLOADS["coarse_512x96x96"]
    shape = (w["nx"], w["nv1"], w["nv2"])
    g = fk.Grid(*shape, w["h_max"], -w["v1_span"], w["v1_span"], -w["v2_span"], w["v2_span"],
                cfl=w["cfl"], precision=fk.FK_F32)
    o = oracle.Oracle(*shape, w["h_max"], -w["v1_span"], w["v1_span"], -w["v2_span"],
                      w["v2_span"], cfl=w["cfl"], threads=os.cpu_count())
    workload_physics(g, o, w)
    f0 = synth.initial_f(shape, w["seed"], w["noise_rel"], w["J"], w["T_fe"])
    g.set_f(f0)
    o.set_state(f0, 0.0)
    g.step(1000)
    o.step(1000)
    fg, fo = g.get_f(), o.get_f()
    print("512x96x96 FP32 vs oracle after 1000 steps: rel L1 %.3e" % rel_l1(fg, fo))
    assert rel_l1(fg, fo) <= 1e-5
    check_edges(fg, fo, 1e-4, "512x96x96 FP32 vs oracle, 1000 steps:")
    assert rel(g.surface_charge(), o.surface_charge()) <= 1e-4
    g.close()


# ----------------------------------------------------------------- limits
@pytest.mark.parametrize("prec,tol", [(fk.FK_F64, 1e-12), (fk.FK_F32, 3e-7)])
def test_longest_x_range(prec, tol):
    """nx = 8192, the largest the ABI accepts: the finalize kernel runs its
    most blocks (64) and the Gauss-law prefix spans them all."""
    shape = (8192, 4, 8)
    g, o = make_pair(shape, prec=prec)
    f0, sigma = strong_physics(g, o, shape, seed=81)
    g.set_state(f0, sigma)
    for _ in range(2):
        o.set_state(g.get_f(), g.surface_charge())
        g.step(1)
        o.step(1)
        assert rel_l1(g.get_f(), o.get_f()) <= tol
        ne_g, ex_g, _, _ = g.moments()
        ne_o, ex_o, _, _ = o.moments()
        assert np.abs(ex_g - ex_o).max() <= 10 * tol * np.abs(ex_o).max()
    g.close()


@pytest.mark.parametrize("prec,tol", [(fk.FK_F64, 1e-12), (fk.FK_F32, 3e-7)])
def test_rows_too_wide_for_the_streaming_kernel(prec, tol):
    """v2 rows wider than one streaming tile (nv2 = 7300) fall back to the
    direct-load kernel, which must give the same step."""
    shape = (3, 4, 7300)
    g, o = make_pair(shape, prec=prec)
    assert g.info()["kernel"] == "direct"
    f0, sigma = strong_physics(g, o, shape, seed=82)
    g.set_state(f0, sigma)
    for _ in range(2):
        o.set_state(g.get_f(), g.surface_charge())
        g.step(1)
        o.step(1)
        assert rel_l1(g.get_f(), o.get_f()) <= tol
    g.close()
