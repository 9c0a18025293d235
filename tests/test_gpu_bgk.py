"""Electron-electron BGK collisions (Eqs. 3-5) on the GPU against the FP64
oracle, with a Coulomb logarithm scaled up so that dt nu_ee is a few
percent and the term is far above rounding."""
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


H, V1, V2 = 20e-6, 6e7, 3e7
T_E = 2.0


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


def setup(shape, prec, seed, dtnu=0.04, c1f=0.2, c2f=0.15):
    """Grid and oracle with every term on and ln(Lambda) chosen so that
    max_k dt nu_ee = dtnu for the initial state."""
    nx, nv1, nv2 = shape
    g = fk.Grid(nx, nv1, nv2, H, -V1, V1, -V2, V2, cfl=0.4, precision=prec)
    o = oracle.Oracle(nx, nv1, nv2, H, -V1, V1, -V2, V2, cfl=0.4)
    info = o.info()
    a2 = c2f * info["dv2"] / info["dt"]
    emax = c1f * info["dv1"] / info["dt"] * ME / QE
    sigma = 2 * EPS0 * emax * 0.8
    n_tot = 1.6 * emax * EPS0 / QE
    amp = 2 * n_tot / (H * 2 * V1 * 2 * V2)
    f0 = synth.random_f(shape, seed, amp)
    n_max = (f0.sum(axis=(1, 2)) * info["dv1"] * info["dv2"]).max()
    lnL = dtnu / (info["dt"] * oracle.nu_ee(n_max, T_E, 1.0))
    for x in (g, o):
        x.set_fields(-a2 * ME / QE, True, 0.0)
        x.set_see(3.0, 400.0, 1.0, 400.0)
        x.set_source(1e7, 0.2 * H, 0.7 * H, 300.0)
        x.set_collisions(T_E, lnL, True)
    g.set_state(f0, sigma)
    o.set_state(f0, sigma)
    return g, o, lnL


@pytest.mark.parametrize("kernel", ["stream", "direct"])
@pytest.mark.parametrize("prec,tol", [(fk.FK_F64, 1e-12), (fk.FK_F32, 3e-7)])
def test_collisions_per_step(kernel, prec, tol, monkeypatch):
    if kernel == "direct":
        monkeypatch.setenv("FK_STEP_KERNEL", "direct")
    else:
        monkeypatch.delenv("FK_STEP_KERNEL", raising=False)
    shape = (19, 48, 44)
    g, o, _ = setup(shape, prec, 31)
    assert g.info()["kernel"] == kernel
    for _ in range(3):
        o.set_state(g.get_f(), g.surface_charge())
        assert o.courant_sum() <= 1.0
        g.step(1)
        o.step(1)
        assert rel_l1(g.get_f(), o.get_f()) <= tol
        assert abs(g.surface_charge() - o.surface_charge()) <= tol * abs(o.surface_charge())
    g.close()


def test_collisions_matter_and_keep_the_plane_densities():
    shape = (11, 32, 30)
    g, _, lnL = setup(shape, fk.FK_F64, 5)
    f0, s0 = g.get_f(), g.surface_charge()
    g.step(1)
    f_on = g.get_f()
    g.set_collisions(T_E, lnL, False)
    g.set_state(f0, s0)
    g.step(1)
    f_off = g.get_f()
    assert np.abs(f_on - f_off).max() > 1e-3 * np.abs(f_off).max()
    assert np.allclose(f_on.sum(axis=(1, 2)), f_off.sum(axis=(1, 2)), rtol=1e-12)
    g.close()


@pytest.mark.parametrize("prec,tol", [(fk.FK_F64, 1e-10), (fk.FK_F32, 1e-5)])
def test_collisions_multi_step_graph_path(prec, tol):
    shape = (24, 32, 32)
    g, o, _ = setup(shape, prec, 77, dtnu=0.02)
    g.step(100)  # three 32-step graph replays and four direct steps
    o.step(100)
    assert rel_l1(g.get_f(), o.get_f()) <= tol
    assert abs(g.surface_charge() - o.surface_charge()) <= 1e-4 * abs(o.surface_charge())
    g.close()


def test_batch_with_and_without_collisions_bitwise():
    shapes = [(16, 24, 24), (20, 32, 21), (12, 16, 16)]
    alone, batched = [], []
    for q, s in enumerate(shapes):
        ga, _, lnL = setup(s, fk.FK_F32, 40 + q)
        gb, _, _ = setup(s, fk.FK_F32, 40 + q)
        if q == 1:  # one grid without collisions
            for x in (ga, gb):
                x.set_collisions(T_E, lnL, False)
        alone.append(ga)
        batched.append(gb)
    with fk.Batch(batched) as b:
        b.step(37)
        assert b.sync() == [fk.FK_OK] * 3
    for g in alone:
        g.step(37)
    for ga, gb in zip(alone, batched):
        assert np.array_equal(ga.get_f(), gb.get_f())
        assert ga.surface_charge() == gb.surface_charge()


def test_switching_collisions_off_restores_the_plain_step():
    shape = (14, 24, 20)
    g, o, lnL = setup(shape, fk.FK_F64, 9)
    g.step(33)  # the graphs of the collision variant
    g.set_collisions(T_E, lnL, False)
    o.set_collisions(T_E, lnL, False)
    o.set_state(g.get_f(), g.surface_charge())
    g.step(40)
    o.step(40)
    assert rel_l1(g.get_f(), o.get_f()) <= 1e-10
    g.close()


# ---- electron reflection at the dielectric (R_f)
@pytest.mark.parametrize("kernel", ["stream", "direct"])
@pytest.mark.parametrize("prec,tol", [(fk.FK_F64, 1e-12), (fk.FK_F32, 3e-7)])
def test_reflection_per_step(kernel, prec, tol, monkeypatch):
    if kernel == "direct":
        monkeypatch.setenv("FK_STEP_KERNEL", "direct")
    else:
        monkeypatch.delenv("FK_STEP_KERNEL", raising=False)
    shape = (17, 40, 36)
    g, o, lnL = setup(shape, prec, 55)
    for x in (g, o):
        x.set_collisions(T_E, lnL, False)
        x.set_reflection(0.4)
    for _ in range(3):
        o.set_state(g.get_f(), g.surface_charge())
        g.step(1)
        o.step(1)
        assert rel_l1(g.get_f(), o.get_f()) <= tol
        assert abs(g.surface_charge() - o.surface_charge()) <= tol * abs(o.surface_charge())
    g.close()


def test_reflection_ledger_and_multi_step():
    shape = (20, 32, 24)
    g, o, lnL = setup(shape, fk.FK_F64, 56, dtnu=0.02)
    for x in (g, o):
        x.set_reflection(0.25)
    g.step(64)
    o.step(64)
    assert rel_l1(g.get_f(), o.get_f()) <= 1e-10
    lg, lo = g.ledger(), o.ledger()
    for key in ("emit", "pe", "see", "vac"):
        assert abs(lg[key] - lo[key]) <= 1e-9 * abs(lo[key]), key
    with pytest.raises(fk.FkError):
        fk.Grid(8, 8, 8, H, -5e7, V1, -V2, V2).set_reflection(0.5)
    g.close()


# ---- Lie splitting (x, then velocity)
@pytest.mark.parametrize("prec,tol", [(fk.FK_F64, 1e-12), (fk.FK_F32, 3e-7)])
def test_lie_per_step_all_terms(prec, tol):
    shape = (18, 40, 34)
    g, o, _ = setup(shape, prec, 61)
    for x in (g, o):
        x.set_reflection(0.2)
        x.set_scheme(fk.FK_SCHEME_LIE)
    for _ in range(3):
        o.set_state(g.get_f(), g.surface_charge())
        g.step(1)
        o.step(1)
        assert rel_l1(g.get_f(), o.get_f()) <= tol
        assert abs(g.surface_charge() - o.surface_charge()) <= tol * abs(o.surface_charge())
    g.close()


def test_lie_multi_step_ledger_and_switching_back():
    shape = (22, 32, 28)
    g, o, lnL = setup(shape, fk.FK_F64, 62, dtnu=0.02)
    for x in (g, o):
        x.set_scheme(fk.FK_SCHEME_LIE)
    g.step(70)  # two graph replays and six direct steps
    o.step(70)
    assert rel_l1(g.get_f(), o.get_f()) <= 1e-10
    lg, lo = g.ledger(), o.ledger()
    for key in ("emit", "pe", "see", "vac", "lv", "inj"):
        assert abs(lg[key] - lo[key]) <= 1e-9 * abs(lo[key]), key
    with pytest.raises(fk.FkError) as e:
        fk.Batch([g])
    assert e.value.status == fk.FK_EINVAL
    # back to the fused unsplit step
    for x in (g, o):
        x.set_scheme(fk.FK_SCHEME_UNSPLIT)
    o.set_state(g.get_f(), g.surface_charge())
    g.step(33)
    o.step(33)
    assert rel_l1(g.get_f(), o.get_f()) <= 1e-10
    g.close()
