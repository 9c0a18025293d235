"""Strang splitting (x over dt/2, velocity over dt, x over dt/2; reading
R14) on the GPU against the FP64 oracle, every term on; and the passes of
both split schemes on the streaming kernel and on the direct-load kernel."""
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


def setup(shape, prec, seed, dtnu=0.03, refl=0.2, scheme=fk.FK_SCHEME_STRANG):
    """Grid and oracle on the Strang scheme with fields, SEE, source,
    reflection and BGK collisions (ln Lambda chosen so that max_k dt nu_ee =
    dtnu for the initial state)."""
    nx, nv1, nv2 = shape
    g = fk.Grid(nx, nv1, nv2, H, -V1, V1, -V2, V2, cfl=0.4, precision=prec)
    o = oracle.Oracle(nx, nv1, nv2, H, -V1, V1, -V2, V2, cfl=0.4)
    info = o.info()
    a2 = 0.15 * info["dv2"] / info["dt"]
    emax = 0.2 * info["dv1"] / info["dt"] * ME / QE
    n_tot = 1.6 * emax * EPS0 / QE
    f0 = synth.random_f(shape, seed, 2 * n_tot / (H * 2 * V1 * 2 * V2))
    n_max = (f0.sum(axis=(1, 2)) * info["dv1"] * info["dv2"]).max()
    lnL = dtnu / (info["dt"] * oracle.nu_ee(n_max, T_E, 1.0))
    for x in (g, o):
        x.set_fields(-a2 * ME / QE, True, 0.0)
        x.set_see(3.0, 400.0, 1.0, 400.0)
        x.set_source(1e7, 0.2 * H, 0.7 * H, 300.0)
        x.set_collisions(T_E, lnL, True)
        x.set_reflection(refl)
        x.set_scheme(scheme)
        x.set_state(f0, 2 * EPS0 * emax * 0.8)
    return g, o


@pytest.mark.parametrize("prec,tol", [(fk.FK_F64, 1e-12), (fk.FK_F32, 5e-7)])
def test_strang_per_step_all_terms(prec, tol):
    shape = (18, 40, 34)
    g, o = setup(shape, prec, 71)
    for _ in range(3):
        o.set_state(g.get_f(), g.surface_charge())
        assert o.courant_sum() <= 1.0
        g.step(1)
        o.step(1)
        assert rel_l1(g.get_f(), o.get_f()) <= tol
        assert abs(g.surface_charge() - o.surface_charge()) <= tol * abs(o.surface_charge())
    g.close()


def test_strang_multi_step_ledger_and_switching():
    shape = (22, 32, 28)
    g, o = setup(shape, fk.FK_F64, 72, dtnu=0.02)
    g.step(70)  # two graph replays and six direct steps
    o.step(70)
    assert rel_l1(g.get_f(), o.get_f()) <= 1e-10
    assert abs(g.surface_charge() - o.surface_charge()) <= 1e-10 * abs(o.surface_charge())
    lg, lo = g.ledger(), o.ledger()
    for key in ("emit", "pe", "see", "vac", "lv", "inj"):
        assert abs(lg[key] - lo[key]) <= 1e-9 * abs(lo[key]), key
    with pytest.raises(fk.FkError) as e:
        fk.Batch([g])
    assert e.value.status == fk.FK_EINVAL
    # on to Lie, then back to the unsplit step
    for scheme in (fk.FK_SCHEME_LIE, fk.FK_SCHEME_UNSPLIT):
        for x in (g, o):
            x.set_scheme(scheme)
        o.set_state(g.get_f(), g.surface_charge())
        g.step(33)
        o.step(33)
        assert rel_l1(g.get_f(), o.get_f()) <= 1e-10
    g.close()


def test_strang_fp32_multi_step():
    shape = (20, 32, 26)
    g, o = setup(shape, fk.FK_F32, 73, dtnu=0.02)
    g.step(64)
    o.step(64)
    assert rel_l1(g.get_f(), o.get_f()) <= 1e-5
    assert abs(g.surface_charge() - o.surface_charge()) <= 1e-4 * abs(o.surface_charge())
    with pytest.raises(fk.FkError):
        g.set_scheme(3)
    g.close()


@pytest.mark.parametrize("scheme", [fk.FK_SCHEME_LIE, fk.FK_SCHEME_STRANG])
@pytest.mark.parametrize("prec,tol", [(fk.FK_F64, 1e-12), (fk.FK_F32, 5e-7)])
@pytest.mark.parametrize("shape", [(18, 40, 34), (12, 96, 72)])
def test_split_passes_on_both_step_kernels(scheme, prec, tol, shape, monkeypatch):
    """Each pass of a split step runs on the streaming kernel as the fused
    step with the other terms' coefficients zeroed (thin tiles two to a CTA
    on the first shape, whole-CTA tiles on the second), or on the
    direct-load kernel (the grids too wide for the streaming kernel, here
    forced): both match the oracle step by step, every term on, and each
    other over a graph replay."""
    finals = []
    for kernel in ("stream", "direct"):
        if kernel == "direct":
            monkeypatch.setenv("FK_STEP_KERNEL", "direct")
        else:
            monkeypatch.delenv("FK_STEP_KERNEL", raising=False)
        g, o = setup(shape, prec, 73, scheme=scheme)
        assert g.info()["kernel"] == kernel
        for _ in range(3):
            o.set_state(g.get_f(), g.surface_charge())
            g.step(1)
            o.step(1)
            assert rel_l1(g.get_f(), o.get_f()) <= tol, kernel
            assert abs(g.surface_charge() - o.surface_charge()) <= tol * abs(o.surface_charge())
        g.step(33)  # a graph replay of the passes
        finals.append((g.get_f(), g.surface_charge(), g.ledger()))
        g.close()
    (fs, ss, ls), (fd, sd, ld) = finals
    assert rel_l1(fs, fd) <= 40 * tol
    assert abs(ss - sd) <= 40 * tol * abs(sd)
    for key in ("emit", "pe", "see", "vac", "inj"):
        assert abs(ls[key] - ld[key]) <= 40 * tol * abs(ld[key]), key
