"""Half-CTA units of the streaming step kernel (two thin tiles per CTA, each
on 3 consumer warps and its own producer warp) against the FP64 oracle and
against the whole-CTA layout (FK_STREAM_HALF=0)."""
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


def layout(monkeypatch, half):
    if half:
        monkeypatch.delenv("FK_STREAM_HALF", raising=False)
    else:
        monkeypatch.setenv("FK_STREAM_HALF", "0")


def setup(shape, prec, seed, v1=(-V1, V1), refl=0.0, dtnu=0.03, with_oracle=True):
    """Grid (and oracle) with fields, SEE, source and BGK collisions on (ln
    Lambda chosen so that max_k dt nu_ee = dtnu for the initial state)."""
    nx, nv1, nv2 = shape
    g = fk.Grid(nx, nv1, nv2, H, v1[0], v1[1], -V2, V2, cfl=0.4, precision=prec)
    info = g.info()
    a2 = 0.15 * info["dv2"] / info["dt"]
    emax = 0.2 * info["dv1"] / info["dt"] * ME / QE
    n_tot = 1.6 * emax * EPS0 / QE
    f0 = synth.random_f(shape, seed, 2 * n_tot / (H * (v1[1] - v1[0]) * 2 * V2))
    n_max = (f0.sum(axis=(1, 2)) * info["dv1"] * info["dv2"]).max()
    lnL = dtnu / (info["dt"] * oracle.nu_ee(n_max, T_E, 1.0))
    xs = [g]
    o = None
    if with_oracle:
        o = oracle.Oracle(nx, nv1, nv2, H, v1[0], v1[1], -V2, V2, cfl=0.4)
        xs.append(o)
    for x in xs:
        x.set_fields(-a2 * ME / QE, True, 0.0)
        x.set_see(3.0, 400.0, 1.0, 400.0)
        x.set_source(1e7, 0.2 * H, 0.7 * H, 300.0)
        x.set_collisions(T_E, lnL, True)
        if refl:
            x.set_reflection(refl)
        x.set_state(f0, 2 * EPS0 * emax * 0.8)
    return g, o


@pytest.mark.parametrize("prec", [fk.FK_F64, fk.FK_F32])
def test_layout_choice_and_override(prec, monkeypatch):
    layout(monkeypatch, True)
    thin = fk.Grid(64, 48, 48, H, -V1, V1, -V2, V2, precision=prec)
    wide = fk.Grid(16, 256, 256, H, -V1, V1, -V2, V2, precision=prec)
    assert thin.info()["units_per_cta"] == 2
    assert thin.info()["n_tiles"] == 2  # one tile per sign of v1
    assert wide.info()["units_per_cta"] == 1
    layout(monkeypatch, False)
    assert fk.Grid(64, 48, 48, H, -V1, V1, -V2, V2, precision=prec).info()["units_per_cta"] == 1


@pytest.mark.parametrize("shape", [(64, 48, 48), (13, 31, 22), (40, 24, 21)])
@pytest.mark.parametrize("prec", [fk.FK_F64, fk.FK_F32])
def test_one_step_is_the_same_in_both_layouts(shape, prec, monkeypatch):
    """Per cell the update is the same arithmetic in both layouts, and the
    first step's fields come from the same moments: f^1 and sigma^1 agree
    bit for bit."""
    out = []
    for half in (True, False):
        layout(monkeypatch, half)
        g, _ = setup(shape, prec, 21, refl=0.3, with_oracle=False)
        assert g.info()["units_per_cta"] == (2 if half else 1)
        g.step(1)
        out.append((g.get_f(), g.surface_charge()))
        g.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


@pytest.mark.parametrize("half", [True, False])
@pytest.mark.parametrize("prec,tol", [(fk.FK_F64, 1e-12), (fk.FK_F32, 3e-7)])
def test_per_step_parity_all_terms(half, prec, tol, monkeypatch):
    layout(monkeypatch, half)
    shape = (23, 40, 30)  # ragged: 23 planes, 30 cells per row
    g, o = setup(shape, prec, 33, refl=0.25)
    assert g.info()["units_per_cta"] == (2 if half else 1)
    for _ in range(3):
        o.set_state(g.get_f(), g.surface_charge())
        assert o.courant_sum() <= 1.0
        g.step(1)
        o.step(1)
        assert rel_l1(g.get_f(), o.get_f()) <= tol
        assert abs(g.surface_charge() - o.surface_charge()) <= tol * abs(o.surface_charge())
    g.close()


@pytest.mark.parametrize("half", [True, False])
@pytest.mark.parametrize("prec,tol", [(fk.FK_F64, 1e-12), (fk.FK_F32, 3e-7)])
def test_halo_zero_row_then_bulk_copy_in_one_stage(half, prec, tol, monkeypatch):
    """Gauss's law makes E_x fall with x, so c_1 < 0 on the planes next to
    the wall and c_1 > 0 past the zero of E_x.  On a plane with c_1 < 0 the
    producer zero-fills the halo row after the last v1 tile (i1 = nv1); the
    same stage comes back 4 planes later, where c_1 > 0 and the bulk copy of
    the tile lands on that row.  With one chunk per tile (a one-grid batch,
    chunk length nx) the zero of E_x lies inside every unit's ring, in both
    layouts, and each step must still match the oracle."""
    layout(monkeypatch, half)
    shape = (48, 40, 30)
    g, o = setup(shape, prec, 41)
    assert g.info()["units_per_cta"] == (2 if half else 1)
    ex = g.moments()[1]
    k0 = int(np.argmax(ex < 0))  # first plane with c_1 > 0
    assert ex[0] > 0 and 8 <= k0 <= shape[0] - 8, (k0, ex[0])
    with fk.Batch([g]) as b:
        b.set_chunks([shape[0]])
        assert list(b.chunks()) == [shape[0]]
        for _ in range(3):
            o.set_state(g.get_f(), g.surface_charge())
            b.step(1)
            assert b.sync() == [fk.FK_OK]
            o.step(1)
            fg, fo = g.get_f(), o.get_f()
            assert rel_l1(fg, fo) <= tol
            # the edge row the zero-fill and the copy share, plane by plane
            edge = np.abs(fg[:, -1, :] - fo[:, -1, :]).max(axis=1)
            assert np.all(edge <= 10 * tol * np.abs(fo).max()), edge.max()
            assert abs(g.surface_charge() - o.surface_charge()) <= tol * abs(o.surface_charge())
    g.close()


@pytest.mark.parametrize("prec,tol", [(fk.FK_F64, 1e-10), (fk.FK_F32, 1e-5)])
def test_multi_step_parity_and_ledger(prec, tol):
    shape = (30, 28, 26)
    g, o = setup(shape, prec, 34, dtnu=0.02)
    assert g.info()["units_per_cta"] == 2
    g.step(75)  # two graph replays and eleven direct steps
    o.step(75)
    assert rel_l1(g.get_f(), o.get_f()) <= tol
    assert abs(g.surface_charge() - o.surface_charge()) <= 1e-4 * abs(o.surface_charge())
    if prec == fk.FK_F64:
        lg, lo = g.ledger(), o.ledger()
        for key in ("emit", "pe", "see", "vac", "lv", "inj"):
            assert abs(lg[key] - lo[key]) <= 1e-9 * abs(lo[key]), key
    g.close()


def test_odd_unit_count_leaves_a_half_idle():
    """Only v1 > 0 rows: one tile, and an odd number of x-chunks puts a
    lone unit on the last CTA."""
    shape = (11, 9, 12)
    g, o = setup(shape, fk.FK_F64, 35, v1=(1e6, V1))
    info = g.info()
    assert info["units_per_cta"] == 2 and info["n_tiles"] == 1
    assert (info["n_tiles"] * info["n_chunks"]) % 2 == 1
    for _ in range(4):
        g.step(1)
        o.step(1)
    assert rel_l1(g.get_f(), o.get_f()) <= 1e-12
    g.close()


MIXED = [(33, 200, 46), (9, 8, 8), (40, 24, 21), (12, 64, 81), (11, 9, 12), (64, 48, 48)]


@pytest.mark.parametrize("prec", [fk.FK_F64, fk.FK_F32])
def test_mixed_batch_bitwise_equals_stepping_alone(prec):
    """A batch of whole-CTA and half-CTA grids (two step-kernel launches per
    batch step, an odd number of half units) steps every grid exactly as
    stepping it alone."""
    def grids():
        out = []
        for q, s in enumerate(MIXED):
            v1 = (1e6, V1) if s == (11, 9, 12) else (-V1, V1)
            g, _ = setup(s, prec, 50 + q, v1=v1, with_oracle=False)
            out.append(g)
        return out
    alone, batched = grids(), grids()
    layouts = [g.info()["units_per_cta"] for g in alone]
    assert 1 in layouts and 2 in layouts
    with fk.Batch(batched) as b:
        info = b.info()
        assert info["whole_ctas"] > 0 and info["half_ctas"] > 0
        assert info["step_launches"] == 2
        b.step(41)
        assert b.sync() == [fk.FK_OK] * len(MIXED)
        b.autotune(2)  # other chunkings, the same results
        b.step(9)
        assert b.sync() == [fk.FK_OK] * len(MIXED)
        _, steps, _, _ = b.scalars()
    for g, n in zip(alone, steps):
        g.step(int(n))
    for ga, gb in zip(alone, batched):
        assert np.array_equal(ga.get_f(), gb.get_f())
        assert ga.surface_charge() == gb.surface_charge()
        ga.close()
        gb.close()
