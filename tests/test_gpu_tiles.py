"""Tile plans of the streaming step kernel (fk_set_tile_rows) and the tile
search of the batch autotuner (fk_batch_autotune_tiles).

A grid's whole-CTA units cover tiles of v1 rows; the per-cell update does
not depend on the tiles, but n_e(x) is summed per (plane, tile), so the tile
plan sets the rounding of everything after the moments.  Here a capped plan
is checked against the FP64 oracle step by step, against the default plan
to rounding, and, in a batch, bit for bit against the same grids stepped
alone with the same caps.
"""
import numpy as np
import pytest

import oracle
from oracle import EPS0, ME, QE
from paper_2303_14119_gb300 import fk, synth

from test_gpu_batch import assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fk.load()


H, V1, V2 = 20e-6, 6e7, 3e7


def setup(shape, prec, seed, with_oracle=True):
    """Grid (and oracle) with E_x changing sign, SEE, source and a large
    E_y; returns (grid, oracle or None, f0, sigma0)."""
    nx, nv1, nv2 = shape
    g = fk.Grid(nx, nv1, nv2, H, -V1, V1, -V2, V2, cfl=0.4, precision=prec)
    info = g.info()
    a2 = 0.15 * info["dv2"] / info["dt"]
    emax = 0.2 * info["dv1"] / info["dt"] * ME / QE
    n_tot = 1.6 * emax * EPS0 / QE
    f0 = synth.random_f(shape, seed, 2 * n_tot / (H * 2 * V1 * 2 * V2))
    sigma = 2 * EPS0 * emax * 0.8
    xs = [g]
    o = None
    if with_oracle:
        o = oracle.Oracle(nx, nv1, nv2, H, -V1, V1, -V2, V2, cfl=0.4)
        xs.append(o)
    for x in xs:
        x.set_fields(-a2 * ME / QE, True, 0.0)
        x.set_see(3.0, 400.0, 1.0, 400.0)
        x.set_source(1e7, 0.2 * H, 0.7 * H, 300.0)
        x.set_state(f0, sigma)
    return g, o, f0, sigma


def rel_l1(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


@pytest.mark.parametrize("prec,tol", [(fk.FK_F64, 1e-12), (fk.FK_F32, 3e-7)])
def test_capped_tiles_keep_the_state_and_step_like_the_oracle(prec, tol):
    shape = (24, 96, 72)  # each sign half too large for a half unit
    g, o, f0, sigma = setup(shape, prec, 61)
    info = g.info()
    assert info["kernel"] == "stream" and info["units_per_cta"] == 1
    assert info["tile_cap"] == 0 and info["tile_rows"] > 7
    before = g.get_f()
    g.set_tile_rows(7)
    info = g.info()
    assert info["tile_cap"] == 7 and info["tile_rows"] <= 7
    assert info["n_tiles"] == 2 * -(-48 // 7)  # 48 rows per sign of v1
    assert np.array_equal(g.get_f(), before)
    for _ in range(3):
        o.set_state(g.get_f(), g.surface_charge())
        g.step(1)
        o.step(1)
        assert rel_l1(g.get_f(), o.get_f()) <= tol
        assert abs(g.surface_charge() - o.surface_charge()) <= tol * abs(o.surface_charge())
    g.step(40)  # a graph replay with the capped plan
    o.set_state(g.get_f(), g.surface_charge())
    g.step(1)
    o.step(1)
    assert rel_l1(g.get_f(), o.get_f()) <= tol
    g.set_tile_rows(0)
    assert g.info()["tile_cap"] == 0 and g.info()["n_tiles"] < 14
    g.close()


@pytest.mark.parametrize("prec,tol", [(fk.FK_F64, 1e-12), (fk.FK_F32, 2e-6)])
def test_the_tile_plan_changes_only_rounding(prec, tol):
    shape = (32, 128, 96)
    runs = []
    for cap in (0, 9):
        g, _, _, _ = setup(shape, prec, 62, with_oracle=False)
        g.set_tile_rows(cap)
        g.step(50)
        runs.append((g.get_f(), g.surface_charge()))
        g.close()
    assert rel_l1(runs[1][0], runs[0][0]) <= tol
    assert abs(runs[1][1] - runs[0][1]) <= tol * abs(runs[0][1])


def test_tile_rows_refused_while_batched_and_checked():
    g, _, _, _ = setup((16, 64, 64), fk.FK_F64, 63, with_oracle=False)
    with pytest.raises(fk.FkError) as ei:
        g.set_tile_rows(-1)
    assert ei.value.status == fk.FK_EINVAL
    with fk.Batch([g]):
        with pytest.raises(fk.FkError) as ei:
            g.set_tile_rows(8)
        assert ei.value.status == fk.FK_ESTATE
    g.set_tile_rows(8)
    assert g.info()["tile_cap"] == 8
    g.close()


SHAPES = [(40, 256, 256), (24, 128, 200), (9, 8, 8), (30, 28, 26)]


def twins(prec, caps):
    a, b = [], []
    for q, s in enumerate(SHAPES):
        ga, _, f0, sigma = setup(s, prec, 70 + q, with_oracle=False)
        gb, _, _, _ = setup(s, prec, 70 + q, with_oracle=False)
        for g in (ga, gb):
            g.set_tile_rows(caps[q])
            g.set_state(f0, sigma)
        a.append(ga)
        b.append(gb)
    return a, b


@pytest.mark.parametrize("prec", [fk.FK_F32, fk.FK_F64])
def test_batch_with_the_tuned_tiles_equals_stepping_alone(prec):
    # the tile search on scratch copies of the grids
    scratch = [setup(s, prec, 70 + q, with_oracle=False)[0] for q, s in enumerate(SHAPES)]
    with fk.Batch(scratch) as b:
        taken = b.autotune(steps_per_trial=1, tiles=True)
        assert taken >= 2 and b.info()["steps"] == taken
        chunks = b.chunks()
        caps = [g.info()["tile_cap"] for g in scratch]
        assert b.sync() == [fk.FK_OK] * len(SHAPES)
    for g, s, c in zip(scratch, SHAPES, caps):
        pitch = s[2] + (-s[2]) % (4 if prec == fk.FK_F32 else 2)
        assert c in (0, max(4, 5120 // pitch), max(4, 4096 // pitch)), (s, c)
        if g.info()["units_per_cta"] == 2:
            assert c == 0  # half units keep their tiles
        g.close()
    # the plan found, and a forced one, step alike in a batch and alone
    for plan in (caps, [16, 12, 0, 0]):
        alone, batched = twins(prec, plan)
        with fk.Batch(batched) as b:
            b.set_chunks(chunks)
            b.step(40)
            for g in alone:
                g.step(40)
            assert b.sync() == [fk.FK_OK] * len(SHAPES)
            for ga, gb in zip(alone, batched):
                assert gb.info()["tile_cap"] == ga.info()["tile_cap"]
                assert_same(ga, gb)
        for g in alone + batched:
            g.close()
