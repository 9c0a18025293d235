"""Runs to SEEA saturation on the GPU against the FP64 oracle's.

The oracle's runs of the ``saturation_64x24x32`` workload (synth.WORKLOADS:
an empty, uncharged 8 um gap driven to saturation at two applied fields)
are stored in tests/golden/saturation_64x24x32.json by
tests/golden/make_saturation.py, which calls only the oracle; the CPU tests
re-run the oracle and check it reproduces them, and pin the saturated state
against Sec. 3 (Eqs. 19-20).  Here the same runs go through the C ABI:

- FP64 grid: the device convergence test of Sec. 2 (finalize kernel) fires
  at the oracle's saturated step exactly, with sigma, Gamma_pe and
  Gamma_see there within 1e-10 relative of the oracle's;
- FP32 grid (f stored and advected in FP32, accumulators FP64): saturated
  surface charge within 1e-4 relative of the FP64 path's.
"""
import json
import os

import numpy as np
import pytest

from paper_2303_14119_gb300 import fk, synth

pytestmark = pytest.mark.gpu

NAME = "saturation_64x24x32"
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", NAME + ".json")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fk.load()


def golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


def run(Ey, precision, steps):
    """The workload at field Ey from f = 0, sigma = 0, stepped `steps` steps;
    returns (saturated step, history rows 0..steps, grid step)."""
    w = synth.WORKLOADS[NAME]
    g = fk.Grid(w["nx"], w["nv1"], w["nv2"], w["h_max"], -w["v1_span"], w["v1_span"],
                -w["v2_span"], w["v2_span"], cfl=w["cfl"], precision=precision,
                history_capacity=1 << 18)
    g.set_fields(Ey)
    g.set_see(w["delta_max"], w["A_max"], w["k_s"], w["T_se"])
    g.set_source(w["J"], w["x_lo"], w["x_hi"], w["T_fe"])
    g.set_convergence(w["sat_window"], w["sat_tol"])
    g.step(steps)
    step, sat = g.step_count()
    hist = g.history(steps + 1)
    g.close()
    assert step == steps
    return sat, hist


@pytest.mark.parametrize("which", [0, 1])
def test_fp64_saturates_at_the_oracle_step(which):
    r = golden()["runs"][which]
    sat, hist = run(r["Ey"], fk.FK_F64, r["sat_step"] + 1)
    assert sat == r["sat_step"]
    row = hist[sat]
    assert row[0] == sat
    for col, key in ((2, "sigma_sat"), (3, "gamma_pe_sat"), (4, "gamma_see_sat")):
        assert abs(row[col] / r[key] - 1.0) <= 1e-10, (key, row[col], r[key])
    # the growth of the charge on the way, every 5000 steps
    s5 = np.array(r["sigma_every_5000"])
    g5 = hist[5000:sat + 1:5000, 2]
    assert np.allclose(g5, s5, rtol=1e-9, atol=0.0)


@pytest.mark.parametrize("which", [0, 1])
def test_fp32_saturated_charge_within_1e4_of_fp64(which):
    r = golden()["runs"][which]
    w = synth.WORKLOADS[NAME]
    n = r["sat_step"] + w["sat_window"]
    sat64, h64 = run(r["Ey"], fk.FK_F64, n)
    sat32, h32 = run(r["Ey"], fk.FK_F32, n)
    assert sat64 == r["sat_step"]
    assert sat32 >= 0, "the FP32 run did not saturate"
    # saturated surface charge (each path at its own saturated step, and
    # both at the end of the run)
    assert abs(h32[sat32, 2] / h64[sat64, 2] - 1.0) <= 1e-4
    assert abs(h32[n, 2] / h64[n, 2] - 1.0) <= 1e-4
    # saturation detected within a few hundred steps of the FP64 path's
    assert abs(sat32 - sat64) <= 0.05 * w["sat_window"]


def test_batched_runs_saturate_at_the_oracle_steps_bitwise_as_alone():
    """Both saturating runs in one batch, beside a grid of several finalize
    blocks (nx = 300) and a grid of five planes: the batch's finalize (one
    warp for each grid of at most 128 planes, four to a CTA; whole blocks
    for the others) fires the convergence test at the oracle's saturated
    steps, and the saturating grids' histories are those of the grids
    stepped alone, bit for bit."""
    runs = golden()["runs"]
    w = synth.WORKLOADS[NAME]
    n = max(r["sat_step"] for r in runs) + 1
    alone = [run(r["Ey"], fk.FK_F64, n) for r in runs]

    def grid(nx, Ey):
        g = fk.Grid(nx, w["nv1"], w["nv2"], w["h_max"], -w["v1_span"], w["v1_span"],
                    -w["v2_span"], w["v2_span"], cfl=w["cfl"], precision=fk.FK_F64,
                    history_capacity=1 << 18)
        g.set_fields(Ey)
        g.set_see(w["delta_max"], w["A_max"], w["k_s"], w["T_se"])
        g.set_source(w["J"], w["x_lo"], w["x_hi"], w["T_fe"])
        g.set_convergence(w["sat_window"], w["sat_tol"])
        return g

    sat_grids = [grid(w["nx"], r["Ey"]) for r in runs]
    grids = [grid(300, runs[0]["Ey"]), sat_grids[0], grid(5, runs[1]["Ey"]), sat_grids[1]]
    with fk.Batch(grids) as b:
        # one finalize CTA per 128 planes of the 300-plane grid, one for the
        # three grids of at most 128
        assert b.info()["finalize_ctas"] == 3 + 1
        b.step(n)
        status = b.sync()
    assert status[1] == fk.FK_OK and status[3] == fk.FK_OK
    for g, r, (sat, hist) in zip(sat_grids, runs, alone):
        step, sat_b = g.step_count()
        assert step == n and sat_b == sat == r["sat_step"]
        assert np.array_equal(g.history(n + 1), hist)
    for g in grids:
        g.close()
