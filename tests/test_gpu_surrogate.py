"""The trained surface-charge surrogates (weights committed with the
package) against the solver: their predictions on held-out runs, and what
they gain the solver as a warm start.

- surrogate_64x48x48.npz: trained on the 4096 training draws of
  synth.surrogate_runs(4608, 11) solved on 64 x 48 x 48; held out: draws
  4096..4607, whose solver labels (sigma(t) profile, saturation step) are
  stored beside the weights.
- surrogate_512x128x128.npz: the same network fine-tuned on the training
  draws solved cold on 512 x 128 x 128 to saturation; held out: 16 draws of
  the held-out set solved cold on that grid, their labels stored beside it.

A cold run of the solver is deterministic (batch results equal stepping
alone bit for bit), so the stored saturation steps are those a cold re-run
gives up to the rounding of later changes to the kernels' sums.
"""
import os

import numpy as np
import pytest

from paper_2303_14119_gb300 import fk, surrogate as S, synth

pytestmark = pytest.mark.gpu

DATA = os.path.join(os.path.dirname(S.__file__), "data")
COARSE = os.path.join(DATA, "surrogate_64x48x48.npz")
FINE = os.path.join(DATA, "surrogate_512x128x128.npz")


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fk.load()
    return torch


def held_out(path):
    d = np.load(path)
    n_train, n_test, seed = int(d["n_train"]), int(d["n_test"]), int(d["seed"])
    runs = synth.surrogate_runs(n_train + n_test, seed)
    if "fine_idx_test" in d.files:
        nx, nv, _ = (int(v) for v in d["grid"])
        runs = [dict(runs[q], nx=nx, nv1=nv, nv2=nv) for q in d["fine_idx_test"]]
    else:
        runs = runs[n_train:]
    return runs, d


def test_predictions_on_held_out_runs(torch):
    runs, d = held_out(COARSE)
    assert len(runs) == 512
    sur = S.Surrogate.load(COARSE)
    ev = S.evaluate(sur, runs, d["test_prof"], d["test_tsat"], d["test_ok"])
    sur.close()
    assert ev["runs"] >= 480
    assert ev["profile_rel_l2"]["median"] <= 0.05
    assert ev["triage_accuracy"] >= 0.95


def test_warm_start_saves_steps_and_reaches_the_same_charge(torch):
    runs, d = held_out(COARSE)
    sel = np.flatnonzero(d["test_ok"] & (d["test_sat_step"] >= 0) & (d["test_tsat"] < S.HORIZON))[:8]
    assert sel.size == 8
    pick = [runs[q] for q in sel]
    sur = S.Surrogate.load(COARSE)
    pp, _ = sur.predict(pick)
    sur.close()
    res = S.solve(pick, sigma0=pp[:, -1], stream=torch.cuda.current_stream().cuda_stream,
                  autotune=False)
    prof_w, _, ok_w = S.labels(res)
    assert ok_w.all()
    cold = d["test_sat_step"][sel].astype(np.int64)
    warm = res["sat_step"]
    assert (warm >= 0).all()
    # the surrogate's charge saves at least a fifth of the steps to saturation
    assert warm.sum() <= 0.8 * cold.sum(), (warm, cold)
    # and the warm runs end where the cold ones did
    end_cold = d["test_prof"][sel, -1].astype(np.float64)
    assert np.all(np.abs(prof_w[:, -1] - end_cold) <= 1e-2 * np.abs(end_cold))


def test_fine_tuned_network_predicts_the_fine_grid_charge(torch):
    """On 512 x 128 x 128 the saturated charge is well below the 64 x 48 x 48
    one (the coarse grid does not resolve the secondaries' hop height).  The
    fine-tuned network predicts the fine grid's saturated charge of the held-
    out points several times better than the coarse network does."""
    runs, d = held_out(FINE)
    assert len(runs) == 16
    out = {}
    for name, path in (("coarse", COARSE), ("fine", FINE)):
        sur = S.Surrogate.load(path)
        pp, _ = sur.predict(runs)
        sur.close()
        end = d["test_prof"][:, -1].astype(np.float64)
        out[name] = np.median(np.abs(pp[:, -1] - end) / np.abs(end))
    assert out["fine"] <= 0.3
    assert out["fine"] <= 0.25 * out["coarse"], out


def test_fine_grid_warm_start_saves_steps(torch):
    """Four held-out points on 512 x 128 x 128, started from the fine-tuned
    network's charge, saturate in fewer steps than their stored cold runs
    and at the same charge."""
    runs, d = held_out(FINE)
    sel = np.flatnonzero(d["test_ok"] & (d["test_sat_step"] >= 0))[:4]
    pick = [runs[q] for q in sel]
    sur = S.Surrogate.load(FINE)
    pp, _ = sur.predict(pick)
    sur.close()
    res = S.solve_to_saturation(pick, 1600000, sigma0=pp[:, -1],
                                stream=torch.cuda.current_stream().cuda_stream, autotune=False)
    prof_w, _, ok_w = S.labels(res)
    assert ok_w.all() and (res["sat_step"] >= 0).all()
    cold = d["test_sat_step"][sel].astype(np.int64)
    assert res["sat_step"].sum() <= 0.8 * cold.sum(), (res["sat_step"], cold)
    end_cold = d["test_prof"][sel, -1].astype(np.float64)
    assert np.all(np.abs(prof_w[:, -1] - end_cold) <= 1e-2 * np.abs(end_cold))
