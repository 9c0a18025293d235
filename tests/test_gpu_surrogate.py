"""The trained surface-charge surrogate (weights committed with the
package) against the solver: its predictions on held-out runs, and what it
gains the solver as a warm start.

The held-out runs are draws 1280..1535 of synth.surrogate_runs(1536, 11);
their solver labels (sigma(t) profile, saturation step) were written by the
same pipeline that trained the network and are stored beside the weights.
A cold run of the solver is deterministic (batch results equal stepping
alone bit for bit), so the stored saturation steps are those a cold re-run
gives.
"""
import os

import numpy as np
import pytest

from paper_2303_14119_gb300 import fk, surrogate as S, synth

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(S.__file__), "data", "surrogate_64x48x48.npz")


@pytest.fixture(scope="module")
def sur():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fk.load()
    s = S.Surrogate.load(WEIGHTS)
    yield s
    s.close()


@pytest.fixture(scope="module")
def held_out():
    d = np.load(WEIGHTS)
    n_train, n_test, seed = int(d["n_train"]), int(d["n_test"]), int(d["seed"])
    runs = synth.surrogate_runs(n_train + n_test, seed)[n_train:]
    return runs, d


def test_predictions_on_held_out_runs(sur, held_out):
    runs, d = held_out
    ok = d["test_ok"]
    pp, pt = sur.predict(runs)
    prof = d["test_prof"].astype(np.float64)
    rel = np.linalg.norm(pp[ok] - prof[ok], axis=1) / np.linalg.norm(prof[ok], axis=1)
    assert np.median(rel) <= 0.10
    sat_true = d["test_tsat"][ok] < S.T_CENSOR
    sat_pred = pt[ok] < S.HORIZON
    assert np.mean(sat_true == sat_pred) >= 0.9


def test_warm_start_saves_steps_and_reaches_the_same_charge(sur, held_out):
    runs, d = held_out
    sel = np.flatnonzero(d["test_ok"] & (d["test_sat_step"] >= 0) & (d["test_tsat"] < S.HORIZON))[:8]
    assert sel.size == 8
    pick = [runs[q] for q in sel]
    pp, _ = sur.predict(pick)
    import torch
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
