"""Host-side logic of the surrogate pipeline (no GPU): features, labels from
sampled histories (interpolation, censoring, invalid runs) and targets."""
import math

import numpy as np

from paper_2303_14119_gb300 import fk, surrogate as S, synth


def test_surrogate_runs_ranges():
    runs = synth.surrogate_runs(2000, 3)
    J = np.array([p["J"] for p in runs])
    h = np.array([p["h_max"] for p in runs])
    assert J.min() >= 1e5 and J.max() <= 1e7 and 0.4 < np.mean(np.log10(J) < 6) < 0.6
    assert h.min() >= 16e-6 and h.max() <= 24e-6
    assert all((p["nx"], p["nv1"], p["nv2"]) == (64, 48, 48) for p in runs)
    assert runs == synth.surrogate_runs(2000, 3)


def test_features_are_the_stated_transforms():
    p = dict(Ey=-2e6, delta_max=3.0, A_max=400.0, T_se=2.0, J=1e6, h_max=20e-6)
    f = S.features([p])[0]
    assert np.allclose(f, [math.log10(2e6), 3.0, 4.0, 2.0, 6.0, 2.0])


def fake_result():
    # two runs sampled every 1000 steps; run 0 saturates at step 5000 with
    # dt = 1e-13 (t = 0.5 ns), run 1 never does, run 2 is frozen (ECFL)
    steps = np.arange(0, 16000, 1000)
    st = np.stack([steps, steps, np.minimum(steps, 3000)], axis=1)
    sig = np.stack([np.minimum(steps, 5000) * 1e-9, steps * 2e-9, np.minimum(steps, 3000) * 1e-9], axis=1)
    return dict(dt=np.array([1e-13, 1e-13, 1e-13]), steps=st, sigma=sig,
                sat_step=np.array([5000, -1, -1]), status=np.array([fk.FK_OK, fk.FK_OK, fk.FK_ECFL]))


def test_labels_interpolate_censor_and_flag():
    res = fake_result()
    horizon = 1.28e-9  # 12800 steps: inside the sampled range
    prof, tsat, ok = S.labels(res, horizon)
    tk = (np.arange(S.N_PROFILE) + 1) * horizon / S.N_PROFILE
    s_k = tk / 1e-13
    assert np.allclose(prof[1], s_k * 2e-9, rtol=1e-12)
    assert np.allclose(prof[0], np.minimum(s_k, 5000) * 1e-9, rtol=1e-12)
    assert tsat[0] == 5000 * 1e-13 and tsat[1] == S.T_CENSOR
    assert list(ok) == [True, True, False]
    # saturation after the horizon is censored too
    res["sat_step"][0] = 13000
    _, tsat2, _ = S.labels(res, horizon)
    assert tsat2[0] == S.T_CENSOR


def test_targets_layout():
    prof = np.ones((3, S.N_PROFILE)) * 2e-4
    tsat = np.array([1e-9, 1e-10, S.T_CENSOR])
    Y = S.targets(prof, tsat)
    assert Y.shape == (3, S.N_PROFILE + 1)
    assert np.allclose(Y[:, :-1], 2.0) and np.allclose(Y[:, -1], np.log10(tsat / 1e-9))
