"""Host-side logic of the surrogate pipeline (no GPU): features, labels from
sampled histories (interpolation, censoring, invalid runs), targets, and the
data set solved in parts and merged."""
import math

import numpy as np
import pytest

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


def _fake_part(runs, idx, seed):
    rng = np.random.default_rng(seed)
    m = idx.size
    res = dict(status=np.zeros(m, dtype=np.int32), sat_step=rng.integers(-1, 9, m),
               dt=rng.random(m), seconds=1.5, batch_steps=100 + seed, cells=float(m * 10))
    prof = rng.random((m, S.N_PROFILE))
    return res, prof, rng.random(m), rng.random(m) > 0.2


def test_parts_cover_the_draws_and_merge_back(tmp_path):
    runs = synth.surrogate_runs(11, 5)
    parts = [S.part_slice(11, "%d/3" % i) for i in range(3)]
    assert np.array_equal(np.concatenate(parts), np.arange(11))
    assert [p.size for p in parts] == [4, 4, 3]
    with pytest.raises(ValueError):
        S.part_slice(11, "3/3")
    paths, want = [], {}
    for i, idx in enumerate(parts):
        res, prof, tsat, ok = _fake_part(runs, idx, i)
        path = str(tmp_path / ("p%d.npz" % i))
        S.save_data(path, idx, runs, res, prof, tsat, ok)
        paths.append(path)
        want[i] = (idx, res, prof, tsat, ok)
    d = S.load_data(paths[::-1], runs)  # any order
    for idx, res, prof, tsat, ok in want.values():
        assert np.array_equal(d["prof"][idx], prof) and np.array_equal(d["tsat"][idx], tsat)
        assert np.array_equal(d["ok"][idx], ok) and np.array_equal(d["sat_step"][idx], res["sat_step"])
    assert d["seconds"] == 4.5 and d["batch_steps"] == 102
    assert d["cell_steps"] == 40 * 100 + 40 * 101 + 30 * 102
    # features made on another machine may differ in the last bit
    z = dict(np.load(paths[0]))
    z["X"] = np.nextafter(z["X"], np.inf)
    np.savez(paths[0], **z)
    assert np.array_equal(S.load_data(paths, runs)["prof"], d["prof"])
    # a missing part, a doubled part, other draws: refused
    with pytest.raises(ValueError, match="no data"):
        S.load_data(paths[:2], runs)
    with pytest.raises(ValueError, match="twice"):
        S.load_data(paths + paths[:1], runs)
    with pytest.raises(ValueError, match="other draws"):
        S.load_data(paths, synth.surrogate_runs(11, 6))
