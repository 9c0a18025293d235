"""The seeded input generator: SplitMix64 against its published outputs,
and the layout of generated distributions."""
import numpy as np

from paper_2303_14119_gb300 import synth


def test_splitmix64_reference_outputs():
    # first outputs of SplitMix64 (Steele, Lea, Flood 2014) for two seeds
    assert int(synth.splitmix64(0, np.arange(1))[0]) == 0xE220A8397B1DCDAF
    assert [int(x) for x in synth.splitmix64(1234567, np.arange(3))] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_uniform_is_counter_based_and_in_range():
    u = synth.uniform(7, 1000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.array_equal(synth.uniform(7, 10, offset=500), u[500:510])
    assert abs(u.mean() - 0.5) < 0.05
    # chunking does not change the stream
    assert np.array_equal(synth.uniform(7, 1000, chunk=37), u)


def test_initial_f_scale_and_shape():
    f = synth.initial_f((4, 3, 5), seed=0, noise_rel=1e-6, J=1.0, T_fe_eV=4.0)
    assert f.shape == (4, 3, 5)
    scale = synth.beam_scale(1.0, 4.0)
    assert f.max() < 1e-6 * scale and f.min() >= 0.0
    flat = 1e-6 * scale * synth.uniform(0, 60)
    assert np.array_equal(f.ravel(), flat)


def test_workloads_are_consistent():
    for name, w in synth.WORKLOADS.items():
        if "sweep" in w or "runs" in w:
            continue
        assert w["nx"] >= 2 and w["Ey"] < 0
        assert f"{w['nx']}x{w['nv1']}x{w['nv2']}" in name


def test_sweep_instances_ranges_and_determinism():
    w = synth.WORKLOADS["sweep_256"]
    ins = synth.sweep_instances(w["sweep"], w["seed"])
    assert len(ins) == 256
    assert ins == synth.sweep_instances(w["sweep"], w["seed"])
    assert ins != synth.sweep_instances(w["sweep"], w["seed"] + 1)
    nx = np.array([p["nx"] for p in ins])
    nv = np.array([p["nv1"] for p in ins])
    e = np.array([-p["Ey"] for p in ins])
    assert nx.min() >= 128 and nx.max() <= 512 and len(set(nx)) > 100
    assert nv.min() >= 64 and nv.max() <= 192 and all(p["nv1"] == p["nv2"] for p in ins)
    assert e.min() >= 3e5 and e.max() <= 5e6
    # log-uniform: about half the draws lie below the geometric midpoint
    frac_low = np.mean(np.log(e) < 0.5 * (np.log(3e5) + np.log(5e6)))
    assert 0.4 < frac_low < 0.6
    for key, lo, hi in (("delta_max", 2.0, 4.0), ("A_max", 250.0, 600.0), ("T_se", 1.0, 5.0)):
        v = np.array([p[key] for p in ins])
        assert v.min() >= lo and v.max() <= hi and v.std() > 0.2 * (hi - lo)
    assert len({p["seed"] for p in ins}) == 256


def test_batched_workload_entries():
    w = synth.WORKLOADS["surrogate_1536"]
    runs = synth.batch_instances(w)
    assert runs == synth.surrogate_runs(1536, 11)
    assert all((p["nx"], p["nv1"], p["nv2"]) == (64, 48, 48) for p in runs)
    # the step count covers the horizon at the smallest gap drawn
    h_min = min(p["h_max"] for p in runs)
    dt = w["cfl"] * (h_min / 64) / w["v1_span"]
    assert h_min >= synth.SURROGATE_H[0] and w["steps"] * dt >= 1.25e-9
    assert synth.batch_instances(synth.WORKLOADS["sweep_256"]) == synth.sweep_instances(256, 2023)
