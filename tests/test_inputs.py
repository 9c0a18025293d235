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
        assert w["nx"] >= 2 and w["Ey"] < 0
        assert f"{w['nx']}x{w['nv1']}x{w['nv2']}" in name
