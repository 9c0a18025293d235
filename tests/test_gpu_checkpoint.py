"""Checkpoints (fk_get_state / fk_set_state): a grid restored into a fresh
grid steps on bit for bit as the original does."""
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


def new_grid(shape, prec, cap=0):
    return fk.Grid(*shape, H, -V1, V1, -V2, V2, cfl=0.4, precision=prec, history_capacity=cap)


def configured(shape, prec, scheme=fk.FK_SCHEME_UNSPLIT):
    g = new_grid(shape, prec)
    info = g.info()
    g.set_fields(-0.15 * info["dv2"] / info["dt"] * ME / QE, True, 0.0)
    g.set_see(3.0, 400.0, 1.0, 400.0)
    g.set_source(1e7, 0.2 * H, 0.7 * H, 300.0)
    emax = 0.2 * info["dv1"] / info["dt"] * ME / QE
    amp = 2 * (1.6 * emax * EPS0 / QE) / (H * 2 * V1 * 2 * V2)
    f0 = synth.random_f(shape, 17, amp)
    # ln(Lambda) scaled so that dt nu_ee is about 3 % for this state
    n_max = (f0.sum(axis=(1, 2)) * info["dv1"] * info["dv2"]).max()
    g.set_collisions(2.0, 0.03 / (info["dt"] * oracle.nu_ee(n_max, 2.0, 1.0)), True)
    g.set_reflection(0.2)
    g.set_scheme(scheme)
    g.set_state(f0, 2 * EPS0 * emax * 0.8)
    return g


def assert_same(a, b):
    assert np.array_equal(a.get_f(), b.get_f())
    assert a.surface_charge() == b.surface_charge()
    assert a.step_count() == b.step_count()
    assert a.ledger() == b.ledger()
    assert np.array_equal(a.history(10 ** 6), b.history(10 ** 6))


@pytest.mark.parametrize("prec", [fk.FK_F64, fk.FK_F32])
@pytest.mark.parametrize("scheme", [fk.FK_SCHEME_UNSPLIT, fk.FK_SCHEME_LIE, fk.FK_SCHEME_STRANG])
def test_restored_grid_continues_bitwise(prec, scheme):
    shape = (20, 32, 26)
    a = configured(shape, prec, scheme)
    a.step(37)
    ck = a.checkpoint()
    a.step(45)  # a graph replay and direct steps
    b = new_grid(shape, prec)  # default parameters: the checkpoint brings its own
    b.restore(ck)
    b.step(45)
    assert_same(a, b)
    a.close()
    b.close()


def test_foreign_or_damaged_checkpoints_are_refused():
    a = configured((12, 16, 16), fk.FK_F32)
    ck = a.checkpoint()
    for other in (new_grid((12, 16, 18), fk.FK_F32), new_grid((12, 16, 16), fk.FK_F64),
                  new_grid((12, 16, 16), fk.FK_F32, cap=1000)):
        with pytest.raises(fk.FkError) as e:
            other.restore(ck)
        assert e.value.status == fk.FK_EINVAL
    b = new_grid((12, 16, 16), fk.FK_F32)
    for bad in (b"nonsense" + ck[8:], ck[:100], ck[:-8]):
        with pytest.raises(fk.FkError) as e:
            b.restore(bad)
        assert e.value.status == fk.FK_EINVAL
    b.restore(ck)
    assert np.array_equal(a.get_f(), b.get_f())


def test_fp32_host_exchange_matches_the_fp64_forms():
    shape = (9, 20, 18)
    g = new_grid(shape, fk.FK_F32)
    f = synth.random_f(shape, 5, 1e2)  # weak enough that its field keeps the CFL bound
    g.set_f32(f.astype(np.float32))
    a = g.get_f32()
    assert np.array_equal(a, f.astype(np.float32))
    assert np.array_equal(g.get_f(), a.astype(np.float64))
    g.set_f(f)  # the FP64 form rounds each value to nearest, the same
    assert np.array_equal(g.get_f32(), a)
    with pytest.raises(fk.FkError):
        new_grid(shape, fk.FK_F64).set_f32(f.astype(np.float32))
    g.close()
