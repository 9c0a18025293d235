"""Failure detection on the GPU, without a GPU fault.

- A bounded wait that runs out: with the test knobs FK_TEST_WAIT_CYCLES
  (a short wait limit) and FK_TEST_WITHHOLD_COPY (one pipeline item whose
  plane copy a work unit does not issue) set at grid creation, the
  streaming step kernel's waits on that item run out.  The step must report
  FK_ETIMEOUT, leave f at the last valid state, do nothing on later steps,
  and leave the GPU usable: a grid created afterwards steps and matches the
  FP64 oracle.  Every copy that was issued lands before the kernel leaves;
  no wait in the kernel is unbounded.
- Negative f: a state with a negative value injected from the host is
  reported as FK_ENEGATIVE by fk_set_f, and the grid refuses to step until a
  valid state is set.
- Allocation failure: with FK_TEST_FAIL_ALLOC=n the n-th device or pinned
  allocation of a grid's or a batch's creation fails on the host (nothing
  reaches the GPU).  Creation must return FK_ENOMEM for every n up to the
  number of allocations, free what it allocated, and leave the device
  usable.
"""
import os

import numpy as np
import pytest

from paper_2303_14119_gb300 import fk, synth

from test_gpu_parity import make_pair, rel_l1, strong_physics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fk.load()


def knobbed_pair(shape, prec, item):
    os.environ["FK_TEST_WAIT_CYCLES"] = "2000000"  # about 1 ms
    os.environ["FK_TEST_WITHHOLD_COPY"] = str(item)
    try:
        return make_pair(shape, prec=prec)
    finally:
        del os.environ["FK_TEST_WAIT_CYCLES"]
        del os.environ["FK_TEST_WITHHOLD_COPY"]


@pytest.mark.parametrize("prec,tol", [(fk.FK_F64, 1e-12), (fk.FK_F32, 3e-7)])
# item: below the 4 planes every chunk has at least; on the long grid the
# chunks are 27 planes and item 9 lies past the first pass of the stage ring
@pytest.mark.parametrize("shape,item", [((16, 24, 20), 2), ((40, 64, 96), 3), ((8192, 4, 8), 9)])
def test_wait_that_runs_out_reports_timeout_and_freezes(prec, tol, shape, item):
    g, o = knobbed_pair(shape, prec, item)
    info = g.info()
    assert info["kernel"] == "stream" and info["chunk_len"] > item
    f0, sigma = strong_physics(g, o, shape, seed=31, c1f=0.05)
    g.set_state(f0, sigma)
    start = g.get_f()  # the state in the grid's storage precision
    assert fk.fk_step_status(g.h, 3) == fk.FK_OK  # enqueued
    assert fk.fk_sync_status(g.h) == fk.FK_ETIMEOUT
    assert "bounded wait" in fk.fk_last_error(g.h)
    assert fk.fk_step_status(g.h, 2) == fk.FK_ETIMEOUT  # frozen: refuses
    out = np.empty(shape)
    with pytest.raises(fk.FkError) as ei:
        g.get_f(out)
    assert ei.value.status == fk.FK_ETIMEOUT
    assert np.array_equal(out, start)  # the last valid state
    with pytest.raises(fk.FkError):
        g.step_count()
    g.close()
    # the GPU is still usable: a fresh grid steps and matches the oracle
    g, o = make_pair(shape, prec=prec)
    f0, sigma = strong_physics(g, o, shape, seed=31, c1f=0.05)
    g.set_state(f0, sigma)
    o.set_state(g.get_f(), sigma)
    g.step(2)
    o.step(2)
    assert rel_l1(g.get_f(), o.get_f()) <= 2 * tol
    g.close()


@pytest.mark.parametrize("prec", [fk.FK_F64, fk.FK_F32])
def test_negative_input_state_is_reported(prec):
    shape = (12, 16, 20)
    g, o = make_pair(shape, prec=prec)
    f0, sigma = strong_physics(g, o, shape, seed=32, c1f=0.05)
    bad = f0.copy()
    bad[3, 5, 7] = -0.5 * bad.max()
    with pytest.raises(fk.FkError) as ei:
        g.set_f(bad)
    assert ei.value.status == fk.FK_ENEGATIVE
    assert fk.fk_step_status(g.h, 1) == fk.FK_ENEGATIVE
    # a valid state clears it and the grid steps again
    g.set_state(f0, sigma)
    g.step(3)
    assert g.step_count()[0] == 3
    g.close()


def _grid(shape, prec=fk.FK_F64):
    return fk.Grid(*shape, 20e-6, -6e7, 6e7, -3e7, 3e7, cfl=0.4, precision=prec)


@pytest.mark.parametrize("prec", [fk.FK_F64, fk.FK_F32])
def test_every_allocation_failure_of_a_creation_is_reported(prec, monkeypatch):
    shape = (16, 24, 20)
    failed = 0
    for n in range(1, 200):
        monkeypatch.setenv("FK_TEST_FAIL_ALLOC", str(n))
        try:
            g = _grid(shape, prec)
        except fk.FkError as e:
            assert e.status == fk.FK_ENOMEM, (n, e)
            failed += 1
            continue
        finally:
            monkeypatch.delenv("FK_TEST_FAIL_ALLOC")
        g.close()
        break
    assert failed >= 20  # every allocation point of the grid was made to fail
    # batches: a grid pair, each allocation of the batch's creation in turn
    grids = [_grid(shape, prec), _grid((9, 8, 8), prec)]
    bfailed = 0
    for n in range(1, 50):
        monkeypatch.setenv("FK_TEST_FAIL_ALLOC", str(n))
        try:
            b = fk.Batch(grids)
        except fk.FkError as e:
            assert e.status == fk.FK_ENOMEM, (n, e)
            bfailed += 1
            continue
        finally:
            monkeypatch.delenv("FK_TEST_FAIL_ALLOC")
        b.step(3)
        assert b.sync() == [fk.FK_OK, fk.FK_OK]
        b.close()
        break
    assert bfailed >= 2
    # the grids (released by every failed batch) and the device still work
    g, o = make_pair(shape, prec=prec)
    f0, sigma = strong_physics(g, o, shape, seed=41, c1f=0.05)
    g.set_state(f0, sigma)
    o.set_state(f0, sigma)
    g.step(5)
    o.step(5)
    assert rel_l1(g.get_f(), o.get_f()) <= (1e-12 if prec == fk.FK_F64 else 1e-6)
    for x in grids + [g]:
        x.step(2)
        x.close()
