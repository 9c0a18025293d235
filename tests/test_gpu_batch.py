"""Batched stepping (fk_batch_*) against stepping each grid alone and against
the FP64 oracle.

A batch only chooses how the x-planes of each grid are cut into chunks; a
cell's update and every partial sum are the same whichever CTA computes
them, so a batch step must equal fk_step on the same grid bit for bit, for
any chunking, including the autotuner's.
"""
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
# mixed sizes: odd nv2 (row padding), nx below and above a chunk, v1 rows
# that need several tiles
SHAPES = [(9, 8, 8), (40, 24, 21), (64, 48, 48), (17, 70, 36), (128, 32, 40)]


def new_grid(shape, prec):
    nx, nv1, nv2 = shape
    return fk.Grid(nx, nv1, nv2, H, -V1, V1, -V2, V2, cfl=0.4, precision=prec)


def physics(g, shape, seed, c1f=0.2, c2f=0.15):
    """Every term active, parameters varied with the seed; returns the
    initial (f, sigma)."""
    info = g.info()
    rng = np.random.default_rng(seed)
    a2 = c2f * info["dv2"] / info["dt"]
    g.set_fields(-a2 * ME / QE, True, 0.0)
    g.set_see(2.0 + rng.uniform(0, 2), 300.0 + rng.uniform(0, 200), 1.0, 200.0 + rng.uniform(0, 300))
    g.set_source(1e7 * (0.5 + rng.uniform()), 0.2 * H, 0.7 * H, 300.0)
    emax = c1f * info["dv1"] / info["dt"] * ME / QE
    sigma = 2 * EPS0 * emax * 0.8
    n_tot = 1.6 * emax * EPS0 / QE
    amp = 2 * n_tot / (H * 2 * V1 * 2 * V2)
    return synth.random_f(shape, seed, amp), sigma


def twins(prec, shapes=SHAPES):
    """Two identical sets of grids with identical states."""
    a, b = [], []
    for q, s in enumerate(shapes):
        ga, gb = new_grid(s, prec), new_grid(s, prec)
        fa, sa = physics(ga, s, 100 + q)
        physics(gb, s, 100 + q)
        ga.set_state(fa, sa)
        gb.set_state(fa, sa)
        a.append(ga)
        b.append(gb)
    return a, b


def assert_same(ga, gb):
    assert np.array_equal(ga.get_f(), gb.get_f())
    assert ga.surface_charge() == gb.surface_charge()
    assert ga.step_count() == gb.step_count()
    la, lb = ga.ledger(), gb.ledger()
    assert la == lb
    na, ea, pa, sa = ga.moments()
    nb, eb, pb, sb = gb.moments()
    assert np.array_equal(na, nb) and np.array_equal(ea, eb) and pa == pb and sa == sb
    ha, hb = ga.history(10**6), gb.history(10**6)
    assert np.array_equal(ha, hb)


# either side of the batched finalize's seam: one warp per grid of at most
# 128 planes (four to a CTA), a block per 128 planes above
SEAM = [(2, 8, 8), (31, 16, 12), (32, 16, 16), (33, 12, 20), (127, 16, 16), (128, 24, 24),
        (129, 16, 16), (300, 16, 16)]


@pytest.mark.parametrize("prec", [fk.FK_F64, fk.FK_F32])
def test_finalize_warp_and_block_paths_equal_stepping_alone(prec):
    """Grids of 2 to 300 planes in one batch with the collision term on, so
    that the finalize also writes each plane's collision rates: 40 batch
    steps equal 40 steps of each grid alone (whose finalize is the block
    path for every size) bit for bit."""
    alone, batched = twins(prec, SEAM)
    for ga, gb in zip(alone, batched):
        info = ga.info()
        n_max = ga.moments()[0].max()
        lnL = 0.02 / (info["dt"] * oracle.nu_ee(n_max, 2.0, 1.0))
        for g in (ga, gb):
            g.set_collisions(2.0, lnL, True)
    with fk.Batch(batched) as b:
        # 3 + 2 blocks for the grids of 300 and 129 planes, 2 CTAs of warps
        # for the six others
        assert b.info()["finalize_ctas"] == 7
        b.step(40)
        for g in alone:
            g.step(40)
        assert b.sync() == [fk.FK_OK] * len(SEAM)
        for ga, gb in zip(alone, batched):
            assert_same(ga, gb)
    for g in alone + batched:
        g.close()


@pytest.mark.parametrize("prec", [fk.FK_F64, fk.FK_F32])
def test_batch_bitwise_equals_stepping_alone(prec):
    alone, batched = twins(prec)
    with fk.Batch(batched) as b:
        info = b.info()
        assert info["grids"] == len(SHAPES) and info["units"] >= len(SHAPES)
        b.step(40)  # one 32-step graph and 8 direct steps
        for g in alone:
            g.step(40)
        assert b.sync() == [fk.FK_OK] * len(SHAPES)
        for ga, gb in zip(alone, batched):
            assert_same(ga, gb)
        # another chunking: same states
        b.set_chunks([max(1, s[0] // 3) for s in SHAPES])
        b.step(7)
        for g in alone:
            g.step(7)
        for ga, gb in zip(alone, batched):
            assert_same(ga, gb)
    # released: the grids step alone again, still in step with their twins
    for g in alone + batched:
        g.step(5)
    for ga, gb in zip(alone, batched):
        assert_same(ga, gb)


def test_batch_matches_oracle_fp64():
    shapes = SHAPES[:3]
    grids, oras = [], []
    for q, s in enumerate(shapes):
        g = new_grid(s, fk.FK_F64)
        f0, sigma = physics(g, s, 7 + q)
        g.set_state(f0, sigma)
        o = oracle.Oracle(s[0], s[1], s[2], H, -V1, V1, -V2, V2, cfl=0.4)
        # the same physics on the oracle, read back from the grid's setters'
        # arguments (re-drawn from the same seed)
        rng = np.random.default_rng(7 + q)
        info = g.info()
        a2 = 0.15 * info["dv2"] / info["dt"]
        o.set_fields(-a2 * ME / QE, True, 0.0)
        o.set_see(2.0 + rng.uniform(0, 2), 300.0 + rng.uniform(0, 200), 1.0,
                  200.0 + rng.uniform(0, 300))
        o.set_source(1e7 * (0.5 + rng.uniform()), 0.2 * H, 0.7 * H, 300.0)
        o.set_state(f0, sigma)
        grids.append(g)
        oras.append(o)
    with fk.Batch(grids) as b:
        b.step(12)
        assert b.sync() == [fk.FK_OK] * len(shapes)
        for g, o in zip(grids, oras):
            o.step(12)
            fg, fo = g.get_f(), o.get_f()
            assert np.abs(fg - fo).sum() / np.abs(fo).sum() <= 1e-11
            assert abs(g.surface_charge() - o.surface_charge()) <= 1e-11 * abs(o.surface_charge())


@pytest.mark.parametrize("prec", [fk.FK_F32, fk.FK_F64])
def test_autotune_keeps_bitwise_equality(prec):
    alone, batched = twins(prec)
    with fk.Batch(batched) as b:
        taken = b.autotune(steps_per_trial=1)
        assert taken >= 2
        assert b.info()["steps"] == taken
        chunks = b.chunks()
        assert all(1 <= c <= s[0] for c, s in zip(chunks, SHAPES))
        b.step(33)
        for g in alone:
            g.step(taken + 33)
        assert b.sync() == [fk.FK_OK] * len(SHAPES)
        for ga, gb in zip(alone, batched):
            assert_same(ga, gb)


def test_member_grid_state_calls_refused():
    alone, batched = twins(fk.FK_F64, SHAPES[:2])
    g = batched[0]
    b = fk.Batch(batched)
    for call in (lambda: g.step(1), lambda: g.set_fields(-1e6), lambda: g.set_convergence(10, 1e-3),
                 lambda: g.set_see(3.0, 400.0), lambda: g.set_source(1.0, 0.0, H, 4.0),
                 lambda: g.set_f(np.zeros(g.shape)), lambda: g.set_surface_charge(0.0),
                 lambda: g.set_kernel_timing(True), lambda: fk.fk_destroy_grid(g.h),
                 lambda: fk.Batch([g])):
        with pytest.raises(fk.FkError) as e:
            call()
        assert e.value.status == fk.FK_ESTATE
    b.step(3)
    alone[0].step(3)
    assert_same(alone[0], g)  # getters see the batch's steps
    b.close()
    g.step(2)
    alone[0].step(2)
    assert_same(alone[0], g)


def test_invalid_batches_rejected():
    g64 = new_grid((8, 8, 8), fk.FK_F64)
    g32 = new_grid((8, 8, 8), fk.FK_F32)
    with pytest.raises(fk.FkError) as e:
        fk.Batch([g64, g32])
    assert e.value.status == fk.FK_EINVAL
    with pytest.raises(fk.FkError) as e:
        fk.Batch([g64, g64])
    assert e.value.status == fk.FK_EINVAL
    # a failed create leaves the grids free
    g64.step(1)
    g32.step(1)


def test_frozen_grid_does_not_stop_the_others():
    alone, batched = twins(fk.FK_F64, SHAPES[:3])
    bad = new_grid((16, 12, 12), fk.FK_F64)
    f0, _ = physics(bad, (16, 12, 12), 5)
    bad.set_f(f0)
    info = bad.info()
    # a wall charge whose field makes |c_1| > 1: the state is flagged at once
    sigma_bad = 2 * EPS0 * 3.0 * info["dv1"] / info["dt"] * ME / QE
    with pytest.raises(fk.FkError) as e:
        bad.set_surface_charge(sigma_bad)
    assert e.value.status == fk.FK_ECFL
    with fk.Batch(batched + [bad]) as b:
        b.step(35)
        st = b.sync()
        assert st[:3] == [fk.FK_OK] * 3 and st[3] == fk.FK_ECFL
        for g in alone:
            g.step(35)
        for ga, gb in zip(alone, batched):
            assert_same(ga, gb)
    # the frozen grid kept its state: step 0 and the f it was given
    lib = fk.load()
    import ctypes as C
    step, sat = C.c_int64(), C.c_int64()
    assert lib.fk_step_count(bad.h, C.byref(step), C.byref(sat)) == fk.FK_ECFL
    assert step.value == 0
    out = np.empty(bad.shape)
    assert lib.fk_get_f(bad.h, fk._dp(out)) == fk.FK_ECFL
    assert np.array_equal(out, f0)


def test_batch_kernel_timing():
    _, batched = twins(fk.FK_F32, SHAPES[:2])
    with fk.Batch(batched) as b:
        b.set_kernel_timing(True)
        b.step(3)
        n, ms = b.kernel_timing()
        assert n == 3 and ms > 0
        b.set_kernel_timing(False)
        b.step(32)
        assert b.sync() == [fk.FK_OK, fk.FK_OK]


def test_batch_scalars_equal_the_grid_getters():
    _, batched = twins(fk.FK_F32, SHAPES[:3])
    with fk.Batch(batched) as b:
        b.step(37)
        sig, step, sat, status = b.scalars()
        for q, g in enumerate(batched):
            assert sig[q] == g.surface_charge()
            assert (step[q], sat[q]) == g.step_count()
            assert status[q] == fk.FK_OK


@pytest.mark.parametrize("prec", [fk.FK_F32, fk.FK_F64])
def test_batch_moments_one_wait_equals_each_grids_getters(prec):
    """fk_batch_moments reads every grid's sigma, wall fluxes, n_e and E_x
    with one wait; the values equal each grid's own getters bit for bit."""
    a, _ = twins(prec)
    with fk.Batch(a) as b:
        b.step(5)
        nxs = [g.shape[0] for g in a]
        n_e = np.full(sum(nxs), np.nan)
        ex = np.full(sum(nxs), np.nan)
        sig, pe, see, _, _ = b.moments(n_e, ex)
        off = 0
        for q, g in enumerate(a):
            ne_g, ex_g, pe_g, see_g = g.moments()
            nx = g.shape[0]
            assert np.array_equal(n_e[off:off + nx], ne_g)
            assert np.array_equal(ex[off:off + nx], ex_g)
            assert sig[q] == g.surface_charge() and pe[q] == pe_g and see[q] == see_g
            off += nx
        # scalars only
        sig2, _, _, _, _ = b.moments()
        assert np.array_equal(sig2, sig)
    for g in a:
        g.close()


def test_pipelined_moments_equal_the_blocking_getter_step_by_step():
    """fk_batch_moments_enqueue / _collect (two pinned slots, the moments of
    step n read while step n + 1 runs) give, step by step, the same values
    as fk_batch_moments on a twin batch stepped the same way."""
    a, b = twins(fk.FK_F32)
    nx = sum(g.shape[0] for g in a)
    got, ref = [], []
    with fk.Batch(a) as ba, fk.Batch(b) as bb:
        with pytest.raises(fk.FkError) as ei:
            ba.moments_collect(0)
        assert ei.value.status == fk.FK_ESTATE
        slot = 0
        for step in range(6):
            ba.step(1)
            ba.moments_enqueue(slot)
            if step > 0:
                ne, ex = np.empty(nx), np.empty(nx)
                sig, pe, see, _, _ = ba.moments_collect(slot ^ 1, ne, ex)
                got.append((sig, pe, see, ne, ex))
            slot ^= 1
            bb.step(1)
            ne, ex = np.empty(nx), np.empty(nx)
            sig, pe, see, _, _ = bb.moments(ne, ex)
            ref.append((sig, pe, see, ne, ex))
        with pytest.raises(fk.FkError) as ei:
            ba.moments_enqueue(slot ^ 1)  # still full
        assert ei.value.status == fk.FK_ESTATE
        ne, ex = np.empty(nx), np.empty(nx)
        got.append(ba.moments_collect(slot ^ 1, ne, ex)[:3] + (ne, ex))
    assert len(got) == len(ref) == 6
    for g_, r_ in zip(got, ref):
        for x, y in zip(g_, r_):
            assert np.array_equal(x, y)
    for g in a + b:
        g.close()


def test_pipelined_moments_are_those_of_the_step_they_followed():
    """The packing kernel runs in order with the batch's steps and the copy
    on the batch's own copy stream: moments enqueued after step 3 and
    collected after 33 more steps (a graph replay among them) are step 3's."""
    a, b = twins(fk.FK_F64, SHAPES[:3])
    nx = sum(g.shape[0] for g in a)
    with fk.Batch(a) as ba, fk.Batch(b) as bb:
        ba.step(3)
        ba.moments_enqueue(1)
        ba.step(33)
        ne, ex = np.empty(nx), np.empty(nx)
        got = ba.moments_collect(1, ne, ex)[:3] + (ne, ex)
        bb.step(3)
        ne, ex = np.empty(nx), np.empty(nx)
        ref = bb.moments(ne, ex)[:3] + (ne, ex)
        for x, y in zip(got, ref):
            assert np.array_equal(x, y)
        bb.step(33)
        assert np.array_equal(ba.moments()[0], bb.moments()[0])
    for g in a + b:
        g.close()
