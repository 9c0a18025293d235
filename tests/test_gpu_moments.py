"""Density moment and conservation ledger of FP32 grids against FP64 sums.

An FP32 grid stores and advects f in FP32; its moments, fluxes, surface
charge and ledger are FP64 (Sec. 2, Eqs. 12-14, 18).  The streaming step
kernel sums f^{n+1} in FP32: each thread adds its cells of a plane (at
most 8 vectors of 4) in sequence, the 32 lanes fold in a 5-level tree, the
producer warp adds the (at most 7) warps' sums, and the plane's sum is
converted to FP64 once.  All terms are >= 0, so the relative error per plane
is at most (31 + 5 + 6) * 2^-24 (about 2.5e-6); the direct-load kernel
keeps a compensated FP32 sum per thread.  Here n_e(x) of
fk_moments and the ledger's N are compared with FP64 numpy sums of the same
FP32 state read back with fk_get_f32.  The wall sums (Gamma_pe and
Gamma_see at x = 0, the outflow at x = h_max) are FP64 sums of the FP32
values in whole-CTA units and FP32 pairs with exact leading products (about
44 bits) in half-CTA units: both are compared with the oracle's FP64 sums
over the same FP32 state.  The FP32 ledger (every cumulative term, and
its closure) is compared with the FP64 oracle over 300 strongly coupled
steps.
"""
import numpy as np
import pytest

import oracle
from paper_2303_14119_gb300 import fk, synth

from test_gpu_parity import make_pair, strong_physics

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
BOUND = 42 * U32  # 31 additions per thread, 5 tree levels per warp, 6 over warps


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fk.load()


def numpy_density(f32, dv1, dv2):
    return f32.astype(np.float64).sum(axis=(1, 2)) * dv1 * dv2


@pytest.mark.parametrize("shape,layout", [((64, 48, 48), 2), ((96, 128, 200), 1),
                                           ((40, 256, 256), 1), ((3, 4, 7300), 0)])
def test_fp32_density_moment_against_fp64_sum(shape, layout):
    """layout: units per CTA of the streaming kernel (2: half-CTA units,
    1: whole-CTA units), 0: the direct-load kernel (rows too wide)."""
    g, o = make_pair(shape, prec=fk.FK_F32)
    info = g.info()
    if layout == 0:
        assert info["kernel"] == "direct"
    else:
        assert info["kernel"] == "stream" and info["units_per_cta"] == layout
    f0, sigma = strong_physics(g, o, shape, seed=21)
    g.set_state(f0, sigma)
    worst = 0.0
    for n in (1, 7, 40):
        g.step(n)
        f32 = g.get_f32()
        ne, _, _, _ = g.moments()
        ref = numpy_density(f32, o.info()["dv1"], o.info()["dv2"])
        err = np.abs(ne - ref) / ref
        worst = max(worst, float(err.max()))
        assert err.max() <= BOUND, (n, err.max())
        N = g.ledger()["N"]
        N_ref = ref.sum() * o.info()["dx"]
        assert abs(N / N_ref - 1.0) <= BOUND
    print("max per-plane relative error of n_e: %.3e (bound %.3e)" % (worst, BOUND))
    g.close()


@pytest.mark.parametrize("shape,layout", [((64, 48, 48), 2), ((96, 128, 200), 1),
                                           ((40, 256, 256), 1)])
def test_fp32_wall_fluxes_against_the_oracle_on_the_same_state(shape, layout):
    """Gamma_pe, Gamma_see and the vacuum outflow that the step kernel sums
    for the new state agree with the oracle's FP64 sums over the same FP32
    values to 1e-11 relative (plain FP32 sums would sit near 1e-7)."""
    g, o = make_pair(shape, prec=fk.FK_F32)
    assert g.info()["kernel"] == "stream" and g.info()["units_per_cta"] == layout
    f0, sigma = strong_physics(g, o, shape, seed=25)
    g.set_state(f0, sigma)
    worst = 0.0
    for n in (1, 6):
        g.step(n)
        _, _, pe, see = g.moments()
        vac = g.history(1)[-1][5]
        o.set_state(g.get_f(), g.surface_charge())
        _, _, pe_o, see_o = o.moments()
        vac_o = o.boundary_fluxes()["vac"]
        for name, got, ref in (("pe", pe, pe_o), ("see", see, see_o), ("vac", vac, vac_o)):
            assert ref != 0.0, name
            err = abs(got - ref) / abs(ref)
            worst = max(worst, err)
            assert err <= 1e-11, (name, n, got, ref)
    print("max relative error of the FP32 grid's wall sums: %.3e" % worst)
    g.close()


def test_fp32_ledger_against_the_oracle():
    """300 steps of the strong state (E_x changing sign, SEE, source) on an
    FP32 grid and on the oracle from the same (FP32-rounded) start: every
    cumulative ledger term within 1e-5 relative, and the FP32 grid's own
    balance N - N0 = emit - pe - vac - lv + inj closed to 1e-6 of N."""
    shape = (24, 40, 36)
    g, o = make_pair(shape, prec=fk.FK_F32)
    f0, sigma = strong_physics(g, o, shape, seed=23, c1f=0.05)
    g.set_state(f0, sigma)
    o.set_state(g.get_f(), sigma)
    g.step(300)
    o.step(300)
    lg, lo = g.ledger(), o.ledger()
    for key in ("N", "emit", "pe", "vac", "lv", "inj", "see"):
        den = max(abs(lo[key]), 1e-300)
        assert abs(lg[key] - lo[key]) / den <= 1e-5, (key, lg[key], lo[key])
    bal = lg["N0"] + lg["emit"] - lg["pe"] - lg["vac"] - lg["lv"] + lg["inj"]
    print("FP32 ledger closure: %.3e of N" % (abs(lg["N"] - bal) / lg["N"]))
    assert abs(lg["N"] - bal) <= 1e-6 * lg["N"]
    g.close()
