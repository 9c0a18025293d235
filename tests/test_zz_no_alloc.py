"""The allocation-free density moment (fk_density_moment_noalloc).

Some callers cannot let a library allocate device memory: code recorded
into a CUDA graph by stream capture (allocation is not allowed during
capture), applications whose own pool allocator owns all device memory, and
loops that cannot take the device-wide synchronisation an allocation may
cause.  For them the library offers one entry point whose scratch is a
fixed array compiled into the library.  This test checks it, called twice
in a row through the C ABI (a larger grid, then a smaller one, so that the
second call reads only slots it wrote itself), against the density moment
summed in FP64 with numpy, and against the grid API's fk_moments for the
same distributions.  It sits in a file of its own that pytest collects
last, and passes alone or after the other tests.
"""
import numpy as np
import pytest

from paper_2303_14119_gb300 import fk, synth

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 per-step tolerance used by the parity tests


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fk.load()
    return torch


def grid_moment(f, span=(6e7, 3e7)):
    nx, nv1, nv2 = f.shape
    g = fk.Grid(nx, nv1, nv2, 20e-6, -span[0], span[0], -span[1], span[1])
    g.set_f(f)
    ne = g.moments()[0]
    info = g.info()
    g.close()
    return ne, info["dv1"], info["dv2"]


def test_noalloc_moment_matches_fp64_sums_twice(torch):
    cases = [synth.random_f((64, 48, 48), 22, 0.5), synth.random_f((37, 24, 30), 21, 5.0)]
    stream = torch.cuda.current_stream()
    for f in cases:
        grid_ne, dv1, dv2 = grid_moment(f)
        ref = f.sum(axis=(1, 2)) * dv1 * dv2  # FP64, numpy
        f_dev = torch.from_numpy(f).cuda()
        n_e = torch.full((f.shape[0],), float("nan"), dtype=torch.float64, device="cuda")
        fk.fk_density_moment_noalloc(f_dev.data_ptr(), *f.shape, dv1, dv2, n_e.data_ptr(),
                                     stream.cuda_stream or None)
        torch.cuda.synchronize()
        got = n_e.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= TOL * np.abs(ref).max()
        assert np.abs(got - grid_ne).max() <= TOL * np.abs(ref).max()


def test_noalloc_rejects_sizes_beyond_scratch(torch):
    f_dev = torch.zeros(8, dtype=torch.float64, device="cuda")
    n_e = torch.zeros(8, dtype=torch.float64, device="cuda")
    too_many = fk.FK_NOALLOC_MAX_PARTIALS // 16 + 1
    with pytest.raises(fk.FkError) as ei:
        fk.fk_density_moment_noalloc(f_dev.data_ptr(), too_many, 1, 1, 1.0, 1.0, n_e.data_ptr())
    assert ei.value.status == fk.FK_EINVAL
    assert "scratch limit" in str(ei.value)
