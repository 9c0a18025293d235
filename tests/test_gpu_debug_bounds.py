"""The debug-bounds build (FK_DEBUG_BOUNDS, libflashkin_bounds.so): the
streaming step kernel checks the index of every shared- and global-memory
access and bulk copy first, sets a sticky flag (FK_EBOUNDS) and skips the
access if one is out of range.  On the GPU, in a process of its own that
loads that library (FK_LIBRARY=bounds): the thin- and whole-tile layouts in
both precisions, a batch with tuned tiles and the split schemes step
without a failed check and still match the FP64 oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CASES = r"""
import numpy as np
from paper_2303_14119_gb300 import fk
assert fk.library_path().endswith("libflashkin_bounds.so")
fk.load()
from test_gpu_parity import make_pair, strong_physics, rel_l1
from test_gpu_tiles import setup as tile_setup
from test_gpu_strang import setup as split_setup
for prec, tol in ((fk.FK_F64, 1e-12), (fk.FK_F32, 3e-7)):
    for shape in ((23, 40, 30), (12, 96, 72), (40, 256, 256)):
        g, o = make_pair(shape, prec=prec)
        f0, sigma = strong_physics(g, o, shape, seed=5)
        g.set_state(f0, sigma)
        if shape[1] == 96:
            g.set_tile_rows(7)
        for n in (1, 1, 40):
            o.set_state(g.get_f(), g.surface_charge())
            g.step(n)
            o.step(n)
            g.sync()
            assert rel_l1(g.get_f(), o.get_f()) <= tol * (30 if n > 1 else 1), (shape, prec)
        g.close()
    grids = [tile_setup(s, prec, 80 + q, with_oracle=False)[0]
             for q, s in enumerate([(40, 256, 256), (24, 128, 200), (9, 8, 8), (30, 28, 26)])]
    with fk.Batch(grids) as b:
        b.autotune(1, tiles=True)
        b.step(40)
        assert b.sync() == [fk.FK_OK] * len(grids)
    for g in grids:
        g.close()
    for scheme in (fk.FK_SCHEME_LIE, fk.FK_SCHEME_STRANG):
        for shape in ((18, 40, 34), (12, 96, 72)):  # thin and whole-CTA tiles
            g, o = split_setup(shape, prec, 7, scheme=scheme)
            g.step(3)
            o.step(3)
            g.sync()
            assert rel_l1(g.get_f(), o.get_f()) <= 10 * tol, (scheme, shape)
            g.close()
print("bounds ok")
"""


def test_debug_bounds_build_steps_without_a_failed_check():
    env = dict(os.environ, FK_LIBRARY="bounds",
               PYTHONPATH=os.pathsep.join([ROOT, HERE, os.environ.get("PYTHONPATH", "")]))
    r = subprocess.run([sys.executable, "-c", CASES], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=1200)
    assert r.returncode == 0 and "bounds ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
