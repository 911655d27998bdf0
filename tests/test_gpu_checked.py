"""The checked build (QPIC_CHECK): the same sources whose kernels test their
invariants -- at most one cell of motion per step, new cells inside the grid,
accumulator and tile-block indices inside their blocks, sort slots inside
their tile -- and report a violation as QPIC_ECHECK instead of trapping.
Runs covering the paths (staged tiles with drift, the global path of a short
box, the moving window with injection, the batched launch) must report none.
Its library is loaded in a child process (QPIC_CHECKED=1)."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent('''
    import sys
    sys.path[:0] = [%r, %r]
    import numpy as np
    import paper_2303_12874_gb300 as q
    import synth
    assert q.library_path().endswith("_build_check/libqpic.so"), q.library_path()
    w = synth.workload("cfg1_small")
    pl, la = w["plasma"], w["laser"]
    for sp in (1, 2, 3):                                   # 3: drift beyond the tile halo
        s = q.Sim(w["nz"], w["nr"], w["dz"], w["dr"], dt=0.13, sort_period=sp)
        s.load_plasma(pl["n0"], pl["z_start"], pl["ramp_len"], pl["ppc"])
        s.add_laser(la["a0"], la["w0"], la["fwhm"], la["z_centroid"], la["z_focus"])
        s.step(20)
    s = q.Sim(24, 19, 0.2, 0.5, dt=0.13)                    # shorter than two staged tiles
    s.load_plasma(0.02, 0.0, 0.0, (2, 2, 2))
    s.add_laser(2.0, 3.0, 3.0, 2.4, 2.4)
    s.step(10)
    win = q.Sim(256, 32, 0.2, 0.5, periodic=False, moving_window=True)
    win.load_plasma(0.01, 10.0, 5.0, (2, 2, 2))
    win.add_laser(2.0, 8.0, 10.0, 30.0, 30.0)
    win.step(40)
    runs = []
    for k in range(3):
        r = q.Sim(96 + 32 * k, 16, 0.2, 0.5, dt=0.12, tile_z=(16, 32, 8)[k], tile_r=8)
        r.load_plasma(0.01, 0.0, 0.0, (2, 2, 2))
        r.add_laser(1.5, 4.0, 6.0, 9.6, 9.6)
        runs.append(r)
    b = q.Batch(runs)
    b.step(2 * b.cycle)
    print("checked runs ok")
''') % (ROOT, os.path.join(ROOT, "tests"))


def test_checked_build_finds_no_violation():
    env = dict(os.environ, QPIC_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0 and "checked runs ok" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
