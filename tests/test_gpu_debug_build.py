"""The bounds-checking build (RUBIX_DEBUG=1; the stand-in for a race and
bounds checker, since compute-sanitizer is not used on these GPUs).

Its kernels check the shared-memory and record indices the deposit and the
adjoint compute (the fast-path rounds' nodes replayed with their own carry
arithmetic, the per-bin paths' slab entries, the adjoint's per-particle
output rows) and set a bit in the device error word instead of faulting.
On cases that take every slab path (tests/_debug_cases.py) the debug build
must report no error and give the release build's cubes and gradients bit
for bit (the checks read indices only)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def _run(kind, tmp_path):
    out = str(tmp_path / f"{kind}.npz")
    r = subprocess.run([sys.executable, os.path.join(HERE, "_debug_cases.py"), kind, out],
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(out)


def test_debug_build_reports_no_bounds_error_and_matches_release(tmp_path):
    dbg = _run("debug", tmp_path)
    rel = _run("release", tmp_path)
    assert sorted(dbg.files) == sorted(rel.files)
    for k in dbg.files:
        if k.endswith("/err"):
            assert int(dbg[k][0]) == 0 and int(rel[k][0]) == 0, (k, int(dbg[k][0]))
        else:
            assert np.array_equal(dbg[k], rel[k]), k
    # the cases took the per-bin / global paths where they were meant to
    assert int(dbg["high_velocity/slow"][0]) > 0
    assert int(dbg["centre_f32/slow"][0]) == 0
