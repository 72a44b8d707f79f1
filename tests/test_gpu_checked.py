"""The bounds-checked debug build (libsllbm_checked.so, -DSLLBM_CHECKED) over
every kernel family: no index that a step kernel takes from a record table or
derives from one leaves its range (the device status word stays 0), the same
kernel runs, and the result is the release build's.

The checked build replaces a memory checker for the step kernels: every
record slot, source population, boundary-state id, source node (per axis and
relative to the arriving node), gather-code cell and row-buffer slot is
range-checked.  It runs in a child process (one library per process).
Tolerances: 1e-6 (FP32) and 1e-13 (FP64) of each velocity's scale; the two
builds run the same arithmetic, so the difference is normally zero.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from tests import checked_runs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def runs(built_lib, tmp_path_factory):
    from paper_2412_09051_gb300 import build
    lib = build.build(checked=True)
    d = tmp_path_factory.mktemp("checked")
    out_c, out_r = str(d / "checked.npz"), str(d / "release.npz")
    r = subprocess.run([sys.executable, "-m", "tests.checked_runs", out_c, lib], cwd=ROOT,
                       capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    checked_runs.run(out_r)                       # the release library of this process
    return np.load(out_c), np.load(out_r)


def test_libraries_report_their_build(runs):
    c, r = runs
    assert int(c["build_flags"]) == 1             # SLLBM_BUILD_CHECKED
    assert int(r["build_flags"]) == 0


@pytest.mark.parametrize("key", checked_runs.keys())
def test_checked_build_keeps_every_index_in_range(runs, key):
    c, r = runs
    assert int(c[key + ".status"]) == 0, f"status bits {int(c[key + '.status']):#x}"
    assert int(r[key + ".status"]) == 0
    assert str(c[key + ".kernel"]) == str(r[key + ".kernel"])
    tol = 1e-13 if "fp64" in key else 1e-6
    worst = 0.0
    for part in ("f", "g"):
        a, b = c[key + "." + part], r[key + "." + part]
        scale = np.maximum(np.abs(b).max(axis=1, keepdims=True), 1e-300)
        worst = max(worst, float((np.abs(a - b) / scale).max()))
    assert worst <= tol, worst
    print(f"CHECKED {key} ({str(r[key + '.kernel'])}): status 0, max difference to release {worst:.1e}")
