"""Memory safety of the recursion tables without compute-sanitizer: the
bounds-checked build of the library (-DBG_CHECKED) compares every table index
with its region's extent, records the first violation and redirects the
access into the thread's own table.  Small ragged batches through every
kernel family (compact kernel in all three table placements, odd dimensions,
four-dimensional legs, both complex fields, all-assignment plans in both
placements, the allocation-free and host-buffer paths) must report no
violation and agree with the oracle."""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_reports_no_out_of_range_index():
    from paper_2502_07060_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, BG_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_case.py")], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    rep = json.loads(r.stdout.strip().splitlines()[-1])
    assert rep["checked"], "the library loaded is not the checked build"
    assert rep["violation"] == 0, f"site {rep['violation'] >> 32}, index {rep['violation'] & 0xffffffff}"
    assert rep["mismatches"] == 0 and rep["cases"] > 50, rep
