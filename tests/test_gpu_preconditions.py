"""The boundary's unchecked preconditions (canonical F_p residues, sum k = 0,
k_i^2 = 0, eps_i . k_i = 0) are checked by the checked build of the library:
a point that breaks one gets status 2 and amplitude 0 instead of a number that
is not the paper's recursion (the kernels use the current conservation these
preconditions imply, Sec. 2.2).  Bad data built on the host, not a device
fault: every access stays inside the caller's buffers."""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_reports_broken_preconditions():
    from paper_2502_07060_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, BG_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "precondition_case.py")], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    rep = json.loads(r.stdout.strip().splitlines()[-1])
    assert rep["checked"], "the library loaded is not the checked build"
    assert len(rep["cases"]) == 8
    for c in rep["cases"]:
        assert c["status2"] == [3, 7, 11, 13], c
        assert c["bad_out_zero"] and c["good_equal"] and c["good_status0"], c
