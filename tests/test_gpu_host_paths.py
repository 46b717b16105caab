"""bg_eval_host from host buffers gives exactly bg_eval's results on each of
its paths: the chunked copy pipeline (pageable buffers, or large batches
whose kernel the host link would bound: F_p at n = 8, d = 6 needs about
350 GB/s of input) and one launch reading and writing page-locked buffers in
place (small batches, and large batches heavy enough per point: complex FP64
at n = 8, d = 6 needs about 60 GB/s)."""

import numpy as np
import pytest

from paper_2502_07060_gb300 import inputs as G

pytestmark = pytest.mark.gpu

P = G.P_DEFAULT


def _check(plan, hk, he, chunk):
    import torch
    ref, rst = plan.eval(hk.cuda(), he.cuda())
    out, st = plan.eval_host(hk, he, chunk=chunk)
    torch.cuda.synchronize()
    assert torch.equal(out, ref.cpu()) and torch.equal(st, rst.cpu()), plan.describe()


@pytest.mark.parametrize("E,pinned", [(1 << 18, True), (3001, True), (3001, False)])
def test_fp_host_paths(E, pinned):
    import torch
    from paper_2502_07060_gb300 import bg
    k, e = G.fp_batch(31, E, 8, 6, 6, P, 0)
    plan = bg.Plan(8, 6, 6, bg.FIELD_FP, P)
    hk, he = torch.from_numpy(k.view(np.int32)), torch.from_numpy(e.view(np.int32))
    if pinned:
        hk, he = hk.pin_memory(), he.pin_memory()
    _check(plan, hk, he, chunk=max(1, E // 7))


def test_complex_real_momenta_large_batch_in_place():
    import torch
    from paper_2502_07060_gb300 import bg
    E = 1 << 16
    k, e = G.c64_batch(32, E, 8, 6, 6, 0)
    plan = bg.Plan(8, 6, 6, bg.FIELD_C64_REAL, 0)
    hk = torch.from_numpy(np.ascontiguousarray(k.real)).pin_memory()
    he = torch.from_numpy(e).pin_memory()
    _check(plan, hk, he, chunk=E // 4)


def test_host_link_rate_is_measured():
    """The in-place decision uses the rate of in-place reads over the host
    link measured on the device (logged under BG_LOG when a server is
    created): a plausible figure, reported as measured."""
    import os
    import re
    import subprocess
    import sys
    code = ("import torch; from paper_2502_07060_gb300 import bg; torch.zeros(1, device='cuda'); "
            "s = bg.Server(1 << 26, max_inflight=1); s.close()")
    env = dict(os.environ, BG_LOG="1")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    m = re.search(r"in-place reads over the host link ([0-9.]+) GB/s \((\w+)", r.stderr)
    assert m, r.stderr[-2000:]
    assert m.group(2) == "measured"
    assert 5.0 < float(m.group(1)) < 2000.0
