"""bg_eval_noalloc, the entry point for callers that cannot allocate device
memory (a framework owning the memory budget, latency-critical loops, code
where CUDA allocation calls are not permitted): through the C-ABI, two calls
in a row must reproduce bg_eval's results (bit-exact over F_p, within the
complex tolerance used by the other GPU tests).  This file is collected last
so that a failure here leaves every other GPU test already run."""

import numpy as np
import pytest

from paper_2502_07060_gb300 import inputs as G

pytestmark = pytest.mark.gpu


def _plan(field, n, d):
    from paper_2502_07060_gb300 import bg
    if field == "fp":
        return bg.Plan(n, d, d, bg.FIELD_FP, G.P_DEFAULT, bg.MOSTLY_MINUS)
    return bg.Plan(n, d, d, bg.FIELD_C64, 0, bg.MOSTLY_MINUS)


def _inputs(field, seed, E, n, d):
    import torch
    if field == "fp":
        k, e = G.fp_batch(seed, E, n, d, d, workers=1)
        return (torch.from_numpy(k.view(np.int32)).cuda(), torch.from_numpy(e.view(np.int32)).cuda())
    k, e = G.c64_batch(seed, E, n, d, d, workers=1)
    return torch.from_numpy(k).cuda(), torch.from_numpy(e).cuda()


@pytest.mark.parametrize("field,n,d,E", [("fp", 8, 6, 70000), ("fp", 12, 8, 3000), ("c64", 8, 6, 20000),
                                         ("fp", 12, 8, 300), ("c64", 8, 6, 200)])   # last two: one point per warp
def test_noalloc_matches_bg_eval_on_two_calls(field, n, d, E):
    import torch
    plan = _plan(field, n, d)
    for seed in (11, 12):                      # two calls in a row on the shared scratch
        k, e = _inputs(field, seed, E, n, d)
        out, st = plan.eval_noalloc(k, e)
        ref, rst = plan.eval(k, e)
        torch.cuda.synchronize()
        assert torch.equal(st, rst)
        if field == "fp":
            assert torch.equal(out, ref)
        else:
            a, b = out.cpu().numpy(), ref.cpu().numpy()
            assert (np.abs(a - b) <= 1e-10 * np.abs(b)).all()


def test_noalloc_with_an_assignment_table_matches_bg_eval():
    """Several state assignments per point (H = 3 rows of an explicit table,
    two states per leg): the table and H reach the kernel the same way as in
    bg_eval; two calls in a row, bit-exact over F_p."""
    import torch
    from paper_2502_07060_gb300 import bg
    n, d, S = 6, 4, 2
    table = np.array([[0] * n, [1] * n, [0, 1, 1, 0, 1, 0]], dtype=np.uint8)
    plan = bg.Plan(n, d, d, bg.FIELD_FP, G.P_DEFAULT, bg.MOSTLY_MINUS, S, table)
    for seed in (21, 22):
        k, e = G.fp_batch(seed, 2000, n, d, d, S=S, workers=1)
        kd = torch.from_numpy(k.view(np.int32)).cuda()
        ed = torch.from_numpy(e.view(np.int32)).cuda()
        out, st = plan.eval_noalloc(kd, ed)
        ref, rst = plan.eval(kd, ed)
        torch.cuda.synchronize()
        assert out.shape == (2000, 3)
        assert torch.equal(st, rst) and torch.equal(out, ref)


def test_noalloc_rejects_sizes_beyond_the_maximum():
    from paper_2502_07060_gb300 import bg
    import torch
    plan = _plan("fp", 8, 6)
    k, e = _inputs("fp", 1, 4, 8, 6)
    out = torch.empty(4, dtype=torch.int32, device="cuda")
    with pytest.raises(bg.BGError) as ei:
        bg._check(bg._lib.bg_eval_noalloc(plan.handle, 1 << 41, bg._ptr(k), bg._ptr(e), bg._ptr(out),
                                          bg._ptr(None), bg._stream_handle(None)))
    assert ei.value.status == bg.BG_ERR_INVALID_ARG
    assert "maximum" in str(ei.value)
