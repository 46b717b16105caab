"""The lane-group kernel for small batches (one point per group of 4 or 8
lanes, one vector component per lane; or per team of the groups of a warp,
which evaluate the ranges of each length in parallel): bit-exact against the
oracle over F_p and within the complex tolerance of reading G8, for n =
4..12, every dimension pair, both metrics and primes, explicit
state-assignment tables and singular points, in both forms; the team form
gives the group form's values bit for bit; the default choice takes them for
small batches only, and the kernels agree at the switch-over size."""

import os

import numpy as np
import pytest

from oracle import coracle as C
from paper_2502_07060_gb300 import inputs as G
from tests.gpu_oracle_check import check_complex, check_fp

pytestmark = pytest.mark.gpu

P, PM = G.P_DEFAULT, G.P_MERSENNE


class _lanes:
    """BG_LANES for the plans created inside the block ("1" always, one point
    per group; "2" always, one point per team; "0" never)."""

    def __init__(self, v):
        self.v = v

    def __enter__(self):
        self.old = os.environ.get("BG_LANES")
        os.environ["BG_LANES"] = self.v

    def __exit__(self, *exc):
        if self.old is None:
            os.environ.pop("BG_LANES", None)
        else:
            os.environ["BG_LANES"] = self.old


def _dev(a):
    import torch
    if a.dtype == np.uint32:
        return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _eval(plan, k, e):
    import torch
    out, st = plan.eval(_dev(k), _dev(e))
    torch.cuda.synchronize()
    return out.cpu().numpy(), st.cpu().numpy()


FP_CASES = [(4, 4, 4, 0, P), (5, 4, 6, 1, PM), (6, 6, 6, 0, P), (7, 5, 7, 0, P), (8, 6, 6, 0, P),
            (8, 8, 8, 1, PM), (9, 4, 4, 1, PM), (10, 6, 8, 0, P), (11, 8, 8, 0, P), (12, 4, 4, 0, P),
            (12, 8, 8, 1, PM)]


MODES = ["1", "2"]                  # one point per group of lanes, per team


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,d,Ds,metric,p", FP_CASES)
def test_lanes_fp_bit_exact(n, d, Ds, metric, p, mode):
    from paper_2502_07060_gb300 import bg
    E = 3 * 16 + 5                              # several blocks of 16 points and a ragged tail
    k, e = G.fp_batch(1500 + 7 * n + d, E, n, d, Ds, p, metric, workers=1)
    with _lanes(mode):
        plan = bg.Plan(n, d, Ds, bg.FIELD_FP, p, metric)
    assert "lanes=%d" % (4 if Ds <= 4 else 8) in plan.describe()
    out, st = _eval(plan, k, e)
    check_fp(out, st, k, e, p, metric)


@pytest.mark.parametrize("field", ["c64", "c64r"])
@pytest.mark.parametrize("n,d,Ds,metric", [(4, 4, 4, 0), (6, 6, 6, 1), (8, 6, 6, 0), (9, 4, 8, 0), (12, 8, 8, 0)])
def test_lanes_complex_within_tolerance(field, n, d, Ds, metric):
    """Both forms against the oracle; the team form equals the group form bit
    for bit (every range runs the same operations in the same order)."""
    from paper_2502_07060_gb300 import bg
    E = 2 * 8 + 3
    k, e = G.c64_batch(1600 + 7 * n + d, E, n, d, Ds, metric, workers=1)
    fid = bg.FIELD_C64_REAL if field == "c64r" else bg.FIELD_C64
    kk = np.ascontiguousarray(k.real) if field == "c64r" else k
    outs = []
    for mode in MODES:
        with _lanes(mode):
            plan = bg.Plan(n, d, Ds, fid, 0, metric)
        out, st = _eval(plan, kk, e)
        check_complex(out, st, k, e, metric)
        outs.append((out, st))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("field", ["fp", "c64"])
def test_lanes_assignment_table(field, mode):
    from paper_2502_07060_gb300 import bg
    n, d, S, E = 6, 4, 2, 21
    table = np.array([[(h >> l) & 1 for l in range(n)] for h in range(1 << n)], dtype=np.uint8)
    if field == "fp":
        k, e = G.fp_batch(1700, E, n, d, d, PM, 1, S=S, workers=1)
        with _lanes(mode):
            plan = bg.Plan(n, d, d, bg.FIELD_FP, PM, bg.ALTERNATING, S, table)
        out, st = _eval(plan, k, e)
        check_fp(out, st, k, e, PM, 1, table)
    else:
        k, e = G.c64_batch(1700, E, n, d, d, 0, S=S, workers=1)
        with _lanes(mode):
            plan = bg.Plan(n, d, d, bg.FIELD_C64, 0, bg.MOSTLY_MINUS, S, table)
        out, st = _eval(plan, k, e)
        check_complex(out, st, k, e, 0, table, max_widened=0.0)


@pytest.mark.parametrize("mode", MODES)
def test_lanes_singular_point(mode):
    from paper_2502_07060_gb300 import bg
    from tests.test_oracle_c import singular_fp_point
    k1, e1 = singular_fp_point(3, 8, 6, 6)
    k, e = G.fp_batch(5, 40, 8, 6, 6, workers=1)
    k[17], e[17] = k1[0], e1[0]
    with _lanes(mode):
        plan = bg.Plan(8, 6, 6, bg.FIELD_FP, P)
    out, st = _eval(plan, k, e)
    assert st[17] == 1 and out[17] == 0
    check_fp(out, st, k, e, P, 0)


@pytest.mark.parametrize("field", ["fp", "c64"])
def test_default_choice_and_switch_over(field):
    """Without BG_LANES the plan takes the lanes kernel up to lanes_max_items
    work items and needs no workspace there; at and just above that size the
    two kernels give the same residues (F_p), or both meet the oracle's
    complex tolerance (their sums run in different orders)."""
    import torch
    from paper_2502_07060_gb300 import bg
    n, d = 7, 6
    fid = bg.FIELD_FP if field == "fp" else bg.FIELD_C64
    pp = P if field == "fp" else 0
    with _lanes("auto"):
        plan = bg.Plan(n, d, d, fid, pp)
    desc = dict(x.split("=", 1) for x in plan.describe().split())
    cut = int(desc["lanes_max_items"])
    assert desc["lanes"] == "8" and 0 < cut < 10 ** 7
    assert plan.workspace_size(cut) == 0 and plan.workspace_size(cut + 1) > 0
    for E in (cut, cut + 1):
        if field == "fp":
            k, e = G.fp_batch(1800, E, n, d, d, workers=1)
        else:
            k, e = G.c64_batch(1800, E, n, d, d, 0, workers=1)
        out, st = _eval(plan, k, e)
        with _lanes("0"):
            ref_plan = bg.Plan(n, d, d, fid, pp)
        ref, rst = _eval(ref_plan, k, e)
        assert np.array_equal(st, rst)
        if field == "fp":
            assert np.array_equal(out, ref)
        else:
            check_complex(out, st, k, e, 0)
            check_complex(ref, rst, k, e, 0)
    sample = np.arange(0, cut, max(1, cut // 300))
    if field == "fp":
        k, e = G.fp_batch(1800, cut, n, d, d, workers=1)
        check_fp(_eval(plan, k, e)[0][sample], None, k[sample], e[sample], P, 0)
    torch.cuda.synchronize()


@pytest.mark.parametrize("mode", MODES)
def test_lanes_host_pipeline_and_empty_batch(mode):
    """bg_eval_host with small chunks runs the lanes kernel per chunk; E = 0
    launches nothing."""
    import torch
    from paper_2502_07060_gb300 import bg
    n, d, E = 9, 6, 500
    k, e = G.fp_batch(1900, E, n, d, d, workers=1)
    with _lanes(mode):
        plan = bg.Plan(n, d, d, bg.FIELD_FP, P)
    out = torch.empty(E, dtype=torch.int32).pin_memory()
    st = torch.empty(E, dtype=torch.uint8).pin_memory()
    plan.eval_host(torch.from_numpy(k.view(np.int32)).pin_memory(), torch.from_numpy(e.view(np.int32)).pin_memory(),
                   out=out, status=st, chunk=70)
    torch.cuda.synchronize()
    check_fp(out.numpy(), st.numpy(), k, e, P, 0)
    o0, s0 = plan.eval(torch.empty((0, n, d), dtype=torch.int32, device="cuda"),
                       torch.empty((0, n, d), dtype=torch.int32, device="cuda"))
    assert o0.numel() == 0 and s0.numel() == 0
