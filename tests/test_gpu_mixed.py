"""Mixed-dimension plans on the GPU (bg_plan_create_mixed): legs flagged as
four-dimensional carry momenta and states that vanish beyond the first four
components (the loop-level setting of Sec. 2.3), and the kernel computes the
currents of ranges made of such legs with four components.

The values must be those of the ordinary plan on the same inputs (bit for
bit over F_p, where only products with exact zeros are skipped) and those of
the oracle; the complex fields within the parity tolerance of the oracle and
of the ordinary plan.
"""

import numpy as np
import pytest

from oracle import coracle as C
from paper_2502_07060_gb300 import inputs as G

from tests.test_gpu_parity import TOL_C64, _dev_c, _dev_u32, _env, check_c64

pytestmark = pytest.mark.gpu

P = G.P_DEFAULT
PM = G.P_MERSENNE


def _cut_mask(n):
    """Legs 1..n-2 four-dimensional: a tree at a one-loop cut with the two
    internal legs (0 and n-1) in d dimensions."""
    return ((1 << (n - 1)) - 1) & ~1


FP_CASES = [
    # n, d, Ds, metric, p, mask
    (5, 6, 6, 0, P, _cut_mask(5)), (6, 8, 8, 1, PM, _cut_mask(6)), (8, 6, 6, 0, P, _cut_mask(8)),
    (8, 8, 8, 0, P, 0b0101010), (8, 4, 6, 0, P, _cut_mask(8)), (9, 6, 8, 1, P, 0b011111100),
    (10, 6, 6, 0, P, _cut_mask(10)), (12, 8, 8, 0, P, _cut_mask(12)), (12, 6, 6, 1, PM, 0b000000000010),
    (7, 7, 7, 0, P, _cut_mask(7)),
]


def _plan(n, d, Ds, field, p, metric, mask, table=None):
    from paper_2502_07060_gb300 import bg
    with _env(BG_TABLE=table):
        return bg.Plan(n, d, Ds, field, p, metric, four_dim_legs=mask)


def _run(plan, kd, ed):
    import torch
    out, st = plan.eval(kd, ed)
    torch.cuda.synchronize()
    return out.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("n,d,Ds,metric,p,mask", FP_CASES)
def test_fp_mixed_bit_exact(n, d, Ds, metric, p, mask):
    from paper_2502_07060_gb300 import bg
    E = 3 * 128 + 41
    k, eps = G.fp_batch(700 + n + d, E, n, d, Ds, p, metric, workers=1, four_d=mask)
    ref, rst = C.amp_fp(k, eps, p, metric)
    kd, ed = _dev_u32(k), _dev_u32(eps)
    plain = bg.Plan(n, d, Ds, bg.FIELD_FP, p, metric)
    out_plain, st_plain = _run(plain, kd, ed)
    for table in (None, "global", "shared"):
        mixed = _plan(n, d, Ds, bg.FIELD_FP, p, metric, mask, table)
        desc = mixed.describe()
        if Ds > 4:
            assert f"four_dim_legs=0x{mask:x}" in desc, desc
        out, st = _run(mixed, kd, ed)
        out = out.view(np.uint32)
        assert np.array_equal(out, ref) and np.array_equal(st, rst), (table, desc)
        assert np.array_equal(out, out_plain.view(np.uint32)) and np.array_equal(st, st_plain)


@pytest.mark.parametrize("field", ["c64", "c64_real"])
@pytest.mark.parametrize("n,d,Ds,metric", [(6, 6, 6, 0), (8, 8, 8, 1), (10, 6, 6, 0)])
def test_c64_mixed_within_tolerance(field, n, d, Ds, metric):
    from paper_2502_07060_gb300 import bg
    E = 2 * 64 + 29
    mask = _cut_mask(n)
    k, eps = G.c64_batch(800 + n + d, E, n, d, Ds, metric, workers=1, four_d=mask)
    if field == "c64":
        f, kd = bg.FIELD_C64, _dev_c(k)
    else:
        import torch
        f, kd = bg.FIELD_C64_REAL, torch.from_numpy(np.ascontiguousarray(k.real)).cuda()
    ed = _dev_c(eps)
    out, st = _run(_plan(n, d, Ds, f, 0, metric, mask), kd, ed)
    out_plain, st_plain = _run(bg.Plan(n, d, Ds, f, 0, metric), kd, ed)
    assert np.array_equal(st, st_plain)
    check_c64(out, k, eps, metric, max_widened=0.02)   # measured: at most 1 of 157 points
    # separately compiled kernels: the same values up to FP64 rounding (FMA
    # contraction may differ), measured below 1e-11 relative
    rel = np.abs(out - out_plain) / np.abs(out_plain)
    assert rel.max() <= TOL_C64, rel.max()


def test_mixed_plan_through_noalloc_and_host_pipeline():
    """The allocation-free and host-buffer entry points run the mixed kernel
    as well and give the same residues."""
    import torch
    from paper_2502_07060_gb300 import bg
    n, d, Ds = 8, 8, 8
    E = 5000
    mask = _cut_mask(n)
    k, eps = G.fp_batch(901, E, n, d, Ds, P, 0, workers=1, four_d=mask)
    ref, _ = C.amp_fp(k, eps, P, 0)
    plan = _plan(n, d, Ds, bg.FIELD_FP, P, 0, mask)
    kd, ed = _dev_u32(k), _dev_u32(eps)
    out = torch.empty(E, dtype=torch.int32, device="cuda")
    st = torch.empty(E, dtype=torch.uint8, device="cuda")
    plan.eval_noalloc(kd, ed, out=out, status=st)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), ref)
    hk = torch.from_numpy(k.view(np.int32)).pin_memory()
    he = torch.from_numpy(eps.view(np.int32)).pin_memory()
    hout = torch.empty(E, dtype=torch.int32).pin_memory()
    hst = torch.empty(E, dtype=torch.uint8).pin_memory()
    plan.eval_host(hk, he, out=hout, status=hst, chunk=1234)
    torch.cuda.synchronize()
    assert np.array_equal(hout.numpy().view(np.uint32), ref)
