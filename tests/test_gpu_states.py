"""All S^n state assignments of a point in one recursion with shared
sub-currents (plan with assign == NULL, H == S^n): every output column equals
the oracle evaluated on that assignment's polarisations, bit-exact over F_p
and within the complex tolerance over C64, for S = 2 (all helicities), S = 3
and S = 4 (D_s - 2 transverse states), shared and global table placements,
ragged batches and singular points."""

import numpy as np
import pytest

from oracle import coracle as C
from paper_2502_07060_gb300 import inputs as G
from tests.test_gpu_parity import _env, check_c64

pytestmark = pytest.mark.gpu

P = G.P_DEFAULT
PM = G.P_MERSENNE


def _assignments(n, S):
    h = np.arange(S ** n)
    return np.stack([(h // S ** l) % S for l in range(n)], axis=1)       # [H][n], leg l's state


def _materialise(eps, assign):
    """eps [E][n][S][Ds] -> [H][E][n][Ds] with leg l taking state assign[h][l]."""
    n = eps.shape[1]
    return eps[:, np.arange(n)[None, :], assign, :].transpose(1, 0, 2, 3)


def _fp_reference(k, eps, p, metric, assign):
    e_h = _materialise(eps, assign)
    H, E = e_h.shape[:2]
    kk = np.broadcast_to(k, (H,) + k.shape).reshape(H * E, *k.shape[1:])
    ref, st = C.amp_fp(np.ascontiguousarray(kk), np.ascontiguousarray(e_h.reshape(H * E, *e_h.shape[2:])),
                       p, metric)
    return ref.reshape(H, E).T, st.reshape(H, E)[0]


def _run(field, k, eps, metric, p=0, table=None):
    import torch
    from paper_2502_07060_gb300 import bg
    E, n, d = k.shape
    S, Ds = eps.shape[2], eps.shape[3]
    fid = {"fp": bg.FIELD_FP, "c64": bg.FIELD_C64, "c64r": bg.FIELD_C64_REAL}[field]
    with _env(BG_TABLE=table):
        plan = bg.Plan(n, d, Ds, fid, p, metric, S, "all")
    if field == "fp":
        dk = torch.from_numpy(k.view(np.int32)).cuda()
        de = torch.from_numpy(eps.view(np.int32)).cuda()
    elif field == "c64r":
        dk = torch.from_numpy(np.ascontiguousarray(k.real)).cuda()
        de = torch.from_numpy(eps).cuda()
    else:
        dk = torch.from_numpy(k).cuda()
        de = torch.from_numpy(eps).cuda()
    out, st = plan.eval(dk, de)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    return (o.view(np.uint32) if field == "fp" else o), st.cpu().numpy(), plan


FP_CASES = [  # n, d, Ds, metric, p, S, E
    (4, 4, 4, 1, PM, 2, 301), (5, 4, 4, 1, PM, 2, 211), (6, 4, 4, 1, PM, 2, 130), (7, 4, 4, 1, PM, 2, 97),
    (8, 4, 4, 1, PM, 2, 70), (8, 6, 6, 0, P, 2, 45), (5, 6, 6, 0, P, 4, 37), (6, 6, 8, 0, P, 3, 23),
    (10, 4, 4, 1, PM, 2, 19), (12, 4, 4, 0, P, 2, 5), (6, 8, 8, 0, P, 4, 7),
]


@pytest.mark.parametrize("n,d,Ds,metric,p,S,E", FP_CASES)
def test_states_fp_bit_exact(n, d, Ds, metric, p, S, E):
    k, eps = G.fp_batch(900 + n * 7 + S, E, n, d, Ds, p, metric, S=S)
    out, st, plan = _run("fp", k, eps, metric, p)
    assert "kernel=states" in plan.describe()
    assert out.shape == (E, S ** n)
    ref, rst = _fp_reference(k, eps, p, metric, _assignments(n, S))
    assert np.array_equal(st, rst)
    assert np.array_equal(out, ref), plan.describe()


@pytest.mark.parametrize("n,S", [(6, 2), (8, 2), (5, 4)])
def test_states_fp_placements_agree(n, S):
    d = 4 if S == 2 else 6
    k, eps = G.fp_batch(77 + n, 33, n, d, d, P, 0, S=S)
    ref, _ = _fp_reference(k, eps, P, 0, _assignments(n, S))
    for table in ("shared", "global"):
        out, _, plan = _run("fp", k, eps, 0, P, table=table)
        assert f"table={table}" in plan.describe()
        assert np.array_equal(out, ref), plan.describe()


def test_states_fp_singular_point():
    from tests.test_oracle_c import singular_fp_point
    n, S = 6, 2
    k1, e1 = singular_fp_point(4, n, 6, 6)
    k, eps = G.fp_batch(8, 20, n, 6, 6, P, 0, S=S)
    k[13] = k1[0]
    eps[13, :, 0] = e1[0]
    out, st, _ = _run("fp", k, eps, 0, P)
    ref, rst = _fp_reference(k, eps, P, 0, _assignments(n, S))
    assert st[13] == 1 and rst[13] == 1 and not out[13].any()
    assert np.array_equal(out, ref) and np.array_equal(st, rst)


@pytest.mark.parametrize("field", ["c64", "c64r"])
@pytest.mark.parametrize("n,d,Ds,metric,S,E", [(5, 4, 4, 0, 2, 40), (7, 4, 4, 0, 2, 21), (6, 6, 6, 1, 4, 6)])
def test_states_c64_within_tolerance(field, n, d, Ds, metric, S, E):
    k, eps = G.c64_batch(600 + n + S, E, n, d, Ds, metric, S=S)
    out, st, plan = _run(field, k, eps, metric)
    assign = _assignments(n, S)
    e_h = _materialise(eps, assign)
    his = np.stack([C.amp_c64dd(k, np.ascontiguousarray(e), metric)[0] for e in e_h], axis=1)
    spt = np.abs(his).max(axis=1)
    for h in range(len(assign)):
        check_c64(out[:, h], k, np.ascontiguousarray(e_h[h]), metric, spt=spt, max_widened=0.0)   # measured: none
    assert not st.any()


def test_states_empty_batch_host_pipeline_and_rejections():
    import torch
    from paper_2502_07060_gb300 import bg
    n, S = 6, 2
    k, eps = G.fp_batch(5, 500, n, 4, 4, PM, 1, S=S)
    plan = bg.Plan(n, 4, 4, bg.FIELD_FP, PM, 1, S, "all")
    hk = torch.from_numpy(k.view(np.int32)).pin_memory()
    he = torch.from_numpy(eps.view(np.int32)).pin_memory()
    ref, rst = plan.eval(hk.cuda(), he.cuda())
    out, st = plan.eval_host(hk, he, chunk=128)
    torch.cuda.synchronize()
    assert torch.equal(out, ref.cpu()) and torch.equal(st, rst.cpu())
    e0, s0 = plan.eval(hk[:0].cuda(), he[:0].cuda())
    assert e0.shape == (0, S ** n)
    with pytest.raises(bg.BGError):                 # the static scratch path takes no such plan
        plan.eval_noalloc(hk.cuda(), he.cuda())
    import ctypes
    h = ctypes.c_void_p()                            # NULL assign needs H == S^n exactly
    assert bg._lib.bg_plan_create(n, 4, 4, bg.FIELD_FP, PM, 1, 2, 2 ** n - 1, None, ctypes.byref(h)) == 1
