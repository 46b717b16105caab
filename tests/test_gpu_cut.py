"""Product plans (bg_plan_create_product: all assignments of per-leg state
sets, shared sub-currents, several points per warp when a point has few
versions) and the cut state sum bg_cut_trace, against the oracle: bit-exact
over F_p, within the complex tolerance over C64."""

import numpy as np
import pytest

from oracle import bg_oracle as O
from oracle import coracle as C
from paper_2502_07060_gb300 import inputs as G
from tests.test_gpu_parity import check_c64

pytestmark = pytest.mark.gpu

P = G.P_DEFAULT
PM = G.P_MERSENNE


def _table(radix):
    """[H][n] assignments in the product order (leg 0 fastest)."""
    H = int(np.prod(radix))
    h = np.arange(H)
    cols, w = [], 1
    for r in radix:
        cols.append((h // w) % r)
        w *= r
    return np.stack(cols, axis=1)


def _materialise(eps, table):
    n = eps.shape[1]
    return eps[:, np.arange(n)[None, :], table, :].transpose(1, 0, 2, 3)     # [H][E][n][Ds]


def _fp_ref(k, eps, p, metric, table):
    e_h = _materialise(eps, table)
    H, E = e_h.shape[:2]
    kk = np.ascontiguousarray(np.broadcast_to(k, (H,) + k.shape).reshape(H * E, *k.shape[1:]))
    ref, st = C.amp_fp(kk, np.ascontiguousarray(e_h.reshape(H * E, *e_h.shape[2:])), p, metric)
    return ref.reshape(H, E).T, st.reshape(H, E)[0]


def _fp_eval(k, eps, p, metric, radix):
    import torch
    from paper_2502_07060_gb300 import bg
    E, n, d = k.shape
    plan = bg.Plan(n, d, eps.shape[3], bg.FIELD_FP, p, metric, eps.shape[2], states_per_leg=radix)
    out, st = plan.eval(torch.from_numpy(k.view(np.int32)).cuda(), torch.from_numpy(eps.view(np.int32)).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32), st.cpu().numpy(), plan


RADIX_CASES = [  # n, d, S, radix, E
    (5, 6, 4, [4, 1, 1, 1, 4], 301),          # cut tree: internal legs first and last
    (6, 6, 4, [4, 1, 1, 1, 1, 4], 77),
    (7, 4, 2, [2, 1, 2, 1, 1, 2, 2], 65),
    (6, 8, 3, [1, 3, 1, 2, 1, 3], 50),
    (8, 4, 2, [2, 2, 1, 2, 2, 1, 2, 2], 33),
    (5, 4, 2, [1, 1, 1, 1, 1], 99),           # a single assignment, 32 points per warp
    (10, 6, 4, [4, 1, 1, 1, 1, 1, 1, 1, 1, 4], 21),
]


@pytest.mark.parametrize("n,d,S,radix,E", RADIX_CASES)
def test_product_plan_fp_bit_exact(n, d, S, radix, E):
    k, eps = G.fp_batch(1300 + n + S, E, n, d, d, P, 0, S=S)
    out, st, plan = _fp_eval(k, eps, P, 0, radix)
    assert "kernel=states" in plan.describe()
    H = int(np.prod(radix))
    assert out.shape == ((E, H) if H > 1 else (E,))
    out = out.reshape(E, H)
    ref, rst = _fp_ref(k, eps, P, 0, _table(radix))
    assert np.array_equal(st, rst)
    assert np.array_equal(out, ref), plan.describe()


def test_product_plan_uniform_equals_all_assignments():
    import torch
    from paper_2502_07060_gb300 import bg
    n, S = 7, 2
    k, eps = G.fp_batch(31, 200, n, 4, 4, PM, 1, S=S)
    a, _, _ = _fp_eval(k, eps, PM, 1, [S] * n)
    plan = bg.Plan(n, 4, 4, bg.FIELD_FP, PM, 1, S, "all")
    out, _ = plan.eval(torch.from_numpy(k.view(np.int32)).cuda(), torch.from_numpy(eps.view(np.int32)).cuda())
    assert np.array_equal(a, out.cpu().numpy().view(np.uint32))


@pytest.mark.parametrize("field", ["c64", "c64r"])
def test_product_plan_complex(field):
    import torch
    from paper_2502_07060_gb300 import bg
    n, d, S, radix, E = 6, 6, 4, [4, 1, 1, 1, 1, 4], 40
    k, eps = G.c64_batch(1400, E, n, d, d, 0, S=S)
    fid = bg.FIELD_C64_REAL if field == "c64r" else bg.FIELD_C64
    plan = bg.Plan(n, d, d, fid, 0, 0, S, states_per_leg=radix)
    kd = torch.from_numpy(np.ascontiguousarray(k.real) if field == "c64r" else k).cuda()
    out, st = plan.eval(kd, torch.from_numpy(eps).cuda())
    out = out.cpu().numpy()
    table = _table(radix)
    e_h = _materialise(eps, table)
    his = np.stack([C.amp_c64dd(k, np.ascontiguousarray(e), 0)[0] for e in e_h], axis=1)
    spt = np.abs(his).max(axis=1)
    for h in range(len(table)):
        check_c64(out[:, h], k, np.ascontiguousarray(e_h[h]), 0, spt=spt, max_widened=0.0)   # measured: none


@pytest.mark.parametrize("k_ring,S", [(1, 3), (2, 4), (4, 4), (5, 2), (3, 8)])
def test_cut_trace_fp_matches_literal_sum(k_ring, S):
    import torch
    from paper_2502_07060_gb300 import bg
    rng = np.random.default_rng(100 * k_ring + S)
    E = 300
    mats = [rng.integers(0, P, size=(E, S, S), dtype=np.uint64).astype(np.uint32) for _ in range(k_ring)]
    out = bg.cut_trace(bg.FIELD_FP, [torch.from_numpy(m.view(np.int32)).cuda() for m in mats], p=P)
    out = out.cpu().numpy().view(np.uint32)
    for e in range(0, E, 37):
        ref = O.cut_state_sum([[[O.GF(int(m[e, r, c]), P) for c in range(S)] for r in range(S)] for m in mats])
        assert int(out[e]) == int(ref)


def test_cut_trace_complex_matches_literal_sum():
    import torch
    from paper_2502_07060_gb300 import bg
    rng = np.random.default_rng(7)
    E, S, kr = 200, 4, 3
    mats = [rng.normal(size=(E, S, S)) + 1j * rng.normal(size=(E, S, S)) for _ in range(kr)]
    out = bg.cut_trace(bg.FIELD_C64, [torch.from_numpy(m).cuda() for m in mats]).cpu().numpy()
    for e in range(0, E, 13):
        ref = O.cut_state_sum([m[e].tolist() for m in mats])
        scale = np.prod([np.abs(m[e]).sum() for m in mats])
        assert abs(out[e] - ref) <= 1e-13 * scale


def test_cut_of_two_trees_end_to_end_fp():
    """Two five-gluon trees with S = 4 states on their internal legs (leg 0
    and leg 4): product plans give the [E][S*S] matrices, bg_cut_trace sums
    the ring; the oracle evaluates every assignment and the literal sum."""
    import torch
    from paper_2502_07060_gb300 import bg
    n, d, S, E = 5, 6, 4, 64
    radix = [S, 1, 1, 1, S]
    trees = []
    refs = []
    for t in range(2):
        k, eps = G.fp_batch(1500 + t, E, n, d, d, P, 0, S=S)
        out, _, _ = _fp_eval(k, eps, P, 0, radix)
        trees.append(torch.from_numpy(out.view(np.int32)).cuda())
        refs.append(_fp_ref(k, eps, P, 0, _table(radix))[0])
    ring = bg.cut_trace(bg.FIELD_FP, trees, p=P).cpu().numpy().view(np.uint32)
    for e in range(E):
        mats = [[[O.GF(int(r[e, so * S + si]), P) for si in range(S)] for so in range(S)] for r in refs]
        assert int(ring[e]) == int(O.cut_state_sum(mats))


def test_product_plan_rejections():
    import ctypes
    from paper_2502_07060_gb300 import bg
    h = ctypes.c_void_p()
    bad = (ctypes.c_uint8 * 5)(2, 0, 1, 1, 2)                # zero states on a leg
    assert bg._lib.bg_plan_create_product(5, 4, 4, bg.FIELD_FP, P, 0, 2, bad, ctypes.byref(h)) == 1
    bad = (ctypes.c_uint8 * 5)(3, 1, 1, 1, 2)                # more than n_states
    assert bg._lib.bg_plan_create_product(5, 4, 4, bg.FIELD_FP, P, 0, 2, bad, ctypes.byref(h)) == 1
    ok = (ctypes.c_uint8 * 5)(2, 1, 1, 1, 2)
    vp = (ctypes.c_void_p * 1)(None)
    assert bg._lib.bg_cut_trace(bg.FIELD_FP, P, 10, 1, 9, vp, None, None) == 1   # S > 8
    assert bg._lib.bg_plan_create_product(5, 4, 4, bg.FIELD_FP, P, 0, 2, ok, ctypes.byref(h)) == 0
    bg._lib.bg_plan_destroy(h)
