"""GPU parity: the CUDA path through the C-ABI against the oracle.

F_p: bit-exact against the C oracle (itself pinned against the exact Python
oracle).  C64: |A_gpu - A_ref| <= 1e-10 max(|A_ref|, S_pt) (reading G8) with
A_ref the double-double evaluation of the C oracle (pinned against mpmath);
on the few points where plain FP64 cannot reach 1e-10 (ill-conditioned
points, measured by the literal FP64 oracle's own error over leg orderings
and over inputs moved by one rounding) the bound is 8x that
FP64 noise floor, and the share of such points is bounded.  Sizes span several
thread blocks and a ragged tail; both shared-memory and global-scratch table
placements are exercised.
"""

import os

import numpy as np
import pytest

from oracle import coracle as C
from paper_2502_07060_gb300 import inputs as G

pytestmark = pytest.mark.gpu

P = G.P_DEFAULT
PM = G.P_MERSENNE
TOL_C64 = 1e-10


def _bg():
    from paper_2502_07060_gb300 import bg
    return bg


def _dev_u32(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def _dev_c(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


class _env:
    """Temporarily set BG_TABLE (read at plan creation)."""

    def __init__(self, **kv):
        self.kv = {k: v for k, v in kv.items() if v is not None}

    def __enter__(self):
        self.old = {k: os.environ.get(k) for k in self.kv}
        os.environ.update(self.kv)

    def __exit__(self, *exc):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def run_fp(k, eps, p, metric, n_states=1, assign=None, table=None):
    bg = _bg()
    E, n, d = k.shape
    Ds = eps.shape[-1]
    with _env(BG_TABLE=table):
        plan = bg.Plan(n, d, Ds, bg.FIELD_FP, p, metric, n_states, assign)
    out, st = plan.eval(_dev_u32(k), _dev_u32(eps))
    import torch
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32), st.cpu().numpy(), plan


def run_c64(k, eps, metric, n_states=1, assign=None):
    bg = _bg()
    E, n, d = k.shape
    Ds = eps.shape[-1]
    plan = bg.Plan(n, d, Ds, bg.FIELD_C64, 0, metric, n_states, assign)
    out, st = plan.eval(_dev_c(k), _dev_c(eps))
    import torch
    torch.cuda.synchronize()
    return out.cpu().numpy(), st.cpu().numpy(), plan


FP_CASES = [
    (4, 4, 4, 0, P), (5, 4, 4, 0, P), (5, 5, 6, 1, PM), (6, 4, 4, 1, PM), (6, 6, 6, 0, P),
    (7, 4, 6, 0, P), (7, 7, 7, 0, P), (8, 6, 6, 0, P), (8, 4, 4, 1, PM), (8, 8, 8, 0, P),
    (9, 6, 6, 0, P), (10, 4, 4, 0, P), (10, 6, 8, 1, P), (11, 8, 8, 0, P), (12, 4, 4, 1, PM),
    (12, 8, 8, 0, P),
]


@pytest.mark.parametrize("n,d,Ds,metric,p", FP_CASES)
def test_fp_bit_exact(n, d, Ds, metric, p):
    E = 3 * 128 + 37                       # several blocks and a ragged tail
    k, eps = G.fp_batch(100 + n * 3 + d, E, n, d, Ds, p, metric)
    ref, rst = C.amp_fp(k, eps, p, metric)
    out, st, plan = run_fp(k, eps, p, metric)
    assert np.array_equal(st, rst)
    assert np.array_equal(out, ref), plan.describe()


@pytest.mark.parametrize("n", [5, 8, 9, 12])
@pytest.mark.parametrize("table", ["shared", "global", "split"])
def test_fp_table_placements_agree(n, table):
    E = 1000
    k, eps = G.fp_batch(7 + n, E, n, 6, 6, P, 0)
    ref, _ = C.amp_fp(k, eps, P, 0)
    out, _, plan = run_fp(k, eps, P, 0, table=table)
    assert f"table={table}" in plan.describe()
    assert np.array_equal(out, ref)


@pytest.mark.parametrize("n,d,Ds,metric,p", [(8, 4, 8, 1, PM), (10, 8, 8, 0, P), (6, 6, 6, 1, PM)])
def test_fp_split_placement_bit_exact(n, d, Ds, metric, p):
    E = 3 * 128 + 37
    k, eps = G.fp_batch(500 + n, E, n, d, Ds, p, metric)
    ref, rst = C.amp_fp(k, eps, p, metric)
    out, st, plan = run_fp(k, eps, p, metric, table="split")
    assert "table=split" in plan.describe()
    assert np.array_equal(st, rst) and np.array_equal(out, ref)


@pytest.mark.parametrize("n,d,expect", [(6, 8, "split"), (8, 7, "split"), (8, 6, "global"), (12, 8, "global")])
def test_fp_default_placement(n, d, expect):
    """Without BG_TABLE, F_p plans with D_s = 8 keep the prefix sums, SA and
    1/P^2 in shared memory while that keeps the resident blocks of the global
    placement (n <= 8 here), and the result is the oracle's."""
    E = 2 * 97280 + 33                           # past one resident wave of threads
    k, eps = G.fp_batch(900 + n + d, E, n, d, d, P, 0)
    out, st, plan = run_fp(k, eps, P, 0)
    assert f"table={expect}" in plan.describe(), plan.describe()
    rng = np.random.default_rng(n)
    sample = np.unique(np.concatenate([rng.choice(E, 1500, replace=False), np.arange(E - 64, E)]))
    ref, rst = C.amp_fp(k[sample], eps[sample], P, 0)
    assert np.array_equal(out[sample], ref) and np.array_equal(st[sample], rst)


def c64_tolerance(k, eps, metric, hi, lo, spt=None):
    """Per-point tolerance of reading G8: 1e-10 max(|A|, S_pt) against the
    double-double value, widened only where FP64 itself cannot reach it: to 8x
    the FP64 noise floor nu_pt, the largest error of the literal FP64 oracle
    over three cyclic orderings of the legs (A is cyclically symmetric, so the
    orderings differ only in rounding) and over two copies of the inputs with
    every real component moved by one unit roundoff (relative 2^-53, seeded
    random signs: the spread of A under the rounding of its inputs, i.e. the
    point's conditioning).  Returns (tol, fraction widened)."""
    scale = np.abs(hi) if spt is None else np.maximum(np.abs(hi), spt)
    nu = np.zeros(len(hi))
    for r in range(3):
        a, _ = C.amp_c64(np.roll(k, -r, axis=1), np.roll(eps, -r, axis=1), metric)
        nu = np.maximum(nu, np.abs((a - hi) - lo))
    rng = np.random.default_rng(20250207)

    def moved(x):
        def part(v):
            return v * (1.0 + rng.choice([-1.0, 1.0], size=v.shape) * 2.0 ** -53)
        return np.ascontiguousarray(part(x.real) + 1j * part(x.imag))
    for _ in range(2):
        a, _ = C.amp_c64(moved(k), moved(eps), metric)
        nu = np.maximum(nu, np.abs((a - hi) - lo))
    tol = np.maximum(TOL_C64 * scale, 8.0 * nu)
    widened = float(np.mean(8.0 * nu > TOL_C64 * scale))
    return tol, widened


def check_c64(out, k, eps, metric, spt=None, max_widened=0.01):
    hi, lo, _ = C.amp_c64dd(k, eps, metric)
    tol, widened = c64_tolerance(k, eps, metric, hi, lo, spt)
    err = np.abs((out - hi) - lo)
    bad = err > tol
    rel = err / np.maximum(np.abs(hi), 1e-300)
    assert not bad.any(), f"{bad.sum()} points out of tolerance, max rel err {rel.max():.3e}"
    assert widened <= max_widened, f"{widened:.3%} of points ill-conditioned in FP64"
    return rel


C64_CASES = [(4, 4, 4, 0), (5, 4, 4, 0), (6, 6, 6, 0), (7, 4, 6, 1), (8, 6, 6, 0), (8, 8, 8, 1),
             (9, 4, 4, 0), (10, 6, 6, 0), (11, 8, 8, 0), (12, 4, 4, 0), (12, 8, 8, 1)]


@pytest.mark.parametrize("n,d,Ds,metric", C64_CASES)
def test_c64_within_tolerance(n, d, Ds, metric):
    E = 2 * 64 + 29
    k, eps = G.c64_batch(200 + n + d, E, n, d, Ds, metric)
    _, rst = C.amp_c64(k, eps, metric)
    out, st, plan = run_c64(k, eps, metric)
    assert np.array_equal(st, rst)
    check_c64(out, k, eps, metric, max_widened=0.02)   # measured: at most 3 of 157 points


def test_c64_metric_workload_strict():
    """n = 8, d = D_s = 6 (the benchmark workload): every point within 1e-10
    of the double-double value, no widening."""
    E = 20000
    k, eps = G.c64_batch(31, E, 8, 6, 6, 0)
    out, _, _ = run_c64(k, eps, 0)
    hi, lo, _ = C.amp_c64dd(k, eps, 0)
    rel = np.abs((out - hi) - lo) / np.abs(hi)
    assert rel.max() <= TOL_C64, rel.max()


def test_golden_rational_fixtures_mod_p():
    """Exact rational amplitudes written by the oracle (tests/golden), reduced
    mod p, are reproduced bit-exactly on the GPU."""
    import json
    from fractions import Fraction
    path = os.path.join(os.path.dirname(__file__), "golden", "rational_amplitudes.json")
    for c in json.load(open(path))["cases"]:
        for p in (P, PM):
            def red(x):
                f = Fraction(x)
                return f.numerator % p * pow(f.denominator % p, -1, p) % p
            k = np.array([[[red(x) for x in v] for v in c["k"]]], dtype=np.uint32)
            eps = np.array([[[red(x) for x in v] for v in c["eps"]]], dtype=np.uint32)
            out, st, _ = run_fp(k, eps, p, c["metric"])
            assert st[0] == 0 and int(out[0]) == red(c["amplitude"])


def test_singular_propagator_status_on_gpu():
    from tests.test_oracle_c import singular_fp_point
    k1, e1 = singular_fp_point(3, 8, 6, 6)
    k, eps = G.fp_batch(5, 200, 8, 6, 6)
    k[77], eps[77] = k1[0], e1[0]
    out, st, _ = run_fp(k, eps, P, 0)
    ref, rst = C.amp_fp(k, eps, P, 0)
    assert st[77] == 1 and out[77] == 0 and rst[77] == 1
    assert np.array_equal(out, ref) and np.array_equal(st, rst)


@pytest.mark.parametrize("field", ["fp", "c64"])
def test_state_assignment_table(field):
    """S = 2 states per leg and all H = 2^n assignments in one launch equal
    the oracle on each explicitly materialised assignment."""
    n, d, Ds, E = 6, 4, 4, 45
    H = 1 << n
    assign = np.array([[(h >> l) & 1 for l in range(n)] for h in range(H)], dtype=np.uint8)
    if field == "fp":
        k, eps = G.fp_batch(9, E, n, d, Ds, PM, 1, S=2)
        out, st, _ = run_fp(k, eps, PM, 1, n_states=2, assign=assign)
    else:
        k, eps = G.c64_batch(9, E, n, d, Ds, 0, S=2)
        out, st, _ = run_c64(k, eps, 0, n_states=2, assign=assign)
    assert out.shape == (E, H)
    idx = np.arange(n)
    refs = []
    for h in range(H):
        e_h = eps[:, idx, assign[h], :]
        if field == "fp":
            ref, _ = C.amp_fp(k, e_h, PM, 1)
            assert np.array_equal(out[:, h], ref)
        else:
            refs.append(e_h)
    if field == "c64":
        his = np.stack([C.amp_c64dd(k, e_h, 0)[0] for e_h in refs], axis=1)
        spt = np.abs(his).max(axis=1)
        for h in range(H):
            check_c64(out[:, h], k, refs[h], 0, spt=spt, max_widened=0.0)   # measured: none


def test_ward_identity_on_gpu_full_batch():
    """Property at any size: eps_i -> k_i gives exactly 0 for every point."""
    E, n, d = 1 << 16, 8, 6
    k, eps = G.fp_batch(12, E, n, d, d)
    for i in (0, 3, n - 1):
        e2 = eps.copy()
        e2[:, i, :] = k[:, i, :]
        out, st, _ = run_fp(k, e2, P, 0)
        assert not out.any()


def test_empty_and_single_point():
    import torch
    bg = _bg()
    plan = bg.Plan(8, 6, 6, bg.FIELD_FP, P)
    e = torch.empty((0, 8, 6), dtype=torch.int32, device="cuda")
    out, st = plan.eval(e, e)
    assert out.numel() == 0
    k, eps = G.fp_batch(1, 1, 8, 6, 6)
    out, st, _ = run_fp(k, eps, P, 0)
    ref, _ = C.amp_fp(k, eps, P, 0)
    assert np.array_equal(out, ref)


def test_eval_rejects_host_pointers_and_small_workspace():
    import torch
    bg = _bg()
    plan = bg.Plan(8, 6, 6, bg.FIELD_FP, P)
    k = torch.zeros((4, 8, 6), dtype=torch.int32)             # host tensors
    with pytest.raises(bg.BGError) as ei:
        plan.eval(k, k, out=torch.zeros(4, dtype=torch.int32, device="cuda"))
    assert ei.value.status == bg.BG_ERR_INVALID_ARG
    c = bg.Plan(8, 6, 6, bg.FIELD_C64, 0)
    E = 20000                                                  # above the lane kernel's batch sizes
    kd = torch.zeros((E, 8, 6), dtype=torch.complex128, device="cuda")
    need = c.workspace_size(E)
    assert need > 0
    small = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(bg.BGError):
        c.eval(kd, kd, workspace=small)


def test_full_size_metric_workload_sampled():
    """The benchmark workload (n = 8, d = D_s = 6, 2^22 points, F_p and C64) in
    the benchmark's launch configuration; sampled points against the oracle."""
    E = 1 << 22
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(E, 4096, replace=False))
    k, eps = G.fp_batch(2025, E, 8, 6, 6, P, 0)
    out, st, _ = run_fp(k, eps, P, 0)
    ref, rst = C.amp_fp(k[sample], eps[sample], P, 0)
    assert np.array_equal(out[sample], ref) and np.array_equal(st[sample], rst)
    del k, eps
    kc, ec = G.c64_batch(2026, E, 8, 6, 6, 0)
    outc, _, _ = run_c64(kc, ec, 0)
    check_c64(outc[sample], kc[sample], ec[sample], 0, max_widened=0.0)


def _resident_threads(plan):
    import torch
    desc = dict(x.split("=", 1) for x in plan.describe().split() if "=" in x)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    return int(desc["blocks_per_sm"]) * int(desc["block"]) * sms


@pytest.mark.parametrize("field,table", [("fp", None), ("fp", "split"), ("c64", None), ("c64r", None)])
def test_several_points_per_thread(field, table):
    """Batches of a little over two resident waves with a ragged last warp: the
    table region of a thread serves several points in turn (its lines are
    dropped from L2 between points), so points after the first of a thread,
    and the last partial warp, are checked against the oracle."""
    import torch
    bg = _bg()
    n, d = 8, 6
    with _env(BG_TABLE=table):
        if field == "fp":
            plan = bg.Plan(n, d, d, bg.FIELD_FP, P, 0)
        else:
            plan = bg.Plan(n, d, d, bg.FIELD_C64_REAL if field == "c64r" else bg.FIELD_C64, 0, 0)
    if table:
        assert "table=" + table in plan.describe()
    else:
        assert "table=global" in plan.describe()
    R = _resident_threads(plan)
    E = 2 * R + 77
    rng = np.random.default_rng(7)
    sample = np.unique(np.concatenate([rng.choice(np.arange(R, E), 1500, replace=False), np.arange(E - 96, E)]))
    if field == "fp":
        k, e = G.fp_batch(2100, E, n, d, d, P, 0)
        out, st = plan.eval(_dev_u32(k), _dev_u32(e))
        torch.cuda.synchronize()
        ref, rst = C.amp_fp(k[sample], e[sample], P, 0)
        assert np.array_equal(out.cpu().numpy().view(np.uint32)[sample], ref)
        assert np.array_equal(st.cpu().numpy()[sample], rst)
    else:
        k, e = G.c64_batch(2101, E, n, d, d, 0)
        kd = torch.from_numpy(np.ascontiguousarray(k.real)).cuda() if field == "c64r" else _dev_c(k)
        out, st = plan.eval(kd, _dev_c(e))
        torch.cuda.synchronize()
        _, rst = C.amp_c64(k[sample], e[sample], 0)
        assert np.array_equal(st.cpu().numpy()[sample], rst)
        check_c64(out.cpu().numpy()[sample], k[sample], e[sample], 0, max_widened=0.01)


@pytest.mark.parametrize("field,pinned", [("fp", True), ("fp", False), ("c64", True)])
def test_eval_host_pipeline_matches_device_eval(field, pinned):
    """bg_eval_host (host buffers, chunked and double buffered) returns exactly
    what bg_eval returns on device copies of the same inputs; chunk sizes
    leave a ragged last chunk."""
    import torch
    bg = _bg()
    n, d, E = 8, 6, 10007
    if field == "fp":
        k, e = G.fp_batch(71, E, n, d, d)
        hk, he = torch.from_numpy(k.view(np.int32)), torch.from_numpy(e.view(np.int32))
        plan = bg.Plan(n, d, d, bg.FIELD_FP, P)
    else:
        k, e = G.c64_batch(71, E, n, d, d)
        hk, he = torch.from_numpy(k), torch.from_numpy(e)
        plan = bg.Plan(n, d, d, bg.FIELD_C64, 0)
    if pinned:
        hk, he = hk.pin_memory(), he.pin_memory()
    ref, rst = plan.eval(hk.cuda(), he.cuda())
    for chunk in (4096, 3000, E):
        out, st = plan.eval_host(hk, he, chunk=chunk)
        torch.cuda.synchronize()
        assert torch.equal(out, ref.cpu()) and torch.equal(st, rst.cpu())


def test_plans_sharing_a_kernel_keep_their_shared_memory():
    """A later plan with a smaller shared-memory table on the same kernel must
    not lower the limit an earlier plan relies on."""
    bg = _bg()
    with _env(BG_TABLE="shared"):
        big = bg.Plan(7, 6, 6, bg.FIELD_FP, P)
        small = bg.Plan(4, 6, 6, bg.FIELD_FP, P)
    assert "table=shared" in big.describe() and "table=shared" in small.describe()
    for plan, n in ((big, 7), (small, 4)):
        k, eps = G.fp_batch(5 + n, 300, n, 6, 6, P, 0)
        ref, _ = C.amp_fp(k, eps, P, 0)
        out, _ = plan.eval(_dev_u32(k), _dev_u32(eps))
        assert np.array_equal(out.cpu().numpy().view(np.uint32), ref)
