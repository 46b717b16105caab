"""Complex FP64 with real momenta (BG_FIELD_C64_REAL), the physical
phase-space points of Sec. 3: the same amplitudes as the complex field under
the same tolerance against the double-double oracle (strict 1e-10 at n = 8,
d = D_s = 6), singular propagators flagged, state-assignment tables, and the
host pipeline and allocation-free entry point equal to bg_eval."""

import numpy as np
import pytest

from oracle import coracle as C
from paper_2502_07060_gb300 import inputs as G
from tests.test_gpu_parity import C64_CASES, TOL_C64, check_c64

pytestmark = pytest.mark.gpu


def _plan(n, d, Ds, metric, n_states=1, assign=None):
    from paper_2502_07060_gb300 import bg
    return bg.Plan(n, d, Ds, bg.FIELD_C64_REAL, 0, metric, n_states, assign)


def _real(k):
    import torch
    assert not np.any(k.imag)
    return torch.from_numpy(np.ascontiguousarray(k.real))


def run_c64r(k, eps, metric, n_states=1, assign=None):
    import torch
    E, n, d = k.shape
    plan = _plan(n, d, eps.shape[-1], metric, n_states, assign)
    out, st = plan.eval(_real(k).cuda(), torch.from_numpy(np.ascontiguousarray(eps)).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy(), st.cpu().numpy(), plan


@pytest.mark.parametrize("n,d,Ds,metric", C64_CASES)
def test_c64_real_within_tolerance(n, d, Ds, metric):
    E = 2 * 64 + 29                        # several blocks and a ragged tail
    k, eps = G.c64_batch(400 + n + d, E, n, d, Ds, metric)
    _, rst = C.amp_c64(k, eps, metric)
    out, st, plan = run_c64r(k, eps, metric)
    assert "field=c64_real" in plan.describe()
    assert np.array_equal(st, rst)
    check_c64(out, k, eps, metric, max_widened=0.02)   # measured: at most 2 of 157 points


def test_c64_real_metric_workload_strict():
    """n = 8, d = D_s = 6: every point within 1e-10 of the double-double
    value, no widening."""
    E = 20000
    k, eps = G.c64_batch(31, E, 8, 6, 6, 0)
    out, _, _ = run_c64r(k, eps, 0)
    hi, lo, _ = C.amp_c64dd(k, eps, 0)
    rel = np.abs((out - hi) - lo) / np.abs(hi)
    assert rel.max() <= TOL_C64, rel.max()


def test_c64_real_singular_status():
    """(k_1 + k_2)^2 = 0 exactly in FP64: status 1 and amplitude 0 for that
    point, the others unaffected."""
    k, eps = G.c64_batch(3, 130, 5, 4, 4, 0)
    k[77, 0] = [1.0, 1.0, 0.0, 0.0]
    k[77, 1] = [2.0, 2.0, 0.0, 0.0]
    out, st, _ = run_c64r(k, eps, 0)
    _, rst = C.amp_c64(k, eps, 0)
    assert st[77] == 1 and out[77] == 0 and rst[77] == 1
    assert np.array_equal(st, rst)
    keep = np.arange(len(k)) != 77
    check_c64(out[keep], k[keep], eps[keep], 0, max_widened=0.01)   # measured: none


def test_c64_real_state_assignment_table():
    n, d, Ds, E = 6, 4, 4, 45
    H = 1 << n
    assign = np.array([[(h >> l) & 1 for l in range(n)] for h in range(H)], dtype=np.uint8)
    k, eps = G.c64_batch(19, E, n, d, Ds, 1, S=2)
    out, _, _ = run_c64r(k, eps, 1, n_states=2, assign=assign)
    assert out.shape == (E, H)
    idx = np.arange(n)
    e_hs = [eps[:, idx, assign[h], :] for h in range(H)]
    his = np.stack([C.amp_c64dd(k, e_h, 1)[0] for e_h in e_hs], axis=1)
    spt = np.abs(his).max(axis=1)
    for h in range(H):
        check_c64(out[:, h], k, e_hs[h], 1, spt=spt, max_widened=0.0)   # measured: none


def test_c64_real_other_entry_points_match_eval():
    """bg_eval_host (host buffers, chunked) and bg_eval_noalloc give exactly
    bg_eval's results."""
    import torch
    n, d, E = 8, 6, 5003
    k, eps = G.c64_batch(72, E, n, d, d, 0)
    plan = _plan(n, d, d, 0)
    hk, he = _real(k).pin_memory(), torch.from_numpy(eps).pin_memory()
    ref, rst = plan.eval(hk.cuda(), he.cuda())
    out, st = plan.eval_host(hk, he, chunk=2000)
    torch.cuda.synchronize()
    assert torch.equal(out, ref.cpu()) and torch.equal(st, rst.cpu())
    out2, st2 = plan.eval_noalloc(hk.cuda(), he.cuda())
    torch.cuda.synchronize()
    assert torch.equal(out2, ref) and torch.equal(st2, rst)


def test_c64_real_rejects_complex_momenta():
    import torch
    k, eps = G.c64_batch(5, 8, 5, 4, 4, 0)
    plan = _plan(5, 4, 4, 0)
    with pytest.raises(TypeError):
        plan.eval(torch.from_numpy(k).cuda(), torch.from_numpy(eps).cuda())
