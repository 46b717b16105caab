"""Failure paths on the GPU, driven by host-side fault injection
(bg_debug_inject_fault): the chosen device allocation, launch or copy fails
as if the CUDA runtime had refused it, without calling the runtime, so no
GPU ever faults.  Each test checks the error code, that nothing was written
where the contract says so, and that the library keeps working afterwards.
"""

import numpy as np
import pytest

from oracle import coracle as C
from paper_2502_07060_gb300 import inputs as G

pytestmark = pytest.mark.gpu

P = G.P_DEFAULT


@pytest.fixture(autouse=True)
def disarm():
    from paper_2502_07060_gb300 import bg
    yield
    for site in (bg.FAULT_DEVICE_ALLOC, bg.FAULT_LAUNCH, bg.FAULT_COPY):
        bg.inject_fault(site, 0, 0)


def _inputs(E=3000, n=7, d=6):
    import torch
    k, eps = G.fp_batch(55, E, n, d, d, P, 0, workers=1)
    ref, _ = C.amp_fp(k, eps, P, 0)
    return k, eps, ref, torch.from_numpy(k.view(np.int32)).cuda(), torch.from_numpy(eps.view(np.int32)).cuda()


def test_plan_allocation_failure_then_recovery():
    from paper_2502_07060_gb300 import bg
    table = np.zeros((3, 6), dtype=np.uint8)
    bg.inject_fault(bg.FAULT_DEVICE_ALLOC, 0, 1)
    with pytest.raises(bg.BGError) as e:
        bg.Plan(6, 4, 4, bg.FIELD_FP, P, bg.MOSTLY_MINUS, 1, table)
    assert e.value.status == 3                       # BG_ERR_NOMEM
    plan = bg.Plan(6, 4, 4, bg.FIELD_FP, P, bg.MOSTLY_MINUS, 1, table)
    assert plan.n_assign == 3


def test_launch_failure_leaves_outputs_untouched():
    import torch
    from paper_2502_07060_gb300 import bg
    k, eps, ref, kd, ed = _inputs()
    E = len(k)
    plan = bg.Plan(7, 6, 6, bg.FIELD_FP, P, bg.MOSTLY_MINUS)
    out = torch.full((E,), 12345, dtype=torch.int32, device="cuda")
    st = torch.full((E,), 7, dtype=torch.uint8, device="cuda")
    bg.inject_fault(bg.FAULT_LAUNCH, 0, 1)
    with pytest.raises(bg.BGError) as e:
        plan.eval(kd, ed, out=out, status=st)
    assert e.value.status == 4                       # BG_ERR_CUDA
    torch.cuda.synchronize()
    assert (out == 12345).all() and (st == 7).all()
    plan.eval(kd, ed, out=out, status=st)            # the plan stays usable
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), ref)
    with pytest.raises(bg.BGError):                  # the allocation-free path too
        bg.inject_fault(bg.FAULT_LAUNCH, 0, 1)
        plan.eval_noalloc(kd, ed, out=out, status=st)


@pytest.mark.parametrize("skip", [0, 3])
def test_host_pipeline_copy_failure_then_recovery(skip):
    """A copy that cannot be enqueued at chunk `skip` ends the call with
    BG_ERR_CUDA after the chunks already in flight have drained; the same
    staging buffer then serves a complete evaluation.  (Pageable buffers: a
    batch this small from page-locked ones is read in place, without copies.)"""
    import torch
    from paper_2502_07060_gb300 import bg
    k, eps, ref, _, _ = _inputs()
    E = len(k)
    plan = bg.Plan(7, 6, 6, bg.FIELD_FP, P, bg.MOSTLY_MINUS)
    hk = torch.from_numpy(k.view(np.int32).copy())
    he = torch.from_numpy(eps.view(np.int32).copy())
    hout = torch.empty(E, dtype=torch.int32)
    hst = torch.empty(E, dtype=torch.uint8)
    bg.inject_fault(bg.FAULT_COPY, skip, 1)
    with pytest.raises(bg.BGError) as e:
        plan.eval_host(hk, he, out=hout, status=hst, chunk=500)
    assert e.value.status == 4
    torch.cuda.synchronize()
    plan.eval_host(hk, he, out=hout, status=hst, chunk=500)
    torch.cuda.synchronize()
    assert np.array_equal(hout.numpy().view(np.uint32), ref)


def test_server_arena_failure_and_failed_request_in_a_mix():
    """bg_serve_create reports an arena that cannot be allocated; inside a
    running server one request whose copy fails completes with BG_ERR_CUDA
    from its wait, while every other request completes correctly."""
    import torch
    from paper_2502_07060_gb300 import bg
    bg.inject_fault(bg.FAULT_DEVICE_ALLOC, 0, 1)
    with pytest.raises(bg.BGError) as e:
        bg.Server(64 << 20, max_inflight=2)
    assert e.value.status == 3
    k, eps, ref, _, _ = _inputs(E=1200)
    plan = bg.Plan(7, 6, 6, bg.FIELD_FP, P, bg.MOSTLY_MINUS)
    srv = bg.Server(256 << 20, max_inflight=2)
    reqs = []
    bg.inject_fault(bg.FAULT_COPY, 2, 1)             # the third admitted request
    for i in range(6):
        lo, hi = 200 * i, 200 * (i + 1)
        hk = torch.from_numpy(k[lo:hi].view(np.int32)).pin_memory()
        he = torch.from_numpy(eps[lo:hi].view(np.int32)).pin_memory()
        ho = torch.empty(hi - lo, dtype=torch.int32).pin_memory()
        hs = torch.empty(hi - lo, dtype=torch.uint8).pin_memory()
        reqs.append((srv.submit(plan, hk, he, ho, hs), lo, hi, ho, hk, he))
    failed = 0
    for t, lo, hi, ho, *_ in reqs:
        try:
            assert srv.wait(t, 10000)
        except bg.BGError as err:
            assert err.status == 4
            failed += 1
            continue
        assert np.array_equal(ho.numpy().view(np.uint32), ref[lo:hi])
    assert failed == 1
    srv.close()
