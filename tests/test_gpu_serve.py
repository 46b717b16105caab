"""Serving: every request's result equals the oracle (bit-exact over F_p, the
complex tolerance rule of reading G8) and is the same alone and in the mix
(identical results, since the same kernel runs), for host-staged, mapped
page-locked and device-resident buffers; waits time out with an error instead
of blocking, and admission respects the device memory budget."""

import numpy as np
import pytest

from paper_2502_07060_gb300 import inputs as G
from tests.gpu_oracle_check import check_complex, check_fp

pytestmark = pytest.mark.gpu

P = G.P_DEFAULT


def _request(bg, field, n, d, E, seed):
    import torch
    if field == "fp":
        k, e = G.fp_batch(seed, E, n, d, d, P, 0, workers=1)
        hk = torch.from_numpy(k.view(np.int32)).pin_memory()
        he = torch.from_numpy(e.view(np.int32)).pin_memory()
        plan = bg.Plan(n, d, d, bg.FIELD_FP, P)
    else:
        k, e = G.c64_batch(seed, E, n, d, d, 0, workers=1)
        if field == "c64r":                       # real momenta
            hk = torch.from_numpy(np.ascontiguousarray(k.real)).pin_memory()
        else:
            hk = torch.from_numpy(k).pin_memory()
        he = torch.from_numpy(e).pin_memory()
        plan = bg.Plan(n, d, d, bg.FIELD_C64_REAL if field == "c64r" else bg.FIELD_C64, 0)
    out = torch.empty(E, dtype=he.dtype).pin_memory()
    st = torch.empty(E, dtype=torch.uint8).pin_memory()
    return plan, hk, he, out, st


def _pageable(req):
    """The same request with pageable host buffers (staged through the arena)."""
    import torch
    plan, hk, he, out, st = req
    return (plan, torch.from_numpy(hk.numpy().copy()), torch.from_numpy(he.numpy().copy()),
            torch.empty(out.shape, dtype=out.dtype), torch.empty(st.shape, dtype=st.dtype))


def _oracle(plan, hk, he, out, st):
    """The served output against the oracle on the request's host inputs."""
    from paper_2502_07060_gb300 import bg
    k, e = hk.cpu().numpy(), he.cpu().numpy()
    if plan.field == bg.FIELD_FP:
        check_fp(out.cpu().numpy(), st.cpu().numpy(), k.view(np.uint32), e.view(np.uint32), P, 0)
    else:
        check_complex(out.cpu().numpy(), st.cpu().numpy(), k.astype(np.complex128), e, 0)


def _alone(plan, hk, he):
    import torch
    o, s = plan.eval(hk.cuda(), he.cuda())
    torch.cuda.synchronize()
    return o.cpu(), s.cpu()


def test_results_alone_equal_results_in_the_mix():
    import torch
    from paper_2502_07060_gb300 import bg
    rng = np.random.default_rng(3)
    reqs = []
    for i in range(40):
        field = "fp" if i % 2 else ("c64r" if i % 4 == 2 else "c64")
        n = int(rng.integers(4, 13))
        d = int(rng.choice([4, 6, 8]))
        E = int(np.exp(rng.uniform(0, np.log(4000))))
        reqs.append(_request(bg, field, n, d, max(E, 1), 500 + i))
    refs = [_alone(p, k, e) for p, k, e, _, _ in reqs]
    srv = bg.Server(256 << 20, max_inflight=6)
    tickets = [srv.submit(p, k, e, o, s) for p, k, e, o, s in reqs]
    for t in tickets[::-1]:                       # wait in reverse order
        assert srv.wait(t, timeout_ms=60000)
    for (p, k, e, o, s), (ro, rs) in zip(reqs, refs):
        assert torch.equal(o, ro), p.describe()
        assert torch.equal(s, rs)
        _oracle(p, k, e, o, s)
    st = srv.stats()
    assert st["completed"] == 40 and st["pending"] == 0 and st["bytes_in_use"] == 0
    assert st["peak_bytes"] <= 256 << 20
    srv.close()


def test_wait_times_out_then_completes():
    from paper_2502_07060_gb300 import bg
    big = [_request(bg, "c64", 12, 8, 65536, 900 + i) for i in range(2)]
    srv = bg.Server(1 << 30, max_inflight=1)
    t1 = srv.submit(*big[0])
    t2 = srv.submit(*big[1])
    assert srv.wait(t2, timeout_ms=0) is False          # still queued behind t1
    with pytest.raises(bg.BGError) as ei:
        bg._check(bg._lib.bg_serve_wait(srv._h, t2, 0))
    assert ei.value.status == bg.BG_ERR_TIMEOUT
    assert srv.wait(t1, timeout_ms=-1) and srv.wait(t2, timeout_ms=-1)
    ref = _alone(*big[1][:3])
    assert np.array_equal(big[1][3].numpy(), ref[0].numpy())
    srv.close()


def test_budget_admission():
    import torch
    from paper_2502_07060_gb300 import bg
    reqs = [_pageable(_request(bg, "fp", 8, 6, 20000, 700 + i)) for i in range(5)]

    def up(x):
        return (x + 255) // 256 * 256
    E = 20000
    one = (up(E * 8 * 6 * 4) * 2 + up(E * 4) + up(E) + up(reqs[0][0].workspace_size(E)))
    budget = int(one * 1.5)
    srv = bg.Server(budget, max_inflight=4)                       # room for one request at a time
    with pytest.raises(bg.BGError) as ei:                              # can never fit
        srv.submit(*_pageable(_request(bg, "fp", 8, 6, 200000, 1)))
    assert ei.value.status == bg.BG_ERR_INVALID_ARG
    ts = [srv.submit(*r) for r in reqs]
    assert all(srv.wait(t, timeout_ms=60000) for t in ts)
    for p, k, e, o, s in reqs:
        assert torch.equal(o, _alone(p, k, e)[0])
    assert one <= srv.stats()["peak_bytes"] <= budget
    srv.close()


def test_device_resident_inputs_and_outputs():
    """Requests may reference a pool of momenta and states kept on the device
    (and leave their outputs there): no copy and no arena bytes for those
    buffers, same results as bg_eval, mixed with staged host requests."""
    import torch
    from paper_2502_07060_gb300 import bg
    n, d, pool = 8, 6, 20000
    k, e = G.fp_batch(77, pool, n, d, d, P, 0)
    dk = torch.from_numpy(k.view(np.int32)).cuda()            # resident pool
    de = torch.from_numpy(e.view(np.int32)).cuda()
    plan = bg.Plan(n, d, d, bg.FIELD_FP, P)
    ref, rst = plan.eval(dk, de)
    torch.cuda.synchronize()
    ref = ref.cpu()
    check_fp(ref.numpy(), rst.cpu().numpy(), k, e, P, 0)
    srv = bg.Server(64 << 20, max_inflight=4)
    jobs = []
    rng = np.random.default_rng(4)
    for i in range(24):
        E = int(rng.integers(1, 3000))
        off = int(rng.integers(0, pool - E))
        if i % 3 == 0:                                       # staged host request
            hk = torch.from_numpy(k[off:off + E].view(np.int32)).pin_memory()
            he = torch.from_numpy(e[off:off + E].view(np.int32)).pin_memory()
            out = torch.empty(E, dtype=torch.int32).pin_memory()
            st = torch.empty(E, dtype=torch.uint8).pin_memory()
            t = srv.submit(plan, hk, he, out, st)
        else:                                                # resident inputs
            out = torch.empty(E, dtype=torch.int32, device="cuda" if i % 3 == 1 else "cpu")
            if out.device.type == "cpu":
                out = out.pin_memory()
            st = torch.empty(E, dtype=torch.uint8, device=out.device)
            if out.device.type == "cpu":
                st = st.pin_memory()
            t = srv.submit(plan, dk[off:off + E], de[off:off + E], out, st)
        jobs.append((t, off, E, out))
    for t, off, E, out in jobs:
        assert srv.wait(t, timeout_ms=60000)
        assert torch.equal(out.cpu(), ref[off:off + E])
    stats = srv.stats()
    assert stats["completed"] == 24 and stats["bytes_in_use"] == 0
    srv.close()


def test_page_locked_requests_are_served_in_place():
    """Page-locked host buffers are used in place: the kernel reads the inputs
    and writes the results over the host link, so no arena bytes beyond the
    kernel workspace are taken.  The same request from pageable host memory is
    staged through the arena.  Both give bg_eval's results."""
    import torch
    from paper_2502_07060_gb300 import bg

    def up(x):
        return (x + 255) // 256 * 256
    for field, n, d, E in (("fp", 8, 6, 1000), ("c64", 6, 4, 300), ("c64r", 5, 8, 257), ("fp", 12, 8, 1),
                           ("c64", 12, 8, 40000)):
        plan, hk, he, out, st = _request(bg, field, n, d, E, 1200 + n)
        ro, rs = _alone(plan, hk, he)
        ws = up(plan.workspace_size(E))
        srv = bg.Server(2 << 30, max_inflight=2)
        assert srv.wait(srv.submit(plan, hk, he, out, st), timeout_ms=60000)
        assert torch.equal(out, ro) and torch.equal(st, rs), plan.describe()
        _oracle(plan, hk, he, out, st)
        assert srv.stats()["peak_bytes"] == ws
        srv.close()
        _, pk, pe, po, ps = _pageable((plan, hk, he, out, st))
        assert not (pk.is_pinned() or pe.is_pinned() or po.is_pinned() or ps.is_pinned())
        srv = bg.Server(2 << 30, max_inflight=2)
        assert srv.wait(srv.submit(plan, pk, pe, po, ps), timeout_ms=60000)
        assert torch.equal(po, ro) and torch.equal(ps, rs), plan.describe()
        assert srv.stats()["peak_bytes"] > ws
        srv.close()


def test_two_threads_wait_on_one_ticket():
    """Several waiters on one ticket all get its result; the ticket is retired
    afterwards (a later wait reports an unknown ticket)."""
    import threading
    from paper_2502_07060_gb300 import bg
    plan, hk, he, out, st = _request(bg, "c64", 10, 6, 3000, 1300)
    srv = bg.Server(1 << 30, max_inflight=2)
    t = srv.submit(plan, hk, he, out, st)
    results = []

    def waiter():
        results.append(bg._lib.bg_serve_wait(srv._h, t, 60000))

    threads = [threading.Thread(target=waiter) for _ in range(3)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert results == [bg.BG_OK] * 3
    assert bg._lib.bg_serve_wait(srv._h, t, 0) == bg.BG_ERR_INVALID_ARG
    _oracle(plan, hk, he, out, st)
    srv.close()
