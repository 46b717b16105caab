"""Parity at the benchmark configurations' full sizes, in the launch
configuration bench.py times, on sampled outputs the oracle computes one by
one:
  * every helicity of n = 10 gluons, d = D_s = 4, two states per leg, 2^20
    points (F_p, p = 2^31 - 1, alternating metric), 32 sampled points with
    all 1024 assignments each, bit-exact;
  * complex FP64 with real momenta, all 256 helicities of n = 8 on 2^20
    points, 16 sampled points against the double-double oracle;
  * d-dimensional F_p, n = 8, d = D_s = 8, 2^22 points (p = 2^31 - 19),
    4096 sampled points, bit-exact.
(n = 8, d = D_s = 6 at 2^22 points: test_gpu_parity.test_full_size_metric_workload_sampled.)
"""

import numpy as np
import pytest

from oracle import coracle as C
from paper_2502_07060_gb300 import inputs as G
from tests.test_gpu_parity import check_c64
from tests.test_gpu_states import _assignments, _fp_reference, _materialise

pytestmark = pytest.mark.gpu

P = G.P_DEFAULT
PM = G.P_MERSENNE


def test_all_helicities_n10_full_size_sampled():
    import torch
    from paper_2502_07060_gb300 import bg
    n, E, S = 10, 1 << 20, 2
    k, eps = G.fp_batch(4000 + n, E, n, 4, 4, PM, 1, S=S)
    plan = bg.Plan(n, 4, 4, bg.FIELD_FP, PM, bg.ALTERNATING, S, "all")
    out, st = plan.eval(torch.from_numpy(k.view(np.int32)).cuda(), torch.from_numpy(eps.view(np.int32)).cuda())
    rng = np.random.default_rng(11)
    sample = np.sort(rng.choice(E, 32, replace=False))
    idx = torch.from_numpy(sample).cuda()
    got = out[idx].cpu().numpy().view(np.uint32)
    gst = st[idx].cpu().numpy()
    del out, st
    ref, rst = _fp_reference(k[sample], eps[sample], PM, 1, _assignments(n, S))
    assert np.array_equal(gst, rst)
    assert np.array_equal(got, ref)


def test_all_helicities_complex_full_size_sampled():
    import torch
    from paper_2502_07060_gb300 import bg
    n, E, S = 8, 1 << 20, 2
    k, eps = G.c64_batch(4000 + n, E, n, 4, 4, 0, S=S)
    plan = bg.Plan(n, 4, 4, bg.FIELD_C64_REAL, 0, bg.MOSTLY_MINUS, S, "all")
    out, _ = plan.eval(torch.from_numpy(np.ascontiguousarray(k.real)).cuda(), torch.from_numpy(eps).cuda())
    rng = np.random.default_rng(12)
    sample = np.sort(rng.choice(E, 16, replace=False))
    got = out[torch.from_numpy(sample).cuda()].cpu().numpy()          # [16][256]
    del out
    assign = _assignments(n, S)
    e_h = _materialise(eps[sample], assign)                            # [H][16][n][Ds]
    H = len(assign)
    kk = np.broadcast_to(k[sample], (H,) + k[sample].shape).reshape(H * 16, n, 4)
    ee = e_h.reshape(H * 16, n, 4)
    hi, _, _ = C.amp_c64dd(np.ascontiguousarray(kk), np.ascontiguousarray(ee), 0)
    spt = np.repeat(np.abs(hi.reshape(H, 16)).max(axis=0)[None, :], H, axis=0).reshape(-1)
    check_c64(got.T.reshape(-1), np.ascontiguousarray(kk), np.ascontiguousarray(ee), 0, spt=spt,
              max_widened=0.01)


def test_d8_full_size_sampled():
    import torch
    from paper_2502_07060_gb300 import bg
    n, d, E = 8, 8, 1 << 22
    k, eps = G.fp_batch(5208, E, n, d, d, P, 0)
    plan = bg.Plan(n, d, d, bg.FIELD_FP, P, bg.MOSTLY_MINUS)
    out, st = plan.eval(torch.from_numpy(k.view(np.int32)).cuda(), torch.from_numpy(eps.view(np.int32)).cuda())
    rng = np.random.default_rng(13)
    sample = np.sort(rng.choice(E, 4096, replace=False))
    got = out.cpu().numpy().view(np.uint32)[sample]
    gst = st.cpu().numpy()[sample]
    ref, rst = C.amp_fp(k[sample], eps[sample], P, 0)
    assert np.array_equal(got, ref) and np.array_equal(gst, rst)
