"""Exact four-dimensional helicity amplitudes over F_p on the GPU.

With the spinor-helicity states of Sec. 2.3 (reference chi_i = k_{i+1}) the
tree amplitudes of Sec. 3.1's validation hold exactly in a prime field:
  * all-plus and single-minus amplitudes vanish;
  * the MHV amplitude equals the Parke-Taylor expression times the constant
    (-1)^n 2^(n-3) derived in the oracle pins (test_parke_taylor_mhv),
    for the two negative-helicity legs anywhere in the ordering.
Both primes and metrics: p = 2^31 - 19 with the mostly-minus metric and
p = 2^31 - 1 (no square root of -1) with the alternating metric.
"""

import numpy as np
import pytest

from paper_2502_07060_gb300 import inputs as G
from tests.oracle_helpers import helicity_point_fp, parke_taylor_fp

pytestmark = pytest.mark.gpu

P = G.P_DEFAULT
PM = G.P_MERSENNE
POINTS = 40


def _batch(n, hel, p, metric, seed0):
    ks, es, pts = [], [], []
    for s in range(POINTS):
        k, eps, lam, _ = helicity_point_fp(seed0 + s, n, list(hel), p, metric)
        ks.append([[x.v for x in v] for v in k])
        es.append([[x.v for x in v] for v in eps])
        pts.append(lam)
    return np.array(ks, dtype=np.uint32), np.array(es, dtype=np.uint32), pts


def _gpu(k, eps, p, metric):
    import torch
    from paper_2502_07060_gb300 import bg
    n = k.shape[1]
    plan = bg.Plan(n, 4, 4, bg.FIELD_FP, p, metric)
    out, st = plan.eval(torch.from_numpy(k.view(np.int32)).cuda(), torch.from_numpy(eps.view(np.int32)).cuda())
    torch.cuda.synchronize()
    assert not st.cpu().numpy().any()
    return out.cpu().numpy().view(np.uint32).astype(np.int64)


@pytest.mark.parametrize("p,metric", [(P, G.MOSTLY_MINUS), (PM, G.ALTERNATING)])
@pytest.mark.parametrize("n", [5, 6, 8])
def test_all_plus_and_single_minus_vanish(n, p, metric):
    for hel in ("+" * n, "-" + "+" * (n - 1), "+" * (n - 2) + "-+"):
        k, eps, _ = _batch(n, hel, p, metric, 100 * n)
        assert not _gpu(k, eps, p, metric).any(), hel


@pytest.mark.parametrize("p,metric", [(P, G.MOSTLY_MINUS), (PM, G.ALTERNATING)])
@pytest.mark.parametrize("n,i,j", [(5, 0, 1), (6, 1, 4), (8, 0, 1), (8, 2, 6)])
def test_mhv_equals_parke_taylor(n, i, j, p, metric):
    hel = ["+"] * n
    hel[i] = hel[j] = "-"
    k, eps, lams = _batch(n, "".join(hel), p, metric, 1000 + 10 * n + i + j)
    out = _gpu(k, eps, p, metric)
    c = ((-1) ** n * 2 ** (n - 3)) % p
    expect = np.array([(c * parke_taylor_fp(lam, i, j, p).v) % p for lam in lams], dtype=np.int64)
    assert np.array_equal(out, expect)
