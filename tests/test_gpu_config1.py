"""The physical d = 4 configuration on the GPU: n = 5 gluons, complex FP64,
helicities (-,-,+,+,+), 1024 RAMBO points at sqrt(s) = 1000 (incoming legs
negated, all momenta outgoing), the spinor-helicity states of Sec. 2.3 with
reference momentum chi_i = k_{i+1}.

Checked three ways, through the C-ABI (both complex plans: real momenta and
complex momenta):
  * against the double-double C oracle, within the tolerance of the parity
    tests (1e-10 relative);
  * against the Parke-Taylor MHV formula of Sec. 3.1: A / PT is the constant
    (-1)^n 2^(n-3) = -4 derived in the oracle pins (test_parke_taylor_mhv);
  * the Ward identity of Sec. 3.1: eps_i -> k_i gives zero, up to rounding
    relative to the size of the physical amplitude.
"""

import numpy as np
import pytest

from oracle import coracle as C
from paper_2502_07060_gb300 import inputs as G

pytestmark = pytest.mark.gpu

N_LEG = 5
E = 1024
HEL = "--+++"
TOL = 1e-10


def _config1_inputs(seed=2025):
    rng = np.random.default_rng(seed)
    ks = G.rambo(rng, E, N_LEG, 1000.0)                       # [E][n][4], real
    ops = G.ComplexOps
    k = ks.astype(np.complex128)
    eps = np.zeros((E, N_LEG, 4), dtype=np.complex128)
    lam_all, lamt_all = [], []
    for e in range(E):
        sp = [G.spinors_from_vector_c(list(map(complex, v))) for v in ks[e]]
        lam = [s[0] for s in sp]
        lamt = [s[1] for s in sp]
        for i, h in enumerate(HEL):
            c = (i + 1) % N_LEG
            f = G.eps_minus if h == "-" else G.eps_plus
            eps[e, i] = f(lam[i], lamt[i], lam[c], lamt[c], G.MOSTLY_MINUS, ops)
        lam_all.append(lam)
        lamt_all.append(lamt)
    return ks, k, eps, lam_all


def _parke_taylor(lam):
    ops = G.ComplexOps
    pt = G.angle(lam[0], lam[1], ops) ** 4
    for i in range(N_LEG):
        pt /= G.angle(lam[i], lam[(i + 1) % N_LEG], ops)
    return pt


def _eval(field, kin, eps):
    import torch
    from paper_2502_07060_gb300 import bg
    plan = bg.Plan(N_LEG, 4, 4, field, 0, bg.MOSTLY_MINUS)
    out, st = plan.eval(torch.from_numpy(np.ascontiguousarray(kin)).cuda(),
                        torch.from_numpy(np.ascontiguousarray(eps)).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy(), st.cpu().numpy()


@pytest.fixture(scope="module")
def config1():
    return _config1_inputs()


@pytest.mark.parametrize("momenta", ["real", "complex"])
def test_config1_against_oracle_and_parke_taylor(config1, momenta):
    from paper_2502_07060_gb300 import bg
    ks, k, eps, lam = config1
    if momenta == "real":
        out, st = _eval(bg.FIELD_C64_REAL, ks.astype(np.float64), eps)
    else:
        out, st = _eval(bg.FIELD_C64, k, eps)
    assert not st.any()
    hi, lo, rst = C.amp_c64dd(k, eps, 0)
    assert not rst.any()
    rel = np.abs((out - hi) - lo) / np.abs(hi)
    assert rel.max() <= TOL, rel.max()
    expect = (-1) ** N_LEG * 2 ** (N_LEG - 3)
    ratio = out / np.array([_parke_taylor(l) for l in lam])
    assert np.abs(ratio - expect).max() <= TOL * abs(expect), np.abs(ratio - expect).max()


def test_config1_ward_identity(config1):
    from paper_2502_07060_gb300 import bg
    ks, k, eps, _ = config1
    phys, _ = _eval(bg.FIELD_C64_REAL, ks.astype(np.float64), eps)
    for i in range(N_LEG):
        e2 = eps.copy()
        e2[:, i, :] = k[:, i, :]
        out, st = _eval(bg.FIELD_C64_REAL, ks.astype(np.float64), e2)
        assert not st.any()
        # eps_i -> k_i rescales the state by |k_i| ~ sqrt(s)/n; compare with
        # |A| times that scale
        scale = np.abs(phys) * np.abs(ks[:, i, 0])
        assert (np.abs(out) <= 1e-10 * scale).all(), (np.abs(out) / scale).max()
