"""Pins of the seeded input generators: on-shell momenta, momentum
conservation, transverse states, RAMBO, spinor points, and the completeness
relations of the d-dimensional states of Sec. 2.3 for d = 4..10."""

import numpy as np
import pytest

from oracle import bg_oracle as O
from paper_2502_07060_gb300 import inputs as G
from tests.oracle_helpers import P, PM


@pytest.mark.parametrize("n,d,Ds,metric,p", [
    (5, 4, 4, 0, P), (8, 6, 6, 0, P), (8, 8, 8, 0, P), (6, 4, 6, 1, PM), (12, 8, 8, 1, P),
])
def test_fp_batch_on_shell_conserved_transverse(n, d, Ds, metric, p):
    E = 257
    k, eps = G.fp_batch(5, E, n, d, Ds, p, metric)
    assert k.dtype == np.uint32 and eps.dtype == np.uint32
    assert (k < p).all() and (eps < p).all()
    eta_d = G.metric_diag(d, metric)
    eta = G.metric_diag(Ds, metric)
    assert not G.fdot(k, k, eta_d, p).any()                        # k_i^2 = 0
    assert not (k.astype(np.uint64).sum(axis=1) % np.uint64(p)).any()   # sum k = 0
    kp = np.zeros((E, n, Ds), dtype=np.uint64)
    kp[..., :d] = k
    assert not G.fdot(kp, eps, eta, p).any()                       # eps_i . k_i = 0
    assert G.fdot(eps, eps, eta, p).any()


def test_fp_batch_states_and_determinism():
    k1, e1 = G.fp_batch(9, 64, 6, 6, 6, S=4)
    k2, e2 = G.fp_batch(9, 64, 6, 6, 6, S=4)
    assert e1.shape == (64, 6, 4, 6)
    assert np.array_equal(k1, k2) and np.array_equal(e1, e2)
    k3, _ = G.fp_batch(10, 64, 6, 6, 6, S=4)
    assert not np.array_equal(k1, k3)
    kp = np.zeros((64, 6, 1, 6), dtype=np.uint64)
    kp[..., 0, :] = k1
    assert not G.fdot(np.broadcast_to(kp, e1.shape), e1, G.metric_diag(6, 0), P).any()


@pytest.mark.parametrize("n,d,Ds,metric", [(8, 6, 6, 0), (5, 4, 4, 0), (7, 8, 8, 1)])
def test_c64_batch_on_shell(n, d, Ds, metric):
    k, eps = G.c64_batch(3, 500, n, d, Ds, metric)
    assert not np.abs(k.imag).any()
    eta = G.metric_diag(Ds, metric)
    eta_d = G.metric_diag(d, metric)
    scale = np.abs(k).max()
    assert np.abs((k * k * eta_d).sum(-1)).max() < 1e-9 * scale ** 2
    assert np.abs(k.sum(axis=1)).max() < 1e-9 * scale
    kp = np.zeros(eps.shape, dtype=complex)
    kp[..., :d] = k
    rel = np.abs((kp * eps * eta).sum(-1)) / (np.abs(kp).max(-1) * np.abs(eps).max(-1))
    assert rel.max() < 1e-12


def test_rambo():
    rng = np.random.default_rng(1)
    k = G.rambo(rng, 1000, 7, 1000.0)
    eta = G.metric_diag(4, 0)
    assert np.abs((k * k * eta).sum(-1)).max() < 1e-7
    assert np.abs(k.sum(axis=1)).max() < 1e-9
    assert (k[:, 2:, 0] > 0).all() and (k[:, :2, 0] < 0).all()
    assert np.allclose(-k[:, :2, 0].sum(axis=1), 1000.0)


@pytest.mark.parametrize("p,metric", [(P, 0), (PM, 1)])
def test_fp_spinor_point(p, metric):
    rng = np.random.Generator(np.random.Philox(2))
    ops = G.FpOps(p)
    eta = G.metric_diag(4, metric)
    for _ in range(5):
        k, lam, lamt = G.fp_spinor_point(rng, 6, p, metric)
        for a in range(6):
            assert sum(int(eta[m]) * k[a][m] * k[a][m] for m in range(4)) % p == 0
        for m in range(4):
            assert sum(k[a][m] for a in range(6)) % p == 0
        # 2 k_a . k_b = <ab>[ab]
        two_dot = 2 * sum(int(eta[m]) * k[0][m] * k[2][m] for m in range(4)) % p
        assert two_dot == ops.mul(G.angle(lam[0], lam[2], ops), G.square(lamt[0], lamt[2], ops))


def _factor_fp(M, p, ops):
    """lam lamt^T = M for a rank-1 2x2 matrix over F_p."""
    m00, m01, m10, m11 = M
    if m00 % p:
        return [m00, m10], [1, ops.div(m01, m00)]
    return [m01, m11], [0, 1]


@pytest.mark.parametrize("d", [4, 5, 6, 7, 8, 9, 10])
def test_completeness_relation(d):
    """sum_i eps_i^mu eps~_i^nu = -g^{mu nu} + (k^mu eta^nu + k^nu eta^mu)/(k.eta)
    (Sec. 2.3, completeness relation), with eta = chi for d = 4 and
    eta = k_4d - k_extra for d > 4, using eps1, eps2 (conjugates eps2, eps1),
    eps3 (conjugate eps3/mu^2) and the extra states (conjugates per the
    documented reading), all exact over F_p."""
    p = P
    ops = G.FpOps(p)
    rng = np.random.Generator(np.random.Philox(40 + d))
    g = [int(x) for x in G.metric_diag(d, 0)]

    def dot(a, b, D):
        return sum(g[m] * a[m] * b[m] for m in range(D)) % p

    for _ in range(3):
        k = [int(x) for x in G.fp_null_vectors(rng, (1,), d, p)[0]]
        lc = [int(x) for x in rng.integers(1, p, 2)]
        ltc = [int(x) for x in rng.integers(1, p, 2)]
        chi = G.vector_from_matrix(G._outer(lc, ltc, ops), 0, ops)
        k4 = k[:4]
        mu2 = dot(k4, k4, 4)
        if d == 4:
            assert mu2 == 0
            kflat = k4
        else:
            c = ops.div(mu2, 2 * dot(chi, k4, 4))
            kflat = [(k4[m] - c * chi[m]) % p for m in range(4)]
        M = [(kflat[0] + kflat[3]) % p, (kflat[1] - ops.i * kflat[2]) % p,
             (kflat[1] + ops.i * kflat[2]) % p, (kflat[0] - kflat[3]) % p]
        lk, ltk = _factor_fp(M, p, ops)
        e1 = G.eps_minus(lk, ltk, lc, ltc, 0, ops) + [0] * (d - 4)
        e2 = G.eps_plus(lk, ltk, lc, ltc, 0, ops) + [0] * (d - 4)
        pairs = [(e1, e2), (e2, e1)]
        if d > 4:
            c3 = ops.div(mu2, dot(chi, k4, 4))
            e3 = [(k4[m] - c3 * chi[m]) % p for m in range(4)] + [0] * (d - 4)
            inv = pow(mu2, -1, p)
            pairs.append((e3, [x * inv % p for x in e3]))
            kf = [O.GF(x, p) for x in k]
            for e, et in G.extra_dim_states(kf, d, lambda v: O.GF(v, p)):
                pairs.append(([int(x) for x in e], [int(x) for x in et]))
        assert len(pairs) == d - 2
        for e, _ in pairs:
            assert dot(e, k, d) == 0
        eta = chi + [0] * (d - 4) if d == 4 else k4 + [(-x) % p for x in k[4:]]
        keta_inv = pow(dot(k, eta, d), -1, p)
        for mu in range(d):
            for nu in range(d):
                lhs = sum(e[mu] * et[nu] for e, et in pairs) % p
                rhs = (-(g[mu] if mu == nu else 0) + (k[mu] * eta[nu] + k[nu] * eta[mu]) * keta_inv) % p
                assert lhs == rhs, (d, mu, nu)


def test_golden_fixtures_reproduce():
    """The stored rational amplitudes (written by tests/golden/make_golden.py
    from the oracle alone) are reproduced by the oracle and are on-shell."""
    import json
    import os
    from fractions import Fraction
    path = os.path.join(os.path.dirname(__file__), "golden", "rational_amplitudes.json")
    cases = json.load(open(path))["cases"]
    assert len(cases) >= 5
    for c in cases:
        k = [[Fraction(x) for x in v] for v in c["k"]]
        eps = [[Fraction(x) for x in v] for v in c["eps"]]
        a, st = O.amplitude(k, eps, c["metric"])
        assert st == 0 and a == Fraction(c["amplitude"])


@pytest.mark.parametrize("n,d,Ds,metric,mask", [(8, 6, 6, 0, 0b1111110), (6, 8, 8, 1, 0b011010),
                                                (5, 4, 6, 0, 0b0110), (12, 8, 8, 0, 0b011111111110)])
def test_mixed_dimension_points(n, d, Ds, metric, mask):
    """Points with four-dimensional legs (the loop-level setting of Sec. 2.3):
    flagged legs have momenta and states that vanish beyond four components;
    every momentum is null, the sum is zero and every state is transverse."""
    k, e = G.fp_batch(9, 300, n, d, Ds, P, metric, workers=1, four_d=mask)
    k = k.astype(np.uint64)
    e = e.astype(np.uint64)
    eta_k = G.metric_diag(d, metric)
    eta_e = G.metric_diag(Ds, metric)
    kp = np.zeros(k.shape[:2] + (Ds,), np.uint64)
    kp[..., :d] = k
    for l in range(n):
        assert (G.fdot(k[:, l], k[:, l], eta_k, P) == 0).all()
        assert (G.fdot(e[:, l], kp[:, l], eta_e, P) == 0).all()
        if (mask >> l) & 1:
            assert not k[:, l, 4:].any() and not e[:, l, 4:].any()
    assert not (k.sum(axis=1) % np.uint64(P)).any()
    if d > 4:
        assert k[:, n - 1, 4:].any()          # the closing leg carries the extra components
    with pytest.raises(ValueError):
        G.fp_batch(9, 4, n, d, Ds, P, metric, workers=1, four_d=1 << (n - 1))
