"""Pins of the C oracle (bulk parity reference and timed CPU baseline).

The C oracle is checked bit-exact over F_p against the Python oracle (itself
pinned in test_oracle_pins.py), against mpmath for complex FP64, and directly
on the Ward identity, reflection symmetry and singular propagators."""

import numpy as np
import pytest

from oracle import bg_oracle as O
from oracle import coracle as C
from paper_2502_07060_gb300 import inputs as G
from tests.oracle_helpers import P, PM, gf_vecs


@pytest.mark.parametrize("n,d,Ds,metric,p", [
    (4, 4, 4, 0, P), (5, 4, 4, 0, P), (6, 6, 6, 0, P), (7, 4, 6, 0, P), (8, 6, 6, 0, P),
    (8, 8, 8, 1, PM), (9, 4, 4, 1, PM), (10, 4, 4, 0, P), (12, 8, 8, 0, P), (6, 5, 7, 1, P),
])
def test_c_fp_matches_python(n, d, Ds, metric, p):
    E = 4 if n < 10 else 2
    k, eps = G.fp_batch(17 + n, E, n, d, Ds, p, metric)
    out, st = C.amp_fp(k, eps, p, metric)
    for e in range(E):
        a, s = O.amplitude(gf_vecs(k[e], p), gf_vecs(eps[e], p), metric)
        assert s == st[e] == 0
        assert int(a) == int(out[e])


@pytest.mark.parametrize("n,d,Ds,metric", [(5, 4, 4, 0), (8, 6, 6, 0), (7, 8, 8, 1), (10, 4, 6, 0)])
def test_c_c64_matches_python(n, d, Ds, metric):
    k, eps = G.c64_batch(23 + n, 6, n, d, Ds, metric)
    out, st = C.amp_c64(k, eps, metric)
    for e in range(6):
        a, s = O.amplitude([list(v) for v in k[e]], [list(v) for v in eps[e]], metric)
        assert s == st[e] == 0
        assert abs(a - out[e]) <= 1e-12 * abs(a)


def test_c_c64_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    k, eps = G.c64_batch(29, 16, 8, 6, 6)
    out, _ = C.amp_c64(k, eps)
    for e in range(16):
        km = [[mp.mpc(x.real, x.imag) for x in v] for v in k[e]]
        em = [[mp.mpc(x.real, x.imag) for x in v] for v in eps[e]]
        a, _ = O.amplitude(km, em)
        assert abs(complex(a) - out[e]) <= 1e-11 * abs(complex(a))


@pytest.mark.parametrize("n,d,Ds,metric,p", [(6, 6, 6, 0, P), (8, 8, 8, 0, P), (7, 4, 4, 1, PM)])
def test_c_ward_identity(n, d, Ds, metric, p):
    E = 64
    k, eps = G.fp_batch(31 + n, E, n, d, Ds, p, metric)
    out, _ = C.amp_fp(k, eps, p, metric)
    assert np.count_nonzero(out) >= E - 1
    for i in range(n):
        e2 = eps.copy()
        e2[:, i, :] = 0
        e2[:, i, :d] = k[:, i, :]
        w, st = C.amp_fp(k, e2, p, metric)
        assert not st.any()
        assert not w.any()


def test_c_reflection_and_cyclic():
    n, E = 7, 32
    k, eps = G.fp_batch(37, E, n, 6, 6)
    a, _ = C.amp_fp(k, eps, P)
    r, _ = C.amp_fp(k[:, ::-1].copy(), eps[:, ::-1].copy(), P)
    assert np.array_equal(r.astype(np.int64), (P - a.astype(np.int64)) % P)   # (-1)^7
    c, _ = C.amp_fp(np.roll(k, 1, axis=1), np.roll(eps, 1, axis=1), P)
    assert np.array_equal(c, a)


def singular_fp_point(seed, n, d, Ds, p=P):
    """A point whose range (legs 1, 2) is on shell: k_2 = c k_1 makes
    (k_1 + k_2)^2 = 0, so an internal propagator is singular."""
    rng = np.random.Generator(np.random.Philox(seed))
    eta = G.metric_diag(d, 0)
    k = np.empty((1, n, d), dtype=np.uint64)
    k[0, :n - 2] = G.fp_null_vectors(rng, (n - 2,), d, p)
    k[0, 1] = G.fmul(k[0, 0], 5, p)
    Q = G.fneg(k[0, :n - 2].sum(axis=0) % np.uint64(p), p)
    while True:
        r = G.fp_null_vectors(rng, (1,), d, p)[0]
        qr = G.fdot(Q, r, eta, p)
        if qr != 0:
            break
    lam = G.fmul(G.fdot(Q, Q, eta, p), G.finv(G.fmul(qr, 2, p), p), p)
    k[0, n - 2] = G.fmul(lam, r, p)
    k[0, n - 1] = G.fsub(Q, k[0, n - 2], p)
    eps = G.fp_transverse_states(rng, k, Ds, p)[:, :, 0, :]
    return k.astype(np.uint32), eps.astype(np.uint32)


def test_singular_propagator_status():
    for n in (5, 8):
        k, eps = singular_fp_point(3, n, 6, 6)
        a, s = O.amplitude(gf_vecs(k[0], P), gf_vecs(eps[0], P))
        assert s == O.SINGULAR and a == O.GF(0, P)
        out, st = C.amp_fp(k, eps, P)
        assert st[0] == 1 and out[0] == 0


def test_thread_count_does_not_change_results():
    k, eps = G.fp_batch(41, 300, 8, 6, 6)
    a1, _ = C.amp_fp(k, eps, P, nthreads=1)
    a2, _ = C.amp_fp(k, eps, P, nthreads=0)
    assert np.array_equal(a1, a2)


def test_bad_arguments_rejected():
    k, eps = G.fp_batch(1, 2, 5, 4, 4)
    with pytest.raises(ValueError):
        C.amp_fp(k, eps, 4294967291)      # p >= 2^31
    with pytest.raises(ValueError):
        C.amp_fp(k[:, :, :4], eps[:, :, :3], P)   # D_s < d


@pytest.mark.parametrize("n,d,Ds,metric", [(4, 4, 4, 0), (8, 6, 6, 0), (7, 8, 8, 1), (12, 4, 4, 0)])
def test_c_double_double_against_mpmath(n, d, Ds, metric):
    """The double-double evaluation (the C64 reference of the GPU tests) agrees
    with a 50-digit mpmath evaluation of the Python oracle to 1e-25."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    E = 6
    k, eps = G.c64_batch(51 + n, E, n, d, Ds, metric)
    hi, lo, st = C.amp_c64dd(k, eps, metric)
    assert not st.any()
    for e in range(E):
        km = [[mp.mpc(x.real, x.imag) for x in v] for v in k[e]]
        em = [[mp.mpc(x.real, x.imag) for x in v] for v in eps[e]]
        a, _ = O.amplitude(km, em, metric)
        v = mp.mpc(hi[e].real, hi[e].imag) + mp.mpc(lo[e].real, lo[e].imag)
        assert abs(v - a) <= mp.mpf("1e-25") * abs(a)


def test_c_double_double_singular():
    k, eps = G.c64_batch(3, 2, 5, 4, 4, 0)
    k[1, 0] = [1.0, 1.0, 0.0, 0.0]          # exactly null, and (k_1 + k_2)^2 = 0
    k[1, 1] = [2.0, 2.0, 0.0, 0.0]          # exactly in FP64
    _, _, st = C.amp_c64dd(k, eps, 0)
    assert st[1] == 1 and st[0] == 0
