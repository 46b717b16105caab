"""Pins of the Python oracle against facts the paper and mathematics fix.

Each test relates ``oracle.bg_oracle`` to something other than itself:
the explicit tensor form of the vertices (brute-force diagram sum), gauge
invariance (Ward identity, current conservation, reference independence),
symmetries of colour-ordered amplitudes (cyclic, reflection, U(1)
decoupling), Lorentz invariance, dimensional embedding, the Parke-Taylor
formula (Sec. 3.1), vanishing helicity amplitudes, exact-rational reduction
mod p and a combinatorial count of the operations.
"""

import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import bg_oracle as O
from paper_2502_07060_gb300 import inputs as G
from tests.oracle_helpers import (P, PM, amp, fp_point, gf_of, gf_vecs, helicity_point_fp,
                                  pad, parke_taylor_fp, permuted, rational_gf)

I_P = G.sqrt_minus_one(P)


# ---------------------------------------------------------------- structure

@pytest.mark.parametrize("n,d,Ds,metric", [
    (4, 4, 4, O.MOSTLY_MINUS), (5, 4, 4, O.MOSTLY_MINUS), (5, 4, 6, O.MOSTLY_MINUS),
    (5, 5, 5, O.ALTERNATING), (6, 4, 4, O.MOSTLY_MINUS),
])
def test_bruteforce_tensor_diagrams_equal_recursion(n, d, Ds, metric):
    """Sum over every planar cubic/quartic diagram, each evaluated with the
    explicit V3/V4 tensors and propagator -i/P^2 of Sec. 2.2 (no memoisation),
    equals i * A.  Generic OFF-shell, non-transverse inputs: this is an
    algebraic identity, so it pins the contraction of the vertices, the
    propagator and the factor of i (reading G1) independently of physics."""
    rng = np.random.Generator(np.random.Philox(1000 + n * 10 + Ds))
    iu = O.GF(I_P, P)
    for _ in range(2):
        k = [[O.GF(int(x), P) for x in rng.integers(0, P, d)] for _ in range(n)]
        eps = [[O.GF(int(x), P) for x in rng.integers(0, P, Ds)] for _ in range(n)]
        a = amp(k, eps, metric)
        M, count = O.bruteforce_diagrams(k, eps, metric, iu)
        assert M == iu * a
        assert count > 0


def test_bruteforce_counts_planar_diagrams():
    """Number of cubic+quartic planar diagrams for the top current: 1, 3, 10, 38
    for 2..5 legs (c(m) = sum over ordered 2- and 3-part compositions)."""
    def c(m):
        if m == 1:
            return 1
        tot = sum(c(a) * c(m - a) for a in range(1, m))
        tot += sum(c(a) * c(b) * c(m - a - b) for a in range(1, m) for b in range(1, m - a))
        return tot
    assert [c(m) for m in range(2, 6)] == [1, 3, 10, 38]
    iu = O.GF(I_P, P)
    for n in (3, 4, 5):
        k = [[O.GF(3 + i + mu, P) for mu in range(4)] for i in range(n)]
        eps = [[O.GF(7 * i + mu + 1, P) for mu in range(4)] for i in range(n)]
        _, count = O.bruteforce_diagrams(k, eps, O.MOSTLY_MINUS, iu)
        assert count == c(n - 1)


def test_bruteforce_complex_matches_recursion():
    rng = np.random.default_rng(7)
    n, d, Ds = 5, 4, 4
    k = [list(rng.standard_normal(d) + 1j * rng.standard_normal(d)) for _ in range(n)]
    eps = [list(rng.standard_normal(Ds) + 1j * rng.standard_normal(Ds)) for _ in range(n)]
    a = amp(k, eps)
    M, _ = O.bruteforce_diagrams(k, eps, O.MOSTLY_MINUS, 1j)
    assert abs(M - 1j * a) <= 1e-12 * abs(M)


def test_op_tally_matches_combinatorics():
    """mul = C(n,3)(3Ds+3d) + C(n,4) 6Ds + (C(n,2)-n)(d+Ds) + Ds: V3 splits,
    V4 pairs, internal propagators and the final contraction."""
    for n, d, Ds in [(4, 4, 4), (5, 4, 6), (8, 6, 6), (8, 4, 4), (10, 4, 4), (12, 8, 8)]:
        t = O.op_tally(n, d, Ds)
        expect = (math.comb(n, 3) * (3 * Ds + 3 * d) + math.comb(n, 4) * 6 * Ds
                  + (math.comb(n, 2) - n) * (d + Ds) + Ds)
        assert t.mul == expect
        assert t.inv == math.comb(n, 2) - n


def test_flop_tally_agrees_with_the_operation_tally():
    """With complex momenta every product costs 6 FP64 operations and every sum
    2, except the sums that start from zero (one per dot product, one per
    component of each range's bracket, one per component of each range-momentum
    row), which cost nothing; a complex reciprocal costs 6.  So the FLOP
    tally, counted by a different mechanism (stand-in numbers instead of the
    operation counters), must equal 6 mul + 2 (add - Z) + 6 inv."""
    for n, d, Ds in [(4, 4, 4), (5, 4, 6), (8, 6, 6), (9, 5, 7), (12, 8, 8)]:
        t = O.op_tally(n, d, Ds)
        N = n - 1
        ranges = N * (N - 1) // 2                      # lengths 2..N
        internal = ranges - 1
        s3, s4 = math.comb(n, 3), math.comb(n, 4)
        dots = 3 * s3 + 3 * s4 + internal + 1
        Z = dots + Ds * ranges + d * N
        assert O.flop_tally(n, d, Ds, real_momenta=False) == 6 * t.mul + 2 * (t.add - Z) + 6 * t.inv
        # real momenta: strictly less work, and no more than the complex count
        assert O.flop_tally(n, d, Ds, real_momenta=True) < O.flop_tally(n, d, Ds, real_momenta=False)


# ----------------------------------------------------------- gauge invariance

@pytest.mark.parametrize("n,d,Ds,metric,p", [
    (4, 4, 4, O.MOSTLY_MINUS, P), (5, 4, 4, O.MOSTLY_MINUS, P), (6, 6, 6, O.MOSTLY_MINUS, P),
    (6, 4, 6, O.MOSTLY_MINUS, P), (7, 8, 8, O.MOSTLY_MINUS, P), (6, 4, 4, O.ALTERNATING, PM),
    (5, 6, 8, O.ALTERNATING, P),
])
def test_ward_identity(n, d, Ds, metric, p):
    """eps_i -> k_i for any one leg gives exactly 0 over F_p (Sec. 3.1)."""
    k, eps = fp_point(11 * n + d, n, d, Ds, p, metric)
    zero = O.GF(0, p)
    assert amp(k, eps, metric) != zero
    for i in range(n):
        e2 = list(eps)
        e2[i] = list(k[i]) + [zero] * (Ds - d)
        assert amp(k, e2, metric) == zero


@pytest.mark.parametrize("n,d,Ds", [(5, 4, 4), (7, 6, 6), (8, 8, 8)])
def test_current_conservation(n, d, Ds):
    """P_{i,j} . J(i,j) = 0 for every internal current (transverse on-shell legs)."""
    k, eps = fp_point(5 + n, n, d, Ds)
    r = O.bg_recursion(k, eps)
    eta = O.metric_signs(Ds)
    zero = O.GF(0, P)
    checked = 0
    for (i, j), J in r.currents.items():
        Pv = r.momenta[(i, j)]
        dot = zero
        for mu in range(Ds):
            dot = dot + eta[mu] * Pv[mu] * J[mu]
        assert dot == zero
        checked += 1
    assert checked == (n - 1) * n // 2 - 1


# ------------------------------------------------------------------ symmetries

@pytest.mark.parametrize("n,d,Ds,metric", [(5, 4, 4, 0), (6, 6, 6, 0), (7, 4, 6, 0), (6, 6, 6, 1)])
def test_cyclic_symmetry(n, d, Ds, metric):
    k, eps = fp_point(21 + n, n, d, Ds, P, metric)
    a = amp(k, eps, metric)
    for shift in range(1, n):
        order = [(i + shift) % n for i in range(n)]
        assert amp(*permuted(k, eps, order), metric) == a


@pytest.mark.parametrize("n,d,Ds", [(4, 4, 4), (5, 4, 4), (6, 6, 6), (7, 8, 8)])
def test_reflection(n, d, Ds):
    k, eps = fp_point(31 + n, n, d, Ds)
    a = amp(k, eps)
    sign = 1 if n % 2 == 0 else -1
    assert amp(*permuted(k, eps, list(range(n - 1, -1, -1)))) == sign * a


@pytest.mark.parametrize("n,d,Ds", [(4, 4, 4), (5, 4, 4), (6, 6, 6), (7, 4, 4)])
def test_u1_decoupling(n, d, Ds):
    """Sum over the n-1 insertions of leg 1 among legs 2..n-1 (leg n last) is 0."""
    k, eps = fp_point(41 + n, n, d, Ds)
    total = O.GF(0, P)
    for pos in range(n - 1):
        rest = list(range(1, n - 1))
        order = rest[:pos] + [0] + rest[pos:] + [n - 1]
        total = total + amp(*permuted(k, eps, order))
    assert total == O.GF(0, P)


# ------------------------------------------------- embedding and Lorentz

@pytest.mark.parametrize("n,d,Ds", [(5, 4, 4), (6, 6, 6), (6, 4, 6)])
def test_dimensional_embedding(n, d, Ds):
    """Zero-padding a (d, D_s) point to (d+2, D_s+2) leaves A unchanged
    (Sec. 2.3: lower-dimensional states are embedded trivially)."""
    k, eps = fp_point(51 + n, n, d, Ds)
    zero = O.GF(0, P)
    a = amp(k, eps)
    assert amp(pad(k, 2, zero), pad(eps, 2, zero)) == a
    assert amp(k, pad(eps, 2, zero)) == a


def _modinv_matrix(M, p):
    n = len(M)
    A = [[x % p for x in row] + [1 if i == j else 0 for j in range(n)] for i, row in enumerate(M)]
    for c in range(n):
        piv = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        inv = pow(A[c][c], -1, p)
        A[c] = [x * inv % p for x in A[c]]
        for r in range(n):
            if r != c and A[r][c]:
                f = A[r][c]
                A[r] = [(x - f * y) % p for x, y in zip(A[r], A[c])]
    return [row[n:] for row in A]


@pytest.mark.parametrize("n,d,Ds,metric", [(5, 4, 4, 0), (6, 6, 6, 0), (5, 4, 6, 0), (6, 6, 6, 1)])
def test_lorentz_invariance(n, d, Ds, metric):
    """A rational Lorentz transformation Lambda = (1 - A)^-1 (1 + A), A = eta S
    with S antisymmetric (Cayley transform), on the first d components, and a
    second one on the extra D_s - d components, leave A unchanged."""
    rng = np.random.Generator(np.random.Philox(61 + n))
    eta = O.metric_signs(Ds, metric)
    Lam = [[1 if i == j else 0 for j in range(Ds)] for i in range(Ds)]
    blocks = [(0, d)] + ([(d, Ds)] if Ds - d >= 2 else [])
    for lo, hi in blocks:
        m = hi - lo
        S = [[0] * m for _ in range(m)]
        for a in range(m):
            for b in range(a + 1, m):
                v = int(rng.integers(1, 50))
                S[a][b], S[b][a] = v, -v
        A = [[eta[lo + a] * S[a][b] for b in range(m)] for a in range(m)]
        Im = [[1 if a == b else 0 for b in range(m)] for a in range(m)]
        inv = _modinv_matrix([[Im[a][b] - A[a][b] for b in range(m)] for a in range(m)], P)
        L = [[sum(inv[a][c] * (Im[c][b] + A[c][b]) for c in range(m)) % P for b in range(m)]
             for a in range(m)]
        for a in range(m):
            for b in range(m):
                Lam[lo + a][lo + b] = L[a][b]
    # Lambda^T eta Lambda = eta
    for a in range(Ds):
        for b in range(Ds):
            s = sum(Lam[c][a] * eta[c] * Lam[c][b] for c in range(Ds)) % P
            assert s == (eta[a] % P if a == b else 0)
    k, eps = fp_point(71 + n, n, d, Ds, P, metric)
    zero = O.GF(0, P)

    def tr(v, D):
        return [sum((O.GF(Lam[a][b], P) * v[b] for b in range(D)), zero) for a in range(D)]

    k2 = [tr(x, d) for x in k]
    e2 = [tr(x, Ds) for x in eps]
    assert amp(k2, e2, metric) == amp(k, eps, metric)


# ------------------------------------------------------ Parke-Taylor (Sec. 3.1)

def _pt_ratio_fp(n, seed, i, j, p, metric):
    hel = ["+"] * n
    hel[i] = hel[j] = "-"
    k, eps, lam, _ = helicity_point_fp(seed, n, hel, p, metric)
    a = amp(k, eps, metric)
    return a / parke_taylor_fp(lam, i, j, p)


@pytest.mark.parametrize("p,metric", [(P, O.MOSTLY_MINUS), (PM, O.ALTERNATING)])
@pytest.mark.parametrize("n", [4, 5, 6, 7])
def test_parke_taylor_mhv(n, p, metric):
    """A(1-2-3+...n+) / [<12>^4/(<12>...<n1>)] = (-1)^n 2^(n-3) for every seed.

    Derivation: the paper's vertices are sqrt2 (V3) and 2 (V4) times the
    standard colour-ordered ones, a factor sqrt2^(n-2) per diagram; its states
    eps1 = eps^-/sqrt2 and eps2 = -sqrt2 eps^+ (reference chi) contribute
    (1/sqrt2)^2 (-sqrt2)^(n-2); the returned A = -i x the paper's amplitude
    (reading G1) cancels the i of Parke-Taylor.  Net: (-1)^n 2^(n-3)."""
    expect = O.GF((-1) ** n * 2 ** (n - 3), p)
    for seed in range(25):
        assert _pt_ratio_fp(n, 100 + seed, 0, 1, p, metric) == expect


@pytest.mark.parametrize("i,j", [(0, 2), (1, 3), (2, 4), (0, 4)])
def test_parke_taylor_other_mhv_positions(i, j):
    n = 5
    expect = O.GF((-1) ** n * 2 ** (n - 3), P)
    for seed in range(10):
        assert _pt_ratio_fp(n, 300 + seed, i, j, P, O.MOSTLY_MINUS) == expect


def test_parke_taylor_many_seeds_n6():
    expect = O.GF(2 ** 3, P)
    for seed in range(100):
        assert _pt_ratio_fp(6, 1000 + seed, 0, 1, P, O.MOSTLY_MINUS) == expect


@pytest.mark.parametrize("hel", ["+++++", "-++++", "+-+++", "++++-", "++++++", "+++-++"])
def test_vanishing_helicity_amplitudes(hel):
    """All-plus and single-minus tree amplitudes vanish exactly (d = 4)."""
    n = len(hel)
    for seed in range(5):
        k, eps, _, _ = helicity_point_fp(500 + seed, n, list(hel))
        assert amp(k, eps) == O.GF(0, P)


def test_reference_vector_independence():
    """Changing the helicity states' reference spinors leaves A unchanged."""
    n = 6
    hel = list("-+-++-")
    k1, e1, lam, lamt = helicity_point_fp(77, n, hel, chi_shift=1)
    ops = G.FpOps(P)
    a1 = amp(k1, e1)
    for shift in (2, 3, n - 1):
        eps = []
        for i, h in enumerate(hel):
            c = (i + shift) % n
            f = G.eps_minus if h == "-" else G.eps_plus
            eps.append(f(lam[i], lamt[i], lam[c], lamt[c], O.MOSTLY_MINUS, ops))
        assert amp(k1, gf_vecs(eps, P)) == a1


def test_parke_taylor_complex_rambo():
    """Physical RAMBO points (sqrt s = 1000), complex spinors: the same
    constant (-1)^n 2^(n-3) within FP64 rounding."""
    rng = np.random.default_rng(5)
    n = 5
    ks = G.rambo(rng, 50, n, 1000.0)
    ops = G.ComplexOps
    for e in range(50):
        k = [list(map(complex, v)) for v in ks[e]]
        sp = [G.spinors_from_vector_c(v) for v in k]
        lam = [s[0] for s in sp]
        lamt = [s[1] for s in sp]
        hel = "--+++"
        eps = []
        for i, h in enumerate(hel):
            c = (i + 1) % n
            f = G.eps_minus if h == "-" else G.eps_plus
            eps.append(f(lam[i], lamt[i], lam[c], lamt[c], O.MOSTLY_MINUS, ops))
        a = amp(k, eps)
        pt = G.angle(lam[0], lam[1], ops) ** 4
        for i in range(n):
            pt /= G.angle(lam[i], lam[(i + 1) % n], ops)
        ratio = a / pt
        assert abs(ratio - (-1) ** n * 2 ** (n - 3)) < 1e-9


# ------------------------------------------------ exact rationals and mpmath

@pytest.mark.parametrize("n,d,Ds,metric", [(5, 4, 4, 0), (6, 6, 6, 0), (5, 4, 6, 1)])
def test_exact_rational_reduces_mod_p(n, d, Ds, metric):
    """Evaluate over Q from rational inputs, reduce mod p; equals the F_p
    evaluation of the reduced inputs (Sec. 1: F_p samples of rational values)."""
    for seed in range(3):
        k, eps = rational_gf(800 + seed, n, d, Ds, metric)
        aq = amp(k, eps, metric)
        assert isinstance(aq, Fraction)
        for p in (P, PM):
            af = amp(gf_of(k, p), gf_of(eps, p), metric)
            assert af == O.to_field(aq, p)


def test_rational_point_is_on_shell():
    for metric in (0, 1):
        k, eps = rational_gf(9, 6, 6, 8, metric)
        eta = O.metric_signs(8, metric)
        for a in range(6):
            assert sum(eta[m] * k[a][m] ** 2 for m in range(6)) == 0
            assert sum(eta[m] * k[a][m] * eps[a][m] for m in range(6)) == 0
        for m in range(6):
            assert sum(k[a][m] for a in range(6)) == 0


def test_complex_oracle_against_mpmath():
    """FP64 evaluation agrees with a 40-digit mpmath evaluation of the same
    oracle on the same inputs (bounds the oracle's own rounding)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    k, eps = G.c64_batch(3, 8, 7, 6, 6)
    for e in range(8):
        kc = [list(v) for v in k[e]]
        ec = [list(v) for v in eps[e]]
        a = amp(kc, ec)
        km = [[mp.mpc(x.real, x.imag) for x in v] for v in kc]
        em = [[mp.mpc(x.real, x.imag) for x in v] for v in ec]
        am = amp(km, em)
        assert abs(complex(am) - a) <= 1e-11 * abs(complex(am))


# --------------------------------------------------- planted mistakes (CPU)

_MUTATIONS = [
    ("R = C.axpy(R, ac + ac, JB, Ds)", "R = C.axpy(R, ac, JB, Ds)"),             # V4 factor 2
    ("R = C.axpy(R, -bc, JA, Ds)", "R = C.axpy(R, bc, JA, Ds)"),                 # V4 sign
    ("R = C.axpy(R, pb_ja + pb_ja, JB, Ds)", "R = C.axpy(R, pb_ja, JB, Ds)"),    # V3 factor 2
    ("diff = [PA[mu] - PB[mu]", "diff = [PB[mu] - PA[mu]"),                      # V3 P-Q sign
    ("J[(s + 1, t)], J[(t + 1, j)]", "J[(s + 1, t)], J[(s + 1, t)]"),            # wrong index
]


@pytest.mark.parametrize("old,new", _MUTATIONS)
def test_planted_mistakes_are_caught(old, new):
    """Each plausible mistake planted in a copy of the oracle breaks the Ward
    identity or the brute-force diagram sum."""
    import inspect
    src = inspect.getsource(O)
    assert old in src
    mod = {}
    exec(compile(src.replace(old, new), "mutant", "exec"), mod)
    k, eps = fp_point(5, 6, 6, 6)
    zero = O.GF(0, P)
    caught = False
    for i in range(6):
        e2 = list(eps)
        e2[i] = list(k[i])
        a, st = mod["amplitude"](k, e2, 0)
        caught |= (a != zero)
    iu = O.GF(I_P, P)
    kk, ee = k[:5], eps[:5]
    M, _ = O.bruteforce_diagrams(kk, ee, 0, iu)
    a, _ = mod["amplitude"](kk, ee, 0)
    caught |= (M != iu * a)
    assert caught
