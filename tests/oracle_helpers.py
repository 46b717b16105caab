"""Helpers shared by the oracle pin tests: mapping generator output into the
oracle's number types and evaluating permuted leg orders.  No recursion
arithmetic lives here."""

from fractions import Fraction

import numpy as np

from oracle import bg_oracle as O
from paper_2502_07060_gb300 import inputs as G

P = G.P_DEFAULT        # 2^31 - 19
PM = G.P_MERSENNE      # 2^31 - 1


def gf_vecs(arr, p):
    """Nested integer array -> list of lists of GF elements."""
    return [[O.GF(int(x), p) for x in row] for row in np.asarray(arr).tolist()]


def gf_of(vs, p):
    return [[O.to_field(x, p) for x in v] for v in vs]


def fp_point(seed, n, d, Ds, p=P, metric=O.MOSTLY_MINUS):
    """One seeded F_p point as GF lists (k [n][d], eps [n][Ds])."""
    k, eps = G.fp_batch(seed, 1, n, d, Ds, p, metric)
    return gf_vecs(k[0], p), gf_vecs(eps[0], p)


def amp(k, eps, metric=O.MOSTLY_MINUS):
    a, st = O.amplitude(k, eps, metric)
    assert st == O.OK
    return a


def permuted(k, eps, order):
    return [k[i] for i in order], [eps[i] for i in order]


def pad(vs, extra, zero):
    return [list(v) + [zero] * extra for v in vs]


def rational_gf(seed, n, d, Ds, metric=O.MOSTLY_MINUS):
    rng = np.random.Generator(np.random.Philox(seed))
    return G.rational_point(rng, n, d, Ds, metric)


def helicity_point_fp(seed, n, helicities, p=P, metric=O.MOSTLY_MINUS, chi_shift=1):
    """F_p point from random spinors with the helicity states of Sec. 2.3:
    '-' -> eps1 = <k|g|chi]/(2[k chi]), '+' -> eps2 = [k|g|chi>/<k chi>, with
    reference chi_i = k_{i+chi_shift mod n}.  Returns (k, eps, lam, lamt) as
    GF lists plus the raw spinors."""
    rng = np.random.Generator(np.random.Philox(seed))
    ops = G.FpOps(p)
    while True:
        k, lam, lamt = G.fp_spinor_point(rng, n, p, metric)
        try:
            eps = []
            for i, h in enumerate(helicities):
                c = (i + chi_shift) % n
                f = G.eps_minus if h == "-" else G.eps_plus
                eps.append(f(lam[i], lamt[i], lam[c], lamt[c], metric, ops))
        except ZeroDivisionError:
            continue
        except ValueError:
            continue
        return gf_vecs(k, p), gf_vecs(eps, p), lam, lamt


def parke_taylor_fp(lam, i, j, p):
    """<ij>^4 / (<12><23>...<n1>) over F_p (legs 0-based)."""
    ops = G.FpOps(p)
    n = len(lam)
    num = pow(G.angle(lam[i], lam[j], ops), 4, p)
    den = 1
    for a in range(n):
        den = den * G.angle(lam[a], lam[(a + 1) % n], ops) % p
    return O.GF(num, p) / O.GF(den, p)
