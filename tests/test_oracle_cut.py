"""Pins of the oracle's cut state sum (Sec. 2.1: sum over internal states of
a ring of tree amplitudes), each against a fact fixed independently of the
literal sum: the closed form for rank-one matrices, the trace for one tree,
the dimension for identity matrices, invariance under rotating the ring, and
multilinearity: with dual states, the state sum of BG amplitudes equals the
contraction of the amplitudes' polarisation tensors with the completeness
projectors (exact over F_p)."""

import random
from fractions import Fraction

import numpy as np
import pytest

from oracle import bg_oracle as O
from paper_2502_07060_gb300 import inputs as G


def _rand_mat(rng, S):
    return [[Fraction(rng.randint(-9, 9), rng.randint(1, 5)) for _ in range(S)] for _ in range(S)]


@pytest.mark.parametrize("k,S", [(1, 3), (2, 2), (3, 4), (4, 3)])
def test_rank_one_closed_form(k, S):
    rng = random.Random(10 * k + S)
    a = [[Fraction(rng.randint(-9, 9), rng.randint(1, 4)) for _ in range(S)] for _ in range(k)]
    b = [[Fraction(rng.randint(-9, 9), rng.randint(1, 4)) for _ in range(S)] for _ in range(k)]
    mats = [[[a[i][r] * b[i][c] for c in range(S)] for r in range(S)] for i in range(k)]
    closed = Fraction(1)
    for i in range(k):                       # s_{i+1} joins a_i (row) and b_{i+1} (column)
        closed *= sum(a[i][s] * b[(i + 1) % k][s] for s in range(S))
    assert O.cut_state_sum(mats) == closed


def test_single_tree_is_trace_and_identity_ring_is_dimension():
    rng = random.Random(3)
    m = _rand_mat(rng, 4)
    assert O.cut_state_sum([m]) == sum(m[s][s] for s in range(4))
    ident = [[Fraction(int(r == c)) for c in range(3)] for r in range(3)]
    assert O.cut_state_sum([ident] * 5) == 3


def test_ring_rotation_invariance_and_order():
    rng = random.Random(4)
    mats = [_rand_mat(rng, 3) for _ in range(4)]
    v = O.cut_state_sum(mats)
    assert O.cut_state_sum(mats[1:] + mats[:1]) == v
    # the ring is ordered: for non-commuting matrices the reversed ring differs
    assert O.cut_state_sum(mats[::-1]) != v


def test_state_sum_equals_projector_contraction_fp():
    """Two trees joined by two internal legs: tree L carries states eps_a on
    its leg 0 and eps_b on its last leg, tree R the dual states.  By
    multilinearity A(eps, ..) = sum_mu eps^mu A(e_mu, ..), so the literal
    state sum equals T_L[mu][nu] Pi[mu][sigma] Pi[nu][rho] T_R[rho][sigma],
    with T the amplitudes on basis vectors and Pi = sum_s eps_s (x) dual_s."""
    p = G.P_DEFAULT
    n, d, Ds, S = 5, 6, 6, 4
    def F(x):
        return O.GF(int(x), p)
    kL, eL = G.fp_batch(21, 1, n, d, Ds, p, 0, S=S)
    kR, eR = G.fp_batch(22, 1, n, d, Ds, p, 0, S=S)
    eta = O.metric_signs(Ds)
    # dual states of leg 0 / leg n-1 of tree L: dual_s . eps_t = delta_st
    # (Gram matrix inverse over F_p, metric dot), placed on tree R
    def dual(vecs):
        gram = [[sum(F(int(eta[m])) * F(int(vecs[s][m])) * F(int(vecs[t][m])) for m in range(Ds))
                 for t in range(S)] for s in range(S)]
        inv = _inverse(gram, F)
        return [[sum((inv[s][t] * F(int(vecs[t][m])) for t in range(S)), F(0)) for m in range(Ds)]
                for s in range(S)]
    epsA = [list(eL[0, 0, s]) for s in range(S)]         # tree L leg 0 states
    epsB = [list(eL[0, n - 1, s]) for s in range(S)]     # tree L last-leg states
    dA, dB = dual(epsA), dual(epsB)
    kLf = [[F(int(x)) for x in v] for v in kL[0]]
    kRf = [[F(int(x)) for x in v] for v in kR[0]]
    eLf = [[F(int(x)) for x in eL[0, l, 0]] for l in range(n)]
    eRf = [[F(int(x)) for x in eR[0, l, 0]] for l in range(n)]

    def amp(kf, ef, first, last):
        e = [first] + ef[1:n - 1] + [last]
        a, st = O.amplitude(kf, e)
        assert st == 0
        return a
    # M_L[s_out][s_in]: tree L's last leg carries state s_out of the ring, leg 0 state s_in;
    # tree R closes the ring with the duals: leg 0 <- dual of tree L's last leg, last leg <- dual of leg 0
    def fe(v):
        return [F(int(x)) for x in v]
    ML = [[amp(kLf, eLf, fe(epsA[si]), fe(epsB[so])) for si in range(S)] for so in range(S)]
    MR = [[amp(kRf, eRf, dB[si], dA[so]) for si in range(S)] for so in range(S)]
    lhs = O.cut_state_sum([ML, MR])
    basis = [[F(int(m == mu)) for m in range(Ds)] for mu in range(Ds)]
    TL = [[amp(kLf, eLf, basis[mu], basis[nu]) for nu in range(Ds)] for mu in range(Ds)]
    TR = [[amp(kRf, eRf, basis[rho], basis[sig]) for sig in range(Ds)] for rho in range(Ds)]
    # Pi_A[mu][sig] = sum_s epsA_s^mu dA_s^sig (leg 0 of L with the last leg of R), Pi_B likewise
    PiA = [[sum((F(int(epsA[s][mu])) * dA[s][sg] for s in range(S)), F(0)) for sg in range(Ds)] for mu in range(Ds)]
    PiB = [[sum((F(int(epsB[s][nu])) * dB[s][rh] for s in range(S)), F(0)) for rh in range(Ds)] for nu in range(Ds)]
    rhs = F(0)
    for mu in range(Ds):
        for nu in range(Ds):
            if TL[mu][nu] == F(0):
                continue
            for rh in range(Ds):
                for sg in range(Ds):
                    rhs = rhs + TL[mu][nu] * PiA[mu][sg] * PiB[nu][rh] * TR[rh][sg]
    assert lhs == rhs


def _inverse(m, F):
    """Gauss-Jordan inverse over the field F."""
    S = len(m)
    a = [list(row) + [F(int(r == c)) for c in range(S)] for r, row in enumerate(m)]
    for c in range(S):
        piv = next(r for r in range(c, S) if a[r][c] != F(0))
        a[c], a[piv] = a[piv], a[c]
        inv = F(1) / a[c][c]
        a[c] = [x * inv for x in a[c]]
        for r in range(S):
            if r != c and a[r][c] != F(0):
                f = a[r][c]
                a[r] = [x - f * y for x, y in zip(a[r], a[c])]
    return [row[S:] for row in a]
