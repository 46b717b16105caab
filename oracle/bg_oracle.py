"""Oracle: a plain, slow, literal Berends-Giele recursion on the CPU.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import or run anything under
``oracle/``.  The product path (``paper_2502_07060_gb300``) never imports it,
and this module imports nothing from the product path.

What it computes (arXiv:2502.07060, Sec. 2.2, the current recursion and the
vertex definitions that follow it):

* ``P_{i,j} = sum_{l=i..j} k_l``                       (range momenta, Sec. 2.2)
* ``J(i,i) = eps_i``; for a range of length m >= 2

      J(i,j) = (-i / P_{i,j}^2) [ sum_s V3(P_A, P_B) J_A J_B
                                + sum_{s<t} V4 J_A J_B J_C ]

  with A = [i,s], B = [s+1,j] for V3 and A = [i,s], B = [s+1,t], C = [t+1,j]
  for V4 (the recursion of Sec. 2.2).
* The amplitude is obtained from the (n-1)-leg current by removing its
  propagator and contracting with the last polarisation (Sec. 2.2).

Contracting the vertices of Sec. 2.2 with currents gives (every factor of i
cancels against the -i of the propagator):

    V3(P,Q) J_A J_B = i [ (J_A.J_B)(P - Q) + 2 (Q.J_A) J_B - 2 (P.J_B) J_A ]
    V4 J_A J_B J_C  = i [ 2 (J_A.J_C) J_B - (J_B.J_C) J_A - (J_A.J_B) J_C ]

so with R(i,j) the bracket divided by i,  J(i,j) = R(i,j) / P_{i,j}^2 and
only integer coefficients appear.  The value returned is

    A = eps_n . R_top,        R_top = R(1, n-1)

i.e. the paper's amplitude i * (eps_n . R_top) divided by i (no factor of i
is needed, so the same code runs over F_p with p = 3 mod 4).  The explicit
tensor form of the vertices, with the factors of i, is evaluated separately
by ``bruteforce_amplitude`` (no memoisation), which pins this contraction.

Readings taken where the paper is silent:
* singular propagator (P^2 = 0 for an internal range): status SINGULAR (1)
  and amplitude 0;
* momenta are d-dimensional, polarisations D_s-dimensional, d <= D_s; momenta
  are embedded by zero padding (Sec. 2.3, padding of lower-dimensional
  states), so dots with a momentum run over its first d components.
* metric: mostly minus diag(+,-,...,-) (Sec. 2.3) or the alternating
  diag(+,-,+,-,...) used for validation (Sec. 3.1).

The code is generic over the number type: ``fractions.Fraction``, Python
``complex``, ``mpmath.mpc`` and the prime field ``GF(p)`` below all work,
because only +, -, *, / and == are used.

``cut_state_sum`` is the sum over internal states of a ring of tree
amplitudes that a one-loop cut needs (Sec. 2.1), literal over all state
tuples.

Pins (tests/test_oracle_pins.py, tests/test_oracle_cut.py) relate this module to facts the paper and
mathematics fix: the tensor-form brute-force diagram sum, the Ward identity,
cyclic and reflection symmetry, U(1) decoupling, current conservation,
dimensional embedding, Lorentz invariance, Parke-Taylor (Sec. 3.1),
vanishing helicity amplitudes and exact-rational reduction mod p.
"""

from __future__ import annotations

import itertools
from dataclasses import dataclass, field

OK = 0
SINGULAR = 1

MOSTLY_MINUS = 0
ALTERNATING = 1


# --------------------------------------------------------------------------
# Number type: the prime field F_p (Sec. 3, finite fields with p < 2^31)
# --------------------------------------------------------------------------

class GF:
    """Element of the prime field F_p.  Plain Python integers, reduced mod p
    after every operation; the inverse is Python's modular inverse."""

    __slots__ = ("v", "p")

    def __init__(self, v, p):
        self.p = p
        self.v = int(v) % p

    def _lift(self, o):
        if isinstance(o, GF):
            if o.p != self.p:
                raise ValueError("mixing different primes")
            return o.v
        return int(o) % self.p

    def __add__(self, o):
        return GF(self.v + self._lift(o), self.p)

    __radd__ = __add__

    def __sub__(self, o):
        return GF(self.v - self._lift(o), self.p)

    def __rsub__(self, o):
        return GF(self._lift(o) - self.v, self.p)

    def __mul__(self, o):
        return GF(self.v * self._lift(o), self.p)

    __rmul__ = __mul__

    def __neg__(self):
        return GF(-self.v, self.p)

    def inverse(self):
        if self.v == 0:
            raise ZeroDivisionError("inverse of 0 in F_p")
        return GF(pow(self.v, -1, self.p), self.p)

    def __truediv__(self, o):
        return self * GF(self._lift(o), self.p).inverse()

    def __rtruediv__(self, o):
        return GF(self._lift(o), self.p) * self.inverse()

    def __eq__(self, o):
        if isinstance(o, GF):
            return self.p == o.p and self.v == o.v
        return self.v == int(o) % self.p

    def __hash__(self):
        return hash((self.v, self.p))

    def __int__(self):
        return self.v

    def __repr__(self):
        return f"GF({self.v}, {self.p})"


def to_field(x, p):
    """Map an integer, a ``Fraction`` or a field element into F_p (a / b -> a b^-1)."""
    from fractions import Fraction
    if isinstance(x, GF):
        return x
    if isinstance(x, Fraction):
        return GF(x.numerator, p) / GF(x.denominator, p)
    return GF(int(x), p)


# --------------------------------------------------------------------------
# Metric and vector helpers
# --------------------------------------------------------------------------

def metric_signs(D, metric=MOSTLY_MINUS):
    """Diagonal of the metric in D dimensions: mostly minus (Sec. 2.3) or the
    alternating diag(1,-1,1,-1,...) (Sec. 3.1)."""
    if metric == MOSTLY_MINUS:
        return [1] + [-1] * (D - 1)
    if metric == ALTERNATING:
        return [1 if mu % 2 == 0 else -1 for mu in range(D)]
    raise ValueError(f"unknown metric {metric}")


@dataclass
class Tally:
    """Operation counts of one literal evaluation (field operations)."""
    mul: int = 0
    add: int = 0
    inv: int = 0


class _Ctx:
    """Arithmetic on vectors with a metric, counting field operations."""

    def __init__(self, eta, zero, tally):
        self.eta = eta
        self.zero = zero
        self.t = tally

    def dot(self, a, b, dims):
        """sum_mu eta_mu a_mu b_mu over the first ``dims`` components."""
        acc = self.zero
        for mu in range(dims):
            term = a[mu] * b[mu]
            acc = acc + term if self.eta[mu] > 0 else acc - term
        self.t.mul += dims
        self.t.add += dims
        return acc

    def scale(self, c, v, dims):
        self.t.mul += dims
        return [c * v[mu] for mu in range(dims)] + list(v[dims:])

    def axpy(self, acc, c, v, dims):
        """acc += c * v on the first ``dims`` components."""
        self.t.mul += dims
        self.t.add += dims
        return [acc[mu] + c * v[mu] for mu in range(dims)] + list(acc[dims:])


# --------------------------------------------------------------------------
# The recursion (Sec. 2.2)
# --------------------------------------------------------------------------

@dataclass
class BGResult:
    amplitude: object
    status: int
    currents: dict = field(default_factory=dict)   # (i, j) -> J(i, j), 0-based legs
    momenta: dict = field(default_factory=dict)    # (i, j) -> P_{i,j} (D_s comps)
    r_top: list | None = None
    tally: Tally = field(default_factory=Tally)


def bg_recursion(k, eps, metric=MOSTLY_MINUS, d=None, zero=None):
    """Literal Berends-Giele recursion for one phase-space point.

    k   : n momenta, each a sequence of d components (d <= D_s), all outgoing,
          sum k = 0 (leg order = colour order, leg n last).
    eps : n polarisation vectors, each of D_s components.
    Returns a ``BGResult`` with amplitude A = eps_n . R_top (module docstring).
    """
    n = len(k)
    if n < 3 or len(eps) != n:
        raise ValueError("need n >= 3 momenta and n polarisations")
    Ds = len(eps[0])
    if d is None:
        d = len(k[0])
    if any(len(e) != Ds for e in eps) or any(len(x) != d for x in k) or d > Ds:
        raise ValueError("inconsistent dimensions")
    if zero is None:
        zero = eps[0][0] * 0
    eta = metric_signs(Ds, metric)
    tally = Tally()
    C = _Ctx(eta, zero, tally)
    N = n - 1

    # Range momenta P_{i,j} = sum_{l=i..j} k_l, zero padded to D_s (Sec. 2.2/2.3).
    P = {}
    for i in range(N):
        acc = [zero] * Ds
        for j in range(i, N):
            acc = [acc[mu] + k[j][mu] for mu in range(d)] + acc[d:]
            tally.add += d
            P[(i, j)] = acc

    J = {(i, i): list(eps[i]) for i in range(N)}
    r_top = None
    for m in range(2, N + 1):
        for i in range(0, N - m + 1):
            j = i + m - 1
            R = [zero] * Ds
            # Three-gluon vertex: split into A = [i, s], B = [s+1, j].
            for s in range(i, j):
                JA, JB = J[(i, s)], J[(s + 1, j)]
                PA, PB = P[(i, s)], P[(s + 1, j)]
                jj = C.dot(JA, JB, Ds)
                pb_ja = C.dot(PB, JA, d)
                pa_jb = C.dot(PA, JB, d)
                diff = [PA[mu] - PB[mu] for mu in range(d)]
                tally.add += d
                R = C.axpy(R, jj, diff, d)
                R = C.axpy(R, pb_ja + pb_ja, JB, Ds)
                R = C.axpy(R, -(pa_jb + pa_jb), JA, Ds)
                tally.add += 2
            # Four-gluon vertex: A = [i, s], B = [s+1, t], C = [t+1, j].
            for s in range(i, j - 1):
                for t in range(s + 1, j):
                    JA, JB, JC = J[(i, s)], J[(s + 1, t)], J[(t + 1, j)]
                    ac = C.dot(JA, JC, Ds)
                    bc = C.dot(JB, JC, Ds)
                    ab = C.dot(JA, JB, Ds)
                    R = C.axpy(R, ac + ac, JB, Ds)
                    R = C.axpy(R, -bc, JA, Ds)
                    R = C.axpy(R, -ab, JC, Ds)
                    tally.add += 1
            if m < N:
                p2 = C.dot(P[(i, j)], P[(i, j)], d)
                if p2 == zero:
                    return BGResult(zero, SINGULAR, J, P, None, tally)
                inv = 1 / p2
                tally.inv += 1
                J[(i, j)] = C.scale(inv, R, Ds)
            else:
                r_top = R
    amp = C.dot(eps[n - 1], r_top, Ds)
    return BGResult(amp, OK, J, P, r_top, tally)


def amplitude(k, eps, metric=MOSTLY_MINUS):
    """(amplitude, status) of one point; see ``bg_recursion``."""
    r = bg_recursion(k, eps, metric)
    return r.amplitude, r.status


def op_tally(n, d, Ds):
    """Field multiplications, additions and inversions of one literal
    evaluation at (n, d, D_s), counted by walking the recursion above on
    F_p inputs (the count does not depend on the values)."""
    p = 2147483629
    k = [[GF(3 + i + mu, p) for mu in range(d)] for i in range(n)]
    eps = [[GF(5 + 7 * i + mu, p) for mu in range(Ds)] for i in range(n)]
    r = bg_recursion(k, eps, MOSTLY_MINUS)
    if r.status != OK:
        raise RuntimeError("tally inputs hit a singular propagator")
    return r.tally


class _FlopValue:
    """Stand-in number that records FP64 work instead of a value.

    Only its kind is tracked: REAL (a double), COMPLEX (a pair of doubles) or
    ZERO (the exact zero every sum of the recursion starts from).  Each
    arithmetic operation adds its cost in FP64 operations to ``counter[0]``:
    a product real x real 1, real x complex 2, complex x complex 6 (four
    products and two sums); a sum or difference with a real operand 1, of two
    complex operands 2; the reciprocal of a real 1, of a complex 6
    (conj(z) / |z|^2: three for |z|^2, one division, two products).
    Operations with the exact zero and negations cost nothing, since no
    floating-point instruction is needed for them."""

    REAL, COMPLEX, ZERO = 0, 1, 2
    __slots__ = ("kind", "counter")

    def __init__(self, kind, counter):
        self.kind = kind
        self.counter = counter

    def _new(self, kind, cost):
        self.counter[0] += cost
        return _FlopValue(kind, self.counter)

    def _kind_of(self, o):
        if isinstance(o, _FlopValue):
            return o.kind
        return self.ZERO if o == 0 else self.REAL

    def __add__(self, o):
        a, b = self.kind, self._kind_of(o)
        if a == self.ZERO:
            return _FlopValue(b, self.counter)
        if b == self.ZERO:
            return _FlopValue(a, self.counter)
        both_c = a == self.COMPLEX and b == self.COMPLEX
        kind = self.COMPLEX if self.COMPLEX in (a, b) else self.REAL
        return self._new(kind, 2 if both_c else 1)

    __radd__ = __add__
    __sub__ = __add__
    __rsub__ = __add__

    def __mul__(self, o):
        a, b = self.kind, self._kind_of(o)
        if self.ZERO in (a, b):
            return _FlopValue(self.ZERO, self.counter)
        if a == self.COMPLEX and b == self.COMPLEX:
            return self._new(self.COMPLEX, 6)
        if self.COMPLEX in (a, b):
            return self._new(self.COMPLEX, 2)
        return self._new(self.REAL, 1)

    __rmul__ = __mul__

    def __neg__(self):
        return _FlopValue(self.kind, self.counter)

    def __rtruediv__(self, o):          # 1 / x, the propagator's reciprocal
        if self.kind == self.ZERO:
            raise ZeroDivisionError("reciprocal of the exact zero")
        return self._new(self.kind, 1 if self.kind == self.REAL else 6)

    def __eq__(self, o):                # only the singular-propagator test
        return self.kind == self.ZERO and self._kind_of(o) == self.ZERO

    __hash__ = object.__hash__


def flop_tally(n, d, Ds, real_momenta=True):
    """FP64 operations of one literal evaluation of the recursion above over
    complex FP64, counted by running it on ``_FlopValue`` stand-ins: momenta
    real (the physical points of Sec. 3) or complex, polarisations complex.
    The count depends only on (n, d, D_s) and the kinds of the inputs."""
    counter = [0]
    kk = _FlopValue.REAL if real_momenta else _FlopValue.COMPLEX
    k = [[_FlopValue(kk, counter) for _ in range(d)] for _ in range(n)]
    eps = [[_FlopValue(_FlopValue.COMPLEX, counter) for _ in range(Ds)] for _ in range(n)]
    r = bg_recursion(k, eps, MOSTLY_MINUS, zero=_FlopValue(_FlopValue.ZERO, counter))
    if r.status != OK:
        raise RuntimeError("flop tally hit the exact zero as a propagator")
    return counter[0]


# --------------------------------------------------------------------------
# Brute-force Feynman-diagram sum with the explicit vertex tensors
# --------------------------------------------------------------------------

def _v3_tensor(P, Q, eta, i_unit):
    """V3^{mu nu rho}(P, Q) of Sec. 2.2, all indices upper, g = diag(eta)."""
    D = len(eta)
    two = i_unit * 0 + 2
    T = {}
    for mu, nu, rho in itertools.product(range(D), repeat=3):
        v = i_unit * 0
        if nu == rho:
            v = v + eta[nu] * (P[mu] - Q[mu])
        if rho == mu:
            v = v + two * eta[rho] * Q[nu]
        if mu == nu:
            v = v - two * eta[mu] * P[rho]
        T[(mu, nu, rho)] = i_unit * v
    return T


def _v4_tensor(eta, i_unit):
    """V4^{mu nu rho sigma} of Sec. 2.2, all indices upper, g = diag(eta)."""
    D = len(eta)
    T = {}
    for mu, nu, rho, sg in itertools.product(range(D), repeat=4):
        v = 0
        if mu == rho and nu == sg:
            v += 2 * eta[mu] * eta[nu]
        if mu == nu and rho == sg:
            v -= eta[mu] * eta[rho]
        if mu == sg and nu == rho:
            v -= eta[mu] * eta[nu]
        T[(mu, nu, rho, sg)] = i_unit * v
    return T


def _lower(v, eta):
    return [eta[mu] * v[mu] for mu in range(len(eta))]


def bruteforce_diagrams(k, eps, metric, i_unit):
    """All planar cubic/quartic tree diagrams for every leg range, each
    evaluated on its own with the explicit vertex tensors and the propagator
    -i/P^2 (no memoisation: a sub-diagram list is re-expanded for every
    parent).  Returns ``(M, count)`` where M = eps_n . B_top is the paper's
    amplitude: the top bracket B_top (current without its propagator)
    contracted with the last polarisation."""
    n = len(k)
    N = n - 1
    Ds = len(eps[0])
    d = len(k[0])
    eta = metric_signs(Ds, metric)
    zero = i_unit * 0
    kk = [list(x) + [zero] * (Ds - d) for x in k]

    def mom(i, j):
        acc = [zero] * Ds
        for l in range(i, j + 1):
            acc = [acc[mu] + kk[l][mu] for mu in range(Ds)]
        return acc

    V4 = _v4_tensor(eta, i_unit)

    def brackets(i, j):
        """Yield B = V3 J J or V4 J J J for every diagram of range [i, j]."""
        for s in range(i, j):
            PA, PB = mom(i, s), mom(s + 1, j)
            V3 = _v3_tensor(PA, PB, eta, i_unit)
            for ja in diagrams(i, s):
                la = _lower(ja, eta)
                for jb in diagrams(s + 1, j):
                    lb = _lower(jb, eta)
                    out = [zero] * Ds
                    for mu in range(Ds):
                        acc = zero
                        for nu in range(Ds):
                            for rho in range(Ds):
                                acc = acc + V3[(mu, nu, rho)] * la[nu] * lb[rho]
                        out[mu] = acc
                    yield out
        for s in range(i, j - 1):
            for t in range(s + 1, j):
                for ja in diagrams(i, s):
                    la = _lower(ja, eta)
                    for jb in diagrams(s + 1, t):
                        lb = _lower(jb, eta)
                        for jc in diagrams(t + 1, j):
                            lc = _lower(jc, eta)
                            out = [zero] * Ds
                            for mu in range(Ds):
                                acc = zero
                                for nu in range(Ds):
                                    for rho in range(Ds):
                                        for sg in range(Ds):
                                            acc = acc + V4[(mu, nu, rho, sg)] * la[nu] * lb[rho] * lc[sg]
                                out[mu] = acc
                            yield out

    def diagrams(i, j):
        if i == j:
            yield list(eps[i])
            return
        P = mom(i, j)
        p2 = zero
        for mu in range(Ds):
            p2 = p2 + eta[mu] * P[mu] * P[mu]
        prop = (zero - i_unit) / p2
        for b in brackets(i, j):
            yield [prop * x for x in b]

    en = _lower(eps[n - 1], eta)
    M = zero
    count = 0
    for b in brackets(0, N - 1):
        count += 1
        for mu in range(Ds):
            M = M + en[mu] * b[mu]
    return M, count


def cut_state_sum(mats):
    """State sum over a ring of tree amplitudes (the leading pole of a
    one-loop cut, Sec. 2.1): with k trees joined in a ring by k internal legs,
    tree i given as its amplitudes M_i[s_out][s_in] for the states of its
    outgoing and incoming internal legs,

        sum over s_1..s_k of  prod_i M_i[s_{i+1}][s_i],    s_{k+1} = s_1,

    evaluated literally, term by term over all S^k state tuples.  ``mats`` is
    a list of k square nested lists (or arrays) of one number type."""
    k = len(mats)
    S = len(mats[0])
    total = None
    for states in itertools.product(range(S), repeat=k):
        term = None
        for i in range(k):
            v = mats[i][states[(i + 1) % k]][states[i]]
            term = v if term is None else term * v
        total = term if total is None else total + term
    return total
