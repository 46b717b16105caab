"""Seeded synthetic inputs: on-shell momenta and polarisation states.

This module builds phase-space points and polarisation vectors only; it holds
none of the recursion's arithmetic (no currents, vertices or propagators) and
imports neither the CUDA binding nor the oracle, so both sides of every parity
check take their inputs from here.

Constructions (arXiv:2502.07060 prepares momenta and states on the host,
Sec. 3; the recipes below are this library's, stated in its design notes):

* Null momenta over F_p, mostly-minus metric: stereographic
  ``k = E (1, 2t/(1+|t|^2), (1-|t|^2)/(1+|t|^2))`` with t uniform in
  F_p^{d-2} and E uniform in F_p^x.  Alternating metric: the projection
  ``k = v - v^2/(2 v.q) q`` of a uniform v along the null q = (1,1,0,...).
* Momentum conservation (all momenta outgoing, sum k = 0): with
  ``Q = -sum_{i<n-1} k_i`` and a seeded null r, ``lam = Q^2/(2 Q.r)``,
  ``k_{n-1} = lam r`` and ``k_n = Q - lam r``.
* Transverse states: ``eps = v - (v.q)/(k.q) k - (v.k)/(k.q) q`` with a seeded
  null reference q and seeded v, giving D_s-2 independent states per leg.
* Complex FP64: the same constructions over the reals (t ~ N(0,1), E ~
  U(1,1000)), complex v; RAMBO (Kleiss, Stirling, Ellis 1986) for physical
  four-dimensional points.
* Spinor-helicity states of Sec. 2.3: eps1 = <k|gamma|chi]/(2[k chi]) and
  eps2 = [k|gamma|chi>/<k chi>, built from two-component spinors; the
  extra-dimensional states of Sec. 2.3 (index reading documented at
  ``extra_dim_states``).

Every array function is vectorised over events with numpy; F_p values are
canonical residues in [0, p) stored as uint32 (uint64 inside).
"""

from __future__ import annotations

import os
from fractions import Fraction

import numpy as np

MOSTLY_MINUS = 0
ALTERNATING = 1

P_DEFAULT = 2147483629      # 2^31 - 19, the paper's default prime (Sec. 3)
P_MERSENNE = 2147483647     # 2^31 - 1


def metric_diag(D, metric):
    if metric == MOSTLY_MINUS:
        return np.array([1] + [-1] * (D - 1), dtype=np.int64)
    if metric == ALTERNATING:
        return np.array([1 if m % 2 == 0 else -1 for m in range(D)], dtype=np.int64)
    raise ValueError(f"unknown metric {metric}")


# --------------------------------------------------------------------------
# Vectorised arithmetic mod p on uint64 arrays (values < 2^31)
# --------------------------------------------------------------------------

def _u64(x):
    return np.asarray(x, dtype=np.uint64)


def fmul(a, b, p):
    return (_u64(a) * _u64(b)) % np.uint64(p)


def fadd(a, b, p):
    return (_u64(a) + _u64(b)) % np.uint64(p)


def fsub(a, b, p):
    return (_u64(a) + np.uint64(p) - _u64(b)) % np.uint64(p)


def fneg(a, p):
    return (np.uint64(p) - _u64(a)) % np.uint64(p)


def _fermat_inv(a, p):
    """Elementwise a^(p-2) by square-and-multiply (0 -> 0)."""
    a = _u64(a)
    r = np.ones_like(a)
    e = p - 2
    for bit in range(e.bit_length() - 1, -1, -1):
        r = (r * r) % np.uint64(p)
        if (e >> bit) & 1:
            r = (r * a) % np.uint64(p)
    return r


def finv(a, p, width=64):
    """Elementwise inverse mod p (0 -> 0).  Montgomery's simultaneous
    inversion along rows of ``width`` elements: prefix products, one Fermat
    inverse per row, then the backward sweep (about 3 products per element
    instead of ~45)."""
    a = _u64(a)
    shape = a.shape
    flat = a.reshape(-1)
    m = flat.size
    if m < 4 * width:
        return _fermat_inv(flat, p).reshape(shape)
    zero = flat == 0
    x = np.where(zero, np.uint64(1), flat)
    rows = -(-m // width)
    pad = rows * width - m
    X = np.concatenate([x, np.ones(pad, dtype=np.uint64)]).reshape(rows, width)
    pref = np.empty_like(X)
    pref[:, 0] = X[:, 0]
    for j in range(1, width):
        pref[:, j] = (pref[:, j - 1] * X[:, j]) % np.uint64(p)
    r = _fermat_inv(pref[:, -1], p)
    out = np.empty_like(X)
    for j in range(width - 1, 0, -1):
        out[:, j] = (pref[:, j - 1] * r) % np.uint64(p)
        r = (r * X[:, j]) % np.uint64(p)
    out[:, 0] = r
    out = out.reshape(-1)[:m]
    out[zero] = 0
    return out.reshape(shape)


def fdot(a, b, eta, p):
    """Metric dot over the last axis; eta is the metric diagonal (+-1)."""
    prod = fmul(a, b, p)
    pos = prod[..., eta > 0].sum(axis=-1) % np.uint64(p)
    neg = prod[..., eta < 0].sum(axis=-1) % np.uint64(p)
    return fsub(pos, neg, p)


def sqrt_minus_one(p):
    """The smaller square root of -1 mod p (p = 1 mod 4); None otherwise."""
    if p % 4 != 1:
        return None
    for a in range(2, 1000):
        if pow(a, (p - 1) // 2, p) == p - 1:          # quadratic non-residue
            r = pow(a, (p - 1) // 4, p)
            return min(r, p - r)
    raise RuntimeError("no non-residue found")


def _fp_uniform(rng, shape, p, nonzero=False):
    lo = 1 if nonzero else 0
    return rng.integers(lo, p, size=shape, dtype=np.uint64)


# --------------------------------------------------------------------------
# F_p null momenta and transverse states
# --------------------------------------------------------------------------

def fp_null_vectors(rng, shape, d, p, metric=MOSTLY_MINUS):
    """Uniform random null vectors in F_p^d, array shape ``shape + (d,)``."""
    shape = tuple(shape)
    if metric == MOSTLY_MINUS:
        # E' (1 + |t|^2, 2t, 1 - |t|^2) with E' uniform in F_p^x: the
        # stereographic vector E (1, 2t/(1+|t|^2), (1-|t|^2)/(1+|t|^2)) with
        # E = E' (1 + |t|^2), which is again uniform when 1 + |t|^2 != 0.
        out = np.empty(shape + (d,), dtype=np.uint64)
        flat = out.reshape(-1, d)
        m = flat.shape[0]
        t = _fp_uniform(rng, (m, d - 2), p)
        s = fmul(t, t, p).sum(axis=-1) % np.uint64(p)
        bad = fadd(s, 1, p) == 0
        while bad.any():
            t[bad] = _fp_uniform(rng, (int(bad.sum()), d - 2), p)
            s = fmul(t, t, p).sum(axis=-1) % np.uint64(p)
            bad = fadd(s, 1, p) == 0
        E = _fp_uniform(rng, (m,), p, nonzero=True)
        flat[:, 0] = fmul(E, fadd(s, 1, p), p)
        flat[:, 1:d - 1] = fmul(fmul(t, 2, p), E[:, None], p)
        flat[:, d - 1] = fmul(E, fsub(1, s, p), p)
        return out
    eta = metric_diag(d, metric)
    q = np.zeros(d, dtype=np.uint64)
    q[0] = 1
    q[1] = 1
    out = np.empty(shape + (d,), dtype=np.uint64)
    todo = np.ones(shape, dtype=bool)
    while todo.any():
        m = int(todo.sum())
        v = _fp_uniform(rng, (m, d), p)
        vq = fdot(v, np.broadcast_to(q, v.shape), eta, p)
        good = vq != 0
        v, vq = v[good], vq[good]
        v2 = fdot(v, v, eta, p)
        c = fmul(v2, finv(fmul(vq, 2, p), p), p)
        k = fsub(v, fmul(c[:, None], q[None, :], p), p)
        idx = np.flatnonzero(todo.ravel())[:len(v)]
        out.reshape(-1, d)[idx] = k
        flat = todo.ravel()
        flat[idx] = False
        todo = flat.reshape(shape)
    return out


def _check_four_d(four_d, n):
    if four_d >> (n - 1):
        raise ValueError("four-dimensional legs must be among 0..n-2 (leg n-1 closes the point)")


def fp_massless_point(rng, E, n, d, p, metric=MOSTLY_MINUS, four_d=0):
    """E points of n null momenta in F_p^d with sum k = 0 (all outgoing).
    four_d: bit mask of legs (among 0..n-2) whose momenta are four-dimensional
    null vectors padded with zeros; the last leg takes the remainder."""
    eta = metric_diag(d, metric)
    k = np.empty((E, n, d), dtype=np.uint64)
    if four_d:
        _check_four_d(four_d, n)
        for l in range(n - 2):
            if (four_d >> l) & 1:
                k[:, l, :4] = fp_null_vectors(rng, (E,), 4, p, metric)
                k[:, l, 4:] = 0
            else:
                k[:, l] = fp_null_vectors(rng, (E,), d, p, metric)
    else:
        k[:, :n - 2] = fp_null_vectors(rng, (E, n - 2), d, p, metric)
    Q = fneg(k[:, :n - 2].sum(axis=1) % np.uint64(p), p)
    todo = np.ones(E, dtype=bool)
    while todo.any():
        idx = np.flatnonzero(todo)
        if (four_d >> (n - 2)) & 1:
            r = np.zeros((len(idx), d), dtype=np.uint64)
            r[:, :4] = fp_null_vectors(rng, (len(idx),), 4, p, metric)
        else:
            r = fp_null_vectors(rng, (len(idx),), d, p, metric)
        Qi = Q[idx]
        qr = fdot(Qi, r, eta, p)
        q2 = fdot(Qi, Qi, eta, p)
        good = (qr != 0) & (q2 != 0)
        idx, r, Qi, qr, q2 = idx[good], r[good], Qi[good], qr[good], q2[good]
        lam = fmul(q2, finv(fmul(qr, 2, p), p), p)
        a = fmul(lam[:, None], r, p)
        k[idx, n - 2] = a
        k[idx, n - 1] = fsub(Qi, a, p)
        todo[idx] = False
    return k


def fp_transverse_states(rng, k, Ds, p, metric=MOSTLY_MINUS, S=1, four_d=0):
    """S seeded states per leg, eps [E][n][S][Ds], transverse to k (padded to
    Ds) and to a seeded null reference q per leg.  Legs in the bit mask
    four_d get four-dimensional states (reference and seed vector in the
    first four components), padded with zeros."""
    if four_d:
        eps = fp_transverse_states(rng, k, Ds, p, metric, S)
        legs = [l for l in range(k.shape[1]) if (four_d >> l) & 1]
        eps[:, legs] = 0
        eps[:, legs, :, :4] = fp_transverse_states(rng, k[:, legs, :4], 4, p, metric, S)
        return eps
    E, n, d = k.shape
    eta = metric_diag(Ds, metric)
    kp = np.zeros((E, n, Ds), dtype=np.uint64)
    kp[..., :d] = k
    q = np.empty((E, n, Ds), dtype=np.uint64)
    kq = np.zeros((E, n), dtype=np.uint64)
    todo = np.ones((E, n), dtype=bool)
    while todo.any():
        idx = np.flatnonzero(todo.ravel())
        qq = fp_null_vectors(rng, (len(idx),), Ds, p, metric)
        kk = kp.reshape(-1, Ds)[idx]
        dots = fdot(kk, qq, eta, p)
        good = dots != 0
        idx = idx[good]
        q.reshape(-1, Ds)[idx] = qq[good]
        kq.reshape(-1)[idx] = dots[good]
        flat = todo.ravel()
        flat[idx] = False
        todo = flat.reshape(E, n)
    inv_kq = finv(kq, p)
    v = _fp_uniform(rng, (E, n, S, Ds), p)
    kpS = kp[:, :, None, :]
    qS = q[:, :, None, :]
    vq = fdot(v, np.broadcast_to(qS, v.shape), eta, p)
    vk = fdot(v, np.broadcast_to(kpS, v.shape), eta, p)
    a = fmul(vq, inv_kq[:, :, None], p)
    b = fmul(vk, inv_kq[:, :, None], p)
    eps = fsub(fsub(v, fmul(a[..., None], kpS, p), p), fmul(b[..., None], qS, p), p)
    return eps


CHUNK = 1 << 16   # points per independently seeded generation chunk


def _chunk_rng(seed, c):
    """Chunk c of a batch draws from Philox seeded by (seed, c)."""
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed), int(c)])))


def _fp_chunk(seed, c, m, n, d, Ds, p, metric, S, four_d=0):
    rng = _chunk_rng(seed, c)
    k = fp_massless_point(rng, m, n, d, p, metric, four_d)
    eps = fp_transverse_states(rng, k, Ds, p, metric, S, four_d)
    return k.astype(np.uint32), (eps[:, :, 0, :] if S == 1 else eps).astype(np.uint32)


def _c64_chunk(seed, c, m, n, d, Ds, metric, S, four_d=0):
    rng = _chunk_rng(seed, c)
    k = c64_massless_point(rng, m, n, d, metric, four_d)
    eps = c64_transverse_states(rng, k, Ds, metric, S, four_d)
    return k.astype(np.complex128), (eps[:, :, 0, :] if S == 1 else eps)


def _run_chunks(fn, seed, E, args, workers):
    """Evaluate fn(seed, c, m, *args) for every chunk, in order; with
    workers > 1 the chunks run in a process pool started with 'spawn' (safe
    next to a CUDA context).  Results do not depend on ``workers``."""
    jobs = [(seed, c, min(CHUNK, E - c * CHUNK)) + tuple(args) for c in range(-(-E // CHUNK))]
    if workers is None:
        workers = 1 if E <= 4 * CHUNK else min(16, os.cpu_count() or 1)
    if workers <= 1 or len(jobs) <= 1:
        return [fn(*j) for j in jobs]
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(fn, *zip(*jobs)))


def fp_batch(seed, E, n, d, Ds, p=P_DEFAULT, metric=MOSTLY_MINUS, S=1, workers=None, four_d=0):
    """Seeded F_p batch: (k uint32 [E][n][d], eps uint32 [E][n][Ds]) when S == 1,
    else eps uint32 [E][n][S][Ds].  four_d: bit mask of four-dimensional legs
    (momenta and states zero beyond the first four components)."""
    parts = _run_chunks(_fp_chunk, seed, E, (n, d, Ds, p, metric, S, four_d), workers)
    if not parts:
        return (np.empty((0, n, d), np.uint32),
                np.empty((0, n, Ds) if S == 1 else (0, n, S, Ds), np.uint32))
    return np.concatenate([a for a, _ in parts]), np.concatenate([b for _, b in parts])


# --------------------------------------------------------------------------
# Complex FP64 momenta and transverse states
# --------------------------------------------------------------------------

def _cdot(a, b, eta):
    return (a * b * eta).sum(axis=-1)


def c64_null_vectors(rng, shape, d, metric=MOSTLY_MINUS, emax=1000.0):
    shape = tuple(shape)
    if metric == MOSTLY_MINUS:
        t = rng.standard_normal(shape + (d - 2,))
        s = (t * t).sum(axis=-1)
        E = rng.uniform(1.0, emax, size=shape)
        k = np.empty(shape + (d,), dtype=np.float64)
        k[..., 0] = E
        k[..., 1:d - 1] = 2 * t * (E / (1 + s))[..., None]
        k[..., d - 1] = E * (1 - s) / (1 + s)
        return k
    eta = metric_diag(d, metric).astype(np.float64)
    q = np.zeros(d)
    q[0] = q[1] = 1.0
    v = rng.standard_normal(shape + (d,)) * (emax / 2)
    vq = _cdot(v, q, eta)
    small = np.abs(vq) < 1e-3 * np.linalg.norm(v, axis=-1)
    while small.any():
        v[small] = rng.standard_normal((int(small.sum()), d)) * (emax / 2)
        vq = _cdot(v, q, eta)
        small = np.abs(vq) < 1e-3 * np.linalg.norm(v, axis=-1)
    v2 = _cdot(v, v, eta)
    return v - (v2 / (2 * vq))[..., None] * q


def c64_massless_point(rng, E, n, d, metric=MOSTLY_MINUS, four_d=0):
    eta = metric_diag(d, metric).astype(np.float64)
    k = np.empty((E, n, d), dtype=np.float64)
    if four_d:
        _check_four_d(four_d, n)
        for l in range(n - 2):
            if (four_d >> l) & 1:
                k[:, l, :4] = c64_null_vectors(rng, (E,), 4, metric)
                k[:, l, 4:] = 0.0
            else:
                k[:, l] = c64_null_vectors(rng, (E,), d, metric)
    else:
        k[:, :n - 2] = c64_null_vectors(rng, (E, n - 2), d, metric)
    Q = -k[:, :n - 2].sum(axis=1)
    todo = np.ones(E, dtype=bool)
    while todo.any():
        idx = np.flatnonzero(todo)
        if (four_d >> (n - 2)) & 1:
            r = np.zeros((len(idx), d))
            r[:, :4] = c64_null_vectors(rng, (len(idx),), 4, metric)
        else:
            r = c64_null_vectors(rng, (len(idx),), d, metric)
        Qi = Q[idx]
        qr = _cdot(Qi, r, eta)
        good = np.abs(qr) >= 1e-3 * np.linalg.norm(Qi, axis=-1) * np.linalg.norm(r, axis=-1)
        idx, r, Qi, qr = idx[good], r[good], Qi[good], qr[good]
        lam = _cdot(Qi, Qi, eta) / (2 * qr)
        k[idx, n - 2] = lam[:, None] * r
        k[idx, n - 1] = Qi - lam[:, None] * r
        todo[idx] = False
    return k


def c64_transverse_states(rng, k, Ds, metric=MOSTLY_MINUS, S=1, four_d=0):
    if four_d:
        eps = c64_transverse_states(rng, k, Ds, metric, S)
        legs = [l for l in range(k.shape[1]) if (four_d >> l) & 1]
        eps[:, legs] = 0
        eps[:, legs, :, :4] = c64_transverse_states(rng, k[:, legs, :4], 4, metric, S)
        return eps
    E, n, d = k.shape
    eta = metric_diag(Ds, metric).astype(np.float64)
    kp = np.zeros((E, n, Ds), dtype=np.complex128)
    kp[..., :d] = k
    q = c64_null_vectors(rng, (E, n), Ds, metric).astype(np.complex128)
    kq = _cdot(kp, q, eta)
    v = rng.standard_normal((E, n, S, Ds)) + 1j * rng.standard_normal((E, n, S, Ds))
    kpS = kp[:, :, None, :]
    qS = q[:, :, None, :]
    a = _cdot(v, qS, eta) / kq[:, :, None]
    b = _cdot(v, kpS, eta) / kq[:, :, None]
    return v - a[..., None] * kpS - b[..., None] * qS


def c64_batch(seed, E, n, d, Ds, metric=MOSTLY_MINUS, S=1, workers=None, four_d=0):
    """Seeded complex batch: (k complex128 [E][n][d] with zero imaginary part,
    eps complex128 [E][n][Ds]) when S == 1, else eps [E][n][S][Ds].  four_d as
    in fp_batch."""
    parts = _run_chunks(_c64_chunk, seed, E, (n, d, Ds, metric, S, four_d), workers)
    if not parts:
        return (np.empty((0, n, d), np.complex128),
                np.empty((0, n, Ds) if S == 1 else (0, n, S, Ds), np.complex128))
    return np.concatenate([a for a, _ in parts]), np.concatenate([b for _, b in parts])


# --------------------------------------------------------------------------
# RAMBO: flat massless phase space (Kleiss, Stirling, Ellis 1986)
# --------------------------------------------------------------------------

def rambo(rng, E, n, sqrt_s=1000.0):
    """E physical points with 2 incoming beams along +-z and n-2 massless
    outgoing momenta; returned all-outgoing (incoming legs 1, 2 negated),
    shape [E][n][4]."""
    m = n - 2
    c = 2 * rng.random((E, m)) - 1
    phi = 2 * np.pi * rng.random((E, m))
    q0 = -np.log(rng.random((E, m)) * rng.random((E, m)))
    st = np.sqrt(1 - c * c)
    q = np.stack([q0, q0 * st * np.cos(phi), q0 * st * np.sin(phi), q0 * c], axis=-1)
    Q = q.sum(axis=1)
    M = np.sqrt(Q[:, 0] ** 2 - (Q[:, 1:] ** 2).sum(axis=-1))
    b = -Q[:, 1:] / M[:, None]
    x = sqrt_s / M
    gamma = Q[:, 0] / M
    a = 1.0 / (1.0 + gamma)
    bq = (b[:, None, :] * q[..., 1:]).sum(axis=-1)
    out = np.empty((E, n, 4))
    out[:, 2:, 0] = x[:, None] * (gamma[:, None] * q[..., 0] + bq)
    out[:, 2:, 1:] = x[:, None, None] * (q[..., 1:] + b[:, None, :] * q[..., :1]
                                         + (a[:, None] * bq)[..., None] * b[:, None, :])
    half = sqrt_s / 2
    out[:, 0] = -np.array([half, 0, 0, half])
    out[:, 1] = -np.array([half, 0, 0, -half])
    return out


# --------------------------------------------------------------------------
# Two-component spinors and the helicity states of Sec. 2.3
# --------------------------------------------------------------------------
#
# A four-vector p is mapped to a 2x2 matrix M(p) with det M(p) = p^2:
#   mostly minus:  [[p0+p3, p1-i p2], [p1+i p2, p0-p3]]
#   alternating :  [[p0+p1, p3+p2], [p3-p2, p0-p1]]   (real; no i needed)
# A null p factorises as M(p) = lam lamt^T.  Brackets: <ab> = det[lam_a lam_b],
# [ab] = det[lamt_a lamt_b], so that 2 a.b = <ab>[ab].  The vector
# <a|gamma^mu|b] has matrix 2 lam_a lamt_b^T.

def vector_from_matrix(M, metric, ops):
    """Inverse of the map above; ``ops`` supplies half, i (or None), sub, add,
    mul, div for the number type in use."""
    a, b, c, dd = M
    if metric == MOSTLY_MINUS:
        p0 = ops.half(ops.add(a, dd))
        p3 = ops.half(ops.sub(a, dd))
        p1 = ops.half(ops.add(b, c))
        p2 = ops.div(ops.sub(c, b), ops.mul(ops.two, ops.i))
        return [p0, p1, p2, p3]
    p0 = ops.half(ops.add(a, dd))
    p1 = ops.half(ops.sub(a, dd))
    p3 = ops.half(ops.add(b, c))
    p2 = ops.half(ops.sub(b, c))
    return [p0, p1, p2, p3]


class FpOps:
    """Scalar arithmetic mod p for the spinor helpers (Python ints)."""

    def __init__(self, p):
        self.p = p
        self.i = sqrt_minus_one(p)
        self.two = 2
        self._half = pow(2, -1, p)

    def add(self, a, b):
        return (a + b) % self.p

    def sub(self, a, b):
        return (a - b) % self.p

    def mul(self, a, b):
        return (a * b) % self.p

    def div(self, a, b):
        return (a * pow(b % self.p, -1, self.p)) % self.p

    def half(self, a):
        return (a * self._half) % self.p

    def neg(self, a):
        return (-a) % self.p


class ComplexOps:
    i = 1j
    two = 2.0

    @staticmethod
    def add(a, b):
        return a + b

    @staticmethod
    def sub(a, b):
        return a - b

    @staticmethod
    def mul(a, b):
        return a * b

    @staticmethod
    def div(a, b):
        return a / b

    @staticmethod
    def half(a):
        return a / 2

    @staticmethod
    def neg(a):
        return -a


def angle(la, lb, ops):
    return ops.sub(ops.mul(la[0], lb[1]), ops.mul(la[1], lb[0]))


def square(ta, tb, ops):
    return ops.sub(ops.mul(ta[0], tb[1]), ops.mul(ta[1], tb[0]))


def _outer(a, b, ops, scale=None):
    m = [ops.mul(a[0], b[0]), ops.mul(a[0], b[1]), ops.mul(a[1], b[0]), ops.mul(a[1], b[1])]
    if scale is not None:
        m = [ops.mul(x, scale) for x in m]
    return m


def eps_minus(lam_k, lamt_k, lam_chi, lamt_chi, metric, ops):
    """eps1 = <k|gamma^mu|chi] / (2 [k chi]) (Sec. 2.3): matrix lam_k lamt_chi^T / [k chi]."""
    s = square(lamt_k, lamt_chi, ops)
    M = _outer(lam_k, lamt_chi, ops, ops.div(1, s))
    return vector_from_matrix(M, metric, ops)


def eps_plus(lam_k, lamt_k, lam_chi, lamt_chi, metric, ops):
    """eps2 = [k|gamma^mu|chi> / <k chi> (Sec. 2.3): matrix 2 lam_chi lamt_k^T / <k chi>."""
    a = angle(lam_k, lam_chi, ops)
    M = _outer(lam_chi, lamt_k, ops, ops.div(ops.two, a))
    return vector_from_matrix(M, metric, ops)


def spinors_from_vector_c(p):
    """(lam, lamt) with lam lamt^T = M(p) for a complex null p, mostly minus."""
    import cmath
    m00, m01, m10, m11 = p[0] + p[3], p[1] - 1j * p[2], p[1] + 1j * p[2], p[0] - p[3]
    if abs(m00) >= abs(m11):
        r = cmath.sqrt(m00)
        return [r, m10 / r], [r, m01 / r]
    r = cmath.sqrt(m11)
    return [m01 / r, r], [m10 / r, r]


def fp_spinor_point(rng, n, p, metric=MOSTLY_MINUS):
    """One F_p point from random spinors: returns (k [n][4] ints, lam, lamt)
    with sum_i lam_i lamt_i^T = 0 (the last two lamt solved)."""
    ops = FpOps(p)
    if metric == MOSTLY_MINUS and ops.i is None:
        raise ValueError("mostly-minus spinors over F_p need i in F_p (p = 1 mod 4)")
    while True:
        lam = [[int(x) for x in rng.integers(0, p, 2)] for _ in range(n)]
        lamt = [[int(x) for x in rng.integers(0, p, 2)] for _ in range(n - 2)]
        Q = [0, 0, 0, 0]
        for a in range(n - 2):
            m = _outer(lam[a], lamt[a], ops)
            Q = [ops.add(Q[t], m[t]) for t in range(4)]
        la, lb = lam[n - 2], lam[n - 1]
        ab = angle(la, lb, ops)
        if ab == 0:
            continue
        # lam_a lamt_a^T + lam_b lamt_b^T = -Q; contract with <b| and <a|.
        # <b x> for a 2x2 matrix row: (<b|Q)_j = b0 Q[1][j] - b1 Q[0][j].
        def contract(l):
            return [ops.sub(ops.mul(l[0], Q[2]), ops.mul(l[1], Q[0])),
                    ops.sub(ops.mul(l[0], Q[3]), ops.mul(l[1], Q[1]))]
        cb = contract(lb)       # <b|Q = -<b a> lamt_a
        ca = contract(la)       # <a|Q = -<a b> lamt_b
        ba = ops.neg(ab)
        lamt_a = [ops.div(ops.neg(x), ba) for x in cb]
        lamt_b = [ops.div(ops.neg(x), ab) for x in ca]
        lamt = lamt + [lamt_a, lamt_b]
        k = [vector_from_matrix(_outer(lam[a], lamt[a], ops), metric, ops) for a in range(n)]
        if any(all(c == 0 for c in v) for v in k):
            continue
        return k, lam, lamt


def extra_dim_states(k, Ds, ops_field):
    """The extra-dimensional states of Sec. 2.3 for a d-dimensional null k
    (mostly-minus metric), square-root free, as vectors of D_s components.

    Reading of the index-garbled general formula (with mu2(x) = sum of k_i^2
    over 0-based components 4 <= i < x): state s, 4 <= s <= d-2, has
    component i = k_i k_{s+1} for 4 <= i <= s, component s+1 = -mu2(s+1) and
    zero elsewhere; its conjugate is eps_s / (mu2(s+1) mu2(s+2)).  s = 4
    reproduces eps4 = {0,0,0,0,k5,-k4} times k4.
    Returns a list of (eps, eps_tilde) pairs; ``ops_field`` is a callable
    mapping ints into the number type (e.g. Fraction)."""
    d = len(k)
    zero = ops_field(0)
    out = []

    def mu2(x):
        acc = zero
        for i in range(4, x):
            acc = acc + k[i] * k[i]
        return acc

    for s in range(4, d - 1):
        e = [zero] * Ds
        for i in range(4, s + 1):
            e[i] = k[i] * k[s + 1]
        e[s + 1] = zero - mu2(s + 1)
        norm = mu2(s + 1) * mu2(s + 2)
        out.append((e, [x / norm for x in e]))
    return out


# --------------------------------------------------------------------------
# Generic scalar generator for small exact tests (Fraction or int mod p)
# --------------------------------------------------------------------------

def rational_point(rng, n, d, Ds, metric=MOSTLY_MINUS, S=1, lo=-9, hi=10):
    """One exact rational point (lists of ``Fraction``): n null momenta in d
    dims with sum 0, and S transverse states of D_s components per leg
    (constructions as in the module docstring, with small random integers)."""
    eta = [int(x) for x in metric_diag(max(d, Ds), metric)]

    def dot(a, b):
        return sum((eta[m] * a[m] * b[m] for m in range(len(a))), Fraction(0))

    def rint(nonzero=False):
        while True:
            v = int(rng.integers(lo, hi))
            if v != 0 or not nonzero:
                return Fraction(v)

    def null(D):
        if metric == MOSTLY_MINUS:
            t = [rint() / rint(True) for _ in range(D - 2)]
            s = sum((x * x for x in t), Fraction(0))
            E = rint(True)
            return [E] + [E * 2 * x / (1 + s) for x in t] + [E * (1 - s) / (1 + s)]
        while True:
            v = [rint() for _ in range(D)]
            q = [Fraction(1), Fraction(1)] + [Fraction(0)] * (D - 2)
            vq = dot(v, q)
            if vq != 0:
                c = dot(v, v) / (2 * vq)
                return [v[m] - c * q[m] for m in range(D)]

    while True:
        k = [null(d) for _ in range(n - 2)]
        Q = [-sum((k[a][m] for a in range(n - 2)), Fraction(0)) for m in range(d)]
        r = null(d)
        qr = dot(Q, r)
        q2 = dot(Q, Q)
        if qr == 0 or q2 == 0:
            continue
        lam = q2 / (2 * qr)
        k.append([lam * x for x in r])
        k.append([Q[m] - lam * r[m] for m in range(d)])
        break
    eps = []
    for a in range(n):
        kp = k[a] + [Fraction(0)] * (Ds - d)
        while True:
            q = null(Ds)
            kq = dot(kp, q)
            if kq != 0:
                break
        states = []
        for _ in range(S):
            v = [rint() for _ in range(Ds)]
            al = dot(v, q) / kq
            be = dot(v, kp) / kq
            states.append([v[m] - al * kp[m] - be * q[m] for m in range(Ds)])
        eps.append(states if S > 1 else states[0])
    return k, eps
