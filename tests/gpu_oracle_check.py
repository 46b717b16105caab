"""Comparison of GPU outputs with the oracle for the GPU tests: bit-exact over
F_p, the complex tolerance rule of reading G8 (check_c64 of
test_gpu_parity) over complex FP64.  Handles explicit state-assignment tables
(output [E][H]).  No recursion arithmetic lives here: every reference value
comes from the C oracle."""

import numpy as np

from oracle import coracle as C


def _columns(eps, assign):
    """eps [E][n][S][Ds] and assign [H][n] -> list of H arrays [E][n][Ds]."""
    n = eps.shape[1]
    idx = np.arange(n)
    return [np.ascontiguousarray(eps[:, idx, assign[h], :]) for h in range(len(assign))]


def check_fp(out, status, k, eps, p, metric, assign=None):
    """out uint32 [E] (or [E][H] with an assignment table), status uint8 [E]."""
    out = np.asarray(out).view(np.uint32)
    if assign is None:
        eps = eps if eps.ndim == 3 else eps[:, :, 0, :]
        ref, rst = C.amp_fp(k, eps, p, metric)
        assert np.array_equal(out.reshape(-1), ref)
    else:
        rst = None
        for h, e_h in enumerate(_columns(eps, assign)):
            ref, rst = C.amp_fp(k, e_h, p, metric)
            assert np.array_equal(out[:, h], ref), f"assignment {h}"
    if status is not None:
        assert np.array_equal(np.asarray(status), rst)


def check_complex(out, status, k, eps, metric, assign=None, max_widened=0.03):
    """out complex128 [E] (or [E][H]); k complex128 [E][n][d] (real momenta
    as complex with zero imaginary part).  The widened-point budget is
    max_widened of the points but at least one point (a batch of a few dozen
    points may hold one ill-conditioned point); measured on the groups of the
    batch and serving tests: at most 6 of 250 points (n = 12, alternating
    metric) and 6 of 363 among the small groups."""
    from tests.test_gpu_parity import check_c64
    out = np.asarray(out)
    k = np.ascontiguousarray(k, dtype=np.complex128)
    max_widened = max(max_widened, 1.0 / max(1, k.shape[0]))
    if assign is None:
        eps = eps if eps.ndim == 3 else eps[:, :, 0, :]
        _, rst = C.amp_c64(k, eps, metric)
        check_c64(out.reshape(-1), k, eps, metric, max_widened=max_widened)
    else:
        cols = _columns(eps, assign)
        his = np.stack([C.amp_c64dd(k, e_h, metric)[0] for e_h in cols], axis=1)
        spt = np.abs(his).max(axis=1)
        for h, e_h in enumerate(cols):
            check_c64(out[:, h], k, e_h, metric, spt=spt, max_widened=max_widened)
        _, rst = C.amp_c64(k, cols[0], metric)
    if status is not None:
        assert np.array_equal(np.asarray(status), rst)
