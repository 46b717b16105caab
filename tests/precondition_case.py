"""Inputs that break the boundary's preconditions, evaluated by the checked
build of the library (BG_LIBRARY = _build/checked/libbg.so, set by
test_gpu_preconditions.py).  Each batch holds valid points and a few points
made invalid on the host: a momentum off its mass shell, a state that is not
transverse, a non-canonical residue, momentum conservation broken while every
leg stays on shell.  Prints one JSON line: per case the points reported with
status 2, whether their amplitudes are 0, and whether every other point equals
the oracle."""

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import coracle as C  # noqa: E402
from paper_2502_07060_gb300 import inputs as G  # noqa: E402

P = G.P_DEFAULT
E = 53
BAD = [3, 7, 11, 13]


def corrupt_fp(k, eps, p):
    """The four kinds of violation on points 3, 7, 11 and 13 (eps [E][n][S][Ds])."""
    k = k.copy()
    eps = eps.copy()
    k[3, 2, 1] = (int(k[3, 2, 1]) + 1) % p                 # off shell (and not conserved)
    eps[7, 1, 0, 0] = (int(eps[7, 1, 0, 0]) + 1) % p       # state not transverse
    eps[11, 2, 0, 1] = int(eps[11, 2, 0, 1]) + p           # not canonical (same residue)
    k[13, 0] = (2 * k[13, 0].astype(np.int64)) % p         # 2 k_0: on shell, transverse, not conserved
    return k, eps


def main():
    import torch
    from paper_2502_07060_gb300 import bg
    torch.cuda.set_device(0)
    report = {"checked": bg.bounds_report()[0], "cases": []}

    def dev_u32(a):
        return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()

    def record(name, out, st, ref):
        st = st.cpu().numpy()
        bad = sorted(int(i) for i in np.nonzero(st == 2)[0])
        good = np.setdiff1d(np.arange(E), BAD)
        report["cases"].append({"case": name, "status2": bad,
                                "bad_out_zero": bool(np.all(out[BAD] == 0)),
                                "good_equal": bool(np.array_equal(out[good], ref[good])),
                                "good_status0": bool(np.all(st[good] == 0))})

    # F_p, compact kernel (both table placements) and lane-group kernel, n = 7, d = D_s = 6
    k, e = G.fp_batch(71, E, 7, 6, 6, P, 0, workers=1)
    ref, _ = C.amp_fp(k, e, P, 0)
    kb, eb = corrupt_fp(k, e[:, :, None, :], P)
    for table, lanes in (("shared", "0"), ("global", "0"), ("global", "1"), ("global", "2")):
        os.environ["BG_TABLE"] = table
        os.environ["BG_LANES"] = lanes
        plan = bg.Plan(7, 6, 6, bg.FIELD_FP, P, bg.MOSTLY_MINUS)
        os.environ.pop("BG_TABLE")
        os.environ.pop("BG_LANES")
        out, st = plan.eval(dev_u32(kb), dev_u32(eb[:, :, 0, :]))
        torch.cuda.synchronize()
        name = f"fp_compact_{table}" if lanes == "0" else "fp_lanes" if lanes == "1" else "fp_team"
        record(name, out.cpu().numpy().view(np.uint32), st, ref)
    # F_p, uneven-batch kernel (the same point body inside the persistent kernel)
    plan = bg.Plan(7, 6, 6, bg.FIELD_FP, P, bg.MOSTLY_MINUS)
    out = torch.empty(E, dtype=torch.int32, device="cuda")
    st = torch.empty(E, dtype=torch.uint8, device="cuda")
    batch = bg.Batch([(plan, dev_u32(kb), dev_u32(eb[:, :, 0, :]), out, st)])
    batch.launch()
    torch.cuda.synchronize()
    record("fp_batch", out.cpu().numpy().view(np.uint32), st, ref)
    # F_p, all-assignment kernel (two states per leg, every assignment)
    n, S = 5, 2
    k2, e2 = G.fp_batch(72, E, n, 4, 4, P, 0, S=S, workers=1)
    kb2, eb2 = corrupt_fp(k2, e2, P)
    plan = bg.Plan(n, 4, 4, bg.FIELD_FP, P, bg.MOSTLY_MINUS, S, "all")
    out, st = plan.eval(dev_u32(kb2), dev_u32(eb2))
    torch.cuda.synchronize()
    H = S ** n
    h = np.arange(H)
    a = np.stack([(h // S ** l) % S for l in range(n)], axis=1)
    eh = e2[:, np.arange(n)[None, :], a, :].transpose(1, 0, 2, 3)
    kk = np.broadcast_to(k2, (H,) + k2.shape).reshape(H * E, *k2.shape[1:])
    r, _ = C.amp_fp(np.ascontiguousarray(kk), np.ascontiguousarray(eh.reshape(H * E, n, 4)), P, 0)
    record("fp_all_assignments", out.cpu().numpy().view(np.uint32).reshape(E, H), st, r.reshape(H, E).T)
    # complex FP64, real momenta and complex momenta, n = 6, d = D_s = 4
    kc, ec = G.c64_batch(73, E, 6, 4, 4, 0, workers=1)
    hi, _, _ = C.amp_c64dd(kc, ec, 0)
    kcb, ecb = kc.copy(), ec.copy()
    kcb[3, 2, 1] *= 1.001                                  # off shell
    ecb[7, 1, 0] += 0.5                                    # not transverse
    kcb[11, 1, 3] += 0.25                                  # off shell
    kcb[13, 0] *= 2.0                                      # not conserved
    for real in (True, False):
        os.environ["BG_LANES"] = "1" if real else "0"      # the real-momentum plan on the lane kernel
        plan = bg.Plan(6, 4, 4, bg.FIELD_C64_REAL if real else bg.FIELD_C64, 0, bg.MOSTLY_MINUS)
        os.environ.pop("BG_LANES")
        kd = torch.from_numpy(np.ascontiguousarray(kcb.real if real else kcb)).cuda()
        out, st = plan.eval(kd, torch.from_numpy(ecb).cuda())
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        good = np.setdiff1d(np.arange(E), BAD)
        rel = np.abs(o - hi) / np.maximum(np.abs(hi), 1e-300)
        close = np.where(rel < 1e-8, hi, o + 1.0)          # equal to the reference within tolerance
        record("c64_real" if real else "c64", np.where(np.isin(np.arange(E), good), close, o), st, hi)
    print(json.dumps(report))


if __name__ == "__main__":
    main()
