"""Small evaluations through every kernel family of the library (the lane-group
kernel of small batches included), compared with
the oracle; run in a child process by test_gpu_bounds.py with BG_LIBRARY set to
the bounds-checked build.  Prints one JSON line: the bounds report and the
number of cases and mismatches."""

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import coracle as C  # noqa: E402
from paper_2502_07060_gb300 import inputs as G  # noqa: E402

P, PM = G.P_DEFAULT, G.P_MERSENNE
E = 97                                   # ragged: not a multiple of any block size


def main():
    import torch
    from paper_2502_07060_gb300 import bg
    torch.cuda.set_device(0)
    cases = mismatches = 0

    def dev_u32(a):
        return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()

    def fp_case(n, d, Ds, metric, p, table=None, mask=None, S=1, assign=None, mode="eval", lanes=False):
        nonlocal cases, mismatches
        k, e = G.fp_batch(100 + n * 10 + d, E, n, d, Ds, p, metric, S=S, workers=1,
                          four_d=mask or 0)
        if table:
            os.environ["BG_TABLE"] = table
        os.environ["BG_LANES"] = lanes if isinstance(lanes, str) else ("1" if lanes else "0")
        plan = bg.Plan(n, d, Ds, bg.FIELD_FP, p, metric, S, assign, four_dim_legs=mask)
        os.environ.pop("BG_TABLE", None)
        os.environ.pop("BG_LANES", None)
        if S == 1:
            ref, _ = C.amp_fp(k, e, p, metric)
        else:
            H = S ** n
            h = np.arange(H)
            a = np.stack([(h // S ** l) % S for l in range(n)], axis=1)
            eh = e[:, np.arange(n)[None, :], a, :].transpose(1, 0, 2, 3)
            kk = np.broadcast_to(k, (H,) + k.shape).reshape(H * E, *k.shape[1:])
            r, _ = C.amp_fp(np.ascontiguousarray(kk), np.ascontiguousarray(eh.reshape(H * E, n, Ds)), p, metric)
            ref = r.reshape(H, E).T
        if mode == "noalloc":
            out = torch.empty(E, dtype=torch.int32, device="cuda")
            plan.eval_noalloc(dev_u32(k), dev_u32(e), out=out)
        elif mode == "host":
            out = torch.empty(E, dtype=torch.int32).pin_memory()
            st = torch.empty(E, dtype=torch.uint8).pin_memory()
            plan.eval_host(torch.from_numpy(k.view(np.int32)).pin_memory(),
                           torch.from_numpy(e.view(np.int32)).pin_memory(), out=out, status=st, chunk=40)
        else:
            out, _ = plan.eval(dev_u32(k), dev_u32(e))
        torch.cuda.synchronize()
        cases += 1
        got = out.cpu().numpy().view(np.uint32).reshape(ref.shape)
        mismatches += int(not np.array_equal(got, ref))

    def c64_case(n, d, Ds, metric, real, lanes=False):
        nonlocal cases, mismatches
        k, e = G.c64_batch(200 + n * 10 + d, E, n, d, Ds, metric, workers=1)
        field = bg.FIELD_C64_REAL if real else bg.FIELD_C64
        os.environ["BG_LANES"] = lanes if isinstance(lanes, str) else ("1" if lanes else "0")
        plan = bg.Plan(n, d, Ds, field, 0, metric)
        os.environ.pop("BG_LANES", None)
        kd = torch.from_numpy(np.ascontiguousarray(k.real if real else k)).cuda()
        out, _ = plan.eval(kd, torch.from_numpy(e).cuda())
        torch.cuda.synchronize()
        hi, _, _ = C.amp_c64dd(k, e, metric)
        cases += 1
        rel = np.abs(out.cpu().numpy() - hi) / np.maximum(np.abs(hi), 1e-300)
        mismatches += int(np.median(rel) > 1e-10)

    for n in range(4, 13):
        for table in ("shared", "global", "split"):
            fp_case(n, 6, 6, 0, P, table)
    for n in (4, 7, 12):
        fp_case(n, 8, 8, 1, PM, "global")
        fp_case(n, 4, 6, 0, P, "shared")
        fp_case(n, 5, 7, 0, P, "global")
    for n in (5, 8, 12):
        mask = ((1 << (n - 1)) - 1) & ~1
        for table in ("shared", "global"):
            fp_case(n, 6, 8, 0, P, table, mask=mask)
    for n in (4, 8, 12):
        for d in (4, 6, 8):
            c64_case(n, d, d, 0, real=(n != 8))
    for n in (4, 6, 8, 10):
        for table in ("shared", "global"):
            fp_case(n, 4, 4, 1, PM, table, S=2, assign="all")
    fp_case(5, 6, 6, 0, P, None, S=3, assign="all")
    fp_case(8, 6, 6, 0, P, None, mode="noalloc")
    fp_case(12, 8, 8, 0, P, None, mode="noalloc")
    fp_case(9, 6, 6, 0, P, None, mode="host")
    for n in (4, 8, 12):                         # lane-group kernel of small batches
        for form in ("1", "2"):                  # one point per group, per team
            fp_case(n, 4, 4, 1, PM, None, lanes=form)
            fp_case(n, 5, 7, 0, P, None, lanes=form)
            c64_case(n, 6, 6, 0, real=(n != 8), lanes=form)
    checked, violation = bg.bounds_report()
    print(json.dumps({"checked": checked, "violation": violation, "cases": cases, "mismatches": mismatches}))


if __name__ == "__main__":
    main()
