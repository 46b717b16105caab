"""Uneven batches (groups of different n, d, D_s, metric, number type and
state tables) in one graph launch reproduce per-group bg_eval exactly: the
same arithmetic runs in both, so F_p and complex results are bit-identical."""

import numpy as np
import pytest

from paper_2502_07060_gb300 import inputs as G

pytestmark = pytest.mark.gpu

P = G.P_DEFAULT
PM = G.P_MERSENNE


def _group(bg, field, n, d, Ds, metric, E, seed, S=1, assign=None):
    import torch
    if field == "fp":
        p = P if metric == 0 else PM
        k, e = G.fp_batch(seed, E, n, d, Ds, p, metric, S=S, workers=1)
        kd = torch.from_numpy(k.view(np.int32)).cuda()
        ed = torch.from_numpy(e.view(np.int32)).cuda()
        plan = bg.Plan(n, d, Ds, bg.FIELD_FP, p, metric, S, assign)
    else:
        k, e = G.c64_batch(seed, E, n, d, Ds, metric, S=S, workers=1)
        if field == "c64r":                       # real momenta
            kd = torch.from_numpy(np.ascontiguousarray(k.real)).cuda()
        else:
            kd = torch.from_numpy(k).cuda()
        ed = torch.from_numpy(e).cuda()
        fid = bg.FIELD_C64_REAL if field == "c64r" else bg.FIELD_C64
        plan = bg.Plan(n, d, Ds, fid, 0, metric, S, assign)
    H = plan.n_assign
    out = torch.empty((E,) if H == 1 else (E, H), dtype=ed.dtype, device="cuda")
    st = torch.empty(E, dtype=torch.uint8, device="cuda")
    return plan, kd, ed, out, st


SPECS = [("fp", 4, 4, 4, 0, 3000), ("fp", 8, 6, 6, 0, 5000), ("fp", 12, 8, 8, 1, 700),
         ("fp", 7, 5, 7, 1, 1234), ("c64", 5, 4, 4, 0, 999), ("c64", 8, 6, 6, 1, 1500),
         ("c64", 11, 8, 8, 0, 300), ("fp", 6, 4, 6, 0, 0), ("c64", 9, 6, 8, 0, 400),
         ("c64r", 8, 6, 6, 0, 1300), ("c64r", 12, 4, 8, 1, 250)]


def test_batch_matches_per_group_eval():
    import torch
    from paper_2502_07060_gb300 import bg
    groups = [_group(bg, *s, seed=50 + i) for i, s in enumerate(SPECS)]
    assign = np.array([[(h >> l) & 1 for l in range(6)] for h in range(64)], dtype=np.uint8)
    groups.append(_group(bg, "fp", 6, 4, 4, 1, 200, 99, S=2, assign=assign))
    groups.append(_group(bg, "c64", 6, 4, 4, 0, 150, 98, S=2, assign=assign))
    groups.append(_group(bg, "c64r", 6, 4, 4, 1, 120, 97, S=2, assign=assign))
    refs = []
    for plan, k, e, _, _ in groups:
        if k.shape[0] == 0:
            refs.append(None)
            continue
        refs.append(plan.eval(k, e))
    batch = bg.Batch(groups)
    for rep in range(2):                               # counters are reset per launch
        for _, _, _, out, st in groups:
            out.zero_()
            st.fill_(7)
        batch.launch()
        torch.cuda.synchronize()
        for (plan, k, _, out, st), ref in zip(groups, refs):
            if ref is None:
                continue
            assert torch.equal(out, ref[0]), plan.describe()
            assert torch.equal(st, ref[1])
    assert "tiles" in batch.describe()


def test_batch_config_variants_and_autotune():
    import torch
    from paper_2502_07060_gb300 import bg
    groups = [_group(bg, *s, seed=80 + i) for i, s in enumerate(SPECS[:7])]
    refs = [plan.eval(k, e)[0] for plan, k, e, _, _ in groups]
    for cfg in (bg.BgBatchConfig(256, 2, 1), bg.BgBatchConfig(4096, 0, 3)):
        batch = bg.Batch(groups, config=cfg)
        batch.launch()
        torch.cuda.synchronize()
        for (_, _, _, out, _), ref in zip(groups, refs):
            assert torch.equal(out, ref)
    best, ms = bg.Batch.autotune(groups, reps=1)
    assert best.tile_points in (256, 1024, 4096) and ms > 0
