"""Uneven batches (groups of different n, d, D_s, metric, number type and
state tables) in one graph launch: every group's output equals the oracle
(bit-exact over F_p, the complex tolerance rule of reading G8), under the
default configuration, explicit ones and the autotuned one, and reproduces
per-group bg_eval exactly (the same arithmetic runs in both)."""

import numpy as np
import pytest

from paper_2502_07060_gb300 import inputs as G
from tests.gpu_oracle_check import check_complex, check_fp

pytestmark = pytest.mark.gpu

P = G.P_DEFAULT
PM = G.P_MERSENNE


def _group(bg, field, n, d, Ds, metric, E, seed, S=1, assign=None):
    """A group and its plan; the plan's own bg_eval runs one point per thread
    at every size (BG_LANES=0), the arithmetic the batch kernels share, so the
    batch reproduces it bit for bit."""
    import os
    import torch
    os.environ["BG_LANES"] = "0"
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
    os.environ.pop("BG_LANES", None)
    H = plan.n_assign
    out = torch.empty((E,) if H == 1 else (E, H), dtype=ed.dtype, device="cuda")
    st = torch.empty(E, dtype=torch.uint8, device="cuda")
    _HOST[id(out)] = (field, metric, p if field == "fp" else 0, k, e, assign)
    return plan, kd, ed, out, st


_HOST = {}      # id(out tensor) -> the group's host inputs for the oracle


def _check_oracle(groups):
    """Every non-empty group's output and status against the oracle."""
    for plan, k, _, out, st in groups:
        if k.shape[0] == 0:
            continue
        field, metric, p, hk, he, assign = _HOST[id(out)]
        o, s = out.cpu().numpy(), st.cpu().numpy()
        if field == "fp":
            check_fp(o, s, hk, he, p, metric, assign)
        else:
            check_complex(o, s, hk, he, metric, assign)


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
    # one item per thread everywhere: bit for bit the per-group bg_eval
    batch = bg.Batch(groups, config=bg.BgBatchConfig(256, 0, 0, 0))
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
        if rep == 0:
            _check_oracle(groups)
    assert "tiles" in batch.describe()
    # the default configuration (lane groups for the small groups): the oracle,
    # and bit for bit over F_p
    default = bg.Batch(groups)
    for _, _, _, out, st in groups:
        out.zero_()
        st.fill_(7)
    default.launch()
    torch.cuda.synchronize()
    _check_oracle(groups)
    for (plan, k, _, out, st), ref in zip(groups, refs):
        if ref is not None and plan.field == bg.FIELD_FP:
            assert torch.equal(out, ref[0]) and torch.equal(st, ref[1])


def test_batch_config_variants_and_autotune():
    import torch
    from paper_2502_07060_gb300 import bg
    groups = [_group(bg, *s, seed=80 + i) for i, s in enumerate(SPECS[:7])]
    refs = [plan.eval(k, e)[0] for plan, k, e, _, _ in groups]
    # explicit configurations: caps (both F_p kernel builds: caps 1-2 the wide
    # one, 0 and 3-4 the one for four blocks), tile sizes, every group on lane
    # groups
    for cfg in (bg.BgBatchConfig(256, 2, 1, 0), bg.BgBatchConfig(4096, 0, 3, 0), bg.BgBatchConfig(64, 3, 2, 0),
                bg.BgBatchConfig(1024, 0, 0, 1 << 20), bg.BgBatchConfig(256, 1, 0, 1 << 20)):
        for _, _, _, out, st in groups:
            out.zero_()
            st.fill_(7)
        batch = bg.Batch(groups, config=cfg)
        assert ("kernel=wide" in batch.describe()) == (cfg.fp_blocks_per_sm in (1, 2))
        batch.launch()
        torch.cuda.synchronize()
        for (plan, _, _, out, _), ref in zip(groups, refs):
            if cfg.lanes_max_items == 0 or plan.field == bg.FIELD_FP:   # lane sums round differently
                assert torch.equal(out, ref)
        _check_oracle(groups)
    best, ms = bg.Batch.autotune(groups, reps=1)
    assert best.tile_points in (64, 256, 1024, 4096) and best.lanes_max_items in (0, 2048) and ms > 0
    for _, _, _, out, st in groups:
        out.zero_()
        st.fill_(7)
    tuned = bg.Batch(groups, config=best)
    tuned.launch()
    torch.cuda.synchronize()
    _check_oracle(groups)


def test_autotune_cache(tmp_path, monkeypatch):
    """With BG_AUTOTUNE_CACHE set, the first autotune of a group mix times the
    candidates and appends its result; the next one for the same mix reads it
    back without timing; a different mix gets its own entry."""
    from paper_2502_07060_gb300 import bg
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("BG_AUTOTUNE_CACHE", str(cache))
    groups = [_group(bg, *s, seed=120 + i) for i, s in enumerate(SPECS[:3])]
    best, ms = bg.Batch.autotune(groups, reps=1)
    lines = cache.read_text().split("\n")
    lines = [l for l in lines if l.strip()]
    assert len(lines) == 1
    key, t, fc, cc, ln, m = lines[0].split()
    assert (int(t), int(fc), int(cc), int(ln)) == (best.tile_points, best.fp_blocks_per_sm, best.c64_blocks_per_sm,
                                                   best.lanes_max_items)
    again, ms2 = bg.Batch.autotune(groups, reps=1)
    assert (again.tile_points, again.fp_blocks_per_sm, again.c64_blocks_per_sm, again.lanes_max_items) == \
        (best.tile_points, best.fp_blocks_per_sm, best.c64_blocks_per_sm, best.lanes_max_items)
    assert abs(ms2 - float(m)) < 1e-5
    assert len([l for l in cache.read_text().split("\n") if l.strip()]) == 1
    other = [_group(bg, *s, seed=130 + i) for i, s in enumerate(SPECS[3:5])]
    bg.Batch.autotune(other, reps=1)
    keys = [l.split()[0] for l in cache.read_text().split("\n") if l.strip()]
    assert len(keys) == 2 and keys[0] != keys[1]


def test_small_groups_on_lane_groups():
    """A batch of small groups (every configuration of the uneven workload, a
    few dozen points each) with lane groups for groups up to 2048 items: every
    group equals the oracle, and equals the same batch run one item per
    thread bit for bit over F_p."""
    import torch
    from paper_2502_07060_gb300 import bg
    specs = [(f, n, d, d, m, 20 + 7 * i) for i, (f, n, d, m) in enumerate(
        [(f, n, d, m) for f in ("fp", "c64", "c64r") for n in (4, 7, 12) for d in (4, 6, 8) for m in (0, 1)])]
    groups = [_group(bg, *s[:5], s[5], seed=300 + i) for i, s in enumerate(specs)]
    lanes = bg.Batch(groups, config=bg.BgBatchConfig(256, 0, 0, 2048))
    lanes.launch()
    torch.cuda.synchronize()
    _check_oracle(groups)
    got = [out.clone() for _, _, _, out, _ in groups]
    plain = bg.Batch(groups, config=bg.BgBatchConfig(256, 0, 0, 0))
    plain.launch()
    torch.cuda.synchronize()
    for (plan, _, _, out, _), g in zip(groups, got):
        if plan.field == bg.FIELD_FP:
            assert torch.equal(out, g)
