"""Benchmark: amplitudes/s of the batched Berends-Giele recursion, n = 8
gluons, d = D_s = 6, over F_p (p = 2^31 - 19) and complex FP64.

One step = one bg_eval over a batch of E synthetic points (all steps of the
hot path run inside that one kernel launch).  Inputs are resident in HBM
before the timed region and larger than L2 (E = 2^22: 1.6 GB for F_p, 6.4 GB
for C64), so no L2 flush is needed between steps.  Timing: W warm-up steps,
then K steps bracketed by barrier + synchronize, timed with CUDA events on
the launching stream; max over ranks.  The printed JSON line's headline
``value`` is F_p amplitudes/s; the complex FP64 leg is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: ``--gpus N`` started as a plain process re-runs itself as N ranks
under torch.distributed.run (started by torchrun, it reads RANK, LOCAL_RANK
and WORLD_SIZE from the environment).  Each rank evaluates its own
independent batch on its own GPU (weak scaling, no data-path collective); the
process group only provides the barrier and the max over ranks of the elapsed
time.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2502_07060_gb300 import inputs as G  # noqa: E402

N_LEG, D, DS = 8, 6, 6
P = G.P_DEFAULT
METRIC = "amplitudes/s for n=8 gluons, d=6 (F_p, C64); serving p50/p99 vs plain launches"


def literal_tally(n, d, Ds):
    """Field multiplications and additions of the literal recursion at
    (n, d, D_s) (the oracle's tally, a closed combinatorial formula)."""
    from math import comb
    mul = comb(n, 3) * (3 * Ds + 3 * d) + comb(n, 4) * 6 * Ds + (comb(n, 2) - n) * (d + Ds) + Ds
    add = None
    return mul, add


def literal_flops(n, d, Ds, real_k):
    """FP64 operations of the literal recursion at (n, d, D_s) over complex
    FP64 (the oracle's FLOP tally, a closed formula): products real x real 1,
    real x complex 2, complex x complex 6; sums 1 with a real operand, 2 with
    two complex ones; reciprocal 1 (real) or 6 (complex); nothing for
    negations and for sums that start from zero.  real_k: real momenta (the
    physical points)."""
    N = n - 1
    tot = 0
    for m in range(2, N + 1):
        s3, s4 = m - 1, (m - 1) * (m - 2) // 2
        per = s4 * (48 * Ds - 4) - 2 * Ds
        if real_k:
            per += s3 * (24 * Ds + 13 * d - 2)
            if m < N:
                per += 2 * d + 2 * Ds                  # P^2, reciprocal, J = R / P^2
        else:
            per += s3 * (24 * Ds + 26 * d - 2)
            if m < N:
                per += 8 * d + 4 + 6 * Ds
        tot += (N - m + 1) * per
    tot += 8 * Ds - 2                                   # final contraction
    tot += (1 if real_k else 2) * d * N * (N - 1) // 2  # range momenta
    return tot


def kernel_mults(n, d, Ds):
    """Field multiplications the CUDA kernel performs per amplitude in its
    regrouped form (dots shared between V3 and V4, one scalar-vector product
    per sub-current, batched inversion), conversion of the momenta to
    Montgomery form included (the states enter as canonical residues)."""
    N = n - 1
    tot = 0
    for m in range(2, N + 1):
        ranges = N - m + 1
        per = (m - 1) * Ds                       # adjacent dots
        per += (m - 1) * 2 * d                   # P.J_B and P.J_A (range momentum P)
        per += (m - 1) * d                       # momentum part of V3
        per += (m - 1) * 2 * Ds                  # prefix and suffix scalar-vector products
        per += (m - 1) * (m - 2) // 2 * 2 * Ds   # gap dots and inner scalar-vector products
        if m < N:
            per += Ds + d                        # J = R / P^2 and P^2
        tot += ranges * per
    ns = N * (N + 1) // 2 - N - 1
    tot += 3 * ns + 45                           # batched inverse + one Fermat power (~45)
    tot += Ds                                    # final contraction
    tot += N * d                                 # momenta to Montgomery form
    return tot


def kernel_fp64_ops(n, d, Ds, real_k):
    """FP64-pipe instructions (FMA, add and multiply each count one) the
    complex kernel issues per amplitude in its regrouped form, a model count
    from the kernel's structure.  real_k: momenta real (two FMAs per momentum
    component in P.J and in the momentum term instead of four)."""
    N = n - 1
    kc = 1 if real_k else 2                    # adds per momentum component
    km = 2 if real_k else 4                    # FMAs per momentum-current component
    tot = 0
    for m in range(2, N + 1):
        ranges = N - m + 1
        per = (m - 1) * 4 * Ds                   # adjacent dots
        per += (m - 1) * 2 * d * km              # P.J_B and P.J_A (current conservation)
        per += (m - 1) * (2 + 2 + 4 + 2)         # coefficient algebra (SA, doubling)
        per += (m - 1) * 8 * Ds                  # prefix and suffix scalar-vector products
        per += (m - 1) * d * km                  # momentum term
        per += (m - 1) * (m - 2) // 2 * (8 * Ds + 2)   # gap dots and inner products
        per += 2 * d * kc + d * km               # P = K_j - K_i, K_i + K_j and -SA (K_i + K_j)
        if m < N:
            per += Ds * (2 if real_k else 4)     # J = R / P^2
            per += d * kc + d * (1 if real_k else 4)   # P^2
            per += 8 if real_k else 12           # reciprocal (Newton steps), complex scaling
        tot += ranges * per
    tot += 4 * Ds                                # final contraction
    tot += N * d * kc                            # prefix sums of the momenta
    return tot


KERNEL_SOURCES = ("paper_2502_07060_gb300/csrc/bg_compact.cuh", "paper_2502_07060_gb300/csrc/bg_field.cuh")


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel):
    """DRAM bytes per 2^22-point launch of `kernel` ("fp" or "c64") from
    bench_traffic.json (ncu counters of a smaller capture scaled by the point
    count), or None when the kernel sources changed since that capture."""
    try:
        with open(os.path.join(ROOT, "bench_traffic.json")) as f:
            rec = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    return float(rec["dram_bytes_per_launch_2p22"])


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [x.strip() for x in l.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------
# distributed plumbing (barrier and max over ranks only)
# --------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist if world > 1 else None


def max_over_ranks(x, dist, device):
    """Largest value of x over the ranks (the step time of the slowest rank)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def launch_ranks(n):
    """Re-run this command as n replica ranks (one process per GPU) under
    torch.distributed.run on this node; returns the launcher's exit code."""
    import socket
    with socket.socket() as sock:
        sock.bind(("127.0.0.1", 0))
        port = sock.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


def launch_check(args, rank, world):
    """The multi-rank path without a GPU (gloo): every rank builds its own
    seeded batch of the metric's workload, times that as its step, and rank 0
    prints the aggregated line with each rank's seed and input digest."""
    import hashlib
    import torch
    dist = init_dist(world, "gloo")
    E = 1 << args.log2_points
    seed = rank_seed(1000, rank)
    t0 = time.perf_counter()
    k, e = G.fp_batch(seed, E, N_LEG, D, DS, P, 0, workers=1)
    ms = (time.perf_counter() - t0) * 1e3
    ms_max = max_over_ranks(ms, dist, torch.device("cpu"))
    mine = {"rank": rank, "seed": seed, "points": E,
            "digest": hashlib.sha256(k.tobytes() + e.tobytes()).hexdigest()[:16]}
    ranks = [mine]
    if dist is not None:
        ranks = [None] * world
        dist.all_gather_object(ranks, mine)
    if rank == 0:
        print(json.dumps({"metric": METRIC, "launch_check": True, "n_gpus": world, "ms_per_step": ms_max,
                          "value": job_value(E, world, ms_max), "scaling": "weak", "ranks": ranks}))
    if dist is not None:
        dist.destroy_process_group()


def rank_seed(base, rank):
    """Each rank evaluates its own independent batch (weak scaling)."""
    return base + rank


def job_value(points_per_rank, world, ms_max):
    """Whole-job amplitudes/s: the points of all ranks over the slowest rank's time."""
    return world * points_per_rank / (ms_max / 1e3)


# --------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, on the host cores
# --------------------------------------------------------------------------

def cpu_baseline(field, target_s=10.0):
    from oracle import coracle
    threads = coracle.max_threads()
    m = 1 << 12
    while True:
        if field == "fp":
            k, e = G.fp_batch(777, m, N_LEG, D, DS, P, 0)
            t0 = time.perf_counter()
            coracle.amp_fp(k, e, P, 0)
        else:
            k, e = G.c64_batch(777, m, N_LEG, D, DS, 0)
            t0 = time.perf_counter()
            coracle.amp_c64(k, e, 0)
        dt = time.perf_counter() - t0
        if dt >= target_s / 4 or m >= (1 << 20):
            break
        m = int(m * min(16.0, max(2.0, target_s / max(dt, 1e-3))))
        m = 1 << max(12, min(20, m.bit_length() - 1))
    return {"value": m / dt, "unit": "amplitudes/s", "cores": threads, "kind": "oracle",
            "sample": f"{m} points of the n=8 d=D_s=6 {field} workload, C oracle (gcc -O3 "
                      f"-ffp-contract=off, OpenMP, one point per iteration), {dt:.2f} s"}


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------

def time_steps(fn, steps, warmup, stream, dist, device):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        fn()
    end.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = start.elapsed_time(end)
    return max_over_ranks(ms, dist, device)


def run_field(field, E, steps, warmup, rank, dist, device, seed, e2e=True):
    import torch
    from paper_2502_07060_gb300 import bg
    if field == "fp":
        k, e = G.fp_batch(seed, E, N_LEG, D, DS, P, 0)
        plan = bg.Plan(N_LEG, D, DS, bg.FIELD_FP, P, bg.MOSTLY_MINUS)
        hk = torch.from_numpy(k.view(np.int32))
        he = torch.from_numpy(e.view(np.int32))
    else:
        # physical points: real momenta (stored with zero imaginary part)
        k, e = G.c64_batch(seed, E, N_LEG, D, DS, 0)
        if field == "c64":
            plan = bg.Plan(N_LEG, D, DS, bg.FIELD_C64_REAL, 0, bg.MOSTLY_MINUS)
            hk = torch.from_numpy(np.ascontiguousarray(k.real))
        else:                                   # "c64c": the general complex-momentum plan
            plan = bg.Plan(N_LEG, D, DS, bg.FIELD_C64, 0, bg.MOSTLY_MINUS)
            hk = torch.from_numpy(k)
        he = torch.from_numpy(e)
    del k, e
    dk = hk.to(device)
    de = he.to(device)
    out = torch.empty(E, dtype=de.dtype, device=device)
    st = torch.empty(E, dtype=torch.uint8, device=device)
    ws = plan.workspace(E, device)
    stream = torch.cuda.current_stream(device)

    def step():
        plan.eval(dk, de, out=out, status=st, workspace=ws, stream=stream)

    with ClockSampler(device.index if device.index is not None else 0) as clk:
        ms = time_steps(step, steps, warmup, stream, dist, device)
    clocks = clk.summary()

    res = {
        "ms_per_step": ms / steps,
        "value_per_rank": E / (ms / steps / 1e3),
        "clocks": clocks,
        "plan": plan.describe(),
    }
    if not e2e:
        return res
    # end to end through the public C-ABI call with HOST buffers
    # (bg_eval_host), pinned inputs and results: every byte crosses the host
    # link each step, either by chunked copies overlapping the kernels (F_p)
    # or read and written in place by the kernel (complex FP64, whose
    # arithmetic per point hides the link traffic)
    pk = hk.pin_memory()
    pe = he.pin_memory()
    hout = torch.empty(E, dtype=de.dtype).pin_memory()
    hst = torch.empty(E, dtype=torch.uint8).pin_memory()
    del dk, de, out, st, ws
    torch.cuda.empty_cache()
    chunk = max(1, E // 16)

    def e2e_step():
        plan.eval_host(pk, pe, out=hout, status=hst, chunk=chunk, stream=stream)

    e2e_steps = max(3, min(steps, 20))
    ms_e2e = time_steps(e2e_step, e2e_steps, 2, stream, dist, device)
    res.update({
        "e2e_ms_per_step": ms_e2e / e2e_steps,
        "e2e_chunk": chunk,
        "h2d_bytes": pk.numel() * pk.element_size() + pe.numel() * pe.element_size(),
        "d2h_bytes": hout.numel() * hout.element_size() + hst.numel(),
    })
    plan._staging = None
    torch.cuda.empty_cache()
    return res


def mixed_workload(args, device):
    """Uneven batches over n = 4..12, d = D_s in {4, 6, 8} and both number
    types (54 groups): 2^22 points spread evenly (about 78 k per group), and
    54 small groups of 512 points (the request mix of a serving step), and
    2^22 points over the 27 F_p groups alone.  Each times (a) the plain
    per-group bg_eval launches (which take the lane-group kernel for small
    groups), (b) one graph launch of the batch with the default configuration
    and (c) with the autotuned configuration (tile size, residency caps and
    with them the F_p kernel build, lane groups for small groups)."""
    return {"large": _mixed(args, device, (1 << args.log2_points) // 54, 3000),
            "small": _mixed(args, device, 512, 3100),
            "fp_large": _mixed(args, device, (1 << args.log2_points) // 27, 3200, fields=("fp",))}


def _mixed(args, device, per, seed0, fields=("fp", "c64")):
    import torch
    from paper_2502_07060_gb300 import bg
    specs = [(f, n, d) for f in fields for n in range(4, 13) for d in (4, 6, 8)]
    groups = []
    for i, (f, n, d) in enumerate(specs):
        if f == "fp":
            k, e = G.fp_batch(seed0 + i, per, n, d, d, P, 0)
            kd = torch.from_numpy(k.view(np.int32)).to(device)
            ed = torch.from_numpy(e.view(np.int32)).to(device)
            plan = bg.Plan(n, d, d, bg.FIELD_FP, P, bg.MOSTLY_MINUS)
        else:
            k, e = G.c64_batch(seed0 + i, per, n, d, d, 0)
            kd = torch.from_numpy(k).to(device)
            ed = torch.from_numpy(e).to(device)
            plan = bg.Plan(n, d, d, bg.FIELD_C64, 0, bg.MOSTLY_MINUS)
        del k, e
        out = torch.empty(per, dtype=kd.dtype, device=device)
        st = torch.empty(per, dtype=torch.uint8, device=device)
        groups.append((plan, kd, ed, out, st))
    stream = torch.cuda.current_stream(device)
    wss = [plan.workspace(per, device) for plan, *_ in groups]

    def plain():
        for (plan, kd, ed, out, st), ws in zip(groups, wss):
            plan.eval(kd, ed, out=out, status=st, workspace=ws, stream=stream)

    steps = max(3, args.steps // 10)
    ms_plain = time_steps(plain, steps, args.warmup, stream, None, device)
    batch = bg.Batch(groups)
    ms_batch = time_steps(lambda: batch.launch(stream), steps, args.warmup, stream, None, device)
    desc_default = batch.describe()
    del batch
    best, _ = bg.Batch.autotune(groups, reps=1, stream=stream)
    tuned = bg.Batch(groups, config=best)
    ms_tuned = time_steps(lambda: tuned.launch(stream), steps, args.warmup, stream, None, device)
    n_pts = per * len(specs)
    what = "F_p and C64" if len(fields) == 2 else "F_p"
    return {"workload": f"uneven batch: {len(specs)} groups (n = 4..12, d = D_s in {{4, 6, 8}}, {what}), "
                        f"{per} points each, {n_pts} points per step",
            "plain_launches": {"ms_per_step": ms_plain / steps, "value": n_pts / (ms_plain / steps / 1e3),
                               "launches_per_step": len(specs)},
            "batch_default": {"ms_per_step": ms_batch / steps, "value": n_pts / (ms_batch / steps / 1e3),
                              "describe": desc_default},
            "batch_autotuned": {"ms_per_step": ms_tuned / steps, "value": n_pts / (ms_tuned / steps / 1e3),
                                "config": {"tile_points": best.tile_points,
                                           "fp_blocks_per_sm": best.fp_blocks_per_sm,
                                           "c64_blocks_per_sm": best.c64_blocks_per_sm,
                                           "lanes_max_items": best.lanes_max_items},
                                "describe": tuned.describe()},
            "unit": "amplitudes/s", "steps": steps}


def helicity_workload(args, device):
    """All 2^n helicity assignments (n = 6..10, d = D_s = 4, two states per
    leg): F_p at p = 2^31 - 1 in the alternating metric and complex FP64 on
    physical points (real momenta), 2^20 points per n.  Times the
    all-assignment plan (shared sub-currents) on the full batch, and the same
    assignments as an explicit table (one full recursion per assignment) on
    the first 2^18 (F_p) / 2^15 (complex) points of it."""
    import torch
    from paper_2502_07060_gb300 import bg
    res = []
    steps = 3
    E = 1 << args.log2_points_helicity
    for field in ("fp", "c64"):
        E_cmp = min(E, 1 << (18 if field == "fp" else 15))
        for n in range(6, 11):
            H = 1 << n
            table = np.array([[(h >> l) & 1 for l in range(n)] for h in range(H)], dtype=np.uint8)
            if field == "fp":
                k, e = G.fp_batch(4000 + n, E, n, 4, 4, G.P_MERSENNE, 1, S=2)
                kd = torch.from_numpy(k.view(np.int32)).to(device)
                ed = torch.from_numpy(e.view(np.int32)).to(device)
                mk = lambda a: bg.Plan(n, 4, 4, bg.FIELD_FP, G.P_MERSENNE, bg.ALTERNATING, 2, a)
            else:
                k, e = G.c64_batch(4000 + n, E, n, 4, 4, 0, S=2)
                kd = torch.from_numpy(np.ascontiguousarray(k.real)).to(device)
                ed = torch.from_numpy(e).to(device)
                mk = lambda a: bg.Plan(n, 4, 4, bg.FIELD_C64_REAL, 0, bg.MOSTLY_MINUS, 2, a)
            del k, e
            out = torch.empty((E, H), dtype=ed.dtype, device=device)
            st = torch.empty(E, dtype=torch.uint8, device=device)
            stream = torch.cuda.current_stream(device)
            row = {"field": field, "n": n, "points": E, "points_per_assignment_run": E_cmp,
                   "assignments": H}
            for mode, a, m in (("shared_currents", "all", E), ("per_assignment", table, E_cmp)):
                plan = mk(a)
                ws = plan.workspace(m, device)
                kv, ev, ov, sv = kd[:m], ed[:m], out[:m], st[:m]
                ms = time_steps(lambda: plan.eval(kv, ev, out=ov, status=sv, workspace=ws, stream=stream),
                                steps, args.warmup, stream, None, device)
                row[mode] = {"ms_per_step": ms / steps, "value": m * H / (ms / steps / 1e3),
                             "plan": plan.describe()}
                del plan, ws
            row["speedup"] = row["shared_currents"]["value"] / row["per_assignment"]["value"]
            res.append(row)
            del kd, ed, out, st
            torch.cuda.empty_cache()
    return {"workload": "all 2^n helicity assignments, n = 6..10, d = D_s = 4, S = 2 states per leg, "
                        f"{E} points per n; F_p p = 2^31-1 (alternating metric) and complex FP64 with "
                        "real momenta",
            "unit": "amplitudes/s", "steps": steps, "rows": res}


def sweep_workload(args, device):
    """Scaling of one bg_eval launch, the analogues of the paper's benchmark
    figures (Sec. 3.2): time against the number of points E = 2^10..2^22 at
    n = 8, d = D_s = 6 (Fig. 1b: flat until the GPU saturates, then linear);
    against the number of gluons n = 4..12 at d = D_s = 8 (Fig. 1a); against
    the dimension d = D_s = 4..8 at n = 6 and 9 (Fig. 2).  F_p at p = 2^31 - 19
    and complex FP64 with real momenta (physical points), mostly-minus metric.
    Each entry: 3 warm-up calls, then CUDA-event timing of enough calls to
    cover 50 ms (at least 3)."""
    import torch
    from paper_2502_07060_gb300 import bg
    stream = torch.cuda.current_stream(device)

    def inputs(field, seed, E, n, d):
        if field == "fp":
            k, e = G.fp_batch(seed, E, n, d, d, P, 0)
            plan = bg.Plan(n, d, d, bg.FIELD_FP, P, bg.MOSTLY_MINUS)
            return plan, torch.from_numpy(k.view(np.int32)).to(device), torch.from_numpy(e.view(np.int32)).to(device)
        k, e = G.c64_batch(seed, E, n, d, d, 0)
        plan = bg.Plan(n, d, d, bg.FIELD_C64_REAL, 0, bg.MOSTLY_MINUS)
        return (plan, torch.from_numpy(np.ascontiguousarray(k.real)).to(device),
                torch.from_numpy(e).to(device))

    def measure(plan, kd, ed, E):
        out = torch.empty(E, dtype=ed.dtype, device=device)
        st = torch.empty(E, dtype=torch.uint8, device=device)
        ws = plan.workspace(E, device)
        kv, ev = kd[:E], ed[:E]
        step = lambda: plan.eval(kv, ev, out=out, status=st, workspace=ws, stream=stream)
        one = time_steps(step, 1, 3, stream, None, device)
        reps = int(min(200, max(3, np.ceil(50.0 / max(one, 1e-3)))))
        ms = time_steps(step, reps, 1, stream, None, device) / reps
        return {"E": E, "ms_per_call": ms, "amplitudes_per_s": E / (ms / 1e3), "calls": reps}

    res = {"E_sweep": [], "n_sweep": [], "d_sweep": []}
    for field, top in (("fp", 22), ("c64", 20)):
        plan, kd, ed = inputs(field, 5100, 1 << top, 8, 6)
        for lg in range(10, top + 1):
            res["E_sweep"].append(dict(field=field, n=8, d=6, **measure(plan, kd, ed, 1 << lg)))
        del kd, ed
        torch.cuda.empty_cache()
    for field, lg in (("fp", 20), ("c64", 17)):
        for n in range(4, 13):
            plan, kd, ed = inputs(field, 5200 + n, 1 << lg, n, 8)
            res["n_sweep"].append(dict(field=field, n=n, d=8, **measure(plan, kd, ed, 1 << lg)))
        for n in (6, 9):
            for d in range(4, 9):
                plan, kd, ed = inputs(field, 5300 + 10 * n + d, 1 << lg, n, d)
                res["d_sweep"].append(dict(field=field, n=n, d=d, **measure(plan, kd, ed, 1 << lg)))
        torch.cuda.empty_cache()
    return {"workload": "one bg_eval launch: E = 2^10..2^22 at n=8 d=6; n = 4..12 at d = D_s = 8; "
                        "d = D_s = 4..8 at n = 6, 9; F_p (p = 2^31-19) and complex FP64 (real momenta)",
            "unit": "amplitudes/s", **res}


def lanes_workload(args, device):
    """Small batches: one bg_eval launch on the one-point-per-thread kernel
    (BG_LANES=0) against the lane-group kernel with one point per group of
    lanes (BG_LANES=1) and per team of the groups of a warp (BG_LANES=2) for
    E = 2^6 .. 2^15 points: F_p (p = 2^31 - 19) at n = 5, 8, 12 and complex
    FP64 (real momenta at n = 8 and 12, complex momenta at n = 6),
    mostly-minus metric.  Each entry: 3 warm-up calls, then the mean of 20
    CUDA-event-timed calls; F_p results compared bit for bit, complex ones by
    their largest relative difference; `default` names the form bg_eval
    takes without BG_LANES."""
    import torch
    from paper_2502_07060_gb300 import bg
    stream = torch.cuda.current_stream(device)
    rows = []
    for field, n, d, lgmax in (("fp", 5, 4, 15), ("fp", 8, 6, 15), ("fp", 12, 8, 15), ("c64r", 8, 6, 15),
                               ("c64r", 12, 8, 13), ("c64", 6, 4, 15)):
        E = 1 << lgmax
        if field == "fp":
            k, e = G.fp_batch(11, E, n, d, d, P, 0)
            kd = torch.from_numpy(k.view(np.int32)).to(device)
            ed = torch.from_numpy(e.view(np.int32)).to(device)
            fid, p = bg.FIELD_FP, P
        else:
            k, e = G.c64_batch(11, E, n, d, d, 0)
            kd = torch.from_numpy(np.ascontiguousarray(k.real) if field == "c64r" else k).to(device)
            ed = torch.from_numpy(e).to(device)
            fid, p = (bg.FIELD_C64_REAL if field == "c64r" else bg.FIELD_C64), 0
        plans = {}
        for v in ("0", "1", "2", "auto"):
            old = os.environ.get("BG_LANES")
            os.environ["BG_LANES"] = v
            plans[v] = bg.Plan(n, d, d, fid, p, bg.MOSTLY_MINUS)
            if old is None:
                os.environ.pop("BG_LANES")
            else:
                os.environ["BG_LANES"] = old
        desc = dict(x.split("=", 1) for x in plans["auto"].describe().split())
        cut, tcut = int(desc["lanes_max_items"]), int(desc["team_max_items"])
        for lg in range(6, lgmax + 1):
            m = 1 << lg
            row = {"field": field, "n": n, "d": d, "E": m,
                   "default": "team" if m <= tcut else "lanes" if m <= cut else "per_thread"}
            outs = {}
            for v, key in (("0", "per_thread_ms"), ("1", "lanes_ms"), ("2", "team_ms")):
                plan = plans[v]
                out = torch.empty(m, dtype=ed.dtype, device=device)
                st = torch.empty(m, dtype=torch.uint8, device=device)
                ws = plan.workspace(m, device)
                fn = lambda: plan.eval(kd[:m], ed[:m], out=out, status=st, workspace=ws, stream=stream)
                row[key] = time_steps(fn, 20, 3, stream, None, device) / 20
                outs[v] = out
            if field == "fp":
                row["bit_identical"] = bool(torch.equal(outs["0"], outs["1"]) and torch.equal(outs["0"], outs["2"]))
            else:
                row["max_rel_diff"] = float(((outs["0"] - outs["1"]).abs() / outs["0"].abs()).max().item())
                row["team_equals_lanes"] = bool(torch.equal(outs["1"], outs["2"]))
            row["speedup"] = row["per_thread_ms"] / row["lanes_ms"]
            row["team_speedup"] = row["per_thread_ms"] / row["team_ms"]
            rows.append(row)
        del kd, ed
        torch.cuda.empty_cache()
    return {"workload": "small batches, one bg_eval launch: per-thread kernel against the lane-group kernel "
                        "(one point per group, per team)",
            "unit": "ms per call", "rows": rows}


def fourdim_workload(args, device):
    """Trees of a one-loop cut (Sec. 2.3): legs 0 and n-1 d-dimensional, legs
    1..n-2 four-dimensional states zero-padded into d dimensions.  Times the
    ordinary plan against the mixed-dimension plan (bg_plan_create_mixed,
    currents of four-dimensional ranges with four components) on the same
    inputs: n = 6, 8, 10, 12, d = D_s = 6 and 8, F_p (2^20 points) and
    complex FP64 with real momenta (2^17 points)."""
    import torch
    from paper_2502_07060_gb300 import bg
    stream = torch.cuda.current_stream(device)
    rows = []
    for field, lg in (("fp", 20), ("c64", 17)):
        E = 1 << lg
        for d in (6, 8):
            for n in (6, 8, 10, 12):
                mask = ((1 << (n - 1)) - 1) & ~1
                if field == "fp":
                    k, e = G.fp_batch(6000 + 10 * n + d, E, n, d, d, P, 0, four_d=mask)
                    kd = torch.from_numpy(k.view(np.int32)).to(device)
                    ed = torch.from_numpy(e.view(np.int32)).to(device)
                    fld, p = bg.FIELD_FP, P
                else:
                    k, e = G.c64_batch(6000 + 10 * n + d, E, n, d, d, 0, four_d=mask)
                    kd = torch.from_numpy(np.ascontiguousarray(k.real)).to(device)
                    ed = torch.from_numpy(e).to(device)
                    fld, p = bg.FIELD_C64_REAL, 0
                del k, e
                out = torch.empty(E, dtype=ed.dtype, device=device)
                st = torch.empty(E, dtype=torch.uint8, device=device)
                row = {"field": field, "n": n, "d": d, "points": E, "four_dim_legs": mask}
                for mode, m in (("plain", None), ("mixed", mask)):
                    plan = bg.Plan(n, d, d, fld, p, bg.MOSTLY_MINUS, four_dim_legs=m)
                    ws = plan.workspace(E, device)
                    step = lambda: plan.eval(kd, ed, out=out, status=st, workspace=ws, stream=stream)
                    ms = time_steps(step, 10, args.warmup, stream, None, device) / 10
                    row[mode] = {"ms_per_call": ms, "value": E / (ms / 1e3), "plan": plan.describe()}
                    del plan, ws
                row["speedup"] = row["mixed"]["value"] / row["plain"]["value"]
                rows.append(row)
                del kd, ed, out, st
                torch.cuda.empty_cache()
    return {"workload": "cut trees: legs 1..n-2 four-dimensional, n = 6..12, d = D_s in {6, 8}; ordinary "
                        "plan against the mixed-dimension plan on the same inputs",
            "unit": "amplitudes/s", "rows": rows}


def serve_workload(args, device):
    """Poisson arrivals (mean rate per second from --serve-rates) of requests
    with log-uniform sizes 1..65536 points, n uniform in 4..12, d = D_s
    uniform in {4, 6, 8}, field uniform; latency = completion - arrival.
    Arms, each on the same request sequence:
      server           bg_server (continuous admission, 8 stream slots) with
                       page-locked host buffers (used in place or staged);
      server_resident  the same server with the momenta and states resident
                       on the device (a pool uploaded once; results still
                       returned to host memory), first rate only;
      plain_1          plain per-request evaluation by one thread in arrival
                       order (copy in, bg_eval, copy out, synchronise);
      plain_8          the same by 8 threads, each on its own stream, without
                       admission control (a request waits only for a free
                       thread)."""
    import queue
    import threading

    import torch
    from paper_2502_07060_gb300 import bg
    configs = [(f, n, d) for f in ("fp", "c64") for n in range(4, 13) for d in (4, 6, 8)]
    pool_pts = 1 << 16
    pools, plans = {}, {}
    for i, (f, n, d) in enumerate(configs):
        if f == "fp":
            k, e = G.fp_batch(7000 + i, pool_pts, n, d, d, P, 0)
            pools[(f, n, d)] = (torch.from_numpy(k.view(np.int32)).pin_memory(),
                                torch.from_numpy(e.view(np.int32)).pin_memory())
            plans[(f, n, d)] = bg.Plan(n, d, d, bg.FIELD_FP, P)
        else:
            k, e = G.c64_batch(7000 + i, pool_pts, n, d, d, 0)
            pools[(f, n, d)] = (torch.from_numpy(k).pin_memory(), torch.from_numpy(e).pin_memory())
            plans[(f, n, d)] = bg.Plan(n, d, d, bg.FIELD_C64, 0)

    def requests(rate, seed):
        rng = np.random.default_rng(seed)
        n_req = int(rate * args.serve_seconds)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
        reqs, placement = [], []
        for _ in range(n_req):
            cfg = configs[rng.integers(len(configs))]
            E = int(np.clip(np.exp(rng.uniform(0, np.log(65536))), 1, 65536))
            off = int(rng.integers(0, pool_pts - E + 1))
            hk, he = pools[cfg]
            out = torch.empty(E, dtype=hk.dtype).pin_memory()
            st = torch.empty(E, dtype=torch.uint8).pin_memory()
            reqs.append((plans[cfg], hk[off:off + E], he[off:off + E], out, st, E))
            placement.append((cfg, off))
        return arrivals, reqs, placement

    def summarise(lat, t0, t_end, total_pts):
        lat = np.array(lat) * 1e3
        n_req = len(lat)
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
                "throughput_points_per_s": total_pts / (t_end - t0),
                "throughput_requests_per_s": n_req / (t_end - t0)}

    def run_server(arrivals, req_list):
        n_req = len(req_list)
        srv = bg.Server(8 << 30, max_inflight=8)
        done_at = [0.0] * n_req
        tickets = queue.Queue()
        failed = []

        def waiter():
            while True:
                item = tickets.get()
                if item is None:
                    return
                i, t = item
                try:
                    if not srv.wait(t, 120000):      # a generous deadline, never an endless wait
                        failed.append(i)
                except Exception:                   # noqa: BLE001 -- reported in the result
                    failed.append(i)
                done_at[i] = time.perf_counter()

        waiters = [threading.Thread(target=waiter) for _ in range(16)]
        for w in waiters:
            w.start()
        t0 = time.perf_counter()
        for i, r in enumerate(req_list):
            delay = t0 + arrivals[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.put((i, srv.submit(r[0], r[1], r[2], r[3], r[4])))
        for _ in waiters:
            tickets.put(None)
        for w in waiters:
            w.join()
        res = summarise([done_at[i] - (t0 + arrivals[i]) for i in range(n_req)], t0, max(done_at),
                        sum(r[5] for r in req_list))
        res["peak_arena_bytes"] = srv.stats()["peak_bytes"]
        res["failed_requests"] = len(failed)
        srv.close()
        return res

    def run_plain(arrivals, req_list, threads):
        n_req = len(req_list)
        work = queue.Queue()
        done_at = [0.0] * n_req

        def worker():
            stream = torch.cuda.Stream(device)
            while True:
                i = work.get()
                if i is None:
                    return
                plan, hk, he, out, st, E = req_list[i]
                with torch.cuda.stream(stream):
                    dk = hk.to(device, non_blocking=True)
                    de = he.to(device, non_blocking=True)
                    o, s_ = plan.eval(dk, de, stream=stream)
                    out.copy_(o, non_blocking=True)
                    st.copy_(s_, non_blocking=True)
                stream.synchronize()
                done_at[i] = time.perf_counter()

        ws = [threading.Thread(target=worker) for _ in range(threads)]
        for w in ws:
            w.start()
        t0 = time.perf_counter()
        for i in range(n_req):
            delay = t0 + arrivals[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            work.put(i)
        for _ in ws:
            work.put(None)
        for w in ws:
            w.join()
        return summarise([done_at[i] - (t0 + arrivals[i]) for i in range(n_req)], t0, max(done_at),
                         sum(r[5] for r in req_list))

    rates = [float(x) for x in args.serve_rates.split(",")]
    rows = []
    for ri, rate in enumerate(rates):
        arrivals, reqs, placement = requests(rate, args.serve_seed + ri)
        row = {"rate_per_s": rate, "requests": len(reqs), "points": sum(r[5] for r in reqs),
               "server": run_server(arrivals, reqs)}
        if ri == 0:
            dpools = {cfg: (hk.to(device), he.to(device)) for cfg, (hk, he) in pools.items()}
            torch.cuda.synchronize(device)
            resident = [(r[0], dpools[cfg][0][off:off + r[5]], dpools[cfg][1][off:off + r[5]], r[3], r[4], r[5])
                        for r, (cfg, off) in zip(reqs, placement)]
            row["server_resident"] = run_server(arrivals, resident)
            del resident, dpools
            torch.cuda.empty_cache()
            row["plain_1"] = run_plain(arrivals, reqs, 1)
        row["plain_8"] = run_plain(arrivals, reqs, 8)
        rows.append(row)
    return {"workload": f"Poisson arrivals for {args.serve_seconds} s per rate (seed {args.serve_seed}), "
                        "sizes log-uniform 1..65536, n uniform 4..12, d = D_s uniform {4, 6, 8}, F_p or C64",
            "rows": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--log2-points", type=int, default=22)
    ap.add_argument("--log2-points-c64", type=int, default=22)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fields", default="fp,c64,c64c",
                    help="comma list of fp, c64 (real momenta, the physical points), c64c (the same "
                         "points through the complex-momentum plan)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving latency leg")
    ap.add_argument("--workload", choices=["metric", "mixed", "serve", "helicity", "sweep", "fourdim",
                                           "lanes", "launchcheck"],
                    default="metric",
                    help="metric: n=8 d=6 headline line; mixed: uneven-batch comparison; "
                         "serve: p50/p99 latency of the request server; helicity: all 2^n "
                         "helicities with shared sub-currents against one recursion per assignment; "
                         "sweep: time against points, gluons and dimension; fourdim: cut trees with "
                         "four-dimensional legs, ordinary against mixed-dimension plans; lanes: small "
                         "batches on the per-thread and lane-group kernels; launchcheck: "
                         "the multi-rank launch on CPU (gloo), no GPU work")
    ap.add_argument("--log2-points-helicity", type=int, default=20,
                    help="points per n of the helicity workload")
    ap.add_argument("--serve-rates", default="2000,1000",
                    help="comma list of mean request rates per second; the first is the metric's")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-seed", type=int, default=2026,
                    help="seed of the arrival times, sizes, configurations and pool offsets")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # started as a plain process: become N replica ranks (one per GPU)
        sys.exit(launch_ranks(args.gpus))
    rank, world, local = dist_env()
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE={world}")
    if args.workload == "launchcheck":
        launch_check(args, rank, world)
        return
    E = 1 << args.log2_points
    Ec = 1 << args.log2_points_c64
    config = {"workload": f"n={N_LEG} gluons, d=D_s={D}, mostly-minus metric, F_p p=2^31-19 and "
                          f"complex FP64, seeded on-shell points, one transverse state per leg",
              "points_per_step_per_gpu": E, "points_per_step_per_gpu_c64": Ec,
              "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas{world}"}

    if args.impl == "reference":
        # the oracle as it stands, on the host cores: every step evaluates a
        # bounded sample (2^14 points) of the same n=8, d=D_s=6 F_p workload
        if rank != 0:
            return
        from oracle import coracle
        m = 1 << 14
        k, e = G.fp_batch(4242, m, N_LEG, D, DS, P, 0)
        for _ in range(args.warmup):
            coracle.amp_fp(k[:1024], e[:1024], P, 0)
        t_all = 0.0
        for _ in range(args.steps):
            t0 = time.perf_counter()
            coracle.amp_fp(k, e, P, 0)
            t_all += time.perf_counter() - t0
        val = args.steps * m / t_all
        cores = coracle.max_threads()
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "amplitudes/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": config,
                "cpu_baseline": {"value": val, "unit": "amplitudes/s", "cores": cores,
                                 "kind": "oracle",
                                 "sample": f"{m} points per step of the n=8 d=D_s=6 F_p workload (of "
                                           f"{E} per GPU step), C oracle (gcc -O3 -ffp-contract=off, "
                                           f"OpenMP, one point per iteration) on {cores} host threads"},
                "e2e": {"value": val, "unit": "amplitudes/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if args.workload == "mixed":
        if rank == 0:
            print(json.dumps({"metric": METRIC, "mixed": mixed_workload(args, device)}))
        return
    if args.workload == "helicity":
        if rank == 0:
            print(json.dumps({"metric": METRIC, "helicity": helicity_workload(args, device)}))
        return
    if args.workload == "fourdim":
        if rank == 0:
            print(json.dumps({"metric": METRIC, "fourdim": fourdim_workload(args, device)}))
        return
    if args.workload == "sweep":
        if rank == 0:
            print(json.dumps({"metric": METRIC, "sweep": sweep_workload(args, device)}))
        return
    if args.workload == "lanes":
        if rank == 0:
            print(json.dumps({"metric": METRIC, "lanes": lanes_workload(args, device)}))
        return
    if args.workload == "serve":
        if rank == 0:
            print(json.dumps({"metric": METRIC, "serve": serve_workload(args, device)}))
        return
    dist = init_dist(world, "nccl")
    fields = args.fields.split(",")
    e2e = not args.no_e2e
    if fields == ["c64"]:
        c64 = run_field("c64", Ec, args.steps, args.warmup, rank, dist, device, rank_seed(2000, rank), e2e)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "c64_only": True, "value": world * c64["value_per_rank"],
                              "unit": "amplitudes/s", "ms_per_step": c64["ms_per_step"],
                              "plan": c64["plan"], "clocks": c64["clocks"]}))
        return
    fp = run_field("fp", E, args.steps, args.warmup, rank, dist, device, rank_seed(1000, rank), e2e)
    c64_steps = max(3, args.steps // 5)
    c64 = c64c = None
    if "c64" in fields:
        c64 = run_field("c64", Ec, c64_steps, args.warmup, rank, dist, device, rank_seed(2000, rank), e2e)
    if "c64c" in fields:
        c64c = run_field("c64c", Ec, c64_steps, args.warmup, rank, dist, device, rank_seed(2000, rank),
                         False)

    value = job_value(E, world, fp["ms_per_step"])
    tally, _ = literal_tally(N_LEG, D, DS)
    peaks = read_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0) or 2070.0
    n_sm = torch.cuda.get_device_properties(device).multi_processor_count
    # F_p roofline: one 32x32 -> 64-bit product per field multiplication
    # (reductions free), at the rate of the 64-bit multiply-add: 32 per SM per
    # clock, half the 64-lane 32-bit IMAD rate (measured: mul.hi 30/clk/SM,
    # four-product accumulation 27 field multiplications/clk/SM).
    peak_mulmod = n_sm * 32 * sm_max * 1e6
    achieved = fp["value_per_rank"] * tally
    c64_flops = literal_flops(N_LEG, D, DS, True)        # real momenta (the c64 leg)
    c64c_flops = literal_flops(N_LEG, D, DS, False)      # complex momenta
    peak_fp64 = n_sm * 2 * 2 * sm_max * 1e6
    peak_fp64_instr = n_sm * 2 * sm_max * 1e6
    ops_c64 = kernel_fp64_ops(N_LEG, D, DS, True)
    ops_c64c = kernel_fp64_ops(N_LEG, D, DS, False)
    kops = kernel_mults(N_LEG, D, DS)
    traffic_fp = profiled_traffic("fp")
    traffic_c64 = profiled_traffic("c64")
    scale = E / float(1 << 22)
    line = {
        "metric": METRIC, "value": value, "unit": "amplitudes/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": fp["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": config,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_mulmod,
                     "unit": "field multiplications/s (F_p, literal tally)",
                     "frac": achieved / peak_mulmod,
                     "traffic": None if traffic_fp is None else traffic_fp * scale,
                     "ops_per_unit": tally, "kernel_ops_per_unit": kops,
                     "frac_kernel_ops": fp["value_per_rank"] * kops / peak_mulmod,
                     "peak_derivation": f"{n_sm} SMs x 32 64-bit products/clk x {sm_max:.0f} MHz, one product "
                                        f"per field multiplication (derived from the IMAD unit: 64 lanes/clk, 64-bit "
                                        f"results at half rate; measured 27/clk/SM for the kernel's accumulation)",
                     "traffic_source": "bench_traffic.json: ncu DRAM counters of a 2^19-point "
                                       "capture scaled by the point count"},
        "c64": None if c64 is None else {
            "value": world * c64["value_per_rank"], "unit": "amplitudes/s",
            "ms_per_step": c64["ms_per_step"], "points_per_step": Ec, "steps": c64_steps,
            "dtype": "f64",
            "momenta": "real (physical points; BG_FIELD_C64_REAL plan)",
            "roofline": {"bound": "alu", "achieved": c64["value_per_rank"] * c64_flops,
                         "peak": peak_fp64, "unit": "FP64 FLOP/s (literal tally, real momenta)",
                         "frac": c64["value_per_rank"] * c64_flops / peak_fp64,
                         "ops_per_unit": c64_flops,
                         "kernel_fp64_instr_per_unit": ops_c64,
                         "frac_kernel_ops": c64["value_per_rank"] * ops_c64 / peak_fp64_instr,
                         "frac_note": "frac counts the literal recursion's FP64 work (oracle tally); the "
                                      "kernel's regrouped recursion issues fewer FP64 operations than the "
                                      "literal one, so frac can exceed 1; frac_kernel_ops is the FP64 pipe's "
                                      "share of its instruction peak",
                         "traffic": None if traffic_c64 is None else traffic_c64 * Ec / float(1 << 22),
                         "peak_derivation": f"{n_sm} SMs x 2 DFMA/clk x 2 x {sm_max:.0f} MHz "
                                            f"(kernel ops: FP64 instructions at 2/clk/SM)"},
            "e2e_value": (world * Ec / (c64["e2e_ms_per_step"] / 1e3)) if e2e else None,
            "clocks": c64["clocks"], "plan": c64["plan"]},
        "c64_complex_momenta": None if c64c is None else {
            "value": world * c64c["value_per_rank"], "unit": "amplitudes/s",
            "ms_per_step": c64c["ms_per_step"], "points_per_step": Ec, "steps": c64_steps,
            "kernel_fp64_instr_per_unit": ops_c64c,
            "literal_flops_per_unit": c64c_flops,
            "frac": c64c["value_per_rank"] * c64c_flops / peak_fp64,
            "frac_kernel_ops": c64c["value_per_rank"] * ops_c64c / peak_fp64_instr,
            "clocks": c64c["clocks"], "plan": c64c["plan"]},
        "e2e": None if not e2e else {
            "value": world * E / (fp["e2e_ms_per_step"] / 1e3), "unit": "amplitudes/s",
            "h2d_bytes_per_step": fp["h2d_bytes"], "d2h_bytes_per_step": fp["d2h_bytes"]},
        "clocks": fp["clocks"],
        "gpu_launches": args.steps,
        "plan": fp["plan"],
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline("fp")
    if rank == 0 and world == 1 and not args.no_serve:
        # the metric's serving half (one GPU): p50/p99 latency of the request
        # server against plain per-request launches (the serve workload)
        try:
            sv = serve_workload(args, device)
            r0 = sv["rows"][0]
            line["serving"] = {
                "workload": sv["workload"], "unit": "ms", "rate_per_s": r0["rate_per_s"],
                "p50_ms": r0["server"]["p50_ms"], "p99_ms": r0["server"]["p99_ms"],
                "throughput_points_per_s": r0["server"]["throughput_points_per_s"],
                "failed_requests": sum(r["server"]["failed_requests"] for r in sv["rows"])
                + r0["server_resident"]["failed_requests"],
                "resident_inputs_p50_ms": r0["server_resident"]["p50_ms"],
                "resident_inputs_p99_ms": r0["server_resident"]["p99_ms"],
                "plain_per_request_p50_ms": r0["plain_1"]["p50_ms"],
                "plain_per_request_p99_ms": r0["plain_1"]["p99_ms"],
                "plain_per_request_throughput_points_per_s": r0["plain_1"]["throughput_points_per_s"],
                "plain_8_streams_p50_ms": r0["plain_8"]["p50_ms"],
                "plain_8_streams_p99_ms": r0["plain_8"]["p99_ms"],
                "other_rates": [{"rate_per_s": r["rate_per_s"], "server_p50_ms": r["server"]["p50_ms"],
                                 "server_p99_ms": r["server"]["p99_ms"],
                                 "plain_8_streams_p50_ms": r["plain_8"]["p50_ms"],
                                 "plain_8_streams_p99_ms": r["plain_8"]["p99_ms"]} for r in sv["rows"][1:]]}
        except Exception as exc:                    # noqa: BLE001 -- keep the throughput line
            line["serving"] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
