"""Multi-rank (replicas) host logic of bench.py on CPU with the gloo backend,
world size 2: each rank evaluates an independent seeded batch, the step time
is the maximum over ranks, and the whole-job value counts every rank's
points.  Per-point results do not depend on which rank computed them."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import coracle as C
    from paper_2502_07060_gb300 import inputs as G
    E = 64
    k, e = G.fp_batch(bench.rank_seed(1000, rank), E, 6, 6, 6, G.P_DEFAULT, 0, workers=1)
    out, _ = C.amp_fp(k, e, G.P_DEFAULT, 0)          # CPU stand-in for the device kernel
    ms = 10.0 + 5.0 * rank                             # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, dist, torch.device("cpu"))
    value = bench.job_value(E, world, ms_max)
    gathered = [torch.zeros(E, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(gathered, torch.from_numpy(out.astype(np.int64)))
    if rank == 0:
        np.save(os.path.join(outdir, "res.npy"), np.stack([g.numpy() for g in gathered]))
        with open(os.path.join(outdir, "val.txt"), "w") as f:
            f.write(f"{ms_max} {value}")
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_gloo(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    ms_max, value = map(float, open(tmp_path / "val.txt").read().split())
    assert ms_max == 15.0
    assert value == pytest.approx(2 * 64 / 0.015)
    res = np.load(tmp_path / "res.npy")
    assert not np.array_equal(res[0], res[1])        # independent batches
    from oracle import coracle as C
    from paper_2502_07060_gb300 import inputs as G
    import bench
    for r in range(world):
        k, e = G.fp_batch(bench.rank_seed(1000, r), 64, 6, 6, 6, G.P_DEFAULT, 0, workers=1)
        ref, _ = C.amp_fp(k, e, G.P_DEFAULT, 0)
        assert np.array_equal(res[r], ref.astype(np.int64))


def test_bench_launches_two_ranks_itself():
    """`bench.py --gpus 2` started as a plain process re-runs itself as two
    ranks under torch.distributed.run (the launch the scaling run uses); the
    launch check (gloo, no GPU work) reports n_gpus = 2, each rank's own
    seeded batch and the whole-job value over the slowest rank's time."""
    import json
    import subprocess
    import sys
    import hashlib
    import bench
    from paper_2502_07060_gb300 import inputs as G
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--workload",
                        "launchcheck", "--log2-points", "8"], capture_output=True, text=True, timeout=600,
                       cwd=root, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1                            # rank 0 alone prints
    line = json.loads(lines[0])
    assert line["n_gpus"] == 2 and line["scaling"] == "weak"
    assert line["value"] == pytest.approx(bench.job_value(256, 2, line["ms_per_step"]))
    ranks = sorted(line["ranks"], key=lambda x: x["rank"])
    assert [x["rank"] for x in ranks] == [0, 1]
    for x in ranks:
        assert x["seed"] == bench.rank_seed(1000, x["rank"]) and x["points"] == 256
        k, e = G.fp_batch(x["seed"], 256, bench.N_LEG, bench.D, bench.DS, bench.P, 0, workers=1)
        assert x["digest"] == hashlib.sha256(k.tobytes() + e.tobytes()).hexdigest()[:16]
    assert ranks[0]["digest"] != ranks[1]["digest"]
