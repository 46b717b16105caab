"""Host logic of bench.py that needs no GPU: the reference arm (the oracle
timed on the host cores) prints the contract's JSON line, and the algorithmic
work per amplitude behind the rooflines (field multiplications over F_p, FP64
operations over complex FP64) is the oracle's counted tally."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    import bench
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "amplitudes/s" and line["higher_is_better"] is True and line["value"] > 0
    assert line["n_gpus"] == 1 and line["steps"] == 1 and line["data"] == "synthetic"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert "workload" in line["config"]


@pytest.mark.parametrize("n,d,Ds", [(4, 4, 4), (5, 4, 4), (8, 6, 6), (8, 4, 8), (10, 6, 6), (12, 8, 8)])
def test_literal_tally_is_the_oracle_count(n, d, Ds):
    import bench
    from oracle.bg_oracle import op_tally
    assert bench.literal_tally(n, d, Ds)[0] == op_tally(n, d, Ds).mul


@pytest.mark.parametrize("n,d,Ds", [(4, 4, 4), (5, 4, 4), (8, 6, 6), (8, 4, 8), (10, 6, 6), (12, 8, 8)])
@pytest.mark.parametrize("real_k", [True, False])
def test_literal_flops_are_the_oracle_count(n, d, Ds, real_k):
    import bench
    from oracle.bg_oracle import flop_tally
    assert bench.literal_flops(n, d, Ds, real_k) == flop_tally(n, d, Ds, real_momenta=real_k)
