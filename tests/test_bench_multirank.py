"""Host-side logic of bench.py, on CPU: the multi-rank path and the clock summary.

Multi-GPU runs are independent replicas (weak scaling): the only exchange is
the maximum of the per-rank step times.  These tests run that exchange with
two gloo ranks, and the reference arm under torchrun with two ranks (rank 0
alone prints its line; the other exits 0)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(1.5 + rank, torch.device("cpu"), world)
        value = bench.job_throughput(1000, world, ms)
        with open(f"{out_path}.{rank}", "w") as f:
            json.dump({"ms": ms, "value": value}, f)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    out = str(tmp_path / "r")
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world,
                       start_method="spawn")
    for r in range(world):
        with open(f"{out}.{r}") as f:
            d = json.load(f)
        assert d["ms"] == 2.5                      # the slowest rank's time, on every rank
        assert d["value"] == pytest.approx(2 * 1000 / 2.5e-3)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.25, None, 1) == 3.25
    assert bench.job_throughput(100, 1, 2.0) == pytest.approx(100 / 2e-3)


def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--workload", "cartpole", "--K", "256", "--steps", "2", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_clock_summary_keeps_the_timed_region():
    import time
    import bench
    t0 = time.mktime(time.strptime("2026/12/03 18:40:01", "%Y/%m/%d %H:%M:%S"))
    lines = [
        "2026/12/03 18:40:00.500, 0, 1200, 2070, 300.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2026/12/03 18:40:01.010, 0, 2070, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active",
        "2026/12/03 18:40:01.030, 0, 2055, 2070, 910.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2026/12/03 18:40:02.000, 0, 1400, 2070, 300.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
    ]
    d = bench.ClockSampler.summarise(lines, (t0, t0 + 0.05))
    assert d["samples"] == 2 and d["in_timed_region"]
    assert d["sm_mhz"] == (2070 + 2055) / 2 and d["sm_max_mhz"] == 2070
    assert d["reasons"] == ["sw_power_cap"]
    # nothing inside: every sample, flagged
    d = bench.ClockSampler.summarise(lines, (t0 + 100, t0 + 101))
    assert d["samples"] == 4 and not d["in_timed_region"]
