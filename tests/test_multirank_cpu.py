"""The multi-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Each rank of `python -m torch.distributed.run --nproc-per-node N bench.py`
runs a full replica of the workload on its own GPU; the job's step time is the
slowest rank's and its throughput counts the samples of every rank.  Here the
same reduction runs over gloo with rank-dependent step times."""

import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from conftest import ROOT

sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    ms = bench.max_over_ranks(10.0 + 2.5 * rank, dist)
    out[rank] = (ms, bench.job_throughput(world, 1000, ms))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_step_time_is_the_slowest_rank(world):
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    slowest = 10.0 + 2.5 * (world - 1)
    for r in range(world):
        ms, value = out[r]
        assert ms == slowest
        assert value == pytest.approx(world * 1000 / (slowest * 1e-3))


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(4.0) == 4.0
    assert bench.job_throughput(1, 500, 2.0) == pytest.approx(250000.0)


def test_reference_arm_prints_its_line():
    """`bench.py --impl reference` (the oracle timed on the host cores) runs
    without a GPU and prints one JSON line with the contract's keys."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--samples-log2", "12"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "ms_per_step", "higher_is_better", "config",
                "cpu_baseline", "e2e"):
        assert key in line
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
