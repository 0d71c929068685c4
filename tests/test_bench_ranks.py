"""Multi-rank logic of bench.py on CPU (gloo, world size 2).

The dense path runs one independent replica per GPU (columns of Z are
independent given Delta, Section 3), so the only cross-rank steps are the
barriers around the timed region and the max over ranks of the measured time;
the reference arm runs on rank 0 alone.
"""

import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, values, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        dist.barrier()
        out[rank] = bench.max_over_ranks(values[rank], world, "cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        values = [3.25, 7.5]
        mp.start_processes(_worker, args=(2, port, values, out), nprocs=2, join=True,
                           start_method="spawn")
        assert dict(out) == {0: 7.5, 1: 7.5}


def test_max_over_ranks_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(4.0, 1, "cpu") == 4.0


def test_reference_arm_runs_on_rank0_only():
    """Rank 1 of a torchrun launch of the reference arm exits without work or output."""
    import bench

    class A:
        n, warmup, steps, cpu_sample_cols, gpus = 8, 0, 1, 0, 2

    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A(), rank=1)
    assert buf.getvalue() == ""


@pytest.mark.parametrize("n", [64])
def test_reference_arm_line_small(n):
    """Rank 0 prints one JSON line with the contract's keys (tiny dense case)."""
    import json

    import bench

    class A:
        warmup, steps, cpu_sample_cols, gpus = 0, 1, 4, 1

    A.n = n
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(A(), rank=0)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "ms" and line["value"] > 0
    for key in ["cpu_baseline", "e2e", "config", "metric", "higher_is_better"]:
        assert key in line
    assert line["cpu_baseline"]["kind"] == "oracle"
