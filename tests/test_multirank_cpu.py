"""The N > 1 path of bench.py on CPU: two gloo ranks, each timing its own
replica of the workload (weak scaling, no collective on the data path).
The slowest rank's time sets the whole-job throughput, every rank sees the
same maximum, and the reference arm prints from rank 0 only."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_s = 1.5 + rank  # rank r "took" 1.5 + r seconds
        s_max = bench.max_over_ranks(local_s, dist)
        cells, steps = 1000, 10
        value = bench.whole_job_mlups(cells, steps, world, s_max)
        # the reference arm: rank 0 alone runs and prints, the others return without work
        buf = io.StringIO()
        if rank != 0:
            with redirect_stdout(buf):
                bench.run_reference(argparse_ns(world), rank)
        out[rank] = (s_max, value, buf.getvalue())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def argparse_ns(world):
    import argparse
    return argparse.Namespace(gpus=world, steps=1, warmup=1)


def test_two_gloo_ranks_max_time_and_whole_job_value():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank in range(world):
        s_max, value, printed = res[rank]
        assert s_max == 2.5  # the slowest rank's time, on every rank
        assert value == pytest.approx(world * 1000 * 10 / 2.5 / 1e6)
        if rank != 0:
            assert printed == ""


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.25) == 0.25
    assert bench.whole_job_mlups(4096, 100, 1, 0.5) == pytest.approx(4096 * 100 / 0.5 / 1e6)
    line = json.dumps({"value": bench.whole_job_mlups(1, 1, 1, 1.0)})
    assert json.loads(line)["value"] == 1e-6
