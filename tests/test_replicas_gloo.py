"""The replica path of bench.py across ranks (world size 2, gloo on CPU):
the job's elapsed time is the slowest rank's and its units are the sum over
ranks, so that `value` is the whole-job throughput."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, inputs, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed, units = inputs[rank]
    out[rank] = bench.over_ranks(dist, "cpu", elapsed, units)
    dist.barrier()
    dist.destroy_process_group()


def test_over_ranks_takes_max_time_and_sums_units():
    world = 2
    inputs = [(100.0, 4), (150.0, 6)]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, _free_port(), inputs, out), nprocs=world,
                           join=True, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1] == (150.0, 10.0)


def test_over_ranks_single_process_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.over_ranks(None, "cpu", 12.5, 3) == (12.5, 3.0)
