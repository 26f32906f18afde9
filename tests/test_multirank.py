"""The N > 1 launch of bench.py on CPU ranks (gloo, world size 2): the whole-job throughput is
the units of all ranks over the slowest rank's time, and the reductions the timing uses agree
on every rank.  The GPU path runs the same helpers over NCCL (one replica per GPU, no
collective in the data path)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units = 1000.0 * (rank + 1)          # rank r processed (r + 1) * 1000 particle-steps
    ms = 10.0 * (rank + 1)               # in (r + 1) * 10 ms
    bench.barrier(world)
    out[rank] = (bench.max_over_ranks(ms, world), bench.sum_over_ranks(units, world),
                 bench.job_rate(units, ms, world))
    dist.destroy_process_group()


def test_job_rate_over_two_gloo_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(rank_main, args=(world, free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in range(world):
        mx, sm, rate = res[r]
        assert mx == 20.0
        assert sm == 3000.0
        assert rate == pytest.approx(3000.0 / 0.020, rel=1e-12)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(5.0, 1) == 5.0
    assert bench.sum_over_ranks(7.0, 1) == 7.0
    assert bench.job_rate(100.0, 50.0, 1) == pytest.approx(2000.0)
