"""The multi-process (replica) path of bench.py on CPU with gloo, world size 2:
the step time is the slowest rank's and the rate counts every replica."""
import os

import pytest
import torch.multiprocessing as mp


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 * (rank + 1), world)
    out[rank] = (ms, bench.whole_job_rate(1000.0, world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_rate_gloo_world2():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1]
    ms, rate = out[0]
    assert ms == 20.0                      # the slower replica
    assert rate == pytest.approx(2 * 1000.0 / 0.020)


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(7.5, 1) == 7.5
    assert bench.whole_job_rate(100.0, 1, 10.0) == pytest.approx(10000.0)
