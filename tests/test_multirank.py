"""The benchmark's replica mode on CPU: world_size 2 over gloo.  Each rank reports its own time; the
job's time is the slowest rank's and the whole-job throughput counts every rank's ops."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    my_ms = 10.0 + 5.0 * rank                      # rank 1 is the slower replica
    t = bench.max_over_ranks(my_ms, world)
    v = bench.whole_job_mops(1_000_000, world, t)
    dist.barrier()
    out[rank] = (t, v)
    dist.destroy_process_group()


def test_replicas_take_max_over_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    t, v = res[0]
    assert t == 15.0
    assert v == pytest.approx(2 * 1_000_000 / 15e-3 / 1e6)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_mops(35_913_728, 1, 10.0) == pytest.approx(3591.3728)
