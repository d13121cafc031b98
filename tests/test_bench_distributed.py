"""bench.py's multi-rank path on CPU (gloo, world size 2): replicas only --
each rank runs the whole workload, the job time is the slowest rank's and the
throughput counts all ranks' steps."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = [2.0, 5.0][rank]
    t, value = bench.aggregate(elapsed, steps=4, world=world, dist=dist, device="cpu")
    out[rank] = (t, value)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, value = res[rank]
        assert t == pytest.approx(5.0)
        assert value == pytest.approx(world * 4 / 5.0)


def test_aggregate_single_rank():
    import bench
    t, value = bench.aggregate(2.5, steps=5, world=1)
    assert (t, value) == (2.5, 2.0)
