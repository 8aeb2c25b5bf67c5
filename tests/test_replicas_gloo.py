"""The N > 1 benchmark path runs independent replicas (one graph's test does
not shard): the only cross-rank step is the max over ranks of the timed
total.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    total_ms, value = bench.aggregate_over_ranks(100.0 * (rank + 1), tests_per_rank=10)
    out[rank] = (total_ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_max_over_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        total_ms, value = res[rank]
        assert total_ms == 200.0                       # the slowest rank
        assert abs(value - 2 * 10 / 0.2) < 1e-9        # all ranks' tests over the slowest time


def test_single_process_is_identity():
    import bench
    total_ms, value = bench.aggregate_over_ranks(50.0, tests_per_rank=4)
    assert total_ms == 50.0 and abs(value - 80.0) < 1e-9
