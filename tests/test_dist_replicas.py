"""The multi-GPU benchmark path runs independent replicas (the solver holds
one grid per GPU; nothing crosses GPUs). Its only collective is the max of
the per-rank times; checked here with two gloo ranks on CPU."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(100.0 + 50.0 * rank, world)
    out[rank] = (ms, bench.replica_throughput(1_000_000, 10, world, ms))
    dist.destroy_process_group()


def test_two_rank_replica_timing():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 150.0
    # 2 replicas x 1M cells x 10 steps in 0.15 s
    assert res[0][1] == pytest.approx(2 * 1e6 * 10 / 0.15 / 1e6)
