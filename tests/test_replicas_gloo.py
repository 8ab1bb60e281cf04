"""The multi-process path of bench.py on CPU: N independent replicas whose timings are reduced by
a max over ranks (world size 2, gloo, 127.0.0.1)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        dist.barrier()
        qps, total = bench.replica_throughput(100.0 + 50.0 * rank, units_per_step=10_000, steps=20)
        out[rank] = (qps, total)
    finally:
        dist.destroy_process_group()


def test_replica_throughput_two_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # both ranks see the slowest rank's time; the job processed 2 x 20 x 10k queries in it
    for rank in range(world):
        qps, total = res[rank]
        assert total == pytest.approx(150.0)
        assert qps == pytest.approx(2 * 20 * 10_000 / 0.150)


def test_replica_throughput_single_process():
    import bench
    qps, total = bench.replica_throughput(200.0, units_per_step=5, steps=4)
    assert total == 200.0 and qps == pytest.approx(5 * 4 / 0.2)
