"""The multi-GPU path of the benchmark is independent replicas (the method
needs no data exchange at one GPU per lattice): check its whole-job
aggregation with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r ran (r + 1) * 1e9 updates in (r + 1) * 0.5 s
    secs, glups = bench.aggregate_replicas(torch, (rank + 1) * 0.5, (rank + 1) * 1e9, world)
    out[rank] = (secs, glups)
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        secs, glups = out[r]
        assert secs == 1.0                      # max over ranks
        assert abs(glups - 3.0) < 1e-12         # (1e9 + 2e9) updates / 1.0 s


def test_single_process_aggregation():
    import bench
    secs, glups = bench.aggregate_replicas(torch, 2.0, 4e9, 1)
    assert secs == 2.0 and glups == 2.0
