"""The multi-GPU path is replicas only: each rank runs its own step; the job reports the summed
iterations over the slowest rank's time.  Checked with two gloo ranks on the CPU."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench._dist()
    ms, it = bench.aggregate(100.0 + 50.0 * rank, 1000.0 + rank, torch.device("cpu"))
    out[rank] = (ws, r, local, ms, it)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    for rank in (0, 1):
        ws, r, local, ms, it = out[rank]
        assert (ws, r, local) == (2, rank, rank)
        assert ms == 150.0 and it == 2001.0


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.aggregate(12.5, 7.0, torch.device("cpu")) == (12.5, 7.0)
