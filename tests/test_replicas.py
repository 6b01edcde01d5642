"""Multi-GPU path of bench.py ("replicas only": the method is not sharded):
each rank runs its own copy of the workload, the job time is the maximum over
ranks and the work the sum.  Checked with world size 2 on the gloo backend
(CPU processes, no GPU)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, upd = bench.reduce_ranks(10.0 + rank, 100.0 * (rank + 1), dist, "cpu")
    out[rank] = (ms, upd)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_reduction_world_size_2():
    import torch.multiprocessing as mp
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    assert out[0] == out[1] == (11.0, 300.0)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_ranks(3.5, 7.0, None, "cpu") == (3.5, 7.0)
