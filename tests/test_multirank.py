"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): each rank
streams its own frames (replicas, weak scaling) and the reported time is the
maximum over ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    frames = bench.rank_frames(rank)
    t = bench.max_over_ranks(10.0 + rank, world, torch.device("cpu"))
    results[rank] = (frames, t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    results = mgr.dict()
    mp.spawn(_worker, args=(world, port, results), nprocs=world, join=True)
    (f0, t0), (f1, t1) = results[0], results[1]
    assert t0 == t1 == 11.0
    assert not set(f0) & set(f1)          # disjoint frames: weak scaling, no shared work
