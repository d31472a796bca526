"""Multi-GPU runs are replicas: each rank labels its own seeded instance and
the job's time is the maximum over ranks. The rank-level host logic of
bench.py, exercised with two gloo ranks on the CPU."""
import os
import socket

import numpy as np
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


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import lattices as L
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spec = bench.replica_spec("hc256", rank)
        spec["L"] = 16                                      # a small instance of the same family
        lat = L.make_instance(spec)
        labels = oracle.uf_label(lat)
        mine = float(1 + rank)                              # stand-in per-rank step time
        job = bench.max_over_ranks(mine, dist)
        out[rank] = (spec["seed"], job, int(labels.sum()), lat.n)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    seeds = {out[r][0] for r in range(world)}
    assert len(seeds) == world                      # independent instances
    assert all(out[r][1] == float(world) for r in range(world))   # max over ranks
    assert out[0][3] == out[1][3]                   # same shape
    assert out[0][2] != out[1][2]                   # different realisations
