"""The multi-rank (N > 1) host logic of bench.py, on CPU with two gloo ranks.

Cells and instances are independent in the collision steps, so `bench.py --gpus N`
runs one independent replica per rank (its own seed, weak scaling) with no
data-path collective; the only cross-rank operations are the barrier around the
timed region and the reduction of the timing: the slowest rank's time and the
units of all ranks.  The reference arm runs on rank 0 alone.
"""
import io
import os
import socket
import contextlib

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # the slowest rank's time, the units of every rank
        t, u = bench.reduce_over_ranks(elapsed=1.0 + rank, units=100.0 * (rank + 1), world=world)
        # each rank draws its own replica (seed = rank): same shape, different particles
        wl, _ = bench.make_workload("relax_64x1000", seed=rank)
        # the reference arm does nothing on ranks other than 0
        buf = io.StringIO()
        if rank != 0:
            with contextlib.redirect_stdout(buf):
                bench.run_reference(type("A", (), {"workload": "relax_64x1000", "steps": 1, "warmup": 3})(),
                                    rank, world)
        out[rank] = (t, u, float(wl["vx"][:8].sum()), wl["vx"].size, buf.getvalue())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_reduction():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, u, _, n, printed = res[r]
        assert t == pytest.approx(2.0)                 # max over ranks
        assert u == pytest.approx(300.0)               # sum over ranks
        assert n == 64 * 1000
    assert res[0][2] != res[1][2]                      # independent replicas
    assert res[1][4] == ""                             # rank 1 printed no reference line


def test_single_rank_reduction_is_identity():
    import bench
    assert bench.reduce_over_ranks(3.5, 42, world=1) == (3.5, 42.0)
