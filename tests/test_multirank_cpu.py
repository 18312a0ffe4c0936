"""The multi-rank (torchrun) path of bench.py, on CPU with the gloo backend and
world_size 2: every rank runs its own replica (independent sub-regions, weak
scaling) and the job value is the units of all ranks over the slowest rank's
time.  No GPU is involved."""
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
    import bench
    ms_local = [10.0, 40.0][rank]          # rank 1 is the slowest
    units_local = [3.0, 5.0][rank]         # Mpix each rank processed per step
    ms, value = bench.aggregate(ms_local, units_local, steps=4, world=world, dist_mod=dist, device="cpu")
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_bench_aggregate_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == 40.0
        assert value == pytest.approx((3.0 + 5.0) * 4 / 0.040)


def test_bench_aggregate_single_rank():
    import bench
    ms, value = bench.aggregate(20.0, 2.0, steps=10, world=1)
    assert ms == 20.0 and value == pytest.approx(2.0 * 10 / 0.020)
