"""Host logic of the multi-rank benchmark path, on CPU with two gloo ranks.

Each rank advances its own lattice (independent chains, no data-path
collective); the job's time is the slowest rank's and its value is all
ranks' site-updates over that time.  Under torchrun the reference arm runs
on rank 0 only.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [12.5, 20.0][rank]
    ms_max = bench.rank_max(local_ms)
    value = bench.job_value(1000, ms_max, world)
    ws, r, lr = bench.dist_setup()
    ref = bench.reference(type("A", (), {"steps": 1, "warmup": 0})()) if rank == 1 else "skipped"
    out[rank] = (ms_max, value, ws, r, lr, ref)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    for rank in (0, 1):
        ms_max, value, ws, r, lr, _ = out[rank]
        assert ms_max == 20.0 and ws == 2 and r == rank and lr == rank
        assert value == pytest.approx(2 * 1000 / 0.020)
    assert out[1][5] is None  # the reference arm does no work on rank 1


def test_single_process_defaults():
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert bench.dist_setup() == (1, 0, 0)
    assert bench.rank_max(3.5) == 3.5
    assert bench.job_value(100, 10.0, 1) == pytest.approx(10000.0)
