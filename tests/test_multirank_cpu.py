"""The multi-GPU logic of bench.py, run as two gloo ranks on the CPU: frames
are independent, so every rank runs its own copy of the workload (replicas,
no collective on the data path); the timed region is the max over ranks and
the throughput is the units of all ranks over that time."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    ws, r = bench.dist_init("gloo")
    assert (ws, r) == (world, rank)
    t_local = 1.0 + rank          # rank 1 is the slow one
    units_local = 100.0 * (rank + 1)
    t = bench.max_over_ranks(t_local)
    u = bench.sum_over_ranks(units_local)
    bench.barrier()
    out[rank] = (t, u)
    dist.destroy_process_group()


def test_max_and_sum_over_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        t, u = out[rank]
        assert t == 2.0            # max over ranks
        assert u == 300.0          # units of all ranks
    # whole-job throughput = all units / slowest rank's time
    assert out[0][1] / out[0][0] == 150.0


def _ref_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    out[rank] = bench.run_reference(bench.parse_args(["--impl", "reference", "--steps", "1", "--warmup", "0",
                                                      "--frames", "1"])) if rank == 1 else 0


def test_reference_arm_runs_on_rank0_only():
    """Under torchrun the reference arm runs on rank 0; other ranks exit 0 at once."""
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_ref_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[1] == 0
