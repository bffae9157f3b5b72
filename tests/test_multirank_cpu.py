"""The multi-GPU logic, run as two gloo ranks on the CPU.

Frames are independent, so N ranks split a sequence round-robin (rank r:
frames r, r + N, ...) with a replica of the handle each and no collective on
the data path; the timed region is the max over ranks, the throughput the
units of all ranks over that time, and the per-frame counts and lists are
gathered back into frame order afterwards.  The per-rank worker here is the
FP64 oracle on tiny frames (no GPU), so the gathered result can be checked
against one process reconstructing every frame."""

import io
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import oracle
from paper_1311_6811_gb300 import replicas
from synth import scene as S


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))


def _worker(rank, world, port, out):
    _env(rank, world, port)
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


def test_round_robin_partition():
    for n in (0, 1, 5, 8, 100, 101):
        for world in (1, 2, 3, 8):
            assert replicas.check_partition(n, world)
            per = replicas.frames_per_rank(n, world)
            assert sum(per) == n and max(per) - min(per) <= 1
    assert replicas.rank_frames(7, 1, 3) == [1, 4]
    with pytest.raises(ValueError):
        replicas.rank_frames(7, 3, 3)


N_SEQ = 5     # frames of the tiny sequence (odd: the ranks hold 3 and 2 frames)
CAP = 140     # list width: smaller than some frames' counts, so truncation is exercised


def _tiny_sequence(frame_ids=None):
    return S.make_scene(seed=9, grid_n=12, cube_side=2.0, n_cams=2, width=48, height=36, focal=45.0,
                        n_frames=N_SEQ, walking=True, frame_ids=frame_ids)


def _oracle_frames(sc):
    counts, lists = [], []
    for f in range(sc.images.shape[0]):
        r = oracle.reconstruct(sc.grid, sc.cams, sc.images[f], sc.mean, sc.var, sc.params)
        counts.append(int(r["list"].size))
        lists.append(r["list"].astype(np.int64))
    return counts, lists


def _gather_worker(rank, world, port, out):
    _env(rank, world, port)
    bench.dist_init("gloo")
    mine = replicas.rank_frames(N_SEQ, rank, world)
    sc = _tiny_sequence(mine)            # this rank renders only its own frames
    counts, lists = _oracle_frames(sc)
    c = torch.tensor(counts, dtype=torch.int32)
    lst = torch.zeros((len(mine), CAP), dtype=torch.int32)
    for i, l in enumerate(lists):
        n = min(len(l), CAP)
        lst[i, :n] = torch.from_numpy(l[:n].astype(np.int32))
    g_counts, g_lists = replicas.gather_frames(c, lst, N_SEQ, rank, world)
    out[rank] = (mine, g_counts, [l.tolist() for l in g_lists])
    dist.destroy_process_group()


def test_sequence_split_across_two_ranks_gathers_the_single_rank_result():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_gather_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert sorted(out[0][0] + out[1][0]) == list(range(N_SEQ))
    counts, lists = _oracle_frames(_tiny_sequence())
    assert max(counts) > CAP > min(counts)   # some lists truncated, some not
    for rank in range(world):
        _, g_counts, g_lists = out[rank]
        assert g_counts == counts            # true counts, in frame order, on every rank
        for f in range(N_SEQ):
            assert g_lists[f] == lists[f][:CAP].tolist()


def _ref_worker(rank, world, port, out):
    _env(rank, world, port)
    calls = []

    def maker(n):
        calls.append(n)
        return _tiny_sequence(list(range(min(n, N_SEQ))))

    buf = io.StringIO()
    old = sys.stdout
    sys.stdout = buf
    try:
        rc = bench.run_reference(bench.parse_args(["--impl", "reference", "--steps", "1", "--warmup", "1",
                                                   "--frames", "2"]), scene_maker=maker, cores=2)
    finally:
        sys.stdout = old
    out[rank] = (rc, len(calls), buf.getvalue())


def test_reference_arm_runs_on_rank0_only():
    """Under torchrun the reference arm runs on rank 0 (one JSON line with a
    positive value); the other ranks exit 0 without building a scene."""
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_ref_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    rc0, calls0, text0 = out[0]
    rc1, calls1, text1 = out[1]
    assert rc0 == 0 and rc1 == 0
    assert calls0 == 1 and calls1 == 0 and text1 == ""
    line = json.loads(text0.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == world
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
