"""Frames of a sequence across ranks, one process per GPU.

The frames of a sequence are independent: each is reconstructed from its own
images against the same rig and background (Section 2.2.2 runs per frame).
So N ranks split a sequence without any exchange on the data path: rank r
takes frames r, r + N, r + 2N, ... (round-robin, so every rank sees the whole
time span and the per-rank counts differ by at most one) with its own handle,
a replica of the same grid, rig and background.  The only collective is the
optional gathering of the results back into frame order: one all-gather of
the per-frame counts and one of the voxel lists padded to the longest list.
"""

from __future__ import annotations

from typing import List, Sequence, Tuple


def rank_frames(n_frames: int, rank: int, world: int) -> List[int]:
    """Global indices of the frames rank `rank` of `world` reconstructs."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    return list(range(rank, max(n_frames, 0), world))


def frames_per_rank(n_frames: int, world: int) -> List[int]:
    return [len(rank_frames(n_frames, r, world)) for r in range(world)]


def gather_frames(counts, lists, n_frames: int, rank: int, world: int, group=None) -> Tuple[list, list]:
    """Gathers every rank's per-frame results into global frame order.

    counts: integer tensor [n_local] of this rank's frames (true counts: a
    count above the list width means the list holds only its first entries);
    lists: integer tensor [n_local][capacity] of voxel lists.  Tensors live on
    the device the process group's backend uses (CUDA for NCCL, CPU for gloo).
    Returns (counts, lists) on every rank: `n_frames` Python ints and
    `n_frames` 1-D tensors of min(count, capacity) voxel indices each."""
    import torch
    import torch.distributed as dist

    mine = rank_frames(n_frames, rank, world)
    if counts.numel() != len(mine) or lists.shape[0] != len(mine):
        raise ValueError(f"rank {rank} holds {counts.numel()} frames, expected {len(mine)}")
    cap = int(lists.shape[1]) if lists.dim() == 2 else 0
    n_max = max(frames_per_rank(n_frames, world))
    dev = counts.device
    c_pad = torch.full((n_max,), -1, dtype=torch.int64, device=dev)
    c_pad[:len(mine)] = counts.to(torch.int64) & 0xFFFFFFFF
    c_all = [torch.empty_like(c_pad) for _ in range(world)]
    dist.all_gather(c_all, c_pad, group=group)
    lengths = [[min(int(c), cap) for c in t.tolist() if c >= 0] for t in c_all]
    width = max([max(l) if l else 0 for l in lengths] + [1])
    l_pad = torch.zeros((n_max, width), dtype=lists.dtype, device=dev)
    if len(mine):
        w = min(width, cap)
        l_pad[:len(mine), :w] = lists[:, :w]
    l_all = [torch.empty_like(l_pad) for _ in range(world)]
    dist.all_gather(l_all, l_pad, group=group)
    out_counts: List[int] = [0] * n_frames
    out_lists: list = [None] * n_frames
    for r in range(world):
        for i, g in enumerate(rank_frames(n_frames, r, world)):
            out_counts[g] = int(c_all[r][i])
            out_lists[g] = l_all[r][i, :lengths[r][i]].clone()
    return out_counts, out_lists


def check_partition(n_frames: int, world: int) -> bool:
    """Every frame on exactly one rank."""
    seen: Sequence[int] = sorted(g for r in range(world) for g in rank_frames(n_frames, r, world))
    return list(seen) == list(range(n_frames))
