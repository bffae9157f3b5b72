"""Shared pieces of the GPU parity tests: run the CUDA path through the C ABI
and compare it with the FP64 oracle on the same seeded inputs.

Tolerances (FP32 path):
  * occupancy within 1e-5 absolute of the oracle, for every voxel whose
    projection is farther than 1e-3 px from a pixel edge in every camera
    (the oracle's `boundary` flag);
  * the occupied set and count bit-exact, except voxels in that boundary
    bucket and voxels whose FP64 log-odds lies within TIE_EPS of the
    threshold's log-odds.  TIE_EPS = 1e-4 bounds the FP32 rounding of the
    log-odds sum: each camera's stored log ratio carries a few 1e-7 of
    rounding and at most 32 cameras are summed.
"""

from __future__ import annotations

import math

import numpy as np
import torch

import oracle
from paper_1311_6811_gb300 import psfs

TIE_EPS = 1e-4
OCC_TOL = 1e-5


def to_dev(a, dev="cuda"):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def gpu_reconstruct(grid, cams, images, mean, var, params=None, map_dtype=None, capacity=None):
    rec = psfs.Reconstructor(grid, cams, params, map_dtype=map_dtype, capacity=capacity)
    rec.set_background(to_dev(mean), to_dev(var))
    occ, lst, cnt = rec.reconstruct(to_dev(images))
    st = rec.sync()
    out = {"occ": occ.cpu().numpy().ravel().astype(np.float64),
           "count": int(cnt.item()) & 0xFFFFFFFF,
           "list": psfs.voxel_list(lst, cnt, rec.capacity).numpy(),
           "status": st}
    rec.close()
    return out


def logit(p):
    return math.log(p / (1 - p))


def compare(got, ref, threshold=0.5, occ_tol=OCC_TOL, exact=True):
    """Returns a report dict; asserts the tolerances when `exact`."""
    keep = ~ref["boundary"]
    d = np.abs(got["occ"] - ref["occ"])
    max_err = float(d[keep].max()) if keep.any() else 0.0
    got_set = np.zeros(ref["occ"].size, bool)
    got_set[got["list"]] = True
    diff = np.flatnonzero(got_set != ref["occupied"])
    tie = np.abs(ref["logodds"] - logit(threshold)) < TIE_EPS
    allowed = ref["boundary"] | tie
    bad = diff[~allowed[diff]]
    report = {"max_abs_err": max_err, "mean_abs_err": float(d[keep].mean()) if keep.any() else 0.0,
              "boundary_voxels": int(ref["boundary"].sum()), "tie_voxels": int(tie.sum()),
              "set_diff": int(diff.size), "set_diff_unexplained": int(bad.size),
              "count": got["count"], "count_ref": int(ref["list"].size)}
    if exact:
        assert max_err <= occ_tol, report
        assert bad.size == 0, report
        assert got["count"] == got["list"].size or got["status"] == psfs.PSFS_ERR_CAPACITY
        explained = int(diff.size)
        assert abs(got["count"] - ref["list"].size) <= explained, report
    return report
