"""torch.autograd.Function wrappers over the CUDA forward and adjoint of
libpsfs (marshalling only: both directions run in the library's kernels).

  occ = psfs_occupancy(rec, images, mean, var)   # grads for mean and var
  occ = psfs_occupancy_from_slm(rec, slm)        # grad for the SLM maps
  occ = psfs_occupancy_sequence(rec, images, mean, var)
      # F frames [F][n_cams][H][W][3] -> [F][nz][ny][nx]: the sequence path
      # forward (frame groups) and the batched adjoint; the background is
      # shared by the frames, so its gradients are summed over them

`rec` is a `Reconstructor`.  The Functions over images keep the uint8 images
and their own output (the occupancy) for the backward, which then forms
dLoss/dL from that occupancy (psfs_backward_from_occupancy) instead of
recomputing the forward; nothing of size n_voxels x n_cams is kept between
the two passes.  The SLM Function keeps the maps and recomputes.
"""

from __future__ import annotations

import torch

from . import psfs


class _Occupancy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rec, images, mean, var):
        rec.set_background(mean.detach().contiguous(), var.detach().contiguous())
        occ, _, _ = rec.reconstruct(images)
        ctx.rec = rec
        ctx.save_for_backward(images, occ)
        ctx.shapes = (mean.shape, var.shape)
        return occ

    @staticmethod
    def backward(ctx, grad_occ):
        images, occ = ctx.saved_tensors
        rec = ctx.rec
        d_mean = torch.empty(ctx.shapes[0], dtype=torch.float32, device=images.device)
        d_var = torch.empty(ctx.shapes[1], dtype=torch.float32, device=images.device)
        # the forward's own occupancy: nothing of the forward is recomputed
        psfs.psfs_backward_from_occupancy(rec.handle, 1, images, occ, grad_occ.contiguous().float(), None, d_mean,
                                          d_var)
        return None, None, d_mean, d_var


class _OccupancyFromSlm(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rec, slm):
        slm_c = slm.detach().contiguous()
        occ, _, _ = rec.fuse_slm(slm_c)
        ctx.rec = rec
        ctx.save_for_backward(slm_c)
        return occ

    @staticmethod
    def backward(ctx, grad_occ):
        (slm,) = ctx.saved_tensors
        d_slm = torch.empty_like(slm)
        psfs.psfs_backward_slm(ctx.rec.handle, slm, grad_occ.contiguous().float(), d_slm)
        return None, d_slm


class _OccupancySequence(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rec, images, mean, var):
        rec.set_background(mean.detach().contiguous(), var.detach().contiguous())
        n = images.shape[0]
        occ = torch.empty((n, *rec.shape), dtype=torch.float32, device=images.device)
        counts = torch.zeros(n, dtype=torch.int32, device=images.device)
        # occupancy only: no voxel lists (capacity 0; counts are still formed)
        psfs.psfs_reconstruct_sequence(rec.handle, n, images, occ, None, 0, counts)
        ctx.rec = rec
        ctx.save_for_backward(images, occ)
        ctx.shapes = (mean.shape, var.shape)
        return occ

    @staticmethod
    def backward(ctx, grad_occ):
        images, occ = ctx.saved_tensors
        d_mean = torch.empty(ctx.shapes[0], dtype=torch.float32, device=images.device)
        d_var = torch.empty(ctx.shapes[1], dtype=torch.float32, device=images.device)
        psfs.psfs_backward_from_occupancy(ctx.rec.handle, images.shape[0], images, occ,
                                          grad_occ.contiguous().float(), None, d_mean, d_var)
        return None, None, d_mean, d_var


def psfs_occupancy_sequence(rec, images, mean, var):
    """Posterior occupancy [F][nz][ny][nx] of F frames; differentiable in the
    shared background `mean` and `var` (gradients summed over the frames)."""
    return _OccupancySequence.apply(rec, images, mean, var)


def psfs_occupancy(rec, images, mean, var):
    """Posterior occupancy [nz][ny][nx]; differentiable in `mean` and `var`."""
    return _Occupancy.apply(rec, images, mean, var)


def psfs_occupancy_from_slm(rec, slm):
    """Posterior occupancy from SLM maps [n_cams][H][W]; differentiable in `slm`."""
    return _OccupancyFromSlm.apply(rec, slm)
