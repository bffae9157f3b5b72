"""Runs one small case of every device entry point and prints, as JSON, each
call's status (psfs_sync) and a digest of its outputs.  tests/test_gpu_bounds.py
runs it under the product build and under the bounds-checked build
(PSFS_BOUNDS_CHECK=1): every status must be ok and the digests equal."""

import json
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1311_6811_gb300 import psfs  # noqa: E402
from synth import scene as S  # noqa: E402


def digest(*ts):
    out = []
    for t in ts:
        a = t.detach().cpu().numpy() if isinstance(t, torch.Tensor) else np.asarray(t)
        if a.dtype.kind == "f":
            out.append(float(np.float64(a.astype(np.float64).sum())))
        else:
            out.append(int(np.sort(a.astype(np.int64).ravel()).sum()))
    return out


def main():
    assert torch.cuda.is_available()
    res = {"lib": psfs.lib_path()}
    sc = S.make_scene(seed=21, grid_n=48, cube_side=2.0, n_cams=4, width=160, height=120, focal=150.0,
                      n_frames=20, walking=True)
    dev = "cuda"
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(torch.from_numpy(sc.mean).to(dev), torch.from_numpy(sc.var).to(dev))
    imgs = torch.from_numpy(sc.images).to(dev)
    F, V = imgs.shape[0], rec.n_voxels
    h = rec.handle

    def sync(name, *outs):
        res[name] = {"status": psfs.psfs_status_string(rec.sync()), "digest": digest(*outs)}

    # one frame per call, every one-frame tile shape (direct and staged)
    for cfg in psfs.FUSE_CONFIGS:
        psfs.psfs_set_fuse_config(h, *cfg)
        o, l, c = rec.reconstruct(imgs[0])
        n = int(c.item())
        sync("reconstruct_%d_%d_%d_%d" % cfg, o, l[:min(n, rec.capacity)], c)
    # the sequence path: groups of 8 and 16 with 32-byte records, 16 with 64-byte records
    occ = torch.empty((F, V), device=dev)
    lists = torch.empty((F, V), dtype=torch.int32, device=dev)
    cnt = torch.zeros(F, dtype=torch.int32, device=dev)
    for g, tz, rb in ((8, 4, 32), (16, 2, 32), (16, 2, 64)):
        psfs.psfs_set_fuse_config(h, 8, 4, 8, 0, 2, g, 8, tz, rb)
        psfs.psfs_reconstruct_sequence(h, F, imgs, occ, lists, V, cnt)
        sync(f"sequence_{g}_{tz}_{rb}", occ, cnt,
             *[lists[f, :int(cnt[f])] for f in range(F)])
    # the adjoint: one frame, batched (recomputed forward), from the occupancy
    n_pix = imgs[0].numel() // 3
    g = torch.Generator().manual_seed(3)
    d_occ = torch.randn((F, V), generator=g).to(dev)
    d_slm = torch.empty((F, n_pix), device=dev)
    d_mean = torch.empty(n_pix * 3, device=dev)
    d_var = torch.empty(n_pix * 3, device=dev)
    psfs.psfs_backward(h, imgs[0], d_occ[0], d_slm[0], d_mean, d_var)
    sync("backward", d_slm[0], d_mean, d_var)
    psfs.psfs_backward_sequence(h, F, imgs, d_occ, d_slm, d_mean, d_var)
    sync("backward_sequence", d_slm, d_mean, d_var)
    psfs.psfs_backward_from_occupancy(h, F, imgs, occ, d_occ, d_slm, d_mean, d_var)
    sync("backward_from_occupancy", d_slm, d_mean, d_var)
    # the NEXT rows
    sl = torch.empty((F, V), dtype=torch.int32, device=dev)
    sn = torch.zeros(F, dtype=torch.int32, device=dev)
    psfs.psfs_surface(h, F, lists, V, cnt, sl, V, sn)
    sync("surface", sn, *[sl[f, :int(sn[f])] for f in range(F)])
    masks = torch.empty((F, len(sc.cams), sc.cams[0].height, sc.cams[0].width), dtype=torch.uint8, device=dev)
    psfs.psfs_reproject(h, F, sl, V, sn, masks)
    sync("reproject", masks)
    sm = torch.empty((F, V), device=dev)
    sml = torch.empty((F, V), dtype=torch.int32, device=dev)
    smc = torch.zeros(F, dtype=torch.int32, device=dev)
    psfs.psfs_smooth(h, F, occ, sm, sml, V, smc)
    sync("smooth", sm, smc)
    rec.close()
    # the batched persistent launch over two frames of the rig
    recs = [psfs.Reconstructor(sc.grid, sc.cams, sc.params) for _ in range(2)]
    outs = []
    for r in recs:
        r.set_background(torch.from_numpy(sc.mean).to(dev), torch.from_numpy(sc.var).to(dev))
        outs.append(r.alloc_outputs())
    b = psfs.psfs_batch_create([(r.handle, imgs[f], o[0], o[1], r.capacity, o[2])
                                for f, (r, o) in enumerate(zip(recs, outs))])
    psfs.psfs_batch_run(b)
    res["batch"] = {"status": psfs.psfs_status_string(psfs.psfs_batch_sync(b)),
                    "digest": digest(*[o[0] for o in outs], *[o[2] for o in outs])}
    psfs.psfs_batch_destroy(b)
    for r in recs:
        r.close()
    print(json.dumps(res))


if __name__ == "__main__":
    main()
