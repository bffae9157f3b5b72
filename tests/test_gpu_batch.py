"""The batched persistent launch: many frames with different grids, camera
counts, image sizes and backgrounds in one CUDA-graph launch must give what
psfs_reconstruct gives frame by frame (the same arithmetic, so the same
bits), and match the FP64 oracle on sampled frames."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1311_6811_gb300 import psfs  # noqa: E402
from synth import scene as S  # noqa: E402
from tests.gpu_helpers import compare, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    psfs.load()


def _frames(specs, seed):
    """Each spec: (grid_n or (nx, ny, nz), cube_side, n_cams, W, H, f)."""
    out = []
    for n, (g, side, K, W, H, f) in enumerate(specs):
        sc = S.make_scene(seed=seed + n, grid_n=g if isinstance(g, int) else g[0], cube_side=side, n_cams=K,
                          width=W, height=H, focal=f)
        if not isinstance(g, int):
            sc.grid = S.Grid(g[0], g[1], g[2], sc.grid.origin, sc.grid.voxel_size)
        out.append(sc)
    return out


def _run_batch(scenes, tune=False):
    recs, frames, outs = [], [], []
    for sc in scenes:
        rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
        rec.set_background(to_dev(sc.mean), to_dev(sc.var))
        img = to_dev(sc.images)
        occ, lst, cnt = rec.alloc_outputs()
        recs.append((rec, img))
        frames.append((rec.handle, img, occ, lst, rec.capacity, cnt))
        outs.append((occ, lst, cnt, rec.capacity))
    b = psfs.psfs_batch_create(frames)
    if tune:
        psfs.psfs_batch_autotune(b, reps=1)
    psfs.psfs_batch_run(b)
    assert psfs.psfs_batch_sync(b) == psfs.PSFS_OK
    return b, recs, outs


def _host(out):
    occ, lst, cnt, cap = out
    return occ.cpu().numpy().ravel(), psfs.voxel_list(lst, cnt, cap).numpy(), int(cnt.item())


# odd camera counts leave partial camera blocks; 3 x 101 x 77 pixels leave a
# last likelihood chunk of 291 pixels (not bulk-copied: plain loads)
SPECS = [(32, 2.0, 3, 160, 120, 150.0), (40, 2.0, 5, 200, 150, 190.0), ((48, 40, 36), 2.0, 4, 160, 120, 150.0),
         (24, 2.0, 6, 128, 96, 120.0), (37, 2.0, 4, 104, 77, 95.0), (56, 2.2, 7, 200, 150, 190.0),
         (23, 2.0, 3, 101, 77, 95.0)]


def test_batch_equals_frame_by_frame_and_oracle():
    scenes = _frames(SPECS, seed=60)
    b, recs, outs = _run_batch(scenes)
    got = [_host(o) for o in outs]
    for (rec, img), g in zip(recs, got):
        occ, lst, cnt = rec.reconstruct(img)
        assert rec.sync() == psfs.PSFS_OK
        np.testing.assert_array_equal(g[0], occ.cpu().numpy().ravel())
        np.testing.assert_array_equal(g[1], psfs.voxel_list(lst, cnt, rec.capacity).numpy())
    # relaunching the graph gives the same bits
    psfs.psfs_batch_run(b)
    assert psfs.psfs_batch_sync(b) == psfs.PSFS_OK
    for o, g in zip(outs, got):
        np.testing.assert_array_equal(_host(o)[0], g[0])
    # every tile shape, and the autotuner's pick, give the same bits
    for cfg in psfs.BATCH_CONFIGS:
        psfs.psfs_batch_set_config(b, *cfg[:3], cameras_per_block=cfg[4], launch=cfg[5])
        psfs.psfs_batch_run(b)
        assert psfs.psfs_batch_sync(b) == psfs.PSFS_OK
        for o, g in zip(outs, got):
            np.testing.assert_array_equal(_host(o)[0], g[0])
    best = psfs.psfs_batch_autotune(b, reps=1)
    assert best in psfs.BATCH_CONFIGS
    with pytest.raises(psfs.PsfsError):
        psfs.psfs_batch_set_config(b, 32, 4, 4, cameras_per_block=2)   # not an instantiated combination
    # FP64 oracle on two frames
    for n in (1, 2):
        sc = scenes[n]
        ref = oracle.reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params)
        compare({"occ": got[n][0].astype(np.float64), "list": got[n][1], "count": got[n][2], "status": 0}, ref)
    psfs.psfs_batch_destroy(b)
    for rec, _ in recs:
        rec.close()


@pytest.mark.slow
def test_batch_64_heterogeneous_frames():
    """64 frames, grids drawn from {96, 128, 160, 192}^3, 4-12 cameras, 640x480
    or 960x540, own pose and background per frame, one graph launch."""
    import os
    scenes = S.batch_64_scenes(seed=64, workers=max(1, min(8, os.cpu_count() or 1)))
    b, recs, outs = _run_batch(scenes, tune=True)
    for k, ((rec, img), o) in enumerate(zip(recs, outs)):
        g = _host(o)
        occ, lst, cnt = rec.reconstruct(img)
        assert rec.sync() == psfs.PSFS_OK
        np.testing.assert_array_equal(g[0], occ.cpu().numpy().ravel())
        assert g[2] == int(cnt.item())
    for n in (0, 37):
        sc = scenes[n]
        g = _host(outs[n])
        ref = oracle.reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params)
        compare({"occ": g[0].astype(np.float64), "list": g[1], "count": g[2], "status": 0}, ref)
    # throughput of the graph launch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        psfs.psfs_batch_run(b)
    e1.record()
    torch.cuda.synchronize()
    evals = sum(sc.grid.n_voxels * sc.n_cams for sc in scenes)
    ms = e0.elapsed_time(e1) / 3
    print(f"batch of 64: {ms:.2f} ms, {evals / ms / 1e6:.1f} Gvox-cam/s")
    assert psfs.psfs_batch_sync(b) == psfs.PSFS_OK
    psfs.psfs_batch_destroy(b)
    for rec, _ in recs:
        rec.close()


def test_batch_wait_timeout_is_reported_and_recovers():
    """Failure detection without a fault: with a 1 ms limit and one frame
    held (its fusion items wait for a chunk that never comes), the bounded
    device-side wait runs out, psfs_batch_sync returns PSFS_ERR_TIMEOUT, and
    the context stays usable: the next launch without the hold returns
    PSFS_OK with every frame as psfs_reconstruct gives it."""
    scenes = _frames([(32, 2.0, 4, 160, 120, 150.0), (40, 2.0, 3, 128, 96, 120.0),
                      (24, 1.5, 5, 96, 80, 90.0)], seed=70)
    b, recs, outs = _run_batch(scenes)
    psfs.psfs_batch_set_wait_limit(b, 1_000_000, hold_frame=1)
    psfs.psfs_batch_run(b)
    with pytest.raises(psfs.PsfsError) as e:
        psfs.psfs_batch_sync(b)
    assert e.value.status == psfs.PSFS_ERR_TIMEOUT
    assert "timed out" in psfs.psfs_last_error_message()
    psfs.psfs_batch_set_wait_limit(b, 1_000_000_000, hold_frame=-1)
    psfs.psfs_batch_run(b)
    assert psfs.psfs_batch_sync(b) == psfs.PSFS_OK
    for (rec, img), out in zip(recs, outs):
        got = _host(out)
        occ, lst, cnt = rec.reconstruct(img)
        assert rec.sync() == psfs.PSFS_OK
        np.testing.assert_array_equal(got[0], occ.cpu().numpy().ravel())
        np.testing.assert_array_equal(got[1], psfs.voxel_list(lst, cnt, rec.capacity).numpy())
    with pytest.raises(psfs.PsfsError):
        psfs.psfs_batch_set_wait_limit(b, 10, hold_frame=-1)        # below 1 us
    with pytest.raises(psfs.PsfsError):
        psfs.psfs_batch_set_wait_limit(b, 1_000_000, hold_frame=3)  # no such frame
    psfs.psfs_batch_destroy(b)
    for rec, _ in recs:
        rec.close()
