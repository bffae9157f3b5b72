"""Voxel silhouettes on the GPU (psfs_reproject) against the oracle's brute
force.  The GPU tests pixel-centre rays in float32, so a pixel whose ray
passes within ~1e-3 voxel of a cube edge may go either way: every pixel the
oracle sets with the cubes shrunk by GROW voxel sizes must be set, and every
pixel it leaves unset with the cubes grown by GROW must be unset."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1311_6811_gb300 import psfs  # noqa: E402
from synth import scene as S  # noqa: E402
from tests.gpu_helpers import to_dev  # noqa: E402

pytestmark = pytest.mark.gpu
GROW = 2e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    psfs.load()


def _gpu_masks(rec, lists, counts, stride):
    F = counts.numel()
    H, W = rec.image_shape[1], rec.image_shape[2]
    masks = torch.full((F, rec.n_cams, H, W), 7, dtype=torch.uint8, device="cuda")
    psfs.psfs_reproject(rec.handle, F, lists, stride, counts, masks)
    assert rec.sync() == psfs.PSFS_OK
    return masks.cpu().numpy()


def _check(grid, cams, lst, got):
    assert set(np.unique(got)) <= {0, 1}
    inner = oracle.reproject(grid, cams, lst, grow=-GROW)
    outer = oracle.reproject(grid, cams, lst, grow=GROW)
    assert np.all(got >= inner), int((got < inner).sum())
    assert np.all(got <= outer), int((got > outer).sum())
    return int((outer != inner).sum())


def test_random_sets_and_a_box():
    sc = S.make_scene(seed=41, grid_n=24, cube_side=2.0, n_cams=3, width=64, height=48, focal=60.0)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    V = sc.grid.n_voxels
    rng = np.random.default_rng(1)
    box = np.zeros((24, 24, 24), bool)
    box[4:15, 6:20, 2:12] = True
    sets = [rng.choice(V, 40, replace=False), rng.choice(V, 400, replace=False), np.flatnonzero(box.ravel()),
            np.array([], np.int64)]
    stride = max(s.size for s in sets)
    lists = torch.zeros((len(sets), stride), dtype=torch.int32)
    counts = torch.zeros((len(sets),), dtype=torch.int32)
    for f, s_ in enumerate(sets):
        lists[f, :s_.size] = torch.from_numpy(s_.astype(np.int32))
        counts[f] = s_.size
    got = _gpu_masks(rec, lists.cuda(), counts.cuda(), stride)
    for f, s_ in enumerate(sets):
        _check(sc.grid, sc.cams, s_.astype(np.uint32), got[f])
    assert got[2].sum() > 500 and got[3].sum() == 0
    rec.close()


def test_reconstructed_surface_silhouettes():
    """A walking sequence: the silhouettes of each frame's surface list (and,
    for one frame, of its full occupied list) against the oracle."""
    sc = S.make_scene(seed=42, grid_n=32, cube_side=2.0, n_cams=4, width=96, height=72, focal=90.0,
                      n_frames=3, walking=True)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    imgs = to_dev(sc.images)
    F, V = imgs.shape[0], rec.n_voxels
    occ = torch.empty((F, V), device="cuda")
    lists = torch.empty((F, V), dtype=torch.int32, device="cuda")
    counts = torch.zeros((F,), dtype=torch.int32, device="cuda")
    psfs.psfs_reconstruct_sequence(rec.handle, F, imgs, occ, lists, V, counts)
    sl = torch.empty((F, V), dtype=torch.int32, device="cuda")
    sc_n = torch.zeros((F,), dtype=torch.int32, device="cuda")
    psfs.psfs_surface(rec.handle, F, lists, V, counts, sl, V, sc_n)
    got_s = _gpu_masks(rec, sl, sc_n, V)
    got_o = _gpu_masks(rec, lists, counts, V)
    for f in range(F):
        surf = sl[f, :int(sc_n[f])].cpu().numpy().astype(np.uint32)
        assert surf.size > 50
        _check(sc.grid, sc.cams, surf, got_s[f])
        # the solid and its surface: the same silhouette up to grazing rays
        assert (got_s[f] != got_o[f]).sum() <= 0.001 * got_o[f].size
    full0 = lists[0, :int(counts[0])].cpu().numpy().astype(np.uint32)
    _check(sc.grid, sc.cams, full0, got_o[0])
    rec.close()


def test_camera_inside_the_grid():
    """Cameras inside an 8 m grid: cubes next to or behind a camera take the
    whole-image path; the exact test still decides."""
    sc = S.make_scene(seed=14, grid_n=12, cube_side=8.0, n_cams=2, width=48, height=40, focal=40.0)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    V = sc.grid.n_voxels
    rng = np.random.default_rng(3)
    s_ = rng.choice(V, 200, replace=False).astype(np.int32)
    lists = torch.from_numpy(s_).cuda().view(1, -1)
    counts = torch.tensor([s_.size], dtype=torch.int32, device="cuda")
    got = _gpu_masks(rec, lists, counts, s_.size)
    _check(sc.grid, sc.cams, s_.astype(np.uint32), got[0])
    rec.close()


@pytest.mark.parametrize("width,height,n_set", [(66, 50, 300), (320, 240, 300)])
def test_staged_and_direct_paths(width, height, n_set):
    """A CTA stages its chunk of 256 voxels in shared memory when the union of
    their boxes fits 32 KB of 4-byte-aligned rows, and stores directly
    otherwise: rows not a multiple of 4 bytes wide (66 px, direct), scattered
    voxels in a 320 x 240 image (unions larger than 32 KB, direct) and a
    solid box in the same rig (staged chunks)."""
    sc = S.make_scene(seed=43, grid_n=24, cube_side=2.0, n_cams=3, width=width, height=height,
                      focal=0.9 * width)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    V = sc.grid.n_voxels
    rng = np.random.default_rng(4)
    box = np.zeros((24, 24, 24), bool)
    box[6:18, 8:16, 4:20] = True
    sets = [rng.choice(V, n_set, replace=False), np.flatnonzero(box.ravel())]
    stride = max(s.size for s in sets)
    lists = torch.zeros((len(sets), stride), dtype=torch.int32)
    counts = torch.zeros((len(sets),), dtype=torch.int32)
    for f, s_ in enumerate(sets):
        lists[f, :s_.size] = torch.from_numpy(s_.astype(np.int32))
        counts[f] = s_.size
    got = _gpu_masks(rec, lists.cuda(), counts.cuda(), stride)
    for f, s_ in enumerate(sets):
        _check(sc.grid, sc.cams, s_.astype(np.uint32), got[f])
        assert got[f].sum() > 100
    rec.close()
