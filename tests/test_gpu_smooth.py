"""Smoothing before the threshold on the GPU (psfs_smooth) against the
oracle's 3 x 3 x 3 box mean over in-grid neighbours, on the same FP32 inputs.

Tolerance: the FP32 sum of 27 probabilities (each in [0, 1]) carries at most
26 roundings of at most 2^-24 of the running sum (<= 27); the scaling by the
FP32 reciprocal of the count (>= 8) adds two more relative roundings of
2^-24 on a result <= 1; that bounds the error by 26 * 27 * 2^-24 / 8 +
2 * 2^-24 < 5.4e-6, so SMOOTH_TOL = 6e-6.  The thresholded
set is exact except voxels whose FP64 smoothed value lies within SMOOTH_TOL of
the threshold (counted)."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1311_6811_gb300 import psfs  # noqa: E402
from synth import scene as S  # noqa: E402
from tests.gpu_helpers import to_dev  # noqa: E402

pytestmark = pytest.mark.gpu
SMOOTH_TOL = 6e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    psfs.load()


def _rec(grid, threshold=0.5):
    sc = S.make_scene(seed=3, grid_n=24, cube_side=2.0, n_cams=2, width=64, height=48, focal=60.0)
    params = S.Params(threshold=threshold)
    return psfs.Reconstructor(grid, sc.cams, params)


def _check(shape, prob_f32, got_sm, got_list, got_count, threshold):
    ref = oracle.smooth(shape, prob_f32.astype(np.float64), threshold)
    if got_sm is not None:
        err = np.abs(got_sm.astype(np.float64) - ref["smoothed"]).max()
        assert err <= SMOOTH_TOL, err
    tie = np.abs(ref["smoothed"] - threshold) < SMOOTH_TOL
    got = np.zeros(prob_f32.size, bool)
    got[got_list] = True
    diff = np.flatnonzero(got != ref["occupied"])
    assert tie[diff].all(), diff[~tie[diff]]
    assert got_count == got_list.size
    return int(diff.size)


@pytest.mark.parametrize("dims", [(37, 29, 23), (64, 64, 64), (8, 8, 8), (33, 9, 17), (150, 20, 12), (132, 35, 9)])
def test_random_fields(dims):
    """Ragged grids: partial tiles along x, y and z, several tiles along
    each axis (150 and 132 columns, 35 rows), odd and small extents."""
    nx, ny, nz = dims
    grid = S.Grid(nx, ny, nz, (-1.0, -1.0, 0.0), 0.05)
    rec = _rec(grid)
    rng = np.random.default_rng(nx * 7 + nz)
    F = 3
    V = nx * ny * nz
    # smooth blobs plus noise: plenty of voxels on both sides of the threshold
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    base = np.exp(-((x - nx / 2) ** 2 / (nx * 2.0) + (y - ny / 2) ** 2 / (ny * 2.0) + (z - nz / 2) ** 2 / (nz * 2.0)))
    probs = np.stack([np.clip(base + 0.3 * rng.standard_normal(base.shape), 0, 1).ravel() for _ in range(F)])
    probs = probs.astype(np.float32)
    occ = torch.from_numpy(probs).cuda()
    sm = torch.full((F, V), -1.0, device="cuda")
    lists = torch.full((F, V), -1, dtype=torch.int32, device="cuda")
    counts = torch.full((F,), 9, dtype=torch.int32, device="cuda")
    psfs.psfs_smooth(rec.handle, F, occ, sm, lists, V, counts)
    assert rec.sync() == psfs.PSFS_OK
    for f in range(F):
        c = int(counts[f])
        _check((nx, ny, nz), probs[f], sm[f].cpu().numpy(), np.sort(lists[f, :c].cpu().numpy()), c, 0.5)
    # without the smoothed output: the same lists
    lists2 = torch.full((F, V), -1, dtype=torch.int32, device="cuda")
    counts2 = torch.zeros((F,), dtype=torch.int32, device="cuda")
    psfs.psfs_smooth(rec.handle, F, occ, None, lists2, V, counts2)
    assert rec.sync() == psfs.PSFS_OK
    for f in range(F):
        c = int(counts[f])
        assert int(counts2[f]) == c
        np.testing.assert_array_equal(np.sort(lists2[f, :c].cpu().numpy()), np.sort(lists[f, :c].cpu().numpy()))
    rec.close()


def test_reconstructed_frames_and_other_threshold():
    sc = S.make_scene(seed=31, grid_n=48, cube_side=2.0, n_cams=4, width=160, height=120, focal=150.0,
                      n_frames=3, walking=True)
    for thr in (0.5, 0.3):
        params = S.Params(threshold=thr)
        rec = psfs.Reconstructor(sc.grid, sc.cams, params)
        rec.set_background(to_dev(sc.mean), to_dev(sc.var))
        imgs = to_dev(sc.images)
        F, V = imgs.shape[0], rec.n_voxels
        occ = torch.empty((F, V), device="cuda")
        lists = torch.empty((F, V), dtype=torch.int32, device="cuda")
        counts = torch.zeros((F,), dtype=torch.int32, device="cuda")
        psfs.psfs_reconstruct_sequence(rec.handle, F, imgs, occ, lists, V, counts)
        sm = torch.empty((F, V), device="cuda")
        sl = torch.empty((F, V), dtype=torch.int32, device="cuda")
        scn = torch.zeros((F,), dtype=torch.int32, device="cuda")
        psfs.psfs_smooth(rec.handle, F, occ, sm, sl, V, scn)
        assert rec.sync() == psfs.PSFS_OK
        shape = (sc.grid.nx, sc.grid.ny, sc.grid.nz)
        for f in range(F):
            c = int(scn[f])
            assert c > 100
            _check(shape, occ[f].cpu().numpy(), sm[f].cpu().numpy(), np.sort(sl[f, :c].cpu().numpy()), c, thr)
        rec.close()


def test_capacity_overflow():
    grid = S.Grid(20, 20, 20, (-1.0, -1.0, 0.0), 0.1)
    rec = _rec(grid)
    prob = np.zeros((20, 20, 20), np.float32)
    prob[5:15, 5:15, 5:15] = 1.0
    occ = torch.from_numpy(prob.ravel()).cuda().view(1, -1)
    lists = torch.full((1, 50), -1, dtype=torch.int32, device="cuda")
    counts = torch.zeros((1,), dtype=torch.int32, device="cuda")
    psfs.psfs_smooth(rec.handle, 1, occ, None, lists, 50, counts)
    assert rec.sync() == psfs.PSFS_ERR_CAPACITY
    ref = oracle.smooth((20, 20, 20), prob.ravel().astype(np.float64), 0.5)
    assert int(counts[0]) == ref["list"].size
    assert np.isin(lists[0].cpu().numpy(), ref["list"]).all()
    rec.close()
