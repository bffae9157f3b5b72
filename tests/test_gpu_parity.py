"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded
synthetic scenes.  Tolerances are stated in tests/gpu_helpers.py."""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1311_6811_gb300 import psfs  # noqa: E402
from synth import scene as S  # noqa: E402
from tests.gpu_helpers import compare, gpu_reconstruct, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    psfs.load()


def test_likelihood_map_matches_oracle():
    """Eq. 1-2 per pixel: FP32 kernel vs FP64 oracle, 64^3 x 4 x 320x240 scene."""
    sc = S.scene_64cube_4cam(seed=0)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    s = rec.likelihood(to_dev(sc.images)).cpu().numpy().astype(np.float64)
    ref = oracle.slm(sc.images, sc.mean, sc.var, sc.params.log_fg_density)
    np.testing.assert_allclose(s, ref, rtol=2e-5, atol=2e-6)
    rec.close()


def test_64cube_4cam_frame():
    sc = S.scene_64cube_4cam(seed=0)
    got = gpu_reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params)
    ref = oracle.reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params)
    rep = compare(got, ref)
    assert ref["list"].size > 1000
    print(rep)


@pytest.mark.slow
def test_128cube_8cam_frames_full_size():
    """Full-size 128^3 x 8 x 640x480 frames of the walking sequence."""
    sc = S.scene_128cube_8cam(seed=1, n_frames=2)
    for f in range(2):
        got = gpu_reconstruct(sc.grid, sc.cams, sc.images[f], sc.mean, sc.var, sc.params)
        ref = oracle.reconstruct(sc.grid, sc.cams, sc.images[f], sc.mean, sc.var, sc.params)
        rep = compare(got, ref)
        assert ref["list"].size > 10000
        print(f, rep)


@pytest.mark.parametrize("width", [101, 104])
def test_ragged_grid_and_odd_image(width):
    """Grid 37 x 29 x 23 (ragged in every tile dimension), 3 cameras of
    width x 77 pixels.  At 101 (3 * 101 * 77 not a multiple of 4) the scalar
    tail of the likelihood kernel runs and rows are not 16-byte aligned, so
    the fuse kernel gathers from global memory; at 104 it stages boxes in
    shared memory with ragged tiles."""
    rng = np.random.default_rng(3)
    cams = S.ring_cameras(rng, 3, width, 77, 95.0, (0.0, 0.0, 1.0))
    grid = S.Grid(37, 29, 23, (-0.9, -0.7, 0.1), 0.05)
    mean, sigma = S.make_background(rng, 3, 77, width)
    var = (sigma ** 2 + 4).astype(np.float32)
    caps = S.body_capsules(S.random_pose(rng), rng.uniform(0, 255, (10, 3)))
    img = S.render_images(rng, cams, caps, mean, sigma)
    p = S.Params()
    got = gpu_reconstruct(grid, cams, img, mean.astype(np.float32), var, p)
    ref = oracle.reconstruct(grid, cams, img, mean.astype(np.float32), var, p)
    compare(got, ref)
    assert ref["list"].size > 50


@pytest.mark.parametrize("prior,thr", [(0.5, 0.5), (0.3, 0.6), (0.7, 0.4)])
def test_other_rates_prior_threshold(prior, thr):
    sc = S.make_scene(seed=8, grid_n=48, cube_side=2.0, n_cams=5, width=200, height=150, focal=190.0)
    p = S.Params(p_detect=0.8, p_false_alarm=0.25, prior=prior, threshold=thr)
    got = gpu_reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, p)
    ref = oracle.reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, p)
    compare(got, ref, threshold=thr)


def test_literal_eq6_to_9_rates():
    """P_D = 1, P_FA = 0 (Eq. 6-9 verbatim): the degenerate branch of the log ratio."""
    sc = S.make_scene(seed=9, grid_n=40, cube_side=2.0, n_cams=4, width=160, height=120, focal=150.0)
    p = S.Params(p_detect=1.0, p_false_alarm=0.0)
    got = gpu_reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, p)
    ref = oracle.reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, p)
    compare(got, ref)


def test_visual_hull_from_binary_maps():
    """psfs_fuse_slm on near-binary maps with P_D = 1, P_FA = 0: the set must
    equal the oracle's (the visual hull), excluding pixel-edge voxels."""
    rng = np.random.default_rng(12)
    cams = S.ring_cameras(rng, 4, 96, 72, 85.0, (0.0, 0.0, 1.0))
    caps = [S.Capsule(np.array([-0.2, 0.1, 0.7]), np.array([0.25, -0.1, 1.35]), 0.2, np.zeros(3))]
    eps = 1e-6
    maps = np.stack([np.where(S.render_labels(c, caps) >= 0, 1 - eps, eps) for c in cams]).astype(np.float32)
    grid = {"nx": 32, "ny": 32, "nz": 32, "origin": (-0.6, -0.6, 0.4), "voxel_size": 1.2 / 32}
    p = {"p_detect": 1.0, "p_false_alarm": 0.0, "prior": 0.5, "threshold": 0.5}
    rec = psfs.Reconstructor(grid, cams, p)
    occ, lst, cnt = rec.fuse_slm(to_dev(maps))
    assert rec.sync() == psfs.PSFS_OK
    got = {"occ": occ.cpu().numpy().ravel().astype(np.float64), "count": int(cnt.item()),
           "list": psfs.voxel_list(lst, cnt, rec.capacity).numpy(), "status": 0}
    ref = oracle.fuse(grid, cams, maps.astype(np.float64), p)
    # the carved set: occupied iff every seeing camera sees the capsule
    compare(got, ref, occ_tol=1e-5)
    assert ref["list"].size > 100
    rec.close()


def test_empty_scene_and_unseen_grid():
    """No body: nothing occupied.  A grid no camera sees keeps the prior."""
    rng = np.random.default_rng(4)
    cams = S.ring_cameras(rng, 4, 128, 96, 120.0, (0.0, 0.0, 1.0))
    mean, sigma = S.make_background(rng, 4, 96, 128)
    img = S.render_images(rng, cams, [], mean, sigma)
    var = (sigma ** 2 + 4).astype(np.float32)
    grid = S.Grid(24, 24, 24, (-1.0, -1.0, 0.0), 2.0 / 24)
    got = gpu_reconstruct(grid, cams, img, mean.astype(np.float32), var, S.Params())
    assert got["count"] == 0
    far = S.Grid(16, 16, 16, (30.0, 30.0, 30.0), 0.1)
    for prior, n_expect in [(0.5, 0), (0.7, 16 ** 3)]:
        got = gpu_reconstruct(far, cams, img, mean.astype(np.float32), var, S.Params(prior=prior))
        assert np.all(np.abs(got["occ"] - prior) <= 1e-7)
        assert got["count"] == n_expect


def test_capacity_overflow_reports_true_count():
    sc = S.scene_64cube_4cam(seed=0)
    ref = oracle.reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params)
    cap = 100
    got = gpu_reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params, capacity=cap)
    assert got["status"] == psfs.PSFS_ERR_CAPACITY
    assert abs(got["count"] - ref["list"].size) <= int(ref["boundary"].sum())
    assert got["list"].size == cap
    assert np.isin(got["list"], np.flatnonzero(ref["occupied"] | ref["boundary"])).all()


def test_host_buffer_path_equals_device_path():
    sc = S.scene_64cube_4cam(seed=2)
    dev = gpu_reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    occ = np.empty(sc.grid.n_voxels, np.float32)
    lst = np.empty(sc.grid.n_voxels, np.uint32)
    cnt = np.zeros(1, np.uint32)
    st = psfs.psfs_reconstruct_host(rec.handle, np.ascontiguousarray(sc.images), occ, lst, lst.size, cnt)
    assert st == psfs.PSFS_OK
    np.testing.assert_array_equal(occ.astype(np.float64), dev["occ"])
    np.testing.assert_array_equal(np.sort(lst[:cnt[0]]), dev["list"])
    # overflow through the host path
    st = psfs.psfs_reconstruct_host(rec.handle, np.ascontiguousarray(sc.images), None, lst, 10, cnt)
    assert st == psfs.PSFS_ERR_CAPACITY and cnt[0] == dev["count"]
    rec.close()


@pytest.mark.parametrize("dtype,bound", [("f16", 5e-3), ("bf16", 5e-2)])
def test_reduced_precision_maps_error_reported(dtype, bound):
    """FP16 / BF16 maps: error against FP64 is reported; a loose sanity bound
    guards against a broken conversion."""
    sc = S.scene_64cube_4cam(seed=0)
    ref = oracle.reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params)
    got = gpu_reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params, map_dtype=dtype)
    rep = compare(got, ref, exact=False)
    print(dtype, rep)
    assert rep["max_abs_err"] < bound
    assert rep["set_diff"] < 0.02 * max(1, ref["list"].size)


def test_background_validation_and_not_ready():
    sc = S.scene_64cube_4cam(seed=0)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    occ, lst, cnt = rec.alloc_outputs()
    with pytest.raises(psfs.PsfsError) as e:
        psfs.psfs_reconstruct(rec.handle, to_dev(sc.images), occ, lst, rec.capacity, cnt)
    assert e.value.status == psfs.PSFS_ERR_NOT_READY
    bad = sc.var.copy()
    bad[1, 2, 3, 1] = 0.0
    with pytest.raises(psfs.PsfsError) as e:
        rec.set_background(to_dev(sc.mean), to_dev(bad))
    assert e.value.status == psfs.PSFS_ERR_INVALID_ARG
    bad = sc.mean.copy()
    bad[0, 0, 0, 0] = np.nan
    with pytest.raises(psfs.PsfsError):
        rec.set_background(to_dev(bad), to_dev(sc.var))
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    # misaligned device pointer
    img = to_dev(sc.images.ravel())
    with pytest.raises(psfs.PsfsError) as e:
        psfs.psfs_reconstruct(rec.handle, img.data_ptr() + 1, occ, lst, rec.capacity, cnt)
    assert e.value.status == psfs.PSFS_ERR_INVALID_ARG
    rec.close()


def test_cameras_inside_the_grid():
    """An 8 m grid that contains the camera ring: voxels behind, beside and in
    front of every camera (tiles that straddle the camera plane take the
    checked path, tiles wholly behind are skipped)."""
    sc = S.make_scene(seed=14, grid_n=48, cube_side=8.0, n_cams=4, width=160, height=120, focal=150.0)
    got = gpu_reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params)
    ref = oracle.reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params)
    compare(got, ref)
    assert (ref["n_seen"] == 0).any() and (ref["n_seen"] == 4).any()


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_reduced_precision_maps_match_oracle_on_stored_maps(dtype):
    """Storage only: the kernel must sum the 16-bit log ratios it stored
    exactly as the FP64 fusion of the same stored values does.  The stored
    maps are read back from the library (psfs_get_log_ratio); the oracle fuses
    SLM values, so with the rates P_D = 1, P_FA = 0 (where g = log(2 s), Eq. 6-9
    verbatim) each stored g is handed to it as s = e^g / 2.  What remains
    between the two is FP32 summation against FP64 products: the 1e-5 bound."""
    sc = S.make_scene(seed=15, grid_n=40, cube_side=2.0, n_cams=4, width=160, height=120, focal=150.0)
    p = S.Params(p_detect=1.0, p_false_alarm=0.0)
    rec = psfs.Reconstructor(sc.grid, sc.cams, p, map_dtype=dtype)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    img = to_dev(sc.images)
    g16 = rec.log_ratio(img)
    assert g16.dtype == (torch.float16 if dtype == "f16" else torch.bfloat16)
    occ, lst, cnt = rec.reconstruct(img)
    assert rec.sync() == psfs.PSFS_OK
    g = g16.double().cpu().numpy()
    s_equiv = np.exp(g) / 2.0
    ref = oracle.fuse(sc.grid, sc.cams, s_equiv, p)
    got = {"occ": occ.cpu().numpy().ravel().astype(np.float64), "count": int(cnt.item()),
           "list": psfs.voxel_list(lst, cnt, rec.capacity).numpy(), "status": 0}
    rep = compare(got, ref)   # the FP32 tolerances: occupancy within 1e-5, sets exact
    print(dtype, rep)
    # the stored values are what the FP32 likelihood rounds to the storage type
    rec32 = psfs.Reconstructor(sc.grid, sc.cams, p)
    rec32.set_background(to_dev(sc.mean), to_dev(sc.var))
    g32 = rec32.log_ratio(img)
    assert torch.equal(g32.to(g16.dtype), g16)
    rec32.close()
    rec.close()


def test_fuse_tile_shapes_give_identical_results_and_autotune():
    """Every supported tile shape sums the same cameras in the same order, so
    occupancy and voxel set are bit-identical; the autotuner picks one of them."""
    sc = S.make_scene(seed=8, grid_n=48, cube_side=2.0, n_cams=5, width=200, height=150, focal=190.0)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    img = to_dev(sc.images)
    results = []
    for cfg in psfs.FUSE_CONFIGS + [(lx, 4, tz, 0) for lx in (8, 16, 32) for tz in (2, 4)]:
        psfs.psfs_set_fuse_config(rec.handle, *cfg)
        assert psfs.psfs_get_fuse_config(rec.handle) == cfg
        occ, lst, cnt = rec.reconstruct(img)
        assert rec.sync() == psfs.PSFS_OK
        results.append((occ.cpu().numpy(), psfs.voxel_list(lst, cnt, rec.capacity).numpy()))
    for occ, lst in results[1:]:
        np.testing.assert_array_equal(occ, results[0][0])
        np.testing.assert_array_equal(lst, results[0][1])
    best = psfs.psfs_autotune(rec.handle, img, reps=2)
    # a frame-group configuration of the sequence path may bring voxels_z = 2 or 4
    assert best in psfs.FUSE_CONFIGS or (best[2] in (2, 4) and best[3] == 0)
    assert psfs.psfs_get_fuse_config(rec.handle) == best
    occ, lst, cnt = rec.reconstruct(img)
    assert rec.sync() == psfs.PSFS_OK
    np.testing.assert_array_equal(occ.cpu().numpy(), results[0][0])
    with pytest.raises(psfs.PsfsError):
        psfs.psfs_set_fuse_config(rec.handle, 12, 4, 8, 0)
    with pytest.raises(psfs.PsfsError):
        psfs.psfs_set_fuse_config(rec.handle, 8, 4, 4, 1)   # the staged kernel has no voxels_z = 4
    rec.close()


def test_sequence_equals_frame_by_frame():
    """psfs_reconstruct_sequence (two streams, double-buffered maps) gives the
    same occupancy bits and voxel sets as one psfs_reconstruct per frame."""
    sc = S.make_scene(seed=16, grid_n=48, cube_side=2.0, n_cams=4, width=160, height=120, focal=150.0,
                      n_frames=5, walking=True)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    imgs = to_dev(sc.images)
    F, V = imgs.shape[0], sc.grid.n_voxels
    cap = V
    occ = torch.empty((F, V), dtype=torch.float32, device="cuda")
    lists = torch.empty((F, cap), dtype=torch.int32, device="cuda")
    counts = torch.zeros((F,), dtype=torch.int32, device="cuda")
    for lk, l2 in ((1, False), (2, True), (4, False)):
        psfs.psfs_set_background_l2(rec.handle, l2)
        cfg = psfs.psfs_get_fuse_config(rec.handle)
        psfs.psfs_set_fuse_config(rec.handle, *cfg, seq_likelihood_ctas=lk)
        psfs.psfs_reconstruct_sequence(rec.handle, F, imgs, occ, lists, cap, counts)
        assert rec.sync() == psfs.PSFS_OK
        for f in range(F):
            o1, l1, c1 = rec.reconstruct(imgs[f])
            assert rec.sync() == psfs.PSFS_OK
            np.testing.assert_array_equal(occ[f].cpu().numpy(), o1.cpu().numpy().ravel())
            assert int(counts[f]) == int(c1.item())
            np.testing.assert_array_equal(psfs.voxel_list(lists[f], counts[f:f + 1], cap).numpy(),
                                          psfs.voxel_list(l1, c1, rec.capacity).numpy())
    rec.close()


@pytest.mark.slow
@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
def test_256cube_16cam_1280x720_two_bodies(dtype):
    """Full-size 256^3 x 16 cameras x 1280x720, two bodies (one partly
    occluding the other): FP32 maps meet the parity tolerances; FP16 / BF16
    maps report their error against FP64 (max, mean |docc| and the
    occupied-set Hamming distance) under loose sanity bounds."""
    sc = S.scene_256cube_16cam(seed=2)
    ref = oracle.reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params)
    got = gpu_reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params, map_dtype=dtype)
    rep = compare(got, ref, exact=(dtype == "f32"))
    print(dtype, rep)
    assert ref["list"].size > 50000
    if dtype != "f32":
        assert rep["max_abs_err"] < (5e-3 if dtype == "f16" else 5e-2)
        assert rep["set_diff"] < 0.01 * ref["list"].size
