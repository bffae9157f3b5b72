"""Frame groups of the sequence path: F frames per likelihood launch (one
pass over the background) and per fusion launch (one projection per voxel
and camera, one vector gather per 32-byte pixel record: 8 FP32 or 16
16-bit frames, one fusion launch per plane of records; or 64-byte records
read by two lanes per voxel).  Each frame's occupancy,
count and voxel set must be bit-identical to one psfs_reconstruct per frame
with the same tile shape, for every group size, map type and a frame count
that leaves trailing frames outside the last group; one group's frame is also
checked against the FP64 oracle directly."""

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


def _scene(n_frames):
    return S.make_scene(seed=21, grid_n=48, cube_side=2.0, n_cams=4, width=160, height=120, focal=150.0,
                        n_frames=n_frames, walking=True)


def _run_sequence(rec, imgs, cap):
    F, V = imgs.shape[0], rec.n_voxels
    occ = torch.full((F, V), -1.0, dtype=torch.float32, device="cuda")
    lists = torch.empty((F, cap), dtype=torch.int32, device="cuda")
    counts = torch.full((F,), 12345, dtype=torch.int32, device="cuda")
    psfs.psfs_reconstruct_sequence(rec.handle, F, imgs, occ, lists, cap, counts)
    assert rec.sync() == psfs.PSFS_OK
    return occ, lists, counts


def _assert_frame_by_frame(rec, imgs, occ, lists, counts, cap):
    for f in range(imgs.shape[0]):
        o1, l1, c1 = rec.reconstruct(imgs[f])
        assert rec.sync() == psfs.PSFS_OK
        np.testing.assert_array_equal(occ[f].cpu().numpy(), o1.cpu().numpy().ravel(), err_msg=f"frame {f}")
        assert int(counts[f]) == int(c1.item()), f
        np.testing.assert_array_equal(psfs.voxel_list(lists[f], counts[f:f + 1], cap).numpy(),
                                      psfs.voxel_list(l1, c1, rec.capacity).numpy())


def _plane_frames(group, dtype):
    """Frames per 32-byte pixel record of the group maps."""
    return min(group, 8 if dtype == "f32" else 16)


def _shape_ok(group, tz, dtype):
    p = _plane_frames(group, dtype)
    return tz in (2, 4) or (tz == 8 and p <= 8) or (tz == 16 and p <= 4)


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("group,tz", [(2, 16), (4, 2), (4, 4), (4, 8), (4, 16), (8, 2), (8, 4), (8, 8), (16, 2),
                                      (16, 4), (16, 8)])
def test_groups_equal_frame_by_frame(group, tz, dtype):
    """33 frames: whole groups, then the trailing frames in smaller groups
    and single frames.  16 FP32 frames are two planes of 8-frame records."""
    if not _shape_ok(group, tz, dtype):
        pytest.skip("tile height not supported for this record size")
    sc = _scene(33)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params, map_dtype=dtype)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    imgs = to_dev(sc.images)
    cap = rec.n_voxels
    for lx in (8, 16):
        psfs.psfs_set_fuse_config(rec.handle, lx, 4, tz, 0, 2, group, 0, 0, 32)
        assert psfs.psfs_get_fuse_config(rec.handle, full=True) == (lx, 4, tz, 0, 2, group, lx, tz, 32)
        occ, lists, counts = _run_sequence(rec, imgs, cap)
        _assert_frame_by_frame(rec, imgs, occ, lists, counts, cap)
    rec.close()


@pytest.mark.parametrize("dtype", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("tz", [2, 4, 8])
def test_groups_of_32_equal_frame_by_frame(tz, dtype):
    """61 frames: one group of 32 frames (four planes of 8-frame records for
    FP32 maps, two of 16 for 16-bit maps), then groups of 16, 8 and 4 and one
    single frame."""
    if not _shape_ok(32, tz, dtype):
        pytest.skip("tile height not supported for this record size")
    sc = _scene(61)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params, map_dtype=dtype)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    imgs = to_dev(sc.images)
    cap = rec.n_voxels
    for lx in (8, 16):
        psfs.psfs_set_fuse_config(rec.handle, lx, 4, tz, 0, 2, 32, 0, 0, 32)
        assert psfs.psfs_get_fuse_config(rec.handle, full=True) == (lx, 4, tz, 0, 2, 32, lx, tz, 32)
        occ, lists, counts = _run_sequence(rec, imgs, cap)
        _assert_frame_by_frame(rec, imgs, occ, lists, counts, cap)
    rec.close()


def test_group_of_32_ragged_grid_and_views():
    """Grid 37 x 29 x 24 (ragged tiles along x, y and z), 3 cameras of 104 x 80
    whose views miss part of the grid, 57 frames: groups of 32, 16 and 8
    and a single frame (the pixel count, 24960, is not a multiple of the
    likelihood's 256-pixel chunks); also the likelihood grid sizes of the
    32-frame group."""
    grid = S.Grid(37, 29, 24, (-0.9, -0.7, 0.1), 0.05)
    sc = S.make_scene(seed=23, grid_n=48, cube_side=2.0, n_cams=3, width=104, height=80, focal=95.0,
                      n_frames=57, walking=True)
    rec = psfs.Reconstructor(grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    imgs = to_dev(sc.images)
    for tz, lk in ((4, 1), (8, 2), (8, 3)):
        psfs.psfs_set_fuse_config(rec.handle, 8, 4, tz, 0, lk, 32, 0, 0, 32)
        occ, lists, counts = _run_sequence(rec, imgs, rec.n_voxels)
        _assert_frame_by_frame(rec, imgs, occ, lists, counts, rec.n_voxels)
    rec.close()


def test_group_of_32_matches_oracle_and_capacity():
    """56 frames (units of 32, 16 and 8): frames 0, 17 and 31 of the group of
    32 and frame 55 against the FP64 oracle; then a capacity below every
    frame's count: full counts, `capacity` valid entries per frame,
    PSFS_ERR_CAPACITY."""
    n = 56
    sc = _scene(n)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    imgs = to_dev(sc.images)
    psfs.psfs_set_fuse_config(rec.handle, 8, 4, 4, 0, 2, 32)
    occ, lists, counts = _run_sequence(rec, imgs, rec.n_voxels)
    for f in (0, 17, 31, 55):
        got = {"occ": occ[f].cpu().numpy().astype(np.float64), "count": int(counts[f]) & 0xFFFFFFFF,
               "list": psfs.voxel_list(lists[f], counts[f:f + 1], rec.n_voxels).numpy(), "status": psfs.PSFS_OK}
        ref = oracle.reconstruct(sc.grid, sc.cams, sc.images[f], sc.mean, sc.var, sc.params)
        assert ref["list"].size > 500
        print(compare(got, ref))
    full = [int(c) for c in counts]
    cap = min(full) // 2
    V = rec.n_voxels
    occ2 = torch.empty((n, V), dtype=torch.float32, device="cuda")
    counts2 = torch.zeros((n,), dtype=torch.int32, device="cuda")
    lists_flat = torch.full((n * cap,), -1, dtype=torch.int32, device="cuda")
    psfs.psfs_reconstruct_sequence(rec.handle, n, imgs, occ2, lists_flat, cap, counts2)
    assert rec.sync() == psfs.PSFS_ERR_CAPACITY
    assert [int(c) for c in counts2] == full
    lf = lists_flat.view(n, cap).cpu().numpy()
    assert (lf >= 0).all() and (lf < V).all()
    for f in range(n):
        assert np.isin(lf[f], psfs.voxel_list(lists[f], counts[f:f + 1], V).numpy()).all()
    rec.close()


@pytest.mark.parametrize("dtype,group,tz", [("f32", 16, 2), ("f32", 16, 4), ("f32", 32, 2), ("f32", 32, 4),
                                            ("f16", 32, 2), ("f16", 32, 4), ("bf16", 32, 2)])
def test_64_byte_records_equal_frame_by_frame(dtype, group, tz):
    """64-byte pixel records (16 FP32 or 32 16-bit frames per plane, two
    lanes per voxel, one 32-byte half each): 61 frames run as groups of
    `group` frames and the trailing units (whose smaller records take the
    one-lane kernel), every frame bit-identical to one frame per call, with
    both lanes_x."""
    sc = _scene(61)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params, map_dtype=dtype)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    imgs = to_dev(sc.images)
    cap = rec.n_voxels
    for lx in (8, 16):
        psfs.psfs_set_fuse_config(rec.handle, lx, 4, tz, 0, 2, group, 0, 0, 64)
        assert psfs.psfs_get_fuse_config(rec.handle, full=True) == (lx, 4, tz, 0, 2, group, lx, tz, 64)
        occ, lists, counts = _run_sequence(rec, imgs, cap)
        _assert_frame_by_frame(rec, imgs, occ, lists, counts, cap)
    rec.close()


def test_64_byte_records_ragged_grid_oracle_and_capacity():
    """64-byte records on the ragged 37 x 29 x 24 grid with 3 cameras whose
    views miss part of it (57 frames: groups of 32 and 16, then 8 and 1);
    one frame of the 32-frame group against the FP64 oracle; then a capacity
    below every frame's count (the two half-warps' frames share the CTA's
    per-frame reservations): full counts, valid entries, PSFS_ERR_CAPACITY."""
    grid = S.Grid(37, 29, 24, (-0.9, -0.7, 0.1), 0.05)
    sc = S.make_scene(seed=23, grid_n=48, cube_side=2.0, n_cams=3, width=104, height=80, focal=95.0,
                      n_frames=57, walking=True)
    rec = psfs.Reconstructor(grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    imgs = to_dev(sc.images)
    n, V = imgs.shape[0], rec.n_voxels
    for tz, lk in ((2, 1), (4, 3)):
        psfs.psfs_set_fuse_config(rec.handle, 8, 4, tz, 0, lk, 32, 0, 0, 64)
        occ, lists, counts = _run_sequence(rec, imgs, V)
        _assert_frame_by_frame(rec, imgs, occ, lists, counts, V)
    f = 21
    got = {"occ": occ[f].cpu().numpy().astype(np.float64), "count": int(counts[f]) & 0xFFFFFFFF,
           "list": psfs.voxel_list(lists[f], counts[f:f + 1], V).numpy(), "status": psfs.PSFS_OK}
    ref = oracle.reconstruct(grid, sc.cams, sc.images[f], sc.mean, sc.var, sc.params)
    assert ref["list"].size > 100
    print(compare(got, ref))
    full = [int(c) for c in counts]
    cap = min(full) // 2
    occ2 = torch.empty((n, V), dtype=torch.float32, device="cuda")
    counts2 = torch.zeros((n,), dtype=torch.int32, device="cuda")
    lists_flat = torch.full((n * cap,), -1, dtype=torch.int32, device="cuda")
    psfs.psfs_reconstruct_sequence(rec.handle, n, imgs, occ2, lists_flat, cap, counts2)
    assert rec.sync() == psfs.PSFS_ERR_CAPACITY
    assert [int(c) for c in counts2] == full
    assert torch.equal(occ2, occ)
    lf = lists_flat.view(n, cap).cpu().numpy()
    assert (lf >= 0).all() and (lf < V).all()
    for f in range(n):
        assert np.isin(lf[f], psfs.voxel_list(lists[f], counts[f:f + 1], V).numpy()).all()
        assert np.unique(lf[f]).size == cap
    rec.close()


def test_64_byte_record_validation():
    """Record sizes 32 and 64 only; with 64-byte records a lane holds 8 FP32
    (16 16-bit) frames of a 16-frame (32-frame) plane: voxels_z 2 or 4; 0
    keeps the current record size; groups whose frames fit 32 bytes keep
    any tile height."""
    sc = _scene(2)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    for bad in [(8, 4, 4, 0, 0, 32, 0, 0, 48), (8, 4, 4, 0, 0, 32, 0, 0, 128), (8, 4, 8, 0, 0, 16, 0, 0, 64),
                (8, 4, 8, 0, 0, 32, 0, 0, 64), (8, 4, 4, 0, 0, 32, 0, 0, -32)]:
        with pytest.raises(psfs.PsfsError):
            psfs.psfs_set_fuse_config(rec.handle, *bad)
    psfs.psfs_set_fuse_config(rec.handle, 8, 4, 8, 0, 0, 8, 0, 0, 64)    # 8 FP32 frames fit 32 bytes
    psfs.psfs_set_fuse_config(rec.handle, 8, 4, 4, 0, 0, 32, 0, 0, 0)
    assert psfs.psfs_get_fuse_config(rec.handle, full=True)[8] == 64
    psfs.psfs_set_fuse_config(rec.handle, 8, 4, 8, 0, 0, 32, 0, 0, 32)
    assert psfs.psfs_get_fuse_config(rec.handle, full=True)[5:] == (32, 8, 8, 32)
    rec.close()


@pytest.mark.parametrize("lk", [1, 2, 3, 4])
def test_group_likelihood_grid_sizes(lk):
    """Every likelihood grid size (CTAs per SM, clamped by shared memory)."""
    sc = _scene(8)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    imgs = to_dev(sc.images)
    psfs.psfs_set_fuse_config(rec.handle, 8, 4, 8, 0, lk, 4)
    occ, lists, counts = _run_sequence(rec, imgs, rec.n_voxels)
    _assert_frame_by_frame(rec, imgs, occ, lists, counts, rec.n_voxels)
    rec.close()


def test_group_ragged_grid():
    """Grid 37 x 29 x 24 (ragged along x and y for every tile shape, along z
    for voxels_z = 16), 3 cameras of 104 x 80 (some voxels outside some
    views), 6 frames in groups of 4 plus 2 single frames."""
    grid = S.Grid(37, 29, 24, (-0.9, -0.7, 0.1), 0.05)
    sc = S.make_scene(seed=22, grid_n=48, cube_side=2.0, n_cams=3, width=104, height=80, focal=95.0,
                      n_frames=6, walking=True)
    rec = psfs.Reconstructor(grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    imgs = to_dev(sc.images)
    for tz in (8, 16):
        psfs.psfs_set_fuse_config(rec.handle, 8, 4, tz, 0, 2, 4)
        occ, lists, counts = _run_sequence(rec, imgs, rec.n_voxels)
        _assert_frame_by_frame(rec, imgs, occ, lists, counts, rec.n_voxels)
    rec.close()


def test_group_frame_matches_oracle():
    """Frame 2 of a group of 4, against the FP64 oracle at the FP32 tolerances."""
    sc = _scene(4)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    imgs = to_dev(sc.images)
    psfs.psfs_set_fuse_config(rec.handle, 8, 4, 8, 0, 2, 4)
    occ, lists, counts = _run_sequence(rec, imgs, rec.n_voxels)
    f = 2
    got = {"occ": occ[f].cpu().numpy().astype(np.float64), "count": int(counts[f]) & 0xFFFFFFFF,
           "list": psfs.voxel_list(lists[f], counts[f:f + 1], rec.n_voxels).numpy(), "status": psfs.PSFS_OK}
    ref = oracle.reconstruct(sc.grid, sc.cams, sc.images[f], sc.mean, sc.var, sc.params)
    rep = compare(got, ref)
    assert ref["list"].size > 500
    print(rep)
    rec.close()


def test_group_capacity_overflow_per_frame():
    """A capacity below the occupied count: every frame's count is still the
    full count, only `capacity` entries are written, and the overflow is
    reported by psfs_sync."""
    sc = _scene(4)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    imgs = to_dev(sc.images)
    full = []
    for f in range(4):
        _, _, c1 = rec.reconstruct(imgs[f])
        assert rec.sync() == psfs.PSFS_OK
        full.append(int(c1.item()))
    cap = min(full) // 2
    psfs.psfs_set_fuse_config(rec.handle, 8, 4, 8, 0, 2, 4)
    V = rec.n_voxels
    occ = torch.empty((4, V), dtype=torch.float32, device="cuda")
    counts = torch.zeros((4,), dtype=torch.int32, device="cuda")
    lists_flat = torch.full((4 * cap,), -1, dtype=torch.int32, device="cuda")
    psfs.psfs_reconstruct_sequence(rec.handle, 4, imgs, occ, lists_flat, cap, counts)
    assert rec.sync() == psfs.PSFS_ERR_CAPACITY
    assert [int(c) for c in counts] == full
    lf = lists_flat.view(4, cap).cpu().numpy()
    assert (lf >= 0).all() and (lf < V).all()
    rec.close()


def test_backward_tile_shapes_identical():
    """The adjoint's voxel pass runs with the handle's tile shape, voxels_z = 4
    included: gradients are bit-identical across shapes."""
    sc = _scene(2)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    img = to_dev(sc.images[0])
    V = rec.n_voxels
    n_pix = img.numel() // 3
    g = torch.Generator().manual_seed(5)
    d_occ = torch.randn(V, generator=g).cuda()
    outs = []
    for cfg in [(8, 4, 16, 0), (8, 4, 4, 0), (16, 4, 4, 0), (32, 4, 4, 0)]:
        psfs.psfs_set_fuse_config(rec.handle, *cfg)
        d_slm = torch.empty(n_pix, device="cuda")
        d_mean = torch.empty(n_pix * 3, device="cuda")
        d_var = torch.empty(n_pix * 3, device="cuda")
        psfs.psfs_backward(rec.handle, img, d_occ, d_slm, d_mean, d_var)
        assert rec.sync() == psfs.PSFS_OK
        outs.append([t.cpu().numpy() for t in (d_slm, d_mean, d_var)])
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            np.testing.assert_array_equal(a, b)
    rec.close()


def test_group_config_validation():
    sc = _scene(2)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    for bad in [(8, 4, 8, 0, 0, 3), (8, 4, 16, 0, 0, 8), (8, 4, 8, 1, 0, 4), (32, 4, 8, 0, 0, 2),
                (8, 4, 8, 0, 0, -1), (32, 4, 4, 0, 0, 4), (8, 4, 16, 0, 0, 16), (8, 4, 16, 0, 0, 32),
                (32, 4, 4, 0, 0, 32), (8, 4, 8, 1, 0, 32), (8, 4, 4, 0, 0, 64)]:
        with pytest.raises(psfs.PsfsError):
            psfs.psfs_set_fuse_config(rec.handle, *bad)
    # FP32 records hold 8 frames: 16 and 32 frames with voxels_z 8 are fine
    for good in [(8, 4, 8, 0, 0, 16, 0, 0, 32), (16, 4, 8, 0, 0, 32, 0, 0, 32)]:
        psfs.psfs_set_fuse_config(rec.handle, *good)
    # 16-bit records hold 16 frames: voxels_z 4 only from 16 frames on
    rec16 = psfs.Reconstructor(sc.grid, sc.cams, sc.params, map_dtype="f16")
    for bad in [(8, 4, 8, 0, 0, 16), (8, 4, 8, 0, 0, 32)]:
        with pytest.raises(psfs.PsfsError):
            psfs.psfs_set_fuse_config(rec16.handle, *bad)
    psfs.psfs_set_fuse_config(rec16.handle, 8, 4, 8, 0, 0, 8, 0, 0, 32)
    psfs.psfs_set_fuse_config(rec16.handle, 8, 4, 4, 0, 0, 32)
    rec16.close()
    psfs.psfs_set_fuse_config(rec.handle, 8, 4, 8, 0, 0, 4)
    assert psfs.psfs_get_fuse_config(rec.handle, full=True)[5] == 4
    # 0 keeps the current group size
    psfs.psfs_set_fuse_config(rec.handle, 16, 4, 8, 0, 0, 0)
    assert psfs.psfs_get_fuse_config(rec.handle, full=True)[5] == 4
    rec.close()


def test_autotune_picks_a_sequence_configuration():
    sc = _scene(2)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    psfs.psfs_autotune(rec.handle, to_dev(sc.images[0]), reps=1)
    cfg = psfs.psfs_get_fuse_config(rec.handle, full=True)
    assert cfg[5] in (1, 2, 4, 8, 16, 32) and 1 <= cfg[4] <= 4
    # the one-frame shape is one of the one-frame candidates; the sequence
    # path's shape supports its group size
    assert cfg[:4] in psfs.FUSE_CONFIGS
    assert cfg[5] == 1 or cfg[7] in (2, 4, 8, 16)
    assert rec.sync() == psfs.PSFS_OK
    rec.close()


def test_autotune_cache_file(tmp_path):
    """The autotuner's choice saved to a file, forgotten, loaded again: a
    handle created afterwards for the same kind of rig starts with it."""
    sc = _scene(2)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    psfs.psfs_autotune(rec.handle, to_dev(sc.images[0]), reps=1)
    tuned = psfs.psfs_get_fuse_config(rec.handle, full=True)
    rec.close()
    path = str(tmp_path / "tune.txt")
    psfs.psfs_tune_cache_save(path)
    psfs.psfs_tune_cache_clear()
    fresh = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    default = psfs.psfs_get_fuse_config(fresh.handle, full=True)
    fresh.close()
    psfs.psfs_tune_cache_load(path)
    assert psfs.psfs_tune_cache_entries() >= 1
    again = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    assert psfs.psfs_get_fuse_config(again.handle, full=True) == tuned
    again.close()
    print("tuned", tuned, "default", default)


def test_sequence_with_its_own_tile_shape():
    """A sequence tile shape of its own (seq_lanes_x, seq_voxels_z) while one
    frame per call keeps another shape: both give the same bits."""
    sc = _scene(5)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    imgs = to_dev(sc.images)
    F, V = imgs.shape[0], rec.n_voxels
    psfs.psfs_set_fuse_config(rec.handle, 32, 4, 16, 0, 2, 4, 16, 2, 32)
    assert psfs.psfs_get_fuse_config(rec.handle, full=True) == (32, 4, 16, 0, 2, 4, 16, 2, 32)
    occ = torch.empty((F, V), device="cuda")
    lst = torch.empty((F, V), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(F, dtype=torch.int32, device="cuda")
    psfs.psfs_reconstruct_sequence(rec.handle, F, imgs, occ, lst, V, cnt)
    assert rec.sync() == psfs.PSFS_OK
    for f in range(F):
        o1, _, c1 = rec.reconstruct(imgs[f])
        assert rec.sync() == psfs.PSFS_OK
        assert torch.equal(o1.view(-1), occ[f]) and int(c1.item()) == int(cnt[f])
    # back to one shape for both
    psfs.psfs_set_fuse_config(rec.handle, 8, 4, 4, 0, 2, 4, 0, 0, 32)
    assert psfs.psfs_get_fuse_config(rec.handle, full=True) == (8, 4, 4, 0, 2, 4, 8, 4, 32)
    with pytest.raises(psfs.PsfsError):
        psfs.psfs_set_fuse_config(rec.handle, 8, 4, 4, 0, 2, 4, 12, 2)   # no such sequence shape
    rec.close()


@pytest.mark.parametrize("pinned", [True, False])
def test_sequence_host_equals_device(pinned):
    """psfs_reconstruct_sequence_host (copies in and out overlapping the
    kernels, three staging slots of 4 frames reused across 18 chunks, the
    last of 2 frames) gives the device sequence's occupancy, counts and
    voxel sets."""
    n = 70
    sc = _scene(n)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    psfs.psfs_set_fuse_config(rec.handle, 8, 4, 8, 0, 2, 2)   # groups of 2
    V, cap = rec.n_voxels, rec.n_voxels // 4
    occ_d, lists_d, counts_d = _run_sequence(rec, to_dev(sc.images), cap)

    def host(shape, dtype):
        t = torch.full(shape, -7, dtype=dtype)
        return t.pin_memory() if pinned else t

    imgs_h = torch.from_numpy(np.ascontiguousarray(sc.images))
    imgs_h = imgs_h.pin_memory() if pinned else imgs_h
    occ_h, lists_h, counts_h = host((n, V), torch.float32), host((n, cap), torch.int32), host((n,), torch.int32)
    assert psfs.psfs_reconstruct_sequence_host(rec.handle, n, imgs_h, occ_h, lists_h, cap, counts_h) == psfs.PSFS_OK
    np.testing.assert_array_equal(occ_h.numpy(), occ_d.cpu().numpy())
    np.testing.assert_array_equal(counts_h.numpy(), counts_d.cpu().numpy())
    for f in range(n):
        c = int(counts_h[f])
        np.testing.assert_array_equal(np.sort(lists_h[f, :c].numpy()),
                                      psfs.voxel_list(lists_d[f], counts_d[f:f + 1], cap).numpy())
        assert (lists_h[f, c:] == -7).all()   # nothing past the count is written
    # without the occupancy copy, and with a capacity below the counts
    small = int(counts_h.min()) // 2
    lists2 = host((n, small), torch.int32)
    counts2 = host((n,), torch.int32)
    st = psfs.psfs_reconstruct_sequence_host(rec.handle, n, imgs_h, None, lists2, small, counts2)
    assert st == psfs.PSFS_ERR_CAPACITY
    np.testing.assert_array_equal(counts2.numpy(), counts_h.numpy())
    l2 = lists2.numpy()
    assert ((l2 >= 0) & (l2 < V)).all()
    assert rec.sync() == psfs.PSFS_OK   # the capacity bit was cleared by the host call
    rec.close()
