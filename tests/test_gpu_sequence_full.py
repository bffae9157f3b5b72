"""The benchmarked launch at full size: psfs_reconstruct_sequence on the
128^3 x 8 cameras x 640x480 walking sequence, in frame groups of 32 with the
background held in L2, exactly as bench.py times it.

36 frames make one 32-frame group (four fusion planes of 8 FP32 frames, two
of 16 half-precision frames) and a trailing 4-frame group.  Every frame must
be bit-identical to psfs_reconstruct of that frame alone (occupancy bits,
count, voxel set), and frames 0, 17, 33 and 35 (first group: its first and a
middle frame; the tail group: its first and last frame) must meet the
parity tolerances against the FP64 oracle (FP32 maps), or report their error
against it (FP16 maps)."""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1311_6811_gb300 import psfs  # noqa: E402
from synth import scene as S  # noqa: E402
from tests.gpu_helpers import compare, to_dev  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N_FRAMES = 36
ORACLE_FRAMES = (0, 17, 33, 35)


@pytest.fixture(scope="module")
def seq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    psfs.load()
    workers = max(1, min(8, os.cpu_count() or 1))
    return S.scene_128cube_8cam(seed=1, n_frames=N_FRAMES, workers=workers)


@pytest.mark.parametrize("dtype,lanes_x,voxels_z,rec_bytes", [("f32", 8, 4, 32), ("f32", 16, 2, 32), ("f16", 8, 2, 32),
                                                              ("f32", 8, 2, 64), ("f16", 16, 2, 64)])
def test_sequence_groups_of_32_full_size(seq, dtype, lanes_x, voxels_z, rec_bytes):
    sc = seq
    V = sc.grid.n_voxels
    cap = 1 << 17
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params, map_dtype=dtype, stream=stream, capacity=cap)
        rec.set_background(to_dev(sc.mean), to_dev(sc.var))
        imgs = to_dev(sc.images)
        occ = torch.empty((N_FRAMES, V), dtype=torch.float32, device="cuda")
        lists = torch.empty((N_FRAMES, cap), dtype=torch.int32, device="cuda")
        counts = torch.zeros((N_FRAMES,), dtype=torch.int32, device="cuda")
    stream.synchronize()
    h = rec.handle
    psfs.psfs_set_background_l2(h, True)
    # the one-frame reference keeps its own shape; the sequence path gets the
    # shape under test (as the autotuner leaves a handle)
    psfs.psfs_set_fuse_config(h, 8, 4, 16, 0, 2, 32, lanes_x, voxels_z, rec_bytes)
    assert psfs.psfs_get_fuse_config(h, full=True)[5:] == (32, lanes_x, voxels_z, rec_bytes)
    with torch.cuda.stream(stream):
        psfs.psfs_reconstruct_sequence(h, N_FRAMES, imgs, occ, lists, cap, counts)
    assert rec.sync() == psfs.PSFS_OK

    # every frame bit-identical to one frame per call
    with torch.cuda.stream(stream):
        o1, l1, c1 = rec.alloc_outputs()
    for f in range(N_FRAMES):
        with torch.cuda.stream(stream):
            rec.reconstruct(imgs[f], (o1, l1, c1))
        assert rec.sync() == psfs.PSFS_OK
        assert torch.equal(occ[f], o1.view(-1)), f"frame {f}: occupancy bits differ"
        assert int(counts[f]) == int(c1.item()), f"frame {f}: counts differ"
        np.testing.assert_array_equal(psfs.voxel_list(lists[f], counts[f:f + 1], cap).numpy(),
                                      psfs.voxel_list(l1, c1, cap).numpy())

    # sampled frames against the FP64 oracle
    reports = {}
    for f in ORACLE_FRAMES:
        ref = oracle.reconstruct(sc.grid, sc.cams, sc.images[f], sc.mean, sc.var, sc.params)
        got = {"occ": occ[f].cpu().numpy().astype(np.float64), "count": int(counts[f]) & 0xFFFFFFFF,
               "list": psfs.voxel_list(lists[f], counts[f:f + 1], cap).numpy(), "status": psfs.PSFS_OK}
        rep = compare(got, ref, exact=(dtype == "f32"))
        reports[f] = rep
        assert ref["list"].size > 10000
        if dtype != "f32":
            assert rep["max_abs_err"] < 5e-3, rep
            assert rep["set_diff"] < 0.01 * ref["list"].size, rep
    print(dtype, lanes_x, voxels_z,
          {f: (r["max_abs_err"], r["set_diff"], r["set_diff_unexplained"]) for f, r in reports.items()})
    rec.close()
