"""psfs_reconstruct_noalloc: the allocation-free entry point, for callers
that cannot call cudaMalloc (hosts that own all device memory, loops that
must not pay an allocation's implicit synchronisation).  Its scratch is a
fixed device array shared by all calls.

Checked through the C ABI against psfs_reconstruct on the same inputs, on two
calls in a row with different frames (the second call must not see the
first one's scratch), within the parity tolerance of the other GPU tests.
This file is collected last so that a failure here stops a run only after
every other test has run."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1311_6811_gb300 import psfs  # noqa: E402
from synth import scene as S  # noqa: E402
from tests.gpu_helpers import OCC_TOL, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    psfs.load()


def _reference(sc, frame):
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    occ, lst, cnt = rec.reconstruct(to_dev(frame))
    assert rec.sync() == psfs.PSFS_OK
    out = occ.cpu().numpy().ravel(), psfs.voxel_list(lst, cnt, rec.capacity).numpy(), int(cnt.item())
    rec.close()
    return out


def test_noalloc_matches_reconstruct_on_two_calls():
    sc = S.make_scene(seed=31, grid_n=48, cube_side=2.0, n_cams=5, width=200, height=150, focal=190.0,
                      n_frames=2, walking=True)
    mean, var = to_dev(sc.mean), to_dev(sc.var)
    V = sc.grid.n_voxels
    occ = torch.empty(V, dtype=torch.float32, device="cuda")
    lst = torch.empty(V, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    for f in range(2):
        ref_occ, ref_list, ref_count = _reference(sc, sc.images[f])
        psfs.psfs_reconstruct_noalloc(sc.grid, sc.cams, sc.params, mean, var, to_dev(sc.images[f]), occ, lst,
                                      V, cnt)
        torch.cuda.synchronize()
        got = occ.cpu().numpy()
        assert np.max(np.abs(got.astype(np.float64) - ref_occ)) <= OCC_TOL
        assert int(cnt.item()) == ref_count and ref_count > 0
        np.testing.assert_array_equal(psfs.voxel_list(lst, cnt, V).numpy(), ref_list)


def test_noalloc_rejects_frames_beyond_its_scratch():
    rng = np.random.default_rng(0)
    cams = S.ring_cameras(rng, 8, 1280, 720, 1200.0, (0.0, 0.0, 1.0))   # 7.4 M pixels > 4 M
    grid = S.Grid(8, 8, 8, (-0.2, -0.2, 0.8), 0.05)
    small = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(psfs.PsfsError) as e:
        psfs.psfs_reconstruct_noalloc(grid, cams, S.Params(), small, small,
                                      torch.zeros(16, dtype=torch.uint8, device="cuda"), small,
                                      torch.zeros(16, dtype=torch.int32, device="cuda"), 16,
                                      torch.zeros(1, dtype=torch.int32, device="cuda"))
    assert e.value.status == psfs.PSFS_ERR_INVALID_ARG
