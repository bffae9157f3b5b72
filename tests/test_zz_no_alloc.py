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
    # raw addresses skip the binding's size checks, so that the library's own
    # limit check is what rejects the call (before any device access)
    with pytest.raises(psfs.PsfsError) as e:
        psfs.psfs_reconstruct_noalloc(grid, cams, S.Params(), small.data_ptr(), small.data_ptr(),
                                      torch.zeros(16, dtype=torch.uint8, device="cuda").data_ptr(),
                                      small.data_ptr(), torch.zeros(16, dtype=torch.int32, device="cuda").data_ptr(),
                                      16, torch.zeros(1, dtype=torch.int32, device="cuda").data_ptr())
    assert e.value.status == psfs.PSFS_ERR_INVALID_ARG
    assert "PSFS_NOALLOC_MAX_PIXELS" in psfs.psfs_last_error_message()
    # through tensors, the binding refuses the undersized buffers itself
    with pytest.raises(ValueError):
        psfs.psfs_reconstruct_noalloc(grid, cams, S.Params(), small, small,
                                      torch.zeros(16, dtype=torch.uint8, device="cuda"), small,
                                      torch.zeros(16, dtype=torch.int32, device="cuda"), 16,
                                      torch.zeros(1, dtype=torch.int32, device="cuda"))


def test_noalloc_overflow_side_stream_and_oracle():
    """A list smaller than the occupied set: count holds the true count and
    the list the first `capacity` entries, all of them occupied voxels.  The
    call is made on a side stream, and the full-capacity result is compared
    with the FP64 oracle at the parity tolerance."""
    import oracle
    from tests.gpu_helpers import compare

    sc = S.make_scene(seed=32, grid_n=40, cube_side=2.0, n_cams=4, width=160, height=120, focal=150.0)
    mean, var, img = to_dev(sc.mean), to_dev(sc.var), to_dev(sc.images)
    V = sc.grid.n_voxels
    occ = torch.empty(V, dtype=torch.float32, device="cuda")
    lst = torch.empty(V, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        psfs.psfs_reconstruct_noalloc(sc.grid, sc.cams, sc.params, mean, var, img, occ, lst, V, cnt, stream=side)
    side.synchronize()
    full = int(cnt.item())
    got = {"occ": occ.cpu().numpy().astype(np.float64), "count": full,
           "list": psfs.voxel_list(lst, cnt, V).numpy(), "status": psfs.PSFS_OK}
    ref = oracle.reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params)
    rep = compare(got, ref)
    assert full > 8, rep
    full_set = set(got["list"].tolist())

    cap = full // 3
    small = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    with torch.cuda.stream(side):
        psfs.psfs_reconstruct_noalloc(sc.grid, sc.cams, sc.params, mean, var, img, occ, small, cap, cnt,
                                      stream=side)
    side.synchronize()
    assert int(cnt.item()) == full   # the true count, beyond the capacity
    head = small.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    assert len(set(head.tolist())) == cap and set(head.tolist()) <= full_set
