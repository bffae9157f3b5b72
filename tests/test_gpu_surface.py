"""Inner-voxel removal on the GPU (psfs_surface) against the oracle's
definition: bit-exact on the same occupied sets (hand-made boxes touching the
grid border, reconstructed frames, several frames per call), consistent with
the oracle's own reconstruction up to the voxels whose occupancy is in the
boundary / tie buckets, and overflow reporting."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1311_6811_gb300 import psfs  # noqa: E402
from synth import scene as S  # noqa: E402
from tests.gpu_helpers import TIE_EPS, logit, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    psfs.load()


def _surface(rec, lists, counts, cap_list, cap_surf):
    n = counts.numel()
    out = torch.full((n, max(cap_surf, 1)), -1, dtype=torch.int32, device="cuda")
    sc = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    psfs.psfs_surface(rec.handle, n, lists, cap_list, counts, out, cap_surf, sc)
    return out, sc


def _sorted(out, sc, f, cap):
    c = min(int(sc[f]), cap)
    return np.sort(out[f, :c].cpu().numpy().astype(np.int64))


def test_boxes_touching_the_grid_border():
    sc = S.make_scene(seed=3, grid_n=24, cube_side=2.0, n_cams=2, width=64, height=48, focal=60.0)
    g = S.Grid(19, 13, 11, (-1.0, -1.0, 0.0), 0.1)
    rec = psfs.Reconstructor(g, sc.cams, sc.params)
    shape = (19, 13, 11)
    occs = []
    a = np.zeros((11, 13, 19), bool)
    a[2:9, 3:10, 4:15] = True           # inside
    b = np.zeros((11, 13, 19), bool)
    b[0:11, 0:5, 12:19] = True          # touches five faces of the grid
    c = np.zeros((11, 13, 19), bool)
    c[5, 6, 7] = True                   # one voxel
    occs = [a, b, c, np.zeros_like(a), np.ones_like(a)]
    V = 19 * 13 * 11
    lists = torch.zeros((len(occs), V), dtype=torch.int32)
    counts = torch.zeros((len(occs),), dtype=torch.int32)
    rng = np.random.default_rng(0)
    for f, o in enumerate(occs):
        idx = np.flatnonzero(o.ravel())
        rng.shuffle(idx)                  # list order is unspecified
        lists[f, :idx.size] = torch.from_numpy(idx.astype(np.int32))
        counts[f] = idx.size
    out, scnt = _surface(rec, lists.cuda(), counts.cuda(), V, V)
    assert rec.sync() == psfs.PSFS_OK
    for f, o in enumerate(occs):
        ref = oracle.surface(shape, o.ravel())
        assert int(scnt[f]) == ref.size
        np.testing.assert_array_equal(_sorted(out, scnt, f, V), ref)
    rec.close()


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_reconstructed_sequence(dtype):
    """Six frames of a walking sequence in one call; each frame's surface
    equals the oracle's surface of the GPU's occupied set, and differs from
    the surface of the oracle's own reconstruction only at voxels next to (or
    at) a voxel in the boundary / tie buckets."""
    sc = S.make_scene(seed=30, grid_n=48, cube_side=2.0, n_cams=4, width=160, height=120, focal=150.0,
                      n_frames=6, walking=True)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params, map_dtype=dtype)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    imgs = to_dev(sc.images)
    F, V = imgs.shape[0], rec.n_voxels
    occ = torch.empty((F, V), device="cuda")
    lists = torch.empty((F, V), dtype=torch.int32, device="cuda")
    counts = torch.zeros((F,), dtype=torch.int32, device="cuda")
    psfs.psfs_reconstruct_sequence(rec.handle, F, imgs, occ, lists, V, counts)
    out, scnt = _surface(rec, lists, counts, V, V)
    assert rec.sync() == psfs.PSFS_OK
    shape = (sc.grid.nx, sc.grid.ny, sc.grid.nz)
    for f in range(F):
        got_occ = np.zeros(V, bool)
        got_occ[lists[f, :int(counts[f])].cpu().numpy()] = True
        got = _sorted(out, scnt, f, V)
        np.testing.assert_array_equal(got, oracle.surface(shape, got_occ))
        assert got.size > 100
        if dtype != "f32":
            continue
        ref = oracle.reconstruct(sc.grid, sc.cams, sc.images[f], sc.mean, sc.var, sc.params)
        ambiguous = ref["boundary"] | (np.abs(ref["logodds"] - logit(0.5)) < TIE_EPS)
        amb = ambiguous.reshape(sc.grid.nz, sc.grid.ny, sc.grid.nx)
        near = amb.copy()
        for ax in range(3):
            near |= np.roll(amb, 1, axis=ax) | np.roll(amb, -1, axis=ax)
        diff = np.setxor1d(got, oracle.surface(shape, ref["occupied"]))
        assert near.ravel()[diff].all(), diff[~near.ravel()[diff]]
    rec.close()


def test_overflow_is_reported():
    sc = S.make_scene(seed=3, grid_n=24, cube_side=2.0, n_cams=2, width=64, height=48, focal=60.0)
    g = S.Grid(16, 16, 16, (-1.0, -1.0, 0.0), 0.1)
    rec = psfs.Reconstructor(g, sc.cams, sc.params)
    o = np.zeros((16, 16, 16), bool)
    o[2:12, 2:12, 2:12] = True
    idx = np.flatnonzero(o.ravel()).astype(np.int32)
    n_surf = 1000 - 512
    lists = torch.from_numpy(idx).cuda().view(1, -1)
    counts = torch.tensor([idx.size], dtype=torch.int32, device="cuda")
    # a surface capacity below the count: the count stays exact, the status says so
    out, scnt = _surface(rec, lists, counts, idx.size, 100)
    assert rec.sync() == psfs.PSFS_ERR_CAPACITY
    assert int(scnt[0]) == n_surf
    w = out[0, :100].cpu().numpy()
    assert np.isin(w, oracle.surface((16, 16, 16), o.ravel())).all()
    # an overflowed input list (count beyond its stride) is reported too
    counts2 = torch.tensor([idx.size + 5], dtype=torch.int32, device="cuda")
    _surface(rec, lists, counts2, idx.size, 1000)
    assert rec.sync() == psfs.PSFS_ERR_CAPACITY
    assert rec.sync() == psfs.PSFS_OK
    rec.close()
