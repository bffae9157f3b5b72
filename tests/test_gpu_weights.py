"""Tracker particle weights on the GPU (psfs_particle_weights) against the
oracle: per camera, S_e and S_r may differ from the oracle's only by the
samples whose projection lies within 1e-3 px of a pixel edge (counted by the
oracle), and log-weights accordingly; closed forms; the whole chain from
images to weights ranks the true pose first."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1311_6811_gb300 import psfs  # noqa: E402
from synth import scene as S  # noqa: E402
from tests.gpu_helpers import to_dev  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    psfs.load()


def _cyl(capsules):
    return np.array([[*c.a, *c.b, c.radius] for c in capsules])


def _particles(seed, n, base):
    rng = np.random.default_rng(seed)
    out = [base]
    for _ in range(n - 1):
        # the whole body shifted, every endpoint jittered, radii kept
        shift = rng.normal(0, 0.05, size=3)
        d = rng.normal(0, 0.02, size=(base.shape[0], 7))
        d[:, 6] = 0.0
        d[:, 0:3] += shift
        d[:, 3:6] += shift
        out.append(base + d)
    return np.stack(out)


def _gpu(rec, parts, masks, kt=8, kw=4):
    P = parts.shape[0]
    w = torch.empty(P, device="cuda")
    t = torch.empty((P, rec.n_cams, 2), device="cuda")
    psfs.psfs_particle_weights(rec.handle, torch.from_numpy(parts.astype(np.float32)).cuda(),
                               torch.from_numpy(masks).cuda(), w, t, kt=kt, kw=kw)
    assert rec.sync() == psfs.PSFS_OK
    return w.cpu().numpy().astype(np.float64), t.cpu().numpy().astype(np.float64)


def _check(cams, masks, parts, w, t, kt=8, kw=4):
    # the oracle sees exactly the float32 particles the GPU gets
    ref = oracle.particle_weights(cams, masks, parts.astype(np.float32).astype(np.float64), kt=kt, kw=kw)
    n_cyl = parts.shape[1]
    n_e, n_r = 2 * n_cyl * kt, n_cyl * kt * kw
    amb = ref["ambiguous"].astype(np.float64)
    assert np.all(np.abs(t[..., 0] - ref["terms"][..., 0]) <= amb / n_e + 1e-6)
    assert np.all(np.abs(t[..., 1] - ref["terms"][..., 1]) <= amb / n_r + 1e-6)
    bound = (amb / n_e + amb / n_r).sum(axis=1) + 1e-5
    assert np.all(np.abs(np.log(w) - np.log(ref["weights"])) <= bound)
    return ref


@pytest.mark.parametrize("kt,kw", [(8, 4), (3, 5)])
def test_against_oracle_on_rendered_silhouettes(kt, kw):
    sc = S.make_scene(seed=51, grid_n=16, cube_side=2.2, n_cams=6, width=200, height=150, focal=180.0)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    caps = S.body_capsules(S.random_pose(np.random.default_rng(7)), np.zeros((10, 3)))
    masks = np.stack([(S.render_labels(c, caps) >= 0).astype(np.uint8) for c in sc.cams])
    parts = _particles(8, 40, _cyl(caps))
    w, t = _gpu(rec, parts, masks, kt, kw)
    ref = _check(sc.cams, masks, parts, w, t, kt, kw)
    assert ref["weights"][0] == ref["weights"].max()
    rec.close()


def test_closed_forms_on_the_gpu():
    sc = S.make_scene(seed=3, grid_n=16, cube_side=2.2, n_cams=4, width=160, height=120, focal=70.0)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    caps = S.body_capsules(S.random_pose(np.random.default_rng(1)), np.zeros((10, 3)))
    cyl = _cyl(caps)[None]
    K = len(sc.cams)
    w, _ = _gpu(rec, cyl, np.ones((K, 120, 160), np.uint8))
    assert w[0] == pytest.approx(np.exp(-K), rel=1e-6)
    w, _ = _gpu(rec, cyl, np.zeros((K, 120, 160), np.uint8))
    assert w[0] == pytest.approx(np.exp(-2 * K), rel=1e-6)
    one = cyl[:, :1]
    w, t = _gpu(rec, one, np.ones((K, 120, 160), np.uint8), kt=1, kw=1)
    np.testing.assert_allclose(t[0, :, 1], 0.0)
    rec.close()


def test_chain_from_images_ranks_the_true_pose_first():
    """Images -> reconstruction -> surface voxels -> silhouettes -> weights of
    particles around the true pose (and of the true pose itself)."""
    sc = S.make_scene(seed=52, grid_n=64, cube_side=2.2, n_cams=4, width=160, height=120, focal=150.0)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    occ, lst, cnt = rec.reconstruct(to_dev(sc.images))
    V = rec.n_voxels
    sl = torch.empty((1, V), dtype=torch.int32, device="cuda")
    sn = torch.zeros((1,), dtype=torch.int32, device="cuda")
    psfs.psfs_surface(rec.handle, 1, lst.view(1, -1), rec.capacity, cnt, sl, V, sn)
    masks = torch.empty((1, rec.n_cams, 120, 160), dtype=torch.uint8, device="cuda")
    psfs.psfs_reproject(rec.handle, 1, sl, V, sn, masks)
    assert rec.sync() == psfs.PSFS_OK
    parts = _particles(9, 30, _cyl(sc.capsules[0]))
    m = masks[0].cpu().numpy()
    w, t = _gpu(rec, parts, m)
    _check(sc.cams, m, parts, w, t)
    assert w[0] >= np.sort(w)[-3]   # the true pose among the best three of 30
    rec.close()
