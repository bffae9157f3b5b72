"""Pins of the oracle's tracker weights (Eq. 14-16) and edge maps: closed
forms for all-set / empty silhouettes and for bodies behind the cameras,
hand-checked edge maps, invariance under cylinder order, and the weight of
the true pose above the weights of displaced poses against silhouettes
rendered from the true pose."""

import numpy as np
import pytest

import oracle
from synth import scene as S


def _cyl(capsules):
    return np.array([[*c.a, *c.b, c.radius] for c in capsules])


def _body(seed=0, root=(0.0, 0.0)):
    rng = np.random.default_rng(seed)
    pose = S.random_pose(rng, root_xy=root)
    return S.body_capsules(pose, np.zeros((10, 3)))


def test_edge_maps():
    m = np.zeros((1, 6, 7), np.uint8)
    assert oracle.edges(m).sum() == 0
    assert oracle.edges(np.ones_like(m)).sum() == 0          # the image border is not an edge
    m[0, 3, 4] = 1
    np.testing.assert_array_equal(oracle.edges(m), m)       # a lone pixel is its own edge
    r = np.zeros((1, 8, 9), np.uint8)
    r[0, 2:6, 1:7] = 1
    ring = r.copy()
    ring[0, 3:5, 2:6] = 0
    np.testing.assert_array_equal(oracle.edges(r), ring)
    t = np.zeros((1, 5, 5), np.uint8)
    t[0, 0:3, 0:5] = 1                                      # touches three image borders
    e = np.zeros_like(t)
    e[0, 2, :] = 1
    np.testing.assert_array_equal(oracle.edges(t), e)


def test_closed_forms():
    # a wide field of view: the whole body is inside every image
    sc = S.make_scene(seed=3, grid_n=16, cube_side=2.2, n_cams=4, width=160, height=120, focal=70.0)
    cyl = _cyl(_body(1))[None]
    K = len(sc.cams)
    full = np.ones((K, 120, 160), np.uint8)
    out = oracle.particle_weights(sc.cams, full, cyl)
    np.testing.assert_allclose(out["terms"][0, :, 1], 0.0)          # every silhouette sample is set
    np.testing.assert_allclose(out["terms"][0, :, 0], 1.0)          # and no pixel is an edge
    assert out["weights"][0] == pytest.approx(np.exp(-K), rel=1e-12)
    empty = np.zeros_like(full)
    assert oracle.particle_weights(sc.cams, empty, cyl)["weights"][0] == pytest.approx(np.exp(-2 * K), rel=1e-12)
    # the body moved 10 km up: above every camera's field of view
    far = cyl.copy()
    far[..., 2] += 1e4
    far[..., 5] += 1e4
    assert oracle.particle_weights(sc.cams, full, far)["weights"][0] == pytest.approx(np.exp(-2 * K), rel=1e-12)


def test_cylinder_order_does_not_matter():
    sc = S.make_scene(seed=4, grid_n=16, cube_side=2.2, n_cams=3, width=120, height=90, focal=110.0)
    caps = _body(2)
    masks = np.stack([(S.render_labels(c, caps) >= 0).astype(np.uint8) for c in sc.cams])
    cyl = _cyl(caps)
    perm = np.random.default_rng(0).permutation(len(caps))
    a = oracle.particle_weights(sc.cams, masks, cyl[None])
    b = oracle.particle_weights(sc.cams, masks, cyl[perm][None])
    np.testing.assert_array_equal(a["terms"], b["terms"])
    assert a["weights"][0] == b["weights"][0]


def test_true_pose_outweighs_displaced_poses():
    sc = S.make_scene(seed=5, grid_n=16, cube_side=2.2, n_cams=4, width=160, height=120, focal=150.0)
    caps = _body(3)
    masks = np.stack([(S.render_labels(c, caps) >= 0).astype(np.uint8) for c in sc.cams])
    cyl = _cyl(caps)
    shifts = [np.zeros(3), np.array([0.15, 0, 0]), np.array([0, -0.2, 0]), np.array([0, 0, 0.3])]
    parts = np.stack([cyl + np.concatenate([d, d, [0.0]]) for d in shifts])
    w = oracle.particle_weights(sc.cams, masks, parts)["weights"]
    assert np.all(w[0] > w[1:]), w
    # silhouette samples of the true pose lie inside the rendered bodies almost everywhere
    assert oracle.particle_weights(sc.cams, masks, cyl[None])["terms"][0, :, 1].max() < 0.1
