"""Pins of the oracle's voxel silhouettes (a pixel is set iff its centre ray
meets a listed voxel's cube in front of the camera): a head-on cube whose
silhouette is its near face, closed form; the silhouette of a solid equals
that of its surface voxels; monotonicity; nothing behind the camera."""

import numpy as np
import pytest

import oracle
from synth import scene as S


def _cam(width, height, f, cx, cy, R=None, t=(0.0, 0.0, 0.0)):
    K = np.array([[f, 0.0, cx], [0.0, f, cy], [0.0, 0.0, 1.0]])
    return {"width": width, "height": height, "K": K, "R": np.eye(3) if R is None else np.asarray(R, float),
            "t": np.asarray(t, float)}


def test_head_on_cube_is_its_near_face():
    """Camera at the origin looking along +z (R = I), f = 100 px, principal
    point (32.25, 24.25).  One voxel: cube [-0.1, 0.1] x [-0.1, 0.1] x [1, 1.2].
    Its silhouette is the near face's projection, u, v in cx +- 10: pixel
    centres x + 1/2 in [22.25, 42.25] -> x = 22..41, likewise y = 14..33."""
    grid = {"nx": 1, "ny": 1, "nz": 1, "origin": (-0.1, -0.1, 1.0), "voxel_size": 0.2}
    cam = _cam(64, 48, 100.0, 32.25, 24.25)
    m = oracle.reproject(grid, [cam], [0])[0]
    expect = np.zeros((48, 64), np.uint8)
    expect[14:34, 22:42] = 1
    np.testing.assert_array_equal(m, expect)


def test_nothing_behind_the_camera():
    grid = {"nx": 1, "ny": 1, "nz": 1, "origin": (-0.1, -0.1, -1.2), "voxel_size": 0.2}
    cam = _cam(64, 48, 100.0, 32.25, 24.25)
    assert oracle.reproject(grid, [cam], [0]).sum() == 0


def test_solid_and_its_surface_have_the_same_silhouette():
    sc = S.make_scene(seed=5, grid_n=16, cube_side=2.0, n_cams=3, width=64, height=48, focal=60.0)
    shape = (16, 16, 16)
    occ = np.zeros((16, 16, 16), bool)
    occ[3:12, 5:14, 2:9] = True
    full = np.flatnonzero(occ.ravel())
    surf = oracle.surface(shape, occ.ravel())
    assert surf.size < full.size
    a = oracle.reproject(sc.grid, sc.cams, full)
    b = oracle.reproject(sc.grid, sc.cams, surf)
    np.testing.assert_array_equal(a, b)
    assert a.sum() > 100


def test_monotone_in_the_voxel_set_and_in_the_cube_size():
    sc = S.make_scene(seed=6, grid_n=12, cube_side=2.0, n_cams=2, width=48, height=40, focal=45.0)
    rng = np.random.default_rng(0)
    lst = np.sort(rng.choice(12 ** 3, 60, replace=False)).astype(np.uint32)
    a = oracle.reproject(sc.grid, sc.cams, lst[:30])
    b = oracle.reproject(sc.grid, sc.cams, lst)
    assert np.all(b >= a) and b.sum() > a.sum()
    shrunk = oracle.reproject(sc.grid, sc.cams, lst, grow=-0.01)
    grown = oracle.reproject(sc.grid, sc.cams, lst, grow=0.01)
    assert np.all(shrunk <= b) and np.all(b <= grown)


def test_voxel_centre_pixel_is_set():
    """The pixel containing a voxel centre's projection is inside the cube's
    silhouette (the centre ray meets the cube at the centre)."""
    sc = S.make_scene(seed=7, grid_n=10, cube_side=2.0, n_cams=2, width=64, height=48, focal=60.0)
    g = sc.grid
    for v in (0, 137, 555, 999):
        m = oracle.reproject(g, sc.cams, [v])
        i, j, k = v % 10, (v // 10) % 10, v // 100
        X = np.asarray(g.origin) + (np.array([i, j, k]) + 0.5) * g.voxel_size
        for c, cam in enumerate(sc.cams):
            xc = cam.R @ X + cam.t
            u, w_, z = cam.K @ xc
            if z <= 0:
                continue
            x, y = u / z, w_ / z
            if 0 <= x < 64 and 0 <= y < 48:
                assert m[c, int(np.floor(y)), int(np.floor(x))] == 1
