"""Pins of the oracle's inner-voxel removal (surface voxels: occupied voxels
with a face neighbour that is not occupied, outside the grid counting as not
occupied): closed forms for boxes, shells and single voxels, and the same
set from morphological erosion with the 6-neighbourhood (scipy.ndimage), a
library routine for the definition."""

import numpy as np
import pytest

import oracle


def _lin(shape, i, j, k):
    nx, ny, _ = shape
    return i + nx * (j + ny * k)


def _grid(shape):
    nx, ny, nz = shape
    return np.zeros((nz, ny, nx), bool)   # [k][j][i]: ravel() is the linear order i + nx (j + ny k)


def test_empty_and_single_voxel():
    shape = (5, 4, 3)
    g = _grid(shape)
    assert oracle.surface(shape, g.ravel()).size == 0
    g[1, 2, 3] = True
    np.testing.assert_array_equal(oracle.surface(shape, g.ravel()), [_lin(shape, 3, 2, 1)])


@pytest.mark.parametrize("box", [(3, 3, 3), (4, 5, 6), (7, 2, 5), (1, 6, 6)])
def test_solid_box_inside_the_grid(box):
    """A solid a x b x c box keeps a b c - (a-2)(b-2)(c-2) surface voxels
    (every voxel when a side is at most 2), and exactly its inner box is
    removed."""
    a, b, c = box
    shape = (a + 4, b + 3, c + 2)
    g = _grid(shape)
    g[1:1 + c, 2:2 + b, 1:1 + a] = True
    surf = oracle.surface(shape, g.ravel())
    inner = max(a - 2, 0) * max(b - 2, 0) * max(c - 2, 0)
    assert surf.size == a * b * c - inner
    removed = np.setdiff1d(np.flatnonzero(g.ravel()), surf)
    expect = _grid(shape)
    if inner:
        expect[2:c, 3:1 + b, 2:a] = True
    np.testing.assert_array_equal(removed, np.flatnonzero(expect.ravel()))


def test_full_grid_keeps_its_boundary_layer():
    shape = (6, 5, 4)
    g = np.ones((4, 5, 6), bool)
    surf = oracle.surface(shape, g.ravel())
    assert surf.size == 6 * 5 * 4 - 4 * 3 * 2
    assert np.all(np.diff(surf.astype(np.int64)) > 0)   # ascending


def test_hollow_shell_is_all_surface():
    shape = (9, 9, 9)
    g = _grid(shape)
    g[1:8, 1:8, 1:8] = True
    g[2:7, 2:7, 2:7] = False
    surf = oracle.surface(shape, g.ravel())
    np.testing.assert_array_equal(surf, np.flatnonzero(g.ravel()))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_matches_erosion_on_random_solids(seed):
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(seed)
    shape = (23, 17, 11)
    z, y, x = np.mgrid[0:11, 0:17, 0:23]
    g = ((x - 11.3) ** 2 / 60 + (y - 8.1) ** 2 / 30 + (z - 5.2) ** 2 / 12) < 1.0
    g |= rng.random(g.shape) < 0.15
    cross = ndi.generate_binary_structure(3, 1)
    eroded = ndi.binary_erosion(g, structure=cross, border_value=0)
    expect = np.flatnonzero((g & ~eroded).ravel())
    np.testing.assert_array_equal(oracle.surface(shape, g.ravel()), expect)
