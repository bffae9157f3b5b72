"""Pins of the oracle's smoothing before the threshold (3 x 3 x 3 box mean of
the voxel probabilities over the neighbours inside the grid): constants and
interior linear fields are unchanged, a single voxel spreads 1/27 (1/8 at a
grid corner), the result equals a normalised scipy.ndimage uniform filter,
and the threshold is strict."""

import numpy as np
import pytest

import oracle


def _vol(shape):
    nx, ny, nz = shape
    return np.zeros((nz, ny, nx))


def test_constant_field_is_unchanged_everywhere():
    shape = (7, 6, 5)
    p = np.full((5, 6, 7), 0.3)
    out = oracle.smooth(shape, p.ravel())
    np.testing.assert_allclose(out["smoothed"], 0.3, rtol=0, atol=1e-15)
    assert out["list"].size == 0


def test_linear_field_unchanged_in_the_interior():
    shape = (9, 8, 7)
    z, y, x = np.mgrid[0:7, 0:8, 0:9].astype(np.float64)
    p = 0.01 * x - 0.02 * y + 0.03 * z + 0.1
    sm = oracle.smooth(shape, p.ravel())["smoothed"].reshape(p.shape)
    np.testing.assert_allclose(sm[1:-1, 1:-1, 1:-1], p[1:-1, 1:-1, 1:-1], rtol=0, atol=1e-14)


def test_single_voxel_spreads_one_27th_and_one_8th_at_a_corner():
    shape = (7, 7, 7)
    p = _vol(shape)
    p[3, 2, 4] = 1.0   # every voxel of its neighbourhood is an interior voxel
    sm = oracle.smooth(shape, p.ravel())["smoothed"].reshape(p.shape)
    np.testing.assert_allclose(sm[2:5, 1:4, 3:6], 1.0 / 27.0, rtol=0, atol=1e-15)
    assert sm.sum() == pytest.approx(1.0)
    shape = (6, 6, 6)
    q = _vol(shape)
    q[0, 0, 0] = 1.0
    sq = oracle.smooth(shape, q.ravel())["smoothed"].reshape(q.shape)
    assert sq[0, 0, 0] == pytest.approx(1.0 / 8.0)   # 8 voxels in the corner's clipped neighbourhood
    assert sq[1, 1, 1] == pytest.approx(1.0 / 27.0)
    assert sq[0, 1, 1] == pytest.approx(1.0 / 18.0)


@pytest.mark.parametrize("seed", [0, 1])
def test_matches_normalised_uniform_filter(seed):
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(seed)
    shape = (13, 11, 9)
    p = rng.random((9, 11, 13))
    num = ndi.uniform_filter(p, size=3, mode="constant", cval=0.0)
    den = ndi.uniform_filter(np.ones_like(p), size=3, mode="constant", cval=0.0)
    out = oracle.smooth(shape, p.ravel(), threshold=0.5)
    np.testing.assert_allclose(out["smoothed"], (num / den).ravel(), rtol=0, atol=1e-12)
    np.testing.assert_array_equal(out["occupied"], (num / den).ravel() > 0.5)


def test_threshold_is_strict():
    shape = (4, 4, 4)
    p = np.full((4, 4, 4), 0.5)
    assert oracle.smooth(shape, p.ravel(), threshold=0.5)["list"].size == 0
    assert oracle.smooth(shape, p.ravel(), threshold=0.4999)["list"].size == 64
