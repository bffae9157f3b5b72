"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test states the passage it follows.  None retypes the oracle's code: the
expected values are hand-derived closed forms, library routines (scipy's
normal density), brute-force carving by exact ray-primitive tests, or
invariants of Eq. 3-9.
"""

import math

import numpy as np
import pytest
from scipy import stats

import oracle
from synth import scene as S

LOG_U = -3.0 * math.log(256.0)


def _cam_down_z(f, W, H, cx, cy, dist):
    """Camera on the -z side at distance `dist`, looking along +z (R = I)."""
    return {"width": W, "height": H,
            "K": np.array([[f, 0, cx], [0, f, cy], [0, 0, 1.0]]),
            "R": np.eye(3), "t": np.array([0.0, 0.0, dist])}


# --------------------------------------------------------------------------- #
# Eq. 1-2: silhouette likelihood map
# --------------------------------------------------------------------------- #
def test_slm_equals_bayes_with_scipy_gaussian():
    """Eq. 1-2 with equal priors: SLM = U / (U + N), N the product of three
    scipy normal densities (diagonal covariance), U = 256^-3."""
    rng = np.random.default_rng(11)
    n = 4000
    img = rng.integers(0, 256, size=(n, 3)).astype(np.uint8)
    mean = rng.uniform(40, 200, size=(n, 3)).astype(np.float32)
    var = (rng.uniform(3, 8, size=(n, 3)) ** 2 + 4).astype(np.float32)
    s = oracle.slm(img, mean, var, LOG_U)
    N = np.prod(stats.norm.pdf(img.astype(np.float64), loc=mean.astype(np.float64),
                               scale=np.sqrt(var.astype(np.float64))), axis=1)
    U = 256.0 ** -3
    expect = (0.5 * U) / (0.5 * U + 0.5 * N)
    np.testing.assert_allclose(s, expect, rtol=1e-12, atol=1e-300)
    assert np.all((s > 0) & (s <= 1))


def test_slm_half_when_gaussian_density_equals_uniform():
    """At I = mu, N = (2 pi var)^(-3/2); choosing var = 256^2 / (2 pi) makes
    N = U, so Eq. 2 gives exactly one half (up to the float32 rounding of var)."""
    var = np.full((1, 3), 256.0 ** 2 / (2 * math.pi), dtype=np.float32)
    mean = np.full((1, 3), 100.0, dtype=np.float32)
    img = np.full((1, 3), 100, dtype=np.uint8)
    s = oracle.slm(img, mean, var, LOG_U)
    assert abs(s[0] - 0.5) < 1e-7


def test_slm_monotone_in_colour_distance():
    """The foreground posterior grows as the colour moves away from the mean."""
    mean = np.full((256, 3), 0.0, dtype=np.float32)
    var = np.full((256, 3), 30.0, dtype=np.float32)
    img = np.repeat(np.arange(256, dtype=np.uint8)[:, None], 3, axis=1)
    s = oracle.slm(img, mean, var, LOG_U)
    assert np.all(np.diff(s) >= 0)
    assert s[0] < 1e-3 and s[-1] == 1.0


# --------------------------------------------------------------------------- #
# camera model (Eq. 3: "the projection of voxel V_i")
# --------------------------------------------------------------------------- #
def test_projection_hand_values():
    cam = _cam_down_z(100.0, 64, 48, 32.0, 24.0, 5.0)
    # X = (0.5, -0.25, 0): x_cam = (0.5, -0.25, 5), u/w = 100*0.1+32 = 42, v/w = -5+24 = 19
    vis, pix, xy, w = oracle.project(cam, [0.5, -0.25, 0.0])
    assert vis and pix == (42, 19) and abs(xy[0] - 42.0) < 1e-12 and abs(xy[1] - 19.0) < 1e-12
    # X = (0.51, -0.2599, 0): u/w = 42.2, v/w = 18.802 -> pixel (42, 18)
    vis, pix, xy, w = oracle.project(cam, [0.51, -0.2599, 0.0])
    assert vis and pix == (42, 18)
    # behind the camera (z_cam = 5 - 6 < 0)
    vis, _, _, w = oracle.project(cam, [0.0, 0.0, -6.0])
    assert not vis and w < 0
    # outside the image: u/w = 100*2/5 + 32 = 72 >= 64
    vis, _, xy, _ = oracle.project(cam, [2.0, 0.0, 0.0])
    assert not vis and abs(xy[0] - 72.0) < 1e-12
    # rotation about z by +90 deg: R maps world (x, y) to (-y, x) in the camera
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    cam_r = dict(cam, R=R)
    vis, pix, xy, _ = oracle.project(cam_r, [0.25, 0.5, 0.0])
    # x_cam = (-0.5, 0.25, 5) -> u/w = -10 + 32 = 22, v/w = 5 + 24 = 29
    assert vis and pix == (22, 29)


# --------------------------------------------------------------------------- #
# Eq. 3-9: one camera, one voxel, by hand
# --------------------------------------------------------------------------- #
ONE_VOXEL_GRID = {"nx": 1, "ny": 1, "nz": 1, "origin": (-0.05, -0.05, -0.05), "voxel_size": 0.1}


@pytest.mark.parametrize("s,expect", [
    # P_D = .9, P_FA = .1, prior = .5.  a = .9 s + .1 (1-s); "nothing" = .1 s + .9 (1-s);
    # b = (nothing + a) / 2 = .5 for every s; occ = .5 a / (.5 a + .5 * .5)
    (0.0, 0.05 / (0.05 + 0.25)),        # a = .1  -> 1/6
    (0.25, 0.15 / (0.15 + 0.25)),       # a = .3  -> .375
    (0.5, 0.5),                         # a = .5
    (1.0, 0.45 / (0.45 + 0.25)),        # a = .9  -> 9/14
])
def test_one_camera_one_voxel(s, expect):
    cam = _cam_down_z(10.0, 1, 1, 0.5, 0.5, 1.0)   # voxel centre projects to (0.5, 0.5)
    out = oracle.fuse(ONE_VOXEL_GRID, [cam], [np.array([[s]])],
                      {"p_detect": 0.9, "p_false_alarm": 0.1, "prior": 0.5, "threshold": 0.5})
    assert out["n_seen"][0] == 1
    assert abs(out["occ"][0] - expect) < 1e-15
    assert out["occupied"][0] == (expect > 0.5)


def test_one_camera_one_voxel_general_rates():
    """P_D = .8, P_FA = .3, prior = .2, s = .75:
    a = .8*.75 + .2*.25 = .65; nothing = .3*.75 + .7*.25 = .4; b = (.4 + .65)/2 = .525;
    occ = .2*.65 / (.2*.65 + .8*.525) = .13 / .55."""
    cam = _cam_down_z(10.0, 1, 1, 0.5, 0.5, 1.0)
    out = oracle.fuse(ONE_VOXEL_GRID, [cam], [np.array([[0.75]])],
                      {"p_detect": 0.8, "p_false_alarm": 0.3, "prior": 0.2, "threshold": 0.5})
    assert abs(out["occ"][0] - 0.13 / 0.55) < 1e-15
    assert abs(out["logodds"][0] - math.log(0.13 / 0.42)) < 1e-13


# --------------------------------------------------------------------------- #
# ring scenes: all-foreground / all-background / uninformative
# --------------------------------------------------------------------------- #
def _ring(n_cams, W=96, H=72, f=90.0, seed=3):
    rng = np.random.default_rng(seed)
    return S.ring_cameras(rng, n_cams, W, H, f, (0.0, 0.0, 1.0), radius=3.0,
                          heights=(1.5, 1.5), jitter_deg=2.0)


SMALL_GRID = {"nx": 12, "ny": 10, "nz": 8, "origin": (-0.3, -0.25, 0.8), "voxel_size": 0.05}


@pytest.mark.parametrize("K,expect_fg", [(4, 10.4976 / 11.4976), (8, 110.19960576 / 111.19960576)])
def test_all_foreground_and_background(K, expect_fg):
    """s = 1 everywhere: every camera contributes a/b = .9/.5 = 1.8, so with
    prior .5 the posterior is 1.8^K / (1 + 1.8^K) (0.913025 at K = 4,
    0.991007 at K = 8).  s = 0: 0.2^K / (1 + 0.2^K)."""
    cams = _ring(K)
    maps = [np.ones((c.height, c.width)) for c in cams]
    out = oracle.fuse(SMALL_GRID, cams, maps)
    assert np.all(out["n_seen"] == K)
    np.testing.assert_allclose(out["occ"], expect_fg, rtol=0, atol=1e-14)
    assert out["occupied"].all() and out["list"].size == out["occ"].size
    assert np.all(np.diff(out["list"].astype(np.int64)) == 1)
    maps0 = [np.zeros((c.height, c.width)) for c in cams]
    out0 = oracle.fuse(SMALL_GRID, cams, maps0)
    np.testing.assert_allclose(out0["occ"], 0.2 ** K / (1 + 0.2 ** K), rtol=1e-13)
    assert out0["list"].size == 0


@pytest.mark.parametrize("prior", [0.5, 0.3, 0.8])
def test_uninformative_maps_and_unseen_voxels_give_prior(prior):
    """s = 1/2 gives a = b = 1/2 for any rates, so the posterior is the prior;
    a voxel that no camera sees also keeps the prior."""
    cams = _ring(4)
    maps = [np.full((c.height, c.width), 0.5) for c in cams]
    p = {"p_detect": 0.85, "p_false_alarm": 0.2, "prior": prior, "threshold": 0.5}
    out = oracle.fuse(SMALL_GRID, cams, maps, p)
    np.testing.assert_allclose(out["occ"], prior, rtol=0, atol=1e-15)
    far = {"nx": 3, "ny": 3, "nz": 3, "origin": (20.0, 20.0, 20.0), "voxel_size": 0.1}
    rng = np.random.default_rng(1)
    out2 = oracle.fuse(far, cams, [rng.uniform(size=(c.height, c.width)) for c in cams], p)
    assert np.all(out2["n_seen"] == 0)
    np.testing.assert_allclose(out2["occ"], prior, rtol=0, atol=1e-15)
    assert out2["occupied"].sum() == (27 if prior > 0.5 else 0)


def test_tie_is_unoccupied():
    """Threshold is strict: posterior exactly equal to the threshold is empty."""
    cams = _ring(4)
    maps = [np.full((c.height, c.width), 0.5) for c in cams]
    out = oracle.fuse(SMALL_GRID, cams, maps, {"prior": 0.5, "threshold": 0.5})
    assert not out["occupied"].any()


def test_literal_eq6_to_9():
    """With P_D = 1, P_FA = 0 the sensor model is Eq. 6-9 verbatim:
    P(S|V=1) = s, P(S|V=0) = (1 - s)/2 + s/2 = 1/2, so
    occ = prior prod s / (prior prod s + (1 - prior) 2^-K).  Maps constant per
    camera, so the lookup position does not matter."""
    K = 5
    cams = _ring(K)
    rng = np.random.default_rng(7)
    sk = rng.uniform(0.05, 0.95, size=K)
    maps = [np.full((c.height, c.width), sk[i]) for i, c in enumerate(cams)]
    prior = 0.35
    out = oracle.fuse(SMALL_GRID, cams, maps,
                      {"p_detect": 1.0, "p_false_alarm": 0.0, "prior": prior})
    assert np.all(out["n_seen"] == K)
    num = prior * np.prod(sk)
    expect = num / (num + (1 - prior) * 2.0 ** -K)
    np.testing.assert_allclose(out["occ"], expect, rtol=1e-13)


# --------------------------------------------------------------------------- #
# special case = visual hull (Sec. 2.2.1): brute-force carving
# --------------------------------------------------------------------------- #
def _pixel_rays(cam):
    W, H = cam.width, cam.height
    xs, ys = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    pix = np.stack([xs.ravel(), ys.ravel(), np.ones(xs.size)], axis=1)
    d = (pix @ np.linalg.inv(cam.K).T) @ cam.R
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return cam.centre, d


def _sphere_silhouette(cam, c, r):
    O, d = _pixel_rays(cam)
    oc = c - O
    tca = d @ oc
    d2 = oc @ oc - tca ** 2
    return ((d2 <= r * r) & (tca > 0)).reshape(cam.height, cam.width)


def _capsule_silhouette(cam, a, b, r):
    O, d = _pixel_rays(cam)
    hit, _ = S._ray_segment_hit(O, d, np.asarray(a, float), np.asarray(b, float), r)
    return hit.reshape(cam.height, cam.width)


def _brute_force_hull(grid, cams, sils):
    """Voxel kept iff seen by >= 1 camera and its centre's pixel is inside the
    silhouette in every camera that sees it (numpy projection, FP64)."""
    nx, ny, nz = grid["nx"], grid["ny"], grid["nz"]
    o = np.asarray(grid["origin"])
    vs = grid["voxel_size"]
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    X = np.stack([o[0] + (i.ravel() + 0.5) * vs, o[1] + (j.ravel() + 0.5) * vs,
                  o[2] + (k.ravel() + 0.5) * vs], axis=1)
    keep = np.ones(len(X), bool)
    seen_any = np.zeros(len(X), bool)
    for cam, sil in zip(cams, sils):
        xc = X @ cam.R.T + cam.t
        uvw = xc @ cam.K.T
        x = uvw[:, 0] / uvw[:, 2]
        y = uvw[:, 1] / uvw[:, 2]
        seen = (uvw[:, 2] > 0) & (x >= 0) & (x < cam.width) & (y >= 0) & (y < cam.height)
        px = np.floor(np.where(seen, x, 0)).astype(int)
        py = np.floor(np.where(seen, y, 0)).astype(int)
        inside = sil[py, px]
        keep &= ~seen | inside
        seen_any |= seen
    return keep & seen_any


@pytest.mark.parametrize("shape", ["sphere", "capsule"])
@pytest.mark.parametrize("n,K", [(16, 2), (24, 3), (32, 4)])
def test_visual_hull_special_case(shape, n, K):
    """Near-binary maps (s = 1 - eps inside, eps outside) with P_D = 1,
    P_FA = 0 and prior 1/2: thresholded PSFS is the classic visual hull."""
    cams = _ring(K, W=80, H=60, f=70.0, seed=n + K)
    centre = np.array([0.05, -0.03, 1.0])
    if shape == "sphere":
        sils = [_sphere_silhouette(c, centre, 0.35) for c in cams]
    else:
        a, b = centre + [-0.25, 0.1, -0.3], centre + [0.2, -0.1, 0.35]
        sils = [_capsule_silhouette(c, a, b, 0.18) for c in cams]
    eps = 1e-9
    maps = [np.where(s, 1 - eps, eps) for s in sils]
    grid = {"nx": n, "ny": n, "nz": n, "origin": (-0.6, -0.6, 0.4), "voxel_size": 1.2 / n}
    out = oracle.fuse(grid, cams, maps, {"p_detect": 1.0, "p_false_alarm": 0.0, "prior": 0.5})
    expect = _brute_force_hull(grid, cams, sils)
    assert expect.any() and not expect.all()
    np.testing.assert_array_equal(out["occupied"], expect)
    np.testing.assert_array_equal(out["list"], np.flatnonzero(expect).astype(np.uint32))


# --------------------------------------------------------------------------- #
# invariants of Eq. 3-4
# --------------------------------------------------------------------------- #
def _random_maps(cams, rng):
    return [rng.uniform(0.0, 1.0, size=(c.height, c.width)) for c in cams]


def test_camera_permutation_invariance():
    cams = _ring(6)
    rng = np.random.default_rng(5)
    maps = _random_maps(cams, rng)
    a = oracle.fuse(SMALL_GRID, cams, maps)
    perm = [3, 0, 5, 1, 4, 2]
    b = oracle.fuse(SMALL_GRID, [cams[p] for p in perm], [maps[p] for p in perm])
    np.testing.assert_allclose(a["occ"], b["occ"], rtol=1e-13, atol=1e-15)


def test_monotone_in_slm():
    """With P_D > P_FA, raising any map value never lowers any posterior."""
    cams = _ring(4)
    rng = np.random.default_rng(6)
    maps = _random_maps(cams, rng)
    base = oracle.fuse(SMALL_GRID, cams, maps)
    up = [np.minimum(1.0, m + rng.uniform(0, 0.3, size=m.shape)) for m in maps]
    hi = oracle.fuse(SMALL_GRID, cams, up)
    assert np.all(hi["occ"] >= base["occ"] - 1e-15)
    assert np.any(hi["occ"] > base["occ"] + 1e-6)


def test_adding_uninformative_camera_changes_nothing():
    cams = _ring(5)
    rng = np.random.default_rng(8)
    maps = _random_maps(cams, rng)
    a = oracle.fuse(SMALL_GRID, cams[:4], maps[:4])
    b = oracle.fuse(SMALL_GRID, cams, maps[:4] + [np.full_like(maps[4], 0.5)])
    np.testing.assert_array_equal(a["occ"], b["occ"])


def test_boundary_flag_marks_pixel_edges():
    """A voxel centre projecting within edge_eps of an integer pixel coordinate is flagged."""
    cam = _cam_down_z(10.0, 4, 4, 2.0, 2.0, 1.0)
    # centre (0, 0, 0) -> (2, 2): exactly on a pixel corner
    g = {"nx": 1, "ny": 1, "nz": 1, "origin": (-0.05, -0.05, -0.05), "voxel_size": 0.1}
    out = oracle.fuse(g, [cam], [np.full((4, 4), 0.7)])
    assert out["boundary"][0]
    # shift by 0.05 m -> (2.5, 2.5): pixel centre, not flagged
    g2 = dict(g, origin=(0.0, 0.0, -0.05))
    out2 = oracle.fuse(g2, [cam], [np.full((4, 4), 0.7)])
    assert not out2["boundary"][0]


def test_fuse_subset_and_voxel_pixels_agree_with_full_fusion():
    """The subset evaluation is the same posterior as the full one, and the
    voxel -> pixel table matches oracle.project."""
    cams = _ring(4)
    rng = np.random.default_rng(17)
    maps = _random_maps(cams, rng)
    full = oracle.fuse(SMALL_GRID, cams, maps)
    idx = rng.choice(full["occ"].size, 50, replace=False)
    sub = oracle.fuse_subset(SMALL_GRID, cams, np.concatenate([m.ravel() for m in maps]), idx)
    np.testing.assert_array_equal(sub, full["occ"][idx])
    pix = oracle.voxel_pixels(SMALL_GRID, cams)
    g = SMALL_GRID
    for v in idx[:10]:
        i, j, k = v % g["nx"], (v // g["nx"]) % g["ny"], v // (g["nx"] * g["ny"])
        X = [g["origin"][0] + (i + .5) * g["voxel_size"], g["origin"][1] + (j + .5) * g["voxel_size"],
             g["origin"][2] + (k + .5) * g["voxel_size"]]
        for c, cam in enumerate(cams):
            vis, (px, py), _, _ = oracle.project(cam, X)
            assert pix[c, v] == (py * cam.width + px if vis else -1)
