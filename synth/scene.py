"""Seeded synthetic multi-camera scenes for probabilistic shape-from-silhouette.

This module only makes inputs: calibrated pinhole cameras on a ring, an
articulated body of ten capsules (the ten body parts of Table 1), a per-pixel
Gaussian colour background and the rendered uint8 images.  It holds none of the
reconstruction arithmetic (no likelihood, no projection of voxels, no fusion);
both the oracle and the CUDA path consume what it returns.

Conventions (shared by every consumer, stated once here):

* world frame: z up, metres;
* a camera maps a world point X to x_cam = R X + t, then (u, v, w) = K x_cam and
  the point lies at image position (u / w, v / w); pixel (x, y) covers
  [x, x+1) x [y, y+1), so a pixel centre sits at (x + 0.5, y + 0.5);
* a grid is (nx, ny, nz, origin, voxel_size); voxel (i, j, k) has its centre at
  origin + (i + 0.5, j + 0.5, k + 0.5) * voxel_size and linear index
  i + nx * (j + ny * k);
* images are uint8 [n_cams][H][W][3]; background mean and variance are float32
  [n_cams][H][W][3]; the variance handed out already contains the sensor noise.

Rendering is CPU ray casting of each pixel-centre ray against the capsules
(no graphics API).  The sensor noise is N(0, 4) per channel (variance 4),
added to foreground and background alike, then rounded and clamped to [0, 255].
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

SENSOR_NOISE_VAR = 4.0


# --------------------------------------------------------------------------- #
# cameras
# --------------------------------------------------------------------------- #
@dataclasses.dataclass
class Camera:
    width: int
    height: int
    K: np.ndarray  # (3, 3) float64
    R: np.ndarray  # (3, 3) float64, world -> camera rotation
    t: np.ndarray  # (3,) float64

    @property
    def centre(self) -> np.ndarray:
        return -self.R.T @ self.t

    def as_dict(self) -> dict:
        return {"width": self.width, "height": self.height,
                "K": self.K.copy(), "R": self.R.copy(), "t": self.t.copy()}


def _rot_x(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]], dtype=np.float64)


def _rot_y(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]], dtype=np.float64)


def _rot_z(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]], dtype=np.float64)


def look_at_camera(centre, target, width, height, focal,
                   jitter_rad=(0.0, 0.0, 0.0)) -> Camera:
    """Pinhole camera at `centre` looking at `target` (x right, y down, z forward).

    `jitter_rad` = (yaw, pitch, roll) applied in the camera frame after the
    look-at rotation.  Principal point at the image centre, square pixels.
    """
    centre = np.asarray(centre, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    fwd = target - centre
    fwd /= np.linalg.norm(fwd)
    up = np.array([0.0, 0.0, 1.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R0 = np.stack([right, down, fwd])
    yaw, pitch, roll = jitter_rad
    Rj = _rot_z(roll) @ _rot_x(pitch) @ _rot_y(yaw)
    R = Rj @ R0
    t = -R @ centre
    K = np.array([[focal, 0.0, width / 2.0],
                  [0.0, focal, height / 2.0],
                  [0.0, 0.0, 1.0]])
    return Camera(width, height, K, R, t)


def ring_cameras(rng: np.random.Generator, n_cams: int, width: int, height: int,
                 focal: float, target, radius: float = 3.0,
                 heights=(1.5, 1.5), jitter_deg: float = 2.0,
                 azimuth0: float = 0.0) -> List[Camera]:
    """`n_cams` cameras evenly spaced on a ring of `radius` around `target`.

    Heights are uniform in `heights` (a degenerate interval gives a fixed
    height); yaw/pitch/roll jitter is uniform in +/- `jitter_deg`.
    """
    cams = []
    tx, ty = float(target[0]), float(target[1])
    for c in range(n_cams):
        az = azimuth0 + 2.0 * math.pi * c / n_cams
        h = heights[0] if heights[0] == heights[1] else rng.uniform(*heights)
        centre = (tx + radius * math.cos(az), ty + radius * math.sin(az), h)
        jit = tuple(math.radians(x) for x in rng.uniform(-jitter_deg, jitter_deg, 3))
        cams.append(look_at_camera(centre, target, width, height, focal, jit))
    return cams


# --------------------------------------------------------------------------- #
# articulated capsule body (Table 1: torso, 2 thighs, 2 calves, 4 arm parts, head)
# --------------------------------------------------------------------------- #
# (length, radius) in metres
PART_DIMS = {
    "torso": (0.55, 0.14),
    "thigh": (0.42, 0.075),
    "calf": (0.42, 0.055),
    "upper_arm": (0.30, 0.045),
    "lower_arm": (0.28, 0.04),
    "head": (0.10, 0.10),
}
PART_ORDER = ["torso", "l_thigh", "l_calf", "r_thigh", "r_calf",
              "l_upper_arm", "l_lower_arm", "r_upper_arm", "r_lower_arm", "head"]


@dataclasses.dataclass
class Capsule:
    a: np.ndarray      # (3,) segment start
    b: np.ndarray      # (3,) segment end
    radius: float
    colour: np.ndarray  # (3,) float64 in [0, 255]


@dataclasses.dataclass
class Pose:
    """Joint angles in radians plus root position and heading."""
    root: np.ndarray           # (3,) pelvis position
    heading: float             # yaw of the body about z
    hip_flex: tuple            # (left, right) forward swing
    hip_abd: tuple             # (left, right) sideways
    knee: tuple                # (left, right) flexion >= 0
    shoulder_flex: tuple
    shoulder_abd: tuple
    elbow: tuple               # flexion >= 0
    torso_lean: float = 0.0
    head_tilt: float = 0.0


def _limb_dir(flex, abd, side_sign):
    """Unit direction of a hanging limb in the body frame (x fwd, y left, z up)."""
    d = np.array([0.0, 0.0, -1.0])
    d = _rot_y(-flex) @ d            # swing forward about the lateral axis
    d = _rot_x(side_sign * abd) @ d  # swing outward
    return d / np.linalg.norm(d)


def body_capsules(pose: Pose, colours: np.ndarray) -> List[Capsule]:
    """Ten capsules for `pose` in world coordinates; `colours` is (10, 3)."""
    Rb = _rot_z(pose.heading)
    root = np.asarray(pose.root, dtype=np.float64)

    def W(p):
        return root + Rb @ p

    caps = []
    tl, tr = PART_DIMS["torso"]
    torso_dir = _rot_y(-pose.torso_lean) @ np.array([0.0, 0.0, 1.0])
    t0 = np.array([0.0, 0.0, 0.0])
    t1 = t0 + tl * torso_dir
    caps.append(("torso", t0, t1, tr))
    # legs
    for side, sgn in (("l", 1.0), ("r", -1.0)):
        si = 0 if side == "l" else 1
        hip = np.array([0.0, sgn * 0.09, -0.02])
        thl, thr = PART_DIMS["thigh"]
        dth = _limb_dir(pose.hip_flex[si], pose.hip_abd[si], sgn)
        knee = hip + thl * dth
        cal, car = PART_DIMS["calf"]
        dca = _limb_dir(pose.hip_flex[si] - pose.knee[si], pose.hip_abd[si], sgn)
        ankle = knee + cal * dca
        caps.append((f"{side}_thigh", hip, knee, thr))
        caps.append((f"{side}_calf", knee, ankle, car))
    # arms
    for side, sgn in (("l", 1.0), ("r", -1.0)):
        si = 0 if side == "l" else 1
        sh = t1 + np.array([0.0, sgn * (tr + 0.05), -0.04])
        ual, uar = PART_DIMS["upper_arm"]
        dua = _limb_dir(pose.shoulder_flex[si], pose.shoulder_abd[si], sgn)
        elb = sh + ual * dua
        lal, lar = PART_DIMS["lower_arm"]
        dla = _limb_dir(pose.shoulder_flex[si] + pose.elbow[si], pose.shoulder_abd[si], sgn)
        wr = elb + lal * dla
        caps.append((f"{side}_upper_arm", sh, elb, uar))
        caps.append((f"{side}_lower_arm", elb, wr, lar))
    hl, hr = PART_DIMS["head"]
    hdir = _rot_y(-pose.head_tilt) @ torso_dir
    h0 = t1 + (0.05 + hr) * torso_dir
    caps.append(("head", h0, h0 + hl * hdir, hr))
    by_name = {c[0]: c for c in caps}
    out = []
    for n, name in enumerate(PART_ORDER):
        _, a, b, r = by_name[name]
        out.append(Capsule(W(a), W(b), float(r), np.asarray(colours[n], dtype=np.float64)))
    return out


def random_pose(rng: np.random.Generator, root_xy=(0.0, 0.0)) -> Pose:
    """A static pose with seeded joint angles inside human limits."""
    d = math.radians
    u = rng.uniform
    root = np.array([root_xy[0], root_xy[1], 0.0])
    pose = Pose(root=root, heading=u(-math.pi, math.pi),
                hip_flex=(d(u(-25, 40)), d(u(-25, 40))),
                hip_abd=(d(u(0, 20)), d(u(0, 20))),
                knee=(d(u(0, 60)), d(u(0, 60))),
                shoulder_flex=(d(u(-30, 80)), d(u(-30, 80))),
                shoulder_abd=(d(u(5, 70)), d(u(5, 70))),
                elbow=(d(u(0, 90)), d(u(0, 90))),
                torso_lean=d(u(-10, 10)), head_tilt=d(u(-15, 15)))
    return _ground(pose)


def _ground(pose: Pose) -> Pose:
    """Raise the root so that the lowest capsule point touches z = 0.02."""
    caps = body_capsules(dataclasses.replace(pose, root=np.array([pose.root[0], pose.root[1], 0.0])),
                         np.zeros((10, 3)))
    zmin = min(min(c.a[2], c.b[2]) - c.radius for c in caps)
    root = np.array([pose.root[0], pose.root[1], 0.02 - zmin])
    return dataclasses.replace(pose, root=root)


def walking_poses(rng: np.random.Generator, n_frames: int, centre_xy=(0.0, 0.0),
                  path_radius: float = 0.35, fps: float = 30.0) -> List[Pose]:
    """Smooth walk: sinusoidal gait plus a root moving on a circle of `path_radius`."""
    d = math.radians
    phase0 = rng.uniform(0, 2 * math.pi)
    ang0 = rng.uniform(0, 2 * math.pi)
    gait_hz = rng.uniform(0.8, 1.1)
    speed = rng.uniform(0.6, 1.0)          # m/s along the path
    amp_hip = d(rng.uniform(20, 30))
    amp_knee = d(rng.uniform(35, 55))
    amp_sh = d(rng.uniform(15, 30))
    poses = []
    for f in range(n_frames):
        tsec = f / fps
        ang = ang0 + speed * tsec / path_radius
        rx = centre_xy[0] + path_radius * math.cos(ang)
        ry = centre_xy[1] + path_radius * math.sin(ang)
        heading = ang + math.pi / 2
        ph = phase0 + 2 * math.pi * gait_hz * tsec
        sl, sr = math.sin(ph), math.sin(ph + math.pi)
        pose = Pose(root=np.array([rx, ry, 0.0]), heading=heading,
                    hip_flex=(amp_hip * sl, amp_hip * sr),
                    hip_abd=(d(4.0), d(4.0)),
                    knee=(amp_knee * max(0.0, -math.cos(ph)) + d(5),
                          amp_knee * max(0.0, -math.cos(ph + math.pi)) + d(5)),
                    shoulder_flex=(amp_sh * sr, amp_sh * sl),
                    shoulder_abd=(d(10.0), d(10.0)),
                    elbow=(d(20) + 0.5 * amp_sh * (1 + sr), d(20) + 0.5 * amp_sh * (1 + sl)),
                    torso_lean=d(3.0), head_tilt=0.0)
        poses.append(_ground(pose))
    return poses


# --------------------------------------------------------------------------- #
# rendering (ray casting of pixel-centre rays against capsules)
# --------------------------------------------------------------------------- #
def _ray_segment_hit(O, D, A, B, r):
    """For rays O + s D (s >= 0, D unit, D is (n, 3)) return (hit mask, depth).

    Hit iff the minimum distance between the ray and segment AB is <= r; the
    depth is the ray parameter of closest approach (used only to pick the
    nearest capsule for colouring).
    """
    e = B - A
    c = float(e @ e)
    w0 = O - A                      # (3,)
    b = D @ e                       # (n,)
    dd = D @ w0                     # (n,)
    ee = float(e @ w0)
    denom = c - b * b               # a = 1
    best = np.full(D.shape[0], np.inf)
    best_s = np.zeros(D.shape[0])
    with np.errstate(divide="ignore", invalid="ignore"):
        s_int = (b * ee - c * dd) / denom
        t_int = (ee - b * dd) / denom
    ok = (denom > 1e-12 * c) & (t_int >= 0) & (t_int <= 1) & (s_int >= 0)
    if np.any(ok):
        P = O + s_int[ok, None] * D[ok]
        Q = A + t_int[ok, None] * e
        dist = np.linalg.norm(P - Q, axis=1)
        best[ok] = dist
        best_s[ok] = s_int[ok]
    for P in (A, B):
        s = np.maximum(D @ (P - O), 0.0)
        dist = np.linalg.norm(O + s[:, None] * D - P, axis=1)
        m = dist < best
        best[m] = dist[m]
        best_s[m] = s[m]
    return best <= r, best_s


def _capsule_pixel_bbox(cam: Camera, cap: Capsule):
    """Conservative pixel box of a capsule (None = whole image)."""
    lo = np.minimum(cap.a, cap.b) - cap.radius
    hi = np.maximum(cap.a, cap.b) + cap.radius
    corners = np.array([[x, y, z] for x in (lo[0], hi[0]) for y in (lo[1], hi[1])
                        for z in (lo[2], hi[2])])
    xc = corners @ cam.R.T + cam.t
    if np.any(xc[:, 2] <= 1e-6):
        return 0, cam.width, 0, cam.height
    uvw = xc @ cam.K.T
    u = uvw[:, 0] / uvw[:, 2]
    v = uvw[:, 1] / uvw[:, 2]
    x0 = max(0, int(math.floor(u.min())) - 1)
    x1 = min(cam.width, int(math.ceil(u.max())) + 2)
    y0 = max(0, int(math.floor(v.min())) - 1)
    y1 = min(cam.height, int(math.ceil(v.max())) + 2)
    if x0 >= x1 or y0 >= y1:
        return None
    return x0, x1, y0, y1


def render_labels(cam: Camera, capsules: Sequence[Capsule]) -> np.ndarray:
    """Per pixel: index of the nearest capsule hit by the pixel-centre ray, or -1."""
    H, W = cam.height, cam.width
    label = np.full((H, W), -1, dtype=np.int32)
    depth = np.full((H, W), np.inf)
    O = cam.centre
    Kinv = np.linalg.inv(cam.K)
    for ci, cap in enumerate(capsules):
        bb = _capsule_pixel_bbox(cam, cap)
        if bb is None:
            continue
        x0, x1, y0, y1 = bb
        xs = np.arange(x0, x1, dtype=np.float64) + 0.5
        ys = np.arange(y0, y1, dtype=np.float64) + 0.5
        gx, gy = np.meshgrid(xs, ys)
        pix = np.stack([gx.ravel(), gy.ravel(), np.ones(gx.size)], axis=1)
        D = (pix @ Kinv.T) @ cam.R          # camera -> world: R^T d
        D /= np.linalg.norm(D, axis=1, keepdims=True)
        hit, s = _ray_segment_hit(O, D, cap.a, cap.b, cap.radius)
        hit = hit.reshape(gy.shape)
        s = s.reshape(gy.shape)
        sub_d = depth[y0:y1, x0:x1]
        sub_l = label[y0:y1, x0:x1]
        closer = hit & (s < sub_d)
        sub_d[closer] = s[closer]
        sub_l[closer] = ci
    return label


def make_background(rng: np.random.Generator, n_cams: int, H: int, W: int,
                    mean_range=(40.0, 200.0), sigma_range=(3.0, 8.0)):
    """Per-pixel, per-channel Gaussian background: (mean, sigma) float64."""
    mean = rng.uniform(*mean_range, size=(n_cams, H, W, 3))
    sigma = rng.uniform(*sigma_range, size=(n_cams, H, W, 3))
    return mean, sigma


def render_images(rng: np.random.Generator, cams: Sequence[Camera], capsules: Sequence[Capsule],
                  bg_mean: np.ndarray, bg_sigma: np.ndarray,
                  labels_out: Optional[list] = None) -> np.ndarray:
    """uint8 [n_cams][H][W][3].

    Background pixel: mean + N(0, sigma^2) + N(0, 4), drawn as one Gaussian of
    variance sigma^2 + 4; foreground pixel: capsule colour + N(0, 4).  Then
    rounded and clamped to [0, 255].
    """
    n = len(cams)
    H, W = cams[0].height, cams[0].width
    z = rng.standard_normal((n, H, W, 3), dtype=np.float32)
    std = np.sqrt(bg_sigma.astype(np.float32) ** 2 + np.float32(SENSOR_NOISE_VAR))
    img = bg_mean.astype(np.float32) + std * z
    cols = np.array([c.colour for c in capsules], np.float32) if len(capsules) else np.zeros((0, 3), np.float32)
    noise_sd = np.float32(math.sqrt(SENSOR_NOISE_VAR))
    for k, cam in enumerate(cams):
        lab = render_labels(cam, capsules)
        if labels_out is not None:
            labels_out.append(lab)
        fg = lab >= 0
        img[k][fg] = cols[lab[fg]] + noise_sd * z[k][fg]
    np.rint(img, out=img)
    np.clip(img, 0, 255, out=img)
    return img.astype(np.uint8)


# --------------------------------------------------------------------------- #
# whole scenes
# --------------------------------------------------------------------------- #
@dataclasses.dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    origin: tuple
    voxel_size: float

    def as_dict(self) -> dict:
        return {"nx": self.nx, "ny": self.ny, "nz": self.nz,
                "origin": tuple(float(x) for x in self.origin),
                "voxel_size": float(self.voxel_size)}

    @property
    def n_voxels(self) -> int:
        return self.nx * self.ny * self.nz


@dataclasses.dataclass
class Params:
    p_detect: float = 0.9
    p_false_alarm: float = 0.1
    prior: float = 0.5
    threshold: float = 0.5
    log_fg_density: float = -3.0 * math.log(256.0)   # uniform over the RGB cube


@dataclasses.dataclass
class Scene:
    grid: Grid
    cams: List[Camera]
    images: np.ndarray        # uint8 [F][K][H][W][3] (F frames) or [K][H][W][3]
    mean: np.ndarray          # float32 [K][H][W][3]
    var: np.ndarray           # float32 [K][H][W][3]
    params: Params
    capsules: list            # per frame: list of Capsule

    @property
    def n_cams(self) -> int:
        return len(self.cams)


def cube_grid(n: int, side: float, centre_xy=(0.0, 0.0)) -> Grid:
    half = side / 2.0
    return Grid(n, n, n, (centre_xy[0] - half, centre_xy[1] - half, 0.0), side / n)


def _colours(rng, n=10):
    return rng.uniform(0.0, 255.0, size=(n, 3))


def _render_frame(args):
    seed, frame, cams, caps, mean, sigma = args
    rng = np.random.default_rng([seed, 1 + frame])
    return render_images(rng, cams, caps, mean, sigma)


def make_scene(*, seed: int, grid_n: int, cube_side: float, n_cams: int, width: int,
               height: int, focal: float, n_frames: int = 1, heights=(1.5, 1.5),
               n_bodies: int = 1, walking: bool = False, ring_radius: float = 3.0,
               params: Optional[Params] = None, workers: int = 1,
               frame_ids: Optional[Sequence[int]] = None) -> Scene:
    """Body (or bodies) on a ring of cameras, per-pixel Gaussian background.

    Cameras, background, colours and poses come from one generator seeded with
    `seed`; the noise of frame f from a generator seeded with (seed, 1 + f), so
    frames can be rendered by `workers` processes (spawned) with identical
    results.  `frame_ids` renders only those frames of the `n_frames`-frame
    sequence, in that order (each exactly as in the whole sequence).
    """
    rng = np.random.default_rng(seed)
    grid = cube_grid(grid_n, cube_side)
    target = (0.0, 0.0, cube_side / 2.0)
    cams = ring_cameras(rng, n_cams, width, height, focal, target, radius=ring_radius,
                        heights=heights)
    mean, sigma = make_background(rng, n_cams, height, width)
    var = sigma ** 2 + SENSOR_NOISE_VAR
    body_cols = [_colours(rng) for _ in range(n_bodies)]
    if n_bodies == 1:
        offsets = [(0.0, 0.0)]
    else:
        offsets = [(-0.35 + 0.7 * b / (n_bodies - 1), 0.25 * (-1) ** b) for b in range(n_bodies)]
    if walking:
        tracks = [walking_poses(rng, n_frames, centre_xy=o) for o in offsets]
    else:
        tracks = [[random_pose(rng, root_xy=o) for _ in range(n_frames)] for o in offsets]
    caps_per_frame = []
    for f in range(n_frames):
        caps = []
        for b in range(n_bodies):
            caps.extend(body_capsules(tracks[b][f], body_cols[b]))
        caps_per_frame.append(caps)
    ids = list(range(n_frames)) if frame_ids is None else [int(f) for f in frame_ids]
    if any(not 0 <= f < n_frames for f in ids):
        raise ValueError("frame_ids outside the sequence")
    jobs = [(seed, f, cams, caps_per_frame[f], mean, sigma) for f in ids]
    if workers > 1 and len(jobs) > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(workers, len(jobs))) as pool:
            frames = pool.map(_render_frame, jobs, chunksize=1)
    else:
        frames = [_render_frame(j) for j in jobs]
    images = np.stack(frames) if (n_frames > 1 or frame_ids is not None) else frames[0]
    return Scene(grid, cams, images, mean.astype(np.float32), var.astype(np.float32),
                 params or Params(), [caps_per_frame[f] for f in ids])


# The workloads, by what they are.
def scene_64cube_4cam(seed: int = 0) -> Scene:
    """64^3 grid over a 2 m cube, 4 cameras 320x240 (f = 300 px) on a 3 m ring at 1.5 m."""
    return make_scene(seed=seed, grid_n=64, cube_side=2.0, n_cams=4, width=320, height=240,
                      focal=300.0)


def scene_128cube_8cam(seed: int = 1, n_frames: int = 100, workers: int = 1, frame_ids=None) -> Scene:
    """128^3 grid over a 2.2 m cube, 8 cameras 640x480 (f = 600 px), heights 1.2-2.2 m,
    a walking sequence of `n_frames` frames (only `frame_ids` of them, if given)."""
    return make_scene(seed=seed, grid_n=128, cube_side=2.2, n_cams=8, width=640, height=480,
                      focal=600.0, n_frames=n_frames, heights=(1.2, 2.2), walking=True,
                      workers=workers, frame_ids=frame_ids)


def scene_256cube_16cam(seed: int = 2) -> Scene:
    """256^3 grid over a 3.0 m cube, 16 cameras 1280x720 (f = 1200 px), two bodies."""
    return make_scene(seed=seed, grid_n=256, cube_side=3.0, n_cams=16, width=1280, height=720,
                      focal=1200.0, heights=(1.2, 2.2), n_bodies=2)


def _scene_from_kwargs(kw):
    return make_scene(**kw)


def batch_64_specs(seed: int = 64, n_frames: int = 64) -> List[dict]:
    """make_scene arguments of the heterogeneous batch: grids drawn uniformly
    from {96, 128, 160, 192}^3 over a 2.2 m cube, 4-12 cameras, 640x480
    (f = 600 px) or 960x540 (f = 900 px), each frame with its own seed (its
    own rig, background and body pose)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_frames):
        n = int(rng.choice([96, 128, 160, 192]))
        K = int(rng.integers(4, 13))
        W, H, f = (640, 480, 600.0) if rng.random() < 0.5 else (960, 540, 900.0)
        out.append(dict(seed=100 + k, grid_n=n, cube_side=2.2, n_cams=K, width=W, height=H, focal=f))
    return out


def batch_64_scenes(seed: int = 64, n_frames: int = 64, workers: int = 1) -> List[Scene]:
    """The 64 heterogeneous frames of the batched launch (batch_64_specs)."""
    specs = batch_64_specs(seed, n_frames)
    if workers > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(workers, len(specs))) as pool:
            return pool.map(_scene_from_kwargs, specs, chunksize=1)
    return [make_scene(**kw) for kw in specs]
