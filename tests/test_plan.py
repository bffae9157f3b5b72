"""Host planning of the fusion kernels, checked on the CPU.

The kernels skip the per-voxel visibility test where the host planner has
marked a (tile, camera) pair "inside", skip the camera where it is marked
"skip", and the staged kernel copies only the planned image box to shared
memory.  A wrong "inside" or box would read the wrong pixel (or outside the
box), a wrong "skip" would drop a camera, so every record is checked here
against the projection of every voxel centre of its tile, including the
clamped lanes of ragged tiles.  The projection is recomputed in float64 from
the planner's float32 matrices; the planner keeps a margin of one pixel
against the float32 rounding of the kernels.
"""

import os
import subprocess

import numpy as np
import pytest

from paper_1311_6811_gb300 import build as libbuild
from synth import scene as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STAGED, INSIDE, SKIP = 1, 2, 4


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    libbuild.build()
    out = tmp_path_factory.mktemp("plan") / "plan_dump"
    objs = [os.path.join(libbuild.BUILD, f) for f in sorted(os.listdir(libbuild.BUILD)) if f.endswith(".o")]
    subprocess.run([libbuild.nvcc(), *libbuild.ARCH, "-std=c++17", "-I", os.path.join(ROOT, "include"),
                    "-I", libbuild.CSRC, os.path.join(ROOT, "tests", "host", "plan_dump.cu"), *objs,
                    "-o", str(out)], check=True, capture_output=True)
    return str(out)


def _plan(driver, grid, cams, map_dtype, tmp_path, shape=(8, 4, 16, 1)):
    inp = tmp_path / "rig.txt"
    with open(inp, "w") as f:
        f.write(f"{grid.nx} {grid.ny} {grid.nz} {grid.origin[0]!r} {grid.origin[1]!r} {grid.origin[2]!r} "
                f"{grid.voxel_size!r} {len(cams)} {map_dtype} {shape[0]} {shape[1]} {shape[2]} {shape[3]}\n")
        for c in cams:
            vals = np.concatenate([c.K.ravel(), c.R.ravel(), c.t.ravel()])
            f.write(f"{c.width} {c.height} " + " ".join(repr(float(v)) for v in vals) + "\n")
    lines = subprocess.run([driver, str(inp)], capture_output=True, text=True, check=True).stdout.splitlines()
    tx_dim, ty_dim, tz_dim, cap = map(int, lines[0].split())
    n = len(cams)
    M = [np.array(lines[1 + c].split(), dtype=np.float32).astype(np.float64).reshape(3, 4) for c in range(n)]
    recs = [tuple(map(int, l.split())) for l in lines[1 + n:] if l.strip()]
    return (tx_dim, ty_dim, tz_dim, cap), M, recs


def _check(driver, grid, cams, map_dtype, tmp_path, shape=(8, 4, 16, 1)):
    (TX, TY, TZ, cap), M, recs = _plan(driver, grid, cams, map_dtype, tmp_path, shape)
    chunk = 4 if map_dtype == 0 else 8
    W, H = cams[0].width, cams[0].height
    ci, cj, ck = 0.5 * (grid.nx - 1), 0.5 * (grid.ny - 1), 0.5 * (grid.nz - 1)
    assert (TX, TY, TZ) == (shape[0], (32 // shape[0]) * shape[1], shape[2])
    n_tiles = (-(-grid.nx // TX)) * (-(-grid.ny // TY)) * (-(-grid.nz // TZ))
    assert len(recs) == n_tiles * len(cams)
    seen_tiles = set()
    counts = {"inside": 0, "skip": 0, "checked": 0, "staged": 0}
    for tc, c, x0, y0, zf, wf in recs:
        tx, ty, tzi = tc & 0x1FFFFF, (tc >> 21) & 0x1FFFFF, tc >> 42
        seen_tiles.add(tc)
        flags, sh = wf >> 16, wf & 0xFFFF
        sw, cls, nby = zf & 0xFFFF, (zf >> 16) & 3, zf >> 18
        i = np.minimum(tx * TX + np.arange(TX), grid.nx - 1)
        j = np.minimum(ty * TY + np.arange(TY), grid.ny - 1)
        k = np.minimum(tzi * TZ + np.arange(TZ), grid.nz - 1)
        I, J, K = np.meshgrid(i, j, k, indexing="ij")
        P = np.stack([I.ravel() - ci, J.ravel() - cj, K.ravel() - ck, np.ones(I.size)], 1)
        uvw = P @ M[c].T
        w = uvw[:, 2]
        with np.errstate(all="ignore"):
            x, y = uvw[:, 0] / w, uvw[:, 1] / w
        if not flags & STAGED:
            assert zf >> 16 == 0, (tc, c)
        if flags & SKIP:
            counts["skip"] += 1
            assert not flags & (STAGED | INSIDE)
            # nothing seen, and nothing within a pixel of the image either
            near = (w > 0) & (x >= -1) & (x < W + 1) & (y >= -1) & (y < H + 1)
            assert not near.any(), (tc, c)
            continue
        if flags & STAGED:
            counts["staged"] += 1
            assert shape[3] == 1
            # tensor boxes of (32 << cls) x 16 pixels, nby of them stacked, from a
            # 16-byte aligned column; the clipped extent fits the smallest class
            assert x0 >= 0 and y0 >= 0 and x0 % chunk == 0, (tc, c)
            assert x0 + sw <= W and y0 + sh <= H, (tc, c)
            assert cls < 3 and (32 << cls) >= sw and (cls == 0 or (16 << cls) < sw), (tc, c, sw, cls)
            assert nby * 16 >= sh > (nby - 1) * 16 and (32 << cls) * nby * 16 <= cap, (tc, c)
            assert np.all(w > 0), (tc, c)
            seen = (x >= 0) & (x < W) & (y >= 0) & (y < H)
            # every seen centre lies at least half a pixel inside the box
            xs, ys = x[seen], y[seen]
            assert np.all((xs >= x0 + 0.5 * (x0 > 0)) & (xs <= x0 + sw - 0.5 * (x0 + sw < W)) &
                          (ys >= y0 + 0.5 * (y0 > 0)) & (ys <= y0 + sh - 0.5 * (y0 + sh < H))), (tc, c)
        if flags & INSIDE:
            counts["inside"] += 1
            assert np.all(w > 0), (tc, c)
            margin = min(x.min(), W - x.max(), y.min(), H - y.max())
            assert margin >= 0.5, (tc, c, margin)
        else:
            counts["checked"] += 1
    assert len(seen_tiles) == n_tiles
    return counts


RIGS = {
    "64cube_4cam_320x240": lambda: S.scene_64cube_4cam(seed=0),
    "48cube_5cam_200x150": lambda: S.make_scene(seed=8, grid_n=48, cube_side=2.0, n_cams=5, width=200,
                                                height=150, focal=190.0),
    "cameras_inside_8m_grid": lambda: S.make_scene(seed=14, grid_n=48, cube_side=8.0, n_cams=4, width=160,
                                                   height=120, focal=150.0),
}


@pytest.mark.parametrize("rig", sorted(RIGS))
@pytest.mark.parametrize("shape", [(8, 4, 16, 1), (16, 4, 8, 1), (32, 4, 8, 0), (8, 4, 4, 0)])
def test_records_cover_every_voxel(driver, rig, shape, tmp_path):
    sc = RIGS[rig]()
    counts = _check(driver, sc.grid, sc.cams, 0, tmp_path, shape)
    assert counts["inside"] > 0
    assert (counts["staged"] > 0) == (shape[3] == 1)


def test_records_f16_staging(driver, tmp_path):
    sc = RIGS["64cube_4cam_320x240"]()
    counts = _check(driver, sc.grid, sc.cams, 1, tmp_path, (8, 4, 16, 1))
    assert counts["staged"] > 0


@pytest.mark.parametrize("shape", [(8, 4, 16, 1), (32, 4, 8, 1)])
@pytest.mark.parametrize("width", [101, 104])
def test_records_ragged_grid(driver, shape, width, tmp_path):
    """Ragged in every tile dimension; 101-pixel rows are not 16-byte aligned,
    so nothing may be staged there."""
    cams = S.ring_cameras(np.random.default_rng(3), 3, width, 77, 95.0, (0.0, 0.0, 1.0))
    counts = _check(driver, S.Grid(37, 29, 23, (-0.9, -0.7, 0.1), 0.05), cams, 0, tmp_path, shape)
    assert counts["inside"] > 0
    assert (counts["staged"] > 0) == (width == 104)


def test_unsupported_shape_is_refused(driver, tmp_path):
    cams = S.ring_cameras(np.random.default_rng(3), 2, 64, 48, 60.0, (0.0, 0.0, 1.0))
    with pytest.raises(subprocess.CalledProcessError):
        _plan(driver, S.Grid(8, 8, 8, (-0.2, -0.2, 0.8), 0.05), cams, 0, tmp_path, (12, 4, 8, 0))


@pytest.mark.slow
def test_records_128cube_8cam(driver, tmp_path):
    sc = S.scene_128cube_8cam(seed=1, n_frames=1)
    counts = _check(driver, sc.grid, sc.cams, 0, tmp_path)
    assert counts["inside"] > 0.8 * (counts["inside"] + counts["checked"] + counts["skip"])
