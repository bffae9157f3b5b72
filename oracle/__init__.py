"""FP64 CPU oracle for probabilistic shape-from-silhouette (test infrastructure).

The arithmetic lives in `psfs_oracle.c` (plain C, double precision), compiled
here with gcc and called through ctypes.  This package is for the test suite,
the smoke check and the CPU-baseline leg of the benchmark only; the CUDA
library never imports it and shares nothing with it.

Inputs are numpy arrays; grids and cameras may be objects or dicts with the
fields (nx, ny, nz, origin, voxel_size) and (width, height, K, R, t).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "psfs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_f32p = ctypes.POINTER(ctypes.c_float)
_i32p = ctypes.POINTER(ctypes.c_int)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, IEEE double, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-std=c11", "-shared",
           "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_slm.argtypes = [ctypes.c_int64, _u8p, _f32p, _f32p, ctypes.c_double, _dp]
            lib.oracle_slm.restype = None
            lib.oracle_edges.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _u8p, _u8p]
            lib.oracle_edges.restype = None
            lib.oracle_particle_weights.argtypes = [ctypes.c_int, _i32p, _dp, _u8p, ctypes.c_int64, ctypes.c_int,
                                                    _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp,
                                                    _i32p]
            lib.oracle_particle_weights.restype = None
            lib.oracle_reproject.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double,
                                             ctypes.c_int, _i32p, _dp, ctypes.c_int64, _u32p, ctypes.c_double,
                                             _u8p]
            lib.oracle_reproject.restype = None
            lib.oracle_smooth.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double, _dp,
                                          _u8p]
            lib.oracle_smooth.restype = None
            lib.oracle_surface.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _u8p, _u32p]
            lib.oracle_surface.restype = ctypes.c_int64
            lib.oracle_project.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, _i32p, _i32p,
                                           _dp, _dp]
            lib.oracle_project.restype = ctypes.c_int
            lib.oracle_fuse.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp,
                                        ctypes.c_double, ctypes.c_int, _i32p, _dp, _dp,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, _dp, _dp, _u8p, _u8p,
                                        _u8p]
            lib.oracle_fuse.restype = None
            lib.oracle_compact.argtypes = [ctypes.c_int64, _u8p, _u32p]
            lib.oracle_compact.restype = ctypes.c_int64
            lib.oracle_backward_slm.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp,
                                                ctypes.c_double, ctypes.c_int, _i32p, _dp, _dp,
                                                ctypes.c_double, ctypes.c_double,
                                                ctypes.c_double, _dp, _dp]
            lib.oracle_backward_slm.restype = None
            lib.oracle_backward_background.argtypes = [ctypes.c_int64, _u8p, _f32p, _f32p, _dp,
                                                       _dp, _dp, _dp]
            lib.oracle_backward_background.restype = None
            _i64p = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_fuse_subset.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double,
                                               ctypes.c_int, _i32p, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_int64, _i64p, _dp]
            lib.oracle_fuse_subset.restype = None
            lib.oracle_voxel_pixels.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double,
                                                ctypes.c_int, _i32p, _dp, _i32p]
            lib.oracle_voxel_pixels.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _get(o, name):
    return o[name] if isinstance(o, dict) else getattr(o, name)


def _grid_args(grid):
    origin = np.ascontiguousarray(np.asarray(_get(grid, "origin"), dtype=np.float64))
    return (int(_get(grid, "nx")), int(_get(grid, "ny")), int(_get(grid, "nz")), origin,
            float(_get(grid, "voxel_size")))


def _cam_args(cams):
    wh = np.array([[int(_get(c, "width")), int(_get(c, "height"))] for c in cams],
                  dtype=np.int32).reshape(-1)
    rec = np.array([np.concatenate([np.asarray(_get(c, "K"), np.float64).ravel(),
                                    np.asarray(_get(c, "R"), np.float64).ravel(),
                                    np.asarray(_get(c, "t"), np.float64).ravel()])
                    for c in cams], dtype=np.float64).reshape(-1)
    return np.ascontiguousarray(wh), np.ascontiguousarray(rec)


def _param(params, name, default=None):
    if params is None:
        return default
    if isinstance(params, dict):
        return params.get(name, default)
    return getattr(params, name, default)


def slm(images: np.ndarray, mean: np.ndarray, var: np.ndarray,
        log_fg_density: float = -3.0 * np.log(256.0)) -> np.ndarray:
    """Silhouette likelihood map (Eq. 1-2), float64 with the images' leading shape."""
    lib = _load()
    img = np.ascontiguousarray(images, dtype=np.uint8)
    mu = np.ascontiguousarray(mean, dtype=np.float32)
    va = np.ascontiguousarray(var, dtype=np.float32)
    assert img.shape == mu.shape == va.shape and img.shape[-1] == 3
    out = np.empty(img.shape[:-1], dtype=np.float64)
    lib.oracle_slm(int(out.size), _ptr(img, _u8p), _ptr(mu, _f32p), _ptr(va, _f32p),
                   float(log_fg_density), _ptr(out, _dp))
    return out


def project(cam, X):
    """(visible, (px, py), (x, y), w) for a world point X, FP64."""
    lib = _load()
    wh, rec = _cam_args([cam])
    Xa = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    px = ctypes.c_int(-1)
    py = ctypes.c_int(-1)
    xy = np.zeros(2)
    w = np.zeros(1)
    vis = lib.oracle_project(_ptr(rec, _dp), int(wh[0]), int(wh[1]), _ptr(Xa, _dp),
                             ctypes.byref(px), ctypes.byref(py), _ptr(xy, _dp), _ptr(w, _dp))
    return bool(vis), (px.value, py.value), (float(xy[0]), float(xy[1])), float(w[0])


def fuse(grid, cams, slm_maps: np.ndarray, params=None, edge_eps: float = 1e-3) -> dict:
    """Voxel posterior (Eq. 3-9) from per-camera SLM maps (list or stacked array)."""
    lib = _load()
    nx, ny, nz, origin, vs = _grid_args(grid)
    wh, rec = _cam_args(cams)
    if isinstance(slm_maps, (list, tuple)):
        flat = np.concatenate([np.asarray(m, np.float64).ravel() for m in slm_maps])
    else:
        flat = np.asarray(slm_maps, np.float64).ravel()
    flat = np.ascontiguousarray(flat)
    expect = int(sum(int(wh[2 * c]) * int(wh[2 * c + 1]) for c in range(len(cams))))
    assert flat.size == expect, (flat.size, expect)
    nv = nx * ny * nz
    occ = np.empty(nv)
    lo = np.empty(nv)
    occupied = np.empty(nv, np.uint8)
    boundary = np.empty(nv, np.uint8)
    n_seen = np.empty(nv, np.uint8)
    lib.oracle_fuse(nx, ny, nz, _ptr(origin, _dp), vs, len(cams), _ptr(wh, _i32p),
                    _ptr(rec, _dp), _ptr(flat, _dp),
                    float(_param(params, "p_detect", 0.9)),
                    float(_param(params, "p_false_alarm", 0.1)),
                    float(_param(params, "prior", 0.5)),
                    float(_param(params, "threshold", 0.5)), float(edge_eps),
                    _ptr(occ, _dp), _ptr(lo, _dp), _ptr(occupied, _u8p), _ptr(boundary, _u8p),
                    _ptr(n_seen, _u8p))
    lst = np.empty(int(occupied.sum()), np.uint32)
    n = lib.oracle_compact(nv, _ptr(occupied, _u8p), _ptr(lst, _u32p) if lst.size else None)
    assert n == lst.size
    return {"occ": occ, "logodds": lo, "occupied": occupied.astype(bool),
            "boundary": boundary.astype(bool), "n_seen": n_seen, "list": lst}


def edges(masks) -> np.ndarray:
    """Edge maps of silhouettes [n_cams][H][W]: set pixels with a 4-neighbour
    inside the image that is not set."""
    lib = _load()
    m = np.ascontiguousarray(np.asarray(masks) != 0, dtype=np.uint8)
    out = np.empty_like(m)
    lib.oracle_edges(m.shape[0], m.shape[2], m.shape[1], _ptr(m, _u8p), _ptr(out, _u8p))
    return out


def particle_weights(cams, masks, cylinders, kt: int = 8, kw: int = 4, edge_eps: float = 1e-3) -> dict:
    """Tracker weights (Eq. 14-16) of particles = cylinders [P][n_cyl][7]
    (a xyz, b xyz, r) against silhouettes [n_cams][H][W]: {"weights" [P],
    "terms" [P][n_cams][2] (S_e, S_r), "ambiguous" [P][n_cams]}."""
    lib = _load()
    wh, rec = _cam_args(cams)
    m = np.ascontiguousarray(np.asarray(masks) != 0, dtype=np.uint8)
    cy = np.ascontiguousarray(np.asarray(cylinders, np.float64))
    P, n_cyl = cy.shape[0], cy.shape[1]
    w = np.empty(P)
    terms = np.empty((P, len(cams), 2))
    amb = np.empty((P, len(cams)), np.int32)
    lib.oracle_particle_weights(len(cams), _ptr(wh, _i32p), _ptr(rec, _dp), _ptr(m, _u8p), P, n_cyl,
                                _ptr(cy, _dp), int(kt), int(kw), float(edge_eps), _ptr(w, _dp), _ptr(terms, _dp),
                                _ptr(amb, _i32p))
    return {"weights": w, "terms": terms, "ambiguous": amb}


def reproject(grid, cams, voxel_list, grow: float = 0.0) -> np.ndarray:
    """Silhouettes of the listed voxels: uint8 masks [n_cams][H][W], pixel set
    iff its centre ray meets a listed voxel's cube (grown by `grow` voxel
    sizes) in front of the camera.  Brute force: small cases only."""
    lib = _load()
    nx, ny, nz, origin, vs = _grid_args(grid)
    wh, rec = _cam_args(cams)
    lst = np.ascontiguousarray(np.asarray(voxel_list, np.uint32).ravel())
    H, W = int(wh[1]), int(wh[0])
    masks = np.zeros((len(cams), H, W), np.uint8)
    lib.oracle_reproject(nx, ny, nz, _ptr(origin, _dp), vs, len(cams), _ptr(wh, _i32p), _ptr(rec, _dp),
                         lst.size, _ptr(lst, _u32p) if lst.size else None, float(grow), _ptr(masks, _u8p))
    return masks


def smooth(shape, prob, threshold: float = 0.5) -> dict:
    """3 x 3 x 3 box mean of the voxel probabilities over the neighbours
    inside the grid, then the strict threshold: {"smoothed", "occupied",
    "list"} (ascending linear indices).  `prob` has nx*ny*nz entries in linear
    order i + nx (j + ny k)."""
    lib = _load()
    nx, ny, nz = (int(x) for x in shape)
    p = np.ascontiguousarray(np.asarray(prob, np.float64).ravel())
    assert p.size == nx * ny * nz
    sm = np.empty_like(p)
    occ = np.empty(p.size, np.uint8)
    lib.oracle_smooth(nx, ny, nz, _ptr(p, _dp), float(threshold), _ptr(sm, _dp), _ptr(occ, _u8p))
    return {"smoothed": sm, "occupied": occ.astype(bool), "list": np.flatnonzero(occ).astype(np.uint32)}


def surface(shape, occupied) -> np.ndarray:
    """Inner-voxel removal: ascending linear indices of the occupied voxels
    with a face neighbour that is not occupied (outside the grid counts as not
    occupied).  `shape` = (nx, ny, nz); `occupied` has nx*ny*nz entries in
    linear order i + nx (j + ny k)."""
    lib = _load()
    nx, ny, nz = (int(x) for x in shape)
    occ = np.ascontiguousarray(np.asarray(occupied).ravel() != 0, dtype=np.uint8)
    assert occ.size == nx * ny * nz
    out = np.empty(max(int(occ.sum()), 1), np.uint32)
    n = lib.oracle_surface(nx, ny, nz, _ptr(occ, _u8p), _ptr(out, _u32p))
    return out[:n].copy()


def reconstruct(grid, cams, images, mean, var, params=None, edge_eps: float = 1e-3) -> dict:
    """Whole path: SLM maps (Eq. 1-2), posterior (Eq. 3-9), threshold, list."""
    lfd = _param(params, "log_fg_density", -3.0 * np.log(256.0))
    s = slm(images, mean, var, lfd)
    out = fuse(grid, cams, s, params, edge_eps)
    out["slm"] = s
    return out


def backward_slm(grid, cams, slm_maps, d_occ, params=None) -> np.ndarray:
    """dLoss/dSLM (same shape as the stacked maps) given dLoss/docc per voxel."""
    lib = _load()
    nx, ny, nz, origin, vs = _grid_args(grid)
    wh, rec = _cam_args(cams)
    s = np.ascontiguousarray(np.asarray(slm_maps, np.float64))
    d = np.ascontiguousarray(np.asarray(d_occ, np.float64).ravel())
    assert d.size == nx * ny * nz
    out = np.empty_like(s)
    lib.oracle_backward_slm(nx, ny, nz, _ptr(origin, _dp), vs, len(cams), _ptr(wh, _i32p),
                            _ptr(rec, _dp), _ptr(s, _dp),
                            float(_param(params, "p_detect", 0.9)),
                            float(_param(params, "p_false_alarm", 0.1)),
                            float(_param(params, "prior", 0.5)), _ptr(d, _dp), _ptr(out, _dp))
    return out


def backward_background(images, mean, var, slm_maps, d_slm):
    """(dLoss/dmean, dLoss/dvar) from dLoss/dSLM through Eq. 1-2."""
    lib = _load()
    img = np.ascontiguousarray(images, dtype=np.uint8)
    mu = np.ascontiguousarray(mean, dtype=np.float32)
    va = np.ascontiguousarray(var, dtype=np.float32)
    s = np.ascontiguousarray(np.asarray(slm_maps, np.float64))
    ds = np.ascontiguousarray(np.asarray(d_slm, np.float64))
    dm = np.empty(img.shape, np.float64)
    dv = np.empty(img.shape, np.float64)
    lib.oracle_backward_background(int(s.size), _ptr(img, _u8p), _ptr(mu, _f32p),
                                   _ptr(va, _f32p), _ptr(s, _dp), _ptr(ds, _dp),
                                   _ptr(dm, _dp), _ptr(dv, _dp))
    return dm, dv


def backward(grid, cams, images, mean, var, d_occ, params=None):
    """(d_slm, d_mean, d_var) for a loss with gradient d_occ on the occupancy."""
    lfd = _param(params, "log_fg_density", -3.0 * np.log(256.0))
    s = slm(images, mean, var, lfd)
    ds = backward_slm(grid, cams, s, d_occ, params)
    dm, dv = backward_background(images, mean, var, s, ds)
    return ds, dm, dv


def fuse_subset(grid, cams, slm_maps, voxels, params=None) -> np.ndarray:
    """Posterior (Eq. 3-4) of the listed voxels only, FP64."""
    lib = _load()
    nx, ny, nz, origin, vs = _grid_args(grid)
    wh, rec = _cam_args(cams)
    flat = np.ascontiguousarray(np.asarray(slm_maps, np.float64).ravel())
    idx = np.ascontiguousarray(np.asarray(voxels, np.int64))
    out = np.empty(idx.size)
    lib.oracle_fuse_subset(nx, ny, nz, _ptr(origin, _dp), vs, len(cams), _ptr(wh, _i32p), _ptr(rec, _dp),
                           _ptr(flat, _dp), float(_param(params, "p_detect", 0.9)),
                           float(_param(params, "p_false_alarm", 0.1)), float(_param(params, "prior", 0.5)),
                           int(idx.size), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(out, _dp))
    return out


def voxel_pixels(grid, cams) -> np.ndarray:
    """int32 [n_cams][n_vox]: pixel offset of each voxel centre, -1 if unseen."""
    lib = _load()
    nx, ny, nz, origin, vs = _grid_args(grid)
    wh, rec = _cam_args(cams)
    out = np.empty((len(cams), nx * ny * nz), np.int32)
    lib.oracle_voxel_pixels(nx, ny, nz, _ptr(origin, _dp), vs, len(cams), _ptr(wh, _i32p), _ptr(rec, _dp),
                            _ptr(out, _i32p))
    return out
