"""ctypes binding of libpsfs (include/psfs.h), one Python function per C entry
point, same names.  Marshalling only: tensors become device pointers, structs
become ctypes structs, statuses become exceptions.  Every step of the
reconstruction runs in the CUDA library; if it cannot be loaded, the calls
raise instead of falling back to anything else.

Device arguments accept CUDA torch tensors (contiguous, the dtype and shape
given in the header) or raw integer pointers.
"""

from __future__ import annotations

import ctypes
import math
import os
import threading
from typing import Optional, Sequence

import numpy as np

from . import build as _build

PSFS_MAX_CAMS = 32

PSFS_OK = 0
PSFS_ERR_INVALID_ARG = 1
PSFS_ERR_NOT_READY = 2
PSFS_ERR_CAPACITY = 3
PSFS_ERR_CUDA = 4
PSFS_ERR_TIMEOUT = 5
PSFS_ERR_NOMEM = 6
PSFS_ERR_BOUNDS = 7

PSFS_MAP_F32 = 0
PSFS_MAP_F16 = 1
PSFS_MAP_BF16 = 2
MAP_DTYPES = {"f32": PSFS_MAP_F32, "f16": PSFS_MAP_F16, "bf16": PSFS_MAP_BF16}


class psfs_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("origin", ctypes.c_double * 3), ("voxel_size", ctypes.c_double)]


class psfs_camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("K", ctypes.c_double * 9), ("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3)]


class psfs_params(ctypes.Structure):
    _fields_ = [("p_detect", ctypes.c_double), ("p_false_alarm", ctypes.c_double),
                ("prior", ctypes.c_double), ("threshold", ctypes.c_double),
                ("log_fg_density", ctypes.c_double), ("map_dtype", ctypes.c_int32)]


class psfs_fuse_config(ctypes.Structure):
    _fields_ = [("lanes_x", ctypes.c_int32), ("warps", ctypes.c_int32), ("voxels_z", ctypes.c_int32),
                ("staged", ctypes.c_int32), ("seq_likelihood_ctas", ctypes.c_int32),
                ("frames_per_group", ctypes.c_int32), ("cameras_per_block", ctypes.c_int32),
                ("seq_lanes_x", ctypes.c_int32), ("seq_voxels_z", ctypes.c_int32),
                ("seq_record_bytes", ctypes.c_int32), ("batch_launch", ctypes.c_int32)]

    def as_tuple(self):
        return (self.lanes_x, self.warps, self.voxels_z, self.staged)


# candidate order of psfs_autotune's timings (PSFS_N_FUSE_CANDIDATES)
FUSE_CONFIGS = ([(lx, 4, tz, 0) for lx in (8, 16, 32) for tz in (2, 4, 8, 16)] +
                [(lx, 4, tz, 1) for lx in (8, 16, 32) for tz in (8, 16)])


class psfs_frame(ctypes.Structure):
    _fields_ = [("handle", ctypes.c_void_p), ("images", ctypes.c_void_p), ("occupancy", ctypes.c_void_p),
                ("voxel_list", ctypes.c_void_p), ("capacity", ctypes.c_uint32), ("count", ctypes.c_void_p)]


class PsfsError(RuntimeError):
    def __init__(self, status: int, func: str, message: str):
        self.status = status
        super().__init__(f"{func}: {_status_name(status)} ({message})")


_lock = threading.Lock()
_lib = None
_vp = ctypes.c_void_p


def lib_path() -> str:
    """The library this process loads: the bounds-checked build when the
    environment sets PSFS_BOUNDS_CHECK=1, else the product build."""
    return _build.BOUNDS_LIB if os.environ.get("PSFS_BOUNDS_CHECK") == "1" else _build.LIB


def load(build_if_missing: bool = True):
    """Load libpsfs.so (building it first if it is missing and nvcc exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise OSError(f"libpsfs.so not built ({path})")
            _build.build(bounds_check=path == _build.BOUNDS_LIB)
        lib = ctypes.CDLL(path)
        st = ctypes.c_int
        sig = {
            "psfs_params_default": (None, [ctypes.POINTER(psfs_params)]),
            "psfs_create": (st, [ctypes.POINTER(psfs_grid), ctypes.POINTER(psfs_camera), ctypes.c_int32,
                                 ctypes.POINTER(psfs_params), _vp, ctypes.POINTER(_vp)]),
            "psfs_set_background": (st, [_vp, _vp, _vp]),
            "psfs_reconstruct": (st, [_vp, _vp, _vp, _vp, ctypes.c_uint32, _vp]),
            "psfs_reconstruct_host": (st, [_vp, _vp, _vp, _vp, ctypes.c_uint32, _vp]),
            "psfs_reconstruct_sequence": (st, [_vp, ctypes.c_int32, _vp, _vp, _vp, ctypes.c_uint32, _vp]),
            "psfs_reconstruct_sequence_host": (st, [_vp, ctypes.c_int32, _vp, _vp, _vp, ctypes.c_uint32, _vp]),
            "psfs_surface": (st, [_vp, ctypes.c_int32, _vp, ctypes.c_uint32, _vp, _vp, ctypes.c_uint32, _vp]),
            "psfs_smooth": (st, [_vp, ctypes.c_int32, _vp, _vp, _vp, ctypes.c_uint32, _vp]),
            "psfs_reproject": (st, [_vp, ctypes.c_int32, _vp, ctypes.c_uint32, _vp, _vp]),
            "psfs_particle_weights": (st, [_vp, ctypes.c_int32, ctypes.c_int32, _vp, ctypes.c_int32, ctypes.c_int32,
                                           _vp, _vp, _vp]),
            "psfs_set_background_l2": (st, [_vp, ctypes.c_int32]),
            "psfs_fuse_slm": (st, [_vp, _vp, _vp, _vp, ctypes.c_uint32, _vp]),
            "psfs_get_likelihood": (st, [_vp, _vp, _vp]),
            "psfs_get_log_ratio": (st, [_vp, _vp, _vp]),
            "psfs_backward": (st, [_vp, _vp, _vp, _vp, _vp, _vp]),
            "psfs_backward_sequence": (st, [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp]),
            "psfs_backward_from_occupancy": (st, [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp]),
            "psfs_backward_slm": (st, [_vp, _vp, _vp, _vp]),
            "psfs_reconstruct_noalloc": (st, [ctypes.POINTER(psfs_grid), ctypes.POINTER(psfs_camera),
                                              ctypes.c_int32, ctypes.POINTER(psfs_params), _vp, _vp, _vp,
                                              _vp, _vp, ctypes.c_uint32, _vp, _vp]),
            "psfs_gather_rows": (st, [_vp, ctypes.c_int64, ctypes.c_int32, _vp, ctypes.c_int64, _vp, _vp]),
            "psfs_sync": (st, [_vp]),
            "psfs_destroy": (None, [_vp]),
            "psfs_set_fuse_config": (st, [_vp, ctypes.POINTER(psfs_fuse_config)]),
            "psfs_get_fuse_config": (st, [_vp, ctypes.POINTER(psfs_fuse_config)]),
            "psfs_autotune": (st, [_vp, _vp, ctypes.c_int32, ctypes.POINTER(psfs_fuse_config),
                                   ctypes.POINTER(ctypes.c_float)]),
            "psfs_tune_cache_save": (st, [ctypes.c_char_p]),
            "psfs_tune_cache_load": (st, [ctypes.c_char_p]),
            "psfs_tune_cache_clear": (None, []),
            "psfs_tune_cache_entries": (ctypes.c_int32, []),
            "psfs_batch_create": (st, [ctypes.POINTER(psfs_frame), ctypes.c_int32, _vp, ctypes.POINTER(_vp)]),
            "psfs_batch_run": (st, [_vp]),
            "psfs_batch_sync": (st, [_vp]),
            "psfs_batch_set_config": (st, [_vp, ctypes.POINTER(psfs_fuse_config)]),
            "psfs_batch_autotune": (st, [_vp, ctypes.c_int32, ctypes.POINTER(psfs_fuse_config),
                                         ctypes.POINTER(ctypes.c_float)]),
            "psfs_batch_set_wait_limit": (st, [_vp, ctypes.c_uint64, ctypes.c_int32]),
            "psfs_batch_destroy": (None, [_vp]),
            "psfs_profile_enable": (st, [_vp, ctypes.c_int32]),
            "psfs_profile_read": (st, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]),
            "psfs_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "psfs_last_error_message": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _status_name(s: int) -> str:
    try:
        return load().psfs_status_string(s).decode()
    except Exception:  # pragma: no cover - only when the library itself is missing
        return f"status {s}"


def _check(status: int, func: str):
    if status != PSFS_OK:
        msg = load().psfs_last_error_message().decode(errors="replace")
        raise PsfsError(status, func, msg)


def _dev_ptr(x, name: str, dtype=None, numel: Optional[int] = None):
    """Device pointer of a CUDA tensor (checked) or a raw integer / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    import torch
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"{name}: expected a CUDA tensor or an int pointer")
    if not x.is_cuda:
        raise ValueError(f"{name}: tensor must be on a CUDA device")
    if not x.is_contiguous():
        raise ValueError(f"{name}: tensor must be contiguous")
    if dtype is not None and x.dtype != dtype:
        raise ValueError(f"{name}: expected dtype {dtype}, got {x.dtype}")
    if numel is not None and x.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {x.numel()}")
    return x.data_ptr()


def _host_ptr(x, name: str, dtype=None, numel: Optional[int] = None):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{name}: array must be C-contiguous")
        if numel is not None and x.size != numel:
            raise ValueError(f"{name}: expected {numel} elements, got {x.size}")
        return x.ctypes.data
    import torch
    if isinstance(x, torch.Tensor):
        if x.is_cuda or not x.is_contiguous():
            raise ValueError(f"{name}: expected a contiguous host tensor")
        if dtype is not None and x.dtype != dtype:
            raise ValueError(f"{name}: expected dtype {dtype}, got {x.dtype}")
        if numel is not None and x.numel() != numel:
            raise ValueError(f"{name}: expected {numel} elements, got {x.numel()}")
        return x.data_ptr()
    raise TypeError(f"{name}: expected a host array")


# --------------------------------------------------------------------------- #
# struct builders
# --------------------------------------------------------------------------- #
def _get(o, name):
    return o[name] if isinstance(o, dict) else getattr(o, name)


def make_grid(grid) -> psfs_grid:
    g = psfs_grid()
    g.nx, g.ny, g.nz = int(_get(grid, "nx")), int(_get(grid, "ny")), int(_get(grid, "nz"))
    g.origin[:] = [float(v) for v in _get(grid, "origin")]
    g.voxel_size = float(_get(grid, "voxel_size"))
    return g


def make_cameras(cams) -> ctypes.Array:
    arr = (psfs_camera * len(cams))()
    for n, c in enumerate(cams):
        arr[n].width = int(_get(c, "width"))
        arr[n].height = int(_get(c, "height"))
        arr[n].K[:] = [float(v) for v in np.asarray(_get(c, "K"), np.float64).ravel()]
        arr[n].R[:] = [float(v) for v in np.asarray(_get(c, "R"), np.float64).ravel()]
        arr[n].t[:] = [float(v) for v in np.asarray(_get(c, "t"), np.float64).ravel()]
    return arr


def psfs_params_default() -> psfs_params:
    p = psfs_params()
    load().psfs_params_default(ctypes.byref(p))
    return p


def make_params(params=None, map_dtype=None) -> psfs_params:
    p = psfs_params_default()
    if params is not None:
        for name in ("p_detect", "p_false_alarm", "prior", "threshold", "log_fg_density"):
            v = params.get(name) if isinstance(params, dict) else getattr(params, name, None)
            if v is not None:
                setattr(p, name, float(v))
        md = params.get("map_dtype") if isinstance(params, dict) else getattr(params, "map_dtype", None)
        if md is not None:
            p.map_dtype = MAP_DTYPES.get(md, md) if isinstance(md, str) else int(md)
    if map_dtype is not None:
        p.map_dtype = MAP_DTYPES[map_dtype] if isinstance(map_dtype, str) else int(map_dtype)
    return p


# --------------------------------------------------------------------------- #
# entry points (names of include/psfs.h)
# --------------------------------------------------------------------------- #
def psfs_create(grid, cams, params=None, stream=None, map_dtype=None) -> int:
    """Returns the handle (an integer pointer).  `stream` is a torch CUDA stream,
    an integer cudaStream_t or None (the current torch stream)."""
    lib = load()
    g = make_grid(grid) if not isinstance(grid, psfs_grid) else grid
    c = make_cameras(cams) if not isinstance(cams, ctypes.Array) else cams
    p = params if isinstance(params, psfs_params) else make_params(params, map_dtype)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    out = _vp()
    _check(lib.psfs_create(ctypes.byref(g), c, len(c), ctypes.byref(p), _vp(stream), ctypes.byref(out)),
           "psfs_create")
    return out.value


def psfs_set_background(h: int, mean, var):
    import torch
    _check(load().psfs_set_background(h, _dev_ptr(mean, "mean", torch.float32),
                                      _dev_ptr(var, "var", torch.float32)), "psfs_set_background")


def psfs_reconstruct(h: int, images, occupancy, voxel_list, capacity: int, count):
    import torch
    _check(load().psfs_reconstruct(h, _dev_ptr(images, "images", torch.uint8),
                                   _dev_ptr(occupancy, "occupancy", torch.float32),
                                   _dev_ptr(voxel_list, "voxel_list"), int(capacity),
                                   _dev_ptr(count, "count")), "psfs_reconstruct")


def psfs_reconstruct_sequence(h: int, n_frames: int, images, occupancy, voxel_lists, capacity: int, counts):
    """n_frames frames in one call; tensors hold the frames back to back."""
    import torch
    _check(load().psfs_reconstruct_sequence(h, int(n_frames), _dev_ptr(images, "images", torch.uint8),
                                            _dev_ptr(occupancy, "occupancy", torch.float32),
                                            _dev_ptr(voxel_lists, "voxel_lists"), int(capacity),
                                            _dev_ptr(counts, "counts")), "psfs_reconstruct_sequence")


def psfs_set_background_l2(h: int, enable: bool = True):
    _check(load().psfs_set_background_l2(h, int(bool(enable))), "psfs_set_background_l2")


def psfs_reconstruct_host(h: int, images, occupancy, voxel_list, capacity: int, count) -> int:
    """Host buffers (numpy arrays or CPU tensors, pinned for speed).  Returns the
    status code: PSFS_OK or PSFS_ERR_CAPACITY (anything else raises)."""
    st = load().psfs_reconstruct_host(h, _host_ptr(images, "images"), _host_ptr(occupancy, "occupancy"),
                                      _host_ptr(voxel_list, "voxel_list"), int(capacity),
                                      _host_ptr(count, "count"))
    if st not in (PSFS_OK, PSFS_ERR_CAPACITY):
        _check(st, "psfs_reconstruct_host")
    return st


def psfs_reconstruct_sequence_host(h: int, n_frames: int, images, occupancy, voxel_lists, capacity: int,
                                   counts) -> int:
    """n_frames frames from and to host buffers (numpy arrays or CPU tensors,
    pinned for speed; occupancy may be None).  Returns PSFS_OK or
    PSFS_ERR_CAPACITY (anything else raises)."""
    st = load().psfs_reconstruct_sequence_host(h, int(n_frames), _host_ptr(images, "images"),
                                               _host_ptr(occupancy, "occupancy") if occupancy is not None else None,
                                               _host_ptr(voxel_lists, "voxel_lists"), int(capacity),
                                               _host_ptr(counts, "counts"))
    if st not in (PSFS_OK, PSFS_ERR_CAPACITY):
        _check(st, "psfs_reconstruct_sequence_host")
    return st


def psfs_particle_weights(h: int, cylinders, masks, weights, terms=None, kt: int = 8, kw: int = 4):
    """Tracker weights (Eq. 14-16) of particles `cylinders` f32 [P][n_cyl][7]
    against silhouettes `masks` uint8 [n_cams][H][W]; writes `weights` [P]
    and, if given, `terms` [P][n_cams][2] (S_e, S_r)."""
    import torch
    P, n_cyl = int(cylinders.shape[0]), int(cylinders.shape[1])
    _check(load().psfs_particle_weights(h, P, n_cyl, _dev_ptr(cylinders, "cylinders", torch.float32), int(kt),
                                        int(kw), _dev_ptr(masks, "masks", torch.uint8),
                                        _dev_ptr(weights, "weights", torch.float32),
                                        _dev_ptr(terms, "terms", torch.float32) if terms is not None else None),
           "psfs_particle_weights")


def psfs_reproject(h: int, n_frames: int, voxel_lists, list_stride: int, counts, masks):
    """Silhouettes of the listed voxels: masks uint8 [n_frames][n_cams][H][W]."""
    import torch
    _check(load().psfs_reproject(h, int(n_frames), _dev_ptr(voxel_lists, "voxel_lists"), int(list_stride),
                                 _dev_ptr(counts, "counts"), _dev_ptr(masks, "masks", torch.uint8)),
           "psfs_reproject")


def psfs_smooth(h: int, n_frames: int, occupancy, smoothed, voxel_lists, capacity: int, counts):
    """Smoothing (3 x 3 x 3 box mean over in-grid neighbours) of n_frames
    posterior grids, strict threshold and compaction; `smoothed` may be None."""
    import torch
    _check(load().psfs_smooth(h, int(n_frames), _dev_ptr(occupancy, "occupancy", torch.float32),
                              _dev_ptr(smoothed, "smoothed", torch.float32) if smoothed is not None else None,
                              _dev_ptr(voxel_lists, "voxel_lists"), int(capacity), _dev_ptr(counts, "counts")),
           "psfs_smooth")


def psfs_surface(h: int, n_frames: int, voxel_lists, list_stride: int, counts, surface_lists,
                 surface_capacity: int, surface_counts):
    """Inner-voxel removal on the device: frame f's surface voxels (listed
    voxels with a face neighbour not listed) from its occupied-voxel list."""
    _check(load().psfs_surface(h, int(n_frames), _dev_ptr(voxel_lists, "voxel_lists"), int(list_stride),
                               _dev_ptr(counts, "counts"), _dev_ptr(surface_lists, "surface_lists"),
                               int(surface_capacity), _dev_ptr(surface_counts, "surface_counts")), "psfs_surface")


def psfs_fuse_slm(h: int, slm, occupancy, voxel_list, capacity: int, count):
    import torch
    _check(load().psfs_fuse_slm(h, _dev_ptr(slm, "slm", torch.float32),
                                _dev_ptr(occupancy, "occupancy", torch.float32),
                                _dev_ptr(voxel_list, "voxel_list"), int(capacity),
                                _dev_ptr(count, "count")), "psfs_fuse_slm")


def psfs_get_likelihood(h: int, images, slm_out):
    import torch
    _check(load().psfs_get_likelihood(h, _dev_ptr(images, "images", torch.uint8),
                                      _dev_ptr(slm_out, "slm_out", torch.float32)), "psfs_get_likelihood")


def psfs_get_log_ratio(h: int, images, map_out):
    """The stored log-ratio maps of `images` in the handle's map dtype
    (map_out: contiguous CUDA tensor of n_cams * H * W float32 / float16 /
    bfloat16 elements)."""
    import torch
    _check(load().psfs_get_log_ratio(h, _dev_ptr(images, "images", torch.uint8),
                                     _dev_ptr(map_out, "map_out")), "psfs_get_log_ratio")


def psfs_backward(h: int, images, d_occ, d_slm=None, d_mean=None, d_var=None):
    import torch
    _check(load().psfs_backward(h, _dev_ptr(images, "images", torch.uint8),
                                _dev_ptr(d_occ, "d_occ", torch.float32),
                                _dev_ptr(d_slm, "d_slm", torch.float32),
                                _dev_ptr(d_mean, "d_mean", torch.float32),
                                _dev_ptr(d_var, "d_var", torch.float32)), "psfs_backward")


def psfs_backward_sequence(h: int, n_frames: int, images, d_occ, d_slm=None, d_mean=None, d_var=None):
    """Adjoint of n_frames frames (see include/psfs.h): d_slm per frame,
    d_mean and d_var summed over the frames in frame order."""
    import torch
    _check(load().psfs_backward_sequence(h, int(n_frames), _dev_ptr(images, "images", torch.uint8),
                                         _dev_ptr(d_occ, "d_occ", torch.float32),
                                         _dev_ptr(d_slm, "d_slm", torch.float32),
                                         _dev_ptr(d_mean, "d_mean", torch.float32),
                                         _dev_ptr(d_var, "d_var", torch.float32)), "psfs_backward_sequence")


def psfs_backward_from_occupancy(h: int, n_frames: int, images, occupancy, d_occ, d_slm=None, d_mean=None,
                                 d_var=None):
    """The adjoint from the forward's occupancy of these frames (no recomputed
    forward); outputs as psfs_backward (one frame) / psfs_backward_sequence."""
    import torch
    _check(load().psfs_backward_from_occupancy(h, int(n_frames), _dev_ptr(images, "images", torch.uint8),
                                               _dev_ptr(occupancy, "occupancy", torch.float32),
                                               _dev_ptr(d_occ, "d_occ", torch.float32),
                                               _dev_ptr(d_slm, "d_slm", torch.float32),
                                               _dev_ptr(d_mean, "d_mean", torch.float32),
                                               _dev_ptr(d_var, "d_var", torch.float32)),
           "psfs_backward_from_occupancy")


PSFS_NOALLOC_MAX_PIXELS = 4 * 1024 * 1024


def psfs_reconstruct_noalloc(grid, cams, params, mean, var, images, occupancy, voxel_list, capacity: int, count,
                             stream=None):
    """One frame without any device allocation (see include/psfs.h); no handle.
    `stream` is a torch CUDA stream, an integer cudaStream_t or None (current).

    The C entry point has no handle that knows the buffer sizes, so this
    wrapper checks every tensor against the sizes the grid and the cameras
    imply, and that each lives on the current CUDA device, before the call:
    an undersized or misplaced buffer would otherwise be an out-of-bounds
    device access."""
    import torch
    g = make_grid(grid) if not isinstance(grid, psfs_grid) else grid
    c = make_cameras(cams) if not isinstance(cams, ctypes.Array) else cams
    p = params if isinstance(params, psfs_params) else make_params(params)
    n_pix = len(c) * int(c[0].width) * int(c[0].height) if len(c) else 0
    n_vox = int(g.nx) * int(g.ny) * int(g.nz)
    dev = torch.cuda.current_device()
    tensors = {"mean": mean, "var": var, "images": images, "occupancy": occupancy, "voxel_list": voxel_list,
               "count": count}
    for name, t in tensors.items():
        if isinstance(t, torch.Tensor) and (not t.is_cuda or t.device.index != dev):
            raise ValueError(f"{name}: tensor must be on the current CUDA device (cuda:{dev})")
    if isinstance(voxel_list, torch.Tensor) and voxel_list.numel() < int(capacity):
        raise ValueError(f"voxel_list: {voxel_list.numel()} entries < capacity {int(capacity)}")
    if isinstance(voxel_list, torch.Tensor) and voxel_list.element_size() != 4:
        raise ValueError("voxel_list: expected 4-byte entries")
    if isinstance(count, torch.Tensor) and (count.numel() < 1 or count.element_size() != 4):
        raise ValueError("count: expected at least one 4-byte element")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    _check(load().psfs_reconstruct_noalloc(ctypes.byref(g), c, len(c), ctypes.byref(p),
                                           _dev_ptr(mean, "mean", torch.float32, n_pix * 3),
                                           _dev_ptr(var, "var", torch.float32, n_pix * 3),
                                           _dev_ptr(images, "images", torch.uint8, n_pix * 3),
                                           _dev_ptr(occupancy, "occupancy", torch.float32, n_vox),
                                           _dev_ptr(voxel_list, "voxel_list"), int(capacity),
                                           _dev_ptr(count, "count"), _vp(stream)), "psfs_reconstruct_noalloc")


def psfs_gather_rows(rows, record_bytes: int, idx, checksum, stream=None):
    """Gathers the rows idx of `rows` (CUDA tensor of whole record_bytes-byte
    rows) with the fusion kernels' loads, XOR-ing every word into checksum
    (int32 CUDA tensor of one element, not cleared); enqueued on `stream`
    (default: torch's current stream)."""
    import torch
    nbytes = rows.numel() * rows.element_size()
    if nbytes % int(record_bytes) != 0:
        raise ValueError("rows: not a whole number of records")
    if checksum.numel() != 1:
        raise ValueError("checksum: expected one element")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    _check(load().psfs_gather_rows(_dev_ptr(rows, "rows"), nbytes // int(record_bytes), int(record_bytes),
                                   _dev_ptr(idx, "idx", torch.int32), idx.numel(), _vp(stream),
                                   _dev_ptr(checksum, "checksum", torch.int32)), "psfs_gather_rows")


def psfs_backward_slm(h: int, slm, d_occ, d_slm):
    import torch
    _check(load().psfs_backward_slm(h, _dev_ptr(slm, "slm", torch.float32), _dev_ptr(d_occ, "d_occ", torch.float32),
                                    _dev_ptr(d_slm, "d_slm", torch.float32)), "psfs_backward_slm")


def psfs_sync(h: int) -> int:
    """Waits for the handle's stream; returns PSFS_OK or PSFS_ERR_CAPACITY."""
    st = load().psfs_sync(h)
    if st not in (PSFS_OK, PSFS_ERR_CAPACITY):
        _check(st, "psfs_sync")
    return st


def psfs_destroy(h: int):
    if h:
        load().psfs_destroy(h)


def psfs_set_fuse_config(h: int, lanes_x: int, warps: int, voxels_z: int, staged: int = 0,
                         seq_likelihood_ctas: int = 0, frames_per_group: int = 0, seq_lanes_x: int = 0,
                         seq_voxels_z: int = 0, seq_record_bytes: int = 0):
    """One-frame tile shape, the sequence path's likelihood CTAs per SM and
    frames per group, (seq_lanes_x, seq_voxels_z > 0) a tile shape of the
    sequence path's own, and (seq_record_bytes 32 or 64) the pixel record of
    its map planes; 0 keeps the current value."""
    cfg = psfs_fuse_config(lanes_x, warps, voxels_z, staged, seq_likelihood_ctas, frames_per_group, 0, seq_lanes_x,
                           seq_voxels_z, seq_record_bytes)
    _check(load().psfs_set_fuse_config(h, ctypes.byref(cfg)), "psfs_set_fuse_config")


def psfs_get_fuse_config(h: int, full: bool = False) -> tuple:
    """(lanes_x, warps, voxels_z, staged), plus (seq_likelihood_ctas,
    frames_per_group, seq_lanes_x, seq_voxels_z, seq_record_bytes) of the
    sequence path when `full` (the argument order of psfs_set_fuse_config)."""
    cfg = psfs_fuse_config()
    _check(load().psfs_get_fuse_config(h, ctypes.byref(cfg)), "psfs_get_fuse_config")
    return cfg.as_tuple() + ((cfg.seq_likelihood_ctas, cfg.frames_per_group, cfg.seq_lanes_x, cfg.seq_voxels_z,
                              cfg.seq_record_bytes) if full else ())


def psfs_autotune(h: int, images, reps: int = 5, timings: Optional[dict] = None) -> tuple:
    """Times every fuse tile shape on `images`, keeps and returns the fastest;
    fills `timings` {config tuple: mean ms} if given."""
    import torch
    cfg = psfs_fuse_config()
    ms = (ctypes.c_float * len(FUSE_CONFIGS))()
    _check(load().psfs_autotune(h, _dev_ptr(images, "images", torch.uint8), int(reps), ctypes.byref(cfg), ms),
           "psfs_autotune")
    if timings is not None:
        for c, t in zip(FUSE_CONFIGS, ms):
            timings[c] = float(t)
    return cfg.as_tuple()


def psfs_tune_cache_save(path: str):
    """Writes the autotuner's remembered choices (per grid size, camera
    count, image size and map type) to a text file."""
    _check(load().psfs_tune_cache_save(os.fsencode(path)), "psfs_tune_cache_save")


def psfs_tune_cache_load(path: str):
    """Adds the choices of a file written by psfs_tune_cache_save; handles
    created afterwards start with them.  Raises PsfsError (nothing changed)
    on an invalid file."""
    _check(load().psfs_tune_cache_load(os.fsencode(path)), "psfs_tune_cache_load")


def psfs_tune_cache_clear():
    load().psfs_tune_cache_clear()


def psfs_tune_cache_entries() -> int:
    return int(load().psfs_tune_cache_entries())


def psfs_batch_create(frames, stream=None) -> int:
    """`frames`: list of dicts/tuples (handle, images, occupancy, voxel_list,
    capacity, count) with CUDA tensors; returns the batch (an int pointer)."""
    import torch
    arr = (psfs_frame * len(frames))()
    for n, fr in enumerate(frames):
        if isinstance(fr, dict):
            fr = (fr["handle"], fr["images"], fr["occupancy"], fr["voxel_list"], fr["capacity"], fr["count"])
        h, img, occ, lst, cap, cnt = fr
        arr[n].handle = h
        arr[n].images = _dev_ptr(img, "images", torch.uint8)
        arr[n].occupancy = _dev_ptr(occ, "occupancy", torch.float32)
        arr[n].voxel_list = _dev_ptr(lst, "voxel_list")
        arr[n].capacity = int(cap)
        arr[n].count = _dev_ptr(cnt, "count")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    out = _vp()
    _check(load().psfs_batch_create(arr, len(frames), _vp(stream), ctypes.byref(out)), "psfs_batch_create")
    return out.value


def psfs_batch_run(b: int):
    _check(load().psfs_batch_run(b), "psfs_batch_run")


def psfs_batch_sync(b: int) -> int:
    st = load().psfs_batch_sync(b)
    if st not in (PSFS_OK, PSFS_ERR_CAPACITY):
        _check(st, "psfs_batch_sync")
    return st


# candidate order of psfs_batch_autotune: (lanes_x, warps, voxels_z, staged,
# cameras_per_block, batch_launch); the last one is the graph of per-frame
# launches, whose tile shapes are each frame handle's own
FRAME_LAUNCH = (0, 0, 0, 0, 0, 1)
BATCH_CONFIGS = ([(lx, 4, tz, 0, 1, 0) for lx in (8, 16, 32) for tz in (8, 16)] +
                 [(lx, 4, tz, 0, 2, 0) for lx in (8, 16) for tz in (4, 8)] +
                 [(lx, 4, 4, 0, 4, 0) for lx in (8, 16)] + [FRAME_LAUNCH])


def psfs_batch_set_config(b: int, lanes_x: int, warps: int, voxels_z: int, cameras_per_block: int = 1,
                          launch: int = 0):
    """The persistent kernel's tile shape and camera block (launch 0), or the
    graph of per-frame launches (launch 1; the shape is then not used)."""
    cfg = psfs_fuse_config(lanes_x, warps, voxels_z, 0, 0, 0, cameras_per_block)
    cfg.batch_launch = int(launch)
    _check(load().psfs_batch_set_config(b, ctypes.byref(cfg)), "psfs_batch_set_config")


def psfs_batch_autotune(b: int, reps: int = 3, timings: Optional[dict] = None) -> tuple:
    """Times every batch candidate; returns the chosen one as in
    BATCH_CONFIGS."""
    cfg = psfs_fuse_config()
    ms = (ctypes.c_float * len(BATCH_CONFIGS))()
    _check(load().psfs_batch_autotune(b, int(reps), ctypes.byref(cfg), ms), "psfs_batch_autotune")
    if timings is not None:
        for c, t in zip(BATCH_CONFIGS, ms):
            timings[c] = float(t)
    if cfg.batch_launch == 1:
        return FRAME_LAUNCH
    return cfg.as_tuple() + (cfg.cameras_per_block, 0)


def psfs_batch_set_wait_limit(b: int, limit_ns: int, hold_frame: int = -1):
    """Limit of the batched fusion items' bounded waits; `hold_frame` (tests
    only) makes one frame's items wait for a chunk that never comes."""
    _check(load().psfs_batch_set_wait_limit(b, int(limit_ns), int(hold_frame)), "psfs_batch_set_wait_limit")


def psfs_batch_destroy(b: int):
    if b:
        load().psfs_batch_destroy(b)


PSFS_N_STAGES = 8
STAGE_NAMES = ["likelihood", "fuse", "backward_voxel", "backward_pixel", "batch", "surface", "smooth",
               "reproject"]


def psfs_profile_enable(h: int, max_launches: int):
    _check(load().psfs_profile_enable(h, int(max_launches)), "psfs_profile_enable")


def psfs_profile_read(h: int) -> dict:
    """{stage name: (milliseconds, launches)} since the previous read."""
    ms = (ctypes.c_double * PSFS_N_STAGES)()
    n = (ctypes.c_int32 * PSFS_N_STAGES)()
    _check(load().psfs_profile_read(h, ms, n), "psfs_profile_read")
    return {STAGE_NAMES[i]: (ms[i], n[i]) for i in range(len(STAGE_NAMES)) if n[i]}


def psfs_status_string(s: int) -> str:
    return load().psfs_status_string(int(s)).decode()


def psfs_last_error_message() -> str:
    return load().psfs_last_error_message().decode(errors="replace")


# --------------------------------------------------------------------------- #
# owning wrapper: handle lifetime + output allocation (torch device memory)
# --------------------------------------------------------------------------- #
class Reconstructor:
    """One grid + camera rig on one CUDA device.  Allocates outputs with torch
    and calls the entry points above; computes nothing itself."""

    def __init__(self, grid, cams, params=None, *, map_dtype=None, stream=None, device=None,
                 capacity: Optional[int] = None):
        import torch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.handle = psfs_create(grid, cams, params, self.stream, map_dtype)
        g = make_grid(grid)
        self.shape = (g.nz, g.ny, g.nx)
        self.n_voxels = g.nx * g.ny * g.nz
        c0 = cams[0]
        self.n_cams = len(cams)
        self.image_shape = (self.n_cams, int(_get(c0, "height")), int(_get(c0, "width")), 3)
        self.capacity = int(capacity) if capacity is not None else self.n_voxels
        self.grid, self.cams, self.params = grid, list(cams), params
        self.map_dtype = int(make_params(params, map_dtype).map_dtype)

    def close(self):
        if getattr(self, "handle", None):
            psfs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_background(self, mean, var):
        psfs_set_background(self.handle, mean, var)

    def alloc_outputs(self):
        import torch
        occ = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        lst = torch.empty(max(self.capacity, 1), dtype=torch.int32, device=self.device)
        cnt = torch.zeros(1, dtype=torch.int32, device=self.device)
        return occ, lst, cnt

    def reconstruct(self, images, out=None):
        """Enqueue one frame; returns (occupancy, list buffer, count tensor)."""
        occ, lst, cnt = out if out is not None else self.alloc_outputs()
        psfs_reconstruct(self.handle, images, occ, lst, self.capacity, cnt)
        return occ, lst, cnt

    def fuse_slm(self, slm, out=None):
        occ, lst, cnt = out if out is not None else self.alloc_outputs()
        psfs_fuse_slm(self.handle, slm, occ, lst, self.capacity, cnt)
        return occ, lst, cnt

    def likelihood(self, images):
        import torch
        out = torch.empty(self.image_shape[:3], dtype=torch.float32, device=self.device)
        psfs_get_likelihood(self.handle, images, out)
        return out

    def log_ratio(self, images):
        """The stored log-ratio maps of `images`, in the handle's map dtype."""
        import torch
        dt = {PSFS_MAP_F32: torch.float32, PSFS_MAP_F16: torch.float16, PSFS_MAP_BF16: torch.bfloat16}
        out = torch.empty(self.image_shape[:3], dtype=dt[self.map_dtype], device=self.device)
        psfs_get_log_ratio(self.handle, images, out)
        return out

    def sync(self) -> int:
        return psfs_sync(self.handle)


def voxel_list(lst, cnt, capacity: int):
    """Occupied-voxel indices as a sorted int64 CPU tensor (after the frame)."""
    n = min(int(cnt.item()) & 0xFFFFFFFF, capacity)
    return (lst[:n].to("cpu").long() & 0xFFFFFFFF).sort().values
