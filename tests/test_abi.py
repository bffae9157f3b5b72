"""The C ABI without a GPU: the library loads, exports every entry point that
include/psfs.h declares, its structs have the C layout, and the host-side
argument checks reject bad input before any CUDA call."""

import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1311_6811_gb300 import build as libbuild
from paper_1311_6811_gb300 import psfs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "psfs.h")


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return psfs.load()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(psfs_\w+)\s*\(", text)))


def test_every_declared_function_is_exported(lib):
    names = _declared_functions()
    assert "psfs_reconstruct" in names and "psfs_backward" in names
    out = subprocess.run(["nm", "-D", "--defined-only", libbuild.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (psfs_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stddef.h>
#include <stdio.h>
#include "psfs.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(psfs_grid), offsetof(psfs_grid, origin),
         offsetof(psfs_grid, voxel_size), (size_t)0);
  printf("%zu %zu %zu %zu\n", sizeof(psfs_camera), offsetof(psfs_camera, K),
         offsetof(psfs_camera, R), offsetof(psfs_camera, t));
  printf("%zu %zu %zu %zu\n", sizeof(psfs_params), offsetof(psfs_params, threshold),
         offsetof(psfs_params, log_fg_density), offsetof(psfs_params, map_dtype));
  printf("%zu %zu %zu %zu\n", sizeof(psfs_fuse_config), offsetof(psfs_fuse_config, cameras_per_block),
         offsetof(psfs_fuse_config, seq_voxels_z), offsetof(psfs_fuse_config, seq_record_bytes));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    rows = [list(map(int, l.split())) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                               check=True).stdout.split("\n") if l]
    assert rows[0][:3] == [ctypes.sizeof(psfs.psfs_grid), psfs.psfs_grid.origin.offset,
                           psfs.psfs_grid.voxel_size.offset]
    assert rows[1] == [ctypes.sizeof(psfs.psfs_camera), psfs.psfs_camera.K.offset,
                       psfs.psfs_camera.R.offset, psfs.psfs_camera.t.offset]
    assert rows[2] == [ctypes.sizeof(psfs.psfs_params), psfs.psfs_params.threshold.offset,
                       psfs.psfs_params.log_fg_density.offset, psfs.psfs_params.map_dtype.offset]
    assert rows[3] == [ctypes.sizeof(psfs.psfs_fuse_config), psfs.psfs_fuse_config.cameras_per_block.offset,
                       psfs.psfs_fuse_config.seq_voxels_z.offset, psfs.psfs_fuse_config.seq_record_bytes.offset]


def test_defaults_and_status_strings(lib):
    p = psfs.psfs_params_default()
    assert (p.p_detect, p.p_false_alarm, p.prior, p.threshold) == (0.9, 0.1, 0.5, 0.5)
    assert abs(p.log_fg_density + 3 * math.log(256)) < 1e-12 and p.map_dtype == psfs.PSFS_MAP_F32
    for s, name in [(0, "ok"), (1, "invalid argument"), (2, "background not set"),
                    (3, "voxel list capacity exceeded"), (4, "CUDA error")]:
        assert psfs.psfs_status_string(s) == name
    assert psfs.psfs_status_string(99) == "unknown status"


def _good():
    grid = psfs.make_grid({"nx": 8, "ny": 8, "nz": 8, "origin": (0, 0, 0), "voxel_size": 0.1})
    cam = {"width": 64, "height": 48, "K": np.eye(3), "R": np.eye(3), "t": np.array([0, 0, 3.0])}
    cams = psfs.make_cameras([cam, cam])
    return grid, cams, psfs.psfs_params_default()


def _create(lib, grid, cams, n, params):
    out = ctypes.c_void_p()
    st = lib.psfs_create(ctypes.byref(grid) if grid is not None else None, cams, n,
                         ctypes.byref(params) if params is not None else None, None, ctypes.byref(out))
    return st, out.value


@pytest.mark.parametrize("case", ["null_grid", "null_cams", "n_cams0", "n_cams_big", "bad_pd", "q0",
                                  "prior1", "thr0", "dtype", "grid0", "vs0", "nan_K", "size_mismatch",
                                  "huge_grid", "null_params"])
def test_create_rejects_bad_arguments(lib, case):
    grid, cams, p = _good()
    n = 2
    if case == "null_grid":
        grid = None
    elif case == "null_cams":
        cams = None
    elif case == "n_cams0":
        n = 0
    elif case == "n_cams_big":
        n = psfs.PSFS_MAX_CAMS + 1
    elif case == "bad_pd":
        p.p_detect = 1.5
    elif case == "q0":
        p.p_detect, p.p_false_alarm = 0.0, 0.0
    elif case == "prior1":
        p.prior = 1.0
    elif case == "thr0":
        p.threshold = 0.0
    elif case == "dtype":
        p.map_dtype = 7
    elif case == "grid0":
        grid.nz = 0
    elif case == "vs0":
        grid.voxel_size = 0.0
    elif case == "nan_K":
        cams[1].K[0] = float("nan")
    elif case == "size_mismatch":
        cams[1].width = 65
    elif case == "huge_grid":
        grid.nx = grid.ny = grid.nz = 1 << 11
    elif case == "null_params":
        p = None
    st, h = _create(lib, grid, cams, n, p)
    assert st == psfs.PSFS_ERR_INVALID_ARG and h is None
    assert psfs.psfs_last_error_message()


def test_calls_reject_null_handle(lib):
    assert lib.psfs_set_background(None, None, None) == psfs.PSFS_ERR_INVALID_ARG
    assert lib.psfs_reconstruct(None, None, None, None, 0, None) == psfs.PSFS_ERR_INVALID_ARG
    assert lib.psfs_reconstruct_host(None, None, None, None, 0, None) == psfs.PSFS_ERR_INVALID_ARG
    assert lib.psfs_reconstruct_sequence_host(None, 1, None, None, None, 0, None) == psfs.PSFS_ERR_INVALID_ARG
    assert lib.psfs_surface(None, 1, None, 0, None, None, 0, None) == psfs.PSFS_ERR_INVALID_ARG
    assert lib.psfs_smooth(None, 1, None, None, None, 0, None) == psfs.PSFS_ERR_INVALID_ARG
    assert lib.psfs_reproject(None, 1, None, 0, None, None) == psfs.PSFS_ERR_INVALID_ARG
    assert lib.psfs_particle_weights(None, 1, 10, None, 8, 4, None, None, None) == psfs.PSFS_ERR_INVALID_ARG
    assert lib.psfs_fuse_slm(None, None, None, None, 0, None) == psfs.PSFS_ERR_INVALID_ARG
    assert lib.psfs_get_likelihood(None, None, None) == psfs.PSFS_ERR_INVALID_ARG
    assert lib.psfs_backward(None, None, None, None, None, None) == psfs.PSFS_ERR_INVALID_ARG
    assert lib.psfs_backward_sequence(None, 2, None, None, None, None, None) == psfs.PSFS_ERR_INVALID_ARG
    assert lib.psfs_backward_from_occupancy(None, 2, None, None, None, None, None, None) == psfs.PSFS_ERR_INVALID_ARG
    assert lib.psfs_get_log_ratio(None, None, None) == psfs.PSFS_ERR_INVALID_ARG
    assert lib.psfs_batch_set_wait_limit(None, 1000000, -1) == psfs.PSFS_ERR_INVALID_ARG
    assert lib.psfs_sync(None) == psfs.PSFS_ERR_INVALID_ARG
    lib.psfs_destroy(None)


@pytest.mark.parametrize("case", ["record_48", "negative_n", "null_rows", "misaligned_rows", "null_idx",
                                  "misaligned_checksum"])
def test_gather_rows_rejects_bad_arguments_before_any_cuda_call(lib, case):
    """psfs_gather_rows checks its arguments on the host and returns
    PSFS_ERR_INVALID_ARG with a message; the stand-in addresses are never
    dereferenced."""
    buf = 1 << 20
    rows, n_rows, rb, idx, n, ck = buf, 100, 64, buf, 10, buf
    if case == "record_48":
        rb = 48
    elif case == "negative_n":
        n = -1
    elif case == "null_rows":
        rows = None
    elif case == "misaligned_rows":
        rows = buf + 32
    elif case == "null_idx":
        idx = None
    elif case == "misaligned_checksum":
        ck = buf + 2
    assert lib.psfs_gather_rows(rows, n_rows, rb, idx, n, None, ck) == psfs.PSFS_ERR_INVALID_ARG
    assert psfs.psfs_last_error_message()


@pytest.mark.parametrize("case", ["null_grid", "null_images", "null_list", "misaligned_occ", "n_cams0",
                                  "n_cams_big", "axis_2_24", "f16_maps", "too_many_pixels", "bad_prior"])
def test_noalloc_rejects_bad_arguments_before_any_cuda_call(lib, case):
    """psfs_reconstruct_noalloc checks everything on the host first, records a
    message and returns PSFS_ERR_INVALID_ARG; the fake device addresses below
    are never dereferenced."""
    grid, cams, p = _good()
    n = 2
    buf = 1 << 20   # a 256-byte aligned stand-in address
    mean = var = images = occ = lst = cnt = buf
    cap = 16
    if case == "null_grid":
        grid = None
    elif case == "null_images":
        images = None
    elif case == "null_list":
        lst = None
    elif case == "misaligned_occ":
        occ = buf + 2
    elif case == "n_cams0":
        n = 0
    elif case == "n_cams_big":
        n = psfs.PSFS_MAX_CAMS + 1
    elif case == "axis_2_24":
        grid.nx, grid.ny, grid.nz = (1 << 24) + 1, 1, 1
    elif case == "f16_maps":
        p.map_dtype = psfs.PSFS_MAP_F16
    elif case == "too_many_pixels":
        cams[0].width = cams[1].width = 4096
        cams[0].height = cams[1].height = 1024   # 2 x 4 Mi pixels > PSFS_NOALLOC_MAX_PIXELS
    elif case == "bad_prior":
        p.prior = 0.0
    psfs.load().psfs_last_error_message()   # any earlier message is replaced below
    st = lib.psfs_reconstruct_noalloc(ctypes.byref(grid) if grid is not None else None, cams, n,
                                      ctypes.byref(p), mean, var, images, occ, lst, cap, cnt, None)
    assert st == psfs.PSFS_ERR_INVALID_ARG
    msg = psfs.psfs_last_error_message()
    assert msg, case
    if case == "axis_2_24":
        assert "2^24" in msg
    if case == "too_many_pixels":
        assert "PSFS_NOALLOC_MAX_PIXELS" in msg
