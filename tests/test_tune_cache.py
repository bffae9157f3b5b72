"""The autotuner's cache file without a GPU: psfs_tune_cache_load accepts
valid files (every line checked against the supported shapes) and changes
nothing on an invalid one; psfs_tune_cache_save writes back what was loaded;
clear and entries.  (That a handle created afterwards starts with a loaded
choice is checked on the GPU in test_gpu_group.py.)"""

import pytest

from paper_1311_6811_gb300 import build as libbuild
from paper_1311_6811_gb300 import psfs

GOOD = [
    # nx ny nz K W H dtype | lx wy tz staged | lk group | own lx wy tz staged | rec
    "128 128 128 8 640 480 0  8 4 16 0  2 32  1 8 4 2 0  64",
    "64 64 64 4 320 240 0  8 4 8 0  3 1  0 8 4 8 0  32",
    "256 256 256 16 1280 720 1  16 4 8 0  2 32  1 8 4 2 0  32",
]


@pytest.fixture(autouse=True)
def lib():
    libbuild.build()
    psfs.load()
    psfs.psfs_tune_cache_clear()
    yield
    psfs.psfs_tune_cache_clear()


def _write(path, lines, header="psfs-tune 1"):
    path.write_text("\n".join(([header] if header is not None else []) + list(lines)) + "\n")
    return str(path)


def _entries(path):
    rows = path.read_text().splitlines()
    assert rows[0] == "psfs-tune 1"
    return sorted(tuple(int(x) for x in r.split()) for r in rows[1:] if r.strip())


def test_load_save_round_trip(tmp_path):
    assert psfs.psfs_tune_cache_entries() == 0
    psfs.psfs_tune_cache_load(_write(tmp_path / "a.txt", GOOD + [""]))
    assert psfs.psfs_tune_cache_entries() == 3
    out = tmp_path / "b.txt"
    psfs.psfs_tune_cache_save(str(out))
    want = sorted(tuple(int(x) for x in r.split()) for r in GOOD)
    # a handle whose sequence path shares the one-frame shape is written with that shape
    assert _entries(out) == want
    # loading again replaces entries of the same kinds
    psfs.psfs_tune_cache_load(str(out))
    assert psfs.psfs_tune_cache_entries() == 3
    psfs.psfs_tune_cache_clear()
    assert psfs.psfs_tune_cache_entries() == 0
    psfs.psfs_tune_cache_save(str(out))
    assert out.read_text() == "psfs-tune 1\n"


@pytest.mark.parametrize("bad", [
    "128 128 128 8 640 480 0  8 4 16 0  2 32  1 8 4 2 0",          # 18 integers
    "128 128 128 8 640 480 0  8 4 16 0  2 32  1 8 4 2 0  64 x",    # trailing characters
    "128 128 128 8 640 480 3  8 4 16 0  2 32  1 8 4 2 0  64",      # no such map type
    "128 128 128 0 640 480 0  8 4 16 0  2 32  1 8 4 2 0  64",      # no camera
    "128 128 128 8 640 480 0  12 4 16 0  2 32  1 8 4 2 0  64",     # lanes_x 12
    "128 128 128 8 640 480 0  8 4 16 0  5 32  1 8 4 2 0  64",      # 5 likelihood CTAs per SM
    "128 128 128 8 640 480 0  8 4 16 0  2 24  1 8 4 2 0  64",      # groups of 24
    "128 128 128 8 640 480 0  8 4 16 0  2 32  1 8 4 8 0  64",      # 64-byte records need voxels_z 2 or 4
    "128 128 128 8 640 480 0  8 4 16 0  2 32  0 8 4 2 0  64",      # the one-frame shape (voxels_z 16) cannot run groups
    "128 128 128 8 640 480 0  8 4 16 0  2 32  1 8 4 2 0  48",      # record size 48
    "128 128 128 8 640 480 0  8 4 16 0  2 32  2 8 4 2 0  64",      # own-shape flag 2
])
def test_invalid_line_changes_nothing(tmp_path, bad):
    psfs.psfs_tune_cache_load(_write(tmp_path / "good.txt", GOOD[:1]))
    assert psfs.psfs_tune_cache_entries() == 1
    with pytest.raises(psfs.PsfsError) as e:
        psfs.psfs_tune_cache_load(_write(tmp_path / "bad.txt", GOOD[1:] + [bad]))
    assert e.value.status == psfs.PSFS_ERR_INVALID_ARG
    assert "line 4" in str(e.value)
    assert psfs.psfs_tune_cache_entries() == 1


def test_bad_files(tmp_path):
    with pytest.raises(psfs.PsfsError):
        psfs.psfs_tune_cache_load(str(tmp_path / "missing.txt"))
    with pytest.raises(psfs.PsfsError):
        psfs.psfs_tune_cache_load(_write(tmp_path / "hdr.txt", GOOD, header="psfs-tune 2"))
    with pytest.raises(psfs.PsfsError):
        psfs.psfs_tune_cache_load(_write(tmp_path / "nohdr.txt", GOOD, header=None))
    (tmp_path / "empty.txt").write_text("")
    with pytest.raises(psfs.PsfsError):
        psfs.psfs_tune_cache_load(str(tmp_path / "empty.txt"))
    with pytest.raises(psfs.PsfsError):
        psfs.psfs_tune_cache_save(str(tmp_path / "no_such_dir" / "x.txt"))
    assert psfs.psfs_tune_cache_entries() == 0
