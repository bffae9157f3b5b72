"""The bounds-checked build (-DPSFS_BOUNDS_CHECK) on every device entry
point: the index checks at the gathers and stores whose indices rest on the
kernels' own arithmetic or on the planner's proofs (a pixel proved inside the
image, an owner list's voxel indices, a silhouette row) must all hold, so
every call returns ok, and the outputs must equal the product build's.
(compute-sanitizer is not available; this and the small cases against the
FP64 oracle stand in for it.)"""

import json
import os
import subprocess
import sys

import pytest

from paper_1311_6811_gb300 import build as libbuild

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(bounds):
    env = dict(os.environ)
    env.pop("PSFS_BOUNDS_CHECK", None)
    if bounds:
        env["PSFS_BOUNDS_CHECK"] = "1"
    out = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_worker.py")], env=env,
                         capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-3000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_bounds_checked_build_matches_and_reports_nothing():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    libbuild.build()
    libbuild.build(bounds_check=True)
    plain, checked = _run(False), _run(True)
    assert checked["lib"].endswith(os.path.join("_build_bounds", "libpsfs.so"))
    assert plain["lib"].endswith(os.path.join("_build", "libpsfs.so"))
    keys = [k for k in plain if k != "lib"]
    assert len(keys) > 15 and set(keys) == set(k for k in checked if k != "lib")
    for k in keys:
        assert plain[k]["status"] == "ok", (k, plain[k])
        assert checked[k]["status"] == "ok", (k, checked[k])
        assert checked[k]["digest"] == plain[k]["digest"], k
