"""Host-side accounting of bench.py (CPU): the unit plan it mirrors from the
sequence path, and the lookup of committed ncu DRAM traffic, which must
refuse a record taken on other kernel sources or another launch shape."""

import json
import math

import numpy as np

import bench


def test_sequence_units_groups_then_smaller_groups():
    # 100 frames in groups of 32: three whole groups, then 4 frames
    assert bench.sequence_units(100, 32, 4, 4) == [32, 32, 32, 4]
    # trailing frames go to the largest smaller groups that fit
    assert bench.sequence_units(61, 32, 4, 4) == [32, 16, 8, 4, 1]
    assert bench.sequence_units(19, 8, 4, 4) == [8, 8, 2, 1]
    # one frame per launch without groups
    assert bench.sequence_units(3, 1) == [1, 1, 1]


def test_sequence_units_respect_the_tile_height():
    # FP32 records hold 8 frames: 16 and 32 frames run at voxels_z 8
    assert bench.sequence_units(40, 32, 8, 4) == [32, 8]
    # 16-bit records hold 16 frames: voxels_z 8 only up to 8 frames
    assert bench.sequence_units(40, 32, 8, 2) == [8, 8, 8, 8, 8]
    # voxels_z 16 only for records of at most 4 frames
    assert bench.sequence_units(10, 8, 16, 4) == [4, 4, 2]


def test_units_cover_every_frame():
    for n in (1, 7, 31, 32, 33, 100, 257):
        for g in (1, 2, 4, 8, 16, 32):
            for tz in (2, 4, 8, 16):
                for elem in (2, 4):
                    for rb in (32, 64):
                        u = bench.sequence_units(n, g, tz, elem, rb)
                        assert sum(u) == n and all(x >= 1 for x in u)


def test_sequence_units_with_64_byte_records():
    # 64-byte records: 16 FP32 / 32 16-bit frames per plane, tile heights 2 and 4 only
    assert bench.sequence_units(100, 32, 4, 4, 64) == [32, 32, 32, 4]
    assert bench.sequence_units(40, 32, 8, 4, 64) == [8, 8, 8, 8, 8]    # groups of 16 and 32 need voxels_z <= 4
    assert bench.sequence_units(40, 32, 8, 2, 64) == [8, 8, 8, 8, 8]    # 16-bit groups of 16 and 32 too
    assert bench.sequence_units(40, 16, 8, 2, 32) == [8, 8, 8, 8, 8]
    assert bench.sequence_units(37, 32, 2, 2, 64) == [32, 4, 1]


def test_ncu_traffic_matches_sources_and_shape(tmp_path, monkeypatch):
    """A traffic record is used only for the launch shape it was taken on and
    only while the kernel sources hash to the recorded digest."""
    import hashlib
    rec = json.load(open(bench.os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")))
    fuse = rec["kernels"]["fuse_group_kernel"]
    fuse = fuse if isinstance(fuse, list) else [fuse]
    names = fuse[0]["sources"]
    csrc = tmp_path / "paper_1311_6811_gb300" / "csrc"
    csrc.mkdir(parents=True)
    h = hashlib.sha256()
    for name in names:
        data = b"// kernel source " + name.encode() + b"\n"
        (csrc / name).write_bytes(data)
        h.update(name.encode())
        h.update(data)
    digest = h.hexdigest()[:16]
    for r in fuse:
        r["sources"], r["sources_sha"] = names, digest
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    shapes = {(r["config"]["lanes_x"], r["config"]["voxels_z"]): r["dram_bytes_per_launch"] for r in fuse}
    for (lx, tz), b in shapes.items():
        got = bench.ncu_traffic("fuse_group_kernel", {"lanes_x": lx, "voxels_z": tz, "frames_per_group": 8})
        assert got == float(b)
    # a launch shape without a record
    assert bench.ncu_traffic("fuse_group_kernel", {"lanes_x": 32, "voxels_z": 4, "frames_per_group": 8}) is None
    assert bench.ncu_traffic("no_such_kernel", {}) is None
    # the same record against edited kernel sources: refused
    (csrc / names[0]).write_bytes((csrc / names[0]).read_bytes() + b"// edited\n")
    lx, tz = next(iter(shapes))
    assert bench.ncu_traffic("fuse_group_kernel", {"lanes_x": lx, "voxels_z": tz, "frames_per_group": 8}) is None


def test_error_report_against_fp64(monkeypatch):
    """The bench's comparison of GPU outputs with the FP64 oracle: the oracle's
    own result reports no error; a flipped voxel outside the boundary and tie
    buckets is counted as unexplained, a shifted occupancy as its error."""
    import numpy as np
    import oracle
    from synth import scene as S
    sc = S.make_scene(seed=3, grid_n=16, cube_side=2.0, n_cams=2, width=64, height=48, focal=60.0)
    for k, v in {"images": sc.images[None], "mean": sc.mean, "var": sc.var, "grid": sc.grid, "cams": sc.cams,
                 "params": sc.params, "oracle": oracle}.items():
        monkeypatch.setitem(bench._W, k, v)
    ref = oracle.reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params)
    occ = ref["occ"].astype(np.float32)
    lst = ref["list"].astype(np.uint32)
    rep = bench._oracle_worker_compare((0, {"same": (occ, lst, lst.size)}))["same"]
    assert rep["set_diff"] == 0 and rep["set_diff_unexplained"] == 0 and rep["max_abs"] < 1e-7
    # flip the clearest voxel outside both buckets and shift one occupancy
    ok = ~ref["boundary"] & (np.abs(ref["logodds"]) > 1.0)
    v = int(np.flatnonzero(ok)[0])
    got = set(lst.tolist()) ^ {v}
    lst2 = np.array(sorted(got), np.uint32)
    occ2 = occ.copy()
    occ2[v] += 0.25
    rep = bench._oracle_worker_compare((0, {"bad": (occ2, lst2, lst2.size)}))["bad"]
    assert rep["set_diff"] == 1 and rep["set_diff_unexplained"] == 1
    assert abs(rep["max_abs"] - 0.25) < 1e-6
    s = bench.summarize_errors({0: rep, 5: rep})
    assert s["frames"] == [0, 5] and s["set_diff_unexplained"] == 2


def test_fp64_comparisons_of_other_workloads_and_adjoints():
    """The CPU leg's comparisons: the oracle's own outputs and gradients
    report no error; a scaled gradient reports its relative error."""
    import numpy as np
    import oracle
    from synth import scene as S
    sc = S.make_scene(seed=4, grid_n=12, cube_side=2.0, n_cams=2, width=48, height=36, focal=45.0)
    ref = oracle.reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params)
    pending = [("c", sc, [(ref["occ"].astype(np.float32), ref["list"], ref["list"].size)])]
    d_occ = np.random.default_rng(0).normal(size=sc.grid.n_voxels).astype(np.float32)
    ds, dm, dv = oracle.backward(sc.grid, sc.cams, sc.images, sc.mean, sc.var, d_occ.astype(np.float64), sc.params)
    adj = [("a", sc, sc.images, d_occ, (ds, dm, dv)), ("b", sc, sc.images, d_occ, (1.01 * ds, dm, dv))]
    out = bench.fp64_comparisons(pending, adj)
    assert out["c"]["hamming"] == 0 and out["c"]["max_abs"] < 1e-7
    assert out["a"]["d_slm"] == 0 and out["a"]["d_mean"] == 0
    assert abs(out["b"]["d_slm"] - 0.01) < 1e-9 and out["b"]["d_var"] == 0


def test_units_with_two_voxel_tiles():
    # voxels_z 2 holds 2 x P accumulators: every record size fits
    assert bench.sequence_units(100, 32, 2, 4) == [32, 32, 32, 4]
    assert bench.sequence_units(100, 32, 2, 2) == [32, 32, 32, 4]


def test_fusion_rows_order_and_membership():
    """The rows the gather ceiling is timed on: per tile of 16 x 8 x 2 voxels,
    camera by camera, the pixel row of every voxel centre that projects into
    the image (checked voxel by voxel with a pinhole projection written out
    here), and nothing else."""
    from synth import scene as S
    sc = S.make_scene(seed=3, grid_n=16, cube_side=2.0, n_cams=3, width=64, height=48, focal=60.0)
    idx, n_rows = bench.fusion_rows(sc)
    g, W, H = sc.grid, 64, 48
    assert n_rows == 3 * W * H
    want = []
    for tz in range(g.nz // 2):
        for ty in range(g.ny // 8):
            for tx in range(g.nx // 16):
                for c, cam in enumerate(sc.cams):
                    for dz in range(2):
                        for dy in range(8):
                            for dx in range(16):
                                i, j, k = 16 * tx + dx, 8 * ty + dy, 2 * tz + dz
                                X = np.asarray(g.origin) + (np.array([i, j, k]) + 0.5) * g.voxel_size
                                u, v, w = cam.K @ (cam.R @ X + cam.t)
                                if w <= 0:
                                    continue
                                px, py = math.floor(u / w), math.floor(v / w)
                                if 0 <= px < W and 0 <= py < H:
                                    want.append(c * W * H + py * W + px)
    assert 0 < len(want) < 3 * g.n_voxels
    np.testing.assert_array_equal(idx, np.asarray(want, dtype=np.int32))
    # a grid that the tile does not divide has no row list
    sc2 = S.make_scene(seed=3, grid_n=12, cube_side=2.0, n_cams=2, width=64, height=48, focal=60.0)
    assert bench.fusion_rows(sc2) is None
