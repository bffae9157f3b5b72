#!/usr/bin/env python
"""Throughput of GB300 probabilistic shape-from-silhouette (PSFS) on the
128^3-voxel x 8-camera (640x480) walking-sequence workload.

One step = the whole hot path (per-pixel likelihood kernel + per-voxel
fusion / threshold / compaction kernel) over every frame of the synthetic
100-frame sequence, inputs resident in HBM.  The metric is Gvoxel-camera
evaluations per second (frames x voxels x cameras / time); frames/s is in
`config`.  With torchrun (N > 1) every rank runs its own copy of the
sequence (frames are independent: weak scaling, no collective on the data
path); the timed region is bracketed by barriers and the max over ranks is
taken.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the FP64 CPU oracle on the host cores instead (one
frame per step, a bounded sample of the same workload).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

GRID_N, N_CAMS, WIDTH, HEIGHT = 128, 8, 640, 480
METRIC = "Gvoxel-camera evals/s (128^3 x 8 cams)"
UNIT = "Gvox-cam/s"
WORKLOAD = "psfs 128^3 grid x 8 cams 640x480, walking sequence"


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--frames", type=int, default=100, help="frames per step (the sequence length)")
    ap.add_argument("--map-dtype", choices=["f32", "f16", "bf16"], default="f32")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--cpu-sample-frames", type=int, default=6,
                    help="frames the CPU oracle baseline times (bounded sample)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--fuse-config", default=None,
                    help="lanes_x,warps,voxels_z,staged[,likelihood_ctas[,frames_per_group[,seq_lanes_x,seq_voxels_z]]]: "
                         "skip the autotuner")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the per-frame FP32/FP16 forward and forward+backward timings")
    ap.add_argument("--forms-frames", type=int, default=20)
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 64^3 x 4, 256^3 x 16 (16-bit maps) and 64-frame batch workloads")
    ap.add_argument("--launch", choices=["sequence", "batch"], default="sequence",
                    help="sequence: psfs_reconstruct_sequence (2 streams); batch: one persistent CUDA-graph launch")
    ap.add_argument("--no-l2-background", action="store_true",
                    help="do not keep the background resident in L2 on the sequence path")
    ap.add_argument("--workers", type=int, default=min(8, os.cpu_count() or 1),
                    help="processes rendering the synthetic frames")
    return ap.parse_args(argv)


# --------------------------------------------------------------------------- #
# distributed plumbing (one process per GPU)
# --------------------------------------------------------------------------- #
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(backend: str):
    import torch.distributed as dist
    ws, rank, _ = dist_env()
    if ws > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return ws, rank


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# --------------------------------------------------------------------------- #
# clocks during the timed region
# --------------------------------------------------------------------------- #
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.15)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------- #
# helpers
# --------------------------------------------------------------------------- #
def sequence_units(n_frames, group, voxels_z=4, map_elem=4, record_bytes=32):
    """Frames per unit of psfs_reconstruct_sequence: groups of `group` frames
    while they fill, then the largest smaller power-of-two groups that fit and
    whose pixel records (P = min(g, record_bytes / map_elem) frames) the tile
    height supports (voxels_z 2 or 4; 8 when P <= 8; 16 when P <= 4; only 2 or
    4 for a 64-byte record, two lanes per voxel), else single frames."""
    def ok(g):
        p = min(g, record_bytes // map_elem)
        if p * map_elem == 64:
            return voxels_z in (2, 4)
        return voxels_z in (2, 4) or (voxels_z == 8 and p <= 8) or (voxels_z == 16 and p <= 4)

    units, left = [], n_frames
    while left > 0:
        g = group
        while g > 1 and (g > left or not ok(g)):
            g //= 2
        g = max(g, 1)
        units.append(g)
        left -= g
    return units


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def csrc_digest() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1311_6811_gb300", "csrc")
    for name in sorted(os.listdir(d)):
        if name.endswith((".cu", ".cuh")):
            with open(os.path.join(d, name), "rb") as f:
                h.update(name.encode())
                h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, config: dict):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current sources of that kernel and the same launch
    configuration; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        with open(path) as f:
            d = json.load(f)
        recs = d.get("kernels", {}).get(kernel)
        if not recs:
            return None
        for rec in (recs if isinstance(recs, list) else [recs]):   # one record per launch configuration
            if any(config.get(k_) != v for k_, v in rec.get("config", {}).items()):
                continue
            h = hashlib.sha256()
            for name in rec["sources"]:
                with open(os.path.join(ROOT, "paper_1311_6811_gb300", "csrc", name), "rb") as f:
                    h.update(name.encode())
                    h.update(f.read())
            if h.hexdigest()[:16] == rec["sources_sha"]:
                return float(rec["dram_bytes_per_launch"])
        return None
    except (ValueError, KeyError, OSError):
        return None


def fusion_rows(sc, tile=(16, 8, 2)):
    """Row of each (voxel, camera) pair that a fusion launch reads: camera c's
    pixel p of the voxel centre's projection (Eq. 3, in float64) is row c *
    n_pix + p of a plane of pixel records.  Pairs outside the image are left
    out; the order is the fusion's (tiles of tile[0] x tile[1] x tile[2]
    voxels in x, y, z, and in each tile camera by camera).  Measurement set-up
    only: the rows to time the device's gather ceiling on."""
    g = sc.grid
    nx, ny, nz = g.nx, g.ny, g.nz
    tx, ty, tz = tile
    if nx % tx or ny % ty or nz % tz:
        return None
    o = np.asarray(g.origin, dtype=np.float64)
    i = (np.arange(nx) + 0.5) * g.voxel_size + o[0]
    j = (np.arange(ny) + 0.5) * g.voxel_size + o[1]
    k = (np.arange(nz) + 0.5) * g.voxel_size + o[2]
    Z, Y, X = np.meshgrid(k, j, i, indexing="ij")   # [nz][ny][nx]
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=0)
    n_pix = sc.cams[0].width * sc.cams[0].height
    rows = np.empty((len(sc.cams), nz * ny * nx), dtype=np.int32)
    for c, cam in enumerate(sc.cams):
        uvw = cam.K @ (cam.R @ P + cam.t.reshape(3, 1))
        w = uvw[2]
        with np.errstate(divide="ignore", invalid="ignore"):
            u, v = np.floor(uvw[0] / w), np.floor(uvw[1] / w)
        ok = (w > 0) & (u >= 0) & (u < cam.width) & (v >= 0) & (v < cam.height)
        rows[c] = np.where(ok, c * n_pix + v * cam.width + u, -1).astype(np.int32)
    # [c][nz/tz][tz][ny/ty][ty][nx/tx][tx] -> tiles (z, y, x), then camera, then voxel in the tile
    r = rows.reshape(len(sc.cams), nz // tz, tz, ny // ty, ty, nx // tx, tx).transpose(1, 3, 5, 0, 2, 4, 6).ravel()
    return np.ascontiguousarray(r[r >= 0]), len(sc.cams) * n_pix


def gather_ceiling(psfs, dev, sc, record_bytes: int, reps: int = 5):
    """The device's rate for the fusion's reads: psfs_gather_rows over the
    rows of every (voxel, camera) pair of the rig that projects into its
    image, in the fusion's order, from a plane of record_bytes-byte records
    (CUDA events, median of `reps` after a warm-up).  Returns (GB/s of rows
    gathered, pairs per frame) or None."""
    import torch
    fr = fusion_rows(sc)
    if fr is None:
        return None
    idx, n_rows = fr
    plane = torch.zeros(n_rows * record_bytes // 4, dtype=torch.int32, device=dev)
    d_idx = torch.from_numpy(idx).to(dev)
    ck = torch.zeros(1, dtype=torch.int32, device=dev)
    psfs.psfs_gather_rows(plane, record_bytes, d_idx, ck)
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        psfs.psfs_gather_rows(plane, record_bytes, d_idx, ck)
        e1.record()
        torch.cuda.synchronize(dev)
        ms.append(e0.elapsed_time(e1))
    t = sorted(ms)[len(ms) // 2]
    return idx.size * record_bytes / (t * 1e-3) / 1e9, int(idx.size)


def make_scene(args):
    """This rank's frames: with N ranks the sequence has N x `--frames` frames
    and rank r renders frames r, r + N, ... of it (round-robin partition;
    per-rank work stays fixed as N grows)."""
    from synth import scene as S
    from paper_1311_6811_gb300 import replicas
    ws, rank, _ = dist_env()
    if ws > 1:
        return S.scene_128cube_8cam(seed=args.seed, n_frames=args.frames * ws, workers=args.workers,
                                    frame_ids=replicas.rank_frames(args.frames * ws, rank, ws))
    return S.scene_128cube_8cam(seed=args.seed, n_frames=args.frames, workers=args.workers)


def host_cores() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


# The oracle over independent frames on all host cores: one spawned worker
# process per core runs the FP64 oracle, as it stands, on whole frames (the
# frames of a sequence are independent).  The background and the images are
# shared with the workers through shared memory.
_W = {}


def _oracle_worker_init(shm_specs, grid, cams, params):
    from multiprocessing import shared_memory
    import oracle
    _W["shm"] = []
    for key, (name, shape, dtype) in shm_specs.items():
        shm = shared_memory.SharedMemory(name=name)
        _W["shm"].append(shm)
        _W[key] = np.ndarray(shape, dtype=dtype, buffer=shm.buf)
    _W["grid"], _W["cams"], _W["params"] = grid, cams, params
    _W["oracle"] = oracle


def _oracle_worker_frame(f):
    out = _W["oracle"].reconstruct(_W["grid"], _W["cams"], _W["images"][f], _W["mean"], _W["var"], _W["params"])
    return int(out["list"].size)


TIE_EPS = 1e-4   # |L_FP64 - logit(threshold)| below this: a near-threshold tie (FP32 summation bound)


def _oracle_worker_compare(job):
    """Reconstructs one frame with the FP64 oracle and compares each GPU
    variant's occupancy and voxel list of that frame with it: occupancy error
    outside the boundary bucket (a voxel whose FP64 projection lies within
    1e-3 px of a pixel edge in some camera), and the occupied-set difference,
    split into boundary, tie and unexplained voxels."""
    pos, variants = job
    p = _W["params"]
    ref = _W["oracle"].reconstruct(_W["grid"], _W["cams"], _W["images"][pos], _W["mean"], _W["var"], p)
    tau = float(getattr(p, "threshold", 0.5))
    keep = ~ref["boundary"]
    tie = np.abs(ref["logodds"] - math.log(tau / (1.0 - tau))) < TIE_EPS
    out = {}
    for name, (occ, lst, count) in variants.items():
        d = np.abs(occ.astype(np.float64) - ref["occ"])
        got = np.zeros(ref["occ"].size, bool)
        got[lst.astype(np.int64) & 0xFFFFFFFF] = True
        diff = np.flatnonzero(got != ref["occupied"])
        out[name] = {"max_abs": float(d[keep].max()) if keep.any() else 0.0,
                     "mean_abs": float(d[keep].mean()) if keep.any() else 0.0,
                     "boundary_voxels": int(ref["boundary"].sum()), "tie_voxels": int(tie.sum()),
                     "set_diff": int(diff.size),
                     "set_diff_boundary": int(ref["boundary"][diff].sum()),
                     "set_diff_unexplained": int((~(ref["boundary"] | tie))[diff].sum()),
                     "count": int(count), "count_fp64": int(ref["list"].size)}
    return out


def summarize_errors(per_frame):
    """Max / mean / sums over the compared frames of one variant."""
    if not per_frame:
        return None
    return {"frames": sorted(per_frame),
            "max_abs": max(r["max_abs"] for r in per_frame.values()),
            "mean_abs": float(np.mean([r["mean_abs"] for r in per_frame.values()])),
            "boundary_voxels": sum(r["boundary_voxels"] for r in per_frame.values()),
            "tie_voxels": sum(r["tie_voxels"] for r in per_frame.values()),
            "set_diff": sum(r["set_diff"] for r in per_frame.values()),
            "set_diff_unexplained": sum(r["set_diff_unexplained"] for r in per_frame.values()),
            "count_diff_max": max(abs(r["count"] - r["count_fp64"]) for r in per_frame.values())}


class OraclePool:
    def __init__(self, sc, images, n_workers):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        import oracle
        oracle.build()   # once, here: the workers only load it
        self.shms = []
        specs = {}
        for key, arr in (("images", images), ("mean", sc.mean), ("var", sc.var)):
            arr = np.ascontiguousarray(arr)
            shm = shared_memory.SharedMemory(create=True, size=max(arr.nbytes, 1))
            np.ndarray(arr.shape, dtype=arr.dtype, buffer=shm.buf)[...] = arr
            self.shms.append(shm)
            specs[key] = (shm.name, arr.shape, arr.dtype.str)
        self.n = n_workers
        self.pool = mp.get_context("spawn").Pool(n_workers, initializer=_oracle_worker_init,
                                                 initargs=(specs, sc.grid, sc.cams, sc.params))

    def run(self, frames):
        return self.pool.map(_oracle_worker_frame, list(frames), chunksize=1)

    def compare(self, jobs):
        """jobs: [(frame position in the pool's images, {variant: (occ, list, count)})]."""
        return self.pool.map(_oracle_worker_compare, list(jobs), chunksize=1)

    def close(self):
        self.pool.close()
        self.pool.join()
        for shm in self.shms:
            shm.close()
            shm.unlink()


def fp64_comparisons(pending, adjoints):
    """The CPU leg's comparisons of other GPU outputs with the FP64 oracle:
    `pending` = [(key, scene, [(occ, list, count)])] frames of the other
    workloads (one per entry, the scene's own frame); `adjoints` = [(key,
    scene, frame images, d_occ, (d_slm, d_mean, d_var))] GPU gradients for the
    given loss gradient.  Returns {key: report}."""
    import oracle
    oracle.build()
    out = {}
    for key, sc, frames in pending:
        ref = oracle.reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params)
        for occ, lst, count in frames:
            out.setdefault(key, []).append(_err_report(occ, lst, count, ref))
    merged = {}
    for key, reps in out.items():
        merged[key] = reps[0] if len(reps) == 1 else {
            "frames": len(reps), "max_abs": max(r["max_abs"] for r in reps),
            "mean_abs": float(np.mean([r["mean_abs"] for r in reps])),
            "hamming": sum(r["hamming"] for r in reps),
            "hamming_unexplained": sum(r["hamming_unexplained"] for r in reps),
            "boundary_voxels": sum(r["boundary_voxels"] for r in reps)}
    masks = {}
    for key, sc, img, d_occ, grads in adjoints:
        ds, dm, dv = oracle.backward(sc.grid, sc.cams, img, sc.mean, sc.var, d_occ.astype(np.float64), sc.params)
        # pixels within one pixel of a boundary voxel's projection may own
        # other voxels in FP32 than in FP64: left out (one mask per frame)
        tag = (id(sc), hash(img.tobytes()))
        if tag not in masks:
            ref = oracle.reconstruct(sc.grid, sc.cams, img, sc.mean, sc.var, sc.params)
            pix = oracle.voxel_pixels(sc.grid, sc.cams)
            W, H = sc.cams[0].width, sc.cams[0].height
            amb = np.zeros((len(sc.cams), H, W), bool)
            for c in range(len(sc.cams)):
                p = pix[c][ref["boundary"] & (pix[c] >= 0)]
                ys, xs = p // W, p % W
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        amb[c, np.clip(ys + dy, 0, H - 1), np.clip(xs + dx, 0, W - 1)] = True
            masks[tag] = ~amb.ravel()
        keep = masks[tag]
        keep3 = np.repeat(keep, 3)
        rep = {}
        for name, got, want, k in (("d_slm", grads[0], ds, keep), ("d_mean", grads[1], dm, keep3),
                                   ("d_var", grads[2], dv, keep3)):
            g, w = np.asarray(got, np.float64).ravel()[k], want.ravel()[k]
            rep[name] = float(np.abs(g - w).max() / max(np.abs(w).max(), 1e-30))
        rep["what"] = "max |GPU - FP64 adjoint| / max |FP64 adjoint| over pixels away from boundary voxels"
        merged[key] = rep
    return merged


def cpu_baseline(sc, n_frames: int, gpu_outputs=None):
    """The FP64 oracle as it stands: whole frames in parallel on every host
    core (frames are independent), and single-threaded for reference.

    gpu_outputs: {frame: {variant: (occ, list, count)}} of the timed GPU
    outputs; the same pool then reconstructs those frames again (outside the
    timing) and compares, giving the error against FP64 per variant."""
    import oracle
    oracle.build()
    v = sc.grid.n_voxels * sc.n_cams
    all_images = sc.images if sc.images.ndim == 5 else sc.images[None]
    images = all_images[:max(1, n_frames)]
    n1 = min(2, len(images))
    t0 = time.perf_counter()
    for f in range(n1):
        oracle.reconstruct(sc.grid, sc.cams, images[f], sc.mean, sc.var, sc.params)
    dt1 = time.perf_counter() - t0
    single = {"value": n1 * v / dt1 / 1e9, "unit": UNIT, "cores": 1, "sample": f"{n1} frames, 1 thread, {dt1:.1f} s"}
    cores = host_cores()
    nf = len(images)
    # frames to compare that lie beyond the timed sample go after it
    extra = sorted(f for f in (gpu_outputs or {}) if f >= nf)
    pos = {f: f for f in range(nf)}
    pos.update({f: nf + i for i, f in enumerate(extra)})
    pool_images = np.concatenate([images, all_images[extra]]) if extra else images
    pool = OraclePool(sc, pool_images, cores)
    errors = None
    try:
        pool.run(range(min(cores, nf)))   # warm-up: workers started and the oracle loaded
        t0 = time.perf_counter()
        pool.run(range(nf))
        dt = time.perf_counter() - t0
        if gpu_outputs:
            frames = sorted(gpu_outputs)
            res = pool.compare([(pos[f], gpu_outputs[f]) for f in frames])
            per_variant = {}
            for f, r in zip(frames, res):
                for name, rep in r.items():
                    per_variant.setdefault(name, {})[f] = rep
            errors = {name: summarize_errors(pf) for name, pf in per_variant.items()}
    finally:
        pool.close()
    return {"value": nf * v / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{nf} frames of the sequence, FP64 C oracle, one frame per process on {cores} host cores, "
                      f"{dt:.1f} s",
            "single_thread": single}, errors


# --------------------------------------------------------------------------- #
# reference arm: the oracle on the host cores
# --------------------------------------------------------------------------- #
def run_reference(args, scene_maker=None, cores=None):
    """The reference arm: the FP64 oracle on the host cores, rank 0 only
    (other ranks return 0 without work).  `scene_maker(n_frames)` and `cores`
    replace the 128^3 x 8 workload and the core count (tests)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from synth import scene as S
    cores = cores or host_cores()
    # each step: one frame per host core, all in parallel (independent frames)
    n_frames = max(1, min(cores, args.frames))
    if scene_maker is None:
        sc = S.scene_128cube_8cam(seed=args.seed, n_frames=n_frames, workers=args.workers)
    else:
        sc = scene_maker(n_frames)
    imgs = sc.images if sc.images.ndim == 5 else sc.images[None]
    v = sc.grid.n_voxels * sc.n_cams
    pool = OraclePool(sc, imgs, cores)
    per_step = [f % len(imgs) for f in range(cores)]
    try:
        for _ in range(max(args.warmup, 1)):
            pool.run(per_step)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.run(per_step)
        dt = time.perf_counter() - t0
    finally:
        pool.close()
    value = args.steps * cores * v / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD + f" ({cores} frames per step, one per host core)", "grid": GRID_N,
                       "cams": N_CAMS, "width": WIDTH, "height": HEIGHT, "frames_per_step": cores},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{cores} frames per step (one per process), {args.steps} steps, "
                                       "FP64 C oracle"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- #
# our arm
# --------------------------------------------------------------------------- #
def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    # render the synthetic sequence before any CUDA call (the renderer may fork workers)
    sc = make_scene(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist_init("nccl")
    from paper_1311_6811_gb300 import psfs

    F = args.frames
    images = sc.images if sc.images.ndim == 5 else sc.images[None]
    F = images.shape[0]
    V = sc.grid.n_voxels
    K = sc.n_cams
    n_pix = K * HEIGHT * WIDTH
    stream = torch.cuda.Stream(device=dev)
    cap = 1 << 20
    with torch.cuda.stream(stream):
        d_images = torch.from_numpy(images).to(dev)
        occ = torch.empty((F, V), dtype=torch.float32, device=dev)
        lists = torch.empty((F, cap), dtype=torch.int32, device=dev)
        counts = torch.zeros((F,), dtype=torch.int32, device=dev)
        rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params, map_dtype=args.map_dtype, stream=stream,
                                 device=dev, capacity=cap)
        rec.set_background(torch.from_numpy(sc.mean).to(dev), torch.from_numpy(sc.var).to(dev))
    stream.synchronize()
    h = rec.handle
    # autotuner: pick the fuse tile shape on the first frame (setup, untimed)
    if not args.no_l2_background:
        psfs.psfs_set_background_l2(h, True)
    tune_ms = {}
    if args.fuse_config:
        cfg = [int(x) for x in args.fuse_config.split(",")]
        psfs.psfs_set_fuse_config(h, *cfg)
    else:
        psfs.psfs_autotune(h, d_images[0], reps=3, timings=tune_ms)
    fuse_cfg = psfs.psfs_get_fuse_config(h, full=True)

    batch = None
    if args.launch == "batch":
        frames = [(h, d_images[f], occ[f], lists[f], cap, counts[f:f + 1]) for f in range(F)]
        batch = psfs.psfs_batch_create(frames, stream=stream)
        psfs.psfs_batch_autotune(batch, reps=2)

    def step():
        if batch is not None:
            # all frames in one persistent kernel (CUDA graph)
            psfs.psfs_batch_run(batch)
        else:
            # the whole sequence in one call: likelihood of frame f+1 overlaps
            # the fusion of frame f on a second stream
            psfs.psfs_reconstruct_sequence(h, F, d_images, occ, lists, cap, counts)

    for _ in range(args.warmup):
        step()
    st = psfs.psfs_sync(h)
    if st != psfs.PSFS_OK:
        raise RuntimeError(f"warm-up frame failed: {psfs.psfs_status_string(st)}")

    # timed region: device time with events on the launching stream; every
    # launch bracketed by the library's event profiler for per-kernel times
    psfs.psfs_profile_enable(h, 2 * F * args.steps + 8)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    ms_local = e0.elapsed_time(e1)
    prof = psfs.psfs_profile_read(h)
    psfs.psfs_profile_enable(h, 0)
    if batch is not None:
        # one persistent launch per step: its events are the step's
        prof = {"batch": (ms_local, args.steps)}
        st_b = psfs.psfs_batch_sync(batch)
        if st_b != psfs.PSFS_OK:
            raise RuntimeError(f"batched frames failed: {psfs.psfs_status_string(st_b)}")
    st = psfs.psfs_sync(h)
    if st != psfs.PSFS_OK:
        raise RuntimeError(f"timed frame failed: {psfs.psfs_status_string(st)}")
    # the timed outputs of a few frames (first group, a middle group, the
    # trailing unit), kept on the host for the comparison with the FP64 oracle
    err_frames = sorted({f for f in (0, 17, 33, 66, F - 1) if 0 <= f < F})
    gpu_outputs = {f: {"f32" if args.map_dtype == "f32" else args.map_dtype: host_frame(occ, lists, counts, f, cap)}
                   for f in err_frames}
    # with N ranks: the per-frame counts and lists of the whole sequence,
    # gathered back into frame order (after the timed region; frames need no
    # exchange while they are reconstructed)
    gathered = None
    if ws > 1:
        from paper_1311_6811_gb300 import replicas
        n_glob = F * ws
        width = int(min(cap, int(counts.max().item()) & 0xFFFFFFFF)) if F else 0
        g_counts, g_lists = replicas.gather_frames(counts, lists[:, :max(width, 1)].contiguous(), n_glob, rank, ws)
        gathered = {"frames": n_glob, "partition": "round-robin (rank r: frames r, r + N, ...)",
                    "occupied_per_frame": float(np.mean(g_counts)),
                    "lists_complete": all(l.numel() == min(c, cap) for c, l in zip(g_counts, g_lists))}
    ms = max_over_ranks(ms_local, dev)
    total_evals = sum_over_ranks(float(F * V * K * args.steps), dev)
    value = total_evals / (ms * 1e-3) / 1e9
    ms_per_step = ms / max(args.steps, 1)
    mean_count = float(counts.double().mean().item())

    # roofline of the dominant kernel (algorithmic bytes / average launch time).
    # The sequence runs in units of G frames (frame groups), then the largest
    # smaller groups that fit the remaining frames, then single frames; per
    # unit of nf frames the likelihood reads the background once (24 B/px), nf
    # images (3 B/px) and writes nf maps, the fusion reads nf maps and writes
    # nf occupancy grids and lists.
    map_elem = 4 if args.map_dtype == "f32" else 2
    G = fuse_cfg[5] if batch is None else 1
    rec_bytes = fuse_cfg[8]
    units = sequence_units(F, G, fuse_cfg[7], map_elem, rec_bytes)   # the sequence path's tile height
    fuse_frame_bytes = n_pix * map_elem + V * 4 + mean_count * 4
    step_bytes = {"likelihood": sum(n_pix * (24 + nf * (3 + map_elem)) for nf in units),
                  "fuse": F * fuse_frame_bytes,
                  "batch": F * (n_pix * (3 + 24 + map_elem) + fuse_frame_bytes)}
    grouped = G > 1
    # frames per plane of pixel records; a plane of 64-byte records runs the
    # two-lanes-per-voxel fusion kernel
    plane = rec_bytes // map_elem
    pair = grouped and min(G, plane) * map_elem == 64
    kern_names = {"likelihood": "likelihood_group_kernel" if grouped else "likelihood_kernel",
                  "fuse": ("fuse_pair_kernel" if pair else "fuse_group_kernel") if grouped else "fuse_kernel",
                  "batch": "batch_kernel"}
    # kernel launches: one likelihood launch per unit, one fusion launch per
    # plane of pixel records (a unit's stage events span its planes)
    fuse_launches = sum(-(-nf // plane) if nf > 1 else 1 for nf in units)
    if batch is None:
        gpu_launches = args.steps * (len(units) + fuse_launches)
    else:
        gpu_launches = sum(n for _, n in prof.values())
    # the profile has one event per unit and stage; a fusion event spans the
    # unit's plane launches, back to back on one stream
    per_unit = {"likelihood": 1.0, "fuse": fuse_launches / len(units)} if batch is None else {}
    stages = {}
    for name, (t_ms, n) in prof.items():
        n_launch = int(round(n * per_unit.get(name, 1.0)))
        avg = t_ms / n_launch
        per_launch = step_bytes[name] * args.steps / n_launch if name in step_bytes else None
        stages[name] = {"launches": n_launch, "events": n, "avg_us": 1e3 * avg, "share": None,
                        "alg_bytes_per_launch": per_launch,
                        "achieved_gbs": per_launch / (avg * 1e-3) / 1e9 if per_launch else None}
    tot = sum(v["avg_us"] * v["launches"] for v in stages.values())
    for v in stages.values():
        v["share"] = v["avg_us"] * v["launches"] / tot if tot else None
    dom = max(stages, key=lambda k: stages[k]["avg_us"] * stages[k]["launches"])
    peak, peak_kind = measured_peaks()
    ach = stages[dom]["achieved_gbs"]
    # the fusion kernel of a group runs per plane of 32-byte records: its
    # launch depends on the frames per record, the likelihood's on G
    traffic = ncu_traffic(kern_names.get(dom, dom),
                          {"lanes_x": fuse_cfg[6], "voxels_z": fuse_cfg[7],
                           "frames_per_group": min(G, plane) if dom == "fuse" else G})
    roofline = {"bound": "hbm", "kernel": kern_names.get(dom, dom), "achieved": ach, "peak": peak,
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
                "unit": "GB/s", "frac": ach / peak if ach else None, "traffic": traffic,
                "alg_bytes_per_launch": stages[dom]["alg_bytes_per_launch"],
                "units_per_step": units,
                "note": ("the fusion kernels are bound by the L2 -> L1 sector rate of their gathers (one 32-byte "
                         "sector per voxel, camera and 8 FP32 frames; ncu: L2 62 %, L1 77 % busy), not by HBM; "
                         "roofline_sequence gives the whole step against HBM")
                        if dom == "fuse" else None}
    # the whole step against the bytes the grouped method moves: per unit of
    # nf frames the background once (24 B per pixel), nf images (3 B per
    # pixel), nf maps written and read back (2 x map bytes per pixel), nf
    # occupancy grids (4 B per voxel) and lists
    step_alg = sum(n_pix * 24 + nf * (n_pix * (3 + 2 * map_elem) + V * 4 + mean_count * 4) for nf in units)
    seq_gbs = step_alg * args.steps / (ms_local * 1e-3) / 1e9
    roofline_sequence = {"alg_bytes_per_frame": step_alg / F, "achieved": seq_gbs, "peak": peak,
                         "unit": "GB/s", "frac": seq_gbs / peak,
                         "note": "whole step: the bytes the grouped method moves per frame (background once per "
                                 "unit, images, maps written and read, occupancy, lists) over the step time"}

    # the fusion against the device's own ceiling for its reads: each (voxel,
    # camera) pair that projects into the image reads map_elem bytes per frame
    # once (one pixel-record row per plane); psfs_gather_rows times the same
    # rows of a plane of the same records with the same loads and nothing else
    roofline_gather = None
    plane_rec = min(G, plane) * map_elem
    if batch is None and grouped and plane_rec in (32, 64) and "fuse" in stages:
        gc = gather_ceiling(psfs, dev, sc, plane_rec)
        if gc is not None:
            ceil_gbs, pairs = gc
            fuse_s = stages["fuse"]["avg_us"] * stages["fuse"]["launches"] / args.steps * 1e-6
            g_bytes = pairs * F * map_elem
            g_ach = g_bytes / fuse_s / 1e9
            roofline_gather = {"kernel": kern_names["fuse"], "bound": "gather", "achieved": g_ach,
                               "ceiling": ceil_gbs, "unit": "GB/s", "frac": g_ach / ceil_gbs,
                               "pairs_per_frame": pairs, "gathered_bytes_per_step": g_bytes,
                               "record_bytes": plane_rec,
                               "note": "fusion stage time of the step (beside the likelihood on the other stream) "
                                       "against psfs_gather_rows timed alone over the same (voxel, camera) rows "
                                       "of one plane: the device's rate for these reads, measured live"}

    # inner-voxel removal on the step's lists (all frames in one call), timed
    # with events on the handle's stream; not part of the headline value
    nxt = None
    if batch is None:
        scap = cap
        s_lists = torch.empty((F, scap), dtype=torch.int32, device=dev)
        s_counts = torch.zeros((F,), dtype=torch.int32, device=dev)
        with torch.cuda.stream(stream):
            psfs.psfs_surface(h, F, lists, cap, counts, s_lists, scap, s_counts)   # warm-up (scratch)
            reps = 10
            t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0e.record(stream)
            for _ in range(reps):
                psfs.psfs_surface(h, F, lists, cap, counts, s_lists, scap, s_counts)
            t1e.record(stream)
        torch.cuda.synchronize(dev)
        st_s = psfs.psfs_sync(h)
        if st_s != psfs.PSFS_OK:
            raise RuntimeError(f"surface pass failed: {psfs.psfs_status_string(st_s)}")
        us_call = 1e3 * t0e.elapsed_time(t1e) / reps
        n_surf = float(s_counts.double().mean().item())
        # per frame: the list read twice, the bitmask zeroed (n_vox / 8 B), six
        # neighbour words read per listed voxel, the surface list written
        surf_bytes = mean_count * 4 * 2 + V / 8 + mean_count * 6 * 4 + n_surf * 4
        peak_s, _ = measured_peaks()
        nxt = {"surface": {"us_per_frame": us_call / F, "frames_per_call": F, "launches_per_call": 3,
                           "occupied_per_frame": mean_count, "surface_voxels_per_frame": n_surf,
                           "alg_bytes_per_frame": surf_bytes,
                           "achieved_gbs": surf_bytes / (us_call / F * 1e-6) / 1e9,
                           "hbm_frac": surf_bytes / (us_call / F * 1e-6) / 1e9 / peak_s,
                           "note": "psfs_surface over the step's lists in one call (memset + 2 kernels); "
                                   "latency-bound: ~30 K listed voxels per frame"}}
        # silhouettes of the surface voxels in every camera
        masks = torch.empty((F, K, HEIGHT, WIDTH), dtype=torch.uint8, device=dev)
        with torch.cuda.stream(stream):
            psfs.psfs_reproject(h, F, s_lists, scap, s_counts, masks)   # warm-up
            t0e.record(stream)
            for _ in range(reps):
                psfs.psfs_reproject(h, F, s_lists, scap, s_counts, masks)
            t1e.record(stream)
        torch.cuda.synchronize(dev)
        st_s = psfs.psfs_sync(h)
        if st_s != psfs.PSFS_OK:
            raise RuntimeError(f"silhouette pass failed: {psfs.psfs_status_string(st_s)}")
        us_rp = 1e3 * t0e.elapsed_time(t1e) / reps / F
        fg = float(masks.float().mean().item())
        rp_bytes = n_pix * 1 + n_surf * 4
        nxt["reproject"] = {"us_per_frame": us_rp, "frames_per_call": F, "launches_per_call": 2,
                            "surface_voxels_per_frame": n_surf, "silhouette_fraction": fg,
                            "alg_bytes_per_frame": rp_bytes,
                            "achieved_gbs": rp_bytes / (us_rp * 1e-6) / 1e9,
                            "hbm_frac": rp_bytes / (us_rp * 1e-6) / 1e9 / peak_s,
                            "note": "psfs_reproject of the step's surface lists in one call (mask memset + "
                                    "1 kernel): one thread per (surface voxel, camera), float32 centre-ray slab "
                                    "tests over the cube's projected box"}
        # tracker weights of 200 particles (10 cylinders each, around frame 0's
        # body) against frame 0's silhouettes
        caps0 = sc.capsules[0]
        base = np.array([[*c_.a, *c_.b, c_.radius] for c_ in caps0], dtype=np.float32)
        prng = np.random.default_rng(args.seed + 17)
        n_part = 200
        parts = np.repeat(base[None], n_part, axis=0)
        jit = prng.normal(0, 0.03, size=parts.shape).astype(np.float32)
        jit[..., 6] = 0.0
        parts = torch.from_numpy(parts + jit).to(dev)
        pw = torch.empty(n_part, device=dev)
        pt = torch.empty((n_part, K, 2), device=dev)
        m0 = masks[0].contiguous()
        with torch.cuda.stream(stream):
            psfs.psfs_particle_weights(h, parts, m0, pw, pt)   # warm-up
            t0e.record(stream)
            for _ in range(reps):
                psfs.psfs_particle_weights(h, parts, m0, pw, pt)
            t1e.record(stream)
        torch.cuda.synchronize(dev)
        us_w = 1e3 * t0e.elapsed_time(t1e) / reps
        n_samples = n_part * K * len(caps0) * (8 * 4 + 2 * 8)
        nxt["particle_weights"] = {"us_per_call": us_w, "particles": n_part, "cylinders": len(caps0),
                                   "samples_per_call": n_samples, "gsamples_per_s": n_samples / (us_w * 1e-6) / 1e9,
                                   "note": "psfs_particle_weights (Eq. 14-16), one launch, one CTA per particle; "
                                           "sample lookups in the L2-resident silhouettes"}
        del masks
        # smoothing + threshold + compaction over the step's occupancy grids
        sm_grid = torch.empty((F, V), dtype=torch.float32, device=dev)
        sm_counts = torch.zeros((F,), dtype=torch.int32, device=dev)
        with torch.cuda.stream(stream):
            psfs.psfs_smooth(h, F, occ, sm_grid, s_lists, scap, sm_counts)   # warm-up
            t0e.record(stream)
            for _ in range(reps):
                psfs.psfs_smooth(h, F, occ, sm_grid, s_lists, scap, sm_counts)
            t1e.record(stream)
        torch.cuda.synchronize(dev)
        st_s = psfs.psfs_sync(h)
        if st_s != psfs.PSFS_OK:
            raise RuntimeError(f"smoothing pass failed: {psfs.psfs_status_string(st_s)}")
        us_sm = 1e3 * t0e.elapsed_time(t1e) / reps / F
        n_sm = float(sm_counts.double().mean().item())
        sm_bytes = V * 4 * 2 + n_sm * 4
        nxt["smooth"] = {"us_per_frame": us_sm, "frames_per_call": F, "launches_per_call": 2,
                         "voxels_above_threshold_per_frame": n_sm, "alg_bytes_per_frame": sm_bytes,
                         "achieved_gbs": sm_bytes / (us_sm * 1e-6) / 1e9,
                         "hbm_frac": sm_bytes / (us_sm * 1e-6) / 1e9 / peak_s,
                         "note": "psfs_smooth over the step's occupancy grids in one call: read the "
                                 "probabilities, write the smoothed grid and the list (memset + 1 kernel)"}
        del sm_grid

    # end to end through the C ABI with host buffers (pinned): the whole
    # sequence per step through psfs_reconstruct_sequence_host, which copies
    # the images in and the occupancy grids, counts and voxel lists out,
    # overlapped with the kernels; the copies are inside the timed region
    e2e = None
    if not args.no_e2e and batch is None:
        cap_e2e = 1 << 17
        h_images = torch.from_numpy(np.ascontiguousarray(images)).pin_memory()
        h_occ = torch.empty((F, V), dtype=torch.float32).pin_memory()
        h_list = torch.empty((F, cap_e2e), dtype=torch.int32).pin_memory()
        h_cnt = torch.zeros((F,), dtype=torch.int32).pin_memory()
        e2e_steps = max(1, min(args.steps, 10))

        def host_blocks(occ_out, n_blocks=3):
            """n_blocks blocks of e2e_steps calls each (the host link is shared
            with the rest of the machine, so single blocks vary); returns the
            seconds of each block (max over ranks) and the bytes copied out
            per step."""
            psfs.psfs_reconstruct_sequence_host(h, F, h_images, occ_out, h_list, cap_e2e, h_cnt)   # warm-up
            secs, out_b = [], 0
            for _ in range(n_blocks):
                barrier()
                t0 = time.perf_counter()
                for _ in range(e2e_steps):
                    st_e = psfs.psfs_reconstruct_sequence_host(h, F, h_images, occ_out, h_list, cap_e2e, h_cnt)
                    if st_e != psfs.PSFS_OK:
                        raise RuntimeError(f"host-buffer sequence failed: {psfs.psfs_status_string(st_e)}")
                    out_b = (F * V * 4 if occ_out is not None else 0) + F * 4 + \
                        4 * int(torch.clamp(h_cnt.long(), max=cap_e2e).sum())
                secs.append(max_over_ranks(time.perf_counter() - t0, dev))
            barrier()
            return secs, out_b

        secs_full, d2h_step = host_blocks(h_occ)
        # the same with the voxel lists and counts as the only result copied
        # out (the reconstruction's output downstream; no occupancy grids)
        secs_lists, d2h_step_l = host_blocks(None)
        dt = sorted(secs_full)[len(secs_full) // 2]     # the median block
        dt_l = sorted(secs_lists)[len(secs_lists) // 2]
        # the host link alone, same pinned buffers: one copy each way
        d_img_tmp = torch.empty(images.shape, dtype=torch.uint8, device=dev)
        link = {}
        for name, dst, src in (("h2d_gbs", d_img_tmp, h_images), ("d2h_gbs", h_occ, occ)):
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize(dev)
            link[name] = src.numel() * src.element_size() / (time.perf_counter() - t0) / 1e9
        # both directions at once on two streams, as the host-buffer path
        # runs them: their combined rate bounds the end-to-end step
        s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        with torch.cuda.stream(s_in):
            d_img_tmp.copy_(h_images, non_blocking=True)
        with torch.cuda.stream(s_out):
            h_occ.copy_(occ, non_blocking=True)
        torch.cuda.synchronize(dev)
        link["both_gbs"] = (h_images.numel() + occ.numel() * 4) / (time.perf_counter() - t0) / 1e9
        del d_img_tmp
        e2e = {"value": sum_over_ranks(float(F * V * K * e2e_steps), dev) / dt / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": F * n_pix * 3, "d2h_bytes_per_step": int(d2h_step),
               "steps": e2e_steps, "ms_per_step": 1e3 * dt / e2e_steps,
               "blocks_ms_per_step": [round(1e3 * x / e2e_steps, 3) for x in secs_full],
               "timing": f"median of {len(secs_full)} blocks of {e2e_steps} steps",
               "link_alone": {k: round(v, 1) for k, v in link.items()},
               "path": "psfs_reconstruct_sequence_host over the step's frames (pinned host buffers; "
                       "copies in and out overlap the kernels)",
               "lists_only": {"value": sum_over_ranks(float(F * V * K * e2e_steps), dev) / dt_l / 1e9,
                              "unit": UNIT, "h2d_bytes_per_step": F * n_pix * 3,
                              "d2h_bytes_per_step": int(d2h_step_l),
                              "ms_per_step": 1e3 * dt_l / e2e_steps,
                              "blocks_ms_per_step": [round(1e3 * x / e2e_steps, 3) for x in secs_lists],
                              "note": "the same call with no occupancy grids copied out (h_occupancy NULL): "
                                      "images in, counts and voxel lists out"}}

    forms = None
    if not args.no_forms:
        forms = time_forms(args, sc, d_images, occ, dev, psfs, fuse_cfg, gpu_outputs)

    configs = None
    pending = []
    if not args.no_configs and rank == 0:
        configs = time_configs(args, dev, psfs, pending)

    cpu = None
    err_vs_fp64 = None
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        cpu, err = cpu_baseline(sc, min(max(args.cpu_sample_frames, 2 * host_cores()), F), gpu_outputs)
        if err:
            headline = "f32" if args.map_dtype == "f32" else args.map_dtype
            err_vs_fp64 = dict(err.get(headline) or {})
            err_vs_fp64["what"] = ("timed outputs of the sampled frames against the FP64 oracle: max / mean "
                                   "|occupancy - FP64| outside the boundary bucket (FP64 projection within 1e-3 px "
                                   "of a pixel edge), occupied-set differences (unexplained = outside the boundary "
                                   f"and |L - logit tau| < {TIE_EPS} tie buckets)")
            for name, rep in err.items():
                if name != headline and forms is not None:
                    forms[f"{name}_batched_err_vs_fp64"] = rep
        extra = fp64_comparisons(pending, (forms or {}).pop("_adjoints", []))
        for key, rep in extra.items():
            if configs is not None and key in configs:
                configs[key]["err_vs_fp64"] = rep
            elif forms is not None:
                forms[key] = rep
    if forms is not None:
        forms.pop("_adjoints", None)

    if batch is not None:
        psfs.psfs_batch_destroy(batch)
    rec.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.map_dtype == "f32" else
                f"f32 (maps {args.map_dtype})", "data": "synthetic",
                "config": {"workload": WORKLOAD, "grid": GRID_N, "cams": N_CAMS, "width": WIDTH,
                           "height": HEIGHT, "frames_per_step": F, "map_dtype": args.map_dtype,
                           "frames_per_s": F * args.steps * ws / (ms * 1e-3),
                           "occupied_voxels_per_frame": mean_count,
                           "l2": f"inputs larger than L2: {F * n_pix * 3 / 1e6:.0f} MB of images per step",
                           "parallelism": f"replicas x{ws} (frames independent)",
                           "sequence_across_ranks": gathered,
                           "fuse_tile": {"lanes_x": fuse_cfg[0], "warps": fuse_cfg[1], "voxels_z": fuse_cfg[2],
                                         "staged": fuse_cfg[3]},
                           "sequence_tile": {"lanes_x": fuse_cfg[6], "warps": 4, "voxels_z": fuse_cfg[7],
                                             "record_bytes": rec_bytes},
                           "likelihood_ctas_per_sm": fuse_cfg[4],
                           "frames_per_group": G,
                           "autotune_fuse_us": {"x".join(map(str, k)): round(1e3 * v, 2) for k, v in tune_ms.items()},
                           "launch": ("psfs_batch_run (one persistent kernel, CUDA graph)" if batch is not None
                                      else f"psfs_reconstruct_sequence (frame groups of {G}: one background pass "
                                      f"per group, one fusion launch per plane of {min(max(G, 1), plane)} "
                                      f"frames ({rec_bytes}-byte pixel records); 2 streams, double-buffered maps)"),
                           "background_l2_resident": not args.no_l2_background},
                "err_vs_fp64": err_vs_fp64,
                "configs": configs,
                "stages": stages, "roofline": roofline, "roofline_sequence": roofline_sequence,
                "roofline_gather": roofline_gather,
                "cpu_baseline": cpu, "e2e": e2e, "forms": forms,
                "next": nxt,
                "gpu_launches": gpu_launches, "clocks": clk}
        print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- #
# the other workloads: 64^3 x 4 (one frame), 256^3 x 16 with 16-bit maps,
# the 64-frame heterogeneous batch in one graph launch
# --------------------------------------------------------------------------- #
def _err_report(occ, lst, count, ref, threshold=0.5):
    """Error of one GPU frame against the FP64 oracle's reconstruction of it."""
    keep = ~ref["boundary"]
    d = np.abs(np.asarray(occ, np.float64).ravel() - ref["occ"])
    got = np.zeros(ref["occ"].size, bool)
    got[np.asarray(lst, np.int64) & 0xFFFFFFFF] = True
    diff = np.flatnonzero(got != ref["occupied"])
    tie = np.abs(ref["logodds"] - math.log(threshold / (1 - threshold))) < TIE_EPS
    return {"max_abs": float(d[keep].max()) if keep.any() else 0.0,
            "mean_abs": float(d[keep].mean()) if keep.any() else 0.0,
            "hamming": int(diff.size), "hamming_unexplained": int((~(ref["boundary"] | tie))[diff].sum()),
            "boundary_voxels": int(ref["boundary"].sum()), "tie_voxels": int(tie.sum()),
            "count": int(count), "count_fp64": int(ref["list"].size)}


def _stage_roofline(prof, stage_bytes, peak):
    """Dominant stage of the library's event profile: algorithmic bytes per
    launch over its average launch time."""
    rows = {}
    for name, (t_ms, n) in prof.items():
        if name in stage_bytes and n:
            rows[name] = (t_ms, n, stage_bytes[name])
    if not rows:
        return None
    dom = max(rows, key=lambda k: rows[k][0])
    t_ms, n, b = rows[dom]
    ach = b / (t_ms / n * 1e-3) / 1e9
    return {"bound": "hbm", "stage": dom, "avg_us": 1e3 * t_ms / n, "alg_bytes_per_launch": b,
            "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "shares": {k: v[0] / sum(r[0] for r in rows.values()) for k, v in rows.items()}}


def time_single_frame(psfs, dev, sc, map_dtype, reps, flush=None):
    """One frame per psfs_reconstruct call: device time per frame (CUDA events
    around each call on the handle's stream; with `flush`, a buffer larger
    than L2 is written before each call), per-stage profile, outputs."""
    import torch
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params, map_dtype=map_dtype, stream=stream, device=dev)
        rec.set_background(torch.from_numpy(sc.mean).to(dev), torch.from_numpy(sc.var).to(dev))
        img = torch.from_numpy(np.ascontiguousarray(sc.images)).to(dev)
        out = rec.alloc_outputs()
        rec.reconstruct(img, out)
    stream.synchronize()
    psfs.psfs_autotune(rec.handle, img, reps=2)
    with torch.cuda.stream(stream):
        rec.reconstruct(img, out)   # warm-up with the chosen shape
    stream.synchronize()
    psfs.psfs_profile_enable(rec.handle, 4 * reps + 8)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    with torch.cuda.stream(stream):
        for e0, e1 in evs:
            if flush is not None:
                flush.add_(1.0)
            e0.record(stream)
            rec.reconstruct(img, out)
            e1.record(stream)
    stream.synchronize()
    assert rec.sync() == psfs.PSFS_OK
    prof = psfs.psfs_profile_read(rec.handle)
    psfs.psfs_profile_enable(rec.handle, 0)
    ms = sum(e0.elapsed_time(e1) for e0, e1 in evs) / reps
    occ, lst, cnt = out
    n = int(cnt.item()) & 0xFFFFFFFF
    res = (occ.cpu().numpy().ravel(), lst[:min(n, rec.capacity)].cpu().numpy(), n)
    cfg = psfs.psfs_get_fuse_config(rec.handle)
    rec.close()
    return ms, prof, res, cfg


def time_configs(args, dev, psfs, pending):
    """The other configurations of the workload list, each with its throughput
    and the roofline of its dominant kernel.  Their outputs are appended to
    `pending` as (config key, scene, frame outputs) for the CPU leg, which
    adds each one's error against the FP64 oracle."""
    import torch
    from synth import scene as S
    peak, _ = measured_peaks()
    out = {}
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)   # 256 MB > L2

    # 64^3 x 4 cameras 320x240, FP32, one frame per call (L2 flushed between calls)
    sc = S.scene_64cube_4cam(seed=0)
    ms, prof, res, cfg = time_single_frame(psfs, dev, sc, "f32", reps=50, flush=flush)
    V, K, n_pix = sc.grid.n_voxels, sc.n_cams, sc.images.size // 3
    pending.append(("c1", sc, [res]))
    out["c1"] = {"workload": "64^3 grid x 4 cams 320x240, FP32, one frame per psfs_reconstruct call",
                 "ms_per_frame": ms, "frames_per_s": 1e3 / ms, "gvox_cam_per_s": V * K / (ms * 1e-3) / 1e9,
                 "timing": "CUDA events around each call; a 256 MB buffer written before each call (L2 flushed)",
                 "fuse_tile": list(cfg),
                 "roofline": _stage_roofline(prof, {"likelihood": n_pix * (3 + 24 + 4),
                                                    "fuse": n_pix * 4 + V * 4 + res[2] * 4}, peak)}

    # 256^3 x 16 cameras 1280x720, two bodies, FP16 then BF16 maps (inputs > L2)
    sc = S.scene_256cube_16cam(seed=2)
    V, K, n_pix = sc.grid.n_voxels, sc.n_cams, sc.images.size // 3
    for dt in ("f16", "bf16"):
        ms, prof, res, cfg = time_single_frame(psfs, dev, sc, dt, reps=10)
        pending.append((f"c3_{dt}", sc, [res]))
        out[f"c3_{dt}"] = {"workload": f"256^3 grid x 16 cams 1280x720, two bodies, {dt} maps (FP32 accumulation), "
                                       "one frame per psfs_reconstruct call",
                           "ms_per_frame": ms, "frames_per_s": 1e3 / ms,
                           "gvox_cam_per_s": V * K / (ms * 1e-3) / 1e9,
                           "timing": "CUDA events around back-to-back calls; inputs (398 MB) larger than L2",
                           "fuse_tile": list(cfg),
                           "roofline": _stage_roofline(prof, {"likelihood": n_pix * (3 + 24 + 2),
                                                              "fuse": n_pix * 2 + V * 4 + res[2] * 4}, peak)}

    # 64 heterogeneous frames in one persistent CUDA-graph launch, FP32
    scenes = S.batch_64_scenes(seed=64, workers=args.workers)
    stream = torch.cuda.Stream(device=dev)
    recs, frames, outs = [], [], []
    with torch.cuda.stream(stream):
        for sc in scenes:
            rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params, stream=stream, device=dev)
            rec.set_background(torch.from_numpy(sc.mean).to(dev), torch.from_numpy(sc.var).to(dev))
            img = torch.from_numpy(np.ascontiguousarray(sc.images)).to(dev)
            o = rec.alloc_outputs()
            recs.append((rec, img))
            frames.append((rec.handle, img, o[0], o[1], rec.capacity, o[2]))
            outs.append(o)
    stream.synchronize()
    b = psfs.psfs_batch_create(frames, stream=stream)
    tune = {}
    best = psfs.psfs_batch_autotune(b, reps=2, timings=tune)
    psfs.psfs_batch_run(b)
    assert psfs.psfs_batch_sync(b) == psfs.PSFS_OK
    reps = 5
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        psfs.psfs_batch_run(b)
    e1.record(stream)
    stream.synchronize()
    assert psfs.psfs_batch_sync(b) == psfs.PSFS_OK
    ms = e0.elapsed_time(e1) / reps
    evals = sum(sc.grid.n_voxels * sc.n_cams for sc in scenes)
    counts = [int(o[2].item()) & 0xFFFFFFFF for o in outs]
    alg = sum(sc.images.size // 3 * (3 + 24 + 2 * 4) + sc.grid.n_voxels * 4 + c * 4 for sc, c in zip(scenes, counts))
    for k in (0, 37):
        occ, lst, cnt = outs[k]
        pending.append(("c4", scenes[k], [(occ.cpu().numpy().ravel(),
                                          lst[:min(counts[k], recs[k][0].capacity)].cpu().numpy(), counts[k])]))
    psfs.psfs_batch_destroy(b)
    for rec, _ in recs:
        rec.close()
    ach = alg / (ms * 1e-3) / 1e9
    frame_launch = len(best) > 5 and best[5] == 1
    out["c4"] = {"workload": "64 frames, grids from {96,128,160,192}^3, 4-12 cams, 640x480 or 960x540, own pose and "
                             "background each, FP32, one psfs_batch_run (CUDA graph) per step: "
                             + ("each frame's likelihood and fusion launches, frames alternating between two "
                                "streams" if frame_launch else "one persistent kernel over all frames"),
                 "launch": "per-frame launches" if frame_launch else "persistent kernel",
                 "ms_per_launch": ms, "ms_per_frame": ms / len(scenes), "frames_per_s": len(scenes) / (ms * 1e-3),
                 "gvox_cam_per_s": evals / (ms * 1e-3) / 1e9, "voxel_camera_evals": evals,
                 "timing": "CUDA events around back-to-back graph launches; inputs (GBs) larger than L2",
                 "tile": list(best), "autotune_ms": {"x".join(map(str, k)): round(v, 3) for k, v in tune.items()},
                 "roofline": {"bound": "hbm", "kernel": "fuse_kernel + likelihood_kernel" if frame_launch else "batch_kernel",
                              "alg_bytes_per_launch": alg, "achieved": ach,
                              "peak": peak, "unit": "GB/s", "frac": ach / peak},
                 "err_vs_fp64_frames": [0, 37]}
    del flush
    return out


def host_frame(occ, lists, counts, f, cap):
    """(occupancy, voxel list, count) of frame f, copied to the host."""
    n = int(counts[f].item()) & 0xFFFFFFFF
    return (occ[f].cpu().numpy(), lists[f, :min(n, cap)].cpu().numpy(), n)


def _adjoint_sample(out, dtype, sc, rec, d_images, occ_f32, stream, psfs):
    """psfs_backward of frame 1 with the loss gradient occ - occ of frame 0
    (FP32 maps' occupancy as the target), kept with its d_occ for the CPU
    leg, which compares the gradients with the FP64 oracle's adjoint for the
    same d_occ."""
    import torch
    f1 = 1 if d_images.shape[0] > 1 else 0
    n_pix = d_images[0].numel() // 3
    dev = d_images.device
    with torch.cuda.stream(stream):
        o, lst, cnt = rec.reconstruct(d_images[f1])
        d_occ = (o.view(-1) - occ_f32[0]).contiguous()
        g = (torch.empty(n_pix, device=dev), torch.empty(n_pix * 3, device=dev), torch.empty(n_pix * 3, device=dev))
        psfs.psfs_backward(rec.handle, d_images[f1], d_occ, *g)
    stream.synchronize()
    assert rec.sync() == psfs.PSFS_OK
    img = d_images[f1].cpu().numpy()
    out.setdefault("_adjoints", []).append((f"{dtype}_adjoint_err_vs_fp64", sc, img, d_occ.cpu().numpy(),
                                            tuple(x.cpu().numpy() for x in g)))


def time_forms(args, sc, d_images, occ_f32, dev, psfs, fuse_cfg, gpu_outputs=None):
    """Per-frame device time of the plain FP32 forward, and of forward +
    adjoint with FP32 and with FP16 maps (the loss is 1/2 sum (occ - target)^2
    with the previous frame's FP32 occupancy as target, so its gradient
    occ - target is one elementwise kernel), CUDA events on the
    handle's stream.  Also the FP16 forward's occupancy error against FP32."""
    import torch
    F = min(args.forms_frames, d_images.shape[0])
    V = sc.grid.n_voxels
    n_pix = d_images[0].numel() // 3
    out = {"frames": F}
    stream = torch.cuda.Stream(device=dev)
    for dtype in ("f32", "f16"):
        with torch.cuda.stream(stream):
            rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params, map_dtype=dtype, stream=stream, device=dev)
            rec.set_background(torch.from_numpy(sc.mean).to(dev), torch.from_numpy(sc.var).to(dev))
            psfs.psfs_set_fuse_config(rec.handle, *fuse_cfg[:4])
            o, lst, cnt = rec.alloc_outputs()
            d_occ = torch.empty(V, dtype=torch.float32, device=dev)
            d_slm = torch.empty(n_pix, dtype=torch.float32, device=dev)
            d_mean = torch.empty(n_pix * 3, dtype=torch.float32, device=dev)
            d_var = torch.empty(n_pix * 3, dtype=torch.float32, device=dev)
            err = 0.0
            for f in range(2):   # warm-up (the torch ops of the loss too: their first launch loads them)
                rec.reconstruct(d_images[f], (o, lst, cnt))
                torch.sub(o.view(-1), occ_f32[f], out=d_occ)
                psfs.psfs_backward(rec.handle, d_images[f], d_occ, d_slm, d_mean, d_var)
                err = max(err, float((o.view(-1) - occ_f32[f]).abs().max()))
            err = 0.0
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            e[0].record(stream)
            for f in range(F):
                rec.reconstruct(d_images[f], (o, lst, cnt))
            e[1].record(stream)
            for f in range(F):
                rec.reconstruct(d_images[f], (o, lst, cnt))
                torch.sub(o.view(-1), occ_f32[max(f - 1, 0)], out=d_occ)
                psfs.psfs_backward(rec.handle, d_images[f], d_occ, d_slm, d_mean, d_var)
            e[2].record(stream)
            for f in range(min(F, 4)):
                rec.reconstruct(d_images[f], (o, lst, cnt))
                err = max(err, float((o.view(-1) - occ_f32[f]).abs().max()))
        stream.synchronize()
        assert rec.sync() == psfs.PSFS_OK
        out[f"{dtype}_forward_us"] = 1e3 * e[0].elapsed_time(e[1]) / F
        out[f"{dtype}_forward_backward_us"] = 1e3 * e[1].elapsed_time(e[2]) / F
        if dtype != "f32":
            out[f"{dtype}_max_abs_occ_diff_vs_f32"] = err
        # batched forward: the sequence path with frame groups (the tuned group
        # size, at least 16 frames for 16-bit maps)
        nseq = min(32, d_images.shape[0])
        G = max(int(fuse_cfg[5]), 16) if dtype != "f32" else max(int(fuse_cfg[5]), 1)
        lx = fuse_cfg[6] if fuse_cfg[6] in (8, 16) else 8
        tz = fuse_cfg[7] if fuse_cfg[7] in (2, 4) else 4   # 16-frame records need a tile height of 2 or 4
        # the record size tuned for FP32 maps; 16-bit maps keep 32-byte records
        # (16 frames per plane): 64-byte records of 32 16-bit frames measured
        # slower (11.1 against 9.7 us per frame at 128^3 x 8)
        rb = fuse_cfg[8] if dtype == "f32" else 32
        psfs.psfs_set_fuse_config(rec.handle, *fuse_cfg[:4], fuse_cfg[4], G, lx, tz, rb)
        cap_s = 1 << 17
        occ_s = torch.empty((nseq, V), dtype=torch.float32, device=dev)
        lst_s = torch.empty((nseq, cap_s), dtype=torch.int32, device=dev)
        cnt_s = torch.zeros((nseq,), dtype=torch.int32, device=dev)
        with torch.cuda.stream(stream):
            psfs.psfs_reconstruct_sequence(rec.handle, nseq, d_images[:nseq], occ_s, lst_s, cap_s, cnt_s)
            e[0].record(stream)
            for _ in range(3):
                psfs.psfs_reconstruct_sequence(rec.handle, nseq, d_images[:nseq], occ_s, lst_s, cap_s, cnt_s)
            e[3].record(stream)
        stream.synchronize()
        assert rec.sync() == psfs.PSFS_OK
        out[f"{dtype}_batched_forward_us"] = 1e3 * e[0].elapsed_time(e[3]) / (3 * nseq)
        out[f"{dtype}_batched_frames_per_group"] = G
        out[f"{dtype}_batched_record_bytes"] = rb
        if dtype != "f32":
            out[f"{dtype}_batched_max_abs_occ_diff_vs_f32"] = float((occ_s - occ_f32[:nseq]).abs().max())
            if gpu_outputs is not None:
                # frames of the batched 16-bit forward, compared with FP64 by the CPU leg
                for f in sorted(gpu_outputs):
                    if f < nseq and dtype not in gpu_outputs[f]:
                        gpu_outputs[f][dtype] = host_frame(occ_s, lst_s, cnt_s, f, cap_s)
        # batched forward + adjoint: the sequence forward, the loss gradient
        # against the FP32 occupancy, psfs_backward_sequence (owner passes of
        # 16 frames; d_slm per frame, d_mean and d_var summed over the frames)
        d_occ_s = torch.empty((nseq, V), dtype=torch.float32, device=dev)
        d_slm_s = torch.empty((nseq, n_pix), dtype=torch.float32, device=dev)
        with torch.cuda.stream(stream):
            for rep in range(2):   # the first pass warms up (allocates the adjoint scratch)
                if rep == 1:
                    e[0].record(stream)
                psfs.psfs_reconstruct_sequence(rec.handle, nseq, d_images[:nseq], occ_s, lst_s, cap_s, cnt_s)
                torch.sub(occ_s, occ_f32[:nseq], out=d_occ_s)
                psfs.psfs_backward_sequence(rec.handle, nseq, d_images[:nseq], d_occ_s, d_slm_s, d_mean, d_var)
            e[3].record(stream)
        stream.synchronize()
        assert rec.sync() == psfs.PSFS_OK
        out[f"{dtype}_batched_forward_backward_us"] = 1e3 * e[0].elapsed_time(e[3]) / nseq
        # the same with the adjoint formed from the forward's own occupancy
        # (psfs_backward_from_occupancy: no recomputed maps or voxel pass)
        with torch.cuda.stream(stream):
            for rep in range(2):
                if rep == 1:
                    e[0].record(stream)
                psfs.psfs_reconstruct_sequence(rec.handle, nseq, d_images[:nseq], occ_s, lst_s, cap_s, cnt_s)
                torch.sub(occ_s, occ_f32[:nseq], out=d_occ_s)
                psfs.psfs_backward_from_occupancy(rec.handle, nseq, d_images[:nseq], occ_s, d_occ_s, d_slm_s,
                                                  d_mean, d_var)
            e[3].record(stream)
        stream.synchronize()
        assert rec.sync() == psfs.PSFS_OK
        out[f"{dtype}_batched_forward_backward_from_occupancy_us"] = 1e3 * e[0].elapsed_time(e[3]) / nseq
        with torch.cuda.stream(stream):
            e[0].record(stream)
            for f in range(F):
                rec.reconstruct(d_images[f], (o, lst, cnt))
                torch.sub(o.view(-1), occ_f32[max(f - 1, 0)], out=d_occ)
                psfs.psfs_backward_from_occupancy(rec.handle, 1, d_images[f], o, d_occ, d_slm, d_mean, d_var)
            e[3].record(stream)
        stream.synchronize()
        assert rec.sync() == psfs.PSFS_OK
        out[f"{dtype}_forward_backward_from_occupancy_us"] = 1e3 * e[0].elapsed_time(e[3]) / F
        _adjoint_sample(out, dtype, sc, rec, d_images, occ_f32, stream, psfs)
        rec.close()
    # the adjoint with BF16 maps, for its error against FP64 only
    with torch.cuda.stream(stream):
        rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params, map_dtype="bf16", stream=stream, device=dev)
        rec.set_background(torch.from_numpy(sc.mean).to(dev), torch.from_numpy(sc.var).to(dev))
    _adjoint_sample(out, "bf16", sc, rec, d_images, occ_f32, stream, psfs)
    rec.close()
    out["note"] = ("*_forward_us / *_forward_backward_us: one frame per call (no stream overlap); backward = "
                   "recomputed maps + voxel pass + per-pixel owner pass + chain rule to SLM, mean, var.  "
                   "*_batched_forward_us: psfs_reconstruct_sequence over 32 frames in frame groups; "
                   "*_batched_forward_backward_us: that forward + loss gradient + psfs_backward_sequence "
                   "(recomputed forward in parts of up to 8 frames, owner passes of 16 frames); "
                   "*_from_occupancy_us: the adjoint from the forward's own occupancy (psfs_backward_from_occupancy)")
    return out


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
