"""The adjoint on the GPU (through the C ABI) against the FP64 oracle's
adjoint and against FP64 central finite differences of the oracle's forward.

Pixels that a "boundary" voxel (FP64 projection within 1e-3 px of a pixel
edge, see tests/gpu_helpers.py) projects into, or next to, are left out of the
element-wise comparison: the FP32 and FP64 projections may hand such a voxel
to neighbouring pixels.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1311_6811_gb300 import psfs  # noqa: E402
from paper_1311_6811_gb300.autograd import (psfs_occupancy, psfs_occupancy_from_slm,  # noqa: E402
                                             psfs_occupancy_sequence)
from synth import scene as S  # noqa: E402
from tests.gpu_helpers import to_dev  # noqa: E402

pytestmark = pytest.mark.gpu
H_FD = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    psfs.load()


def _ambiguous_pixels(grid, cams, boundary):
    """[n_cams * H * W] bool: pixels within one pixel of a boundary voxel's projection."""
    pix = oracle.voxel_pixels(grid, cams)
    W, H = cams[0].width, cams[0].height
    mask = np.zeros((len(cams), H, W), bool)
    for c in range(len(cams)):
        p = pix[c][boundary & (pix[c] >= 0)]
        ys, xs = p // W, p % W
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                mask[c, np.clip(ys + dy, 0, H - 1), np.clip(xs + dx, 0, W - 1)] = True
    return mask.ravel()


def _compare(got, ref, keep, rel=1e-3):
    g, r = got.ravel()[keep].astype(np.float64), ref.ravel()[keep]
    scale = max(np.abs(r).max(), 1e-30)
    err = np.abs(g - r)
    assert np.all(err <= rel * np.abs(r) + 1e-4 * scale), (err.max(), scale)
    return float(err.max() / scale)


def _frame(sc_seed=41, grid_n=48, n_cams=4, W=160, H=120, f=150.0):
    sc = S.make_scene(seed=sc_seed, grid_n=grid_n, cube_side=2.0, n_cams=n_cams, width=W, height=H, focal=f)
    rng = np.random.default_rng(sc_seed)
    target = rng.uniform(0, 1, size=sc.grid.n_voxels)
    return sc, target


def test_backward_matches_oracle_adjoint():
    sc, target = _frame()
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    img = to_dev(sc.images)
    occ, _, _ = rec.reconstruct(img)
    d_occ = 2 * (occ.reshape(-1) - to_dev(target.astype(np.float32)))
    n_pix = sc.images.size // 3
    d_slm = torch.empty(n_pix, dtype=torch.float32, device="cuda")
    d_mean = torch.empty(sc.images.shape, dtype=torch.float32, device="cuda")
    d_var = torch.empty(sc.images.shape, dtype=torch.float32, device="cuda")
    psfs.psfs_backward(rec.handle, img, d_occ.contiguous(), d_slm, d_mean, d_var)
    assert rec.sync() == psfs.PSFS_OK
    ref = oracle.reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params)
    ds, dm, dv = oracle.backward(sc.grid, sc.cams, sc.images, sc.mean, sc.var, 2 * (ref["occ"] - target), sc.params)
    keep = ~_ambiguous_pixels(sc.grid, sc.cams, ref["boundary"])
    e1 = _compare(d_slm.cpu().numpy(), ds, keep)
    keep3 = np.repeat(keep, 3)
    e2 = _compare(d_mean.cpu().numpy(), dm, keep3)
    e3 = _compare(d_var.cpu().numpy(), dv, keep3)
    # pixels no voxel projects into get exactly zero
    owned = (ds.ravel() != 0)
    assert np.all(d_slm.cpu().numpy()[~owned & keep] == 0)
    print("rel err d_slm %.2e d_mean %.2e d_var %.2e" % (e1, e2, e3))
    rec.close()


def test_backward_slm_matches_finite_differences():
    """dLoss/dSLM from psfs_backward_slm against FP64 central differences of
    the oracle's forward on 200 seeded pixels (150 owned, 50 not)."""
    sc, target = _frame(sc_seed=43, grid_n=40)
    p = {"p_detect": 0.8, "p_false_alarm": 0.3, "prior": 0.4, "threshold": 0.5}
    s64 = oracle.slm(sc.images, sc.mean, sc.var)
    s32 = s64.astype(np.float32)
    rec = psfs.Reconstructor(sc.grid, sc.cams, p)
    slm = to_dev(s32)
    occ, _, _ = rec.fuse_slm(slm)
    d_occ = 2 * (occ.reshape(-1) - to_dev(target.astype(np.float32)))
    d_slm = torch.empty_like(slm)
    psfs.psfs_backward_slm(rec.handle, slm, d_occ.contiguous(), d_slm)
    assert rec.sync() == psfs.PSFS_OK
    g = d_slm.cpu().numpy().ravel().astype(np.float64)
    s_in = s32.astype(np.float64)
    ref = oracle.fuse(sc.grid, sc.cams, s_in, p)
    keep = ~_ambiguous_pixels(sc.grid, sc.cams, ref["boundary"])
    pixtab = oracle.voxel_pixels(sc.grid, sc.cams)
    n_cam_pix = sc.cams[0].width * sc.cams[0].height
    owned = np.zeros(s_in.size, bool)
    for c in range(len(sc.cams)):
        q = pixtab[c][pixtab[c] >= 0]
        owned[c * n_cam_pix + q] = True
    rng = np.random.default_rng(7)
    pick = np.concatenate([rng.choice(np.flatnonzero(owned & keep), 150, replace=False),
                           rng.choice(np.flatnonzero(~owned & keep), 50, replace=False)])
    for idx in pick:
        c, q = divmod(int(idx), n_cam_pix)
        vox = np.flatnonzero(pixtab[c] == q)
        if vox.size == 0:
            assert g[idx] == 0.0
            continue
        sp, sm = s_in.ravel().copy(), s_in.ravel().copy()
        sp[idx] += H_FD
        sm[idx] -= H_FD
        op = oracle.fuse_subset(sc.grid, sc.cams, sp, vox, p)
        om = oracle.fuse_subset(sc.grid, sc.cams, sm, vox, p)
        t = target[vox]
        fd = float(np.sum((op - om) * (op + om - 2 * t))) / (2 * H_FD)
        assert abs(g[idx] - fd) <= 2e-3 * abs(fd) + 1e-5, (idx, g[idx], fd)
    rec.close()


def test_autograd_functions_match_the_c_abi():
    sc, target = _frame(sc_seed=44, grid_n=32)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    img = to_dev(sc.images)
    mean = to_dev(sc.mean).requires_grad_(True)
    var = to_dev(sc.var).requires_grad_(True)
    tgt = to_dev(target.astype(np.float32)).reshape(sc.grid.nz, sc.grid.ny, sc.grid.nx)
    occ = psfs_occupancy(rec, img, mean, var)
    loss = ((occ - tgt) ** 2).sum()
    loss.backward()
    d_occ = (2 * (occ.detach() - tgt)).reshape(-1).contiguous()
    dm = torch.empty_like(mean)
    dv = torch.empty_like(var)
    psfs.psfs_backward(rec.handle, img, d_occ, None, dm, dv)
    torch.cuda.synchronize()
    assert torch.equal(mean.grad, dm) and torch.equal(var.grad, dv)
    assert float(mean.grad.abs().max()) > 0
    slm = torch.full((len(sc.cams), sc.cams[0].height, sc.cams[0].width), 0.3, device="cuda", requires_grad=True)
    occ2 = psfs_occupancy_from_slm(rec, slm)
    occ2.sum().backward()
    assert slm.grad is not None and float(slm.grad.abs().max()) > 0
    rec.close()


@pytest.mark.slow
def test_backward_full_size_128cube():
    """128^3 x 8 x 640x480: target occupancy from a pose perturbed by N(0, 5 deg)
    on the joints; loss = sum (occ - target)^2; GPU adjoint against the oracle's
    adjoint, and against finite differences of the oracle on 200 pixels."""
    sc = S.scene_128cube_8cam(seed=5, n_frames=1)
    rng = np.random.default_rng(5)
    # target: the oracle's occupancy of the same rig seeing a perturbed pose
    pose = S.random_pose(rng)
    import dataclasses
    import math
    jitter = lambda v: tuple(x + math.radians(rng.normal(0, 5)) for x in v)  # noqa: E731
    pose2 = dataclasses.replace(pose, hip_flex=jitter(pose.hip_flex), knee=jitter(pose.knee),
                                shoulder_flex=jitter(pose.shoulder_flex), elbow=jitter(pose.elbow))
    cols = rng.uniform(0, 255, (10, 3))
    mean64, sigma = sc.mean.astype(np.float64), np.sqrt(np.maximum(sc.var.astype(np.float64) - 4, 0))
    img = S.render_images(rng, sc.cams, S.body_capsules(pose, cols), mean64, sigma)
    img_t = S.render_images(rng, sc.cams, S.body_capsules(pose2, cols), mean64, sigma)
    target = oracle.reconstruct(sc.grid, sc.cams, img_t, sc.mean, sc.var, sc.params)["occ"]
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    d_img = to_dev(img)
    occ, _, _ = rec.reconstruct(d_img)
    d_occ = (2 * (occ.reshape(-1).double() - to_dev(target))).float().contiguous()
    n_pix = img.size // 3
    d_slm = torch.empty(n_pix, dtype=torch.float32, device="cuda")
    d_mean = torch.empty(img.shape, dtype=torch.float32, device="cuda")
    d_var = torch.empty(img.shape, dtype=torch.float32, device="cuda")
    psfs.psfs_backward(rec.handle, d_img, d_occ, d_slm, d_mean, d_var)
    assert rec.sync() == psfs.PSFS_OK
    ref = oracle.reconstruct(sc.grid, sc.cams, img, sc.mean, sc.var, sc.params)
    ds, dm, dv = oracle.backward(sc.grid, sc.cams, img, sc.mean, sc.var, 2 * (ref["occ"] - target), sc.params)
    keep = ~_ambiguous_pixels(sc.grid, sc.cams, ref["boundary"])
    e1 = _compare(d_slm.cpu().numpy(), ds, keep)
    keep3 = np.repeat(keep, 3)
    e2 = _compare(d_mean.cpu().numpy(), dm, keep3)
    e3 = _compare(d_var.cpu().numpy(), dv, keep3)
    print("128^3 rel err d_slm %.2e d_mean %.2e d_var %.2e" % (e1, e2, e3))
    # finite differences of the oracle on 200 pixels of the SLM
    s64 = ref["slm"].ravel()
    g = d_slm.cpu().numpy().astype(np.float64)
    pixtab = oracle.voxel_pixels(sc.grid, sc.cams)
    n_cam_pix = sc.cams[0].width * sc.cams[0].height
    owned = np.zeros(s64.size, bool)
    for c in range(len(sc.cams)):
        owned[c * n_cam_pix + pixtab[c][pixtab[c] >= 0]] = True
    cand = np.flatnonzero(owned & keep & (np.abs(ds.ravel()) > 1e-6))
    pick = np.concatenate([rng.choice(cand, 150, replace=False),
                           rng.choice(np.flatnonzero(~owned & keep), 50, replace=False)])
    for idx in pick:
        c, q = divmod(int(idx), n_cam_pix)
        vox = np.flatnonzero(pixtab[c] == q)
        if vox.size == 0:
            assert g[idx] == 0.0
            continue
        sp, sm = s64.copy(), s64.copy()
        sp[idx] += H_FD
        sm[idx] -= H_FD
        op = oracle.fuse_subset(sc.grid, sc.cams, sp, vox, sc.params)
        om = oracle.fuse_subset(sc.grid, sc.cams, sm, vox, sc.params)
        t = target[vox]
        fd = float(np.sum((op - om) * (op + om - 2 * t))) / (2 * H_FD)
        assert abs(g[idx] - fd) <= 5e-3 * abs(fd) + 1e-5 * np.abs(g).max(), (idx, g[idx], fd)
    rec.close()


def test_backward_sequence_equals_per_frame():
    """27 frames (pixel passes of 16 frames, records of 8 + 8, and of 11
    frames, records of 8 + 3): psfs_backward_sequence's d_slm of every frame
    is bit-identical to psfs_backward's, and its d_mean and d_var are the
    frame-ordered FP32 sums of psfs_backward's; NULL outputs are skipped."""
    n = 27
    sc = S.make_scene(seed=31, grid_n=48, cube_side=2.0, n_cams=4, width=160, height=120, focal=150.0,
                      n_frames=n, walking=True)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    imgs = to_dev(sc.images)
    V = rec.n_voxels
    n_pix = imgs[0].numel() // 3
    g = torch.Generator().manual_seed(9)
    d_occ = torch.randn(n, V, generator=g).cuda()
    d_slm = torch.full((n, n_pix), 7.0, device="cuda")
    d_mean = torch.full((n_pix * 3,), 7.0, device="cuda")
    d_var = torch.full((n_pix * 3,), 7.0, device="cuda")
    psfs.psfs_backward_sequence(rec.handle, n, imgs, d_occ, d_slm, d_mean, d_var)
    assert rec.sync() == psfs.PSFS_OK
    sum_m = torch.zeros(n_pix * 3, device="cuda")
    sum_v = torch.zeros(n_pix * 3, device="cuda")
    owned = 0
    for f in range(n):
        s1 = torch.empty(n_pix, device="cuda")
        m1 = torch.empty(n_pix * 3, device="cuda")
        v1 = torch.empty(n_pix * 3, device="cuda")
        psfs.psfs_backward(rec.handle, imgs[f], d_occ[f], s1, m1, v1)
        assert rec.sync() == psfs.PSFS_OK
        np.testing.assert_array_equal(d_slm[f].cpu().numpy(), s1.cpu().numpy(), err_msg=f"frame {f}")
        owned += int((s1 != 0).sum())
        sum_m += m1
        sum_v += v1
    assert owned > 1000
    np.testing.assert_array_equal(d_mean.cpu().numpy(), sum_m.cpu().numpy())
    np.testing.assert_array_equal(d_var.cpu().numpy(), sum_v.cpu().numpy())
    # only the mean gradient
    d_mean2 = torch.full((n_pix * 3,), 7.0, device="cuda")
    psfs.psfs_backward_sequence(rec.handle, n, imgs, d_occ, None, d_mean2, None)
    assert rec.sync() == psfs.PSFS_OK
    np.testing.assert_array_equal(d_mean2.cpu().numpy(), sum_m.cpu().numpy())
    rec.close()


def test_backward_cameras_inside_the_grid_and_deterministic():
    """An 8 m grid that contains the camera ring (voxels behind, beside and in
    front of every camera; long owner segments near the cameras): the adjoint
    against the oracle's, and two calls give the same bits."""
    sc = S.make_scene(seed=14, grid_n=48, cube_side=8.0, n_cams=4, width=160, height=120, focal=150.0)
    rng = np.random.default_rng(14)
    target = rng.uniform(0, 1, size=sc.grid.n_voxels)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    img = to_dev(sc.images)
    occ, _, _ = rec.reconstruct(img)
    d_occ = (2 * (occ.reshape(-1) - to_dev(target.astype(np.float32)))).contiguous()
    n_pix = sc.images.size // 3
    outs = []
    for _ in range(2):
        d_slm = torch.empty(n_pix, dtype=torch.float32, device="cuda")
        d_mean = torch.empty(sc.images.shape, dtype=torch.float32, device="cuda")
        d_var = torch.empty(sc.images.shape, dtype=torch.float32, device="cuda")
        psfs.psfs_backward(rec.handle, img, d_occ, d_slm, d_mean, d_var)
        assert rec.sync() == psfs.PSFS_OK
        outs.append((d_slm.cpu().numpy(), d_mean.cpu().numpy(), d_var.cpu().numpy()))
    for a, b in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(a, b)
    ref = oracle.reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params)
    ds, dm, dv = oracle.backward(sc.grid, sc.cams, sc.images, sc.mean, sc.var, 2 * (ref["occ"] - target), sc.params)
    keep = ~_ambiguous_pixels(sc.grid, sc.cams, ref["boundary"])
    _compare(outs[0][0], ds, keep)
    keep3 = np.repeat(keep, 3)
    _compare(outs[0][1], dm, keep3)
    _compare(outs[0][2], dv, keep3)
    rec.close()


@pytest.mark.parametrize("dtype,bound", [("f16", 2e-2), ("bf16", 2e-1)])
def test_reduced_precision_adjoint_error_vs_fp64(dtype, bound):
    """The adjoint with 16-bit maps (the forward it recomputes sums stored
    16-bit log ratios) against the FP64 oracle's adjoint: the error of d_slm,
    d_mean and d_var relative to each gradient's largest magnitude is
    reported, under a loose sanity bound."""
    sc, target = _frame(sc_seed=45, grid_n=48)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params, map_dtype=dtype)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    img = to_dev(sc.images)
    ref = oracle.reconstruct(sc.grid, sc.cams, sc.images, sc.mean, sc.var, sc.params)
    # the same d_occ on both sides: the FP64 loss gradient at the FP64 occupancy
    d_occ64 = 2 * (ref["occ"] - target)
    d_occ = to_dev(d_occ64.astype(np.float32))
    n_pix = sc.images.size // 3
    d_slm = torch.empty(n_pix, dtype=torch.float32, device="cuda")
    d_mean = torch.empty(sc.images.shape, dtype=torch.float32, device="cuda")
    d_var = torch.empty(sc.images.shape, dtype=torch.float32, device="cuda")
    psfs.psfs_backward(rec.handle, img, d_occ, d_slm, d_mean, d_var)
    assert rec.sync() == psfs.PSFS_OK
    ds, dm, dv = oracle.backward(sc.grid, sc.cams, sc.images, sc.mean, sc.var, d_occ64, sc.params)
    keep = ~_ambiguous_pixels(sc.grid, sc.cams, ref["boundary"])
    keep3 = np.repeat(keep, 3)
    errs = {}
    for name, got, want, k in (("d_slm", d_slm, ds, keep), ("d_mean", d_mean, dm, keep3),
                               ("d_var", d_var, dv, keep3)):
        g, w = got.cpu().numpy().ravel()[k].astype(np.float64), want.ravel()[k]
        errs[name] = float(np.abs(g - w).max() / max(np.abs(w).max(), 1e-30))
    print(dtype, "adjoint error vs FP64 (max |err| / max |grad|):", errs)
    assert max(errs.values()) < bound, errs
    rec.close()


def test_autograd_sequence_function_matches_per_frame():
    """psfs_occupancy_sequence over 10 frames (the sequence forward and the
    batched adjoint): its occupancy equals psfs_occupancy frame by frame bit for
    bit, and its background gradients are the frame-ordered sums of the
    per-frame Function's."""
    n = 10
    sc = S.make_scene(seed=47, grid_n=32, cube_side=2.0, n_cams=4, width=160, height=120, focal=150.0,
                      n_frames=n, walking=True)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    psfs.psfs_set_fuse_config(rec.handle, 8, 4, 4, 0, 2, 8)
    imgs = to_dev(sc.images)
    tgt = torch.from_numpy(np.random.default_rng(47).uniform(0, 1, (n, *rec.shape)).astype(np.float32)).cuda()
    mean = to_dev(sc.mean).requires_grad_(True)
    var = to_dev(sc.var).requires_grad_(True)
    occ = psfs_occupancy_sequence(rec, imgs, mean, var)
    ((occ - tgt) ** 2).sum().backward()
    gm, gv = mean.grad.clone(), var.grad.clone()
    sm = torch.zeros_like(gm)
    sv = torch.zeros_like(gv)
    for f in range(n):
        m1 = to_dev(sc.mean).requires_grad_(True)
        v1 = to_dev(sc.var).requires_grad_(True)
        o1 = psfs_occupancy(rec, imgs[f], m1, v1)
        assert torch.equal(o1, occ[f].detach()), f
        ((o1 - tgt[f]) ** 2).sum().backward()
        sm += m1.grad
        sv += v1.grad
    torch.cuda.synchronize()
    assert torch.equal(gm, sm) and torch.equal(gv, sv)
    assert float(gm.abs().max()) > 0
    rec.close()


def test_backward_from_occupancy_equals_recomputing_adjoint():
    """With the forward's own occupancy the adjoint skips the recomputed maps
    and voxel pass; its outputs must be those of psfs_backward (one frame) and
    psfs_backward_sequence (19 frames: groups of 16 and 3) bit for bit."""
    n = 19
    sc = S.make_scene(seed=48, grid_n=40, cube_side=2.0, n_cams=4, width=160, height=120, focal=150.0,
                      n_frames=n, walking=True)
    rec = psfs.Reconstructor(sc.grid, sc.cams, sc.params)
    rec.set_background(to_dev(sc.mean), to_dev(sc.var))
    imgs = to_dev(sc.images)
    V = rec.n_voxels
    n_pix = imgs[0].numel() // 3
    occ = torch.empty((n, V), device="cuda")
    lst = torch.empty((n, V), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    psfs.psfs_reconstruct_sequence(rec.handle, n, imgs, occ, lst, V, cnt)
    d_occ = torch.randn((n, V), generator=torch.Generator().manual_seed(3)).cuda()
    outs = []
    for fn in ("recompute", "occupancy"):
        s_ = torch.full((n, n_pix), 7.0, device="cuda")
        m_ = torch.full((n_pix * 3,), 7.0, device="cuda")
        v_ = torch.full((n_pix * 3,), 7.0, device="cuda")
        if fn == "recompute":
            psfs.psfs_backward_sequence(rec.handle, n, imgs, d_occ, s_, m_, v_)
        else:
            psfs.psfs_backward_from_occupancy(rec.handle, n, imgs, occ, d_occ, s_, m_, v_)
        assert rec.sync() == psfs.PSFS_OK
        outs.append((s_.cpu(), m_.cpu(), v_.cpu()))
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    # one frame
    s1, m1, v1 = (torch.empty(n_pix, device="cuda"), torch.empty(n_pix * 3, device="cuda"),
                  torch.empty(n_pix * 3, device="cuda"))
    s2, m2, v2 = (torch.empty(n_pix, device="cuda"), torch.empty(n_pix * 3, device="cuda"),
                  torch.empty(n_pix * 3, device="cuda"))
    psfs.psfs_backward(rec.handle, imgs[4], d_occ[4], s1, m1, v1)
    psfs.psfs_backward_from_occupancy(rec.handle, 1, imgs[4], occ[4], d_occ[4], s2, m2, v2)
    assert rec.sync() == psfs.PSFS_OK
    assert torch.equal(s1, s2) and torch.equal(m1, m2) and torch.equal(v1, v2)
    assert torch.equal(s1, outs[0][0][4].cuda())
    rec.close()
