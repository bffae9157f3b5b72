"""Pins of the oracle's adjoint: FP64 central finite differences of the
oracle's forward (Eq. 1-9), an independent computation from the analytic
adjoint (which scatters dLoss/docc through the derivative of Eq. 4-9 and of
Eq. 1-2).

Loss = sum_v (occ_v - target_v)^2.  The loss difference of a central pair is
summed as (occ+ - occ-)(occ+ + occ- - 2 target), so that voxels the
perturbation does not reach contribute exactly zero.
"""

import numpy as np
import pytest

import oracle
from synth import scene as S

H_FD = 1e-4
P = {"p_detect": 0.9, "p_false_alarm": 0.1, "prior": 0.5}


def _scene():
    sc = S.make_scene(seed=21, grid_n=20, cube_side=2.0, n_cams=4, width=96, height=72,
                      focal=90.0)
    return sc, sc.grid.as_dict()


def _dloss(occ_p, occ_m, target):
    return float(np.sum((occ_p - occ_m) * (occ_p + occ_m - 2 * target)))


@pytest.mark.parametrize("P", [P, {"p_detect": 0.8, "p_false_alarm": 0.3, "prior": 0.4}])
def test_backward_slm_matches_finite_differences(P):
    """dLoss/dSLM on 200 seeded pixels: 150 that some voxel projects to and
    50 that none does (gradient exactly 0 on both sides).  The second rate
    pair has P_D + P_FA != 1, so P(S|V=0) depends on s and its term counts."""
    sc, grid = _scene()
    s = oracle.slm(sc.images, sc.mean, sc.var)
    rng = np.random.default_rng(4)
    target = rng.uniform(0, 1, size=sc.grid.n_voxels)
    occ = oracle.fuse(grid, sc.cams, s, P)["occ"]
    ds = oracle.backward_slm(grid, sc.cams, s, 2 * (occ - target), P)
    owned = np.flatnonzero(ds.ravel() != 0)
    unowned = np.flatnonzero(ds.ravel() == 0)
    assert owned.size >= 150 and unowned.size >= 50
    pick_owned = rng.choice(owned, 150, replace=False)
    pick_unowned = rng.choice(unowned, 50, replace=False)
    for idx, is_owned in [(i, True) for i in pick_owned] + [(i, False) for i in pick_unowned]:
        sp = s.copy().ravel()
        sm = s.copy().ravel()
        sp[idx] += H_FD
        sm[idx] -= H_FD
        op = oracle.fuse(grid, sc.cams, sp.reshape(s.shape), P)["occ"]
        om = oracle.fuse(grid, sc.cams, sm.reshape(s.shape), P)["occ"]
        fd = _dloss(op, om, target) / (2 * H_FD)
        an = ds.ravel()[idx]
        if is_owned:
            assert abs(fd - an) <= 1e-4 * abs(an) + 1e-12, (idx, fd, an)
        else:
            assert fd == 0.0 and an == 0.0


def test_backward_background_matches_finite_differences():
    """dLoss/dmean and dLoss/dvar through Eq. 1-2, one seeded channel per pixel.
    The step is 2^-13 (~1.2e-4), a multiple of the float32 spacing of every
    mean and variance in the scene, so both perturbed inputs are exact."""
    sc, grid = _scene()
    rng = np.random.default_rng(9)
    target = rng.uniform(0, 1, size=sc.grid.n_voxels)
    s = oracle.slm(sc.images, sc.mean, sc.var)
    occ = oracle.fuse(grid, sc.cams, s, P)["occ"]
    ds, dm, dv = oracle.backward(grid, sc.cams, sc.images, sc.mean, sc.var, 2 * (occ - target), P)
    ssum = (s * (1 - s)).ravel()
    cand = np.flatnonzero((np.abs(ds.ravel()) > 1e-3) & (ssum > 1e-2))
    assert cand.size >= 40
    pick = rng.choice(cand, 40, replace=False)
    h = 2.0 ** -13
    assert sc.mean.max() < 256 and sc.var.max() < 256

    def occ_of(mean, var):
        return oracle.fuse(grid, sc.cams, oracle.slm(sc.images, mean, var), P)["occ"]

    for idx in pick:
        c = int(rng.integers(0, 3))
        flat = idx * 3 + c
        for which, an_arr in (("mean", dm), ("var", dv)):
            arr = sc.mean if which == "mean" else sc.var
            ap = arr.copy().ravel()
            am = arr.copy().ravel()
            ap[flat] = np.float32(float(ap[flat]) + h)
            am[flat] = np.float32(float(am[flat]) - h)
            assert float(ap[flat]) - float(arr.ravel()[flat]) == h
            if which == "mean":
                op, om = occ_of(ap.reshape(arr.shape), sc.var), occ_of(am.reshape(arr.shape), sc.var)
            else:
                op, om = occ_of(sc.mean, ap.reshape(arr.shape)), occ_of(sc.mean, am.reshape(arr.shape))
            fd = _dloss(op, om, target) / (2 * h)
            an = an_arr.ravel()[flat]
            assert abs(fd - an) <= 1e-5 * abs(an) + 1e-12, (which, idx, c, fd, an)
