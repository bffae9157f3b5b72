"""The FP64 oracle against the exact posteriors of tests/golden/
one_voxel_posteriors.txt: one voxel seen by K cameras (K coincident pinhole
cameras, each with its own one-pixel likelihood map), the product form of
Eq. 3-4 with Eq. 5's occlusion marginalisation, P(O) = 1/2 (Eq. 6-9 for
P_D = 1, P_FA = 0).  The stored values come from exact rational arithmetic
(make_one_voxel_posteriors.py), not from the oracle or the GPU path."""

import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "one_voxel_posteriors.txt")
ONE_VOXEL_GRID = {"nx": 1, "ny": 1, "nz": 1, "origin": (-0.05, -0.05, -0.05), "voxel_size": 0.1}
CAM = {"width": 1, "height": 1, "K": np.array([[10.0, 0, 0.5], [0, 10.0, 0.5], [0, 0, 1.0]]),
       "R": np.eye(3), "t": np.array([0.0, 0.0, 1.0])}   # the voxel centre projects to (0.5, 0.5)


def _cases():
    with open(GOLDEN) as fh:
        for ln in fh:
            if ln.startswith("#") or not ln.strip():
                continue
            pd, pfa, prior, slms, occ = ln.split()
            yield (float(Fraction(pd)), float(Fraction(pfa)), float(Fraction(prior)),
                   [float(Fraction(s)) for s in slms.split(",")], float(occ))


CASES = list(_cases())


def test_golden_file_has_the_cases():
    assert len(CASES) == 35
    assert any(len(c[3]) == 8 for c in CASES) and any(c[4] == 0.0 for c in CASES)


@pytest.mark.parametrize("pd,pfa,prior,slms,occ", CASES)
def test_oracle_matches_exact_posterior(pd, pfa, prior, slms, occ):
    out = oracle.fuse(ONE_VOXEL_GRID, [CAM] * len(slms), [np.array([[s]]) for s in slms],
                      {"p_detect": pd, "p_false_alarm": pfa, "prior": prior, "threshold": 0.5})
    assert out["n_seen"][0] == len(slms)
    assert abs(out["occ"][0] - occ) < 1e-14
    if abs(occ - 0.5) > 1e-12:
        assert bool(out["occupied"][0]) == (occ > 0.5)


GOLDEN_ADJ = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "one_voxel_adjoint.txt")


def _adjoint_cases():
    with open(GOLDEN_ADJ) as fh:
        for ln in fh:
            if ln.startswith("#") or not ln.strip():
                continue
            pd, pfa, prior, slms, ds = ln.split()
            yield (float(Fraction(pd)), float(Fraction(pfa)), float(Fraction(prior)),
                   [float(Fraction(s)) for s in slms.split(",")], [float(d) for d in ds.split(",")])


ADJ_CASES = list(_adjoint_cases())


@pytest.mark.parametrize("pd,pfa,prior,slms,ds", ADJ_CASES)
def test_oracle_adjoint_matches_exact_derivative(pd, pfa, prior, slms, ds):
    """dLoss/dSLM with dLoss/docc = 1 is d occ / d s_k for every camera k."""
    assert len(ADJ_CASES) >= 30
    maps = np.array([[[s]] for s in slms])
    got = oracle.backward_slm(ONE_VOXEL_GRID, [CAM] * len(slms), maps, np.array([1.0]),
                              {"p_detect": pd, "p_false_alarm": pfa, "prior": prior})
    np.testing.assert_allclose(got.reshape(-1), ds, rtol=1e-12, atol=1e-15)
