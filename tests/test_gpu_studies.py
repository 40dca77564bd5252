"""The two study drivers (§4) on the GPU against the FP64 oracle, each run
through the same driver with the oracle's lattice class in place of the
library's:

- the single-ellipsoid adsorption study's own box (64^3, walls, radii 12 and
  6, Θ = 90°) for 200 steps: the centre's height above the far interface
  and the tilt after every 100 steps;
- the domain-size study on a 64^3 bijel box (aspect ratio 2 at concentration
  0.12, g = 0.08) for 200 steps: the domain size L after every 100 steps.

The tolerances are those of the other 200-step comparisons: positions 1e-5
lattice units, orientations 1e-5 rad; the domain size, a statistic of the
whole field, to 1e-5 relative."""
import numpy as np
import pytest

from oracle import lbref
from paper_1109_3277_gb300 import adsorption as AD
from paper_1109_3277_gb300 import domain as DS

pytestmark = pytest.mark.gpu


def test_adsorption_study_box_matches_the_oracle():
    gpu = AD.trajectories([30.0], steps=200, chunk=100)
    ref = AD.trajectories([30.0], steps=200, chunk=100, lattice=lbref.Lattice)
    assert gpu["step"] == ref["step"] == [100, 200]
    zg, zr = np.array(gpu["z"][0]), np.array(ref["z"][0])
    pg, pr = np.array(gpu["phi_deg"][0]), np.array(ref["phi_deg"][0])
    assert np.max(np.abs(zg - zr)) < 1e-5, (zg, zr)
    assert np.max(np.abs(np.radians(pg - pr))) < 1e-5, (pg, pr)
    # the particle moved (the comparison is not of a resting state)
    assert abs(zr[-1] - zr[0]) > 1e-3 or abs(pr[-1] - pr[0]) > 1e-3


def test_domain_size_study_matches_the_oracle():
    kw = dict(n=64, steps=200, checkpoint=100)
    gpu = DS.study([0.12], storage="f32", **kw)
    ref = DS.study([0.12], lattice=lbref.Lattice, **kw)
    assert gpu["particles"] == ref["particles"] and gpu["particles"][0] > 10
    Lg, Lr = np.array(gpu["L"][0]), np.array(ref["L"][0])
    assert np.all(np.isfinite(Lr)) and np.all(Lr > 2.0)
    assert np.max(np.abs(Lg - Lr) / Lr) < 1e-5, (Lg, Lr)
