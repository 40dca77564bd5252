"""Contact-angle calibration Θ(Δρ) (§2, the particle colour) on the GPU.

The library steps the boxes as one batch; the contact angle follows from the
sphere's height above the far interface (paper_1109_3277_gb300.contact_angle).
Parity: a short run against the FP64 oracle, both analysed through their own
analysis code.  Calibration: Θ(0) = 90° by symmetry, Θ grows with Δρ (the
sign of the paper's fit), and opposite colours give supplementary angles."""
import numpy as np
import pytest

from oracle import analysis, lbref
from paper_1109_3277_gb300 import contact_angle as CA
from paper_1109_3277_gb300 import lbe
from paper_1109_3277_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_short_run_matches_the_oracle():
    """Sphere of radius 4, Δρ = 0.05, in a 24 x 24 x 24 box, 150 steps: the
    sphere height within 1e-5, the far interface within 1e-4 and the
    contact angle within 0.01°."""
    w = W.contact_angle_box(0.05, shape=(24, 24, 24), radius=4.0, steps=150)
    g = lbe.Lattice(w.shape, w.rho0, **w.params)
    r = lbref.Lattice(w.shape, w.rho0, **w.params)
    p = w.particles
    for L in (g, r):
        L.add_particles(p["pos"], p["quat"], p["r_par"], p["r_perp"], p["delta_rho"])
    g.step(w.steps)
    r.step(w.steps)
    zg = g.read_particles()["pos"][0]
    zr = r.read_particles()["pos"][0]
    assert abs(zg[2] - zr[2]) < 1e-5
    col = CA.far_column(w.shape, zg)
    ig = CA.interface_height(g.read_fields(vel=False)[0], *col)
    ir = analysis.interface_z(r.read_fields()[0], col)
    assert abs(ig - ir) < 1e-4
    assert abs(CA.contact_angle(zg[2], ig, 4.0) - analysis.sphere_contact_angle(zr[2], ir, 4.0)) < 1e-2
    g.close()


def test_calibration_is_monotonic_and_symmetric():
    """Δρ in {-0.04, 0, 0.04}, sphere of radius 5 in 48 x 48 x 40, 6000 steps
    (the height settles within about 4000)."""
    res = CA.calibrate([-0.04, 0.0, 0.04], steps=6000, chunk=1000)
    t = res["theta_deg"]
    assert all(res["attached"])
    assert abs(t[1] - 90.0) < 2.0
    assert t[0] < t[1] < t[2]
    assert abs(t[0] + t[2] - 180.0) < 4.0
    assert res["slope_deg"] > 0
    # settled: the last two chunks moved the spheres by less than 0.2
    last = np.asarray(res["trace"][-1]) - np.asarray(res["trace"][-2])
    assert np.all(np.abs(last) < 0.2)
