"""Single-ellipsoid adsorption (§4) through the batched GPU path: an
ellipsoid of aspect ratio 2 and Θ = 90° that starts at φ = 0.0057°, just
dipping into the interface, first moves across the interface without
turning, then turns to the stable point φ ≈ 90°, as the paper's snapshot
series shows; one started at 30° ends there too, and both centres end on
the interface (z = 0 at Θ = 90°)."""
import pytest

from paper_1109_3277_gb300 import adsorption as AD

pytestmark = pytest.mark.gpu


def test_approach_then_rotation_to_the_stable_point():
    res = AD.trajectories([0.0057, 30.0], steps=8000, chunk=1000)
    z, phi = res["z"], res["phi_deg"]
    # first stage: the centre moves more than 5 nodes while the axis stays
    # within 10 degrees of the normal
    assert phi[0][0] < 10.0
    assert abs(z[0][0] - 10.0) > 5.0
    # end: lying in the interface, centre on it
    assert phi[0][-1] > 80.0 and phi[1][-1] > 80.0
    assert abs(z[0][-1]) < 1.5 and abs(z[1][-1]) < 1.5
