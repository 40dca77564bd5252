"""Pins of the observables of §4 (domain size L(t), interface area, tilt)."""
import numpy as np
import pytest

from oracle import analysis
from paper_1109_3277_gb300 import workloads as W


@pytest.mark.parametrize("lam", [8, 16, 32])
def test_single_mode_domain_size_is_wavelength(lam):
    """A single sine mode of wavelength λ along x gives <k_x^2> = (2π/λ)^2
    and L_x = λ exactly (both the squared reading and the printed |·|)."""
    n = 64
    x = np.arange(n)
    phi = np.sin(2 * np.pi * x / lam)[None, None, :] * np.ones((n // 2, n // 4, 1))
    rho = np.stack([0.5 + 0.1 * phi, 0.5 - 0.1 * phi])
    _, (lx, ly, lz) = analysis.domain_size(rho)
    assert abs(lx - lam) < 1e-9
    assert np.isinf(ly) and np.isinf(lz)
    _, (lx2, _, _) = analysis.domain_size(rho, squared=False)
    assert abs(lx2 - lam) < 1e-9


def test_two_modes_mixed_size():
    n = 64
    z, y, x = np.mgrid[0:n, 0:n, 0:n]
    phi = np.sin(2 * np.pi * x / 16) + np.sin(2 * np.pi * y / 32)
    rho = np.stack([phi, -phi]) * 0.05 + 0.5
    _, (lx, ly, lz) = analysis.domain_size(rho)
    # S has equal weight on both modes: <k_x^2> = (2π/16)^2 / 2
    assert abs(lx - 16 * np.sqrt(2)) < 1e-9
    assert abs(ly - 32 * np.sqrt(2)) < 1e-9


def test_flat_interface_area():
    """Reading: area = number of axis links crossing the sign of φ.  A
    periodic slab has two flat interfaces of nx*ny links each; with walls
    the open z direction has one."""
    shape = (12, 10, 20)
    rho = W.flat_interface(shape, 10, 0.7, 0.04, 0.0)
    assert analysis.interface_area(rho) == 2 * 12 * 10
    assert analysis.interface_area(rho, periodic=(True, True, False)) == 12 * 10
    fluid = np.ones((20, 10, 12), dtype=bool)
    fluid[:, :, :3] = False
    assert analysis.interface_area(rho, fluid=fluid, periodic=(True, True, False)) == 9 * 10


def test_tilt_closed_forms():
    for t in (0.0, 0.3, np.pi / 4, 1.2, np.pi / 2):
        q = W.axis_tilt_quaternion(t, 0.7)
        assert abs(analysis.tilt(q)[0] - t) < 1e-12
    # a symmetry axis pointing down is the same tilt as pointing up
    assert abs(analysis.tilt(W.axis_tilt_quaternion(np.pi - 0.4, 1.0))[0] - 0.4) < 1e-12


def _column_field(phi_z, nx=4, ny=3):
    """rho [2, nz, ny, nx] whose φ = ρ_r − ρ_b is phi_z on every column."""
    phi_z = np.asarray(phi_z, dtype=np.float64)
    r = 0.5 + 0.5 * phi_z
    b = 0.5 - 0.5 * phi_z
    return np.stack([np.broadcast_to(r[:, None, None], (phi_z.size, ny, nx)),
                     np.broadcast_to(b[:, None, None], (phi_z.size, ny, nx))])


def test_interface_height_closed_forms():
    z = np.arange(40, dtype=np.float64)
    # a linear profile crosses exactly where the line does
    assert analysis.interface_z(_column_field(0.03 * (17.3 - z)), (1, 2)) == pytest.approx(17.3, abs=1e-12)
    # a profile odd about a midpoint between nodes crosses at the midpoint
    assert analysis.interface_z(_column_field(np.tanh((20.5 - z) / 2.0)), (0, 0)) == pytest.approx(20.5, abs=1e-12)
    # no crossing between the walls
    assert np.isnan(analysis.interface_z(_column_field(np.ones(40)), (0, 0)))
    # a slab has two crossings: the one nearest mid-height
    slab = np.where((z > 8) & (z < 25), 1.0, -1.0)
    assert analysis.interface_z(_column_field(slab), (0, 0)) == pytest.approx(24.5, abs=1e-12)


@pytest.mark.parametrize("theta", [0.0, 30.0, 90.0, 131.0, 180.0])
def test_sphere_contact_angle_against_wetted_area(theta):
    """The fraction of a sphere's surface below a plane through the contact
    circle is (1 + cos Θ)/2 (Archimedes); a seeded uniform sample of the
    surface recovers Θ from the centre height through that fraction."""
    R, zi = 5.0, 19.5
    zc = zi - R * np.cos(np.radians(theta))
    assert analysis.sphere_contact_angle(zc, zi, R) == pytest.approx(theta, abs=1e-9)
    u = W.uniform(7, (200000,), stream=9, lo=-1.0, hi=1.0)  # z of uniform points on the unit sphere
    below = np.mean(zc + R * u < zi)
    est = np.degrees(np.arccos(np.clip(2 * below - 1, -1, 1)))
    assert est == pytest.approx(theta, abs=1.0)


def test_package_contact_angle_analysis_matches_the_oracle():
    """The library's host analysis (used by the calibration and the bench)
    and the oracle's give the same heights and angles on the same fields."""
    from paper_1109_3277_gb300 import contact_angle as CA
    z = np.arange(36, dtype=np.float64)
    for z0, w in ((17.3, 1.5), (20.0, 2.0), (12.75, 3.0)):
        rho = _column_field(np.tanh((z0 - z) / w))
        a = CA.interface_height(rho, 2, 1)
        b = analysis.interface_z(rho, (2, 1))
        assert a == pytest.approx(b, abs=1e-12)
        for zc in (z0 - 4.0, z0, z0 + 2.5):
            assert CA.contact_angle(zc, a, 5.0) == pytest.approx(analysis.sphere_contact_angle(zc, b, 5.0), abs=1e-9)


def test_package_tilt_matches_the_oracle():
    """The adsorption driver's tilt and the oracle's agree on seeded random
    orientations and on the axis-tilt construction."""
    from paper_1109_3277_gb300 import adsorption as AD
    q = W.random_quaternions(5, 64)
    for k in range(64):
        assert AD.tilt_deg(q[k]) == pytest.approx(np.degrees(analysis.tilt(q[k])[0]), abs=1e-9)
    for t in (0.0, 0.0057, 10.0, 45.0, 89.0, 90.0):
        assert AD.tilt_deg(W.axis_tilt_quaternion(np.radians(t))) == pytest.approx(t, abs=1e-7)


def test_package_domain_size_matches_the_oracle():
    """The study's real-FFT domain size and the oracle's full-FFT one agree
    on seeded fields with and without solid nodes, and give the wavelength
    of a single mode."""
    from paper_1109_3277_gb300 import domain as D
    shape = (24, 20, 16)
    nx, ny, nz = shape
    rho = W.uniform(3, (2, nz, ny, nx), stream=11, lo=0.0, hi=1.0)
    fluid = W.uniform(3, (nz, ny, nx), stream=12) > 0.2
    for fl in (None, fluid):
        a = D.domain_size(rho, fl)
        b = analysis.domain_size(rho, fl)
        assert a[0] == pytest.approx(b[0], rel=1e-12)
        assert np.allclose(a[1], b[1], rtol=1e-12)
    x = np.arange(nx)
    phi = np.broadcast_to(np.sin(2 * np.pi * x / 8.0)[None, None, :], (nz, ny, nx))
    L, (lx, _, _) = D.domain_size(np.stack([0.5 + 0.5 * phi, 0.5 - 0.5 * phi]))
    assert lx == pytest.approx(8.0, rel=1e-12)
    assert D.fit_inverse([0.1, 0.2, 0.25], [2.2 / 0.1 + 11.08, 2.2 / 0.2 + 11.08, 2.2 / 0.25 + 11.08]) == \
        pytest.approx((2.2, 11.08), rel=1e-12)


def test_study_drivers_run_on_the_oracle():
    """The calibration and domain-size drivers, with the oracle's lattice
    class standing in for the library's (tiny boxes, few steps): their
    bookkeeping of chunks, heights, angles, concentrations and fits."""
    from oracle import lbref
    from paper_1109_3277_gb300 import contact_angle as CA
    from paper_1109_3277_gb300 import domain as D
    r = CA.calibrate([-0.05, 0.05], steps=30, shape=(16, 16, 16), radius=3.0, chunk=15,
                     lattice=lbref.Lattice)
    assert len(r["trace"]) == 2 and all(len(t) == 2 for t in r["trace"])
    assert all(np.isfinite(r["theta_deg"])) and all(0.0 <= t <= 180.0 for t in r["theta_deg"])
    for h, t in zip(r["height"], r["theta_deg"]):
        assert t == pytest.approx(np.degrees(np.arccos(np.clip(-h / 3.0, -1, 1))), abs=1e-9)
    d = D.study([0.1, 0.2], n=32, steps=20, checkpoint=10, lattice=lbref.Lattice)
    assert d["step"] == [10, 20] and all(len(s) == 2 for s in d["L"])
    assert all(np.isfinite(d["L_final"])) and all(L > 0 for L in d["L_final"])
    vol = 4.0 / 3.0 * np.pi * 8.0 * 4.0 * 4.0
    assert d["C_placed"] == pytest.approx([p * vol / 32 ** 3 for p in d["particles"]], rel=1e-12)
    assert np.isfinite(d["a"]) and np.isfinite(d["b"])
    from paper_1109_3277_gb300 import adsorption as AD
    t = AD.trajectories([10.0, 80.0], steps=20, chunk=10, lattice=lbref.Lattice, edge=24, r_par=6.0,
                        r_perp=3.0)
    assert t["step"] == [10, 20] and all(len(z) == 2 for z in t["z"])
    # after 10 of the first steps the ellipsoids have barely moved or turned
    assert t["phi_deg"][0][0] == pytest.approx(10.0, abs=0.5) and t["phi_deg"][1][0] == pytest.approx(80.0, abs=0.5)
    for k, tilt in enumerate((10.0, 80.0)):
        half = np.hypot(6.0 * np.cos(np.radians(tilt)), 3.0 * np.sin(np.radians(tilt)))
        assert t["z"][k][0] == pytest.approx(half - 2.0 + 0.5, abs=0.3)
