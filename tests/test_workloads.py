"""The seeded input generators: SplitMix64 against its published test
sequence, determinism, placement without overlap."""
import numpy as np
import pytest

from paper_1109_3277_gb300 import workloads as W


def test_splitmix64_reference_sequence():
    # state 1234567: first outputs of the reference SplitMix64 generator
    got = W.splitmix64(0, 5, stream=1234567)
    assert [int(v) for v in got] == [6457827717110365317, 3203168211198807973,
                                     9817491932198370423, 4593380528125082431,
                                     16408922859458223821]


def test_uniform_deterministic_and_in_range():
    a = W.uniform(5, (1000,), stream=3)
    b = W.uniform(5, (1000,), stream=3)
    assert np.array_equal(a, b)
    assert a.min() >= 0 and a.max() < 1 and abs(a.mean() - 0.5) < 0.05
    assert not np.array_equal(a, W.uniform(5, (1000,), stream=4))


def test_quaternions_unit_and_uniform_axis():
    q = W.random_quaternions(3, 4000)
    assert np.allclose(np.linalg.norm(q, axis=1), 1.0)
    w, x, y, z = q.T
    axz = 2 * (x * z - w * y)
    # uniform axis directions: cos(polar angle) uniform on [-1, 1]
    assert abs(axz.mean()) < 0.05 and abs((axz ** 2).mean() - 1 / 3) < 0.03


def test_placement_no_overlap():
    shape = (40, 40, 40)
    pos, quat = W.place_ellipsoids(shape, 30, 4.0, 2.0, seed=2)
    assert len(pos) == 30
    occ = np.zeros((40, 40, 40), dtype=int)
    for p, q in zip(pos, quat):
        X, Y, Z = W._inflated_nodes(shape, p, q, 4.0, 2.0, 0.0, (True, True, True))
        occ[Z, Y, X] += 1
    assert occ.max() == 1


def test_workload_recipes():
    w = W.adsorption_box()
    assert w.shape == (32, 32, 48) and w.params["walls_z"]
    assert w.rho0.shape == (2, 48, 32, 32)
    assert abs(w.rho0[0, 10].mean() - 0.7) < 1e-3 and abs(w.rho0[0, 40].mean() - 0.04) < 1e-3
    r = W.adsorption_request(7, 3)
    e = r.shape[0]
    assert 32 <= e <= 96 and r.shape == (e, e, e)
    rmax = max(r.particles["r_par"][0], r.particles["r_perp"][0])
    assert 2 * rmax + 6 <= e
    assert r.particles["pos"][0, 2] + rmax < e - 1


def test_study_recipes():
    """The calibration and study boxes: shapes, walls, the interface, and
    particles placed as stated."""
    c = W.contact_angle_box(0.04)
    assert c.shape == (48, 48, 40) and c.params["walls_z"]
    assert np.allclose(c.particles["pos"][0], [24.0, 24.0, 20.0])
    assert c.particles["r_par"][0] == c.particles["r_perp"][0] == 5.0 and c.particles["delta_rho"][0] == 0.04
    assert abs(c.rho0[0, 10].mean() - 0.7) < 1e-3 and abs(c.rho0[1, 30].mean() - 0.7) < 1e-3
    for tilt in (0.0057, 45.0, 90.0):
        a = W.adsorption_study_box(tilt)
        q = a.particles["quat"][0]
        axis_z = 2 * (q[1] * q[3] - q[0] * q[2])
        assert np.degrees(np.arccos(min(1.0, abs(axis_z)))) == pytest.approx(tilt, abs=1e-6)
        # the lowest point dips 2 nodes below the interface plane z = 32
        t = np.radians(tilt)
        half = np.hypot(12.0 * np.cos(t), 6.0 * np.sin(t))
        assert a.particles["pos"][0, 2] - half == pytest.approx(30.0, abs=1e-12)
    b = W.bijel_study_box(0.2, n=64)
    vol = 4.0 / 3.0 * np.pi * 8.0 * 4.0 * 4.0
    assert len(b.particles["pos"]) == int(round(0.2 * 64 ** 3 / vol))
    assert b.params["g_br"] == 0.08 and not b.params["walls_z"]
    # random initial densities, 1:1, uniform in [0, 1.4) per component
    assert b.rho0.min() >= 0.0 and b.rho0.max() < 1.4
    assert np.allclose(b.rho0.reshape(2, -1).mean(axis=1), 0.7, atol=0.01)
