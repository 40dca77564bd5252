"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP32 storage and arithmetic against FP64.  One step from random
populations agrees to 2e-6 absolute on populations of order 0.03 (a few FP32
ulps of the largest intermediate); densities after many steps to 1e-5, the
bound of the FP32 path after 200 steps; particle position and orientation to
1e-5 lattice units."""
import numpy as np
import pytest

from oracle import lbref
from paper_1109_3277_gb300 import lbe
from paper_1109_3277_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_F_ONE_STEP = 2e-6
TOL_RHO = 1e-5
TOL_PART = 1e-5


def _pair(shape, rho0, **params):
    mode = params.pop("particle_mode", "free")
    g = lbe.Lattice(shape, rho0, particle_mode=mode, **params)
    r = lbref.Lattice(shape, rho0, particle_mode=lbe.MODES[mode], **params)
    return g, r


def _add(g, r, **p):
    for L in (g, r):
        L.add_particles(p["pos"], p["quat"], p["r_par"], p["r_perp"], p["delta_rho"],
                        vel=p.get("vel"), omega=p.get("omega"))


@pytest.mark.parametrize("flags", [0, lbe.FLAG_TWO_PASS])
@pytest.mark.parametrize("shape,walls,tau", [((8, 8, 8), False, (1.0, 1.0)),
                                             ((13, 7, 5), True, (0.8, 1.3)),
                                             ((33, 17, 9), False, (1.0, 0.7)),
                                             ((70, 35, 40), True, (1.0, 1.0)),
                                             ((1, 1, 1), False, (1.0, 1.0)),
                                             ((3, 2, 1), False, (0.9, 1.1)),
                                             ((2, 1, 3), True, (1.0, 1.0))])
def test_one_step_populations(shape, walls, tau, flags):
    """Several tiles plus a ragged tail (the fused kernel's tiles are 32x8
    and walk z in chunks), walls or not, τ ≠ 1; fused and two-pass fluid
    kernels.  Degenerate lattices: one node (every neighbour is the node
    itself), a single periodic plane, and one fluid plane between walls."""
    nx, ny, nz = shape
    f0 = W.random_populations(shape, seed=21)
    g = lbe.Lattice(shape, np.full((2, nz, ny, nx), 0.5), walls_z=walls, tau=tau, g_br=0.1,
                    body_force=(1e-4, 0.0, -2e-4), flags=flags)
    r = lbref.Lattice(shape, np.full((2, nz, ny, nx), 0.5), walls_z=walls, tau=tau, g_br=0.1,
                      body_force=(1e-4, 0.0, -2e-4))
    g.set_populations(f0)
    r.set_populations(f0)
    g.step(1)
    r.step(1)
    _, _, typ = r.read_fields()
    fl = typ == 0
    fg, fr = g.get_populations(), r.get_populations()
    assert np.max(np.abs(fg[:, :, fl] - fr[:, :, fl])) < TOL_F_ONE_STEP


@pytest.mark.parametrize("flags", [0, lbe.FLAG_TWO_PASS])
def test_spinodal_densities_many_steps(flags):
    shape = (24, 20, 16)
    rho0 = W.uniform_mixture(shape, 0.7, 0.01, seed=22)
    g = lbe.Lattice(shape, rho0, g_br=0.1, flags=flags)
    r = lbref.Lattice(shape, rho0, g_br=0.1)
    g.step(60)
    r.step(60)
    rg, vg, _ = g.read_fields()
    rr, vr, _ = r.read_fields()
    assert np.max(np.abs(rg - rr)) < TOL_RHO
    assert np.max(np.abs(vg - vr)) < TOL_RHO


def test_static_particle_one_step():
    shape = (12, 11, 10)
    f0 = W.random_populations(shape, seed=23)
    g, r = _pair(shape, np.full((2, 10, 11, 12), 0.5), walls_z=True, g_br=0.1,
                 particle_mode="static")
    _add(g, r, pos=[[5.6, 5.2, 4.9]], quat=[W.axis_tilt_quaternion(0.6, 0.3)], r_par=3.6,
         r_perp=2.1, delta_rho=-0.15, vel=[[0.01, -0.02, 0.005]], omega=[[0.003, 0.002, -0.004]])
    _, _, tg = g.read_fields()
    _, _, tr = r.read_fields()
    assert np.array_equal(tg, tr)
    g.set_populations(f0)
    r.set_populations(f0)
    g.step(1)
    r.step(1)
    fl = tr == 0
    fg, fr = g.get_populations(), r.get_populations()
    assert np.max(np.abs(fg[:, :, fl] - fr[:, :, fl])) < TOL_F_ONE_STEP
    pg, pr = g.read_particles(), r.read_particles()
    scale = max(1.0, np.abs(pr["force"]).max())
    assert np.max(np.abs(pg["force"] - pr["force"])) < 1e-5 * scale
    assert np.max(np.abs(pg["torque"] - pr["torque"])) < 1e-5 * max(1.0, np.abs(pr["torque"]).max())


def test_large_particle_links_beyond_the_shell_buffer():
    """A sphere of radius 14 has about 3,000 shell nodes, more than the
    shell kernel collects per particle in shared memory (1,024): the rest
    enter the link list directly.  One step of a moving static sphere
    against the oracle: populations, and the momentum exchange."""
    shape = (40, 40, 40)
    f0 = W.random_populations(shape, seed=29)
    g, r = _pair(shape, np.full((2, 40, 40, 40), 0.5), g_br=0.1, particle_mode="static")
    _add(g, r, pos=[[19.6, 20.3, 19.8]], quat=[W.axis_tilt_quaternion(0.4, 0.7)], r_par=14.2,
         r_perp=13.8, delta_rho=0.05, vel=[[0.01, -0.015, 0.02]], omega=[[0.001, -0.002, 0.0015]])
    _, _, tg = g.read_fields()
    _, _, tr = r.read_fields()
    assert np.array_equal(tg, tr)
    g.set_populations(f0)
    r.set_populations(f0)
    g.step(1)
    r.step(1)
    fl = tr == 0
    fg, fr = g.get_populations(), r.get_populations()
    assert np.max(np.abs(fg[:, :, fl] - fr[:, :, fl])) < TOL_F_ONE_STEP
    pg, pr = g.read_particles(), r.read_particles()
    scale = max(1.0, np.abs(pr["force"]).max())
    assert np.max(np.abs(pg["force"] - pr["force"])) < 1e-5 * scale
    assert np.max(np.abs(pg["torque"] - pr["torque"])) < 1e-5 * max(1.0, np.abs(pr["torque"]).max())


def test_prescribed_motion_fill_empty():
    """A particle driven through the lattice: coverage changes every few
    steps, exercising fill and empty."""
    shape = (24, 20, 20)
    rho0 = W.flat_interface(shape, 10, 0.7, 0.04, 1e-3, seed=24)
    g, r = _pair(shape, rho0, walls_z=True, g_br=0.1, particle_mode="prescribed")
    _add(g, r, pos=[[8.2, 9.7, 10.3]], quat=[W.axis_tilt_quaternion(0.7, 0.2)], r_par=5.0,
         r_perp=2.5, delta_rho=0.1, vel=[[0.06, 0.01, -0.02]], omega=[[0.0, 0.01, 0.004]])
    for _ in range(4):
        g.step(10)
        r.step(10)
        rg, _, tg = g.read_fields()
        rr, _, tr = r.read_fields()
        assert np.array_equal(tg, tr)
        assert np.max(np.abs(rg - rr)) < TOL_RHO
    pg, pr = g.read_particles(), r.read_particles()
    assert np.max(np.abs(pg["pos"] - pr["pos"])) < 1e-9
    assert np.max(np.abs(pg["force"] - pr["force"])) < 1e-4 * max(1.0, np.abs(pr["force"]).max())


@pytest.mark.parametrize("flags", [0, lbe.FLAG_TWO_PASS])
def test_adsorption_box_200_steps(flags):
    """The 32x32x48 adsorption box with one free prolate ellipsoid (r_par 6,
    r_perp 3) tilted 45 degrees on the interface, 200 steps: densities within
    1e-5, particle position and orientation within 1e-5."""
    w = W.adsorption_box()
    g = lbe.Lattice(w.shape, w.rho0, flags=flags, **w.params)
    r = lbref.Lattice(w.shape, w.rho0, **w.params)
    p = w.particles
    _add(g, r, **p)
    g.step(w.steps)
    r.step(w.steps)
    rg, _, tg = g.read_fields()
    rr, _, tr = r.read_fields()
    both = (tg == 0) & (tr == 0)
    assert (tg != tr).sum() == 0
    assert np.max(np.abs(rg[:, both] - rr[:, both])) < TOL_RHO
    pg, pr = g.read_particles(), r.read_particles()
    assert np.max(np.abs(pg["pos"] - pr["pos"])) < TOL_PART
    qg, qr = pg["quat"] * np.sign(pg["quat"][:, :1]), pr["quat"] * np.sign(pr["quat"][:, :1])
    assert np.max(np.abs(qg - qr)) < TOL_PART
    # the particle did move
    assert np.linalg.norm(pr["pos"][0] - p["pos"][0]) > 1e-3


def test_free_particles_hertz_contact():
    """Free ellipsoids in a periodic box, two of them in slight end-to-end
    Hertz overlap (Eq. 6-8), one straddling the periodic corner;
    lubrication off."""
    shape = (36, 30, 28)
    rho0 = W.random_phases(shape, 0.5, seed=25)
    g, r = _pair(shape, rho0, g_br=0.1, lub_cut=0.0)
    pos = [[10.0, 10.0, 10.0], [10.0, 10.0, 17.97], [22.5, 10.5, 10.0], [30.0, 22.0, 20.0],
           [1.0, 25.5, 1.5]]
    quats = [W.axis_tilt_quaternion(0.0), W.axis_tilt_quaternion(0.0),
             W.axis_tilt_quaternion(np.pi / 2, 0.0), W.axis_tilt_quaternion(1.0, 2.0),
             W.axis_tilt_quaternion(0.4, 1.0)]
    _add(g, r, pos=pos, quat=quats, r_par=4.0, r_perp=2.0, delta_rho=[0.0, 0.1, -0.1, 0.05, 0.0],
         vel=[[0.0, 0.0, 0.002], [0.0, 0.0, -0.002], [-0.005, 0, 0], [0.002, 0.001, 0.0],
              [0.0, 0.0, 0.0]])
    g.step(1)
    r.step(1)
    pg, pr = g.read_particles(), r.read_particles()
    scale = max(1.0, np.abs(pr["force"]).max())
    assert np.abs(pr["force"]).max() > 0.1  # Hertz overlap is active
    assert np.max(np.abs(pg["force"] - pr["force"])) < 1e-5 * scale
    assert np.max(np.abs(pg["torque"] - pr["torque"])) < 1e-5 * max(scale, np.abs(pr["torque"]).max())
    g.step(39)
    r.step(39)
    pg, pr = g.read_particles(), r.read_particles()
    assert np.max(np.abs(pg["vel"])) < 0.05  # a physically sane run
    assert np.max(np.abs(pg["pos"] - pr["pos"])) < TOL_PART
    qg, qr = pg["quat"] * np.sign(pg["quat"][:, :1]), pr["quat"] * np.sign(pr["quat"][:, :1])
    assert np.max(np.abs(qg - qr)) < TOL_PART
    rg, _, tg = g.read_fields()
    rr, _, tr = r.read_fields()
    assert np.array_equal(tg, tr)
    assert np.max(np.abs(rg - rr)) < TOL_RHO


def test_lubrication_gap():
    """Two ellipsoids side by side at a gap of 0.45 < Δc closing slowly: the
    lubrication correction (Eq. 9 generalised with σ) opposes the approach."""
    shape = (32, 24, 24)
    rho0 = W.uniform_mixture(shape, 0.7, 0.0, seed=1)
    g, r = _pair(shape, rho0, g_br=0.0)
    q = W.axis_tilt_quaternion(np.pi / 2, 0.0)  # both axes along x, separation along y
    pos = [[16.0, 9.775, 12.0], [16.0, 14.225, 12.0]]
    vel = [[0.0, 0.001, 0.0], [0.0, -0.001, 0.0]]
    _add(g, r, pos=pos, quat=[q, q], r_par=5.0, r_perp=2.0, delta_rho=0.0, vel=vel)
    g.step(1)
    r.step(1)
    pg, pr = g.read_particles(), r.read_particles()
    # the pair force on particle 0 points away from particle 1 (-y)
    assert pr["force"][0, 1] < 0 and pr["force"][1, 1] > 0
    # the momentum exchange sums O(100) FP32 link terms of order 0.03: its
    # rounding floor is absolute, ~1e-6, whatever the net force
    assert np.max(np.abs(pg["force"] - pr["force"])) < 1e-5 * max(1.0, np.abs(pr["force"]).max())
    g.step(29)
    r.step(29)
    pg, pr = g.read_particles(), r.read_particles()
    assert np.max(np.abs(pg["pos"] - pr["pos"])) < TOL_PART


def test_mass_sums_and_conservation():
    shape = (40, 36, 30)
    rho0 = W.random_phases(shape, 0.5, seed=26)
    g, r = _pair(shape, rho0, g_br=0.1)
    m0 = g.mass()
    assert np.allclose(m0, r.mass(), rtol=1e-7)
    g.step(100)
    m1 = g.mass()
    assert np.all(np.abs(m1 - m0) / m0 < 1e-6)


@pytest.mark.parametrize("storage,tol", [("f16", 2e-4), ("bf16", 2e-3)])
def test_16bit_offset_storage(storage, tol):
    """FP32 arithmetic with populations stored as 16-bit offsets from
    w_i ρ_ref: error against the FP64 oracle bounded by the storage
    precision after 20 steps."""
    shape = (20, 18, 16)
    rho0 = W.random_phases(shape, 0.5, seed=27)
    g = lbe.Lattice(shape, rho0, g_br=0.1, storage=storage, rho_ref=(0.37, 0.37))
    r = lbref.Lattice(shape, rho0, g_br=0.1)
    g.step(20)
    r.step(20)
    rg, _, _ = g.read_fields()
    rr, _, _ = r.read_fields()
    assert np.max(np.abs(rg - rr)) < tol
    m = g.mass()
    assert np.allclose(m, r.mass(), rtol=5 * tol)


def test_graph_and_direct_launches_agree():
    """lbe_step(n) replays a captured 2-step graph; odd counts launch
    directly.  Both routes give bit-identical results."""
    shape = (16, 16, 16)
    rho0 = W.uniform_mixture(shape, 0.7, 0.01, seed=28)
    a = lbe.Lattice(shape, rho0, g_br=0.1)
    b = lbe.Lattice(shape, rho0, g_br=0.1)
    a.step(10)
    for _ in range(10):
        b.step(1)
    fa, fb = a.get_populations(), b.get_populations()
    assert np.array_equal(fa, fb)


def test_invalid_arguments_are_rejected():
    shape = (8, 8, 8)
    rho0 = np.full((2, 8, 8, 8), 0.5)
    with pytest.raises(lbe.LbeError):
        lbe.Lattice(shape, rho0, tau=(0.4, 1.0))
    with pytest.raises(lbe.LbeError):
        lbe.Lattice((8, 8, 2), rho0[:, :2], walls_z=True)
    g = lbe.Lattice(shape, rho0)
    with pytest.raises(lbe.LbeError):
        g.add_particles([[9.0, 1.0, 1.0]], [[1, 0, 0, 0]], 2.0, 1.0, 0.0)
    with pytest.raises(lbe.LbeError):
        g.add_particles([[4.0, 4.0, 4.0]], [[1, 0, 0, 0]], -2.0, 1.0, 0.0)
    g.step(2)
    assert np.all(np.isfinite(g.mass()))


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_wide_store_offsets_give_identical_results(storage):
    """The fused kernel's 32-bit store offsets (from the node's component)
    and its 64-bit ones (from the array base) address the same slots: walls,
    a moving particle and periodic wraps, with and without TMA staging
    (nx = 24 and nx = 13), bit for bit."""
    for shape, walls in (((24, 20, 20), True), ((13, 11, 10), False)):
        nx, ny, nz = shape
        rho0 = W.flat_interface(shape, nz // 2, 0.7, 0.04, 1e-3, seed=41)
        out = []
        for flags in (0, lbe.FLAG_WIDE_OFFSETS):
            g = lbe.Lattice(shape, rho0, walls_z=walls, g_br=0.1, storage=storage, flags=flags)
            g.add_particles([[nx / 2 - 0.3, ny / 2 + 0.2, nz / 2]], [W.axis_tilt_quaternion(0.7, 0.2)],
                            4.0, 2.0, 0.1, vel=[[0.02, 0.01, -0.01]], omega=[[0.0, 0.01, 0.004]])
            g.step(12)
            out.append((g.get_populations(), g.read_particles()["pos"]))
            g.close()
        assert np.array_equal(out[0][0], out[1][0])
        assert np.array_equal(out[0][1], out[1][1])
