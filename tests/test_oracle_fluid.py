"""Pins of the oracle's fluid step (Eq. 1-3 and the shifted-velocity forcing
of §2) against closed forms, conservation laws, textbook flows and a literal
brute-force evaluation."""
import numpy as np
import pytest

from oracle import lbref
from paper_1109_3277_gb300 import workloads as W
from tests import bruteforce


def _lattice(shape, rho0, **kw):
    return lbref.Lattice(shape, rho0, **kw)


@pytest.mark.parametrize("walls", [False, True])
def test_bruteforce_one_step_fluid(walls):
    shape = (8, 8, 8)
    f0 = W.random_populations(shape, seed=7)
    L = _lattice(shape, np.full((2, 8, 8, 8), 0.5), walls_z=walls, tau=(1.0, 0.8), g_br=0.1,
                 body_force=(1e-3, -2e-3, 5e-4))
    L.set_populations(f0)
    L.step(1)
    got = L.get_populations()
    want, _, _, typ = bruteforce.step(shape, f0, walls, (1.0, 0.8), 0.1, (1e-3, -2e-3, 5e-4), [])
    fluid = np.zeros((8, 8, 8), dtype=bool)
    for (x, y, z), t in typ.items():
        fluid[z, y, x] = t == 0
    assert np.max(np.abs(got[:, :, fluid] - want[:, :, fluid])) < 1e-14


def test_bruteforce_one_step_static_particle():
    """Moving bounce-back (Eq. 4) and momentum exchange (Eq. 5) with a
    particle that is held in place but carries a surface velocity."""
    shape = (8, 8, 8)
    f0 = W.random_populations(shape, seed=8)
    P = dict(pos=[3.6, 4.2, 3.9], quat=W.axis_tilt_quaternion(0.6, 0.3), r_par=2.6, r_perp=1.7,
             delta_rho=-0.15, vel=[0.01, -0.02, 0.005], omega=[0.003, 0.002, -0.004])
    L = _lattice(shape, np.full((2, 8, 8, 8), 0.5), walls_z=True, tau=(1.0, 1.0), g_br=0.1,
                 particle_mode=1)
    L.add_particles([P["pos"]], [P["quat"]], P["r_par"], P["r_perp"], P["delta_rho"],
                    vel=[P["vel"]], omega=[P["omega"]])
    L.set_populations(f0)
    L.step(1)
    got = L.get_populations()
    _, _, typ_o = L.read_fields()
    want, forces, torques, typ = bruteforce.step(shape, f0, True, (1.0, 1.0), 0.1, (0, 0, 0), [P])
    fluid = np.zeros((8, 8, 8), dtype=bool)
    tb = np.zeros((8, 8, 8), dtype=np.uint8)
    for (x, y, z), t in typ.items():
        fluid[z, y, x] = t == 0
        tb[z, y, x] = t
    assert np.array_equal(tb, typ_o)
    assert (tb == 2).sum() > 10
    assert np.max(np.abs(got[:, :, fluid] - want[:, :, fluid])) < 1e-14
    part = L.read_particles()
    assert np.allclose(part["force"][0], forces[0], atol=1e-13)
    assert np.allclose(part["torque"][0], torques[0], atol=1e-13)


@pytest.mark.parametrize("walls", [False, True])
def test_mass_conservation(walls):
    shape = (16, 12, 10)
    rho0 = W.uniform_mixture(shape, 0.7, 0.05, seed=3)
    L = _lattice(shape, rho0, walls_z=walls, g_br=0.1, tau=(1.0, 0.7))
    m0 = L.mass()
    L.step(40)
    assert np.all(np.abs(L.mass() - m0) / m0 < 1e-12)


def test_mass_conservation_static_particles():
    shape = (20, 20, 20)
    rho0 = W.random_phases(shape, 0.5, seed=4)
    L = _lattice(shape, rho0, walls_z=True, g_br=0.1, particle_mode=1)
    L.add_particles([[6.3, 7.1, 9.4], [14.2, 12.6, 9.9]],
                    [W.axis_tilt_quaternion(0.3), W.axis_tilt_quaternion(1.2, 0.7)],
                    [4.0, 3.0], [2.0, 2.5], [0.1, -0.2])
    m0 = L.mass()
    L.step(30)
    assert np.all(np.abs(L.mass() - m0) / m0 < 1e-12)


def test_momentum_conservation_shan_chen():
    """Σ_x F^c = 0 on a periodic lattice (pairwise-antisymmetric Eq. 3) and
    the shifted-velocity collision changes the momentum by exactly Σ F, so
    the total momentum is conserved for any τ."""
    shape = (12, 10, 14)
    rho0 = W.uniform_mixture(shape, 0.7, 0.05, seed=5)
    L = _lattice(shape, rho0, walls_z=False, g_br=0.12, tau=(1.0, 0.75))
    p0 = L.momentum()["fluid"]
    L.step(30)
    p1 = L.momentum()["fluid"]
    assert np.max(np.abs(p1 - p0)) < 1e-11


def test_body_force_momentum_rate():
    """With a body force g per unit density the momentum grows by g Σρ per
    step exactly (Poiseuille driving term)."""
    shape = (6, 6, 6)
    rho0 = W.uniform_mixture(shape, 0.7, 0.05, seed=6)
    g = np.array([1e-4, -3e-5, 2e-5])
    L = _lattice(shape, rho0, g_br=0.1, body_force=tuple(g))
    p0 = L.momentum()["fluid"]
    m = L.mass().sum()
    L.step(10)
    p1 = L.momentum()["fluid"]
    assert np.allclose(p1 - p0, 10 * g * m, rtol=1e-10, atol=1e-14)


def test_poiseuille_curvature():
    """Single component between halfway bounce-back walls driven by a body
    force: the steady profile is a parabola with u'' = -g/ν, ν = (τ-1/2)/3,
    where u is the observable velocity (j + F/2)/ρ."""
    nz = 34
    shape = (4, 4, nz)
    rho0 = np.zeros((2, nz, 4, 4))
    rho0[0] = 1.0
    g = 1e-6
    for tau in (1.0, 0.8):
        L = _lattice(shape, rho0, walls_z=True, tau=(tau, tau), g_br=0.0, body_force=(g, 0, 0))
        L.step(7000 if tau == 1.0 else 9000)
        _, vel, _ = L.read_fields()
        u = vel[0, :, 1, 1]
        nu = (tau - 0.5) / 3.0
        curv = u[2:-3] - 2 * u[3:-2] + u[4:-1]
        assert np.allclose(curv, -g / nu, rtol=2e-3)
        assert np.allclose(u[1:-1], u[1:-1][::-1], rtol=1e-9)
        assert np.max(np.abs(vel[1:])) < 1e-12 * g / nu * nz ** 2 + 1e-20


def _pressure(rho, g):
    psi = 1.0 - np.exp(-rho)
    return (rho[0] + rho[1]) / 3.0 + 10.0 * g * psi[0] * psi[1]


def test_flat_interface_pressure_balance():
    """Mechanical equilibrium across a flat interface: the bulk pressures
    p = c_s^2 (ρ_r + ρ_b) + 10 g ψ_r ψ_b (leading order of Eq. 3 with the
    unweighted stencil, Σ c c = 10 I) on both sides agree."""
    nz = 48
    shape = (2, 2, nz)
    rho0 = W.flat_interface(shape, nz // 2, 0.7, 0.04, 0.0)
    rho0[:, : nz // 4] = rho0[:, ::-1][:, : nz // 4]  # periodic slab: two interfaces
    g = 0.1
    L = _lattice(shape, rho0, walls_z=False, g_br=g)
    L.step(4000)
    rho, vel, _ = L.read_fields()
    p = _pressure(rho, g)[:, 0, 0]
    red = rho[0, :, 0, 0] > rho[1, :, 0, 0]
    p_red = p[red][len(p[red]) // 2]
    p_blue = p[~red][len(p[~red]) // 2]
    assert abs(p_red - p_blue) / p_red < 2e-3
    # the interface carries only the small spurious current of the
    # Shan-Chen forcing
    assert np.max(np.abs(vel)) < 1e-4
    # demixed bulks (coexistence densities of the g = 0.1 system)
    assert rho[0, :, 0, 0].max() > 0.6 and rho[0, :, 0, 0].min() < 0.1


def test_laplace_law_cylinders():
    """Static cylindrical droplets: Δp = γ / R, so Δp is linear in 1/R with
    an intercept near zero and a common γ."""
    n = 48
    g = 0.1
    dps, inv_r = [], []
    for R in (8.0, 11.0, 14.0):
        y, x = np.mgrid[0:n, 0:n]
        inside = (x - n / 2 + 0.5) ** 2 + (y - n / 2 + 0.5) ** 2 < R * R
        rho0 = np.zeros((2, 1, n, n))
        rho0[0, 0] = np.where(inside, 0.69, 0.07)
        rho0[1, 0] = np.where(inside, 0.07, 0.69)
        L = _lattice((n, n, 1), rho0, walls_z=False, g_br=g)
        L.step(3000)
        rho, _, _ = L.read_fields()
        p = _pressure(rho, g)[0]
        dps.append(p[n // 2, n // 2] - p[0, 0])
        inv_r.append(1.0 / R)
    slope, icpt = np.polyfit(inv_r, dps, 1)
    assert slope > 0
    assert abs(icpt) < 0.05 * max(dps)
    gam = np.array(dps) / np.array(inv_r)
    assert gam.std() / gam.mean() < 0.05


@pytest.mark.parametrize("g,demix", [(0.1, True), (0.02, False), (-0.1, False)])
def test_demixing_sign_of_coupling(g, demix):
    """Reading of the sign of g (Eq. 3 with F = -ψ Σ g ψ' (x'-x)): g > 0
    repels the components and a noisy mixture coarsens; small or negative g
    stays mixed."""
    shape = (16, 16, 16)
    rho0 = W.uniform_mixture(shape, 0.7, 0.01, seed=9)
    L = _lattice(shape, rho0, g_br=g)
    s0 = np.std(rho0[0] - rho0[1])
    L.step(300)
    rho, _, _ = L.read_fields()
    s1 = np.std(rho[0] - rho[1])
    if demix:
        assert s1 > 10 * s0
    else:
        assert s1 < s0


def test_walls_leave_a_uniform_mixture_at_rest():
    """Readings c11, c13: a wall node takes the mean ρ of its fluid
    neighbours (Δρ = 0), so next to a flat wall a uniform mixture at rest
    sees the same ψ on every side and no Shan–Chen force.  It stays uniform
    and at rest to rounding over many steps.  Walls that kept ψ = 0 instead
    would pull the fluid towards themselves at once."""
    shape = (6, 5, 12)
    nx, ny, nz = shape
    rho0 = np.zeros((2, nz, ny, nx))
    rho0[0], rho0[1] = 0.6, 0.3
    L = _lattice(shape, rho0, walls_z=True, g_br=0.1, tau=(1.0, 0.8))
    L.step(60)
    rho, vel, typ = L.read_fields()
    fl = typ == 0
    assert np.max(np.abs(rho[0][fl] - 0.6)) < 1e-13 and np.max(np.abs(rho[1][fl] - 0.3)) < 1e-13
    assert np.max(np.abs(vel[:, fl])) < 1e-14
