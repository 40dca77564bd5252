"""Pins of the oracle's particle side: the Berne–Pechukas Hertz interaction
(Eq. 6-8), the rigid-body update, the node coverage, the moving
bounce-back / momentum-exchange signs (Eq. 4-5) and the fill/empty
bookkeeping."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import lbref
from paper_1109_3277_gb300 import workloads as W


def _axis(q):
    w, x, y, z = q
    return np.array([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)])


# ------------------------------------------------------- Eq. 6-8 closed forms

def test_sigma_limits_side_and_end():
    """σ is 2 r_perp side by side and 2 r_par end to end (Eq. 8 with
    χ = (R_p^2 - R_o^2)/(R_p^2 + R_o^2))."""
    rp, ro = 8.0, 4.0
    ex, ey = np.array([1.0, 0, 0]), np.array([0, 1.0, 0])
    side = lbref.pair_hertz(100.0, rp, ro, [0, 0, 20.0], ex, ex)
    assert abs(side["sigma"] - 2 * ro) < 1e-12
    end = lbref.pair_hertz(100.0, rp, ro, [20.0, 0, 0], ex, ex)
    assert abs(end["sigma"] - 2 * rp) < 1e-12
    # parallel axes side by side along y also 2 r_perp
    s2 = lbref.pair_hertz(100.0, rp, ro, [0, 20.0, 0], ex, ex)
    assert abs(s2["sigma"] - 2 * ro) < 1e-12
    # crossed axes, both across the separation: side contact again
    c = lbref.pair_hertz(100.0, rp, ro, [0, 0, 20.0], ex, ey)
    assert abs(c["sigma"] - 2 * ro) < 1e-12
    # T shape (separation along one axis): σ = σ̄ / sqrt(1 - χ), between the two
    t = lbref.pair_hertz(100.0, rp, ro, [20.0, 0, 0], ex, ey)
    chi = (rp * rp - ro * ro) / (rp * rp + ro * ro)
    assert abs(t["sigma"] - 2 * ro / np.sqrt(1 - chi)) < 1e-12
    assert 2 * ro < t["sigma"] < 2 * rp


@pytest.mark.parametrize("r", [7.0, 9.5, 9.999])
def test_sphere_limit_is_hertz(r):
    """R_p = R_o gives χ = 0, ε = ε̄, σ = 2R and φ = K_H (2R - r)^{5/2}."""
    R, K = 5.0, 100.0
    o1 = np.array([0.3, 0.4, np.sqrt(1 - 0.25)])
    o2 = np.array([1.0, 0.0, 0.0])
    d = np.array([0.6, -0.8, 0.0]) * r
    h = lbref.pair_hertz(K, R, R, d, o1, o2)
    assert abs(h["sigma"] - 2 * R) < 1e-12
    assert abs(h["energy"] - K * (2 * R - r) ** 2.5) < 1e-9 * max(1.0, h["energy"])
    fmag = 2.5 * K * (2 * R - r) ** 1.5
    assert np.allclose(h["f_j"], fmag * d / r, rtol=1e-10, atol=1e-12)
    assert np.allclose(h["t_i"], 0, atol=1e-12) and np.allclose(h["t_j"], 0, atol=1e-12)
    far = lbref.pair_hertz(K, R, R, d / r * 10.5, o1, o2)
    assert far["energy"] == 0 and np.all(far["f_j"] == 0)


def _rot(v, axis, ang):
    axis = axis / np.linalg.norm(axis)
    return (v * np.cos(ang) + np.cross(axis, v) * np.sin(ang)
            + axis * (axis @ v) * (1 - np.cos(ang)))


def test_forces_torques_are_minus_gradients():
    """Finite differences of the energy pin the analytic force on j and the
    torques (rigid rotations of each axis)."""
    rp, ro, K = 8.0, 4.0, 100.0
    rng = np.random.default_rng(1)
    for _ in range(6):
        oi = rng.normal(size=3)
        oi /= np.linalg.norm(oi)
        oj = rng.normal(size=3)
        oj /= np.linalg.norm(oj)
        d = rng.normal(size=3)
        d = d / np.linalg.norm(d)
        sig = lbref.pair_hertz(K, rp, ro, d * 30, oi, oj)["sigma"]
        r = d * sig * 0.93
        h = lbref.pair_hertz(K, rp, ro, r, oi, oj)
        assert h["energy"] > 0
        eps = 1e-6
        grad = np.zeros(3)
        for k in range(3):
            e = np.zeros(3)
            e[k] = eps
            grad[k] = (lbref.pair_hertz(K, rp, ro, r + e, oi, oj)["energy"]
                       - lbref.pair_hertz(K, rp, ro, r - e, oi, oj)["energy"]) / (2 * eps)
        assert np.allclose(h["f_j"], -grad, rtol=1e-5, atol=1e-6)
        for k in range(3):
            ax = np.zeros(3)
            ax[k] = 1.0
            ti = -(lbref.pair_hertz(K, rp, ro, r, _rot(oi, ax, eps), oj)["energy"]
                   - lbref.pair_hertz(K, rp, ro, r, _rot(oi, ax, -eps), oj)["energy"]) / (2 * eps)
            tj = -(lbref.pair_hertz(K, rp, ro, r, oi, _rot(oj, ax, eps))["energy"]
                   - lbref.pair_hertz(K, rp, ro, r, oi, _rot(oj, ax, -eps))["energy"]) / (2 * eps)
            assert abs(h["t_i"][k] - ti) < 1e-5 * max(1.0, abs(ti))
            assert abs(h["t_j"][k] - tj) < 1e-5 * max(1.0, abs(tj))
        # rotational invariance of φ: no net torque on the pair
        tot = h["t_i"] + h["t_j"] + np.cross(r, h["f_j"])
        assert np.allclose(tot, 0, atol=1e-8 * max(1.0, np.abs(h["f_j"]).max() * sig))


# ------------------------------------------------------ rigid-body update

def test_translation_closed_form():
    M = 3.0
    F = np.array([0.01, -0.02, 0.003])
    pos, q, v, w = np.array([5.0, 6, 7]), np.array([1.0, 0, 0, 0]), np.array([0.1, 0, 0]), np.zeros(3)
    for _ in range(10):
        pos, q, v, w = lbref.rigid_update(M, 1.0, 1.0, F, np.zeros(3), pos, q, v, w)
    assert np.allclose(v, [0.1, 0, 0] + 10 * F / M, rtol=1e-14)
    assert np.allclose(pos, [5.0, 6, 7] + 10 * np.array([0.1, 0, 0]) + F / M * 55, rtol=1e-13)
    assert np.allclose(q, [1, 0, 0, 0])


def test_symmetric_top_free_precession():
    """Torque-free symmetric top: in the body frame the transverse ω
    rotates about the symmetry axis at Ω = (I_par - I_perp)/I_perp ω_par;
    the lab angular momentum is conserved (to the scheme's order)."""
    rp, ro = 6.0, 3.0
    M = 4 / 3 * np.pi * rp * ro * ro
    ipar, iperp = 0.4 * M * ro * ro, 0.2 * M * (rp * rp + ro * ro)
    wpar, wt = 0.01, 0.004
    q = np.array([1.0, 0, 0, 0])
    w = np.array([wpar, wt, 0.0])
    pos, v = np.zeros(3), np.zeros(3)
    L0 = np.array([ipar * wpar, iperp * wt, 0.0])
    n = 400
    for _ in range(n):
        pos, q, v, w = lbref.rigid_update(M, ipar, iperp, np.zeros(3), np.zeros(3), pos, q, v, w)
    w2, x2, y2, z2 = q
    R = np.array([[1 - 2 * (y2 * y2 + z2 * z2), 2 * (x2 * y2 - w2 * z2), 2 * (x2 * z2 + w2 * y2)],
                  [2 * (x2 * y2 + w2 * z2), 1 - 2 * (x2 * x2 + z2 * z2), 2 * (y2 * z2 - w2 * x2)],
                  [2 * (x2 * z2 - w2 * y2), 2 * (y2 * z2 + w2 * x2), 1 - 2 * (x2 * x2 + y2 * y2)]])
    wb = R.T @ w
    Om = (ipar - iperp) / iperp * wpar
    ang = np.arctan2(wb[2], wb[1])
    want = np.angle(np.exp(1j * n * Om))
    assert abs(np.angle(np.exp(1j * (ang - want)))) < 0.02 * abs(n * Om)
    assert abs(wb[0] - wpar) < 1e-12
    Lb = np.array([ipar, iperp, iperp]) * wb
    Llab = R @ Lb
    assert np.linalg.norm(Llab - L0) / np.linalg.norm(L0) < 0.02
    assert abs(np.linalg.norm(q) - 1) < 1e-14


# ------------------------------------------------------------- coverage

def _exact_inside(node, pos, a, b, perm):
    """Exact rational inside test for an axis-aligned ellipsoid whose
    symmetry axis is lattice axis perm[0]."""
    d = [Fraction(node[k]) - Fraction(pos[k]) for k in range(3)]
    v = (d[perm[0]] / Fraction(a)) ** 2 + (d[perm[1]] / Fraction(b)) ** 2 + (d[perm[2]] / Fraction(b)) ** 2
    return v <= 1, abs(v - 1)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_coverage_matches_exact_rational_count(axis):
    shape = (24, 22, 20)
    pos = [11.3, 10.6, 9.85]
    a, b = 6.5, 3.25
    quats = {0: [1.0, 0, 0, 0],
             1: [np.sqrt(0.5), 0, 0, np.sqrt(0.5)],      # x -> y
             2: [np.sqrt(0.5), 0, -np.sqrt(0.5), 0]}     # x -> z
    perms = {0: (0, 1, 2), 1: (1, 0, 2), 2: (2, 1, 0)}
    L = lbref.Lattice(shape, np.full((2, 20, 22, 24), 0.5), particle_mode=1)
    L.add_particles([pos], [quats[axis]], a, b, 0.0)
    _, _, typ = L.read_fields()
    want = np.zeros_like(typ)
    margin = 1.0
    for z in range(20):
        for y in range(22):
            for x in range(24):
                ins, dist = _exact_inside((x, y, z), pos, a, b, perms[axis])
                margin = min(margin, float(dist))
                want[z, y, x] = 2 if ins else 0
    assert margin > 1e-12  # no node sits on the surface
    assert np.array_equal(typ, want)
    vol = 4 / 3 * np.pi * a * b * b
    assert abs((want == 2).sum() - vol) < 0.15 * vol


def test_coverage_periodic_wrap_and_lowest_owner():
    shape = (16, 16, 16)
    L = lbref.Lattice(shape, np.full((2, 16, 16, 16), 0.5), particle_mode=1)
    # one particle straddles the periodic corner; two overlap
    L.add_particles([[0.4, 15.7, 0.2], [8.0, 8.0, 8.0], [10.0, 8.0, 8.0]],
                    [[1.0, 0, 0, 0]] * 3, [3.0, 3.0, 3.0], [2.0, 2.0, 2.0], [0.0, 0.0, 0.0])
    _, _, typ = L.read_fields()
    assert typ[0, 15, 0] == 2 and typ[0, 15, 15] == 2 and typ[15, 0, 0] == 2
    assert typ[8, 8, 9] == 2  # shared by particles 1 and 2


# ------------------------------------------- moving bounce-back, Eq. 4-5

def _sphere_setup(vel=(0, 0, 0), omega=(0, 0, 0), u_fluid=None, mode=1, g=0.0, n=20):
    shape = (n, n, n)
    rho0 = np.zeros((2, n, n, n))
    rho0[0] = 1.0
    L = lbref.Lattice(shape, rho0, g_br=g, particle_mode=mode)
    L.add_particles([[n / 2 + 0.1, n / 2 - 0.2, n / 2 + 0.15]], [[1.0, 0, 0, 0]], 4.0, 4.0, 0.0,
                    vel=[vel], omega=[omega])
    if u_fluid is not None:
        f = L.get_populations()
        _, _, typ = L.read_fields()
        feq = lbref.feq(1.0, np.array(u_fluid))
        f[0] = np.where(typ[None] == 0, feq[:, None, None, None], 0.0)
        f[1] = 0.0
        L.set_populations(f)
    return L


def test_static_wall_drag_direction():
    """A particle moving through fluid at rest feels a force opposite to
    its velocity; co-moving fluid removes the linear part of that force
    (the C term of Eq. 4 reproduces the moving-wall equilibrium)."""
    U = np.array([0.02, -0.01, 0.005])
    L = _sphere_setup(vel=U)
    L.step(1)
    F_rest = L.read_particles()["force"][0]
    assert F_rest @ U < 0
    assert np.allclose(np.cross(F_rest, U) / (np.linalg.norm(F_rest) * np.linalg.norm(U)), 0,
                       atol=0.2)
    L2 = _sphere_setup(vel=U, u_fluid=U)
    L2.step(1)
    F_co = L2.read_particles()["force"][0]
    assert np.linalg.norm(F_co) < 0.05 * np.linalg.norm(F_rest)


def test_rotating_sphere_torque_opposes_spin():
    om = np.array([0.0, 0.0, 0.01])
    L = _sphere_setup(omega=om)
    L.step(1)
    T = L.read_particles()["torque"][0]
    assert T @ om < 0
    assert abs(T[2]) > 20 * max(abs(T[0]), abs(T[1]))


def test_momentum_conservation_free_particle():
    """Without Shan-Chen coupling or walls, fluid + particle + pending
    fill/empty momentum is conserved exactly (signs of Eq. 4-5 and of the
    fill/empty transfers)."""
    L = _sphere_setup(vel=(0.05, 0.02, -0.03), omega=(0.002, -0.001, 0.003), mode=0)
    def total():
        m = L.momentum()
        return m["fluid"] + m["particles"] + m["pending"]
    p0 = total()
    moved = False
    for _ in range(40):
        L.step(1)
        d = L.diagnostics()
        moved = moved or d["created"].sum() > 0 or d["deleted"].sum() > 0
        assert np.max(np.abs(total() - p0)) < 1e-11
    assert moved


def test_fill_empty_mass_bookkeeping():
    """Per step: Σρ(t+1) - Σρ(t) = created - deleted + Σ_links C, per
    component (reading of the fill/empty rule)."""
    shape = (24, 20, 20)
    rho0 = W.flat_interface(shape, 10, 0.7, 0.04, 1e-3, seed=11)
    L = lbref.Lattice(shape, rho0, walls_z=True, g_br=0.1, particle_mode=2)
    L.add_particles([[8.2, 9.7, 10.3]], [W.axis_tilt_quaternion(0.7, 0.2)], 5.0, 2.5, 0.1,
                    vel=[[0.06, 0.01, -0.02]], omega=[[0.0, 0.01, 0.004]])
    m = L.mass()
    events = 0
    for _ in range(40):
        L.step(1)
        d = L.diagnostics()
        m1 = L.mass()
        events += int(d["created"].sum() > 0) + int(d["deleted"].sum() > 0)
        assert np.allclose(m1 - m, d["created"] - d["deleted"] + d["sum_c"], rtol=0,
                           atol=1e-12 * m.sum())
        m = m1
    assert events > 10


def test_co_moving_fluid_is_left_at_equilibrium_exactly():
    """Eq. 4 with C = 6 w_i ρ (u_surf·c_i) (readings c5, c6): a sphere centred
    on a node (its links come in inversion pairs) that moves with the
    uniform fluid.  The bounced population plus C is then exactly the
    equilibrium of the moving fluid, so after one step every fluid node is
    still at f^eq(ρ, U), to rounding, and the net force and torque vanish: in
    (2 f*_ī + C) c_ī the terms odd in c cancel, and the even ones sum to zero
    over each inversion pair.  A wrong sign or factor in C leaves the odd
    terms, which do not cancel."""
    n = 16
    U = np.array([0.02, -0.01, 0.005])
    rho0 = np.zeros((2, n, n, n))
    rho0[0] = 1.0
    L = lbref.Lattice((n, n, n), rho0, g_br=0.0, particle_mode=1)
    # radius 4.3: no node lies within 0.05 of the surface
    L.add_particles([[8.0, 8.0, 8.0]], [[1.0, 0, 0, 0]], 4.3, 4.3, 0.0, vel=[U])
    f = L.get_populations()
    _, _, typ = L.read_fields()
    feq = lbref.feq(1.0, U)
    fluid = typ == 0
    f[0] = np.where(fluid[None], feq[:, None, None, None], 0.0)
    f[1] = 0.0
    L.set_populations(f)
    L.step(1)
    f1 = L.get_populations()
    assert np.max(np.abs(f1[0][:, fluid] - feq[:, None])) < 1e-14
    p = L.read_particles()
    assert np.max(np.abs(p["force"][0])) < 1e-12
    assert np.max(np.abs(p["torque"][0])) < 1e-12
    # the same sphere at rest in that flow feels a drag along U
    L2 = lbref.Lattice((n, n, n), rho0, g_br=0.0, particle_mode=1)
    L2.add_particles([[8.0, 8.0, 8.0]], [[1.0, 0, 0, 0]], 4.3, 4.3, 0.0)
    L2.set_populations(f)
    L2.step(1)
    F = L2.read_particles()["force"][0]
    assert F @ U > 0 and np.linalg.norm(F) > 1e-3


@pytest.mark.parametrize("gap", [0.1, 0.4, 0.6])
def test_lubrication_sphere_limit(gap):
    """Eq. 9 for two spheres of radius R approaching at relative speed v
    with a gap h = r - 2R below the cut-off Δc = 2/3: the correction is
    (3π μ R^2 / 2) v (1/h - 1/Δc) along the line of centres, pushing them
    apart, with μ = ρ̄ ν and ν = (τ - 1/2)/3 (reading c10).  It is isolated
    as the difference between runs with and without the cut-off; the Hertz
    term is zero at a positive gap."""
    R, tau, rho_bar, cut = 4.0, 0.8, 1.4, 2.0 / 3.0
    n = (32, 16, 16)
    rho0 = np.zeros((2, 16, 16, 32))
    rho0[0] = 1.0
    v = 0.01
    xa = 10.0
    xb = xa + 2 * R + gap
    F = []
    for c in (cut, 0.0):
        L = lbref.Lattice(n, rho0, g_br=0.0, tau=(tau, tau), particle_mode=1, lub_cut=c, lub_rho=rho_bar)
        L.add_particles([[xa, 8.0, 8.0], [xb, 8.0, 8.0]], [[1.0, 0, 0, 0]] * 2, R, R, 0.0,
                        vel=[[v, 0, 0], [-v, 0, 0]])
        L.step(1)
        F.append(L.read_particles()["force"])
    dF = F[0] - F[1]
    mu = rho_bar * (tau - 0.5) / 3.0
    want = 1.5 * np.pi * mu * R * R * (2 * v) * (1.0 / gap - 1.0 / cut)
    assert dF[0, 0] == pytest.approx(-want, rel=1e-10)
    assert dF[1, 0] == pytest.approx(want, rel=1e-10)
    assert np.allclose(dF[:, 1:], 0.0, atol=1e-14)


@pytest.mark.parametrize("rho_p", [1.0, 3.0])
def test_lubrication_capped_at_reduced_mass(rho_p):
    """At a gap where the coefficient K (1/h - 1/Δc) of Eq. 9 exceeds the
    pair's reduced mass (two spheres of radius 4 at h = 0.01: about 1,040
    against M/2 = 134 ρ_p), the correction is the reduced mass times the
    normal approach speed, so one update (Δt = 1) removes the approach
    (reading: the cap keeps the explicit update from reversing the approach
    with a growing speed).  The mass is the particle density ρ_p times the
    sphere's volume.  Two spheres started a little further apart, at h =
    0.03, close in without flying apart."""
    R, tau, rho_bar, cut = 4.0, 0.8, 1.4, 2.0 / 3.0
    n = (32, 16, 16)
    rho0 = np.zeros((2, 16, 16, 32))
    rho0[0] = 1.0
    v, xa, gap = 0.01, 10.0, 0.01
    M = rho_p * 4.0 / 3.0 * np.pi * R ** 3
    F = []
    for c in (cut, 0.0):
        L = lbref.Lattice(n, rho0, g_br=0.0, tau=(tau, tau), particle_mode=1, lub_cut=c, lub_rho=rho_bar,
                          rho_particle=rho_p)
        L.add_particles([[xa, 8.0, 8.0], [xa + 2 * R + gap, 8.0, 8.0]], [[1.0, 0, 0, 0]] * 2, R, R, 0.0,
                        vel=[[v, 0, 0], [-v, 0, 0]])
        L.step(1)
        F.append(L.read_particles()["force"])
    dF = F[0] - F[1]
    assert dF[0, 0] == pytest.approx(-0.5 * M * 2 * v, rel=1e-10)
    assert dF[1, 0] == pytest.approx(0.5 * M * 2 * v, rel=1e-10)
    L = lbref.Lattice(n, rho0, g_br=0.0, tau=(tau, tau), particle_mode=1, lub_cut=cut, lub_rho=rho_bar,
                      rho_particle=rho_p)
    L.add_particles([[xa, 8.0, 8.0], [xa + 2 * R + 0.03, 8.0, 8.0]], [[1.0, 0, 0, 0]] * 2, R, R, 0.0,
                    vel=[[v, 0, 0], [-v, 0, 0]])
    for _ in range(8):
        L.step(1)
        p = L.read_particles()
        assert np.all(np.abs(p["vel"]) <= 2 * v)
    assert p["pos"][1, 0] - p["pos"][0, 0] > 2 * R - 0.1


@pytest.mark.parametrize("drho", [0.15, -0.15])
def test_colour_rule_sign(drho):
    """The colour rule of §2: Δρ > 0 adds red density to the particle's
    shell, Δρ < 0 adds |Δρ| to blue.  The extra density repels the other
    component (g > 0), so after some steps in a uniform mixture the fluid
    next to the particle is richer in the colour's component than the bulk:
    red for Δρ > 0, blue for Δρ < 0."""
    n = 16
    rho0 = np.full((2, n, n, n), 0.35)
    L = lbref.Lattice((n, n, n), rho0, g_br=0.1, particle_mode=1)
    L.add_particles([[8.0, 8.0, 8.0]], [[1.0, 0, 0, 0]], 3.3, 3.3, drho)
    L.step(40)
    rho, _, typ = L.read_fields()
    fluid = typ == 0
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.sqrt((x - 8.0) ** 2 + (y - 8.0) ** 2 + (z - 8.0) ** 2)
    near = fluid & (r < 5.0)
    far = fluid & (r > 7.0)
    phi_near = (rho[0] - rho[1])[near].mean()
    phi_far = (rho[0] - rho[1])[far].mean()
    assert np.sign(phi_near - phi_far) == np.sign(drho)
    assert abs(phi_near - phi_far) > 1e-3


def test_hertz_pair_force_applied_to_both_particles():
    """The pair step applies the Berne–Pechukas Hertz interaction (Eq. 6-8)
    of lbref_pair_hertz with r = X_B − X_A: +f_j on B, −f_j on A, and each
    particle's own torque.  Isolated as the difference between runs with and
    without the Hertz constant (no lubrication), two overlapping ellipsoids
    held in place."""
    n = (32, 24, 24)
    rho0 = np.zeros((2, 24, 24, 32))
    rho0[0] = 1.0
    qa, qb = W.axis_tilt_quaternion(0.7, 0.2), W.axis_tilt_quaternion(1.2, -0.4)
    xa, xb = np.array([13.0, 12.0, 12.0]), np.array([19.5, 12.8, 11.6])
    out = []
    for k in (100.0, 0.0):
        L = lbref.Lattice(n, rho0, g_br=0.0, particle_mode=1, k_hertz=k, lub_cut=0.0)
        L.add_particles([xa, xb], [qa, qb], 6.0, 3.0, 0.0)
        L.step(1)
        p = L.read_particles()
        out.append((p["force"], p["torque"]))
    dF, dT = out[0][0] - out[1][0], out[0][1] - out[1][1]
    h = lbref.pair_hertz(100.0, 6.0, 3.0, xb - xa, _axis(qa), _axis(qb))
    assert h["energy"] > 0  # they overlap
    assert np.allclose(dF[1], h["f_j"], rtol=1e-12, atol=1e-14)
    assert np.allclose(dF[0], -h["f_j"], rtol=1e-12, atol=1e-14)
    assert np.allclose(dT[0], h["t_i"], rtol=1e-12, atol=1e-14)
    assert np.allclose(dT[1], h["t_j"], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("case", ["translating sphere", "spinning ellipsoid"])
def test_uncovered_node_gets_the_local_equilibrium(case):
    """Reading c12 for a node the particle leaves: its populations become
    f^eq(ρ̄^c, u_surf(x)), where ρ̄^c is the mean density of its neighbours that
    are fluid before and after the update, and u_surf = V + ω × (x − X) is
    the particle's surface velocity at the node.  Checked on every node a
    particle uncovers in one step, against the fields read back.  In the
    spinning case some uncovered nodes border nodes the particle covers in
    the same step, which the density mean must leave out."""
    n = 20
    rho0 = W.uniform_mixture((n, n, n), 0.5, 0.05, seed=9)
    L = lbref.Lattice((n, n, n), rho0, g_br=0.0, particle_mode=2)
    if case == "translating sphere":
        V, om = np.array([0.35, 0.0, 0.0]), np.array([0.0, 0.0, 0.01])
        L.add_particles([[9.9, 10.1, 9.95]], [[1.0, 0, 0, 0]], 3.6, 3.6, 0.0, vel=[V], omega=[om])
    else:
        V, om = np.array([0.05, 0.0, 0.0]), np.array([0.0, 0.0, 0.15])
        L.add_particles([[9.9, 10.1, 9.95]], [W.axis_tilt_quaternion(np.pi / 2, 0.3)], 7.0, 2.5, 0.0,
                        vel=[V], omega=[om])
    _, _, t0 = L.read_fields()
    L.step(1)
    _, _, t1 = L.read_fields()
    f = L.get_populations()
    X = L.read_particles()["pos"][0]
    c, w, _ = lbref.lattice_tables()
    gone = np.argwhere((t0 == 2) & (t1 == 0))
    newly = (t0 == 0) & (t1 == 2)
    assert len(gone) > 3
    bordering = 0
    for z, y, x in gone:
        sums, cnt = np.zeros(2), 0
        for i in range(1, 19):
            xm, ym, zm = (x + c[i][0]) % n, (y + c[i][1]) % n, (z + c[i][2]) % n
            bordering += int(newly[zm, ym, xm])
            if t0[zm, ym, xm] == 0 and t1[zm, ym, xm] == 0:
                sums += f[:, :, zm, ym, xm].sum(axis=1)
                cnt += 1
        rbar = sums / cnt
        r = np.array([x, y, z], dtype=np.float64) - X
        r -= n * np.round(r / n)
        us = V + np.cross(om, r)
        for comp in range(2):
            assert np.allclose(f[comp, :, z, y, x], lbref.feq(rbar[comp], us), rtol=0, atol=1e-14)
    if case == "spinning ellipsoid":
        assert bordering > 0


def test_prescribed_motion_closed_form():
    """Prescribed mode (the driven particles of the parity and serving
    tests): the centre moves by V every step and the orientation turns about
    the fixed lab-frame ω by |ω| per step, whatever the fluid does."""
    n = 24
    rho0 = W.uniform_mixture((n, n, n), 0.5, 0.05, seed=4)
    V = np.array([0.03, -0.02, 0.01])
    om = np.array([0.01, 0.02, -0.015])
    q0 = W.axis_tilt_quaternion(0.4, 1.1)
    L = lbref.Lattice((n, n, n), rho0, g_br=0.1, particle_mode=2)
    L.add_particles([[11.0, 12.0, 12.5]], [q0], 5.0, 2.5, 0.05, vel=[V], omega=[om])
    steps = 25
    L.step(steps)
    p = L.read_particles()
    assert np.allclose(p["pos"][0], np.array([11.0, 12.0, 12.5]) + steps * V, atol=1e-12)
    ang = np.linalg.norm(om) * steps
    ax = om / np.linalg.norm(om)

    def rot(v):  # Rodrigues: rotation by ang about ax
        return v * np.cos(ang) + np.cross(ax, v) * np.sin(ang) + ax * (ax @ v) * (1 - np.cos(ang))

    assert np.allclose(_axis(p["quat"][0]), rot(_axis(q0)), atol=1e-10)
    assert np.allclose(p["vel"][0], V) and np.allclose(p["omega"][0], om)
