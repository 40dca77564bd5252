"""Batched stepping (lbe_batch_*): several lattices of different shapes,
parameters and particle modes stepped by one launch per kernel.

Every node and particle of a member is computed by the same code as when the
member steps alone: the node arithmetic is written with rounding intrinsics
and the particle kernels compile without contraction, the link sums are
exact fixed-point integers, and the pair forces are summed over the same
splits in the same order.  So a member's populations and particles are
bit-identical to stepping it alone, and never depend on the other members."""
import numpy as np
import pytest

from paper_1109_3277_gb300 import lbe
from paper_1109_3277_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _adsorption(storage="f32"):
    w = W.adsorption_box()
    g = lbe.Lattice(w.shape, w.rho0, **dict(w.params, storage=storage))
    p = w.particles
    g.add_particles(p["pos"], p["quat"], p["r_par"], p["r_perp"], p["delta_rho"])
    return g


def _spinodal(storage="f32"):
    shape = (24, 20, 16)
    return lbe.Lattice(shape, W.uniform_mixture(shape, 0.7, 0.01, seed=22), g_br=0.1, storage=storage)


def _prescribed(storage="f32"):
    shape = (24, 20, 20)
    g = lbe.Lattice(shape, W.flat_interface(shape, 10, 0.7, 0.04, 1e-3, seed=24), walls_z=True,
                    g_br=0.1, particle_mode="prescribed", storage=storage)
    g.add_particles([[8.2, 9.7, 10.3]], [W.axis_tilt_quaternion(0.7, 0.2)], 5.0, 2.5, 0.1,
                    vel=[[0.06, 0.01, -0.02]], omega=[[0.0, 0.01, 0.004]])
    return g


def _static(storage="f32"):
    shape = (13, 11, 10)
    g = lbe.Lattice(shape, W.random_phases(shape, 0.5, seed=23), walls_z=True, tau=(0.8, 1.3),
                    g_br=0.1, particle_mode="static", storage=storage)
    g.add_particles([[5.6, 5.2, 4.9]], [W.axis_tilt_quaternion(0.6, 0.3)], 3.6, 2.1, -0.15,
                    vel=[[0.01, -0.02, 0.005]], omega=[[0.003, 0.002, -0.004]])
    return g


def _pair(storage="f32"):
    """Two free ellipsoids at a lubrication gap in a noisy mixture."""
    shape = (32, 24, 24)
    g = lbe.Lattice(shape, W.uniform_mixture(shape, 0.7, 0.01, seed=1), g_br=0.1, storage=storage)
    q = W.axis_tilt_quaternion(np.pi / 2, 0.0)
    g.add_particles([[16.0, 9.775, 12.0], [16.0, 14.225, 12.0]], [q, q], 5.0, 2.0, 0.0,
                    vel=[[0.0, 0.001, 0.0], [0.0, -0.001, 0.0]])
    return g


def _many(storage="f32"):
    """150 free ellipsoids packed with a 0.8 margin (Hertz contacts and
    lubrication gaps), more than one tile of 128 particles, so that the
    pair sums run over two splits.  The fluid (total density about 0.74)
    is lighter than the particles (density 1): the oracle keeps this run
    stable for 30 steps (|V| < 0.04)."""
    shape = (40, 40, 36)
    pos, quat = W.place_ellipsoids(shape, 150, 3.0, 1.5, seed=31, margin=0.8)
    assert len(pos) == 150
    g = lbe.Lattice(shape, W.random_phases(shape, 0.5, seed=32), g_br=0.1, storage=storage)
    g.add_particles(pos, quat, 3.0, 1.5, np.where(np.arange(150) % 2, 0.05, -0.05),
                    vel=W.uniform(33, (150, 3), lo=-2e-3, hi=2e-3))
    return g


MAKERS = [_adsorption, _spinodal, _prescribed, _static, _pair, _many]


def _state(g):
    out = {"f": g.get_populations()}
    if g.np:
        out.update(g.read_particles())
    out["types"] = g.read_fields(rho=False, vel=False)[2]
    return out


def _equal(a, b):
    return all(np.array_equal(a[k], b[k]) for k in a)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_matches_members_stepped_alone(storage):
    alone = [m(storage) for m in MAKERS]
    mixed = [m(storage) for m in MAKERS]
    batch = lbe.Batch(mixed)
    assert batch.kernels_per_step() == 11
    for g in alone:
        g.step(30)
    batch.step(30)
    for k, (a, b) in enumerate(zip(alone, mixed)):
        assert _equal(_state(a), _state(b)), MAKERS[k].__name__
    batch.close()


def test_member_alone_or_in_a_mix_is_identical():
    """The result of a member does not depend on what else is batched with
    it: bit-identical outputs, pair forces included."""
    solo = _pair()
    b1 = lbe.Batch([solo])
    mix = [m() for m in MAKERS]
    b2 = lbe.Batch(mix)
    b1.step(25)
    b2.step(25)
    assert _equal(_state(solo), _state(mix[MAKERS.index(_pair)]))
    assert b1.kernels_per_step() == 11


def test_odd_steps_and_interleaving_with_member_steps():
    """Parities of the populations and of the owner maps stay consistent
    when batched steps (odd counts) and a member's own steps alternate."""
    a = _prescribed()
    b = _prescribed()
    other = _spinodal()
    batch = lbe.Batch([other, b])
    a.step(7)
    batch.step(3)
    b.step(2)
    batch.step(1)
    b.step(1)
    assert _equal(_state(a), _state(b))


def test_batch_without_particles():
    a = [_spinodal(), _spinodal()]
    b = [_spinodal(), _spinodal()]
    batch = lbe.Batch(b)
    assert batch.kernels_per_step() == 4
    for g in a:
        g.step(11)
    batch.step(11)
    for x, y in zip(a, b):
        assert _equal(_state(x), _state(y))


def test_autotuners_keep_results_bit_identical():
    """The z-chunk of the fused kernel and the persistent CTA count change
    only the order in which tiles run, never a result."""
    a, b = _adsorption(), _adsorption()
    a.step(3)
    b.step(3)
    zc = a.autotune()
    assert zc >= 1
    a.step(20)
    b.step(20)
    assert _equal(_state(a), _state(b))
    for z in (1, 5, 10 ** 6, 0):
        a.set_zchunk(z)
        a.step(4)
        b.step(4)
        assert _equal(_state(a), _state(b)), z
    with pytest.raises(lbe.LbeError):
        a.set_zchunk(-1)
    m1 = [m() for m in MAKERS]
    m2 = [m() for m in MAKERS]
    b1, b2 = lbe.Batch(m1), lbe.Batch(m2)
    b1.step(2)
    b2.step(2)
    c = b1.autotune()
    assert c >= 1
    b1.step(20)
    b2.step(20)
    for x, y in zip(m1, m2):
        assert _equal(_state(x), _state(y))


def test_invalid_batches_are_rejected():
    a = _spinodal("f32")
    with pytest.raises(lbe.LbeError):
        lbe.Batch([])
    with pytest.raises(lbe.LbeError):
        lbe.Batch([a, _spinodal("f16")])
    with pytest.raises(lbe.LbeError):
        lbe.Batch([a, a])
    shape = (8, 8, 8)
    t = lbe.Lattice(shape, np.full((2, 8, 8, 8), 0.5), flags=lbe.FLAG_TWO_PASS)
    with pytest.raises(lbe.LbeError):
        lbe.Batch([a, t])
