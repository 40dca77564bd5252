"""Failure detection without a GPU fault.

- A bounded wait that runs out: the fused kernel is made to wait for a
  barrier phase that no copy completes, with a limit of 64 tries; the CTA
  gives up, waits (with the full limit) for its copies in flight, flags the
  lattice's status word, and the next synchronising call returns
  LBE_ETIMEOUT.  The device stays usable.
- Allocation failures made on the host: lbe_fail_allocations lets the n-th
  device allocation fail as if the device were full; lbe_init_lattice,
  lbe_add_particles and server admission return LBE_ENOMEM and keep nothing.
- The bounds-checked build (every computed index verified) runs a small
  moving-particle case clean, in a child process."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1109_3277_gb300 import lbe
from paper_1109_3277_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ENOMEM, ETIMEOUT = -2, -6
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_bytes():
    torch = pytest.importorskip("torch")
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info(0)[0]


@pytest.mark.parametrize("particles", [False, True])
def test_copy_wait_that_runs_out_is_reported(particles):
    shape = (64, 48, 40)  # row pitch a multiple of 16 bytes: box copies by TMA
    g = lbe.Lattice(shape, W.uniform_mixture(shape, 0.7, 0.01, seed=3), storage="f16", device=0)
    if particles:
        g.add_particles([[30.2, 22.7, 19.4]], [W.axis_tilt_quaternion(0.5, 0.2)], 6.0, 3.0, 0.05)
    g.set_wait_limit(64, unreachable=True)  # a phase no copy completes: the wait runs out
    g.step(3)
    with pytest.raises(lbe.LbeError) as e:
        g.mass()
    assert e.value.status == ETIMEOUT
    g.close()
    # the device and a new lattice work normally
    h = lbe.Lattice(shape, W.uniform_mixture(shape, 0.7, 0.01, seed=3), storage="f16", device=0)
    m0 = h.mass()
    h.step(4)
    assert np.allclose(h.mass(), m0, rtol=1e-4)  # 16-bit storage conserves mass to its rounding
    h.close()


def test_allocation_failures_keep_nothing():
    shape = (96, 64, 48)
    rho0 = W.uniform_mixture(shape, 0.7, 0.01, seed=4)
    pos, quat = [[40.1, 30.3, 20.7]], [W.axis_tilt_quaternion(0.4, 0.1)]
    warm = lbe.Lattice(shape, rho0, device=0)  # context and module loaded
    warm.close()
    free0 = _free_bytes()
    failures = 0
    for k in range(40):
        lbe.fail_allocations(k)
        try:
            g = lbe.Lattice(shape, rho0, device=0)
        except lbe.LbeError as e:
            assert e.status == ENOMEM
            failures += 1
            continue
        try:
            g.add_particles(pos, quat, 6.0, 3.0, 0.0)
            added = True
        except lbe.LbeError as e:
            assert e.status == ENOMEM
            failures += 1
            added = False
        lbe.fail_allocations(-1)
        # the lattice is whole either way: it steps, with or without the particle
        g.step(2)
        assert np.all(np.isfinite(g.mass()))
        if added:
            assert g.read_particles()["pos"].shape == (1, 3)
        g.close()
        if added and k > 20:
            break
    lbe.fail_allocations(-1)
    assert failures > 5
    # nothing leaked (allocations come in driver pages; a leak per attempt
    # would add up to far more than the slack)
    assert free0 - _free_bytes() < (8 << 20)


def test_server_request_failing_allocation_is_reported():
    w = W.adsorption_request(7, 0, edge_range=(32, 36))
    p = w.particles
    blob = lbe.particle_blob(p["pos"], p["quat"], p["r_par"], p["r_perp"], p["delta_rho"])
    srv = lbe.Server(4 << 30, 2, "f32")
    try:
        lbe.fail_allocations(0)
        rid = srv.submit(w.shape, w.rho0, blob, 200, 1e-9, **w.params)
        with pytest.raises(lbe.LbeError) as e:
            srv.wait(rid, 60.0)
        assert e.value.status == ENOMEM
        lbe.fail_allocations(-1)
        # the budget was released: a new request runs to its step limit
        rid2 = srv.submit(w.shape, w.rho0, blob, 200, 1e-9, **w.params)
        done, steps, out = srv.wait(rid2, 120.0)
        assert done and steps == 200 and np.all(np.isfinite(out))
    finally:
        lbe.fail_allocations(-1)
        srv.close()


CHECKED_RUN = r"""
import numpy as np
import paper_1109_3277_gb300.lbe as lbe
from oracle import lbref
from paper_1109_3277_gb300 import workloads as W
shape = (24, 20, 22)
rho0 = W.flat_interface(shape, 11, 0.7, 0.04, 1e-3, seed=6)
params = dict(walls_z=True, g_br=0.1, particle_mode="prescribed")
part = ([[11.2, 9.8, 11.3]], [W.axis_tilt_quaternion(0.7, 0.3)], 4.5, 2.2, 0.05)
kin = dict(vel=[[0.03, -0.01, 0.01]], omega=[[0.0, 0.005, 0.003]])
g = lbe.Lattice(shape, rho0, device=0, **params)
g.add_particles(*part, **kin)
g.step(30)  # a bounds-check failure would make this read raise
rg, _, tg = g.read_fields()
r = lbref.Lattice(shape, rho0, walls_z=True, g_br=0.1, particle_mode=2)
r.add_particles(*part, **kin)
r.step(30)
rr, _, tr = r.read_fields()
assert np.array_equal(tg, tr)
assert np.max(np.abs(rg - rr)) < 1e-5
print("checked build ok")
"""


def test_bounds_checked_build_runs_clean():
    from paper_1109_3277_gb300 import build as b
    lib = b.build(check=True)
    env = dict(os.environ, LBE_LIB=lib)
    r = subprocess.run([sys.executable, "-c", CHECKED_RUN], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "checked build ok" in r.stdout
