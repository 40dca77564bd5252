"""Serving of adsorption requests with continuous batching (lbe_server_*):
admission by slots and HBM footprint, retirement on tilt convergence or the
step limit, and results identical alone and in the mix."""
import numpy as np
import pytest

from paper_1109_3277_gb300 import lbe
from paper_1109_3277_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GB = 1 << 30


def _requests(n, seed=7, edge_range=(32, 44)):
    return [W.adsorption_request(seed, i, edge_range=edge_range) for i in range(n)]


def _submit(srv, w, max_steps, tol):
    p = w.particles
    blob = lbe.particle_blob(p["pos"], p["quat"], p["r_par"], p["r_perp"], p["delta_rho"])
    return srv.submit(w.shape, w.rho0, blob, max_steps, tol, **w.params)


def _alone(w, steps, storage):
    g = lbe.Lattice(w.shape, w.rho0, storage=storage, **w.params)
    p = w.particles
    g.add_particles(p["pos"], p["quat"], p["r_par"], p["r_perp"], p["delta_rho"])
    g.step(steps)
    r = g.read_particles()
    g.close()
    return np.concatenate([r["pos"], r["quat"], r["vel"], r["omega"], r["force"], r["torque"]], axis=1)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_results_alone_and_in_the_mix_are_identical(storage):
    """Six uneven boxes with different step limits through a 3-slot server
    (boxes join while others run), against the same requests one at a time
    and against plain lattices: bit-identical particle results."""
    reqs = _requests(6)
    limits = [200, 500, 300, 400, 200, 300]
    mixed = lbe.Server(8 * GB, 3, storage)
    ids = [_submit(mixed, w, m, 0.0) for w, m in zip(reqs, limits)]
    out_mixed = [mixed.wait(i, 120.0) for i in ids]
    st = mixed.stats()
    mixed.close()
    assert st["completed"] == 6 and st["max_running"] == 3
    single = lbe.Server(8 * GB, 1, storage)
    out_single = [single.wait(_submit(single, w, m, 0.0), 120.0) for w, m in zip(reqs, limits)]
    assert single.stats()["max_running"] == 1
    single.close()
    for w, m, a, b in zip(reqs, limits, out_mixed, out_single):
        assert a[0] and b[0] and a[1] == m and b[1] == m
        assert np.array_equal(a[2], b[2])
        assert np.array_equal(a[2], _alone(w, m, storage))
        assert np.all(np.isfinite(a[2]))


def test_tilt_convergence_and_step_limit():
    """A tolerance above any tilt change stops a request at the first check
    (100 steps); tolerance 0 runs it to its limit, rounded up to 100."""
    w = _requests(1, seed=9)[0]
    srv = lbe.Server(4 * GB, 2, "f32")
    a = _submit(srv, w, 1000, 10.0)
    b = _submit(srv, w, 250, 0.0)
    ra, rb = srv.wait(a, 60.0), srv.wait(b, 60.0)
    assert ra[0] and ra[1] == 100
    assert rb[0] and rb[1] == 300
    qa, ta = srv.timing(a)
    assert 0.0 <= qa <= ta
    srv.close()


def test_admission_by_hbm_footprint():
    """With a budget that holds one box, boxes run one at a time although
    more slots are free; with room for all, they run together."""
    reqs = _requests(4, seed=11, edge_range=(40, 40))
    fp = max(lbe.footprint(w.shape, 1, storage="f32", **w.params) for w in reqs)
    assert fp > 0
    tight = lbe.Server(int(1.5 * fp), 8, "f32")
    ids = [_submit(tight, w, 200, 0.0) for w in reqs]
    for i in ids:
        assert tight.wait(i, 60.0)[0]
    assert tight.stats()["max_running"] == 1
    tight.close()
    roomy = lbe.Server(int(4.5 * fp), 8, "f32")
    ids = [_submit(roomy, w, 200, 0.0) for w in reqs]
    for i in ids:
        assert roomy.wait(i, 60.0)[0]
    assert roomy.stats()["max_running"] == 4
    roomy.close()


def test_footprint_bounds_the_allocation():
    w = _requests(1, seed=13)[0]
    for storage in ("f32", "f16"):
        g = lbe.Lattice(w.shape, w.rho0, storage=storage, **w.params)
        p = w.particles
        g.add_particles(p["pos"], p["quat"], p["r_par"], p["r_perp"], p["delta_rho"])
        fp = lbe.footprint(w.shape, 1, storage=storage, **w.params)
        held = g.device_bytes()
        g.close()
        # the footprint adds the transient initial-density buffer (2 N
        # doubles) and a bound on the pair cell list (1.5 bytes per node)
        n = w.rho0[0].size
        assert held <= fp <= held + 16 * n + 12 * (n // 8) + 1024


def test_oversized_and_invalid_requests_are_rejected():
    w = _requests(1, seed=15)[0]
    srv = lbe.Server(1 << 20, 2, "f32")
    with pytest.raises(lbe.LbeError) as e:
        _submit(srv, w, 100, 0.0)
    assert e.value.status == -2
    with pytest.raises(lbe.LbeError):
        srv.poll(12345)
    srv.close()


def test_batch_first_quat_in_member_order():
    reqs = _requests(3, seed=17)
    lats = []
    for w in reqs:
        g = lbe.Lattice(w.shape, w.rho0, **w.params)
        p = w.particles
        g.add_particles(p["pos"], p["quat"], p["r_par"], p["r_perp"], p["delta_rho"])
        lats.append(g)
    b = lbe.Batch(lats)
    b.step(3)
    q = b.first_quat()
    for k, g in enumerate(lats):
        assert np.array_equal(q[k], g.read_particles()["quat"][0])


def test_idle_server_starts_and_stops():
    """A server that never gets a request runs no chunk and shuts down cleanly."""
    import time
    srv = lbe.Server(1 * GB, 2, "f32")
    time.sleep(0.2)
    st = srv.stats()
    srv.close()
    assert st == {"completed": 0, "node_steps": 0, "max_running": 0, "chunks": 0}
