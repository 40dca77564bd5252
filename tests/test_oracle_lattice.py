"""Pins of the oracle's lattice tables and equilibrium against the
isotropy conditions that any D3Q19 model must meet (§2: "a D3Q19
implementation"; the weights and velocities are not printed in the paper)."""
import itertools

import numpy as np

from oracle import lbref


def test_d3q19_velocity_set():
    c, w, opp = lbref.lattice_tables()
    rows = {tuple(v) for v in c}
    assert len(rows) == 19
    # rest + 6 axis + 12 face diagonals, no body diagonals
    norms = sorted(int((v * v).sum()) for v in c)
    assert norms == [0] + [1] * 6 + [2] * 12
    for i in range(19):
        assert np.all(c[opp[i]] == -c[i])
        assert w[opp[i]] == w[i]


def test_isotropy_moments():
    c, w, _ = lbref.lattice_tables()
    c = c.astype(np.float64)
    cs2 = 1.0 / 3.0
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w @ c, 0.0, atol=1e-16)
    m2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(m2, cs2 * np.eye(3), atol=1e-15)
    m3 = np.einsum("i,ia,ib,ic->abc", w, c, c, c)
    assert np.allclose(m3, 0.0, atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    want = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                       + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(m4, want, atol=1e-15)


def test_equilibrium_moments():
    c, _, _ = lbref.lattice_tables()
    c = c.astype(np.float64)
    for rho, u in [(0.7, (0.0, 0.0, 0.0)), (1.3, (0.05, -0.02, 0.01)), (0.04, (-0.1, 0.07, 0.03))]:
        u = np.array(u)
        f = lbref.feq(rho, u)
        assert abs(f.sum() - rho) < 1e-15
        assert np.allclose(f @ c, rho * u, atol=1e-16)
        pi = np.einsum("i,ia,ib->ab", f, c, c)
        assert np.allclose(pi, rho * (np.eye(3) / 3.0 + np.outer(u, u)), atol=1e-15)


def test_equilibrium_at_rest_is_weights():
    _, w, _ = lbref.lattice_tables()
    for rho in (0.04, 0.7):
        assert np.allclose(lbref.feq(rho, np.zeros(3)), rho * w, rtol=0, atol=1e-17)


def test_unweighted_stencil_second_moment():
    """The reading of Eq. 3 (unweighted sum over the 18 neighbours) has
    Σ_i c_i c_i = 10 I, the factor in the equation of state used by the
    Laplace check."""
    c, _, _ = lbref.lattice_tables()
    c = c.astype(np.float64)
    assert np.allclose(c.T @ c, 10.0 * np.eye(3))
    for a, b in itertools.product(range(3), repeat=2):
        assert (c[:, a] * c[:, b]).sum() == (10 if a == b else 0)
