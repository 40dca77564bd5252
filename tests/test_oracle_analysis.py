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
