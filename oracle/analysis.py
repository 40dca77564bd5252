"""Observables of §4 of Günther et al., arXiv:1109.3277, computed on host
fields in FP64.

TEST INFRASTRUCTURE ONLY (part of the oracle).  Applied to the oracle's
fields and to fields read back from the CUDA library alike, so that a
statistic is compared through one definition.
"""
import numpy as np


def domain_size(rho, fluid=None, squared=True):
    """Lateral domain size of §4: L = (L_x + L_y + L_z)/3 with
    L_i = 2π / sqrt(<k_i^2>), <k_i^2> = Σ_k k_i^2 S(k) / Σ_k S(k), the structure
    function of the order-parameter fluctuation φ' = φ - <φ>, φ = ρ_r - ρ_b.

    The paper prints S(k) = |φ'_k| / N; the reading used here is the squared
    modulus (the standard structure factor), selected by ``squared``.
    ``rho`` is [2, nz, ny, nx]; solid nodes (``fluid`` False) are set to the
    mean before the transform.  Returns (L, (L_x, L_y, L_z))."""
    phi = np.asarray(rho[0], dtype=np.float64) - np.asarray(rho[1], dtype=np.float64)
    if fluid is not None:
        m = phi[fluid].mean()
        phi = np.where(fluid, phi, m)
    phi = phi - phi.mean()
    nz, ny, nx = phi.shape
    fk = np.fft.fftn(phi)
    S = np.abs(fk) ** 2 if squared else np.abs(fk)
    S = S / phi.size
    kz = 2 * np.pi * np.fft.fftfreq(nz)[:, None, None]
    ky = 2 * np.pi * np.fft.fftfreq(ny)[None, :, None]
    kx = 2 * np.pi * np.fft.fftfreq(nx)[None, None, :]
    tot = S.sum()
    out = []
    for k in (kx, ky, kz):
        m2 = float((np.broadcast_to(k * k, S.shape) * S).sum() / tot)
        out.append(2 * np.pi / np.sqrt(m2) if m2 > 0 else np.inf)
    return (out[0] + out[1] + out[2]) / 3.0, tuple(out)


def interface_area(rho, fluid=None, periodic=(True, True, True)):
    """Interface area (reading; the paper does not define a discrete
    measure): the number of axis-aligned nearest-neighbour links whose two
    ends are fluid and carry opposite signs of φ = ρ_r - ρ_b."""
    phi = np.asarray(rho[0], dtype=np.float64) - np.asarray(rho[1], dtype=np.float64)
    if fluid is None:
        fluid = np.ones(phi.shape, dtype=bool)
    count = 0
    for axis, per in zip((2, 1, 0), periodic):  # x, y, z axes of a [z, y, x] array
        a = phi
        b = np.roll(phi, -1, axis=axis)
        fa = fluid
        fb = np.roll(fluid, -1, axis=axis)
        cut = (a > 0) != (b > 0)
        ok = fa & fb
        if not per:
            sl = [slice(None)] * 3
            sl[axis] = slice(0, phi.shape[axis] - 1)
            cut = cut[tuple(sl)]
            ok = ok[tuple(sl)]
        count += int(np.count_nonzero(cut & ok))
    return count


def tilt(quat, normal=(0.0, 0.0, 1.0)):
    """Tilt φ of §4: the angle between the particle's main (symmetry) axis,
    the body x axis, and the interface normal, in [0, π/2]."""
    q = np.asarray(quat, dtype=np.float64).reshape(-1, 4)
    w, x, y, z = q.T
    n = np.sqrt(w * w + x * x + y * y + z * z)
    w, x, y, z = w / n, x / n, y / n, z / n
    axis = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)], axis=1)
    c = np.abs(axis @ np.asarray(normal, dtype=np.float64))
    return np.arccos(np.clip(c, 0.0, 1.0))


def interface_z(rho, col, walls=True):
    """Height of the φ = ρ_r − ρ_b = 0 crossing on lattice column col = (x,
    y): the zero of the straight line through the two nodes where φ changes
    sign (the crossing nearest mid-height if there are several), over the
    fluid planes (1 .. nz−2 between walls).  NaN without a crossing."""
    x, y = col
    phi = np.asarray(rho[0], dtype=np.float64)[:, y, x] - np.asarray(rho[1], dtype=np.float64)[:, y, x]
    nz = phi.size
    lo, hi = (1, nz - 2) if walls else (0, nz - 1)
    zs = []
    for z in range(lo, hi):
        if phi[z] == 0.0:
            zs.append(float(z))
        elif phi[z] * phi[z + 1] < 0.0:
            zs.append(z + phi[z] / (phi[z] - phi[z + 1]))
    if not zs:
        return float("nan")
    zs = np.asarray(zs)
    return float(zs[np.argmin(np.abs(zs - 0.5 * (lo + hi)))])


def sphere_contact_angle(z_centre, z_interface, radius):
    """Contact angle (degrees, through the lower, red phase) of a sphere whose
    centre is z_centre − z_interface above a flat interface.  The interface
    cuts the sphere in the circle at polar angle β from the upward axis,
    cos β = (z_interface − z_centre) / radius.  There the sphere's outward
    normal makes the angle β with the interface normal, so the angle between
    the two surfaces measured through the lower phase is Θ = β (a sphere
    below the interface, fully wetted by red, has Θ = 0)."""
    c = (z_interface - z_centre) / radius
    return float(np.degrees(np.arccos(min(1.0, max(-1.0, c)))))
