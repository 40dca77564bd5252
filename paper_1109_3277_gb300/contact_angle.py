"""Contact-angle calibration Θ(Δρ) of the particle colour (§2).

The paper fits the contact angle of a particle against its colour Δρ with a
straight line: 243.2° per unit Δρ through 90° at Δρ = 0, and it notes that
the slope depends on the simulation parameters.

Here a sphere of radius R starts centred on a flat interface between the
red-rich (lower) and blue-rich (upper) phases. It settles at the height
where the interface meets its surface at the contact angle. With h the
height of its centre above the flat interface far from it,

    cos Θ = -h / R,

so Θ is measured through the red phase. Θ = 0 is a sphere fully wetted by
red and Θ = 180° one fully in blue. Raising Δρ (more red density in the
shell) drives the sphere into the blue phase, so Θ grows with Δρ, the sign
of the paper's fit. The far interface is located on the lattice column
farthest from the sphere, where φ = ρ_r − ρ_b changes sign, by linear
interpolation between the two nodes around the crossing. A sphere with
|h| ≥ R has left the interface, and the fit leaves it out.

All boxes of a calibration run together as one batch (one launch per
kernel for all of them). The analysis here is host-side post-processing of
fields and particle state read back through the C ABI.
"""
import time

import numpy as np

from . import lbe
from . import workloads as W


def interface_height(rho, x, y, z_lo=1, z_hi=None):
    """Height z of the φ = ρ_r − ρ_b = 0 crossing on the column (x, y) of
    ``rho`` [2, nz, ny, nx], between planes z_lo and z_hi (the fluid planes
    between the walls by default): the crossing nearest the column's middle,
    interpolated linearly.  NaN if φ does not change sign."""
    phi = np.asarray(rho[0][:, y, x], dtype=np.float64) - np.asarray(rho[1][:, y, x], dtype=np.float64)
    nz = phi.shape[0]
    z_hi = nz - 2 if z_hi is None else z_hi
    best = np.nan
    mid = 0.5 * (z_lo + z_hi)
    for z in range(z_lo, z_hi):
        a, b = phi[z], phi[z + 1]
        if a == 0.0:
            cand = float(z)
        elif (a > 0.0) != (b > 0.0) and b != 0.0:
            cand = z + a / (a - b)
        else:
            continue
        if np.isnan(best) or abs(cand - mid) < abs(best - mid):
            best = cand
    return best


def contact_angle(z_particle, z_interface, radius):
    """Θ in degrees, measured through the red (lower) phase: cos Θ =
    (z_interface − z_particle) / radius, clipped to [−1, 1]."""
    c = (float(z_interface) - float(z_particle)) / float(radius)
    return float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))


def far_column(shape, pos):
    """The lattice column farthest from ``pos`` in a box periodic in x and y."""
    nx, ny, _ = shape
    return int(np.floor(pos[0] + nx / 2.0)) % nx, int(np.floor(pos[1] + ny / 2.0)) % ny


def calibrate(delta_rhos, steps=6000, shape=(48, 48, 40), radius=5.0, storage="f32", chunk=500, seed=1115,
              lattice=None):
    """Run one box per Δρ together and return the contact angles.

    ``lattice`` replaces the library's lattice class (then the boxes step one
    after the other instead of as a batch); any class with the constructor,
    add_particles, step, read_particles, read_fields and close of
    ``lbe.Lattice`` will do.

    Returns a dict: ``delta_rho``; ``theta_deg`` (per box, after ``steps``);
    ``height`` (sphere centre minus far interface height, per box); the
    least-squares line ``slope_deg`` and ``intercept_deg`` of Θ against Δρ;
    ``trace`` (per chunk of ``chunk`` steps: the sphere heights); the
    node updates per second of the batch (``mlups``)."""
    boxes = [W.contact_angle_box(float(d), seed=seed, shape=shape, radius=radius, steps=steps)
             for d in delta_rhos]
    lats = []
    for w in boxes:
        g = (lattice or lbe.Lattice)(w.shape, w.rho0, storage=storage, **w.params)
        p = w.particles
        g.add_particles(p["pos"], p["quat"], p["r_par"], p["r_perp"], p["delta_rho"])
        lats.append(g)
    batch = lbe.Batch(lats) if lattice is None else None
    trace = []
    done = 0
    t0 = time.perf_counter()
    while done < steps:
        n = min(chunk, steps - done)
        if batch is not None:
            batch.step(n)
        else:
            for g in lats:
                g.step(n)
        done += n
        trace.append([float(g.read_particles()["pos"][0, 2]) for g in lats])
    dt = time.perf_counter() - t0
    thetas, heights = [], []
    for g in lats:
        pos = g.read_particles()["pos"][0]
        rho, _, _ = g.read_fields()
        x, y = far_column(shape, pos)
        zi = interface_height(rho, x, y)
        heights.append(float(pos[2] - zi))
        thetas.append(contact_angle(pos[2], zi, radius))
    if batch is not None:
        batch.close()
    for g in lats:
        g.close()
    d = np.asarray(delta_rhos, dtype=np.float64)
    attached = np.abs(np.asarray(heights)) < radius
    th = np.asarray(thetas)
    if attached.sum() >= 2:
        slope, intercept = np.polyfit(d[attached], th[attached], 1)
    else:
        slope, intercept = np.nan, np.nan
    nodes = int(np.prod(shape)) * len(lats)
    return {"delta_rho": [float(v) for v in d], "theta_deg": thetas, "height": heights,
            "attached": [bool(a) for a in attached], "slope_deg": float(slope),
            "intercept_deg": float(intercept), "trace": trace, "steps": steps,
            "mlups": nodes * steps / dt / 1e6, "seconds": dt}
