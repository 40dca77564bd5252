"""Single-ellipsoid adsorption at a flat interface (§4, NEXT-2).

An ellipsoid of aspect ratio m = 2 and colour Δρ = 0 (Θ = 90°) starts just
touching the interface between two lamellae, with its symmetry axis at the
angle φ(0) to the interface normal.  The paper reports two stages:
- the particle first moves toward the interface without turning;
- then it turns to φ ≈ 90° (the stable point).
A particle that starts at φ = 0 stays there, at a metastable point. Both
end points have the centre on the interface (z = 0) at Θ = 90°.

All starting angles run together as one batch. After every chunk of steps
the driver reads each particle's centre and orientation and the far
interface height. The tilt and the distance are host-side post-processing
of state read back through the C ABI.
"""
import time

import numpy as np

from . import contact_angle as CA
from . import lbe
from . import workloads as W


def tilt_deg(quat):
    """Angle (degrees, in [0, 90]) between the body x axis (the symmetry axis)
    of the unit quaternion (w, x, y, z) and the z axis."""
    w, x, y, z = np.asarray(quat, dtype=np.float64) / np.linalg.norm(quat)
    az = 2.0 * (x * z - w * y)  # z component of the rotated body x axis
    return float(np.degrees(np.arccos(min(1.0, abs(az)))))


def trajectories(tilts_deg, steps=8000, chunk=250, storage="f32", lattice=None, **box):
    """Run one box per starting angle together.

    Returns a dict with ``tilt0_deg`` and ``step`` (the chunk ends), and per
    box ``z`` (the centre minus the far interface height) and ``phi_deg``
    (the tilt) at every chunk end, plus ``mlups`` and ``seconds``.
    ``lattice`` replaces the library's lattice class (the boxes then step one
    after the other instead of as a batch)."""
    works = [W.adsorption_study_box(float(t), **box) for t in tilts_deg]
    lats = []
    for w in works:
        g = (lattice or lbe.Lattice)(w.shape, w.rho0, storage=storage, **w.params)
        p = w.particles
        g.add_particles(p["pos"], p["quat"], p["r_par"], p["r_perp"], p["delta_rho"])
        lats.append(g)
    batch = lbe.Batch(lats) if lattice is None else None
    z = [[] for _ in lats]
    phi = [[] for _ in lats]
    marks = []
    done, busy = 0, 0.0
    while done < steps:
        n = min(chunk, steps - done)
        t0 = time.perf_counter()
        if batch is not None:
            batch.step(n)
        else:
            for g in lats:
                g.step(n)
        for k, g in enumerate(lats):
            st = g.read_particles()
            pos = st["pos"][0]
            if k == 0:
                busy += time.perf_counter() - t0
            rho, _, _ = g.read_fields()
            zi = CA.interface_height(rho, *CA.far_column(g.shape, pos))
            z[k].append(float(pos[2] - zi))
            phi[k].append(tilt_deg(st["quat"][0]))
        done += n
        marks.append(done)
    if batch is not None:
        batch.close()
    for g in lats:
        g.close()
    nodes = sum(int(np.prod(w.shape)) for w in works)
    return {"tilt0_deg": [float(t) for t in tilts_deg], "step": marks, "z": z, "phi_deg": phi,
            "mlups": nodes * steps / busy / 1e6, "seconds": busy}
