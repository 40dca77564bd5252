"""Seeded synthetic inputs shaped like the workloads of Günther et al.,
arXiv:1109.3277 (§3 benchmark system, §4 adsorption box and emulsions).

This module holds no lattice Boltzmann arithmetic: only a counter-based
random generator (SplitMix64), density fields, particle placement and the
workload recipes.  It is the one module that both the CUDA path and the
oracle's tests draw their inputs from.
"""
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, count, stream=0):
    """SplitMix64 outputs number 1..count of the sequence started at
    seed * 2^32 + stream (Steele, Lea, Flood 2014), as uint64."""
    with np.errstate(over="ignore"):
        base = np.uint64((int(seed) << 32) + int(stream) & 0xFFFFFFFFFFFFFFFF)
        k = np.arange(1, count + 1, dtype=np.uint64)
        z = base + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, shape, stream=0, lo=0.0, hi=1.0):
    """Uniform doubles in [lo, hi) from the top 53 bits of SplitMix64."""
    n = int(np.prod(shape)) if np.ndim(shape) else int(shape)
    z = splitmix64(seed, n, stream)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return (lo + (hi - lo) * u).reshape(shape)


def random_quaternions(seed, n, stream=0):
    """Uniformly distributed unit quaternions (w, x, y, z) by Shoemake's
    subgroup algorithm (Graphics Gems III, 1992)."""
    u = uniform(seed, (n, 3), stream)
    a = np.sqrt(1.0 - u[:, 0])
    b = np.sqrt(u[:, 0])
    t1 = 2 * np.pi * u[:, 1]
    t2 = 2 * np.pi * u[:, 2]
    return np.stack([b * np.cos(t2), a * np.sin(t1), a * np.cos(t1), b * np.sin(t2)], axis=1)


def axis_tilt_quaternion(tilt, azimuth=0.0):
    """Quaternion that turns the body x axis (the symmetry axis) to the
    direction at polar angle ``tilt`` from +z and azimuth ``azimuth``."""
    # rotate e_x onto e_z first (about y by -90 deg), then tilt about y, then
    # spin about z: compose as a single axis-angle from e_x to the target.
    tgt = np.array([np.sin(tilt) * np.cos(azimuth), np.sin(tilt) * np.sin(azimuth), np.cos(tilt)])
    ex = np.array([1.0, 0.0, 0.0])
    c = float(np.clip(ex @ tgt, -1.0, 1.0))
    ax = np.cross(ex, tgt)
    s = np.linalg.norm(ax)
    if s < 1e-15:
        return np.array([1.0, 0.0, 0.0, 0.0]) if c > 0 else np.array([0.0, 0.0, 0.0, 1.0])
    ax = ax / s
    ang = np.arctan2(s, c)
    return np.array([np.cos(ang / 2), *(np.sin(ang / 2) * ax)])


# ---------------------------------------------------------------- fields

def uniform_mixture(shape, rho=0.7, noise=0.01, seed=0):
    """Both components at ``rho`` plus independent uniform noise in
    [-noise, noise) per node and component (spinodal start, §4)."""
    nx, ny, nz = shape
    return rho + uniform(seed, (2, nz, ny, nx), stream=1, lo=-noise, hi=noise)


def flat_interface(shape, z_interface, major=0.7, minor=0.04, noise=1e-3, seed=0):
    """Red-rich below ``z_interface`` and blue-rich above, as the two
    lamellae of the adsorption box of §4, plus uniform noise."""
    nx, ny, nz = shape
    z = np.arange(nz)[:, None, None]
    low = np.broadcast_to(z < z_interface, (nz, ny, nx))
    r = np.where(low, major, minor)
    b = np.where(low, minor, major)
    out = np.stack([r, b]).astype(np.float64)
    if noise:
        out = out + uniform(seed, out.shape, stream=2, lo=-noise, hi=noise)
    return out


def random_phases(shape, p_red, major=0.7, minor=0.04, seed=0):
    """Each node red-rich (major/minor) with probability ``p_red``, else
    blue-rich: the random initial densities of the emulsion runs of §4."""
    nx, ny, nz = shape
    red = uniform(seed, (nz, ny, nx), stream=3) < p_red
    return np.stack([np.where(red, major, minor), np.where(red, minor, major)]).astype(np.float64)


def random_populations(shape, seed=0, rho=0.5, spread=0.3):
    """Positive, non-equilibrium populations f[2][19][nz][ny][nx] for
    single-step checks: w_i-free uniform values around rho/19."""
    nx, ny, nz = shape
    return (rho / 19.0) * (1.0 + uniform(seed, (2, 19, nz, ny, nx), stream=4, lo=-spread, hi=spread))


# ------------------------------------------------------------- particles

def _inflated_nodes(shape, pos, quat, r_par, r_perp, margin, periodic):
    """Integer nodes inside the ellipsoid inflated by ``margin`` (used only
    to keep placements apart)."""
    w, x, y, z = quat / np.linalg.norm(quat)
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    a, b = r_par + margin, r_perp + margin
    h = int(np.ceil(max(a, b))) + 1
    rng = np.arange(-h, h + 1)
    gz, gy, gx = np.meshgrid(rng + int(np.floor(pos[2])), rng + int(np.floor(pos[1])),
                             rng + int(np.floor(pos[0])), indexing="ij")
    d = np.stack([gx - pos[0], gy - pos[1], gz - pos[2]], axis=-1) @ R
    qv = (d[..., 0] / a) ** 2 + (d[..., 1] / b) ** 2 + (d[..., 2] / b) ** 2
    sel = qv <= 1.0
    nx, ny, nz = shape
    X, Y, Z = gx[sel], gy[sel], gz[sel]
    if periodic[2]:
        Z = Z % nz
    else:
        keep = (Z >= 0) & (Z < nz)
        X, Y, Z = X[keep], Y[keep], Z[keep]
    return X % nx, Y % ny, Z


def place_ellipsoids(shape, count, r_par, r_perp, seed=0, margin=1.0, periodic=(True, True, True),
                     z_range=None, max_tries=None):
    """Random sequential addition: uniform centres and Shoemake orientations,
    rejected while the margin-inflated node sets overlap.  Returns (pos,
    quat) arrays; may return fewer than ``count`` if the space fills."""
    nx, ny, nz = shape
    occ = np.zeros((nz, ny, nx), dtype=bool)
    max_tries = max_tries or 50 * count + 1000
    u = uniform(seed, (max_tries, 3), stream=5)
    quats = random_quaternions(seed, max_tries, stream=6)
    lo = np.zeros(3)
    hi = np.array([nx, ny, nz], dtype=np.float64)
    if z_range is not None:
        lo[2], hi[2] = z_range
    pos_out, q_out = [], []
    for t in range(max_tries):
        if len(pos_out) >= count:
            break
        p = lo + (hi - lo) * u[t]
        X, Y, Z = _inflated_nodes(shape, p, quats[t], r_par, r_perp, margin, periodic)
        if occ[Z, Y, X].any():
            continue
        occ[Z, Y, X] = True
        pos_out.append(p)
        q_out.append(quats[t])
    return np.array(pos_out).reshape(-1, 3), np.array(q_out).reshape(-1, 4)


# ------------------------------------------------------------ workloads

@dataclass
class Workload:
    name: str
    shape: tuple
    params: dict
    rho0: np.ndarray
    steps: int
    particles: dict = field(default_factory=dict)
    storage: str = "f32"
    note: str = ""


def _particles(pos, quat, r_par, r_perp, delta_rho):
    n = len(pos)
    return {"pos": np.asarray(pos, dtype=np.float64).reshape(n, 3),
            "quat": np.asarray(quat, dtype=np.float64).reshape(n, 4),
            "r_par": np.full(n, float(r_par)), "r_perp": np.full(n, float(r_perp)),
            "delta_rho": np.full(n, float(delta_rho)) if np.ndim(delta_rho) == 0
            else np.asarray(delta_rho, dtype=np.float64)}


def adsorption_box(seed=1110, shape=(32, 32, 48), steps=200):
    """32x32x48 box, walls at z=0 and z=47, flat interface at z=24 (0.7 /
    0.04 + 1e-3 noise), one prolate ellipsoid r_par=6, r_perp=3 at the box
    centre on the interface, axis tilted 45 degrees from the normal, Δρ=0,
    τ=1, g=0.1, 200 steps."""
    nx, ny, nz = shape
    rho0 = flat_interface(shape, nz // 2, 0.7, 0.04, 1e-3, seed)
    q = axis_tilt_quaternion(np.pi / 4)
    return Workload("adsorption-32x32x48-1ellipsoid", shape,
                    dict(walls_z=True, tau=(1.0, 1.0), g_br=0.1, rho_ref=(0.37, 0.37)),
                    rho0, steps,
                    _particles([[nx / 2, ny / 2, nz / 2]], [q], 6.0, 3.0, 0.0))


def spinodal(seed=1111, n=128, steps=2000):
    """n^3 periodic, both components 0.7 + uniform noise in [-0.01, 0.01),
    g=0.1, τ=1, no particles.  The 16-bit offset base is each component's
    initial mean density, so the seeding noise is stored at full relative
    precision."""
    shape = (n, n, n)
    return Workload(f"spinodal-{n}^3", shape,
                    dict(walls_z=False, tau=(1.0, 1.0), g_br=0.1, rho_ref=(0.7, 0.7)),
                    uniform_mixture(shape, 0.7, 0.01, seed), steps)


def bijel(seed=1112, n=256, steps=5000, volume_fraction=0.15):
    """n^3 periodic 50/50 random mixture, oblate ellipsoids r_par=4,
    r_perp=8 at the given volume fraction, Δρ=0, g=0.1."""
    shape = (n, n, n)
    vol = 4.0 / 3.0 * np.pi * 4.0 * 8.0 * 8.0
    count = int(round(volume_fraction * n ** 3 / vol))
    pos, quat = place_ellipsoids(shape, count, 4.0, 8.0, seed)
    return Workload(f"bijel-{n}^3-{len(pos)}oblate", shape,
                    dict(walls_z=False, tau=(1.0, 1.0), g_br=0.1, rho_ref=(0.37, 0.37)),
                    random_phases(shape, 0.5, seed=seed), steps,
                    _particles(pos, quat, 4.0, 8.0, 0.0))


def pickering(seed=1113, n=512, steps=10000, volume_fraction=0.10, storage="f16"):
    """n^3 periodic, nodes red-rich with probability 0.8 (80/20), prolate
    ellipsoids r_par=8, r_perp=4 at the given volume fraction, Δρ=0.1."""
    shape = (n, n, n)
    vol = 4.0 / 3.0 * np.pi * 8.0 * 4.0 * 4.0
    count = int(round(volume_fraction * n ** 3 / vol))
    pos, quat = place_ellipsoids(shape, count, 8.0, 4.0, seed)
    return Workload(f"pickering-{n}^3-{len(pos)}prolate", shape,
                    dict(walls_z=False, tau=(1.0, 1.0), g_br=0.1, rho_ref=(0.37, 0.37)),
                    random_phases(shape, 0.8, seed=seed), steps,
                    _particles(pos, quat, 8.0, 4.0, 0.1), storage=storage)


def adsorption_request(seed, index, edge_range=(32, 96), m_range=(0.25, 4.0), r_perp=4.0,
                       drho_range=(-0.2, 0.2)):
    """One serving request: a cubic box with walls in z and a flat interface
    at mid-height holding one ellipsoid of aspect ratio m (r_par = m r_perp),
    random Δρ and a random tilt, its centre just above the interface."""
    u = uniform(seed, (64, 6), stream=100 + index)
    for row in u:
        edge = int(edge_range[0] + np.floor(row[0] * (edge_range[1] - edge_range[0] + 1)))
        m = m_range[0] + (m_range[1] - m_range[0]) * row[1]
        r_par = m * r_perp
        rmax = max(r_par, r_perp)
        # resampled: particles that do not fit between the walls, and discs
        # thinner than 2 lattice units (r_par < 2), which the lattice cannot
        # resolve (the method diverges on them, in FP64 too)
        if 2 * rmax + 6 <= edge and r_par >= 2.0:
            break
    drho = drho_range[0] + (drho_range[1] - drho_range[0]) * row[2]
    tilt = 0.5 * np.pi * row[3]
    az = 2 * np.pi * row[4]
    shape = (edge, edge, edge)
    zc = edge / 2.0 + min(rmax + 1.0, edge / 2.0 - rmax - 2.0)
    rho0 = flat_interface(shape, edge // 2, 0.7, 0.04, 1e-3, seed * 1000 + index)
    q = axis_tilt_quaternion(tilt, az)
    return Workload(f"request-{index}-edge{edge}", shape,
                    dict(walls_z=True, tau=(1.0, 1.0), g_br=0.1, rho_ref=(0.37, 0.37)),
                    rho0, 20000,
                    _particles([[edge / 2.0 + 0.25, edge / 2.0 + 0.25, zc]], [q], r_par, r_perp, drho))


def contact_angle_box(delta_rho, seed=1115, shape=(48, 48, 40), radius=5.0, steps=6000):
    """Contact-angle calibration (§2, the particle colour): a box with walls
    in z and a flat interface at mid-height (red-rich below, 0.7 / 0.04 with
    1e-3 noise), one sphere of radius ``radius`` and colour ``delta_rho``
    centred on the interface, τ = 1, g = 0.1.  The sphere settles at the
    height where the interface meets it at its contact angle."""
    nx, ny, nz = shape
    rho0 = flat_interface(shape, nz // 2, 0.7, 0.04, 1e-3, seed)
    return Workload(f"contact-angle-{nx}x{ny}x{nz}-R{radius:g}-drho{delta_rho:+.3f}", shape,
                    dict(walls_z=True, tau=(1.0, 1.0), g_br=0.1, rho_ref=(0.37, 0.37)),
                    rho0, steps,
                    _particles([[nx / 2.0, ny / 2.0, nz / 2.0]], [[1.0, 0.0, 0.0, 0.0]], radius, radius,
                               delta_rho))


def adsorption_study_box(tilt_deg, seed=1116, edge=64, r_par=12.0, r_perp=6.0, delta_rho=0.0, gap=2.0):
    """Single-ellipsoid adsorption of §4: a cube of edge 64 with walls at
    z = 0 and 63 and two lamellae (red-rich below z = 32, blue-rich above,
    0.7 / 0.04 with 1e-3 noise), g = 0.1, τ = 1, one ellipsoid of radii
    r_par = 12, r_perp = 6 (aspect ratio 2) and colour Δρ = 0 (Θ = 90°) whose
    axis makes the angle ``tilt_deg`` with the interface normal.  Its centre
    starts above the interface by its half-extent along z minus ``gap``, so
    that its lowest point dips ``gap`` nodes into the interface."""
    shape = (edge, edge, edge)
    t = np.radians(tilt_deg)
    half = np.sqrt((r_par * np.cos(t)) ** 2 + (r_perp * np.sin(t)) ** 2)
    zc = edge / 2.0 + half - gap
    rho0 = flat_interface(shape, edge // 2, 0.7, 0.04, 1e-3, seed)
    return Workload(f"adsorption-study-{edge}-m{r_par / r_perp:g}-tilt{tilt_deg:g}", shape,
                    dict(walls_z=True, tau=(1.0, 1.0), g_br=0.1, rho_ref=(0.37, 0.37)),
                    rho0, 10000,
                    _particles([[edge / 2.0 + 0.25, edge / 2.0 + 0.25, zc]], [axis_tilt_quaternion(t)],
                               r_par, r_perp, delta_rho))


def bijel_study_box(concentration, seed=1117, n=256, r_par=8.0, r_perp=4.0, g_br=0.08, steps=20000):
    """Domain size against particle concentration (§4): an n^3 periodic box
    with random initial densities, g = 0.08, and prolate ellipsoids of
    aspect ratio r_par / r_perp = 2 with Δρ = 0 (Θ = 90°) placed by random
    sequential addition to the volume fraction ``concentration``.  Each
    node's two densities are independent and uniform in [0, 1.4) (fluid
    ratio 1:1, mean 0.7 per component as in the spinodal start): at g =
    0.08 this mixture separates, while nodes that are red- or blue-rich at
    0.7 / 0.04 (mean 0.37) stay mixed.  The particles' mass density is 8,
    about six times the fluid's 1.4: lighter particles made the explicit
    update diverge at 256^3 and C = 0.24 (densities 1 and 2 within 5,000
    steps, 4 by step 9,000; 8 ran 20,000).  The paper gives no particle
    mass.  The placement keeps half a node
    between particles, so that random sequential addition still reaches C =
    0.24 (with a whole node it stalls near 0.18); the concentration reached
    is the number placed times the particle volume over n^3."""
    shape = (n, n, n)
    vol = 4.0 / 3.0 * np.pi * r_par * r_perp * r_perp
    count = int(round(concentration * n ** 3 / vol))
    pos, quat = place_ellipsoids(shape, count, r_par, r_perp, seed, margin=0.5)
    rho0 = uniform(seed, (2, n, n, n), stream=7, lo=0.0, hi=1.4)
    return Workload(f"bijel-study-{n}^3-C{concentration:g}-{len(pos)}prolate", shape,
                    dict(walls_z=False, tau=(1.0, 1.0), g_br=g_br, rho_ref=(0.7, 0.7), rho_particle=8.0),
                    rho0, steps, _particles(pos, quat, r_par, r_perp, 0.0), storage="f16")
