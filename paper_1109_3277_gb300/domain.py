"""Domain size of particle-stabilised emulsions against the particle
concentration, L(C) (§4, NEXT-3).

The paper measures the lateral domain size L = (L_x + L_y + L_z)/3 of
bijels at 256^3 for volume concentrations C = 0.08 ... 0.24 of ellipsoids
of aspect ratio 2 at Θ = 90°.  It fits L = a/C + b, with a ≈ 2.20 and
b ≈ 11.08 for m = 2.  Here each concentration is one lattice stepped by the
library; L(t) is computed on the host from the densities read back at
checkpoints.

L_i = 2π / sqrt(<k_i^2>), where <k_i^2> is the second moment of the
structure factor S(k) = |φ'_k|^2 / N of the order-parameter fluctuation
φ' = φ − <φ>, φ = ρ_r − ρ_b. The paper prints |φ'_k| without the square;
the squared modulus (the standard structure factor) is the reading taken.
Solid nodes take the mean φ of the fluid nodes. The transform is a real
FFT over x; the bins 0 < k_x < n_x/2 stand for two conjugate bins.
"""
import time

import numpy as np

from . import lbe
from . import workloads as W


def domain_size(rho, fluid=None):
    """(L, (L_x, L_y, L_z)) of the fields ``rho`` [2, nz, ny, nx]."""
    phi = np.asarray(rho[0], dtype=np.float64) - np.asarray(rho[1], dtype=np.float64)
    if fluid is not None:
        phi = np.where(fluid, phi, phi[fluid].mean())
    phi = phi - phi.mean()
    nz, ny, nx = phi.shape
    S = np.abs(np.fft.rfftn(phi)) ** 2 / phi.size
    mult = np.full(S.shape[2], 2.0)
    mult[0] = 1.0
    if nx % 2 == 0:
        mult[-1] = 1.0
    S = S * mult[None, None, :]
    k2 = [(2 * np.pi * np.fft.rfftfreq(nx)) ** 2,
          (2 * np.pi * np.fft.fftfreq(ny)) ** 2,
          (2 * np.pi * np.fft.fftfreq(nz)) ** 2]
    tot = S.sum()
    mx = (S.sum(axis=(0, 1)) * k2[0]).sum() / tot
    my = (S.sum(axis=(0, 2)) * k2[1]).sum() / tot
    mz = (S.sum(axis=(1, 2)) * k2[2]).sum() / tot
    L = [2 * np.pi / np.sqrt(m) if m > 0 else np.inf for m in (mx, my, mz)]
    return (L[0] + L[1] + L[2]) / 3.0, tuple(L)


def fit_inverse(concentrations, sizes):
    """Least-squares a, b of L = a / C + b."""
    x = 1.0 / np.asarray(concentrations, dtype=np.float64)
    a, b = np.polyfit(x, np.asarray(sizes, dtype=np.float64), 1)
    return float(a), float(b)


def study(concentrations, n=256, steps=20000, checkpoint=5000, storage="f16", lattice=None, **box):
    """One lattice per concentration, run for ``steps`` with L recorded at
    every ``checkpoint``; returns the L(t) series, the final sizes, the fit
    of L = a/C + b and the node updates per second of the stepping.
    ``lattice`` is the lattice class (default: the library's ``lbe.Lattice``;
    any class with its constructor, add_particles, step, mass, read_fields
    and close will do)."""
    make = lattice or lbe.Lattice
    out = {"C": [], "C_placed": [], "particles": [], "step": [], "L": [], "L_final": []}
    busy, nodes = 0.0, 0
    for C in concentrations:
        w = W.bijel_study_box(float(C), n=n, steps=steps, **box)
        g = make(w.shape, w.rho0, storage=storage, **w.params)
        p = w.particles
        g.add_particles(p["pos"], p["quat"], p["r_par"], p["r_perp"], p["delta_rho"])
        series, marks, done = [], [], 0
        while done < steps:
            k = min(checkpoint, steps - done)
            t0 = time.perf_counter()
            g.step(k)
            g.mass()  # synchronises
            busy += time.perf_counter() - t0
            done += k
            rho, _, typ = g.read_fields()
            series.append(domain_size(rho, typ == 0)[0])
            marks.append(done)
        g.close()
        nodes += int(np.prod(w.shape)) * steps
        out["C"].append(float(C))
        vol = 4.0 / 3.0 * np.pi * p["r_par"] * p["r_perp"] * p["r_perp"]
        out["C_placed"].append(float(vol.sum() / np.prod(w.shape)))
        out["particles"].append(len(p["pos"]))
        out["step"] = marks
        out["L"].append(series)
        out["L_final"].append(series[-1])
    # the fit uses the concentrations the placement reached
    a, b = fit_inverse(out["C_placed"], out["L_final"]) if len(concentrations) > 1 else (np.nan, np.nan)
    out.update({"a": a, "b": b, "mlups": nodes / busy / 1e6 if busy > 0 else np.nan, "seconds": busy})
    return out
