"""Literal, per-equation evaluation of one time step of §2 of Günther et al.,
arXiv:1109.3277, for tiny lattices: direct Python loops over nodes x,
directions i and components c, nothing vectorised or fused.  Used only to
pin the oracle (tests/test_oracle_fluid.py).

Covers: Eq. 1 (streaming), Eq. 2 (BGK), Eq. 3 (Shan-Chen force, unweighted
neighbour sum), the shifted-velocity forcing, Eq. 4-5 (moving bounce-back and
momentum exchange), Eq. 10 + colour rule (shell fill).  Particles are held
static (no integration, no coverage change)."""
import math

import numpy as np

# D3Q19, written out independently of the oracle's table
VEL = [(0, 0, 0)]
for a in range(3):
    for s in (1, -1):
        v = [0, 0, 0]
        v[a] = s
        VEL.append(tuple(v))
for a, b in ((0, 1), (0, 2), (1, 2)):
    for sa, sb in ((1, 1), (-1, -1), (1, -1), (-1, 1)):
        v = [0, 0, 0]
        v[a], v[b] = sa, sb
        VEL.append(tuple(v))
WGT = [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12
OPP = [VEL.index(tuple(-x for x in v)) for v in VEL]


def quat_to_matrix(q):
    w, x, y, z = q
    return [[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
            [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
            [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]]


def nearest_image(d, n):
    return d - n * round(d / n)


def node_types(shape, walls, particles):
    nx, ny, nz = shape
    typ = {}
    owner = {}
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if walls and z in (0, nz - 1):
                    typ[x, y, z] = 1
                    continue
                typ[x, y, z] = 0
                for p, P in enumerate(particles):
                    R = quat_to_matrix(P["quat"])
                    d = [nearest_image(x - P["pos"][0], nx), nearest_image(y - P["pos"][1], ny),
                         (z - P["pos"][2]) if walls else nearest_image(z - P["pos"][2], nz)]
                    b = [sum(R[j][k] * d[j] for j in range(3)) for k in range(3)]
                    if (b[0] / P["r_par"]) ** 2 + (b[1] / P["r_perp"]) ** 2 + (b[2] / P["r_perp"]) ** 2 <= 1:
                        typ[x, y, z] = 2
                        owner[x, y, z] = p
                        break
    return typ, owner


def step(shape, f, walls, tau, g, body, particles):
    """One step.  f is [2][19][nz][ny][nx]; returns (f_new, forces, torques)."""
    nx, ny, nz = shape
    typ, owner = node_types(shape, walls, particles)

    def nb(x, y, z, v):
        xx, yy, zz = (x + v[0]) % nx, (y + v[1]) % ny, z + v[2]
        if walls:
            if zz < 0 or zz >= nz:
                return None
        else:
            zz %= nz
        return xx, yy, zz

    nodes = list(typ.keys())
    rho, j = {}, {}
    for n in nodes:
        x, y, z = n
        for c in range(2):
            if typ[n] == 0:
                rho[n, c] = sum(f[c][i][z][y][x] for i in range(19))
                j[n, c] = [sum(f[c][i][z][y][x] * VEL[i][a] for i in range(19)) for a in range(3)]
            else:
                rho[n, c] = 0.0
                j[n, c] = [0.0, 0.0, 0.0]
    psi = {}
    for n in nodes:
        if typ[n] == 0:
            for c in range(2):
                psi[n, c] = 1 - math.exp(-rho[n, c])
            continue
        fl = [m for m in (nb(*n, VEL[i]) for i in range(1, 19)) if m is not None and typ[m] == 0]
        if not fl:
            psi[n, 0] = psi[n, 1] = 0.0
            continue
        rn = [sum(rho[m, c] for m in fl) / len(fl) for c in range(2)]
        dr = particles[owner[n]]["delta_rho"] if typ[n] == 2 else 0.0
        if dr > 0:
            rn[0] += dr
        else:
            rn[1] += abs(dr)
        for c in range(2):
            psi[n, c] = 1 - math.exp(-rn[c])
    force = {}
    for n in nodes:
        if typ[n] != 0:
            continue
        for c in range(2):
            other = 1 - c
            s = [0.0, 0.0, 0.0]
            for i in range(1, 19):
                m = nb(*n, VEL[i])
                for a in range(3):
                    s[a] += psi[m, other] * VEL[i][a]
            force[n, c] = [-g * psi[n, c] * s[a] + rho[n, c] * body[a] for a in range(3)]
    fstar = {}
    for n in nodes:
        if typ[n] != 0:
            continue
        x, y, z = n
        den = sum(rho[n, c] / tau[c] for c in range(2))
        up = [sum(j[n, c][a] / tau[c] for c in range(2)) / den if den > 0 else 0.0 for a in range(3)]
        for c in range(2):
            r = rho[n, c]
            ue = [up[a] + tau[c] * force[n, c][a] / r if r > 0 else up[a] for a in range(3)]
            uu = sum(v * v for v in ue)
            for i in range(19):
                cu = sum(VEL[i][a] * ue[a] for a in range(3))
                feq = WGT[i] * r * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)
                fstar[n, c, i] = f[c][i][z][y][x] - (f[c][i][z][y][x] - feq) / tau[c]
    fnew = np.array(f, dtype=np.float64, copy=True)
    forces = [np.zeros(3) for _ in particles]
    torques = [np.zeros(3) for _ in particles]
    for n in nodes:
        if typ[n] != 0:
            continue
        x, y, z = n
        for i in range(19):
            src = nb(x, y, z, tuple(-v for v in VEL[i]))
            for c in range(2):
                if src is not None and typ[src] == 0:
                    fnew[c][i][z][y][x] = fstar[src, c, i]
                elif src is not None and typ[src] == 2:
                    P = particles[owner[src]]
                    rb = [nearest_image(x - P["pos"][0], nx) - VEL[i][0] / 2,
                          nearest_image(y - P["pos"][1], ny) - VEL[i][1] / 2,
                          ((z - P["pos"][2]) if walls else nearest_image(z - P["pos"][2], nz))
                          - VEL[i][2] / 2]
                    us = np.array(P["vel"]) + np.cross(P["omega"], rb)
                    C = 2 * WGT[i] / (1 / 3) * rho[n, c] * float(us @ np.array(VEL[i]))
                    fr = fstar[n, c, OPP[i]]
                    fnew[c][i][z][y][x] = fr + C
                    F = (2 * fr + C) * np.array(VEL[OPP[i]], dtype=np.float64)
                    forces[owner[src]] += F
                    torques[owner[src]] += np.cross(rb, F)
                else:
                    fnew[c][i][z][y][x] = fstar[n, c, OPP[i]]
    return fnew, forces, torques, typ
