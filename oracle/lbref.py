"""ctypes binding of the FP64 CPU oracle (``liblbref.so``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only users.  The oracle shares no code with the CUDA
library; this module imports nothing from the product package.

The oracle computes the time step of Günther et al., arXiv:1109.3277, §2:
D3Q19 BGK (Eq. 1-2), Shan-Chen force (Eq. 3), moving bounce-back and momentum
exchange (Eq. 4-5), anisotropic Hertz/Berne-Pechukas and lubrication pair
forces (Eq. 6-9), outer-shell fill with the particle colour (Eq. 10).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbref.c")
_LIB = os.path.join(_HERE, "liblbref.so")

Q = 19


_LIB_OMP = os.path.join(_HERE, "liblbref_omp.so")


def build(force=False, omp=False):
    """Compile the oracle with plain gcc (no contraction of multiply-adds).
    omp=True builds liblbref_omp.so, whose per-node phases (moments, psi,
    force, collision) run over OpenMP threads; every node is computed by the
    same operations, and the particle sums stay serial, so its results equal
    the serial build's bit for bit.  The pins run the serial build."""
    lib_path = _LIB_OMP if omp else _LIB
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lbref.h"))):
        return lib_path
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC,
           "-o", lib_path + ".tmp", "-lm"]
    if omp:
        cmd[1:1] = ["-fopenmp", "-DLBREF_OMP"]
    subprocess.check_call(cmd)
    os.replace(lib_path + ".tmp", lib_path)
    return lib_path


class LatticeDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("walls_z", ctypes.c_int32),
        ("tau", ctypes.c_double * 2),
        ("g_br", ctypes.c_double),
        ("body_force", ctypes.c_double * 3),
        ("rho_ref", ctypes.c_double * 2),
        ("storage", ctypes.c_int32),
        ("particle_mode", ctypes.c_int32),
        ("k_hertz", ctypes.c_double),
        ("lub_cut", ctypes.c_double),
        ("lub_rho", ctypes.c_double),
        ("cuda_stream", ctypes.c_void_p),
        ("device", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("rho_particle", ctypes.c_double),
    ]


_lib = None


def lib():
    """The oracle library: the in-tree build, or the file named by the
    environment variable LBREF_LIB (the mutation tests load deliberately
    broken builds of the oracle this way, in subprocesses)."""
    global _lib
    if _lib is None:
        path = os.environ.get("LBREF_LIB") or build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        D = ctypes.POINTER(ctypes.c_double)
        L.lbref_init_lattice.argtypes = [ctypes.POINTER(LatticeDesc), D, ctypes.POINTER(P)]
        L.lbref_add_particles.argtypes = [P, ctypes.c_int32, D, D, D, D, D, D, D]
        L.lbref_step.argtypes = [P, ctypes.c_int32]
        L.lbref_read_fields.argtypes = [P, D, D, ctypes.POINTER(ctypes.c_uint8)]
        L.lbref_read_particles.argtypes = [P, D, D, D, D, D, D]
        L.lbref_mass.argtypes = [P, D]
        L.lbref_get_populations.argtypes = [P, D]
        L.lbref_set_populations.argtypes = [P, D]
        L.lbref_diagnostics.argtypes = [P, D]
        L.lbref_momentum.argtypes = [P, D]
        L.lbref_last_error.argtypes = [P]
        L.lbref_last_error.restype = ctypes.c_char_p
        L.lbref_destroy.argtypes = [P]
        L.lbref_destroy.restype = None
        L.lbref_lattice.argtypes = [ctypes.POINTER(ctypes.c_int32), D, ctypes.POINTER(ctypes.c_int32)]
        L.lbref_lattice.restype = None
        L.lbref_feq.argtypes = [ctypes.c_double, D, D]
        L.lbref_feq.restype = None
        L.lbref_pair_hertz.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, D, D, D,
                                       D, D, D, D, D]
        L.lbref_pair_hertz.restype = None
        L.lbref_rigid_update.argtypes = [ctypes.c_double] * 3 + [D] * 6
        L.lbref_rigid_update.restype = None
        L.lbref_inside.argtypes = [D, D, D, ctypes.c_double, ctypes.c_double]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def make_desc(shape, walls_z=False, tau=(1.0, 1.0), g_br=0.1, body_force=(0.0, 0.0, 0.0),
              rho_ref=(0.7, 0.7), particle_mode=0, k_hertz=100.0, lub_cut=2.0 / 3.0, lub_rho=1.4,
              rho_particle=1.0, **_ignored):
    nx, ny, nz = shape
    d = LatticeDesc()
    d.nx, d.ny, d.nz = nx, ny, nz
    d.walls_z = int(bool(walls_z))
    d.tau[0], d.tau[1] = tau
    d.g_br = g_br
    for k in range(3):
        d.body_force[k] = body_force[k]
    d.rho_ref[0], d.rho_ref[1] = rho_ref
    d.storage = 0
    d.particle_mode = particle_mode
    d.k_hertz = k_hertz
    d.lub_cut = lub_cut
    d.lub_rho = lub_rho
    d.cuda_stream = None
    d.device = -1
    d.flags = 0
    d.rho_particle = rho_particle
    return d


class OracleError(RuntimeError):
    pass


class Lattice:
    """One oracle lattice.  ``shape`` is (nx, ny, nz); ``rho0`` is [2, nz, ny, nx]."""

    def __init__(self, shape, rho0, **params):
        self.shape = tuple(shape)
        nx, ny, nz = self.shape
        self.N = nx * ny * nz
        self.desc = make_desc(self.shape, **params)
        r = _f64(rho0, (2, nz, ny, nx))
        self._ptr = ctypes.c_void_p()
        st = lib().lbref_init_lattice(ctypes.byref(self.desc), _dp(r), ctypes.byref(self._ptr))
        if st != 0:
            raise OracleError(f"lbref_init_lattice failed: {st}")
        self.np = 0

    def _check(self, st, what):
        if st != 0:
            msg = lib().lbref_last_error(self._ptr)
            raise OracleError(f"{what} failed ({st}): {msg.decode() if msg else ''}")

    def add_particles(self, pos, quat, r_par, r_perp, delta_rho, vel=None, omega=None):
        pos = _f64(pos).reshape(-1, 3)
        n = pos.shape[0]
        quat = _f64(quat).reshape(n, 4)
        vel = _f64(np.zeros((n, 3)) if vel is None else vel).reshape(n, 3)
        omega = _f64(np.zeros((n, 3)) if omega is None else omega).reshape(n, 3)
        rp = _f64(np.broadcast_to(r_par, (n,)))
        ro = _f64(np.broadcast_to(r_perp, (n,)))
        dr = _f64(np.broadcast_to(delta_rho, (n,)))
        self._check(lib().lbref_add_particles(self._ptr, n, _dp(pos), _dp(quat), _dp(vel),
                                              _dp(omega), _dp(rp), _dp(ro), _dp(dr)),
                    "add_particles")
        self.np += n

    def step(self, n=1):
        self._check(lib().lbref_step(self._ptr, int(n)), "step")

    def read_fields(self):
        nx, ny, nz = self.shape
        rho = np.zeros((2, nz, ny, nx))
        vel = np.zeros((3, nz, ny, nx))
        typ = np.zeros((nz, ny, nx), dtype=np.uint8)
        self._check(lib().lbref_read_fields(self._ptr, _dp(rho), _dp(vel),
                                            typ.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))),
                    "read_fields")
        return rho, vel, typ

    def read_particles(self):
        n = self.np
        out = {k: np.zeros((n, 4 if k == "quat" else 3)) for k in
               ("pos", "quat", "vel", "omega", "force", "torque")}
        self._check(lib().lbref_read_particles(self._ptr, _dp(out["pos"]), _dp(out["quat"]),
                                               _dp(out["vel"]), _dp(out["omega"]),
                                               _dp(out["force"]), _dp(out["torque"])),
                    "read_particles")
        return out

    def mass(self):
        out = np.zeros(2)
        self._check(lib().lbref_mass(self._ptr, _dp(out)), "mass")
        return out

    def get_populations(self):
        nx, ny, nz = self.shape
        f = np.zeros((2, Q, nz, ny, nx))
        self._check(lib().lbref_get_populations(self._ptr, _dp(f)), "get_populations")
        return f

    def set_populations(self, f):
        nx, ny, nz = self.shape
        f = _f64(f, (2, Q, nz, ny, nx))
        self._check(lib().lbref_set_populations(self._ptr, _dp(f)), "set_populations")

    def diagnostics(self):
        out = np.zeros(6)
        self._check(lib().lbref_diagnostics(self._ptr, _dp(out)), "diagnostics")
        return {"created": out[0:2].copy(), "deleted": out[2:4].copy(), "sum_c": out[4:6].copy()}

    def momentum(self):
        out = np.zeros(9)
        self._check(lib().lbref_momentum(self._ptr, _dp(out)), "momentum")
        return {"fluid": out[0:3].copy(), "particles": out[3:6].copy(),
                "pending": out[6:9].copy()}

    def close(self):
        if self._ptr:
            lib().lbref_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lattice_tables():
    c = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, dtype=np.int32)
    lib().lbref_lattice(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(w),
                        opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return c, w, opp


def feq(rho, u):
    u = _f64(u, (3,))
    out = np.zeros(Q)
    lib().lbref_feq(float(rho), _dp(u), _dp(out))
    return out


def pair_hertz(k_hertz, r_par, r_perp, r, oi, oj):
    r, oi, oj = _f64(r, (3,)), _f64(oi, (3,)), _f64(oj, (3,))
    e = np.zeros(1)
    fj, ti, tj = np.zeros(3), np.zeros(3), np.zeros(3)
    sig = np.zeros(1)
    lib().lbref_pair_hertz(float(k_hertz), float(r_par), float(r_perp), _dp(r), _dp(oi),
                           _dp(oj), _dp(e), _dp(fj), _dp(ti), _dp(tj), _dp(sig))
    return {"energy": e[0], "f_j": fj, "t_i": ti, "t_j": tj, "sigma": sig[0]}


def rigid_update(mass, i_par, i_perp, force, torque, pos, quat, vel, omega):
    force, torque = _f64(force, (3,)), _f64(torque, (3,))
    pos, quat = _f64(pos, (3,)).copy(), _f64(quat, (4,)).copy()
    vel, omega = _f64(vel, (3,)).copy(), _f64(omega, (3,)).copy()
    lib().lbref_rigid_update(float(mass), float(i_par), float(i_perp), _dp(force), _dp(torque),
                             _dp(pos), _dp(quat), _dp(vel), _dp(omega))
    return pos, quat, vel, omega


def inside(node, pos, quat, r_par, r_perp):
    node, pos, quat = _f64(node, (3,)), _f64(pos, (3,)), _f64(quat, (4,))
    return bool(lib().lbref_inside(_dp(node), _dp(pos), _dp(quat), float(r_par), float(r_perp)))
