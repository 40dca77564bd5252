"""Python binding of liblbe.so (include/lbe.h): argument marshalling only.

Every step of the lattice Boltzmann path runs in the library's CUDA kernels.
There is no fallback: if the library or a GPU is missing the calls raise.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("LBE_LIB") or os.path.join(HERE, "liblbe.so")
Q = 19

STORAGE = {"f32": 0, "bf16": 1, "f16": 2}
MODES = {"free": 0, "static": 1, "prescribed": 2}
FLAG_TWO_PASS = 1
FLAG_WIDE_OFFSETS = 2
PARTICLE_IN = 16   # pos[3], quat[4], vel[3], omega[3], r_par, r_perp, delta_rho
PARTICLE_OUT = 19  # pos[3], quat[4], vel[3], omega[3], force[3], torque[3]

STATUS = {0: "LBE_OK", -1: "LBE_EINVAL", -2: "LBE_ENOMEM", -3: "LBE_ECUDA", -4: "LBE_ENUMERIC",
          -5: "LBE_EOVERLAP", -6: "LBE_ETIMEOUT", -7: "LBE_EBUSY"}


class LbeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


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


# Every symbol include/lbe.h declares, with (restype, argtypes).
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "lbe_init_lattice": (ctypes.c_int, [ctypes.POINTER(LatticeDesc), _D, ctypes.POINTER(_P)]),
    "lbe_add_particles": (ctypes.c_int, [_P, ctypes.c_int32, _D, _D, _D, _D, _D, _D, _D]),
    "lbe_step": (ctypes.c_int, [_P, ctypes.c_int32]),
    "lbe_read_fields": (ctypes.c_int, [_P, _D, _D, ctypes.POINTER(ctypes.c_uint8)]),
    "lbe_read_particles": (ctypes.c_int, [_P, _D, _D, _D, _D, _D, _D]),
    "lbe_mass": (ctypes.c_int, [_P, _D]),
    "lbe_get_populations": (ctypes.c_int, [_P, _D]),
    "lbe_set_populations": (ctypes.c_int, [_P, _D]),
    "lbe_profile_enable": (ctypes.c_int, [_P, ctypes.c_int32]),
    "lbe_profile_read": (ctypes.c_int, [_P, _D, ctypes.POINTER(ctypes.c_int64)]),
    "lbe_kernels_per_step": (ctypes.c_int32, [_P]),
    "lbe_device_bytes": (ctypes.c_size_t, [_P]),
    "lbe_mass_noalloc": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int64, ctypes.c_int64, _D,
                                         ctypes.c_int32, _P, _P]),
    "lbe_autotune": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "lbe_set_zchunk": (ctypes.c_int, [_P, ctypes.c_int32]),
    "lbe_set_tile": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "lbe_get_tile": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "lbe_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "lbe_fail_allocations": (None, [ctypes.c_int32]),
    "lbe_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, ctypes.POINTER(_P)]),
    "lbe_batch_step": (ctypes.c_int, [_P, ctypes.c_int32]),
    "lbe_batch_autotune": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "lbe_batch_kernels_per_step": (ctypes.c_int32, [_P]),
    "lbe_batch_destroy": (None, [_P]),
    "lbe_footprint": (ctypes.c_size_t, [ctypes.POINTER(LatticeDesc), ctypes.c_int32]),
    "lbe_batch_first_quat": (ctypes.c_int, [_P, _D]),
    "lbe_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_P)]),
    "lbe_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(LatticeDesc), _D, ctypes.c_int32, _D, ctypes.c_int32,
                                         ctypes.c_double, ctypes.POINTER(ctypes.c_uint64)]),
    "lbe_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_int32), _D]),
    "lbe_server_wait": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int32]),
    "lbe_server_timing": (ctypes.c_int, [_P, ctypes.c_uint64, _D, _D]),
    "lbe_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "lbe_server_destroy": (None, [_P]),
    "lbe_last_error": (ctypes.c_char_p, [_P]),
    "lbe_destroy": (None, [_P]),
}

_lib = None


def load(path=LIB_PATH):
    """Load liblbe.so (build it first with paper_1109_3277_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(shape) if shape is not None else a


def make_desc(shape, walls_z=False, tau=(1.0, 1.0), g_br=0.1, body_force=(0.0, 0.0, 0.0),
              rho_ref=(0.37, 0.37), storage="f32", particle_mode="free", k_hertz=100.0,
              lub_cut=2.0 / 3.0, lub_rho=1.4, stream=None, device=-1, flags=0, rho_particle=1.0):
    nx, ny, nz = shape
    d = LatticeDesc()
    d.nx, d.ny, d.nz = nx, ny, nz
    d.walls_z = int(bool(walls_z))
    d.tau[0], d.tau[1] = tau
    d.g_br = g_br
    for k in range(3):
        d.body_force[k] = body_force[k]
    d.rho_ref[0], d.rho_ref[1] = rho_ref
    d.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    d.particle_mode = MODES[particle_mode] if isinstance(particle_mode, str) else int(particle_mode)
    d.k_hertz = k_hertz
    d.lub_cut = lub_cut
    d.lub_rho = lub_rho
    d.cuda_stream = stream
    d.device = int(device)
    d.flags = int(flags)
    d.rho_particle = rho_particle
    return d


class Lattice:
    """One lattice on the current CUDA device.  ``shape`` is (nx, ny, nz);
    ``rho0`` is [2, nz, ny, nx] (host)."""

    def __init__(self, shape, rho0, **params):
        self.shape = tuple(shape)
        nx, ny, nz = self.shape
        self.N = nx * ny * nz
        self.desc = make_desc(self.shape, **params)
        r = _f64(rho0, (2, nz, ny, nx))
        self._ptr = ctypes.c_void_p()
        st = load().lbe_init_lattice(ctypes.byref(self.desc), _dp(r), ctypes.byref(self._ptr))
        if st != 0:
            raise LbeError(st, "lbe_init_lattice")
        self.np = 0

    def _check(self, st, what):
        if st != 0:
            msg = load().lbe_last_error(self._ptr)
            raise LbeError(st, f"{what}: {msg.decode() if msg else ''}")

    def add_particles(self, pos, quat, r_par, r_perp, delta_rho, vel=None, omega=None):
        pos = _f64(pos).reshape(-1, 3)
        n = pos.shape[0]
        quat = _f64(quat).reshape(n, 4)
        vel = None if vel is None else _f64(vel).reshape(n, 3)
        omega = None if omega is None else _f64(omega).reshape(n, 3)
        rp = _f64(np.broadcast_to(r_par, (n,)))
        ro = _f64(np.broadcast_to(r_perp, (n,)))
        dr = _f64(np.broadcast_to(delta_rho, (n,)))
        self._check(load().lbe_add_particles(self._ptr, n, _dp(pos), _dp(quat), _dp(vel), _dp(omega),
                                             _dp(rp), _dp(ro), _dp(dr)), "add_particles")
        self.np += n

    def step(self, n=1):
        self._check(load().lbe_step(self._ptr, int(n)), "step")

    def read_fields(self, rho=True, vel=True, types=True):
        nx, ny, nz = self.shape
        r = np.zeros((2, nz, ny, nx)) if rho else None
        v = np.zeros((3, nz, ny, nx)) if vel else None
        t = np.zeros((nz, ny, nx), dtype=np.uint8) if types else None
        self._check(load().lbe_read_fields(self._ptr, _dp(r), _dp(v),
                                           t.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
                                           if t is not None else None), "read_fields")
        return r, v, t

    def read_particles(self):
        n = self.np
        out = {k: np.zeros((n, 4 if k == "quat" else 3)) for k in
               ("pos", "quat", "vel", "omega", "force", "torque")}
        self._check(load().lbe_read_particles(self._ptr, _dp(out["pos"]), _dp(out["quat"]),
                                              _dp(out["vel"]), _dp(out["omega"]), _dp(out["force"]),
                                              _dp(out["torque"])), "read_particles")
        return out

    def mass(self):
        out = np.zeros(2)
        self._check(load().lbe_mass(self._ptr, _dp(out)), "mass")
        return out

    def get_populations(self):
        nx, ny, nz = self.shape
        f = np.zeros((2, Q, nz, ny, nx))
        self._check(load().lbe_get_populations(self._ptr, _dp(f)), "get_populations")
        return f

    def set_populations(self, f):
        nx, ny, nz = self.shape
        f = _f64(f, (2, Q, nz, ny, nx))
        self._check(load().lbe_set_populations(self._ptr, _dp(f)), "set_populations")

    def profile_enable(self, on=True):
        self._check(load().lbe_profile_enable(self._ptr, int(bool(on))), "profile_enable")

    def profile_read(self):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(load().lbe_profile_read(self._ptr, ctypes.byref(ms), ctypes.byref(n)),
                    "profile_read")
        return ms.value, n.value

    def kernels_per_step(self):
        return int(load().lbe_kernels_per_step(self._ptr))

    def autotune(self):
        """Time the fused kernel's z-chunk candidates; returns the one chosen."""
        zc = ctypes.c_int32()
        self._check(load().lbe_autotune(self._ptr, ctypes.byref(zc)), "autotune")
        return zc.value

    def set_zchunk(self, zc):
        """Fix the fused kernel's z chunk (0: default); results do not depend on it."""
        self._check(load().lbe_set_zchunk(self._ptr, int(zc)), "set_zchunk")

    def set_tile(self, rows, zc=0):
        """Fix the fused kernel's tile height (4 or 8) and z chunk (0: default)."""
        self._check(load().lbe_set_tile(self._ptr, int(rows), int(zc)), "set_tile")

    def tile(self):
        """(rows, z chunk) of the fused kernel's tiles in use."""
        r, z = ctypes.c_int32(), ctypes.c_int32()
        self._check(load().lbe_get_tile(self._ptr, ctypes.byref(r), ctypes.byref(z)), "get_tile")
        return r.value, z.value

    def set_wait_limit(self, tries, unreachable=False):
        """Tries of each bounded wait for a box copy (0: the default);
        unreachable: wait for a phase no copy completes (timeout tests)."""
        self._check(load().lbe_set_wait_limit(self._ptr, int(tries), int(bool(unreachable))), "set_wait_limit")

    def device_bytes(self):
        return int(load().lbe_device_bytes(self._ptr))

    def close(self):
        if self._ptr:
            load().lbe_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several lattices stepped together by one launch per kernel (a
    persistent fused kernel over the tiles of all members).  The members stay
    ordinary Lattice objects for reading; they must outlive the batch and
    must not gain particles while it exists."""

    def __init__(self, members):
        self.members = list(members)
        arr = (ctypes.c_void_p * len(self.members))(*[m._ptr.value for m in self.members])
        self._ptr = ctypes.c_void_p()
        st = load().lbe_batch_create(arr, len(self.members), ctypes.byref(self._ptr))
        if st != 0:
            raise LbeError(st, "lbe_batch_create")

    def step(self, n=1):
        st = load().lbe_batch_step(self._ptr, int(n))
        if st != 0:
            raise LbeError(st, "lbe_batch_step")

    def autotune(self):
        """Time the persistent CTAs per SM; returns the number chosen."""
        c = ctypes.c_int32()
        st = load().lbe_batch_autotune(self._ptr, ctypes.byref(c))
        if st != 0:
            raise LbeError(st, "lbe_batch_autotune")
        return c.value

    def kernels_per_step(self):
        return int(load().lbe_batch_kernels_per_step(self._ptr))

    def first_quat(self):
        """Orientation of each member's first particle, [n_members, 4]."""
        out = np.zeros((len(self.members), 4))
        st = load().lbe_batch_first_quat(self._ptr, _dp(out))
        if st != 0:
            raise LbeError(st, "lbe_batch_first_quat")
        return out

    def close(self):
        if self._ptr:
            load().lbe_batch_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fail_allocations(after):
    """Make the library's device allocations fail after `after` more (tests of
    the out-of-memory paths); -1 lifts the limit."""
    load().lbe_fail_allocations(int(after))


def footprint(shape, nparticles=0, **params):
    """Device bytes a lattice of this shape and particle count holds at most."""
    d = make_desc(tuple(shape), **params)
    return int(load().lbe_footprint(ctypes.byref(d), int(nparticles)))


def particle_blob(pos, quat, r_par, r_perp, delta_rho, vel=None, omega=None):
    """Pack particles into the [n, PARTICLE_IN] layout of lbe_server_submit."""
    pos = _f64(pos).reshape(-1, 3)
    n = pos.shape[0]
    b = np.zeros((n, PARTICLE_IN))
    b[:, 0:3] = pos
    b[:, 3:7] = _f64(quat).reshape(n, 4)
    if vel is not None:
        b[:, 7:10] = _f64(vel).reshape(n, 3)
    if omega is not None:
        b[:, 10:13] = _f64(omega).reshape(n, 3)
    b[:, 13] = np.broadcast_to(r_par, (n,))
    b[:, 14] = np.broadcast_to(r_perp, (n,))
    b[:, 15] = np.broadcast_to(delta_rho, (n,))
    return b


class Server:
    """Continuous-batching server of adsorption requests on the current
    device (lbe_server_*)."""

    def __init__(self, hbm_budget_bytes, max_slots, storage="f32"):
        self._ptr = ctypes.c_void_p()
        st = load().lbe_server_create(int(hbm_budget_bytes), int(max_slots),
                                      STORAGE[storage] if isinstance(storage, str) else int(storage),
                                      ctypes.byref(self._ptr))
        if st != 0:
            raise LbeError(st, "lbe_server_create")
        self._np = {}

    def submit(self, shape, rho0, blob, max_steps, tilt_tol, **params):
        nx, ny, nz = shape
        d = make_desc(tuple(shape), **params)
        r = _f64(rho0, (2, nz, ny, nx))
        blob = _f64(blob).reshape(-1, PARTICLE_IN)
        rid = ctypes.c_uint64()
        st = load().lbe_server_submit(self._ptr, ctypes.byref(d), _dp(r), blob.shape[0],
                                      _dp(blob) if blob.shape[0] else None, int(max_steps),
                                      float(tilt_tol), ctypes.byref(rid))
        if st != 0:
            raise LbeError(st, "lbe_server_submit")
        self._np[rid.value] = blob.shape[0]
        return rid.value

    def poll(self, rid):
        """(done, steps_run, particles [n, PARTICLE_OUT] or None)."""
        done = ctypes.c_int32()
        steps = ctypes.c_int32()
        out = np.zeros((max(1, self._np.get(rid, 0)), PARTICLE_OUT))
        st = load().lbe_server_poll(self._ptr, ctypes.c_uint64(rid), ctypes.byref(done),
                                    ctypes.byref(steps), _dp(out))
        if st != 0:
            raise LbeError(st, "lbe_server_poll")
        return bool(done.value), steps.value, out[:self._np.get(rid, 0)] if done.value else None

    def wait(self, rid, timeout_s=60.0):
        st = load().lbe_server_wait(self._ptr, ctypes.c_uint64(rid), int(timeout_s * 1000))
        if st != 0:
            raise LbeError(st, "lbe_server_wait")
        return self.poll(rid)

    def timing(self, rid):
        q = np.zeros(1)
        t = np.zeros(1)
        st = load().lbe_server_timing(self._ptr, ctypes.c_uint64(rid), _dp(q), _dp(t))
        if st != 0:
            raise LbeError(st, "lbe_server_timing")
        return float(q[0]), float(t[0])

    def stats(self):
        out = (ctypes.c_int64 * 4)()
        st = load().lbe_server_stats(self._ptr, out)
        if st != 0:
            raise LbeError(st, "lbe_server_stats")
        return {"completed": out[0], "node_steps": out[1], "max_running": out[2], "chunks": out[3]}

    def close(self):
        if self._ptr:
            load().lbe_server_destroy(self._ptr)
            self._ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
