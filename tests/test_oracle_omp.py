"""The OpenMP build of the oracle (the all-core CPU baseline) computes what
the serial build computes, bit for bit (CPU only).

Its per-node phases run over threads, but every node is computed by the same
operations and the particle sums stay serial, so a run with free particles,
walls, pair forces and coverage changes must give identical populations,
fields and particle states.  Each build runs in a child process, since the
oracle's loader binds one library per process (LBREF_LIB)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import lbref

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUN = r"""
import sys
import numpy as np
from oracle import lbref
from paper_1109_3277_gb300 import workloads as W
shape = (24, 22, 20)
rho0 = W.flat_interface(shape, 10, 0.7, 0.04, 1e-3, seed=8)
L = lbref.Lattice(shape, rho0, walls_z=True, g_br=0.1, rho_ref=(0.37, 0.37))
L.add_particles([[8.3, 10.2, 9.6], [15.1, 11.4, 10.3]],
                [W.axis_tilt_quaternion(0.6, 0.2), W.axis_tilt_quaternion(1.1, 0.9)], 4.5, 2.5, 0.05,
                vel=[[0.02, 0.0, 0.01], [-0.02, 0.005, 0.0]])
L.step(12)
rho, vel, typ = L.read_fields()
p = L.read_particles()
np.savez(sys.argv[1], f=L.get_populations(), rho=rho, u=vel, typ=typ,
         **{"p_" + k: v for k, v in p.items()}, mass=np.array(L.mass()))
"""


def _run(lib, out, threads):
    env = dict(os.environ, LBREF_LIB=lib, OMP_NUM_THREADS=str(threads))
    r = subprocess.run([sys.executable, "-c", RUN, out], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    return np.load(out)


def test_openmp_build_equals_serial_build(tmp_path):
    serial = lbref.build()
    try:
        omp = lbref.build(omp=True)
    except subprocess.CalledProcessError:
        pytest.skip("the OpenMP build needs gcc with -fopenmp")
    a = _run(serial, str(tmp_path / "serial.npz"), 1)
    b = _run(omp, str(tmp_path / "omp.npz"), 4)
    assert set(a.files) == set(b.files)
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k
    # the run did move the particles across nodes (coverage changes)
    assert not np.array_equal(a["p_pos"], np.array([[8.3, 10.2, 9.6], [15.1, 11.4, 10.3]]))
