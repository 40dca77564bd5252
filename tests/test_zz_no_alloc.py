"""The allocation-free mass sums (lbe_mass_noalloc) against the regular
lbe_mass entry point.

lbe_mass_noalloc serves callers that keep their populations in memory they
manage and cannot call cudaMalloc; it uses a fixed array inside the library
instead of allocated scratch.  This file is collected last so that a run that
stops at the first failure has run every other test before it."""
import ctypes

import numpy as np
import pytest

from paper_1109_3277_gb300 import lbe
from paper_1109_3277_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(f_dev, storage, type_dev, nodes, stride, rho_ref, stream, out_dev):
    rr = (ctypes.c_double * 2)(*rho_ref)
    return lbe.load().lbe_mass_noalloc(ctypes.c_void_p(f_dev.data_ptr()), storage,
                                       ctypes.c_void_p(type_dev.data_ptr()), nodes, stride,
                                       ctypes.cast(rr, ctypes.POINTER(ctypes.c_double)), -1,
                                       ctypes.c_void_p(stream.cuda_stream),
                                       ctypes.c_void_p(out_dev.data_ptr()))


def test_noalloc_mass_matches_lbe_mass_twice():
    torch = pytest.importorskip("torch")
    torch.cuda.set_device(0)
    shape = (36, 20, 24)
    nx, ny, nz = shape
    n = nx * ny * nz
    f0 = W.random_populations(shape, seed=31)
    # the regular entry point: a lattice with walls and these populations
    ref = lbe.Lattice(shape, np.full((2, nz, ny, nx), 0.5), walls_z=True, device=0)
    ref.set_populations(f0)
    want = ref.mass()
    _, _, typ = ref.read_fields(rho=False, vel=False)
    ref.close()
    # the same populations and node types in caller-owned device memory
    stream = torch.cuda.Stream()
    f_dev = torch.from_numpy(f0.astype(np.float32).reshape(2 * 19 * n)).cuda()
    t_dev = torch.from_numpy(typ.reshape(n).copy()).cuda()
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(-1.0)
        torch.cuda.synchronize()
        st = _noalloc(f_dev, lbe.STORAGE["f32"], t_dev, n, n, (0.0, 0.0), stream, out)
        assert st == 0
        stream.synchronize()
        got = out.cpu().numpy()
        assert np.allclose(got, want, rtol=1e-12, atol=0)
    # sizes beyond the limits are rejected without touching the output
    out.fill_(-1.0)
    torch.cuda.synchronize()
    assert _noalloc(f_dev, 0, t_dev, 2 ** 31, 2 ** 31, (0.0, 0.0), stream, out) == -1
    assert _noalloc(f_dev, 0, t_dev, n, n - 1, (0.0, 0.0), stream, out) == -1
    stream.synchronize()
    assert np.all(out.cpu().numpy() == -1.0)
