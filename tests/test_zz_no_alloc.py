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

RHO_REF = (0.6, 0.35)
W_I = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def _noalloc(f_dev, storage, type_dev, nodes, stride, rho_ref, stream, out_dev, device=-1):
    rr = (ctypes.c_double * 2)(*rho_ref)
    return lbe.load().lbe_mass_noalloc(ctypes.c_void_p(f_dev.data_ptr()), storage,
                                       ctypes.c_void_p(type_dev.data_ptr()), nodes, stride,
                                       ctypes.cast(rr, ctypes.POINTER(ctypes.c_double)), device,
                                       ctypes.c_void_p(stream.cuda_stream),
                                       ctypes.c_void_p(out_dev.data_ptr()))


def _caller_buffer(torch, f0, storage, stride):
    """f0 [2][19][n] as the caller's device buffer in the library's layout:
    the two components of direction i at node n side by side, element
    2 (i stride + n) + c; the 16-bit modes hold f - w_i rho_ref^c rounded to
    nearest, as the library stores them."""
    n = f0.shape[-1]
    f32 = f0.astype(np.float32)
    if storage != "f32":
        base = (W_I[None, :] * np.array(RHO_REF)[:, None]).astype(np.float32)   # [2][19]
        f32 = (f32 - base[:, :, None]).astype(np.float32)
    pairs = np.zeros((19, stride, 2), dtype=np.float32)
    pairs[:, :n, 0] = f32[0]
    pairs[:, :n, 1] = f32[1]
    t = torch.from_numpy(pairs.reshape(-1))
    dtype = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[storage]
    return t.to(dtype).cuda()


@pytest.mark.parametrize("storage,pad", [("f32", 0), ("f16", 0), ("bf16", 0), ("f16", 100), ("f32", 37)])
def test_noalloc_mass_matches_lbe_mass_twice(storage, pad):
    torch = pytest.importorskip("torch")
    torch.cuda.set_device(0)
    shape = (36, 20, 24)
    nx, ny, nz = shape
    n = nx * ny * nz
    f0 = W.random_populations(shape, seed=31).reshape(2, 19, n)
    # the regular entry point: a lattice with walls and these populations
    ref = lbe.Lattice(shape, np.full((2, nz, ny, nx), 0.5), walls_z=True, device=0, storage=storage,
                      rho_ref=RHO_REF)
    ref.set_populations(f0.reshape(2, 19, nz, ny, nx))
    want = ref.mass()
    _, _, typ = ref.read_fields(rho=False, vel=False)
    ref.close()
    # the same populations and node types in caller-owned device memory
    stream = torch.cuda.Stream()
    stride = n + pad
    f_dev = _caller_buffer(torch, f0, storage, stride)
    t_dev = torch.from_numpy(typ.reshape(n).copy()).cuda()
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    before = torch.cuda.current_device()
    for _ in range(2):
        out.fill_(-1.0)
        torch.cuda.synchronize()
        st = _noalloc(f_dev, lbe.STORAGE[storage], t_dev, n, stride, RHO_REF, stream, out, device=0)
        assert st == 0
        stream.synchronize()
        got = out.cpu().numpy()
        assert np.allclose(got, want, rtol=1e-12, atol=0)
        assert torch.cuda.current_device() == before
    # sizes beyond the limits and bad devices are rejected without touching the output
    out.fill_(-1.0)
    torch.cuda.synchronize()
    st_id = lbe.STORAGE[storage]
    assert _noalloc(f_dev, st_id, t_dev, 2 ** 31, 2 ** 31, RHO_REF, stream, out) == -1
    assert _noalloc(f_dev, st_id, t_dev, n, n - 1, RHO_REF, stream, out) == -1
    assert _noalloc(f_dev, st_id, t_dev, n, stride, RHO_REF, stream, out, device=-2) == -1
    stream.synchronize()
    assert np.all(out.cpu().numpy() == -1.0)
    assert torch.cuda.current_device() == before
