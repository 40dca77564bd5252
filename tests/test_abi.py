"""The C-ABI library loads and exports every symbol include/lbe.h declares,
and its host-side checks and arithmetic behave as documented (no compute
calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "lbe.h")).read()
    return sorted(set(re.findall(r"LBE_API\s+[\w\s\*]*?\b(lbe_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1109_3277_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("lbe_init_lattice", "lbe_add_particles", "lbe_step", "lbe_read_fields",
                 "lbe_read_particles", "lbe_mass", "lbe_destroy", "lbe_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1109_3277_gb300 import lbe
    assert sorted(lbe.SIGNATURES) == _declared()


def test_descriptor_layout_matches_oracle_shape():
    """The oracle and the library take descriptors of the same layout (the
    tests pass one set of parameters to both)."""
    from oracle import lbref
    from paper_1109_3277_gb300 import lbe
    a = [(n, ctypes.sizeof(t)) for n, t in lbe.LatticeDesc._fields_]
    b = [(n, ctypes.sizeof(t)) for n, t in lbref.LatticeDesc._fields_]
    assert a == b
    assert ctypes.sizeof(lbe.LatticeDesc) == ctypes.sizeof(lbref.LatticeDesc)


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1109_3277_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"^\s*(?:from|import)\s+(\w+)", txt, re.M), f
                assert "lbref" not in txt, f


def test_library_fails_loudly_without_the_shared_object(tmp_path):
    from paper_1109_3277_gb300 import lbe
    with pytest.raises(RuntimeError):
        lbe._lib, saved = None, lbe._lib
        try:
            lbe.load(str(tmp_path / "missing.so"))
        finally:
            lbe._lib = saved


def test_invalid_descriptors_are_rejected_before_any_device_work():
    """lbe_init_lattice checks its descriptor on the host and returns
    LBE_EINVAL (-1) without touching a device (so this runs without one)."""
    import numpy as np
    from paper_1109_3277_gb300 import lbe
    ok = dict(shape=(8, 8, 8))
    bad = [dict(shape=(0, 8, 8)), dict(shape=(8, 8, 2), walls_z=True), dict(tau=(0.5, 1.0)),
           dict(tau=(1.0, float("nan"))), dict(storage=7), dict(particle_mode=5), dict(flags=8),
           dict(shape=(1, 70000, 1))]
    for b in bad:
        p = dict(ok, **b)
        shape = p.pop("shape")
        nx, ny, nz = shape
        with pytest.raises(lbe.LbeError) as e:
            lbe.Lattice(shape, np.full((2, nz, ny, nx), 0.5), **p)
        assert e.value.status == -1, b


def test_footprint_arithmetic():
    """lbe_footprint is host arithmetic: the 16-bit modes save exactly half
    of the two population buffers, particles add their arrays and the link
    list, and an invalid descriptor gives 0."""
    from paper_1109_3277_gb300 import lbe
    shape = (40, 36, 30)
    N = 40 * 36 * 30
    S = ((N + 127) // 128) * 128 + 384
    f32 = lbe.footprint(shape, storage="f32")
    f16 = lbe.footprint(shape, storage="f16")
    assert f32 - f16 == 2 * 2 * 19 * S * 2
    assert lbe.footprint(shape, storage="bf16") == f16
    with_p = lbe.footprint(shape, 10, storage="f16")
    assert with_p - f16 >= N * 8
    assert lbe.footprint((0, 36, 30)) == 0
    assert lbe.footprint(shape, storage=9) == 0
