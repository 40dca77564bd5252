"""The C-ABI library loads and exports every symbol include/lbe.h declares
(no compute calls: this runs without a GPU)."""
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
