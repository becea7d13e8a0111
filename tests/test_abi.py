"""The C-ABI library builds, loads and exports every entry point that
include/eb.h declares (CPU only: no compute call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "eb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char|eb_handle)\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    import paper_2204_06083_gb300 as pkg
    return ctypes.CDLL(pkg.library_path())


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("eb_build", "eb_apply", "eb_rhs", "amg_setup", "pcg_solve", "heat_step", "wave_step",
                 "eb_last_error", "eb_destroy", "amg_destroy"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    import paper_2204_06083_gb300 as pkg
    assert set(_declared()) <= set(pkg.exported_symbols())


def test_invalid_arguments_are_reported_without_a_gpu(lib):
    import paper_2204_06083_gb300 as pkg
    L = pkg.load()
    assert L.eb_build(None, None, None, None) == pkg.EB_ERR_INVALID
    assert b"NULL" in L.eb_last_error()
    assert L.eb_apply(None, 0, None, None, None) == pkg.EB_ERR_INVALID
    assert L.pcg_solve(None, None, None, 1e-10, 10, None, None, None) == pkg.EB_ERR_INVALID
    assert L.wave_step(None, 0, 0.1, None, None, 1, None) == pkg.EB_ERR_INVALID
