"""The C-ABI library loads and exports every entry point include/ptim.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ptim.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pt_[a-zA-Z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2501_03061_gb300 import _lib, build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pt_create", "pt_destroy", "pt_apply_exchange", "pt_build_ace", "pt_apply_ace",
                     "pt_ptim_step", "pt_apply_H", "pt_diag_occupations"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_prototypes_cover_the_header():
    from paper_2501_03061_gb300 import _lib
    assert set(declared_functions()) == set(_lib.PROTOTYPES)


def test_version_string(lib):
    from paper_2501_03061_gb300 import _lib
    l = _lib.load()
    assert b"sm_103a" in l.pt_version()
