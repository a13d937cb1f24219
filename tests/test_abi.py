"""The C ABI: the library builds, loads and exports every declared entry point.

CPU only: no compute call is made (there may be no GPU here).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cup_gb300.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cup_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1112_5717_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("cup_factor", "cup_rank_profile", "cup_rref", "cup_det", "cup_inverse",
                 "cup_solve", "cup_mm_sub", "cup_trsm_ruu", "cup_laswp_cols", "cup_create",
                 "cup_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_the_header(lib_path):
    import paper_1112_5717_gb300 as cup
    assert sorted(cup.SIGNATURES) == _declared()
    lib = cup.load()
    for name in cup.SIGNATURES:
        assert getattr(lib, name).argtypes is not None


def test_status_codes_match_header():
    import paper_1112_5717_gb300 as cup
    text = open(HEADER).read()
    for name, val in re.findall(r"(CUP_[A-Z_]+)\s*=\s*(-?\d+)", text):
        if name.startswith(("CUP_OK", "CUP_SINGULAR", "CUP_INCONSISTENT", "CUP_ERR")):
            assert cup.STATUS[int(val)] == name


def test_null_handle_is_rejected(lib_path):
    import paper_1112_5717_gb300 as cup
    lib = cup.load()
    r = ctypes.c_int64(0)
    assert lib.cup_factor(None, None, 0, 0, 1, 7, None, None, ctypes.byref(r), None) == -1
    assert lib.cup_set_option(None, 0, 0) == -1
    assert lib.cup_destroy(None) == -1
