"""The C-ABI library loads and exports every entry point that include/cmm.h
declares (no GPU needed: nothing here calls into the device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "cmm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(cmm_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1309_7473_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    syms = declared_symbols()
    for s in ("cmm_apply_A", "cmm_rhs", "cmm_precon_create", "cmm_precon_apply", "cmm_solve",
              "cmm_pointing_create", "cmm_noise_create", "cmm_op_create"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_version_and_error_string(lib):
    lib.cmm_version.restype = ctypes.c_char_p
    lib.cmm_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.cmm_version()
    assert isinstance(lib.cmm_last_error(), bytes)


def test_binding_wraps_every_symbol(lib):
    from paper_1309_7473_gb300 import cmm
    assert sorted(cmm.EXPORTED) == declared_symbols()
