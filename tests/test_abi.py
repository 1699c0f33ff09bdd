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


def test_null_arguments_are_rejected_before_any_device_work(lib):
    """Every entry point checks its handles and pointers first: with null ones it
    returns CMM_ERR_ARG and says why (no crash, no device call); destroying a null
    handle is a no-op that returns CMM_OK."""
    from paper_1309_7473_gb300 import cmm
    ints = (ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64)
    for name, argtypes in cmm._SIGS.items():
        f = getattr(cmm._lib, name)
        args = [0 if t in ints else 0.0 if t in (ctypes.c_double, ctypes.c_float) else None for t in argtypes]
        rc = f(*args)
        if name.endswith("_destroy"):
            assert rc == 0, name
        else:
            assert rc == 1, (name, rc)
            assert cmm._lib.cmm_last_error(), name


def test_context_without_a_gpu_fails_loudly(lib):
    """No CPU fallback: without a usable device the context cannot be made, and the
    error names the CUDA call that failed."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1309_7473_gb300 import cmm
    h = ctypes.c_void_p()
    assert cmm._lib.cmm_ctx_create(0, None, ctypes.byref(h)) == 2   # CMM_ERR_CUDA
    assert h.value is None
    assert b"cuda" in cmm._lib.cmm_last_error().lower()
